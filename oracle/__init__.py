"""Independent CPU FP64 oracle of the Chebyshev typicality method.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check of the
repository entry point and by the benchmark's CPU-baseline leg, never by the
library.  It shares no code with the CUDA path.
"""
