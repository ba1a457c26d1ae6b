// Device helpers shared by the kernels of libkpm: the counter-based random
// signs, rank/unrank of S^z sector states, 16-byte vector chunks and warp
// reductions.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kpm_internal.h"

namespace kpm {

// splitmix64 output for generator state x (Steele, Lea and Flood; the
// published mixing constants of the splitmix64 reference generator).
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Rank of bitstring t inside its popcount sector, from the split tables.
__device__ __forceinline__ uint32_t sector_rank(uint64_t t, const TablesDev &tb) {
  const uint32_t lomask = (1u << tb.L) - 1u;
  const uint32_t lo = (uint32_t)t & lomask;
  const uint32_t hi = (uint32_t)(t >> tb.L);
  const uint32_t c = __popc(lo);
  return __ldg(tb.lo_rank + lo) + __ldg(tb.hi_rank + ((size_t)c << tb.H) + hi);
}

// Walks hi-block index b forward to the block holding rank r (ranks of one
// caller only increase), then returns the bitstring of rank r in sector k.
__device__ __forceinline__ uint64_t sector_unrank(uint32_t r, int k, uint32_t b_last, uint32_t &b,
                                                  const TablesDev &tb) {
  while (b < b_last && __ldg(tb.hb_off + b + 1) <= r) ++b;
  const uint32_t hi = __ldg(tb.hb_hi + b);
  const int c = k - __popc(hi);
  const uint32_t lo = __ldg(tb.lo_list + __ldg(tb.lo_start + c) + (r - __ldg(tb.hb_off + b)));
  return ((uint64_t)hi << tb.L) | lo;
}

template <typename T>
struct Chunk;
template <>
struct Chunk<float> {
  using type = float4;
  static constexpr int W = 4;
  __device__ static __forceinline__ float get(const float4 &v, int i) {
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
  }
  __device__ static __forceinline__ void set(float4 &v, int i, float x) {
    if (i == 0) v.x = x; else if (i == 1) v.y = x; else if (i == 2) v.z = x; else v.w = x;
  }
};
template <>
struct Chunk<double> {
  using type = double2;
  static constexpr int W = 2;
  __device__ static __forceinline__ double get(const double2 &v, int i) { return i == 0 ? v.x : v.y; }
  __device__ static __forceinline__ void set(double2 &v, int i, double x) {
    if (i == 0) v.x = x; else v.y = x;
  }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block reduction of NQ values per thread; result valid in thread 0.
// `scratch` holds kWarps * NQ doubles.  All threads of the block must call it.
template <int NQ>
__device__ __forceinline__ void block_sum(double (&v)[NQ], double *scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) scratch[warp * NQ + q] = v[q];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double x = lane < kWarps ? scratch[lane * NQ + q] : 0.0;
      v[q] = warp_sum(x);
    }
  }
  __syncthreads();
}

// Compensated (Kahan) FP32 accumulator: the FP32 form keeps its running dot
// products in FP32 pairs and hands them to FP64 at the end of a tile.
struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

}  // namespace kpm
