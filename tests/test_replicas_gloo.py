"""Two ranks over gloo (CPU): disjoint random-vector ranges averaged with one
all-reduce give the moments of a single run over all vectors."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import kpm_workloads as W
from oracle import kpm_oracle as O
from paper_2104_13218_gb300.replicas import combine_moments, vector_offset


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, R, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    model = W.ring(10)
    runs = O.sector_moments(model.arrays(), 10, -1, 5.0, -0.1, 24, R, 7, r0=vector_offset(rank, R))
    mom = {k: torch.tensor(runs[k]) for k in ("mu", "mu_M", "mu_M2")}
    combine_moments(mom, world)
    if rank == 0:
        np.save(out_path, np.stack([mom[k].numpy() for k in ("mu", "mu_M", "mu_M2")]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_average_to_the_joint_run(tmp_path):
    R, world = 3, 2
    out = str(tmp_path / "mu.npy")
    mp.start_processes(_rank, args=(world, _free_port(), R, out), nprocs=world, start_method="spawn")
    got = np.load(out)
    joint = O.sector_moments(W.ring(10).arrays(), 10, -1, 5.0, -0.1, 24, world * R, 7)
    ref = np.stack([joint[k] for k in ("mu", "mu_M", "mu_M2")])
    assert np.max(np.abs(got - ref)) < 1e-14
