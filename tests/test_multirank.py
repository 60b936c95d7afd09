"""Two CPU ranks over gloo (127.0.0.1): the multi-rank host logic.

* The measurement partition of Sec. III-B as a real exchange: each rank
  evaluates its contiguous shard of the settings with the oracle (global B),
  the loss, h and G psi are all-reduced (sum), and every rank then holds the
  unsharded values.
* The bench's aggregation: job time = slowest rank, units = all ranks'."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2607_19577_b300 import replicas, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        n, M, K = 6, 13, 3
        inst = synth.random_instance(n, M, K, shots=120, seed=77)
        psi = inst.psi.astype(np.complex128)
        w = inst.w.astype(np.float64)
        lo, hi = replicas.shard(M, rank, world)
        a, b = inst.row_ptr[lo], inst.row_ptr[hi]
        rp = inst.row_ptr[lo:hi + 1] - a
        f = oracle.forward(n, inst.basis[lo:hi], psi, w, rp, inst.outcome[a:b], inst.count[a:b],
                           inst.shots[lo:hi], B=M)
        g = oracle.adjoint(n, inst.basis[lo:hi], psi, w, rp, inst.outcome[a:b], f["c_obs"], B=M)
        G = torch.from_numpy(np.ascontiguousarray(g["G_psi"]).view(np.float64).copy())
        hL = torch.tensor(list(g["h"]) + [f["loss"]], dtype=torch.float64)
        dist.all_reduce(G, op=dist.ReduceOp.SUM)
        dist.all_reduce(hL, op=dist.ReduceOp.SUM)
        full = oracle.forward(n, inst.basis, psi, w, inst.row_ptr, inst.outcome, inst.count, inst.shots)
        fadj = oracle.adjoint(n, inst.basis, psi, w, inst.row_ptr, inst.outcome, full["c_obs"])
        np.testing.assert_allclose(G.numpy().view(np.complex128).reshape(K, -1), fadj["G_psi"], atol=1e-14)
        np.testing.assert_allclose(hL.numpy()[:K], fadj["h"], rtol=1e-12)
        assert abs(hL[K].item() - full["loss"]) <= 1e-12 * max(1.0, abs(full["loss"]))
        # aggregation: rank r reports (10 + r) ms and (r + 1) * 100 units
        ms, units = replicas.aggregate(10.0 + rank, (rank + 1) * 100.0, dist)
        assert ms == 10.0 + (world - 1) and units == 100.0 * world * (world + 1) / 2
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_sum_and_aggregate():
    mp.spawn(_worker, args=(2, _free_port()), nprocs=2, join=True)


def test_shard_ranges_cover_settings():
    for M in (1, 2, 7, 4096):
        for world in (1, 2, 3, 8):
            spans = [replicas.shard(M, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == M
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1


def test_aggregate_single_process():
    assert replicas.aggregate(3.5, 7, None) == (3.5, 7.0)
