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
        rp, a, b = replicas.shard_rows(inst.row_ptr, lo, hi)
        f = oracle.forward(n, inst.basis[lo:hi], psi, w, rp, inst.outcome[a:b], inst.count[a:b],
                           inst.shots[lo:hi], B=M)
        g = oracle.adjoint(n, inst.basis[lo:hi], psi, w, rp, inst.outcome[a:b], f["c_obs"], B=M)
        # the exchange the GPU shards use (replicas.allreduce_evaluation), here over gloo in FP64
        loss = torch.tensor([f["loss"]], dtype=torch.float64)
        grad = torch.from_numpy(g["grad_psi"].copy())
        gw = torch.from_numpy(g["grad_w"].copy())
        replicas.allreduce_evaluation(loss, grad, gw, dist)
        full = oracle.forward(n, inst.basis, psi, w, inst.row_ptr, inst.outcome, inst.count, inst.shots)
        fadj = oracle.adjoint(n, inst.basis, psi, w, inst.row_ptr, inst.outcome, full["c_obs"])
        np.testing.assert_allclose(grad.numpy(), fadj["grad_psi"], atol=1e-14)
        np.testing.assert_allclose(gw.numpy(), fadj["grad_w"], rtol=1e-12)
        assert abs(loss.item() - full["loss"]) <= 1e-12 * max(1.0, abs(full["loss"]))
        # the same exchange in FP32 complex64 / float32 (the GPU path's dtypes)
        g32 = torch.from_numpy(np.ascontiguousarray(g["grad_psi"]).astype(np.complex64))
        gw32 = torch.from_numpy(np.ascontiguousarray(g["grad_w"]).astype(np.float32))
        replicas.allreduce_evaluation(torch.tensor([f["loss"]], dtype=torch.float64), g32, gw32, dist)
        np.testing.assert_allclose(g32.numpy(), fadj["grad_psi"], atol=1e-6 * np.abs(fadj["grad_psi"]).max())
        np.testing.assert_allclose(gw32.numpy(), fadj["grad_w"], rtol=1e-5)
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
