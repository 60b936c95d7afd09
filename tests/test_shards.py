"""Master-worker shard evaluation with failure detection, on CPU ranks.

Three processes share a TCPStore on 127.0.0.1: the master (rank 0) and two
workers.  Each shard is a contiguous range of settings evaluated by the oracle
with the global B (the measurement partition of Sec. III-B).  Failures are made
on the host -- a worker that stops answering, one that stalls past the
deadline -- and the master must reassign their shards and still produce sums
that are bitwise those of an in-order evaluation of every shard, and equal to
the unsharded oracle up to rounding."""
import socket
import time

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2607_19577_b300 import shards, synth

N, M, K, N_SHARDS = 5, 12, 3, 4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _instance():
    inst = synth.random_instance(N, M, K, shots=150, seed=91)
    return inst, inst.psi.astype(np.complex128), inst.w.astype(np.float64)


def _shard_fn(lo, hi):
    """(G psi, h, loss) of settings [lo, hi) with B = M, by the oracle."""
    inst, psi, w = _instance()
    a, b = inst.row_ptr[lo], inst.row_ptr[hi]
    rp = inst.row_ptr[lo:hi + 1] - a
    f = oracle.forward(N, inst.basis[lo:hi], psi, w, rp, inst.outcome[a:b], inst.count[a:b], inst.shots[lo:hi], B=M)
    g = oracle.adjoint(N, inst.basis[lo:hi], psi, w, rp, inst.outcome[a:b], f["c_obs"], B=M)
    return [np.asarray(g["G_psi"]), np.asarray(g["h"]), np.float64(f["loss"])]


def _rank(rank, world, port, scenario, out):
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timeout=__import__("datetime").timedelta(seconds=30))
    if rank == 0:
        master = shards.ShardMaster(store, world, M, n_shards=N_SHARDS, timeout_s=0.6, heartbeat_timeout_s=0.6)
        t0 = time.time()
        while len(master.alive()) < world - 1 and time.time() - t0 < 5.0:
            time.sleep(0.01)
        reports = [master.evaluate(it, _shard_fn) for it in range(2)]
        master.stop()
        expect = shards.sum_results([_shard_fn(*span) for span in master.spans])
        inst, psi, w = _instance()
        full = oracle.forward(N, inst.basis, psi, w, inst.row_ptr, inst.outcome, inst.count, inst.shots)
        fadj = oracle.adjoint(N, inst.basis, psi, w, inst.row_ptr, inst.outcome, full["c_obs"])
        for rep in reports:
            got = shards.sum_results(rep.results)
            assert all(np.array_equal(a, b) for a, b in zip(got, expect))  # bitwise: fixed shard order
            np.testing.assert_allclose(got[0], fadj["G_psi"], rtol=1e-12, atol=1e-15)
            np.testing.assert_allclose(got[1], fadj["h"], rtol=1e-12)
            assert abs(got[2] - full["loss"]) <= 1e-12 * abs(full["loss"])
        out.put({"owners": [r.owner for r in reports], "reassigned": [r.reassigned for r in reports],
                 "dead": sorted(reports[-1].dead)})
        return
    worker = shards.ShardWorker(store, rank, heartbeat_s=0.05)
    if scenario == "dead" and rank == 2:
        time.sleep(0.2)          # heartbeats start, then the rank leaves before serving anything
        worker.stop_heartbeat()
        return
    calls = {"n": 0}

    def fn(lo, hi):
        calls["n"] += 1
        if scenario == "stall" and rank == 1 and calls["n"] == 1:
            time.sleep(1.5)      # past the master's deadline: the result arrives too late
        return _shard_fn(lo, hi)

    worker.serve(fn, max_wait_s=30.0)


@pytest.mark.parametrize("scenario", ["none", "dead", "stall"])
def test_master_reassigns_failed_shards(scenario):
    ctx = mp.get_context("spawn")
    out = ctx.SimpleQueue()
    mp.start_processes(_rank, args=(3, _free_port(), scenario, out), nprocs=3, join=True, start_method="spawn")
    rep = out.get()
    owners = [o for it in rep["owners"] for o in it]
    if scenario == "none":
        assert rep["dead"] == [] and rep["reassigned"] == [{}, {}]
        assert set(owners) == {1, 2}
    elif scenario == "dead":
        assert 2 in rep["dead"] or 2 not in owners
        assert 2 not in owners   # no result of the departed rank is used
    else:
        assert rep["dead"] == [1]
        assert rep["reassigned"][0] and all(v == [1] for v in rep["reassigned"][0].values())
        assert all(o != 1 for o in rep["owners"][1])  # a failed rank gets no further work


def test_sum_results_in_shard_order():
    rs = [[np.array([1.0, 2.0]), 3.0], [np.array([0.5, 0.25]), 1.0]]
    tot = shards.sum_results(rs)
    assert np.array_equal(tot[0], np.array([1.5, 2.25])) and tot[1] == 4.0
