"""Batched evaluation of uneven instances (one captured CUDA graph): parity with
the oracle per instance on a reduced version of the batched workload, bitwise
equality of graph replays, and bitwise equality with single-plan evaluation on
the full 64-instance shapes."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_19577_b300 import qst, synth

pytestmark = pytest.mark.gpu


def _alloc(insts):
    datas = [qst.Data.from_numpy(i.n, i.basis, i.row_ptr, i.outcome, i.count, i.shots) for i in insts]
    psis = [torch.from_numpy(i.psi).cuda() for i in insts]
    ws = [torch.from_numpy(i.w).cuda() for i in insts]
    losses = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in insts]
    cs = [torch.zeros(i.nnz, dtype=torch.float32, device="cuda") for i in insts]
    gs = [torch.zeros_like(p) for p in psis]
    gws = [torch.zeros_like(w) for w in ws]
    return datas, psis, ws, losses, cs, gs, gws


def test_batch_matches_oracle_per_instance():
    insts = synth.make_batch(seed=1, count=10, n_range=(3, 12), M_range=(15, 60), shots_range=(100, 800),
                             rank_range=(1, 4))
    b = qst.Batch([(i.n, i.M, i.K, i.nnz) for i in insts])
    datas, psis, ws, losses, cs, gs, gws = _alloc(insts)
    b.evaluate(psis, ws, datas, losses, cs, gs, gws)
    torch.cuda.synchronize()
    first = [(l.item(), g.cpu().numpy().copy(), gw.cpu().numpy().copy()) for l, g, gw in zip(losses, gs, gws)]
    for inst, l, c, g, gw in zip(insts, losses, cs, gs, gws):
        psi = inst.psi.astype(np.complex128)
        w = inst.w.astype(np.float64)
        f = oracle.forward(inst.n, inst.basis, psi, w, inst.row_ptr, inst.outcome, inst.count, inst.shots)
        a = oracle.adjoint(inst.n, inst.basis, psi, w, inst.row_ptr, inst.outcome, f["c_obs"])
        assert abs(l.item() - f["loss"]) <= 1e-5 * abs(f["loss"])
        np.testing.assert_allclose(c.cpu().numpy(), f["c_obs"], rtol=1e-4)
        gg = g.cpu().numpy().astype(np.complex128)
        for k in range(inst.K):
            assert np.max(np.abs(gg[k] - a["grad_psi"][k])) <= 1e-4 * np.max(np.abs(a["grad_psi"][k]))
        np.testing.assert_allclose(gw.cpu().numpy(), a["grad_w"], rtol=1e-4)
    # the second call replays the captured graph: identical bits
    for x in gs + gws:
        x.zero_()
    b.evaluate(psis, ws, datas, losses, cs, gs, gws)
    torch.cuda.synchronize()
    for (l0, g0, gw0), l, g, gw in zip(first, losses, gs, gws):
        assert l.item() == l0 and np.array_equal(g.cpu().numpy(), g0) and np.array_equal(gw.cpu().numpy(), gw0)
    b.close()


def test_full_batched_workload_equals_single_plans():
    """The graph evaluation equals direct calls of the batch's own plans bitwise,
    and plans made alone (which size their bins for the whole GPU, so they may
    bin the settings, and pick chunk kernels, differently) within the parity
    tolerances."""
    insts = synth.make_batch(seed=0, count=64)
    b = qst.Batch([(i.n, i.M, i.K, i.nnz) for i in insts])
    datas, psis, ws, losses, cs, gs, gws = _alloc(insts)
    b.evaluate(psis, ws, datas, losses, cs, gs, gws)
    torch.cuda.synchronize()
    for idx in [0, 7, 21, 42, 63]:
        inst = insts[idx]
        bp = b.plan(idx)
        _, c1, l1 = bp.forward(psis[idx], ws[idx], datas[idx])
        g1, gw1 = bp.adjoint(psis[idx], ws[idx], datas[idx], c1)
        torch.cuda.synchronize()
        assert l1.item() == losses[idx].item()
        assert torch.equal(g1, gs[idx]) and torch.equal(gw1, gws[idx])
        plan = qst.Plan(inst.n, inst.M, inst.K, inst.nnz)
        _, c2, l2 = plan.forward(psis[idx], ws[idx], datas[idx])
        g2, gw2 = plan.adjoint(psis[idx], ws[idx], datas[idx], c2)
        torch.cuda.synchronize()
        assert abs(l2.item() - l1.item()) <= 1e-6 * abs(l1.item())
        gn = g1.abs().amax(dim=1)
        assert torch.all((g2 - g1).abs().amax(dim=1) <= 1e-5 * gn)
        assert torch.all((gw2 - gw1).abs() <= 1e-5 * gw1.abs())
        plan.close()
    # <psi_k | G psi_k> = h_k on every instance (Eqs. weight-gradient, atom-response)
    for inst, g, gw in zip(insts, gs, gws):
        psi = inst.psi.astype(np.complex128)
        w = inst.w.astype(np.float64)
        inner = np.sum(np.conj(psi) * (-g.cpu().numpy().astype(np.complex128) / w[:, None]), axis=1).real
        np.testing.assert_allclose(inner, -gw.cpu().numpy(), rtol=1e-4)
    b.close()


def test_full_batched_workload_largest_instances_match_oracle():
    """The instances of the full 64-instance workload with the most qubits (n = 14,
    and the largest n = 13 one), evaluated in the batch, against the FP64 oracle
    over all of their settings (sharded over the host cores)."""
    insts = synth.make_batch(seed=0, count=64)
    b = qst.Batch([(i.n, i.M, i.K, i.nnz) for i in insts])
    datas, psis, ws, losses, cs, gs, gws = _alloc(insts)
    b.evaluate(psis, ws, datas, losses, cs, gs, gws)
    torch.cuda.synchronize()
    pick = []
    for n in (14, 13):
        cand = [j for j, i in enumerate(insts) if i.n == n]
        pick += sorted(cand, key=lambda j: -insts[j].M * insts[j].K)[:1 if n == 13 else 2]
    assert pick
    for j in pick:
        inst = insts[j]
        psi, w = inst.psi.astype(np.complex128), inst.w.astype(np.float64)
        f = oracle.forward_sharded(inst.n, inst.basis, psi, w, inst.row_ptr, inst.outcome, inst.count, inst.shots)
        c = cs[j].cpu().numpy().astype(np.float64)
        a = oracle.adjoint_sharded(inst.n, inst.basis, psi, w, inst.row_ptr, inst.outcome, c)
        assert abs(losses[j].item() - f["loss"]) <= 1e-5 * abs(f["loss"])
        np.testing.assert_allclose(c, f["c_obs"], rtol=1e-4)
        gg = gs[j].cpu().numpy().astype(np.complex128)
        for k in range(inst.K):
            assert np.max(np.abs(gg[k] - a["grad_psi"][k])) <= 1e-4 * np.max(np.abs(a["grad_psi"][k])), (j, k)
        np.testing.assert_allclose(gws[j].cpu().numpy(), a["grad_w"], rtol=1e-4)
    b.close()


def test_batch_autotuner_per_size_class():
    """qst.autotune_batch times each size class's instances as one batch under its
    candidate layouts; the batch built with the chosen per-instance parameters
    (qst_batch_create_each) agrees with the oracle on every instance."""
    insts = synth.make_batch(seed=3, count=8, n_range=(6, 12), M_range=(20, 60), shots_range=(100, 400),
                             rank_range=(1, 3))
    shapes = [(i.n, i.M, i.K, i.nnz) for i in insts]
    datas, psis, ws, losses, cs, gs, gws = _alloc(insts)
    chosen, table = qst.autotune_batch(shapes, psis, ws, datas, warmup=1, reps=1)
    assert len(chosen) == len(insts) and table
    for i, c in zip(insts, chosen):
        assert c in qst.batch_candidates(i.n)
    b = qst.Batch(shapes, params=chosen)
    b.evaluate(psis, ws, datas, losses, cs, gs, gws)
    torch.cuda.synchronize()
    for j, inst in enumerate(insts):
        assert b.plan(j).status() == 0
        psi, w = inst.psi.astype(np.complex128), inst.w.astype(np.float64)
        f = oracle.forward(inst.n, inst.basis, psi, w, inst.row_ptr, inst.outcome, inst.count, inst.shots)
        a = oracle.adjoint(inst.n, inst.basis, psi, w, inst.row_ptr, inst.outcome, f["c_obs"])
        assert abs(losses[j].item() - f["loss"]) <= 1e-5 * abs(f["loss"])
        gg = gs[j].cpu().numpy().astype(np.complex128)
        for k in range(inst.K):
            assert np.max(np.abs(gg[k] - a["grad_psi"][k])) <= 1e-4 * np.max(np.abs(a["grad_psi"][k]))
    b.close()


def test_batch_iterate_equals_per_instance_iterate():
    """qst_batch_iterate (every instance's Algorithm 1 sequence on its own forked
    stream of one captured graph) equals each instance's own qst_iterate on the
    same plan bitwise: atoms, weights, J after every iteration, acceptances; a
    replay of the batch graph from the same start reproduces it."""
    insts = synth.make_batch(seed=5, count=6, n_range=(6, 12), M_range=(20, 50), shots_range=(100, 400),
                             rank_range=(1, 3))
    b = qst.Batch([(i.n, i.M, i.K, i.nnz) for i in insts])
    datas = [qst.Data.from_numpy(i.n, i.basis, i.row_ptr, i.outcome, i.count, i.shots) for i in insts]
    psi0 = []
    for inst in insts:
        p = inst.psi.astype(np.complex128)
        psi0.append((p / np.linalg.norm(p, axis=1, keepdims=True)).astype(np.complex64))
    kw = dict(T_alpha=3, T_ref=5, delta_window=0, max_oracle_calls=0)
    T = 8
    ps = [torch.from_numpy(p.copy()).cuda() for p in psi0]
    ws = [torch.from_numpy(i.w.copy()).cuda() for i in insts]
    Jb, ab = b.iterate(T, 0, ps, ws, datas, **kw)
    torch.cuda.synchronize()
    first = [(J.cpu().numpy().copy(), a.cpu().numpy().copy(), p.clone(), w.clone()) for J, a, p, w in zip(Jb, ab, ps, ws)]
    for p, w, p0, inst in zip(ps, ws, psi0, insts):
        p.copy_(torch.from_numpy(p0))
        w.copy_(torch.from_numpy(inst.w))
    Jb, ab = b.iterate(T, 0, ps, ws, datas, J_hists=Jb, accepteds=ab, **kw)
    torch.cuda.synchronize()
    for (J0, a0, p0, w0), J, a, p, w in zip(first, Jb, ab, ps, ws):
        assert np.array_equal(J.cpu().numpy(), J0) and np.array_equal(a.cpu().numpy(), a0)
        assert torch.equal(p, p0) and torch.equal(w, w0)
    for idx, inst in enumerate(insts):
        plan = b.plan(idx)
        p = torch.from_numpy(psi0[idx].copy()).cuda()
        w = torch.from_numpy(inst.w.copy()).cuda()
        J, a = plan.iterate(T, 0, p, w, datas[idx], **kw)
        torch.cuda.synchronize()
        assert plan.status() == 0
        assert np.array_equal(J.cpu().numpy(), first[idx][0]) and np.array_equal(a.cpu().numpy(), first[idx][1])
        assert torch.equal(p, first[idx][2]) and torch.equal(w, first[idx][3])
    assert sum(int(f[1].sum()) for f in first) > 0
    b.close()


def test_batch_with_cluster_and_small_chunk_plans():
    """A batch holding a 16-qubit-chunk plan (CTA clusters: the batch then runs
    every instance's own launch sequence in the graph) beside two-round plans of
    10, 11 qubits equals the same plans called directly, bitwise, and the oracle."""
    insts = [synth.random_instance(17, 6, 2, 1500, 41), synth.random_instance(11, 30, 3, 400, 42),
             synth.random_instance(10, 25, 5, 1500, 43)]
    params = [dict(chunk_qubits=16), dict(), dict()]
    b = qst.Batch([(i.n, i.M, i.K, i.nnz) for i in insts], params=params)
    datas, psis, ws, losses, cs, gs, gws = _alloc(insts)
    b.evaluate(psis, ws, datas, losses, cs, gs, gws)
    torch.cuda.synchronize()
    assert b.plan(0).geometry()["fixed_rounds"] == 4
    assert b.plan(1).geometry()["fixed_rounds"] == 2 and b.plan(2).geometry()["fixed_rounds"] == 2
    for idx, inst in enumerate(insts):
        p1, c1, l1, g1, gw1 = b.plan(idx).evaluate(psis[idx], ws[idx], datas[idx])
        torch.cuda.synchronize()
        assert l1.item() == losses[idx].item()
        assert torch.equal(c1, cs[idx]) and torch.equal(g1, gs[idx]) and torch.equal(gw1, gws[idx])
        psi = inst.psi.astype(np.complex128)
        w = inst.w.astype(np.float64)
        f = oracle.forward(inst.n, inst.basis, psi, w, inst.row_ptr, inst.outcome, inst.count, inst.shots)
        a = oracle.adjoint(inst.n, inst.basis, psi, w, inst.row_ptr, inst.outcome, f["c_obs"])
        assert abs(losses[idx].item() - f["loss"]) <= 1e-5 * abs(f["loss"])
        gg = gs[idx].cpu().numpy().astype(np.complex128)
        for k in range(inst.K):
            assert np.max(np.abs(gg[k] - a["grad_psi"][k])) <= 1e-4 * np.max(np.abs(a["grad_psi"][k]))
    b.close()
