"""GPU simplex projection (+ P_tau) and spectral refactorisation against the
FP64 oracle.  The refactor is compared through rho-level quantities (atoms
carry a free phase and degenerate eigenvalues a free basis): weights, the
Frobenius distance between the old and new rho computed from Gram matrices,
and orthonormality of the new atoms."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_19577_b300 import qst, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("K,seed,tau", [(1, 0, 1e-3), (2, 1, 1e-3), (7, 2, 0.0), (16, 3, 1e-3), (100, 4, 1e-3),
                                        (1024, 5, 1e-4), (33, 6, 0.05)])
def test_simplex_project_matches_oracle(K, seed, tau):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(K) * 0.3 + 1.0 / K
    beta, keep, kout = qst.simplex_project(torch.from_numpy(v).cuda(), tau)
    torch.cuda.synchronize()
    ref = oracle.simplex_project(v)
    rkeep, rb = oracle.prune(ref, tau)
    k = int(kout.item())
    assert k == rkeep.size
    assert list(keep.cpu().numpy()[:k]) == list(rkeep)
    full = np.zeros(K)
    full[rkeep] = rb
    np.testing.assert_allclose(beta.cpu().numpy(), full, atol=1e-14)


def test_simplex_project_ties_and_nothing_survives():
    v = np.array([0.25, 0.25, 0.25, 0.25])
    beta, keep, kout = qst.simplex_project(torch.from_numpy(v).cuda(), 0.3)  # all equal, none > 0.3
    assert int(kout.item()) == 1 and int(keep[0].item()) == 0
    np.testing.assert_allclose(beta.cpu().numpy(), [1, 0, 0, 0])


def _gram_frob2(A, wa, B, wb):
    """||A^T diag(wa) A^* - B^T diag(wb) B^*||_F^2 through K x K Gram matrices."""
    def cross(X, wx, Y, wy):
        G = X.conj() @ Y.T
        return float(np.real(np.sum(np.outer(wx, wy) * np.abs(G) ** 2)))
    return cross(A, wa, A, wa) + cross(B, wb, B, wb) - 2 * cross(A, wa, B, wb)


@pytest.mark.parametrize("n,K,seed", [(4, 3, 0), (8, 8, 1), (12, 16, 2), (16, 16, 3), (10, 32, 4)])
def test_refactor_matches_oracle(n, K, seed):
    rng = synth.rng_for(seed, 55)
    psi = synth.random_atoms(n, K, rng).astype(np.complex64)
    w = synth.dirichlet_weights(K, rng)
    w[-1] = 2e-4  # below tau after renormalisation: gets pruned
    w = (w / w.sum()).astype(np.float32)
    tau = 1e-3
    plan = qst.Plan(n, 4, K, 0)
    tp, tw = torch.from_numpy(psi.copy()).cuda(), torch.from_numpy(w.copy()).cuda()
    kout = plan.refactor(tp, tw, tau)
    torch.cuda.synchronize()
    k = int(kout.item())
    phi, wk = oracle.refactor(psi.astype(np.complex128), w.astype(np.float64), tau)
    assert k == phi.shape[0]
    gp = tp.cpu().numpy().astype(np.complex128)
    gw = tw.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(gw[:k], wk, rtol=1e-5, atol=1e-7)
    assert np.all(gw[k:] == 0) and np.all(gp[k:] == 0)
    np.testing.assert_allclose(gp[:k].conj() @ gp[:k].T, np.eye(k), atol=2e-5)
    # rho' against the oracle's rho' (same pruning) and, before pruning effects, against rho
    d2 = _gram_frob2(gp[:k], gw[:k], phi, wk)
    assert d2 <= 1e-9, d2
    plan.close()


def test_refactor_of_orthonormal_atoms_is_identity_on_rho():
    n, K = 9, 5
    a = synth.random_atoms(n, K, synth.rng_for(9), orthonormal=True).astype(np.complex64)
    w = np.array([0.4, 0.25, 0.2, 0.1, 0.05], np.float32)
    plan = qst.Plan(n, 4, K, 0)
    tp, tw = torch.from_numpy(a.copy()).cuda(), torch.from_numpy(w.copy()).cuda()
    plan.refactor(tp, tw, 0.0)
    gp, gw = tp.cpu().numpy().astype(np.complex128), tw.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(gw, w, atol=1e-6)
    assert _gram_frob2(gp, gw, a.astype(np.complex128), w.astype(np.float64)) <= 1e-10
    plan.close()


def test_step_sequence_matches_oracle():
    """A sequence of Algorithm-1 slots (atom, coefficient and refactor slots) on the
    GPU and in the oracle: same acceptance decisions and step sizes, J within 1e-5,
    and the same state at the rho level; J never increases."""
    inst = synth.make_instance("n4_all81", seed=7, K=4)
    n = inst.n
    psi0 = inst.psi.astype(np.complex128)
    psi0 /= np.linalg.norm(psi0, axis=1, keepdims=True)
    w0 = inst.w.astype(np.float64)
    data = dict(basis=inst.basis, row_ptr=inst.row_ptr, outcome=inst.outcome, count=inst.count, shots=inst.shots)
    plan = qst.Plan(n, inst.M, inst.K, inst.nnz)
    d = qst.Data.from_numpy(n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    tp = torch.from_numpy(psi0.astype(np.complex64)).cuda()
    tw = torch.from_numpy(w0.astype(np.float32)).cuda()
    op = tp.cpu().numpy().astype(np.complex128)
    ow = tw.cpu().numpy().astype(np.float64)
    J_prev = None
    for slot, r in [(0, 0), (1, 0), (0, 1), (0, 2), (0, 3), (1, 0), (2, 0), (0, 0), (1, 0), (0, 1)]:
        J, acc, eta = plan.step(slot, r, tp, tw, d)
        op, ow, oJ, oacc, oeta = oracle.step(n, data, op, ow, slot, r)
        assert acc == oacc and abs(eta - oeta) <= 1e-12 * max(1.0, oeta), (slot, r, acc, oacc, eta, oeta)
        assert abs(J - oJ) <= 1e-5 * abs(oJ), (J, oJ)
        gp = tp.cpu().numpy().astype(np.complex128)
        gw = tw.cpu().numpy().astype(np.float64)
        a = gw > 0
        b = ow > 0
        d2 = _gram_frob2(gp[a], gw[a], op[b], ow[b])
        assert d2 <= 1e-9, (slot, d2)
        if J_prev is not None:
            assert J <= J_prev + 1e-12
        J_prev = J
        # continue the oracle from the GPU state (FP32), so differences do not accumulate
        op, ow = gp, gw
    plan.close()


def _schedule(t, T_alpha, T_ref):
    if T_ref > 0 and (t + 1) % T_ref == 0:
        return 2
    if T_alpha > 0 and (t + 1) % T_alpha == 0:
        return 1
    return 0


@pytest.mark.parametrize("name,n,K,T,T_alpha,T_ref,rounds", [("n4_all81", None, 4, 14, 3, 7, -1),
                                                              ("n12_m60_k6", 12, 6, 9, 4, 0, -1),
                                                              ("n12_m60_k5", 12, 5, 8, 3, 7, 2),
                                                              ("n11_m40_k5", 11, 5, 8, 3, 7, 2),
                                                              ("n17_m12_k3", 17, 3, 6, 3, 5, 4)])
def test_device_iterations_equal_host_steps(name, n, K, T, T_alpha, T_ref, rounds):
    """qst_iterate (every decision on the device, one captured graph) equals the same
    schedule driven from the host with qst_step: bitwise the same atoms and weights
    and the same J after every iteration.  A second run continues (t0 = T) and a
    replay of the first run's graph on the same buffers reproduces it.  The last
    case runs the two-round chunk kernels (odd K: a CTA with one atom), whose
    forward honours the device skip flag inside conditional graph nodes.  The
    11-qubit case runs the two-round kernels with four atoms per CTA, the 17-qubit
    case the 16-qubit chunks on CTA clusters (fixed_rounds = 4)."""
    inst = synth.make_instance(name, seed=11, K=K)
    psi0 = inst.psi.astype(np.complex128)
    psi0 /= np.linalg.norm(psi0, axis=1, keepdims=True)
    psi0 = psi0.astype(np.complex64)
    w0 = inst.w.astype(np.float32)
    plan = qst.Plan(inst.n, inst.M, K, inst.nnz, fixed_rounds=rounds)
    if rounds == 2:
        assert plan.geometry()["fixed_rounds"] == 2
    d = qst.Data.from_numpy(inst.n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    # host-driven reference
    hp, hw = torch.from_numpy(psi0.copy()).cuda(), torch.from_numpy(w0.copy()).cuda()
    Jh, acc_h, count = [], [], 0
    for t in range(2 * T):
        slot = _schedule(t, T_alpha, T_ref)
        r = 0
        if slot == 0:
            act = [k for k, v in enumerate(hw.cpu().numpy()) if v > 0]
            r = act[count % len(act)]
            count += 1
        J, acc, _ = plan.step(slot, r, hp, hw, d)
        Jh.append(J)
        acc_h.append(acc)
    # device-driven: first T iterations, a replay of the same graph from the
    # same start, then the next T iterations (t0 = T continues the atom cycle)
    dp, dw = torch.from_numpy(psi0.copy()).cuda(), torch.from_numpy(w0.copy()).cuda()
    off = dict(delta_window=0, max_oracle_calls=0)  # this test compares schedules, not stopping rules
    J1, a1 = plan.iterate(T, 0, dp, dw, d, T_alpha=T_alpha, T_ref=T_ref, **off)
    first = (J1.cpu().numpy().copy(), a1.cpu().numpy().copy(), dp.clone(), dw.clone())
    dp.copy_(torch.from_numpy(psi0))
    dw.copy_(torch.from_numpy(w0))
    J1, a1 = plan.iterate(T, 0, dp, dw, d, J_hist=J1, accepted=a1, T_alpha=T_alpha, T_ref=T_ref, **off)
    torch.cuda.synchronize()
    assert np.array_equal(J1.cpu().numpy(), first[0]) and np.array_equal(a1.cpu().numpy(), first[1])
    assert torch.equal(dp, first[2]) and torch.equal(dw, first[3])
    J2, a2 = plan.iterate(T, T, dp, dw, d, T_alpha=T_alpha, T_ref=T_ref, **off)
    torch.cuda.synchronize()
    plan.check()
    Jd = list(first[0]) + list(J2.cpu().numpy())
    ad = list(first[1]) + list(a2.cpu().numpy())
    assert [bool(x) for x in ad] == acc_h
    assert Jd == Jh
    assert torch.equal(dp, hp) and torch.equal(dw, hw)
    assert sum(acc_h) > 0
    plan.close()


@pytest.mark.parametrize("name,K,T,T_alpha,T_ref", [("n8_m40_k4", 4, 11, 3, 4), ("n10_m60_k8", 8, 9, 4, 3)])
def test_iterate_with_spectral_slots_equals_host_steps(name, K, T, T_alpha, T_ref):
    """qst_iterate with spectral = 1: the T_rho slots run qst_step slot 3 between graph
    segments (one graph replayed for segments with the same slots).  Bitwise the same
    atoms, weights, J and acceptances as the schedule driven from the host with
    qst_step (slot 3 at the T_rho slots), over a first run and a continued one; the
    device's oracle-call count adds the spectral slots' calls."""
    inst = synth.make_instance(name, seed=21, K=K)
    psi0 = inst.psi.astype(np.complex128)
    psi0 /= np.linalg.norm(psi0, axis=1, keepdims=True)
    psi0 = psi0.astype(np.complex64)
    w0 = inst.w.astype(np.float32)
    plan = qst.Plan(inst.n, inst.M, K, inst.nnz)
    d = qst.Data.from_numpy(inst.n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    hp, hw = torch.from_numpy(psi0.copy()).cuda(), torch.from_numpy(w0.copy()).cuda()
    Jh, acc_h, count = [], [], 0
    for t in range(2 * T):
        slot = _schedule(t, T_alpha, T_ref)
        r = 0
        if slot == 0:
            act = [k for k, v in enumerate(hw.cpu().numpy()) if v > 0]
            r = act[count % len(act)]
            count += 1
        J, acc, _ = plan.step(3 if slot == 2 else slot, r, hp, hw, d)
        Jh.append(J)
        acc_h.append(acc)
    dp, dw = torch.from_numpy(psi0.copy()).cuda(), torch.from_numpy(w0.copy()).cuda()
    off = dict(delta_window=0, max_oracle_calls=0)
    J1, a1 = plan.iterate(T, 0, dp, dw, d, T_alpha=T_alpha, T_ref=T_ref, spectral=True, **off)
    J1, a1 = J1.cpu().numpy().copy(), a1.cpu().numpy().copy()
    calls1 = plan.iterate_state()["oracle_calls"]
    J2, a2 = plan.iterate(T, T, dp, dw, d, T_alpha=T_alpha, T_ref=T_ref, spectral=True, **off)
    torch.cuda.synchronize()
    plan.check()
    assert [bool(x) for x in list(a1) + list(a2.cpu().numpy())] == acc_h
    assert list(J1) + list(J2.cpu().numpy()) == Jh
    assert torch.equal(dp, hp) and torch.equal(dw, hw)
    assert any(acc_h[t] for t in range(2 * T) if _schedule(t, T_alpha, T_ref) == 2)
    assert plan.iterate_state()["oracle_calls"] > calls1 > 0
    plan.close()


@pytest.mark.parametrize("name,K,seed,rank_fix", [("n4_all81", 4, 3, 0), ("n8_m40_k4", 4, 5, 0),
                                                  ("n10_m60_k8", 8, 7, 0), ("n8_m40_k4", 4, 5, 2),
                                                  ("n10_m60_k8", 8, 7, 3)])
def test_spectral_step_matches_oracle(name, K, seed, rank_fix):
    """qst_step slot 3 (Sec. III-C: block Krylov Ritz pairs of S = rho + eta G, the
    scored candidates, the best one, acceptance over the step grid) against the
    oracle's slot 3: same acceptance and step, J within 1e-5, and the same state at
    the rho level.  At n = 4 the Krylov space spans C^16 (exact eigenpairs).  rank_fix
    > 0 is the known-rank variant (only the candidate with that many Ritz pairs)."""
    inst = synth.make_instance(name, seed=seed, K=K)
    n = inst.n
    psi0 = inst.psi.astype(np.complex128)
    psi0 /= np.linalg.norm(psi0, axis=1, keepdims=True)
    w0 = inst.w.astype(np.float64)
    data = dict(basis=inst.basis, row_ptr=inst.row_ptr, outcome=inst.outcome, count=inst.count, shots=inst.shots)
    plan = qst.Plan(n, inst.M, K, inst.nnz)
    d = qst.Data.from_numpy(n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    tp = torch.from_numpy(psi0.astype(np.complex64)).cuda()
    tw = torch.from_numpy(w0.astype(np.float32)).cuda()
    J, acc, eta = plan.step(3, 0, tp, tw, d, rank_fix=rank_fix)
    # the oracle starts from the same (FP32-rounded) state
    op, ow, oJ, oacc, oeta = oracle.step(n, data, psi0.astype(np.complex64).astype(np.complex128),
                                         w0.astype(np.float32).astype(np.float64), 3, 0, n_krylov=30,
                                         rank_fix=rank_fix)
    assert acc == oacc and abs(eta - oeta) <= 1e-12 * max(1.0, oeta), (acc, oacc, eta, oeta)
    assert abs(J - oJ) <= 1e-5 * abs(oJ), (J, oJ)
    gp = tp.cpu().numpy().astype(np.complex128)
    gw = tw.cpu().numpy().astype(np.float64)
    a, b = gw > 0, ow > 0
    assert a.sum() == b.sum()
    np.testing.assert_allclose(np.sort(gw[a]), np.sort(ow[b]), atol=2e-5)
    assert _gram_frob2(gp[a], gw[a], op[b], ow[b]) <= 1e-8
    if acc:  # an accepted spectral step leaves orthonormal Ritz vectors (a rejected one the old atoms)
        np.testing.assert_allclose(gp[a].conj() @ gp[a].T, np.eye(a.sum()), atol=2e-5)
        if rank_fix:
            assert a.sum() <= rank_fix
    plan.close()


def _host_calls(slot, acc, eta, R_new, n_eta=11, eta0=1.0, ratio=0.5):
    """Serial-equivalent oracle calls of one Algorithm 1 slot (the reading the device
    counter uses): atom slot 1 + 2 per trial, coefficient slot 1 + 1 per trial,
    refactor slot (new atoms) + 1; trials = accepted index + 1, else the grid."""
    trials = int(round(np.log(eta / eta0) / np.log(ratio))) + 1 if acc else n_eta
    if slot == 0:
        return 1 + 2 * trials
    if slot == 1:
        return 1 + trials
    return R_new + 1


@pytest.mark.parametrize("window,tol,max_calls", [(4, 2e-3, 0), (0, 0.0, 60), (6, 5e-3, 100000)])
def test_device_stopping_rules_match_the_host_rule(window, tol, max_calls):
    """Table I's stopping rules inside qst_iterate (no host synchronisation): the
    relative decrease of J over the last `window` accepted updates below `tol`,
    or `max_calls` serial-equivalent oracle calls.  The same schedule driven from
    the host with qst_step, with the rule evaluated on the host, stops at the same
    iteration with the same J history (bitwise), oracle-call count and accepted
    updates; after the stop the device leaves the state unchanged."""
    inst = synth.make_instance("n8_m40_k4", seed=21, K=4)
    psi0 = inst.psi.astype(np.complex128)
    psi0 /= np.linalg.norm(psi0, axis=1, keepdims=True)
    psi0 = psi0.astype(np.complex64)
    w0 = inst.w.astype(np.float32)
    plan = qst.Plan(inst.n, inst.M, 4, inst.nnz)
    d = qst.Data.from_numpy(inst.n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    T, T_alpha = 40, 5
    hp, hw = torch.from_numpy(psi0.copy()).cuda(), torch.from_numpy(w0.copy()).cuda()
    R0 = int(np.count_nonzero(w0 > 0))
    calls = R0 + 1
    _, _, loss0 = plan.forward(hp, hw, d)
    Jrec = [loss0.item() + 1e-3 * R0]  # J after accepted update i (i = 0: the start; mu = 1e-3)
    Jh, acc_h, count, stop_at = [], [], 0, None
    for t in range(T):
        slot = _schedule(t, T_alpha, 0)
        r = 0
        if slot == 0:
            act = [k for k, v in enumerate(hw.cpu().numpy()) if v > 0]
            r = act[count % len(act)]
            count += 1
        J, acc, eta = plan.step(slot, r, hp, hw, d)
        Jh.append(J)
        acc_h.append(acc)
        calls += _host_calls(slot, acc, eta, int(np.count_nonzero(hw.cpu().numpy() > 0)))
        if acc:
            Jrec.append(J)
        n_acc = len(Jrec) - 1
        fired = window > 0 and acc and n_acc >= window and (Jrec[n_acc - window] - J) / abs(Jrec[n_acc - window]) < tol
        if fired or (max_calls > 0 and calls >= max_calls):
            stop_at = t
            break
    assert stop_at is not None, "the rule must fire within the run"
    dp, dw = torch.from_numpy(psi0.copy()).cuda(), torch.from_numpy(w0.copy()).cuda()
    Jd, ad = plan.iterate(T, 0, dp, dw, d, T_alpha=T_alpha, T_ref=0, delta_window=window, delta_tol=tol,
                          max_oracle_calls=max_calls)
    st = plan.iterate_state()
    Jd, ad = Jd.cpu().numpy(), ad.cpu().numpy()
    assert st["stopped"]
    assert list(Jd[:stop_at + 1]) == Jh and [bool(x) for x in ad[:stop_at + 1]] == acc_h
    assert np.all(Jd[stop_at + 1:] == Jh[-1]) and not ad[stop_at + 1:].any()
    assert st["oracle_calls"] == calls and st["accepted_updates"] == sum(acc_h)
    assert torch.equal(dp, hp) and torch.equal(dw, hw)
    plan.close()
