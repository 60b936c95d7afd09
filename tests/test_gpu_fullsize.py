"""Full-size parity in the benchmark's launch configuration (n = 16, M = 4096,
K = 16, default plan), on outputs the oracle can compute one by one, and on
properties that hold at any size."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_19577_b300 import qst, synth

pytestmark = pytest.mark.gpu

P_TOL, C_TOL, G_TOL, H_TOL = 1e-5, 1e-4, 1e-4, 1e-4


@pytest.fixture(scope="module")
def c3():
    inst = synth.make_instance("n16_m4096_k16", seed=0)
    plan = qst.Plan(inst.n, inst.M, inst.K, inst.nnz)
    data = qst.Data.from_numpy(inst.n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    psi, w = torch.from_numpy(inst.psi).cuda(), torch.from_numpy(inst.w).cuda()
    p_obs, c_obs, loss = plan.forward(psi, w, data)
    g, gw = plan.adjoint(psi, w, data, c_obs)
    torch.cuda.synchronize()
    assert plan.status() == 0
    yield dict(inst=inst, plan=plan, data=data, psi=psi, w=w, p_obs=p_obs, c_obs=c_obs, loss=loss, g=g, gw=gw)
    plan.close()


def _rows(inst, sel):
    rp = [0]
    outs, cnts = [], []
    for s in sel:
        lo, hi = inst.row_ptr[s], inst.row_ptr[s + 1]
        outs.append(inst.outcome[lo:hi])
        cnts.append(inst.count[lo:hi])
        rp.append(rp[-1] + hi - lo)
    return np.array(rp, np.int64), np.concatenate(outs), np.concatenate(cnts)


def test_sampled_settings_forward(c3):
    inst = c3["inst"]
    sel = synth.rng_for(1234).choice(inst.M, 6, replace=False)
    rp, out, cnt = _rows(inst, sel)
    ref = oracle.forward(inst.n, inst.basis[sel], inst.psi.astype(np.complex128), inst.w.astype(np.float64),
                         rp, out, cnt, inst.shots[sel], eps=inst.eps, B=inst.M)
    p = c3["p_obs"].cpu().numpy()
    c = c3["c_obs"].cpu().numpy()
    for j, s in enumerate(sel):
        lo, hi = inst.row_ptr[s], inst.row_ptr[s + 1]
        r = ref["p_obs"][rp[j]:rp[j + 1]]
        assert np.max(np.abs(p[lo:hi] - r)) / np.max(r) <= P_TOL
        np.testing.assert_allclose(c[lo:hi], ref["c_obs"][rp[j]:rp[j + 1]], rtol=C_TOL)


def test_loss_is_the_fp64_sum_of_its_terms(c3):
    inst = c3["inst"]
    p = c3["p_obs"].cpu().numpy().astype(np.float64)
    shots = np.repeat(inst.shots, np.diff(inst.row_ptr)).astype(np.float64)
    pihat = inst.count / (inst.M * shots)
    L = -np.sum(pihat * np.log(p / inst.M + inst.eps))
    assert abs(c3["loss"].item() - L) <= 1e-5 * abs(L)


def test_sampled_settings_adjoint(c3):
    """G restricted to a few settings (c zeroed elsewhere) in the same launch
    configuration, against the oracle on those settings."""
    inst = c3["inst"]
    sel = np.sort(synth.rng_for(99).choice(inst.M, 4, replace=False))
    mask = np.zeros(inst.nnz, bool)
    for s in sel:
        mask[inst.row_ptr[s]:inst.row_ptr[s + 1]] = True
    c_full = c3["c_obs"].cpu().numpy()
    c_masked = torch.from_numpy(np.where(mask, c_full, 0).astype(np.float32)).cuda()
    g, gw = c3["plan"].adjoint(c3["psi"], c3["w"], c3["data"], c_masked)
    rp, out, _ = _rows(inst, sel)
    ref = oracle.adjoint(inst.n, inst.basis[sel], inst.psi.astype(np.complex128), inst.w.astype(np.float64),
                         rp, out, c_full[mask].astype(np.float64), B=inst.M)
    g = g.cpu().numpy().astype(np.complex128)
    for k in range(inst.K):
        nrm = np.max(np.abs(ref["grad_psi"][k]))
        assert np.max(np.abs(g[k] - ref["grad_psi"][k])) / nrm <= G_TOL
    np.testing.assert_allclose(gw.cpu().numpy(), ref["grad_w"], rtol=H_TOL)


def test_h_equals_atom_inner_product_with_G(c3):
    """<psi_k|G psi_k> = h_k, with G psi_k from the gradient path and h_k from
    the weight-gradient path (Eqs. weight-gradient, atom-wirtinger-gradient)."""
    psi = c3["psi"].cpu().numpy().astype(np.complex128)
    w = c3["w"].cpu().numpy().astype(np.float64)
    g = c3["g"].cpu().numpy().astype(np.complex128)
    h = -c3["gw"].cpu().numpy().astype(np.float64)
    inner = np.sum(np.conj(psi) * (-g / w[:, None]), axis=1)
    np.testing.assert_allclose(inner.real, h, rtol=1e-4)


def test_weighted_h_sum_matches_forward(c3):
    """sum_k w_k h_k = sum_m c_m pi_m, from the forward's c and p."""
    inst = c3["inst"]
    w = c3["w"].cpu().numpy().astype(np.float64)
    h = -c3["gw"].cpu().numpy().astype(np.float64)
    c = c3["c_obs"].cpu().numpy().astype(np.float64)
    p = c3["p_obs"].cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(np.dot(w, h), np.sum(c * p / inst.M), rtol=1e-5)


def test_povm_completeness_at_n16():
    """32 full settings with c = 1 at every outcome: G = I, so grad = -w psi."""
    n, M, K = 16, 32, 2
    D = 1 << n
    basis = synth.pauli_settings(n, M, synth.rng_for(5))
    row_ptr = np.arange(M + 1, dtype=np.int64) * D
    outcome = np.tile(np.arange(D, dtype=np.uint32), M)
    plan = qst.Plan(n, M, K, M * D)
    data = qst.Data.from_numpy(n, basis, row_ptr, outcome, np.ones(M * D, np.uint32), np.full(M, D, np.uint32))
    psi = torch.from_numpy(synth.random_atoms(n, K, synth.rng_for(6)).astype(np.complex64)).cuda()
    w = torch.tensor([-1.0, -1.0], device="cuda")
    g, _ = plan.adjoint(psi, w, data, torch.ones(M * D, device="cuda"))
    err = (g - psi).abs().max().item() / psi.abs().max().item()
    assert err <= 1e-5
    plan.close()


@pytest.fixture(scope="module")
def c3k2():
    """The bench workload's settings and counts with its first two atoms (w = 1/2 each)
    in the bench's per-unit launch configuration: two-round chunk kernels and bins of
    up to 96 settings (a plan for K = 16 chooses both on its own)."""
    inst = synth.make_instance("n16_m4096_k16", seed=0)
    inst.psi = np.ascontiguousarray(inst.psi[:2])
    inst.w = np.full(2, 0.5, np.float32)
    plan = qst.Plan(inst.n, inst.M, 2, inst.nnz, fixed_rounds=2, max_bin_settings=96)
    assert plan.geometry()["fixed_rounds"] == 2
    data = qst.Data.from_numpy(inst.n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    psi, w = torch.from_numpy(inst.psi).cuda(), torch.from_numpy(inst.w).cuda()
    p_obs, c_obs, loss = plan.forward(psi, w, data)
    g, gw = plan.adjoint(psi, w, data, c_obs)
    torch.cuda.synchronize()
    assert plan.status() == 0
    out = dict(inst=inst, p_obs=p_obs.cpu().numpy().astype(np.float64), c_obs=c_obs.cpu().numpy().astype(np.float64),
               loss=loss.item(), g=g.cpu().numpy().astype(np.complex128), gw=gw.cpu().numpy().astype(np.float64))
    plan.close()
    return out


def test_all_settings_forward_k2(c3k2):
    """p and c at every observed outcome of all 4096 settings against the FP64 oracle
    (settings sharded over the host cores).  The p error is taken relative to the
    largest observed p of its setting, which is no larger than the setting's largest
    p, so the bound is at least as strict as the normwise one."""
    inst = c3k2["inst"]
    ref = oracle.forward_sharded(inst.n, inst.basis, inst.psi.astype(np.complex128), inst.w.astype(np.float64),
                                 inst.row_ptr, inst.outcome, inst.count, inst.shots, eps=inst.eps)
    p = c3k2["p_obs"]
    worst = 0.0
    for s in range(inst.M):
        lo, hi = inst.row_ptr[s], inst.row_ptr[s + 1]
        r = ref["p_obs"][lo:hi]
        worst = max(worst, np.max(np.abs(p[lo:hi] - r)) / np.max(r))
    assert worst <= P_TOL, worst
    np.testing.assert_allclose(c3k2["c_obs"], ref["c_obs"], rtol=C_TOL)
    assert abs(c3k2["loss"] - ref["loss"]) <= 1e-5 * abs(ref["loss"])


def test_all_settings_adjoint_k2(c3k2):
    """G psi_k summed over all 4096 settings, element by element against the FP64
    oracle given the same c (the sum over settings of the headline size)."""
    inst = c3k2["inst"]
    ref = oracle.adjoint_sharded(inst.n, inst.basis, inst.psi.astype(np.complex128), inst.w.astype(np.float64),
                                 inst.row_ptr, inst.outcome, c3k2["c_obs"])
    for k in range(2):
        nrm = np.max(np.abs(ref["grad_psi"][k]))
        err = np.max(np.abs(c3k2["g"][k] - ref["grad_psi"][k])) / nrm
        assert err <= G_TOL, (k, err)
    np.testing.assert_allclose(c3k2["gw"], ref["grad_w"], rtol=H_TOL)


def test_evaluate_equals_forward_then_adjoint_at_full_size(c3):
    """qst_evaluate in the bench's configuration (transform cache on) gives the
    bits of qst_forward + qst_adjoint on the whole n = 16, M = 4096, K = 16 workload."""
    p_obs, c_obs, loss, g, gw = c3["plan"].evaluate(c3["psi"], c3["w"], c3["data"])
    torch.cuda.synchronize()
    assert c3["plan"].status() == 0
    assert torch.equal(p_obs, c3["p_obs"]) and torch.equal(c_obs, c3["c_obs"])
    assert loss.item() == c3["loss"].item()
    assert torch.equal(g, c3["g"]) and torch.equal(gw, c3["gw"])
