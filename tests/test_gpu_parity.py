"""Parity of the CUDA forward/adjoint (through the C ABI) with the FP64 oracle.

Tolerances (FP32 path against FP64; the rotation is add-only, so each of the
<= n butterfly stages adds at most one rounding of relative size 2^-24 to every
amplitude, and |.|^2 doubles it):
  * probabilities: per setting max_u |dp_u| / max_u p_u <= 1e-5, the maximum of
    p taken over all 2^n outcomes of the setting (the normwise error of the
    setting's distribution), the difference over the outcomes the kernel
    outputs (all of them for the dense output, the observed ones for p_obs)
  * likelihood ratio c: relative 1e-4; loss: relative 1e-5
  * gradients: per atom ||d grad_k||_inf / ||grad_k||_inf <= 1e-4; h: relative 1e-4
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_19577_b300 import qst, synth

pytestmark = pytest.mark.gpu

P_TOL, C_TOL, L_TOL, G_TOL, H_TOL = 1e-5, 1e-4, 1e-5, 1e-4, 1e-4


def run_gpu(inst, dense=False, **plan_kw):
    plan = qst.Plan(inst.n, inst.M, inst.K, inst.nnz, eps=inst.eps, **plan_kw)
    data = qst.Data.from_numpy(inst.n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    psi = torch.from_numpy(inst.psi).cuda()
    w = torch.from_numpy(inst.w).cuda()
    p_dense = torch.zeros(inst.M, inst.D, dtype=torch.float32, device="cuda") if dense else None
    p_obs, c_obs, loss = plan.forward(psi, w, data, p_dense=p_dense)
    g, gw = plan.adjoint(psi, w, data, c_obs)
    torch.cuda.synchronize()
    assert plan.status() == 0
    out = dict(p_obs=p_obs.cpu().numpy().astype(np.float64), c_obs=c_obs.cpu().numpy().astype(np.float64),
               loss=float(loss.item()), grad_psi=g.cpu().numpy().astype(np.complex128),
               grad_w=gw.cpu().numpy().astype(np.float64))
    if dense:
        out["p_dense"] = p_dense.cpu().numpy().astype(np.float64)
    plan.close()
    return out


def setting_pmax(n, basis, psi, w):
    """max_u p_{s,u} over all 2^n outcomes of every setting (FP64 oracle, dense)."""
    M, D = basis.shape[0], 1 << n
    step = max(1, (1 << 24) // D)
    out = np.zeros(M)
    for lo in range(0, M, step):
        hi = min(M, lo + step)
        f = oracle.forward(n, basis[lo:hi], psi, w, np.zeros(hi - lo + 1, np.int64), np.zeros(0, np.uint32),
                           np.zeros(0, np.uint32), np.ones(hi - lo, np.uint32), dense=True)
        out[lo:hi] = f["p_dense"].max(axis=1)
    return out


def run_oracle(inst, dense=False):
    psi = inst.psi.astype(np.complex128)
    w = inst.w.astype(np.float64)
    f = oracle.forward(inst.n, inst.basis, psi, w, inst.row_ptr, inst.outcome, inst.count, inst.shots,
                       eps=inst.eps, dense=dense)
    a = oracle.adjoint(inst.n, inst.basis, psi, w, inst.row_ptr, inst.outcome, f["c_obs"])
    pmax = f["p_dense"].max(axis=1) if dense else setting_pmax(inst.n, inst.basis, psi, w)
    return {**f, **a, "p_max": pmax}


def compare(inst, gpu, ref, dense=False):
    if dense:
        err = np.max(np.abs(gpu["p_dense"] - ref["p_dense"]), axis=1) / np.max(ref["p_dense"], axis=1)
        assert err.max() <= P_TOL, err.max()
    for s in range(inst.M):
        lo, hi = inst.row_ptr[s], inst.row_ptr[s + 1]
        if hi > lo:
            scale = max(ref["p_max"][s], 1e-300)
            err = np.max(np.abs(gpu["p_obs"][lo:hi] - ref["p_obs"][lo:hi])) / scale
            assert err <= P_TOL, (s, err)
    if inst.nnz:
        np.testing.assert_allclose(gpu["c_obs"], ref["c_obs"], rtol=C_TOL, atol=1e-12)
    assert abs(gpu["loss"] - ref["loss"]) <= L_TOL * max(abs(ref["loss"]), 1e-30)
    for k in range(inst.K):
        gk, rk = gpu["grad_psi"][k], ref["grad_psi"][k]
        nrm = np.max(np.abs(rk))
        if nrm > 0:
            assert np.max(np.abs(gk - rk)) / nrm <= G_TOL, (k, np.max(np.abs(gk - rk)) / nrm)
        else:
            assert np.max(np.abs(gk)) == 0
    np.testing.assert_allclose(gpu["grad_w"], ref["grad_w"], rtol=H_TOL, atol=1e-12)


@pytest.mark.parametrize("n,M,K,shots,seed", [
    (1, 3, 1, 20, 0), (2, 5, 2, 30, 1), (3, 7, 3, 50, 2), (4, 9, 2, 100, 3), (5, 11, 3, 100, 4),
    (6, 13, 4, 200, 5), (7, 10, 2, 300, 6), (9, 17, 3, 400, 7), (10, 23, 3, 500, 8),
    (11, 9, 2, 800, 9), (12, 21, 2, 1000, 10), (13, 12, 2, 1500, 11), (14, 10, 2, 2000, 12),
])
def test_parity_shapes(n, M, K, shots, seed):
    inst = synth.random_instance(n, M, K, shots, seed)
    dense = n <= 12
    compare(inst, run_gpu(inst, dense=dense), run_oracle(inst, dense=dense), dense=dense)


@pytest.mark.parametrize("chunk", [3, 5, 6, 7, 8, 9])
def test_parity_forced_high_bits(chunk):
    """Small n with a forced small chunk exercises the binned high-bit path
    (r = n - chunk up to 4) against the oracle."""
    n = min(chunk + 4, 12)
    inst = synth.random_instance(n, 40, 3, 300, 100 + chunk)
    compare(inst, run_gpu(inst, dense=True, chunk_qubits=chunk),
            run_oracle(inst, dense=True), dense=True)


@pytest.mark.parametrize("n,chunk,reg_bits", [(12, 0, 4), (14, 0, 4), (16, 0, 4), (11, 7, 4), (9, 5, 4),
                                              (9, 5, 5), (13, 9, 5)])
def test_parity_register_layouts(n, chunk, reg_bits):
    """Both register blockings (16 or 32 amplitudes per thread and round)."""
    inst = synth.random_instance(n, 12 if n >= 14 else 30, 2, 1500, 900 + n + reg_bits)
    compare(inst, run_gpu(inst, chunk_qubits=chunk, reg_bits=reg_bits), run_oracle(inst))


@pytest.mark.parametrize("smax", [1, 2, 5])
def test_parity_split_bins(smax):
    inst = synth.random_instance(8, 37, 3, 200, 200 + smax)
    compare(inst, run_gpu(inst, dense=True, max_bin_settings=smax), run_oracle(inst, dense=True), dense=True)


def test_parity_n16_several_tiles():
    """n = 16 uses the production split (12 chunk bits, 4 binned high bits)."""
    inst = synth.random_instance(16, 6, 2, 2000, 300)
    compare(inst, run_gpu(inst), run_oracle(inst))


def test_parity_edge_settings_and_empty_rows():
    """All-Z, all-X, all-Y settings, empty rows and a row observing every outcome."""
    n, K = 8, 3
    D = 1 << n
    rng = synth.rng_for(400)
    basis = np.concatenate([np.zeros((1, n), np.uint8), np.ones((1, n), np.uint8), np.full((1, n), 2, np.uint8),
                            synth.pauli_settings(n, 5, rng)])
    M = basis.shape[0]
    rows, outs, cnts = [0], [], []
    for s in range(M):
        if s in (2, 5):
            o = np.zeros(0, np.uint32)          # empty rows
        elif s == 3:
            o = np.arange(D, dtype=np.uint32)   # dense row
        else:
            o = np.unique(rng.integers(0, D, 40)).astype(np.uint32)
        outs.append(o)
        cnts.append(rng.integers(1, 9, o.size).astype(np.uint32))
        rows.append(rows[-1] + o.size)
    shots = np.array([max(1, int(c.sum())) for c in cnts], np.uint32)
    inst = synth.Instance(name="edge", n=n, basis=basis, shots=shots, row_ptr=np.array(rows, np.int64),
                          outcome=np.concatenate(outs), count=np.concatenate(cnts),
                          psi=synth.random_atoms(n, K, rng).astype(np.complex64),
                          w=np.array([0.5, 0.3, 0.2], np.float32))
    compare(inst, run_gpu(inst, dense=True), run_oracle(inst, dense=True), dense=True)


def test_parity_n4_all_81_settings():
    """The n = 4 workload (all 3^4 Pauli strings, counts drawn from the truth's
    Born probabilities given by the oracle)."""
    def probs(basis, tw, ta):
        D = 1 << 4
        return np.stack([oracle.forward(4, basis[s:s + 1], ta, tw, np.array([0, D]), np.arange(D),
                                        np.ones(D), np.array([D]), dense=True)["p_dense"][0]
                         for s in range(basis.shape[0])])
    inst = synth.make_instance("n4_all81", seed=0, probs_fn=probs)
    compare(inst, run_gpu(inst, dense=True), run_oracle(inst, dense=True), dense=True)


def test_parity_n12_workload_prefix():
    """The first 120 settings of the n = 12, M = 2000, K = 8 workload."""
    inst = synth.make_instance("n12_m2000_k8", seed=0)
    m = 120
    e = inst.row_ptr[m]
    sub = synth.Instance(name="n12_prefix", n=12, basis=inst.basis[:m], shots=inst.shots[:m],
                         row_ptr=inst.row_ptr[:m + 1], outcome=inst.outcome[:e], count=inst.count[:e],
                         psi=inst.psi, w=inst.w)
    compare(sub, run_gpu(sub), run_oracle(sub))


def test_repeat_calls_are_bitwise_deterministic():
    inst = synth.random_instance(12, 30, 3, 800, 500)
    a, b = run_gpu(inst), run_gpu(inst)
    for key in ["p_obs", "c_obs", "grad_psi", "grad_w"]:
        assert np.array_equal(a[key], b[key]), key
    assert a["loss"] == b["loss"]


def test_host_buffer_entry_point_matches_device_path():
    inst = synth.random_instance(10, 25, 3, 500, 600)
    plan = qst.Plan(inst.n, inst.M, inst.K, inst.nnz)
    loss, g, gw = plan.evaluate_host(inst.psi, inst.w, inst.basis, inst.row_ptr, inst.outcome, inst.count,
                                     inst.shots)
    ref = run_gpu(inst)
    assert loss == ref["loss"]
    assert np.array_equal(g.astype(np.complex128), ref["grad_psi"])
    assert np.array_equal(gw.astype(np.float64), ref["grad_w"])


def test_device_validation_flags_bad_data():
    inst = synth.random_instance(6, 5, 2, 50, 700)
    plan = qst.Plan(inst.n, inst.M, inst.K, inst.nnz)
    bad = inst.basis.copy()
    bad[1, 2] = 7
    data = qst.Data.from_numpy(inst.n, bad, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    psi, w = torch.from_numpy(inst.psi).cuda(), torch.from_numpy(inst.w).cuda()
    plan.forward(psi, w, data)
    assert plan.status() & 1
    out = inst.outcome.copy()
    lo = inst.row_ptr[2]
    if inst.row_ptr[3] - lo >= 2:
        out[lo], out[lo + 1] = out[lo + 1], out[lo]  # breaks the ascending order
    else:
        out[lo] = 1 << 6                             # out of range
    data = qst.Data.from_numpy(inst.n, inst.basis, inst.row_ptr, out, inst.count, inst.shots)
    plan.forward(psi, w, data)
    assert plan.status() & 2
    plan.forward(psi, w, qst.Data.from_numpy(inst.n, inst.basis, inst.row_ptr, inst.outcome, inst.count,
                                             inst.shots))
    assert plan.status() == 0


def test_autograd_function_matches_oracle_gradient():
    """torch's complex gradient of a real loss is 2 dL/dpsi^*; the wrapper's
    backward must give exactly that (checked against the oracle) and a
    finite-difference directional derivative of the GPU loss."""
    inst = synth.random_instance(9, 30, 3, 500, 800)
    plan = qst.Plan(inst.n, inst.M, inst.K, inst.nnz, eps=1e-3)
    inst.eps = 1e-3
    data = qst.Data.from_numpy(inst.n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    psi = torch.from_numpy(inst.psi).cuda().requires_grad_(True)
    w = torch.from_numpy(inst.w).cuda().requires_grad_(True)
    L = qst.qst_loss(psi, w, plan, data)
    L.backward()
    ref = run_oracle(inst)
    g = psi.grad.cpu().numpy().astype(np.complex128)
    np.testing.assert_allclose(g, 2 * ref["grad_psi"], atol=G_TOL * np.max(np.abs(ref["grad_psi"])) * 2)
    np.testing.assert_allclose(w.grad.cpu().numpy(), ref["grad_w"], rtol=H_TOL)
    # directional derivative of the GPU loss in FP64 oracle terms
    rng = synth.rng_for(801)
    delta = (rng.standard_normal(inst.psi.shape) + 1j * rng.standard_normal(inst.psi.shape))
    t = 1e-4
    lp = oracle.forward(inst.n, inst.basis, inst.psi.astype(np.complex128) + t * delta, inst.w.astype(np.float64),
                        inst.row_ptr, inst.outcome, inst.count, inst.shots, eps=1e-3)["loss"]
    lm = oracle.forward(inst.n, inst.basis, inst.psi.astype(np.complex128) - t * delta, inst.w.astype(np.float64),
                        inst.row_ptr, inst.outcome, inst.count, inst.shots, eps=1e-3)["loss"]
    fd = (lp - lm) / (2 * t)
    an = float(np.real(np.sum(np.conj(g) * delta)))  # <torch grad, delta> = 2 Re<dL/dpsi^*, delta>
    assert abs(fd - an) <= 1e-3 * max(1.0, abs(fd))


def test_autotuner_returns_a_valid_fastest_layout():
    inst = synth.random_instance(13, 40, 2, 1000, 1300)
    data = qst.Data.from_numpy(inst.n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    psi, w = torch.from_numpy(inst.psi).cuda(), torch.from_numpy(inst.w).cuda()
    best, table = qst.autotune(psi, w, data, reps=1, warmup=1)
    assert table and best == table[0][0] and all(t > 0 for _, t in table)
    compare(inst, run_gpu(inst, **best), run_oracle(inst))


@pytest.mark.parametrize("n,fixed", [(n, fx) for n in (12, 13, 16) for fx in (2, 1, 0)])
def test_parity_fixed_and_per_setting_rounds(n, fixed):
    """12-qubit chunks run two 6-qubit rounds (bits 6..11, 0..5; two atoms per
    CTA), three fixed 4-qubit rounds (bits 8..11, 4..7, 0..3) or rounds chosen
    per setting; all against the oracle, with settings whose whole 4- or
    6-qubit groups are Z (skipped rounds), all-X, all-Y and random.  K = 3 is
    odd, so the last two-round CTA has one atom only."""
    rng = synth.rng_for(700 + n)
    M_rand = 14
    special = []
    for q0, width in ((0, 4), (4, 4), (8, 4), (0, 6), (6, 6)):  # chunk bits q0.. all Z, the rest random X/Y
        row = rng.integers(1, 3, n).astype(np.uint8)
        for b in range(q0, q0 + width):
            row[n - 1 - b] = 0                # qubit n-1-b carries outcome bit b
        special.append(row)
    special += [np.zeros(n, np.uint8), np.ones(n, np.uint8), np.full(n, 2, np.uint8)]
    basis = np.concatenate([np.stack(special), synth.pauli_settings(n, M_rand, rng)])
    inst = synth.random_instance(n, basis.shape[0], 3, 800, 710 + n, basis=basis)
    dense = n <= 12
    compare(inst, run_gpu(inst, dense=dense, fixed_rounds=fixed), run_oracle(inst, dense=dense), dense=dense)


@pytest.mark.parametrize("n,M,K,smax,seed", [(12, 23, 1, 96, 0), (12, 31, 2, 3, 1), (13, 29, 5, 1, 2),
                                              (14, 40, 1, 7, 3), (15, 18, 3, 96, 4), (16, 9, 1, 2, 5)])
def test_parity_two_round_bins_and_atoms(n, M, K, smax, seed):
    """The two-round kernels with one atom per CTA (K = 1, odd K), bins split to
    a few settings or a single one, and 0..4 high bits, against the oracle."""
    inst = synth.random_instance(n, M, K, 600, 900 + seed)
    dense = n <= 12
    compare(inst, run_gpu(inst, dense=dense, fixed_rounds=2, max_bin_settings=smax), run_oracle(inst, dense=dense),
            dense=dense)


@pytest.mark.parametrize("n,M,K,smax,shots,seed", [(11, 23, 3, 96, 1500, 0), (11, 37, 4, 5, 300, 1),
                                                    (11, 19, 9, 1, 1500, 2), (10, 29, 5, 96, 1500, 3),
                                                    (10, 33, 8, 7, 150, 4), (10, 21, 11, 2, 1500, 5)])
def test_parity_two_round_small_chunks(n, M, K, smax, shots, seed):
    """Whole states of 10 and 11 qubits on the two-round kernels (8 and 4 atoms
    per CTA, atoms past K inactive): qst_forward + qst_adjoint (the recomputing
    adjoint), qst_evaluate with the transform cache (the cached adjoint) and with
    the automatic choice (cache only for sparse outcomes) against the oracle,
    dense p, and bitwise equal."""
    inst = synth.random_instance(n, M, K, shots, 1300 + seed)
    geo = qst.Plan(n, M, K, inst.nnz, max_bin_settings=smax).geometry()
    assert geo == {"chunk_qubits": n, "high_qubits": 0, "fixed_rounds": 2}
    ref = run_oracle(inst, dense=True)
    sep = run_gpu(inst, dense=True, max_bin_settings=smax)
    compare(inst, sep, ref, dense=True)
    ev = run_gpu_evaluate(inst, max_bin_settings=smax, phi_cache=1)
    compare(inst, ev, ref)
    auto = run_gpu_evaluate(inst, max_bin_settings=smax)
    for other in (ev, auto):
        for key in ["p_obs", "c_obs", "grad_psi", "grad_w"]:
            assert np.array_equal(other[key], sep[key]), key


@pytest.mark.parametrize("n,M,K,seed", [(5, 14, 3, 0), (12, 20, 4, 1), (16, 6, 2, 2)])
def test_tangent_matches_oracle(n, M, K, seed):
    """qst_tangent (Eq. atom-projected-descent-direction) from the adjoint's outputs,
    against the oracle's d_k = w_k (I - psi_k psi_k^*) G psi_k; for unit-norm atoms
    d_k is orthogonal to psi_k."""
    inst = synth.random_instance(n, M, K, 800, 1200 + seed)
    psi = inst.psi.astype(np.complex128)
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    inst.psi = psi.astype(np.complex64)
    plan = qst.Plan(n, inst.M, K, inst.nnz, eps=inst.eps)
    d = qst.Data.from_numpy(n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    tp, tw = torch.from_numpy(inst.psi).cuda(), torch.from_numpy(inst.w).cuda()
    _, c_obs, _ = plan.forward(tp, tw, d)
    g, gw = plan.adjoint(tp, tw, d, c_obs)
    t = plan.tangent(tp, tw, g, gw).cpu().numpy().astype(np.complex128)
    ref = run_oracle(inst)
    want = oracle.tangent(inst.psi.astype(np.complex128), inst.w.astype(np.float64), ref["G_psi"])
    for k in range(K):
        # normwise against the size of the terms that are subtracted (w_k G psi_k)
        nrm = max(np.max(np.abs(want[k])), inst.w[k] * np.max(np.abs(ref["G_psi"][k])))
        assert np.max(np.abs(t[k] - want[k])) / nrm <= G_TOL
        p = inst.psi[k].astype(np.complex128)
        assert abs(np.vdot(p, t[k])) <= 1e-4 * np.linalg.norm(t[k])
    # aliasing the output onto grad_psi gives the same result
    t2 = plan.tangent(tp, tw, g, gw, out=g).cpu().numpy().astype(np.complex128)
    np.testing.assert_array_equal(t2, t)
    plan.close()


def run_gpu_evaluate(inst, **plan_kw):
    """qst_evaluate (forward, then the adjoint with the transform cache when the
    plan has one) -> the same dict as run_gpu."""
    plan = qst.Plan(inst.n, inst.M, inst.K, inst.nnz, eps=inst.eps, **plan_kw)
    data = qst.Data.from_numpy(inst.n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    psi = torch.from_numpy(inst.psi).cuda()
    w = torch.from_numpy(inst.w).cuda()
    p_obs, c_obs, loss, g, gw = plan.evaluate(psi, w, data)
    torch.cuda.synchronize()
    assert plan.status() == 0
    out = dict(p_obs=p_obs.cpu().numpy().astype(np.float64), c_obs=c_obs.cpu().numpy().astype(np.float64),
               loss=float(loss.item()), grad_psi=g.cpu().numpy().astype(np.complex128),
               grad_w=gw.cpu().numpy().astype(np.float64))
    plan.close()
    return out


@pytest.mark.parametrize("n,M,K,smax,seed", [(12, 40, 3, 0, 0), (13, 31, 2, 7, 1), (14, 45, 5, 96, 2),
                                              (16, 9, 1, 2, 3), (16, 14, 4, 0, 4)])
def test_evaluate_with_transform_cache_matches_oracle(n, M, K, smax, seed):
    """qst_evaluate on two-round plans (transform cache on: the adjoint applies only
    the inverse rounds to c .* the stored transforms) against the oracle, and
    bitwise equal to qst_forward + qst_adjoint (the same arithmetic in another
    order of launches); odd K leaves the last CTA's second atom idle."""
    inst = synth.random_instance(n, M, K, 700, 1400 + seed)
    kw = dict(fixed_rounds=2, max_bin_settings=smax, phi_cache=1)
    ev = run_gpu_evaluate(inst, **kw)
    compare(inst, ev, run_oracle(inst))
    sep = run_gpu(inst, **kw)
    for key in ["p_obs", "c_obs", "grad_psi", "grad_w"]:
        assert np.array_equal(ev[key], sep[key]), key
    assert ev["loss"] == sep["loss"]


def test_evaluate_without_cache_and_other_families():
    """Without the cache (or on plans whose kernels have no cached adjoint)
    qst_evaluate is qst_forward + qst_adjoint."""
    inst = synth.random_instance(13, 20, 3, 600, 1450)
    for kw in (dict(fixed_rounds=2, phi_cache=0), dict(fixed_rounds=1), dict(fixed_rounds=0)):
        ev = run_gpu_evaluate(inst, **kw)
        sep = run_gpu(inst, **kw)
        for key in ["p_obs", "c_obs", "grad_psi", "grad_w"]:
            assert np.array_equal(ev[key], sep[key]), (kw, key)
    with pytest.raises(qst.QSTError):
        qst.Plan(inst.n, inst.M, inst.K, inst.nnz, fixed_rounds=1, phi_cache=1)


@pytest.mark.parametrize("n,M,K,smax,seed", [(5, 20, 3, 0, 0), (6, 37, 2, 5, 1), (8, 64, 5, 0, 2), (9, 30, 4, 96, 3),
                                              (9, 41, 3, 1, 4)])
def test_warp_unit_kernels(n, M, K, smax, seed):
    """States of 5..9 qubits in one chunk: a warp per (bin, atom), butterflies on
    the low five bits by lane shuffles (fixed_rounds = 3, the automatic choice)
    and the per-setting-round CTA kernels (fixed_rounds = 0), both against the
    oracle, dense p included; odd K, single-setting and full bins."""
    inst = synth.random_instance(n, M, K, 40 << min(n, 8), 1700 + seed)
    ref = run_oracle(inst, dense=True)
    for fr in (3, 0):
        compare(inst, run_gpu(inst, dense=True, fixed_rounds=fr, max_bin_settings=smax), ref, dense=True)
    plan = qst.Plan(n, M, K, inst.nnz)
    assert plan.geometry()["fixed_rounds"] == 3
    plan.close()
    with pytest.raises(qst.QSTError):
        qst.Plan(10, M, K, inst.nnz, fixed_rounds=3)
