"""The tensor-core chunk transforms (plan precision T = 1, 2, 3: six-qubit group
products on tcgen05.mma kind::f16, the data split into T BF16 terms, operators
exact in BF16, FP32 accumulation) against the FP64 oracle.

Error bound (a priori, per amplitude).  Each group product multiplies data
rows by an exact matrix with entries 0, +-1; the data enter as T BF16 terms,
x = x_1 + ... + x_T + r with |r| <= 2^-8T |x| per real component (each term
rounds the previous residual to 8 significant bits; BF16 has FP32's exponent
range).  The tensor core adds at most 2^m_g T nonzero products into an FP32
accumulator (m_g <= 6 X/Y qubits of the group); charging 2^-23 of the sum of
their magnitudes per addition (one unit of FP32 rounding, whether the
accumulator rounds to nearest or truncates), and the same for each of the n
FP32 additions of the source build, the transform of an atom at outcome u
differs from the exact one by at most

    beta_T * A_u,   beta_T = 2 * 2^-8T (1 + 2^-7) + (2 * 64 T + 2 n) 2^-23,
    A_u = (|V_s| (|Re psi| + |Im psi|))_u,

|V_s| the entrywise absolute value of the rotation (2^-m/2 times sums over
the qubits rotated by X or Y).  Then |dp_u| <= sum_k w_k (2 |phi_ku| + beta_T A_ku)
beta_T A_ku.  The tests check this bound on every outcome at n = 12.

Refined (observed) behaviour: the data-split errors enter with random signs,
so the error of the setting's distribution is about 2^-8T relative to its
largest probability, and the gradient error a few times that.  T = 3 meets
the FP32 path's tolerances (p: 1e-5 of the setting's largest probability;
c, gradients, h: 1e-4; loss 1e-5); T = 2 is checked against 8 * 2^-16 and
T = 1 against 8 * 2^-8 in p, 64 * 2^-8T in the gradients.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_19577_b300 import qst, synth
from test_gpu_parity import compare, run_gpu, run_gpu_evaluate, run_oracle

pytestmark = pytest.mark.gpu


def abs_rotation(n, basis_row, x):
    """|V_s| x for a real nonnegative vector x (qubit q <-> bit n - 1 - q)."""
    y = x.copy()
    m = 0
    for q in range(n):
        if basis_row[q] == 0:
            continue
        m += 1
        bit = 1 << (n - 1 - q)
        y = y.reshape(-1, 2, bit)
        s = y[:, 0, :] + y[:, 1, :]
        y = np.stack([s, s], axis=1).reshape(-1)
    return y * 2.0 ** (-m / 2)


def beta(T, n):
    return 2 * 2.0 ** (-8 * T) * (1 + 2.0 ** -7) + (2 * 64 * T + 2 * n) * 2.0 ** -23


@pytest.mark.parametrize("T", [1, 2, 3])
def test_dense_probabilities_within_the_a_priori_bound(T):
    n, M, K = 12, 30, 3
    inst = synth.random_instance(n, M, K, 600, 5100 + T)
    gpu = run_gpu(inst, dense=True, fixed_rounds=2, precision=T)
    ref = run_oracle(inst, dense=True)
    psi = inst.psi.astype(np.complex128)
    w = inst.w.astype(np.float64)
    # |phi_ku|^2 of each atom alone (dense oracle forward with one unit weight)
    phi2 = [oracle.forward(n, inst.basis, psi[k:k + 1], np.ones(1), np.zeros(M + 1, np.int64),
                           np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.ones(M, np.uint32),
                           dense=True)["p_dense"] for k in range(K)]
    b = beta(T, n)
    for s in range(M):
        dp = np.abs(gpu["p_dense"][s] - ref["p_dense"][s])
        bound = 4 * 2.0 ** -24 * np.abs(ref["p_dense"][s])  # the scale and |.|^2 in FP32
        for k in range(K):
            A = abs_rotation(n, inst.basis[s], np.abs(psi[k].real) + np.abs(psi[k].imag))
            bound += w[k] * (2 * np.sqrt(phi2[k][s]) + b * A) * b * A
        assert np.all(dp <= bound), (s, float(np.max(dp / np.maximum(bound, 1e-300))))


@pytest.mark.parametrize("T", [1, 2])
def test_fewer_terms_within_the_refined_bounds(T):
    """BF16 x 1 and x 2: the distribution's error about 2^-8T of its largest
    probability, the gradients within 64 2^-8T; fewer terms, larger error."""
    inst = synth.random_instance(14, 24, 3, 1500, 5200 + T)
    ref = run_oracle(inst)
    errs = {}
    for t in (T, 3):
        gpu = run_gpu(inst, fixed_rounds=2, precision=t)
        pe = 0.0
        for s in range(inst.M):
            lo, hi = inst.row_ptr[s], inst.row_ptr[s + 1]
            if hi > lo:
                pe = max(pe, np.max(np.abs(gpu["p_obs"][lo:hi] - ref["p_obs"][lo:hi])) / ref["p_max"][s])
        ge = max(np.max(np.abs(gpu["grad_psi"][k] - ref["grad_psi"][k])) / np.max(np.abs(ref["grad_psi"][k]))
                 for k in range(inst.K))
        errs[t] = (pe, ge)
    pe, ge = errs[T]
    assert pe <= 8 * 2.0 ** (-8 * T), pe
    assert ge <= 64 * 2.0 ** (-8 * T), ge
    assert pe > errs[3][0] and ge > errs[3][1]


@pytest.mark.parametrize("n,M,K,shots,seed", [(12, 40, 3, 800, 1), (13, 30, 2, 1000, 2), (14, 20, 4, 1500, 3),
                                              (15, 12, 1, 1500, 4), (16, 6, 2, 2000, 5)])
def test_bf16x3_meets_the_fp32_tolerances(n, M, K, shots, seed):
    """BF16 x 3 against the oracle at the FP32 path's tolerances: qst_forward +
    qst_adjoint (the adjoint recomputes the transforms on the tensor cores) and
    qst_evaluate (the adjoint reads the forward's stored transforms) give the
    same bits."""
    inst = synth.random_instance(n, M, K, shots, 5300 + seed)
    ref = run_oracle(inst)
    sep = run_gpu(inst, fixed_rounds=2, precision=3)
    compare(inst, sep, ref)
    ev = run_gpu_evaluate(inst, fixed_rounds=2, precision=3)
    for key in ["p_obs", "c_obs", "grad_psi", "grad_w"]:
        assert np.array_equal(ev[key], sep[key]), key
    assert ev["loss"] == sep["loss"]


def test_bf16x3_without_the_cache_and_with_split_bins():
    """phi_cache = 0 (qst_evaluate's adjoint recomputes the transforms), bins of
    one and of five settings, empty rows."""
    inst = synth.random_instance(13, 33, 3, 300, 5401)
    ref = run_oracle(inst)
    for smax in (1, 5):
        compare(inst, run_gpu_evaluate(inst, fixed_rounds=2, precision=3, phi_cache=0, max_bin_settings=smax), ref)


def test_refusals():
    with pytest.raises(qst.QSTError):  # three-round kernels have no tensor-core form
        qst.Plan(12, 4, 2, 10, fixed_rounds=1, precision=3)
    with pytest.raises(qst.QSTError):  # chunks below 12 qubits
        qst.Plan(10, 4, 2, 10, precision=1)
    with pytest.raises(qst.QSTError):
        qst.Plan(12, 4, 2, 10, fixed_rounds=2, precision=4)


def test_full_workload_against_fp32_and_sampled_oracle_settings():
    """The n = 16, M = 4096, K = 16 workload with BF16 x 3 in the bench's plan:
    the gradients against the FP32 plan's (oracle-checked elsewhere) over all
    settings, and p / c on sampled settings against the oracle."""
    inst = synth.make_instance("n16_m4096_k16", seed=0)
    data = qst.Data.from_numpy(inst.n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    psi, w = torch.from_numpy(inst.psi).cuda(), torch.from_numpy(inst.w).cuda()
    tc = qst.Plan(inst.n, inst.M, inst.K, inst.nnz, precision=3)
    p_t, c_t, l_t, g_t, gw_t = tc.evaluate(psi, w, data)
    fp = qst.Plan(inst.n, inst.M, inst.K, inst.nnz)
    p_f, c_f, l_f, g_f, gw_f = fp.evaluate(psi, w, data)
    torch.cuda.synchronize()
    assert tc.status() == 0 and fp.status() == 0
    gn = g_f.abs().amax(dim=1)
    assert torch.all((g_t - g_f).abs().amax(dim=1) <= 1e-4 * gn)
    assert torch.all((gw_t - gw_f).abs() <= 1e-4 * gw_f.abs())
    assert abs(l_t.item() - l_f.item()) <= 1e-5 * abs(l_f.item())
    sel = synth.rng_for(4321).choice(inst.M, 4, replace=False)
    rp, outs, cnts = [0], [], []
    for s in sel:
        lo, hi = inst.row_ptr[s], inst.row_ptr[s + 1]
        outs.append(inst.outcome[lo:hi])
        cnts.append(inst.count[lo:hi])
        rp.append(rp[-1] + hi - lo)
    rp = np.array(rp, np.int64)
    ref = oracle.forward(inst.n, inst.basis[sel], inst.psi.astype(np.complex128), inst.w.astype(np.float64), rp,
                         np.concatenate(outs), np.concatenate(cnts), inst.shots[sel], eps=inst.eps, B=inst.M)
    p = p_t.cpu().numpy()
    c = c_t.cpu().numpy()
    for j, s in enumerate(sel):
        lo, hi = inst.row_ptr[s], inst.row_ptr[s + 1]
        r = ref["p_obs"][rp[j]:rp[j + 1]]
        assert np.max(np.abs(p[lo:hi] - r)) / np.max(r) <= 1e-5
        np.testing.assert_allclose(c[lo:hi], ref["c_obs"][rp[j]:rp[j + 1]], rtol=1e-4)
    tc.close()
    fp.close()
