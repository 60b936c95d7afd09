"""Pins of the FP64 oracle against things other than itself.

Each test fixes the oracle to an independent route: explicit Kronecker
matrices and traces (Eq. born-map with the Pauli POVM of Sec. IV), closed-form
distributions, linear inversion with the Pauli operator basis, POVM
completeness, and central finite differences of the loss (Eqs. weight-gradient
and atom-wirtinger-gradient).  A dropped term, a wrong sign, a wrong bit order
or a transposed rotation fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2607_19577_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")

# Textbook single-qubit objects, written out independently of the oracle's C code.
PAULI = {
    "I": np.eye(2, dtype=complex),
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
}
CODE = {0: "Z", 1: "X", 2: "Y"}


def eigen_rotation(code):
    """V whose row u is the conjugated eigenvector of the Pauli with eigenvalue (-1)^u,
    found numerically from the Pauli matrix (not typed in)."""
    P = PAULI[CODE[code]]
    vals, vecs = np.linalg.eigh(P)
    order = np.argsort(-vals)  # +1 first
    V = vecs[:, order].conj().T
    # fix each row's global phase so the first nonzero entry is real positive
    for r in range(2):
        j = np.flatnonzero(np.abs(V[r]) > 1e-12)[0]
        V[r] *= np.exp(-1j * np.angle(V[r, j]))
    return V


def dense_rotation(b):
    U = np.array([[1.0 + 0j]])
    for code in b:  # qubit 1 is the leftmost Kronecker factor
        U = np.kron(U, eigen_rotation(int(code)))
    return U


def dense_rho(psi, w):
    psi = np.asarray(psi, dtype=complex)
    return (psi.T * np.asarray(w)) @ psi.conj()


def csr_all_outcomes(M, D):
    row_ptr = np.arange(M + 1, dtype=np.int64) * D
    outcome = np.tile(np.arange(D, dtype=np.uint32), M)
    return row_ptr, outcome


@pytest.mark.parametrize("n,M,K,seed", [(1, 3, 1, 0), (2, 7, 2, 1), (3, 9, 3, 2), (5, 11, 4, 3), (7, 6, 3, 4)])
def test_forward_matches_dense_trace(n, M, K, seed):
    """p_{s,u} = <u|V_s rho V_s^*|u> with rho = Psi diag(w) Psi^* and dense Kronecker V_s."""
    inst = synth.random_instance(n, M, K, shots=50, seed=seed)
    psi = inst.psi.astype(np.complex128)
    w = inst.w.astype(np.float64)
    out = oracle.forward(n, inst.basis, psi, w, inst.row_ptr, inst.outcome, inst.count,
                         inst.shots, eps=1e-8, dense=True)
    rho = dense_rho(psi, w)
    for s in range(M):
        U = dense_rotation(inst.basis[s])
        p_ref = np.real(np.diag(U @ rho @ U.conj().T))
        np.testing.assert_allclose(out["p_dense"][s], p_ref, atol=1e-13, rtol=0)
    # loss and likelihood ratio from the dense probabilities (Eq. qst-loss, Eq. likelihood-ratio-vector)
    B = M
    L = 0.0
    for s in range(M):
        U = dense_rotation(inst.basis[s])
        p_ref = np.real(np.diag(U @ rho @ U.conj().T))
        for i in range(inst.row_ptr[s], inst.row_ptr[s + 1]):
            u = inst.outcome[i]
            pi, pihat = p_ref[u] / B, inst.count[i] / (B * inst.shots[s])
            L -= pihat * math.log(pi + 1e-8)
            assert abs(out["c_obs"][i] - pihat / (pi + 1e-8)) <= 1e-9 * max(1.0, out["c_obs"][i])
    assert abs(out["loss"] - L) <= 1e-12 * max(1.0, abs(L))


def test_golden_closed_forms():
    cases = json.load(open(GOLDEN))["cases"]
    for c in cases:
        n = c["n"]
        psi = (np.array(c["state_re"]) + 1j * np.array(c["state_im"]))[None, :]
        basis = np.array([c["basis"]], dtype=np.uint8)
        D = 1 << n
        row_ptr, outcome = csr_all_outcomes(1, D)
        out = oracle.forward(n, basis, psi, [1.0], row_ptr, outcome, np.ones(D, np.uint32),
                             np.array([D], np.uint32), dense=True)
        np.testing.assert_allclose(out["p_dense"][0], c["p"], atol=1e-14, err_msg=c["name"])


def _zbits_xy(b):
    return sum(1 for x in b if x != 0)


@pytest.mark.parametrize("n", [1, 3, 6, 9])
def test_zero_state_closed_form(n):
    """|0...0>: p(u) = 2^-n_XY if the Z-measured bits of u are 0, else 0."""
    rng = synth.rng_for(11, n)
    basis = synth.pauli_settings(n, 12, rng)
    D = 1 << n
    psi = np.zeros((1, D), complex)
    psi[0, 0] = 1
    row_ptr, outcome = csr_all_outcomes(12, D)
    out = oracle.forward(n, basis, psi, [1.0], row_ptr, outcome, np.ones(12 * D, np.uint32),
                         np.full(12, D, np.uint32), dense=True)
    for s in range(12):
        b = basis[s]
        nxy = _zbits_xy(b)
        for u in range(D):
            zbits_zero = all(((u >> (n - 1 - j)) & 1) == 0 for j in range(n) if b[j] == 0)
            want = 2.0 ** -nxy if zbits_zero else 0.0
            assert abs(out["p_dense"][s, u] - want) < 1e-14


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_ghz_closed_form(n):
    """GHZ parity statistics.  No Z: p(u) = 2^-n (1 + (-1)^|u| cos(m pi/2)), m = #Y.
    With Z present: 2^-(n_XY+1) if the Z-bits of u agree, else 0."""
    D = 1 << n
    psi = np.zeros((1, D), complex)
    psi[0, 0] = psi[0, D - 1] = 1 / math.sqrt(2)
    rng = synth.rng_for(5, n)
    basis = np.concatenate([synth.pauli_settings(n, 20, rng),
                            np.zeros((1, n), np.uint8),           # all Z
                            np.ones((1, n), np.uint8),            # all X
                            np.full((1, n), 2, np.uint8)])        # all Y
    M = basis.shape[0]
    row_ptr, outcome = csr_all_outcomes(M, D)
    out = oracle.forward(n, basis, psi, [1.0], row_ptr, outcome, np.ones(M * D, np.uint32),
                         np.full(M, D, np.uint32), dense=True)
    for s in range(M):
        b = basis[s]
        zq = [j for j in range(n) if b[j] == 0]
        m = sum(1 for x in b if x == 2)
        nxy = n - len(zq)
        for u in range(D):
            bits = [(u >> (n - 1 - j)) & 1 for j in range(n)]
            if not zq:
                want = 2.0 ** -n * (1 + (-1) ** sum(bits) * math.cos(m * math.pi / 2))
            else:
                zb = [bits[j] for j in zq]
                want = 2.0 ** -(nxy + 1) if (all(x == 0 for x in zb) or all(x == 1 for x in zb)) else 0.0
            assert abs(out["p_dense"][s, u] - want) < 1e-13, (s, u)


def test_product_state_closed_form():
    """Product of single-qubit eigenstates measured in matching / unbiased bases."""
    n = 6
    # per qubit: (state, basis, distribution over outcome bit)
    h = 1 / math.sqrt(2)
    kets = {"0": [1, 0], "1": [0, 1], "+": [h, h], "-": [h, -h], "+i": [h, 1j * h], "-i": [h, -1j * h]}
    choice = [("1", 0, [0, 1]), ("+", 1, [1, 0]), ("-i", 2, [0, 1]), ("0", 1, [0.5, 0.5]),
              ("+i", 0, [0.5, 0.5]), ("-", 2, [0.5, 0.5])]
    psi = np.array([1.0 + 0j])
    for st, _, _ in choice:
        psi = np.kron(psi, np.array(kets[st], complex))
    basis = np.array([[b for _, b, _ in choice]], np.uint8)
    D = 1 << n
    row_ptr, outcome = csr_all_outcomes(1, D)
    out = oracle.forward(n, basis, psi[None, :], [1.0], row_ptr, outcome, np.ones(D, np.uint32),
                         np.array([D], np.uint32), dense=True)
    for u in range(D):
        want = 1.0
        for j, (_, _, dist) in enumerate(choice):
            want *= dist[(u >> (n - 1 - j)) & 1]
        assert abs(out["p_dense"][0, u] - want) < 1e-14


def test_linear_inversion_full_pauli_set():
    """n = 4, all 81 settings: rho = 2^-n sum_P <P> P must equal Psi diag(w) Psi^*."""
    n = 4
    inst = synth.make_instance("n4_all81", seed=0, probs_fn=None)
    psi = inst.psi.astype(np.complex128)
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    w = np.array([0.4, 0.3, 0.2, 0.1])
    D = 1 << n
    row_ptr, outcome = csr_all_outcomes(81, D)
    out = oracle.forward(n, inst.basis, psi, w, row_ptr, outcome, np.ones(81 * D, np.uint32),
                         np.full(81, D, np.uint32), dense=True)
    key = {tuple(b): s for s, b in enumerate(inst.basis.tolist())}
    rho = np.zeros((D, D), complex)
    import itertools
    for labels in itertools.product("IXYZ", repeat=n):
        # any setting whose basis matches P on its support
        b = tuple({"X": 1, "Y": 2, "Z": 0, "I": 0}[l] for l in labels)
        s = key[b]
        expv = 0.0
        for u in range(D):
            sign = 1
            for j, l in enumerate(labels):
                if l != "I" and (u >> (n - 1 - j)) & 1:
                    sign = -sign
            expv += sign * out["p_dense"][s, u]
        P = np.array([[1.0 + 0j]])
        for l in labels:
            P = np.kron(P, PAULI[l])
        rho += expv * P / D
    np.testing.assert_allclose(rho, dense_rho(psi, w), atol=1e-13)


def test_probability_invariants():
    inst = synth.random_instance(8, 15, 5, shots=40, seed=21)
    psi = inst.psi.astype(np.complex128)
    w = inst.w.astype(np.float64)
    out = oracle.forward(8, inst.basis, psi, w, inst.row_ptr, inst.outcome, inst.count, inst.shots, dense=True)
    p = out["p_dense"]
    assert p.min() >= -1e-15
    norm = float(np.sum(w * np.sum(np.abs(psi) ** 2, axis=1)))
    np.testing.assert_allclose(p.sum(axis=1), norm, rtol=1e-13)


def test_loss_closed_form_all_z_zero_state():
    """All-Z settings on |0...0> with every shot on u = 0: pi = pihat = 1/B and
    L = -log(1/B + eps)."""
    n, B = 5, 7
    D = 1 << n
    psi = np.zeros((1, D), complex)
    psi[0, 0] = 1
    basis = np.zeros((B, n), np.uint8)
    row_ptr = np.arange(B + 1, dtype=np.int64)
    outcome = np.zeros(B, np.uint32)
    count = np.full(B, 100, np.uint32)
    eps = 1e-3
    out = oracle.forward(n, basis, psi, [1.0], row_ptr, outcome, count, np.full(B, 100, np.uint32), eps=eps)
    assert abs(out["loss"] + math.log(1.0 / B + eps)) < 1e-14
    np.testing.assert_allclose(out["c_obs"], (1.0 / B) / (1.0 / B + eps), rtol=1e-14)


def _loss(n, inst, psi, w, eps):
    return oracle.forward(n, inst.basis, psi, w, inst.row_ptr, inst.outcome, inst.count,
                          inst.shots, eps=eps)["loss"]


@pytest.mark.parametrize("n,M,K,seed", [(3, 9, 2, 0), (6, 14, 3, 1)])
def test_adjoint_finite_differences(n, M, K, seed):
    """dL/dt along a complex direction delta equals 2 Re<dJ/dpsi^*, delta>, and
    dL/dw_k = -h_k (central differences, FP64)."""
    inst = synth.random_instance(n, M, K, shots=200, seed=seed)
    psi = inst.psi.astype(np.complex128)
    w = inst.w.astype(np.float64)
    eps = 1e-3  # keeps the loss smooth at the FD step
    fw = oracle.forward(n, inst.basis, psi, w, inst.row_ptr, inst.outcome, inst.count, inst.shots, eps=eps)
    adj = oracle.adjoint(n, inst.basis, psi, w, inst.row_ptr, inst.outcome, fw["c_obs"])
    rng = synth.rng_for(99, seed)
    t = 1e-6
    for _ in range(3):
        delta = rng.standard_normal(psi.shape) + 1j * rng.standard_normal(psi.shape)
        fd = (_loss(n, inst, psi + t * delta, w, eps) - _loss(n, inst, psi - t * delta, w, eps)) / (2 * t)
        an = 2 * np.real(np.sum(np.conj(adj["grad_psi"]) * delta))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)
    for k in range(K):
        e = np.zeros(K)
        e[k] = t
        fd = (_loss(n, inst, psi, w + e, eps) - _loss(n, inst, psi, w - e, eps)) / (2 * t)
        assert abs(fd - adj["grad_w"][k]) <= 1e-6 * max(1.0, abs(fd))


def test_povm_completeness_gives_identity():
    """c == 1 at every outcome of every setting: G = sum_m E_m = I, so G v = v."""
    n, M = 6, 9
    D = 1 << n
    basis = synth.pauli_settings(n, M, synth.rng_for(3))
    row_ptr, outcome = csr_all_outcomes(M, D)
    v = synth.random_atoms(n, 3, synth.rng_for(4))
    Gv = oracle.apply_G(n, basis, row_ptr, outcome, np.ones(M * D), v)
    np.testing.assert_allclose(Gv, v, atol=1e-14)


def test_adjoint_identities_and_dense_G():
    """<psi_k|G psi_k> = h_k; sum_k w_k h_k = sum pihat pi/(pi+eps); G v against a
    dense G = sum_m c_m E_m built from Kronecker matrices."""
    n, M, K = 5, 10, 3
    inst = synth.random_instance(n, M, K, shots=300, seed=8)
    psi = inst.psi.astype(np.complex128)
    w = inst.w.astype(np.float64)
    fw = oracle.forward(n, inst.basis, psi, w, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    adj = oracle.adjoint(n, inst.basis, psi, w, inst.row_ptr, inst.outcome, fw["c_obs"])
    inner = np.sum(np.conj(psi) * adj["G_psi"], axis=1)
    np.testing.assert_allclose(inner.real, adj["h"], rtol=1e-12)
    assert np.max(np.abs(inner.imag)) < 1e-14
    pi = fw["p_obs"] / M
    pihat = inst.count / (M * np.repeat(inst.shots, np.diff(inst.row_ptr)))
    np.testing.assert_allclose(np.dot(w, adj["h"]), np.sum(pihat * pi / (pi + 1e-8)), rtol=1e-12)
    D = 1 << n
    G = np.zeros((D, D), complex)
    for s in range(M):
        U = dense_rotation(inst.basis[s])
        for i in range(inst.row_ptr[s], inst.row_ptr[s + 1]):
            e = np.zeros(D)
            e[inst.outcome[i]] = 1
            G += fw["c_obs"][i] * (U.conj().T @ np.diag(e) @ U) / M
    np.testing.assert_allclose(adj["G_psi"], (G @ psi.T).T, atol=1e-13)
    np.testing.assert_allclose(adj["grad_psi"], -w[:, None] * adj["G_psi"], atol=1e-15)
    # the tangent direction is orthogonal to its (unit-norm) atom
    psi_u = psi / np.linalg.norm(psi, axis=1, keepdims=True)
    d = oracle.tangent(psi_u, w, (G @ psi_u.T).T)
    assert np.max(np.abs(np.sum(np.conj(psi_u) * d, axis=1))) < 1e-13


def test_direct_amplitude_matches_transform():
    """The direct-summation amplitude (used for spot checks at large n) agrees with
    the dense Kronecker rotation."""
    n = 6
    rng = synth.rng_for(17)
    basis = synth.pauli_settings(n, 4, rng)
    psi = synth.random_atoms(n, 1, rng)[0]
    for s in range(4):
        U = dense_rotation(basis[s])
        phi = U @ psi
        for u in [0, 5, 33, 63]:
            assert abs(oracle.amplitude(n, basis[s], psi, u) - phi[u]) < 1e-13


def test_sharded_sums_equal_unsharded():
    """The measurement partition of Sec. III-B: loss, h and G psi summed over
    disjoint setting shards (with the global B) equal the unsharded values."""
    n, M, K = 6, 12, 3
    inst = synth.random_instance(n, M, K, shots=100, seed=31)
    psi = inst.psi.astype(np.complex128)
    w = inst.w.astype(np.float64)
    full = oracle.forward(n, inst.basis, psi, w, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    fadj = oracle.adjoint(n, inst.basis, psi, w, inst.row_ptr, inst.outcome, full["c_obs"])
    L, h, G = 0.0, np.zeros(K), np.zeros_like(psi)
    for lo, hi in [(0, 5), (5, 6), (6, 12)]:
        a, b = inst.row_ptr[lo], inst.row_ptr[hi]
        rp = inst.row_ptr[lo:hi + 1] - a
        f = oracle.forward(n, inst.basis[lo:hi], psi, w, rp, inst.outcome[a:b], inst.count[a:b],
                           inst.shots[lo:hi], B=M)
        g = oracle.adjoint(n, inst.basis[lo:hi], psi, w, rp, inst.outcome[a:b], f["c_obs"], B=M)
        L += f["loss"]
        h += g["h"]
        G += g["G_psi"]
    assert abs(L - full["loss"]) < 1e-13 * max(1, abs(L))
    np.testing.assert_allclose(h, fadj["h"], rtol=1e-13)
    np.testing.assert_allclose(G, fadj["G_psi"], atol=1e-15)


def test_sharded_oracle_equals_the_serial_oracle():
    """forward_sharded / adjoint_sharded (contiguous setting shards on host threads,
    summed in shard order) give the serial oracle's values: per-entry outputs
    exactly, sums to rounding."""
    inst = synth.random_instance(7, 23, 3, 300, 41)
    psi = inst.psi.astype(np.complex128)
    w = inst.w.astype(np.float64)
    f1 = oracle.forward(7, inst.basis, psi, w, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    a1 = oracle.adjoint(7, inst.basis, psi, w, inst.row_ptr, inst.outcome, f1["c_obs"])
    for threads in (1, 3, 8):
        f2 = oracle.forward_sharded(7, inst.basis, psi, w, inst.row_ptr, inst.outcome, inst.count, inst.shots,
                                    threads=threads)
        np.testing.assert_array_equal(f2["p_obs"], f1["p_obs"])
        np.testing.assert_array_equal(f2["c_obs"], f1["c_obs"])
        assert abs(f2["loss"] - f1["loss"]) <= 1e-14 * abs(f1["loss"])
        a2 = oracle.adjoint_sharded(7, inst.basis, psi, w, inst.row_ptr, inst.outcome, f1["c_obs"], threads=threads)
        np.testing.assert_allclose(a2["G_psi"], a1["G_psi"], rtol=0, atol=1e-14 * np.max(np.abs(a1["G_psi"])))
        np.testing.assert_allclose(a2["h"], a1["h"], rtol=1e-13)
        np.testing.assert_allclose(a2["grad_w"], a1["grad_w"], rtol=1e-13)
