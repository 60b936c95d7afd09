"""Pins of the oracle's update-rule helpers: simplex projection (KKT conditions,
closed forms, fixed points), the truncation map P_tau (its definition's cases),
and the spectral refactorisation (rho invariance, orthonormal atoms, eigenvalues
of a dense eigh of rho, which is a different route from the K x K Gram)."""
import numpy as np
import pytest

import oracle
from paper_2607_19577_b300 import synth


@pytest.mark.parametrize("seed", range(8))
def test_simplex_projection_kkt(seed):
    rng = np.random.default_rng(seed)
    K = int(rng.integers(1, 40))
    v = rng.standard_normal(K) * rng.choice([0.1, 1.0, 10.0])
    b = oracle.simplex_project(v)
    assert np.all(b >= 0) and abs(b.sum() - 1) < 1e-12
    # KKT: b = max(v - theta, 0) for one theta; active entries share v - b = theta,
    # inactive entries have v <= theta
    act = b > 0
    theta = np.mean(v[act] - b[act])
    np.testing.assert_allclose(v[act] - b[act], theta, atol=1e-12)
    assert np.all(v[~act] <= theta + 1e-12)
    # optimality against random feasible points (the projection is the closest)
    for _ in range(20):
        q = rng.dirichlet(np.ones(K))
        assert np.sum((v - b) ** 2) <= np.sum((v - q) ** 2) + 1e-12


def test_simplex_projection_closed_forms():
    np.testing.assert_allclose(oracle.simplex_project([0.2, 0.3, 0.5]), [0.2, 0.3, 0.5])  # fixed point
    np.testing.assert_allclose(oracle.simplex_project([3.0, 1.0]), [1.0, 0.0])            # 2D: theta = 2
    np.testing.assert_allclose(oracle.simplex_project([0.5, 0.5 + 0.2]), [0.4, 0.6])      # theta = 0.1
    np.testing.assert_allclose(oracle.simplex_project([0.0, 0.0, 0.0, 0.0]), [0.25] * 4)  # uniform shift


def test_prune_cases():
    keep, b = oracle.prune([0.5, 0.0005, 0.4995], 1e-3)
    assert list(keep) == [0, 2] and abs(b.sum() - 1) < 1e-15
    keep, b = oracle.prune([1e-4, 3e-4, 2e-4], 1e-3)  # nothing survives: keep the largest
    assert list(keep) == [1] and b[0] == 1.0
    keep, b = oracle.prune([0.001, 0.999], 1e-3)      # strict inequality drops 0.001
    assert list(keep) == [1]


@pytest.mark.parametrize("n,K,seed", [(3, 2, 0), (5, 4, 1), (7, 6, 2)])
def test_refactor_preserves_rho_and_gives_its_eigenpairs(n, K, seed):
    rng = synth.rng_for(seed, 77)
    psi = synth.random_atoms(n, K, rng)
    w = synth.dirichlet_weights(K, rng)
    rho = (psi.T * w) @ psi.conj()
    phi, wk = oracle.refactor(psi, w, 0.0)
    rho2 = (phi.T * wk) @ phi.conj()
    np.testing.assert_allclose(rho2, rho, atol=1e-12)
    np.testing.assert_allclose(phi.conj() @ phi.T, np.eye(phi.shape[0]), atol=1e-12)
    ev = np.sort(np.linalg.eigvalsh(rho))[::-1][:phi.shape[0]]
    np.testing.assert_allclose(wk, ev / ev.sum(), atol=1e-12)
    assert np.all(np.diff(wk) <= 1e-15)


def test_refactor_prunes_and_merges_duplicate_atoms():
    """Two copies of one atom are one eigenvector: the refactor returns rank 2 with the
    merged weight, and P_tau drops a negligible third atom."""
    rng = synth.rng_for(5)
    a = synth.random_atoms(6, 3, rng)
    psi = np.stack([a[0], a[0], a[1], a[2]])
    w = np.array([0.3, 0.3, 0.3995, 0.0005])
    phi, wk = oracle.refactor(psi, w, 1e-3)
    assert phi.shape[0] == 2
    rho = (psi.T * w) @ psi.conj()
    top = np.sort(np.linalg.eigvalsh(rho))[::-1][:2]
    np.testing.assert_allclose(wk, top / top.sum(), atol=1e-12)


def _data(inst):
    return dict(basis=inst.basis, row_ptr=inst.row_ptr, outcome=inst.outcome, count=inst.count, shots=inst.shots)


def test_oracle_step_is_monotone_and_feasible():
    """The acceptance rule makes J non-increasing; atoms stay unit norm and the
    weights stay on the simplex through every kind of slot."""
    inst = synth.make_instance("n4_all81", seed=3, K=4)
    data = _data(inst)
    psi = inst.psi.astype(np.complex128)
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    w = inst.w.astype(np.float64)
    J_prev = None
    for slot, r in [(0, 0), (1, 0), (0, 1), (0, 2), (1, 0), (2, 0), (0, 0), (1, 0)]:
        psi, w, J, acc, eta = oracle.step(4, data, psi, w, slot, r)
        if J_prev is not None:
            assert J <= J_prev + 1e-15
        J_prev = J
        act = w > 0
        assert abs(w.sum() - 1) < 1e-12 and np.all(w >= 0)
        np.testing.assert_allclose(np.linalg.norm(psi[act], axis=1), 1.0, atol=1e-12)


def test_oracle_atom_step_decreases_loss_for_small_eta():
    """The tangent direction is an ascent direction of the log-likelihood: for a small
    enough step the loss decreases (first-order check of Eq. atom-direction)."""
    inst = synth.random_instance(5, 20, 3, 400, 12)
    data = _data(inst)
    psi = inst.psi.astype(np.complex128)
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    w = inst.w.astype(np.float64)
    J0, f0 = oracle.objective(5, data, psi, w, 1e-8, 1e-3)
    adj = oracle.adjoint(5, data["basis"], psi, w, data["row_ptr"], data["outcome"], f0["c_obs"])
    g = oracle.tangent(psi[:1], w[:1], adj["G_psi"][:1])[0]
    t = psi[0] + 1e-4 * g
    pt = psi.copy()
    pt[0] = t / np.linalg.norm(t)
    J1, _ = oracle.objective(5, data, pt, w, 1e-8, 1e-3)
    assert J1 < J0


# ----------------------------------------------------------------- spectral step (Sec. III-C)

def _dense_S(inst, psi, w, c_obs, eta):
    """S = Psi diag(w) Psi^* + eta sum_m c_m E_m with E_m from Kronecker products of
    the single-qubit eigenbases (a route independent of the oracle's butterflies)."""
    from test_oracle_pins import dense_rotation
    D = 1 << inst.n
    M = inst.basis.shape[0]
    G = np.zeros((D, D), complex)
    for s in range(M):
        U = dense_rotation(inst.basis[s])
        for i in range(inst.row_ptr[s], inst.row_ptr[s + 1]):
            u = int(inst.outcome[i])
            G += c_obs[i] * np.outer(U[u].conj(), U[u]) / M
    rho = (psi.T * w) @ psi.conj()
    return rho + eta * G


def _spectral_setup(seed=3, K=4):
    inst = synth.make_instance("n4_all81", seed=seed, K=K)
    psi = inst.psi.astype(np.complex128)
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    w = inst.w.astype(np.float64)
    f = oracle.forward(inst.n, inst.basis, psi, w, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    return inst, psi, w, f["c_obs"]


@pytest.mark.parametrize("eta", [1.0, 0.25, 1e-3])
def test_krylov_ritz_spanning_the_space_gives_the_dense_eigenpairs(eta):
    """At n = 4 the block Krylov space reaches all of C^16, so its Ritz pairs are the
    eigenpairs of the dense S (Eq. ritz-pairs with zero residual)."""
    inst, psi, w, c = _spectral_setup()
    lam, Phi = oracle.krylov_ritz(inst.n, _data(inst), psi, w, c, eta)
    S = _dense_S(inst, psi, w, c, eta)
    assert lam.size == 16
    np.testing.assert_allclose(lam, np.sort(np.linalg.eigvalsh(S))[::-1], atol=1e-12)
    np.testing.assert_allclose(Phi.conj() @ Phi.T, np.eye(16), atol=1e-12)
    res = np.linalg.norm((S @ Phi.T).T - lam[:, None] * Phi, axis=1)
    assert res.max() < 1e-11


def test_krylov_ritz_partial_space_is_rayleigh_ritz():
    """With fewer Krylov vectors than D the Ritz values interlace the spectrum: the
    largest Ritz value lies below the largest eigenvalue, and every Ritz value is a
    Rayleigh quotient of its unit Ritz vector."""
    inst, psi, w, c = _spectral_setup()
    lam, Phi = oracle.krylov_ritz(inst.n, _data(inst), psi, w, c, 0.5, n_krylov=8)
    S = _dense_S(inst, psi, w, c, 0.5)
    assert lam.size == 8
    ev = np.sort(np.linalg.eigvalsh(S))[::-1]
    assert lam[0] <= ev[0] + 1e-12 and lam[-1] >= ev[-1] - 1e-12
    rq = np.real(np.einsum("id,de,ie->i", Phi.conj(), S, Phi))
    np.testing.assert_allclose(rq, lam, atol=1e-12)


def _frob2(a, b):
    return float(np.sum(np.abs(a - b) ** 2))


@pytest.mark.parametrize("eta", [1.0, 0.1])
def test_spectral_candidates_theorem_1(eta):
    """Theorem 1 with exact eigenpairs and tau = 0: (i) candidate s minimises
    ||rho_X - S||_F over feasible X of rank <= s (checked against many random
    feasible states); (ii) the selected candidate minimises Q_t over all of them;
    and the A15 score equals the dense Frobenius form up to the constant ||S||^2."""
    inst, psi, w, c = _spectral_setup()
    K, mu = psi.shape[0], 1e-3
    lam, Phi = oracle.krylov_ritz(inst.n, _data(inst), psi, w, c, eta)
    S = _dense_S(inst, psi, w, c, eta)
    s_star, cands = oracle.spectral_candidates(lam, eta, mu, 0.0, K)
    rng = np.random.default_rng(0)
    Qfull = []
    for s_, (keep, b, q) in enumerate(cands, start=1):
        rho_x = (Phi[keep].T * b) @ Phi[keep].conj()
        f2 = _frob2(rho_x, S)
        np.testing.assert_allclose(q, (f2 - _frob2(0 * S, S)) / (2 * eta) + mu * keep.size, rtol=1e-10, atol=1e-12)
        Qfull.append(f2 / (2 * eta) + mu * keep.size)
        for _ in range(200):  # random feasible states of rank <= s
            R = int(rng.integers(1, s_ + 1))
            A = rng.standard_normal((R, 16)) + 1j * rng.standard_normal((R, 16))
            A /= np.linalg.norm(A, axis=1, keepdims=True)
            a = rng.dirichlet(np.ones(R))
            rho_r = (A.T * a) @ A.conj()
            assert _frob2(rho_r, S) >= f2 - 1e-12
            assert _frob2(rho_r, S) / (2 * eta) + mu * R >= min(Qfull) - 1e-12 or s_ < s_star
    assert int(np.argmin(Qfull)) + 1 == s_star


def test_spectral_step_small_eta_reduces_to_the_refactor():
    """As eta -> 0, S_t -> rho_t and the spectral candidate with the most atoms is the
    exact eigen-refactorisation of rho_t."""
    inst, psi, w, c = _spectral_setup()
    K = psi.shape[0]
    lam, Phi = oracle.krylov_ritz(inst.n, _data(inst), psi, w, c, 1e-9)
    _, cands = oracle.spectral_candidates(lam, 1e-9, 0.0, 1e-3, K)
    keep, b, _ = cands[-1]
    phi, wk = oracle.refactor(psi, w, 1e-3)
    np.testing.assert_allclose(b, wk, atol=1e-6)
    rho_a = (Phi[keep].T * b) @ Phi[keep].conj()
    rho_b = (phi.T * wk) @ phi.conj()
    assert _frob2(rho_a, rho_b) < 1e-10


def test_oracle_spectral_slot_is_monotone_and_feasible():
    inst, psi, w, _ = _spectral_setup(seed=5)
    data = _data(inst)
    J_prev = None
    for slot in (3, 0, 1, 3):
        psi, w, J, acc, eta = oracle.step(inst.n, data, psi, w, slot, 0)
        assert np.all(w >= 0) and abs(w.sum() - 1) < 1e-12
        act = w > 0
        np.testing.assert_allclose(np.linalg.norm(psi[act], axis=1), 1.0, atol=1e-12)
        if J_prev is not None:
            assert J <= J_prev + 1e-15
        J_prev = J


# ----------------------------------------------------------------- Algorithm 1 slots against a dense route
#
# The helpers below recompute every slot of Algorithm 1 from dense matrices: rho as a
# D x D matrix, p_s from the diagonal of V_s rho V_s^* with Kronecker V_s, G as
# sum_m c_m E_m, the tangent with the explicit projector I - psi psi^*, the simplex
# projection by bisection on its threshold, and the spectral candidates from a dense
# eigh of S = rho + eta G.  None of them calls the oracle.

STEP_EPS, STEP_MU, STEP_TAU, STEP_TAU_ACC = 1e-8, 1e-3, 1e-3, 1e-10
GRID = [2.0 ** -j for j in range(11)]  # Table I step grid, largest first


def _dense_objective(inst, psi, w):
    """J = -sum pihat log(p/B + eps) + mu #{w > 0} from dense probabilities; also c."""
    from test_oracle_pins import dense_rotation
    psi = np.asarray(psi, complex)
    rho = (psi.T * np.asarray(w)) @ psi.conj()
    M = inst.basis.shape[0]
    L, c = 0.0, np.zeros(inst.outcome.shape[0])
    for s in range(M):
        U = dense_rotation(inst.basis[s])
        p = np.real(np.einsum("ud,de,ue->u", U, rho, U.conj()))
        for i in range(inst.row_ptr[s], inst.row_ptr[s + 1]):
            pihat = inst.count[i] / (M * inst.shots[s])
            pi = p[inst.outcome[i]] / M
            L -= pihat * np.log(pi + STEP_EPS)
            c[i] = pihat / (pi + STEP_EPS)
    return L + STEP_MU * int(np.count_nonzero(np.asarray(w) > 0)), c


def _dense_G(inst, c):
    from test_oracle_pins import dense_rotation
    D, M = 1 << inst.n, inst.basis.shape[0]
    G = np.zeros((D, D), complex)
    for s in range(M):
        U = dense_rotation(inst.basis[s])
        for i in range(inst.row_ptr[s], inst.row_ptr[s + 1]):
            row = U[int(inst.outcome[i])]
            G += c[i] * np.outer(row.conj(), row) / M
    return G


def _proj_bisect(v):
    """Euclidean projection onto the simplex as max(v - theta, 0) with theta found by
    bisection on sum max(v - theta, 0) = 1 (a different route from sorting)."""
    v = np.asarray(v, float)
    lo, hi = v.min() - 1.0, v.max()
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.maximum(v - mid, 0.0).sum() > 1.0:
            lo = mid
        else:
            hi = mid
    b = np.maximum(v - 0.5 * (lo + hi), 0.0)
    return b / b.sum()


def _prune_dense(beta):
    keep = [i for i in range(len(beta)) if beta[i] > STEP_TAU]
    if not keep:
        keep = [int(np.argmax(beta))]
    b = np.asarray([beta[i] for i in keep])
    return keep, b / b.sum()


def _dense_step(inst, psi, w, slot, r, rank_fix=0):
    """(psi~, w~, J, accepted, eta) of one Algorithm 1 slot, dense route (rank_fix:
    the spectral slot takes the candidate with that many eigenpairs)."""
    psi = np.array(psi, complex)
    w = np.array(w, float)
    K, D = psi.shape
    J0, c0 = _dense_objective(inst, psi, w)
    G = _dense_G(inst, c0)
    rho = (psi.T * w) @ psi.conj()
    if slot == 2:
        act = int(np.count_nonzero(w > 0))
        lam, V = np.linalg.eigh(rho)
        lam, V = lam[::-1][:act], V[:, ::-1][:, :act]
        lam = np.maximum(lam, 0.0)
        keep, b = _prune_dense(lam / lam.sum())
        pt, wt = np.zeros_like(psi), np.zeros_like(w)
        pt[:len(keep)] = V[:, keep].T
        wt[:len(keep)] = b
        Jt, _ = _dense_objective(inst, pt, wt)
        return (pt, wt, Jt, True, 0.0) if Jt <= J0 - STEP_TAU_ACC else (psi, w, J0, False, 0.0)
    for eta in GRID:
        if slot == 0:
            x = psi[r]
            P = np.eye(D) - np.outer(x, x.conj())
            d = w[r] * (P @ (G @ x))
            t = x + eta * d
            pt, wt = psi.copy(), w
            pt[r] = t / np.linalg.norm(t)
        elif slot == 1:
            h = np.real(np.einsum("kd,de,ke->k", psi.conj(), G, psi))
            act = np.nonzero(w > 0)[0]
            keep, b = _prune_dense(_proj_bisect(w[act] + eta * h[act]))
            pt, wt = psi, np.zeros_like(w)
            wt[act[keep]] = b
        else:  # slot 3: exact eigenpairs of S = rho + eta G (the Krylov space is all of C^D here)
            lam, V = np.linalg.eigh(rho + eta * G)
            lam, V = lam[::-1], V[:, ::-1]
            best = None
            L = min(K, D)
            for s_ in (range(1, L + 1) if rank_fix <= 0 else [min(rank_fix, L)]):
                keep, b = _prune_dense(_proj_bisect(lam[:s_]))
                q = (np.dot(b, b) - 2.0 * np.dot(b, lam[keep])) / (2.0 * eta) + STEP_MU * len(keep)
                if best is None or q < best[0]:
                    best = (q, keep, b)
            _, keep, b = best
            pt, wt = np.zeros_like(psi), np.zeros_like(w)
            pt[:len(keep)] = V[:, keep].T
            wt[:len(keep)] = b
        Jt, _ = _dense_objective(inst, pt, wt)
        if Jt <= J0 - STEP_TAU_ACC:
            return pt, wt, Jt, True, eta
    return psi, w, J0, False, GRID[-1]


def _rho_of(psi, w):
    return (np.asarray(psi).T * np.asarray(w)) @ np.asarray(psi).conj()


def _step_case(seed, K, shots):
    inst = synth.make_instance("n4_all81", seed=seed, K=K, shots=shots)
    psi = inst.psi.astype(np.complex128)
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    w = synth.dirichlet_weights(K, synth.rng_for(seed, 55))  # distinct, non-uniform weights
    return inst, psi, w


@pytest.mark.parametrize("seed,K,shots", [(3, 4, 1000), (8, 3, 200)])
def test_oracle_step_equals_dense_route(seed, K, shots):
    """Every slot of oracle.step against the dense route: the same accepted flag, the
    same eta from the Table I grid, the same J, and the same state (compared through
    rho, which is free of atom phases and of the basis of degenerate eigenspaces).
    The sequence must accept in the three step-grid slot kinds and at least once below
    eta = 1; the refactor (slot 2) is accepted only when it lowers the rank, which the
    second half checks on a state with a duplicated atom."""
    inst, psi, w = _step_case(seed, K, shots)
    data = _data(inst)
    accepted, etas = set(), []
    for slot, r in [(0, 0), (0, 1), (1, 0), (3, 0), (0, 2), (1, 0), (2, 0), (0, 0), (3, 0), (1, 0)]:
        if slot == 0 and r >= K:
            continue
        po, wo, Jo, acc_o, eta_o = oracle.step(4, data, psi, w, slot, r)
        pd, wd, Jd, acc_d, eta_d = _dense_step(inst, psi, w, slot, r)
        assert acc_o == acc_d and eta_o == eta_d, (slot, r, acc_o, acc_d, eta_o, eta_d)
        assert abs(Jo - Jd) <= 1e-10 * max(1.0, abs(Jd)), (slot, Jo, Jd)
        np.testing.assert_allclose(_rho_of(po, wo), _rho_of(pd, wd), atol=1e-10)
        if acc_o:
            accepted.add(slot)
            etas.append(eta_o)
        psi, w = po, wo
    assert {0, 1, 3} <= accepted, accepted
    assert any(0.0 < e < 1.0 for e in etas), etas
    # a duplicated atom: the refactor merges the two copies (rank K - 1), so mu R drops
    psi[1] = psi[0]
    w = np.full(K, 1.0 / K)
    po, wo, Jo, acc_o, _ = oracle.step(4, data, psi, w, 2, 0)
    pd, wd, Jd, acc_d, _ = _dense_step(inst, psi, w, 2, 0)
    assert acc_o and acc_d and np.count_nonzero(wo > 0) == K - 1
    assert abs(Jo - Jd) <= 1e-10 * max(1.0, abs(Jd))
    np.testing.assert_allclose(_rho_of(po, wo), _rho_of(pd, wd), atol=1e-10)


@pytest.mark.parametrize("n,K,seed", [(3, 3, 4), (4, 4, 6)])
def test_oracle_tangent_against_dense_projector_and_fd(n, K, seed):
    """oracle.tangent = w_k (I - psi_k psi_k^*) G psi_k with the projector as a dense
    matrix and distinct, non-unit weights; along the normalised trial
    (psi_k + t d_k)/||psi_k + t d_k|| the objective changes at rate -2 ||d_k||^2
    (central differences of the dense objective), which fixes the w_k factor."""
    inst = synth.random_instance(n, 3 ** n if n <= 3 else 40, K, shots=400, seed=seed)
    psi = inst.psi.astype(np.complex128)
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    w = np.array([0.55, 0.3, 0.1, 0.05][:K])
    w = w / w.sum()
    J0, c = _dense_objective(inst, psi, w)
    G = _dense_G(inst, c)
    Gpsi = (G @ psi.T).T
    d = oracle.tangent(psi, w, Gpsi)
    D = 1 << n
    for k in range(K):
        P = np.eye(D) - np.outer(psi[k], psi[k].conj())
        np.testing.assert_allclose(d[k], w[k] * (P @ Gpsi[k]), atol=1e-14)
        t = 1e-5
        vals = []
        for sgn in (1, -1):
            x = psi[k] + sgn * t * d[k]
            pt = psi.copy()
            pt[k] = x / np.linalg.norm(x)
            vals.append(_dense_objective(inst, pt, w)[0])
        fd = (vals[0] - vals[1]) / (2 * t)
        want = -2.0 * np.sum(np.abs(d[k]) ** 2)
        assert abs(fd - want) <= 1e-6 * abs(want) + 1e-12, (k, fd, want)


@pytest.mark.parametrize("rank_fix", [1, 2, 3])
def test_oracle_spectral_slot_with_a_fixed_rank_equals_dense_route(rank_fix):
    """The known-rank variant of the spectral slot (Sec. IV ablation: the candidate with
    R Ritz pairs) against the dense route: same acceptance, step, J and rho."""
    inst, psi, w = _step_case(3, 4, 1000)
    po, wo, Jo, acc_o, eta_o = oracle.step(4, _data(inst), psi, w, 3, 0, rank_fix=rank_fix)
    pd, wd, Jd, acc_d, eta_d = _dense_step(inst, psi, w, 3, 0, rank_fix=rank_fix)
    assert acc_o == acc_d and eta_o == eta_d
    assert abs(Jo - Jd) <= 1e-10 * max(1.0, abs(Jd))
    np.testing.assert_allclose(_rho_of(po, wo), _rho_of(pd, wd), atol=1e-10)
    if acc_o:
        assert np.count_nonzero(wo > 0) <= rank_fix
