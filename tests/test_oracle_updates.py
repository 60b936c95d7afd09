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
