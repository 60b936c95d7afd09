"""The ablation driver of Algorithm 1 (Sec. IV: v_atom, v_coeff, v_kr, v_full) on a
small instance: every variant's recorded J decreases with every accepted update,
the oracle-call count grows, the atom-only variant keeps its support, the
known-rank variant never keeps more than R* atoms after a spectral step, and the
full variant reaches an objective no worse than the atom-only one."""
import numpy as np
import pytest
import torch

from paper_2607_19577_b300 import ablation

pytestmark = pytest.mark.gpu


def test_ablation_variants_on_a_small_instance():
    n, M, shots, R_star, K = 6, 80, 800, 2, 4
    *data, tw, ta = ablation.make_data(n, M, shots, R_star, seed=5)
    runs = {v: ablation.run_variant(v, n, tuple(data), (tw, ta), K, R_star, T_ref=10, max_iter=60, seed=5)
            for v in ablation.VARIANTS}
    for v, run in runs.items():
        rec = run["records"]
        J = [r["J"] for r in rec]
        calls = [r["calls"] for r in rec]
        assert len(rec) > 1, v
        assert all(b <= a for a, b in zip(J, J[1:])), v
        assert all(b > a for a, b in zip(calls, calls[1:])), v
        assert all(0.0 <= r["e_rho"] <= 2.0 for r in rec), v
    assert all(r["R"] == K for r in runs["v_atom"]["records"])
    assert all(r["R"] <= R_star for r in runs["v_kr"]["records"] if r["slot"] == 3)
    assert runs["v_full"]["records"][-1]["J"] <= runs["v_atom"]["records"][-1]["J"] + 1e-9


def test_recovery_error_from_inner_products():
    """e_rho from atom inner products equals the dense Frobenius norm."""
    rng = np.random.default_rng(0)
    a = rng.standard_normal((3, 16)) + 1j * rng.standard_normal((3, 16))
    b = rng.standard_normal((2, 16)) + 1j * rng.standard_normal((2, 16))
    wa, wb = np.array([0.5, 0.3, 0.2]), np.array([0.7, 0.3])
    rho_a = (a.T * wa) @ a.conj()
    rho_b = (b.T * wb) @ b.conj()
    want = np.linalg.norm(rho_a - rho_b) / np.linalg.norm(rho_b)
    got = ablation.recovery_error(torch.from_numpy(a), torch.from_numpy(wa), torch.from_numpy(b),
                                  torch.from_numpy(wb))
    assert abs(got - want) <= 1e-12
