"""Algorithmic ablation of Algorithm 1 (Sec. IV, the variants v_atom, v_coeff,
v_kr, v_full): the same data, stabilised likelihood, initialisation, step grid
and acceptance rule, with different candidate moves enabled:

  v_atom   atom trials only (weights and support fixed);
  v_coeff  atom trials and the simplex coefficient update (T_alpha schedule);
  v_kr     as v_coeff, plus the spectral refactorisation step of Sec. III-C every
           T_ref iterations, restricted to the true rank R* (qst_step_params.rank_fix);
  v_full   as v_kr with the candidate chosen by the rank-penalised score Q_t.

Every move runs on the GPU through qst_step (one slot per call).  After each
accepted update the driver records the serial-equivalent oracle calls (one
primitive of Sec. III-B over all outcomes for one atom, or one loss or A^T c
evaluation, as Algorithm 1 issues them), J, the active rank R_t and the recovery
error e_rho = ||rho - rho*||_F / ||rho*||_F (from atom inner products; rho is
never formed).  A run stops at Table I's rules (relative decrease of J over the
last 20 accepted updates below 1e-4, or 1e5 oracle calls) or after max_iter
iterations.

Data: n qubits, M random Pauli strings, `shots` multinomial draws per setting
from the truth's Born probabilities (computed by qst_forward on the truth's
atoms and weights), a rank-R* truth with complex-Gaussian atoms and Dirichlet
weights; initial state R_max random atoms with weights 1/R_max (Table I).

    python -m paper_2607_19577_b300.ablation [--n 12 --M 2000 --shots 1000 --rank 4 --K 8]
prints one JSON object (the four curves and a summary)."""
from __future__ import annotations

import argparse
import json
import math

import numpy as np
import torch

from . import qst, synth

VARIANTS = ("v_atom", "v_coeff", "v_kr", "v_full")


def schedule(variant: str, t: int, T_alpha: int, T_ref: int) -> int:
    """Slot of iteration t: 0 atom, 1 coefficients, 3 spectral step."""
    if variant in ("v_kr", "v_full") and T_ref > 0 and (t + 1) % T_ref == 0:
        return 3
    if variant != "v_atom" and T_alpha > 0 and (t + 1) % T_alpha == 0:
        return 1
    return 0


def oracle_calls(slot: int, accepted: bool, eta: float, R_new: int, K: int, n_krylov: int, n_eta: int = 11,
                 eta0: float = 1.0, ratio: float = 0.5) -> int:
    """Serial-equivalent oracle calls of one slot.  Trials = accepted index + 1, or
    the whole grid.  Atom slot: G psi_r, then per trial the trial atom's response
    and the loss.  Coefficient slot: A^T c, then per trial the loss.  Spectral slot:
    per trial, G applied to every vector of the block Krylov basis (K per block,
    floor(n_krylov / K) blocks at most) plus the new atoms' responses and the loss."""
    trials = int(round(math.log(eta / eta0) / math.log(ratio))) + 1 if accepted else n_eta
    if slot == 0:
        return 1 + 2 * trials
    if slot == 1:
        return 1 + trials
    blocks = max(1, n_krylov // K)
    return trials * (blocks * K + R_new + 1)


def recovery_error(psi: torch.Tensor, w: torch.Tensor, phi: torch.Tensor, lam: torch.Tensor) -> float:
    """||Psi diag(w) Psi^* - Phi diag(lam) Phi^*||_F / ||Phi diag(lam) Phi^*||_F from
    the inner products of the rows (atoms) of psi and phi, in float64."""
    a, b = psi.to(torch.complex128), phi.to(torch.complex128)
    wa, wb = w.to(torch.float64), lam.to(torch.float64)

    def tr(x, wx, y, wy):  # tr(rho_x rho_y) = sum_ij wx_i wy_j |<x_i, y_j>|^2
        g = x.conj() @ y.T
        return float((wx[:, None] * wy[None, :] * (g.abs() ** 2)).sum())
    saa, sbb, sab = tr(a, wa, a, wa), tr(b, wb, b, wb), tr(a, wa, b, wb)
    return math.sqrt(max(saa + sbb - 2 * sab, 0.0) / sbb)


def make_data(n, M, shots, rank, seed):
    """Pauli strings, a rank-R* truth and multinomial counts from its Born probabilities."""
    rng = synth.rng_for(seed, 0)
    basis = synth.pauli_settings(n, M, rng)
    tw = synth.dirichlet_weights(rank, synth.rng_for(seed, 1))
    ta = synth.random_atoms(n, rank, synth.rng_for(seed, 2))
    D = 1 << n
    # Born probabilities of the truth for every outcome (qst_forward's dense output)
    row_ptr = np.zeros(M + 1, np.int64)
    plan = qst.Plan(n, M, rank, 0)
    d0 = qst.Data.from_numpy(n, basis, row_ptr, np.zeros(0, np.uint32), np.zeros(0, np.uint32),
                             np.ones(M, np.uint32))
    p_dense = torch.zeros(M, D, dtype=torch.float32, device="cuda")
    plan.forward(torch.from_numpy(ta.astype(np.complex64)).cuda(), torch.from_numpy(tw.astype(np.float32)).cuda(),
                 d0, p_dense=p_dense)
    probs = p_dense.double().cpu().numpy()
    plan.close()
    rp, out, cnt = synth.counts_from_probs(probs, np.full(M, shots, np.uint32), synth.rng_for(seed, 3))
    return basis, rp, out, cnt, np.full(M, shots, np.uint32), tw, ta


def run_variant(variant, n, data, truth, K, R_star, T_alpha=5, T_ref=50, max_iter=400, seed=0, n_krylov=30,
                delta_window=20, delta_tol=1e-4, max_calls=100000):
    basis, rp, out, cnt, shots = data
    tw, ta = truth
    M = basis.shape[0]
    plan = qst.Plan(n, M, K, out.shape[0])
    d = qst.Data.from_numpy(n, basis, rp, out, cnt, shots)
    psi = torch.from_numpy(synth.random_atoms(n, K, synth.rng_for(seed, 1000)).astype(np.complex64)).cuda()
    w = torch.full((K,), 1.0 / K, dtype=torch.float32, device="cuda")
    phi = torch.from_numpy(ta.astype(np.complex64)).cuda()
    lam = torch.from_numpy(tw.astype(np.float64)).cuda()
    _, _, loss = plan.forward(psi, w, d)
    J = loss.item() + 1e-3 * K
    calls = K + 1
    rec = [{"i": 0, "t": -1, "calls": calls, "J": J, "e_rho": recovery_error(psi, w, phi, lam), "R": K, "slot": None}]
    cycle = 0
    stop = "max_iter"
    for t in range(max_iter):
        slot = schedule(variant, t, T_alpha, T_ref)
        r = 0
        if slot == 0:
            act = torch.nonzero(w > 0).flatten().tolist()
            r = act[cycle % len(act)]
            cycle += 1
        kw = {"rank_fix": R_star} if (slot == 3 and variant == "v_kr") else {}
        J, acc, eta = plan.step(slot, r, psi, w, d, n_krylov=n_krylov, **kw)
        R = int((w > 0).sum().item())
        calls += oracle_calls(slot, acc, eta, R, K, n_krylov)
        if acc:
            rec.append({"i": len(rec), "t": t, "calls": calls, "J": J, "e_rho": recovery_error(psi, w, phi, lam),
                        "R": R, "slot": slot})
            if delta_window and len(rec) > delta_window:
                J0 = rec[-1 - delta_window]["J"]
                if (J0 - J) / abs(J0) < delta_tol:
                    stop = "delta"
                    break
        if max_calls and calls >= max_calls:
            stop = "oracle_calls"
            break
    plan.close()
    return {"records": rec, "stop": stop, "iterations": t + 1}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=12)
    ap.add_argument("--M", type=int, default=2000)
    ap.add_argument("--shots", type=int, default=1000)
    ap.add_argument("--rank", type=int, default=4, help="R*, the truth's rank")
    ap.add_argument("--K", type=int, default=8, help="R_max, the initial number of atoms")
    ap.add_argument("--max-iter", type=int, default=400)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)
    torch.cuda.set_device(0)
    *data, tw, ta = make_data(args.n, args.M, args.shots, args.rank, args.seed)
    runs = {v: run_variant(v, args.n, tuple(data), (tw, ta), args.K, args.rank, max_iter=args.max_iter,
                           seed=args.seed) for v in VARIANTS}
    J_best = min(r["J"] for run in runs.values() for r in run["records"])
    summary = {}
    for v, run in runs.items():
        last = run["records"][-1]
        summary[v] = {"accepted_updates": len(run["records"]) - 1, "iterations": run["iterations"],
                      "stop": run["stop"], "oracle_calls": last["calls"], "delta_J": last["J"] - J_best,
                      "e_rho": last["e_rho"], "R": last["R"]}
    print(json.dumps({"workload": vars(args), "J_best": J_best, "summary": summary,
                      "curves": {v: run["records"] for v, run in runs.items()}}))


if __name__ == "__main__":
    main()
