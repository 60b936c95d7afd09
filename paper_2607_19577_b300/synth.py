"""Seeded synthetic inputs shaped like the paper's workloads (Sec. IV).

This module draws random numbers and lays them out; it holds none of the
method's arithmetic (no rotation, no Born rule, no loss).  Where counts must
follow a state's Born distribution, the caller passes the per-setting
probabilities in (``counts_from_probs``); otherwise counts come from a
Porter-Thomas surrogate (``surrogate_counts``), which reproduces the sparsity
structure of measurements on Haar-like states: per setting, N_s shots spread
over 2^n outcomes with exponentially distributed outcome weights.

Recipes (Sec. IV "Numerical tests", Table I):
  * Pauli strings: each qubit's basis uniform in {Z, X, Y} (codes 0, 1, 2),
    qubit 1 first (most significant outcome bit); n=4 uses all 3^4 strings in
    lexicographic order.
  * Truth weights: Dirichlet(1), sorted non-increasing.
  * Truth atoms: xi / ||xi||, xi ~ CN(0, I_D); optionally orthonormalised (QR).
  * Counts: Multinomial(N_s, P(.|s)) per setting, stored as CSR with outcomes
    ascending inside each row.
  * Evaluation point: atoms = truth atoms + 0.1 CN noise, renormalised, padded
    with fresh random atoms up to K; weights 1/K.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rng_for(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([seed, stream]))


def pauli_settings(n: int, M: int, rng: np.random.Generator, all_strings: bool = False) -> np.ndarray:
    """uint8 [M][n] basis codes (0=Z, 1=X, 2=Y)."""
    if all_strings:
        M = 3 ** n
        idx = np.arange(M)
        out = np.zeros((M, n), dtype=np.uint8)
        for q in range(n):  # qubit 1 varies slowest
            out[:, q] = (idx // 3 ** (n - 1 - q)) % 3
        return out
    return rng.integers(0, 3, size=(M, n), dtype=np.uint8)


def random_atoms(n: int, R: int, rng: np.random.Generator, orthonormal: bool = False) -> np.ndarray:
    """complex128 [R][2^n] unit vectors, xi / ||xi|| with xi ~ CN(0, I)."""
    D = 1 << n
    xi = (rng.standard_normal((R, D)) + 1j * rng.standard_normal((R, D))) / np.sqrt(2.0)
    if orthonormal:
        q, _ = np.linalg.qr(xi.T)
        return np.ascontiguousarray(q.T[:R])
    return xi / np.linalg.norm(xi, axis=1, keepdims=True)


def dirichlet_weights(R: int, rng: np.random.Generator) -> np.ndarray:
    return np.sort(rng.dirichlet(np.ones(R)))[::-1].copy()


def counts_from_probs(probs: np.ndarray, shots: np.ndarray, rng: np.random.Generator):
    """Multinomial counts per setting from given probabilities [M][D].

    Returns CSR (row_ptr int64 [M+1], outcome uint32 [nnz], count uint32 [nnz])."""
    M = probs.shape[0]
    rows, outs, cnts = [0], [], []
    for s in range(M):
        p = np.clip(np.asarray(probs[s], dtype=np.float64), 0.0, None)
        p = p / p.sum()
        c = rng.multinomial(int(shots[s]), p)
        nz = np.nonzero(c)[0]
        outs.append(nz.astype(np.uint32))
        cnts.append(c[nz].astype(np.uint32))
        rows.append(rows[-1] + nz.size)
    return (np.asarray(rows, dtype=np.int64),
            np.concatenate(outs) if outs else np.zeros(0, np.uint32),
            np.concatenate(cnts) if cnts else np.zeros(0, np.uint32))


def surrogate_counts(n: int, shots: np.ndarray, weights: np.ndarray, rng: np.random.Generator):
    """Counts with the statistics of Haar-like states, drawn without the Born rule.

    For D <= 2^16 each setting gets Porter-Thomas outcome weights (a rank-R
    mixture sum_r weights_r e_{r,u}, e ~ Exp(1), when R*D <= 2^18, else a single
    exponential per outcome) and N_s categorical draws by inverse CDF.  For
    larger D the N_s shots land uniformly (collisions are rare there, so the
    sparsity pattern is the same).  Returns CSR like ``counts_from_probs``."""
    D = 1 << n
    M = shots.shape[0]
    R = weights.shape[0]
    rows, outs, cnts = [0], [], []
    for s in range(M):
        ns = int(shots[s])
        if D <= (1 << 16):
            if R * D <= (1 << 18):
                p = weights @ rng.exponential(1.0, size=(R, D))
            else:
                p = rng.exponential(1.0, size=D)
            cdf = np.cumsum(p)
            draws = np.searchsorted(cdf, rng.random(ns) * cdf[-1], side="right")
            o, k = np.unique(np.minimum(draws, D - 1), return_counts=True)
        else:
            o, k = np.unique(rng.integers(0, D, size=ns), return_counts=True)
        outs.append(o.astype(np.uint32))
        cnts.append(k.astype(np.uint32))
        rows.append(rows[-1] + o.size)
    return (np.asarray(rows, dtype=np.int64), np.concatenate(outs), np.concatenate(cnts))


def eval_point(truth_atoms: np.ndarray, K: int, rng: np.random.Generator, noise: float = 0.1):
    """Atoms near the truth (perturbed, renormalised), padded with random atoms to K."""
    R, D = truth_atoms.shape
    n = D.bit_length() - 1
    take = min(R, K)
    pert = truth_atoms[:take] + noise * random_atoms(n, take, rng)
    pert /= np.linalg.norm(pert, axis=1, keepdims=True)
    if K > take:
        pert = np.concatenate([pert, random_atoms(n, K - take, rng)], axis=0)
    return np.ascontiguousarray(pert), np.full(K, 1.0 / K)


@dataclass
class Instance:
    """One tomography instance: measurement data and an evaluation point."""
    name: str
    n: int
    basis: np.ndarray          # uint8 [M][n]
    shots: np.ndarray          # uint32 [M]
    row_ptr: np.ndarray        # int64 [M+1]
    outcome: np.ndarray        # uint32 [nnz]
    count: np.ndarray          # uint32 [nnz]
    psi: np.ndarray            # complex64 [K][D] evaluation atoms
    w: np.ndarray              # float32 [K] evaluation weights
    eps: float = 1e-8
    truth_w: np.ndarray = field(default=None)
    truth_atoms: np.ndarray = field(default=None)

    @property
    def M(self):
        return self.basis.shape[0]

    @property
    def K(self):
        return self.psi.shape[0]

    @property
    def D(self):
        return 1 << self.n

    @property
    def nnz(self):
        return self.outcome.shape[0]


def truth_for(name: str, n: int, rng: np.random.Generator):
    """Truth (weights, atoms) for the named workload."""
    if name == "n4_all81":
        return dirichlet_weights(2, rng), random_atoms(n, 2, rng, orthonormal=True)
    if name == "n16_m4096_k16":
        # rank-8 truth mixed 95/5 with an independent rank-8 perturbation
        wa, aa = dirichlet_weights(8, rng), random_atoms(n, 8, rng)
        wb, ab = dirichlet_weights(8, rng), random_atoms(n, 8, rng)
        return np.concatenate([0.95 * wa, 0.05 * wb]), np.concatenate([aa, ab])
    rank = {"n12_m2000_k8": 4, "n20_m1024_k8": 4, "n20_m64_k8": 4}.get(name, 4)
    return dirichlet_weights(rank, rng), random_atoms(n, rank, rng)


WORKLOADS = {
    # name: (n, M, shots, K)
    "n4_all81": (4, 81, 1000, 4),
    "n12_m2000_k8": (12, 2000, 1000, 8),
    "n16_m4096_k16": (16, 4096, 2000, 16),
    "n20_m1024_k8": (20, 1024, 10000, 8),
    # per-launch shape of the n = 20 workload with 1/16 of its settings (profiling)
    "n20_m64_k8": (20, 64, 10000, 8),
}


def make_instance(name: str, seed: int = 0, probs_fn=None, n=None, M=None, shots=None, K=None) -> Instance:
    """Build a named workload (or a custom one with the same recipe).

    ``probs_fn(basis, truth_w, truth_atoms) -> [M][D]`` supplies Born
    probabilities of the truth for the counts; without it the Porter-Thomas
    surrogate is used."""
    if name not in WORKLOADS and n is None:
        import re
        mt = re.fullmatch(r"n(\d+)_m(\d+)_k(\d+)(?:_s(\d+))?", name)
        if not mt:
            raise ValueError(f"unknown workload {name!r}")
        n, M, K = int(mt.group(1)), int(mt.group(2)), int(mt.group(3))
        shots = int(mt.group(4) or 2000)
    dn, dM, dshots, dK = WORKLOADS.get(name, (n, M, shots, K))
    n, M, shots, K = n or dn, M or dM, shots or dshots, K or dK
    rng = rng_for(seed, 0)
    basis = pauli_settings(n, M, rng, all_strings=(name == "n4_all81"))
    M = basis.shape[0]
    tw, ta = truth_for(name, n, rng_for(seed, 1))
    shots_arr = np.full(M, shots, dtype=np.uint32)
    if probs_fn is not None:
        row_ptr, outcome, count = counts_from_probs(probs_fn(basis, tw, ta), shots_arr, rng_for(seed, 2))
    else:
        row_ptr, outcome, count = surrogate_counts(n, shots_arr, tw, rng_for(seed, 2))
    psi, w = eval_point(ta, K, rng_for(seed, 1000))
    return Instance(name=name, n=n, basis=basis, shots=shots_arr, row_ptr=row_ptr,
                    outcome=outcome, count=count, psi=psi.astype(np.complex64),
                    w=w.astype(np.float32), truth_w=tw, truth_atoms=ta)


def random_instance(n: int, M: int, K: int, shots: int, seed: int, dense_frac: float = None,
                    basis: np.ndarray = None) -> Instance:
    """A small instance with surrogate counts, random atoms and Dirichlet weights
    (used for parity sweeps over shapes).  `basis` ([M][n] codes) replaces the
    random Pauli strings when given."""
    rng = rng_for(seed, 7)
    if basis is None:
        basis = pauli_settings(n, M, rng)
    else:
        basis = np.ascontiguousarray(basis, dtype=np.uint8)
        M = basis.shape[0]
    tw = dirichlet_weights(max(1, min(K, 4)), rng)
    shots_arr = np.full(M, shots, dtype=np.uint32)
    row_ptr, outcome, count = surrogate_counts(n, shots_arr, tw, rng_for(seed, 8))
    psi = random_atoms(n, K, rng_for(seed, 9)).astype(np.complex64)
    w = dirichlet_weights(K, rng_for(seed, 10)).astype(np.float32) if K > 0 else np.zeros(0, np.float32)
    return Instance(name="random", n=n, basis=basis, shots=shots_arr, row_ptr=row_ptr,
                    outcome=outcome, count=count, psi=psi, w=w)


def make_batch(seed: int = 0, count: int = 64, n_range=(6, 14), M_range=(200, 3000), shots_range=(500, 5000),
               rank_range=(1, 8), probs_fn=None):
    """The batched workload: `count` independent instances with n uniform in n_range,
    truth rank uniform in rank_range, M uniform in M_range random Pauli strings,
    shots uniform in shots_range, K = 2 x rank atoms; instance i draws from stream i
    of the seed."""
    out = []
    for i in range(count):
        rng = rng_for(seed, 10_000 + i)
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        rank = int(rng.integers(rank_range[0], rank_range[1] + 1))
        M = int(rng.integers(M_range[0], M_range[1] + 1))
        shots = int(rng.integers(shots_range[0], shots_range[1] + 1))
        basis = pauli_settings(n, M, rng)
        tw, ta = dirichlet_weights(rank, rng), random_atoms(n, rank, rng)
        shots_arr = np.full(M, shots, dtype=np.uint32)
        if probs_fn is not None:
            row_ptr, outcome, count_ = counts_from_probs(probs_fn(basis, tw, ta), shots_arr, rng_for(seed, 20_000 + i))
        else:
            row_ptr, outcome, count_ = surrogate_counts(n, shots_arr, tw, rng_for(seed, 20_000 + i))
        psi, w = eval_point(ta, 2 * rank, rng_for(seed, 30_000 + i))
        out.append(Instance(name=f"batch{i}", n=n, basis=basis, shots=shots_arr, row_ptr=row_ptr, outcome=outcome,
                            count=count_, psi=psi.astype(np.complex64), w=w.astype(np.float32),
                            truth_w=tw, truth_atoms=ta))
    return out
