"""FP64 CPU oracle for the forward and adjoint of matrix-free atomic QST.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its binding) never imports this package, and this package
imports nothing from the product.

The arithmetic lives in ``qst_oracle.c`` (plain C, FP64, one qubit and one
outcome at a time); this module only compiles it with gcc, loads it with
ctypes and marshals numpy arrays.  The definitions it follows are listed in the
header of ``qst_oracle.c`` (Sec. II Eqs. atomic-density, born-map, qst-loss,
atom-response, atomic-born-map; Sec. III Eqs. likelihood-ratio-vector,
weight-gradient, atom-wirtinger-gradient, atom-projected-descent-direction,
negative-gradient-product; Sec. IV Pauli POVM).

Parity pins (tests/test_oracle_*.py): dense brute force with explicit Kronecker
matrices, closed forms (|0...0>, GHZ, product states), linear inversion on the
full n=4 Pauli set, POVM completeness (c == 1 gives G v = v), the identities
<psi_k|G psi_k> = h_k and sum_k w_k h_k = sum pihat*pi/(pi+eps), and central
finite differences of the loss.  The update-rule helpers are pinned too:
simplex projection by its KKT conditions, refactor by dense eigh of rho, the
Krylov Ritz pairs by dense eigenpairs of S, and every slot of ``step`` (accepted
flag, step size, J and state) plus ``tangent`` (dense projector, and the rate
-2||d||^2 of the objective along the normalised trial) against a route built
from dense D x D matrices.  No function here is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "qst_oracle.c"
_LIB = _HERE / "liboracle.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile qst_oracle.c into liboracle.so with gcc (plain -O2, FP64, no fast-math)."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(".so.tmp%d" % os.getpid())
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(tmp), str(_SRC), "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(str(build()))
        P = ctypes.c_void_p
        i32, f64 = ctypes.c_int, ctypes.c_double
        lib.qst_oracle_forward.argtypes = [i32, i32, i32, i32, P, P, P, P, P, P, P, f64, P, P, P, P]
        lib.qst_oracle_forward.restype = i32
        lib.qst_oracle_adjoint.argtypes = [i32, i32, i32, i32, P, P, P, P, P, P, P, P, P]
        lib.qst_oracle_adjoint.restype = i32
        lib.qst_oracle_apply_G.argtypes = [i32, i32, i32, P, P, P, P, i32, P, P]
        lib.qst_oracle_apply_G.restype = i32
        lib.qst_oracle_amplitude.argtypes = [i32, P, P, ctypes.c_uint32, P]
        lib.qst_oracle_amplitude.restype = None
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _cplx(psi):
    """complex array [..., D] -> contiguous interleaved float64 view source."""
    return np.ascontiguousarray(np.asarray(psi, dtype=np.complex128))


def forward(n, basis, psi, w, row_ptr, outcome, count, shots, eps=1e-8, B=None,
            dense=False):
    """Born probabilities, loss and likelihood ratio (FP64).

    Returns dict(p_obs, c_obs, loss[, p_dense]).  ``B`` is the normalising number
    of settings (defaults to the number passed in)."""
    lib = _load()
    basis = _c(basis, np.uint8)
    M = basis.shape[0]
    psi = _cplx(psi).reshape(-1, 1 << n)
    K = psi.shape[0]
    w = _c(w, np.float64)
    row_ptr, outcome = _c(row_ptr, np.int64), _c(outcome, np.uint32)
    count, shots = _c(count, np.uint32), _c(shots, np.uint32)
    nnz = outcome.shape[0]
    p_obs = np.zeros(nnz)
    c_obs = np.zeros(nnz)
    loss = np.zeros(1)
    p_dense = np.zeros((M, 1 << n)) if dense else None
    rc = lib.qst_oracle_forward(n, M, int(B or M), K, _ptr(basis), _ptr(psi), _ptr(w),
                                _ptr(row_ptr), _ptr(outcome), _ptr(count), _ptr(shots),
                                float(eps), _ptr(p_dense), _ptr(p_obs), _ptr(c_obs), _ptr(loss))
    if rc != 0:
        raise ValueError("oracle forward rejected its input")
    out = dict(p_obs=p_obs, c_obs=c_obs, loss=float(loss[0]))
    if dense:
        out["p_dense"] = p_dense
    return out


def adjoint(n, basis, psi, w, row_ptr, outcome, c_obs, B=None):
    """Atom gradients and coefficient gradient (FP64).

    Returns dict(G_psi [K][D] complex, grad_psi = -w_k G psi_k, h [K],
    grad_w = -h)."""
    lib = _load()
    basis = _c(basis, np.uint8)
    M = basis.shape[0]
    D = 1 << n
    psi = _cplx(psi).reshape(-1, D)
    K = psi.shape[0]
    w = _c(w, np.float64)
    row_ptr, outcome = _c(row_ptr, np.int64), _c(outcome, np.uint32)
    c_obs = _c(c_obs, np.float64)
    G = np.zeros((K, D), dtype=np.complex128)
    g = np.zeros((K, D), dtype=np.complex128)
    h = np.zeros(K)
    rc = lib.qst_oracle_adjoint(n, M, int(B or M), K, _ptr(basis), _ptr(psi), _ptr(w),
                                _ptr(row_ptr), _ptr(outcome), _ptr(c_obs), _ptr(G), _ptr(g), _ptr(h))
    if rc != 0:
        raise ValueError("oracle adjoint rejected its input")
    return dict(G_psi=G, grad_psi=g, h=h, grad_w=-h)


def apply_G(n, basis, row_ptr, outcome, c_obs, v, B=None):
    """G v = (1/B) sum_s V_s^*(c_s .* V_s v) for each row of v (FP64)."""
    lib = _load()
    basis = _c(basis, np.uint8)
    M = basis.shape[0]
    D = 1 << n
    v = _cplx(v).reshape(-1, D)
    out = np.zeros_like(v)
    rc = lib.qst_oracle_apply_G(n, M, int(B or M), _ptr(basis), _ptr(_c(row_ptr, np.int64)),
                                _ptr(_c(outcome, np.uint32)), _ptr(_c(c_obs, np.float64)),
                                v.shape[0], _ptr(v), _ptr(out))
    if rc != 0:
        raise ValueError("oracle apply_G rejected its input")
    return out


def _shards(M, parts):
    """Contiguous setting ranges [lo, hi) covering 0..M-1, at most `parts` of them."""
    parts = max(1, min(int(parts), M)) if M else 1
    edges = [round(M * j / parts) for j in range(parts + 1)]
    return [(edges[j], edges[j + 1]) for j in range(parts) if edges[j + 1] > edges[j]] or [(0, 0)]


def _threads(threads):
    if threads:
        return int(threads)
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def forward_sharded(n, basis, psi, w, row_ptr, outcome, count, shots, eps=1e-8, B=None, threads=None):
    """forward() over contiguous setting shards on a thread pool (the measurement
    partition of Sec. III-B: every shard uses the global B, so the per-entry
    outputs are those of forward() and the loss is the sum of the shard losses,
    added in shard order).  The C routine releases the GIL, so the shards run on
    separate host cores.  The arithmetic per setting is forward()'s."""
    from concurrent.futures import ThreadPoolExecutor
    basis = _c(basis, np.uint8)
    M = basis.shape[0]
    row_ptr = _c(row_ptr, np.int64)
    B = int(B or M)
    parts = _shards(M, _threads(threads))

    def run(r):
        lo, hi = r
        a, b = int(row_ptr[lo]), int(row_ptr[hi])
        return forward(n, basis[lo:hi], psi, w, row_ptr[lo:hi + 1] - a, outcome[a:b], count[a:b], shots[lo:hi],
                       eps=eps, B=B)
    with ThreadPoolExecutor(len(parts)) as ex:
        res = list(ex.map(run, parts))
    loss = 0.0
    for r in res:
        loss += r["loss"]
    return dict(p_obs=np.concatenate([r["p_obs"] for r in res]), c_obs=np.concatenate([r["c_obs"] for r in res]),
                loss=loss)


def adjoint_sharded(n, basis, psi, w, row_ptr, outcome, c_obs, B=None, threads=None):
    """adjoint() over contiguous setting shards on a thread pool, summed in shard
    order (G psi, h and the gradients are sums over settings, Eqs.
    negative-gradient-product and weight-gradient; each shard uses the global B).
    The arithmetic per setting is adjoint()'s."""
    from concurrent.futures import ThreadPoolExecutor
    basis = _c(basis, np.uint8)
    M = basis.shape[0]
    row_ptr = _c(row_ptr, np.int64)
    c_obs = _c(c_obs, np.float64)
    B = int(B or M)
    parts = _shards(M, _threads(threads))

    def run(r):
        lo, hi = r
        a, b = int(row_ptr[lo]), int(row_ptr[hi])
        return adjoint(n, basis[lo:hi], psi, w, row_ptr[lo:hi + 1] - a, outcome[a:b], c_obs[a:b], B=B)
    with ThreadPoolExecutor(len(parts)) as ex:
        res = list(ex.map(run, parts))
    out = {key: res[0][key].copy() for key in ("G_psi", "grad_psi", "h")}
    for r in res[1:]:
        for key in out:
            out[key] += r[key]
    out["grad_w"] = -out["h"]
    return out


def amplitude(n, b, psi, u):
    """(V_s psi)_u by direct summation over all basis states (independent of the
    axis-by-axis transform)."""
    lib = _load()
    b = _c(b, np.uint8)
    psi = _cplx(psi).reshape(-1)
    out = np.zeros(2)
    lib.qst_oracle_amplitude(n, _ptr(b), _ptr(psi), int(u), _ptr(out))
    return complex(out[0], out[1])


def tangent(psi, w, G_psi):
    """Projected descent direction d_k = w_k (I - psi_k psi_k^*) G psi_k
    (Eq. atom-projected-descent-direction), row by row, FP64."""
    psi = np.asarray(psi, dtype=np.complex128)
    G_psi = np.asarray(G_psi, dtype=np.complex128)
    inner = np.sum(np.conj(psi) * G_psi, axis=1)  # <psi_k | G psi_k>
    return np.asarray(w, dtype=np.float64)[:, None] * (G_psi - psi * inner[:, None])


# ----------------------------------------------------------------- update-rule helpers (FP64 numpy)

def simplex_project(v):
    """Euclidean projection of v onto the probability simplex (Eq. coefficient-update's
    proj_Delta): the sort-based exact method (Held, Wolfe and Crowder 1974; Duchi et al.
    2008).  Sort descending u, take the largest j with u_j - (sum_{i<=j} u_i - 1)/j > 0,
    theta = (sum_{i<=j} u_i - 1)/j, beta = max(v - theta, 0)."""
    v = np.asarray(v, dtype=np.float64)
    if v.size == 0:
        return v.copy()
    u = np.sort(v)[::-1]
    css = np.cumsum(u)
    j = np.arange(1, v.size + 1)
    ok = u - (css - 1.0) / j > 0
    rho = int(np.nonzero(ok)[0][-1]) + 1
    theta = (css[rho - 1] - 1.0) / rho
    return np.maximum(v - theta, 0.0)


def prune(beta, tau):
    """The truncation map P_tau of Sec. III-A (Eq. truncation-map): keep the indices with
    beta_r > tau (strict), renormalise them to sum 1.  When no index survives, keep the
    largest one (lowest index on ties).  Returns (kept indices, renormalised weights)."""
    beta = np.asarray(beta, dtype=np.float64)
    keep = np.nonzero(beta > tau)[0]
    if keep.size == 0:
        keep = np.array([int(np.argmax(beta))])
    b = beta[keep]
    return keep, b / b.sum()


def refactor(psi, w, tau):
    """Exact spectral refactorisation of rho = Psi diag(w) Psi^* (the spectral step of
    Sec. III-C with eta_rho = 0, where its Ritz pairs are exact): through the K x K Gram
    matrix C = diag(sqrt w) Psi^* Psi diag(sqrt w) = V Lambda V^*, the eigenvectors of rho
    are phi_j = Psi diag(sqrt w) v_j / sqrt(lambda_j) with eigenvalues lambda_j.  Eigenpairs
    are sorted descending, weights lambda / sum(lambda), then P_tau.
    Returns (atoms [K'][D], weights [K'])."""
    psi = np.asarray(psi, dtype=np.complex128)
    w = np.asarray(w, dtype=np.float64)
    sw = np.sqrt(np.maximum(w, 0.0))
    B = psi.T * sw                     # D x K: columns sqrt(w_k) psi_k
    C = B.conj().T @ B                 # K x K Hermitian PSD
    lam, V = np.linalg.eigh(C)
    order = np.argsort(lam)[::-1]
    lam, V = lam[order], V[:, order]
    lam = np.maximum(lam, 0.0)
    weights = lam / lam.sum()
    keep, wk = prune(weights, tau)
    phi = (B @ V[:, keep]) / np.sqrt(lam[keep])
    return np.ascontiguousarray(phi.T), wk


def objective(n, data, psi, w, eps, mu):
    """J = L_eps(A(Psi) w) + mu R (Eq. fixed-rank-objective), R = number of atoms with
    w_r > 0 (zero-weight slots are not part of the state)."""
    f = forward(n, data["basis"], psi, w, data["row_ptr"], data["outcome"], data["count"], data["shots"], eps=eps)
    R = int(np.count_nonzero(np.asarray(w) > 0))
    return f["loss"] + mu * R, f


def _orth_block(W, drop, scale):
    """Orthonormal rows spanning the rows of W: from the Gram matrix
    C_ij = <w_i, w_j> = V Lambda V^*, u_j = sum_i V_ij w_i / sqrt(lambda_j) for the
    eigenvalues lambda_j > drop * scale (scale: the squared Frobenius norm of the
    block before any projection), sorted descending."""
    C = W.conj() @ W.T
    lam, V = np.linalg.eigh(C)
    order = np.argsort(lam)[::-1]
    lam, V = lam[order], V[:, order]
    keep = lam > drop * scale
    return (V[:, keep] / np.sqrt(lam[keep])[None, :]).T @ W


def krylov_ritz(n, data, psi, w, c_obs, eta, n_krylov=30, drop=1e-10, B=None):
    """Ritz pairs of S = Psi diag(w) Psi^* + eta G (Eqs. density-proposal,
    density-product, ritz-pairs) from a block Krylov space started at the atoms
    (the block of K vectors; one product with G per block, as the adjoint gives):
      Q_0 = orth(Psi);  W = S Q_j minus its components on every previous block,
      taken twice (full reorthogonalisation);  Q_{j+1} = orth(W);
    while the basis stays within n_krylov vectors.  Rayleigh-Ritz on
    T = Q^* S Q (Hermitian part).  A block direction is dropped when its squared
    norm after the projections is below drop times the block's squared norm
    before them.  Returns (lam descending, Phi [m][D] Ritz vectors)."""
    psi = np.asarray(psi, dtype=np.complex128)
    w = np.asarray(w, dtype=np.float64)
    K = psi.shape[0]

    def S(V):  # rows of V are vectors
        G = apply_G(n, data["basis"], data["row_ptr"], data["outcome"], c_obs, V, B)
        rho = (psi.T @ (w[:, None] * (psi.conj() @ V.T))).T
        return rho + eta * G

    blocks = [_orth_block(psi, drop, float(np.sum(np.abs(psi) ** 2)))]
    sblocks = []
    while True:
        SQ = S(blocks[-1])
        sblocks.append(SQ)
        m = sum(b.shape[0] for b in blocks)
        if m + K > n_krylov or blocks[-1].shape[0] == 0:
            break
        W = SQ.copy()
        for _ in range(2):
            for Qb in blocks:
                W = W - (Qb.conj() @ W.T).T @ Qb
        Qn = _orth_block(W, drop, float(np.sum(np.abs(SQ) ** 2)))
        if Qn.shape[0] == 0:
            break
        blocks.append(Qn)
    Q = np.vstack(blocks)
    SQ = np.vstack(sblocks[:len(blocks)])
    T = Q.conj() @ SQ.T
    T = 0.5 * (T + T.conj().T)
    lam, Y = np.linalg.eigh(T)
    order = np.argsort(lam)[::-1]
    lam, Y = lam[order], Y[:, order]
    return lam, Y.T @ Q


def spectral_candidates(lam, eta, mu, tau, L):
    """Candidates of Eq. spectral-candidates and their scores (Eq.
    proximal-surrogate): for s = 1..L, beta = P_tau(proj_Delta(lam_1..s)); with
    orthonormal Ritz vectors ||rho_X - S||_F^2 = ||beta||^2 - 2 beta^T lam_I + ||S||_F^2,
    and the last term is the same for every candidate, so
    Q_s = (||beta||^2 - 2 beta^T lam_I) / (2 eta) + mu |I|.  Returns
    (s* (1-based, first minimum), [(kept indices, weights, Q_s) for s = 1..L])."""
    out = []
    for s_ in range(1, L + 1):
        beta = simplex_project(lam[:s_])
        keep, b = prune(beta, tau)
        q = (np.dot(b, b) - 2.0 * np.dot(b, lam[keep])) / (2.0 * eta) + mu * keep.size
        out.append((keep, b, q))
    qs = [c[2] for c in out]
    return int(np.argmin(qs)) + 1, out


def step(n, data, psi, w, slot, r, eps=1e-8, mu=1e-3, tau=1e-3, tau_acc=1e-10, eta0=1.0, eta_ratio=0.5,
         n_eta=11, n_krylov=30, rank_fix=0):
    """One slot of Algorithm 1 with the step grid of Sec. IV (eta = eta0 * eta_ratio^j,
    j = 0..n_eta-1, largest first; the first accepted proposal is kept) and the
    acceptance rule J(X~) <= J_t - tau_acc (Eq. state-acceptance-rule).
      slot 0 (T_psi): atom r, direction g = w_r (I - psi psi^*) G psi_r (Eq. atom-direction),
             trial psi~ = (psi + eta g)/||psi + eta g|| (Eq. atom-trial).
      slot 1 (T_alpha): beta = proj_Delta(w + eta h) over the active atoms (Eq.
             coefficient-update), then P_tau.
      slot 2 (T_rho): the exact spectral refactorisation of rho_t (eta_rho = 0), then P_tau;
             one proposal, no step grid.
      slot 3 (T_rho): the spectral step of Sec. III-C with eta_rho from the step grid:
             Ritz pairs of S_t = rho_t + eta G_t (krylov_ritz), candidates and their
             scores (spectral_candidates, L_t = K), the best candidate, acceptance;
             with rank_fix > 0 the candidate with min(rank_fix, L_t) Ritz pairs is taken
             instead of the best (the known-rank variant of the ablation in Sec. IV).
    Zero-weight slots are inactive.  Returns (psi, w, J, accepted, eta)."""
    psi = np.array(psi, dtype=np.complex128)
    w = np.array(w, dtype=np.float64)
    J0, f0 = objective(n, data, psi, w, eps, mu)
    etas = [eta0 * eta_ratio ** j for j in range(n_eta)]
    if slot == 2:
        active = np.nonzero(w > 0)[0]
        phi, wk = refactor(psi[active], w[active], tau)
        pt = np.zeros_like(psi)
        wt = np.zeros_like(w)
        pt[:phi.shape[0]] = phi
        wt[:wk.size] = wk
        Jt, _ = objective(n, data, pt, wt, eps, mu)
        if Jt <= J0 - tau_acc:
            return pt, wt, Jt, True, 0.0
        return psi, w, J0, False, 0.0
    if slot == 3:
        K = psi.shape[0]
        for eta in etas:
            lam, Phi = krylov_ritz(n, data, psi, w, f0["c_obs"], eta, n_krylov)
            L = min(K, lam.size)
            s_star, cands = spectral_candidates(lam, eta, mu, tau, L)
            if rank_fix > 0:
                s_star = min(rank_fix, L)
            keep, b, _ = cands[s_star - 1]
            pt = np.zeros_like(psi)
            wt = np.zeros_like(w)
            pt[:keep.size] = Phi[keep]
            wt[:keep.size] = b
            Jt, _ = objective(n, data, pt, wt, eps, mu)
            if Jt <= J0 - tau_acc:
                return pt, wt, Jt, True, eta
        return psi, w, J0, False, etas[-1]
    adj = adjoint(n, data["basis"], psi, w, data["row_ptr"], data["outcome"], f0["c_obs"])
    if slot == 0:
        g = tangent(psi[r:r + 1], w[r:r + 1], adj["G_psi"][r:r + 1])[0]
        for eta in etas:
            t = psi[r] + eta * g
            pt = psi.copy()
            pt[r] = t / np.linalg.norm(t)
            Jt, _ = objective(n, data, pt, w, eps, mu)
            if Jt <= J0 - tau_acc:
                return pt, w, Jt, True, eta
        return psi, w, J0, False, etas[-1]
    h = adj["h"]
    active = np.nonzero(w > 0)[0]
    for eta in etas:
        beta = simplex_project(w[active] + eta * h[active])
        keep, b = prune(beta, tau)
        wt = np.zeros_like(w)
        wt[active[keep]] = b
        Jt, _ = objective(n, data, psi, wt, eps, mu)
        if Jt <= J0 - tau_acc:
            return psi, wt, Jt, True, eta
    return psi, w, J0, False, etas[-1]
