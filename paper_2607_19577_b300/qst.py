"""Thin Python binding of libqst.so (include/qst.h): argument marshalling only.

Every step of the forward/adjoint runs in the library's CUDA kernels; this
module checks dtypes/shapes, passes device pointers and the current CUDA
stream, and raises on a non-OK status.  There is no CPU fallback: if the
library is missing, ``load()`` raises.

PyTorch supplies device memory and streams only.  ``QSTLoss`` wraps
forward + adjoint as a ``torch.autograd.Function``: for a real loss PyTorch
expects 2 * dL/dpsi^* as the gradient of a complex tensor, so backward returns
2 * grad_output * (-w_k G psi_k) for the atoms and grad_output * (-h_k) for
the weights.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from pathlib import Path

import numpy as np
import torch

LIB_PATH = Path(__file__).resolve().parent / "libqst.so"

QST_OK = 0
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "unsupported size", 3: "CUDA error",
                4: "out of device memory", 5: "device-side error"}
DEV_BITS = {1: "bad basis code", 2: "malformed CSR counts", 4: "zero shots on a non-empty row",
            8: "non-finite loss", 16: "bounded wait of a kernel on its own copies timed out"}
KERNEL_KINDS = ["pack", "validate", "forward", "loss", "adjoint", "reduce", "hsum", "epilogue", "refactor", "step",
                "high", "tangent"]


class QSTError(RuntimeError):
    pass


class _Params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("norm_settings", ctypes.c_int),
                ("chunk_qubits", ctypes.c_int), ("max_bin_settings", ctypes.c_int),
                ("validate", ctypes.c_int), ("reg_bits", ctypes.c_int), ("fixed_rounds", ctypes.c_int),
                ("phi_cache", ctypes.c_int), ("precision", ctypes.c_int)]


class _StepParams(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("tau", ctypes.c_double), ("tau_acc", ctypes.c_double),
                ("eta0", ctypes.c_double), ("eta_ratio", ctypes.c_double), ("n_eta", ctypes.c_int),
                ("n_krylov", ctypes.c_int), ("rank_fix", ctypes.c_int)]


class _IterParams(ctypes.Structure):
    _fields_ = [("step", _StepParams), ("T_alpha", ctypes.c_int), ("T_ref", ctypes.c_int),
                ("delta_window", ctypes.c_int), ("delta_tol", ctypes.c_double),
                ("max_oracle_calls", ctypes.c_longlong), ("spectral", ctypes.c_int)]


_lib = None


def load():
    """Load libqst.so (fails loudly when it has not been built)."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise QSTError(f"{LIB_PATH} is missing: build it with paper_2607_19577_b300/build.py")
        lib = ctypes.CDLL(str(LIB_PATH))
        P, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.qst_params_default.argtypes = [ctypes.POINTER(_Params)]
        lib.qst_params_default.restype = None
        lib.qst_status_string.argtypes = [i32]
        lib.qst_status_string.restype = ctypes.c_char_p
        lib.qst_plan_create.argtypes = [ctypes.POINTER(P), i32, i32, i32, i64, ctypes.POINTER(_Params)]
        lib.qst_plan_destroy.argtypes = [P]
        lib.qst_plan_workspace_bytes.argtypes = [P, ctypes.POINTER(i64)]
        lib.qst_plan_geometry.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
        lib.qst_tangent.argtypes = [P, P, P, P, P, P, P]
        lib.qst_iter_params_default.argtypes = [ctypes.POINTER(_IterParams)]
        lib.qst_iter_params_default.restype = None
        lib.qst_iterate.argtypes = [P, i32, i32, P, P, P, P, P, P, P, ctypes.POINTER(_IterParams), P, P, P]
        lib.qst_iterate_state.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_longlong),
                                          ctypes.POINTER(i32), ctypes.POINTER(f64)]
        lib.qst_forward.argtypes = [P] + [P] * 11 + [P]
        lib.qst_adjoint.argtypes = [P] + [P] * 8 + [P]
        lib.qst_evaluate_host.argtypes = [P] + [P] * 11 + [P]
        lib.qst_evaluate.argtypes = [P] + [P] * 12 + [P]
        lib.qst_plan_status.argtypes = [P, ctypes.POINTER(i32)]
        lib.qst_plan_set_timing.argtypes = [P, i32]
        lib.qst_plan_kernel_stats.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(f64), i32]
        lib.qst_plan_reset_stats.argtypes = [P]
        lib.qst_plan_launch_count.argtypes = [P, ctypes.POINTER(i64)]
        lib.qst_adjoint_noalloc.argtypes = [i32, i32, i32, i64, ctypes.POINTER(_Params)] + [P] * 9 + [P]
        lib.qst_simplex_project.argtypes = [P, i32, f64, P, P, P, P]
        lib.qst_refactor.argtypes = [P, P, P, f64, P, P]
        lib.qst_batch_create.argtypes = [ctypes.POINTER(P), i32, P, P, P, P, ctypes.POINTER(_Params)]
        lib.qst_batch_create_each.argtypes = [ctypes.POINTER(P), i32, P, P, P, P, ctypes.POINTER(_Params)]
        lib.qst_batch_destroy.argtypes = [P]
        lib.qst_batch_plan.argtypes = [P, i32, ctypes.POINTER(P)]
        lib.qst_batch_evaluate.argtypes = [P] + [P] * 11 + [P]
        lib.qst_batch_iterate.argtypes = [P, i32, i32] + [P] * 7 + [ctypes.POINTER(_IterParams), P, P, P]
        lib.qst_step_params_default.argtypes = [ctypes.POINTER(_StepParams)]
        lib.qst_step_params_default.restype = None
        lib.qst_step.argtypes = [P, i32, i32, P, P, P, P, P, P, P, ctypes.POINTER(_StepParams),
                                 ctypes.POINTER(f64), ctypes.POINTER(i32), ctypes.POINTER(f64), P]
        for name in ["qst_plan_create", "qst_plan_destroy", "qst_plan_workspace_bytes", "qst_plan_geometry", "qst_tangent", "qst_iterate", "qst_iterate_state", "qst_forward",
                     "qst_adjoint", "qst_evaluate", "qst_evaluate_host", "qst_plan_status", "qst_plan_set_timing",
                     "qst_plan_kernel_stats", "qst_plan_reset_stats", "qst_plan_launch_count",
                     "qst_adjoint_noalloc", "qst_simplex_project", "qst_refactor", "qst_step",
                     "qst_batch_create", "qst_batch_create_each", "qst_batch_destroy", "qst_batch_plan",
                     "qst_batch_evaluate", "qst_batch_iterate"]:
            getattr(lib, name).restype = i32
        _lib = lib
    return _lib


def _check(rc, what):
    if rc != QST_OK:
        raise QSTError(f"{what}: {STATUS_NAMES.get(rc, rc)}")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need(t, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise QSTError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise QSTError(f"{name}: expected contiguous {dtype} {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")


@dataclass
class Data:
    """Measurement data resident on the device (Sec. IV): Pauli strings and CSR counts."""
    n: int
    basis: torch.Tensor     # uint8 [M][n]
    row_ptr: torch.Tensor   # int64 [M+1]
    outcome: torch.Tensor   # int32 view of uint32 [nnz]
    count: torch.Tensor     # int32 view of uint32 [nnz]
    shots: torch.Tensor     # int32 view of uint32 [M]

    @property
    def M(self):
        return self.basis.shape[0]

    @property
    def nnz(self):
        return self.outcome.shape[0]

    @staticmethod
    def from_numpy(n, basis, row_ptr, outcome, count, shots, device="cuda"):
        def dev(a, dt):
            return torch.from_numpy(np.ascontiguousarray(a).view(dt)).to(device)
        return Data(n=n, basis=dev(np.asarray(basis, np.uint8), np.uint8),
                    row_ptr=dev(np.asarray(row_ptr, np.int64), np.int64),
                    outcome=dev(np.asarray(outcome, np.uint32), np.int32),
                    count=dev(np.asarray(count, np.uint32), np.int32),
                    shots=dev(np.asarray(shots, np.uint32), np.int32))


class Plan:
    """Owns a qst_plan (device workspace for one problem shape)."""

    def __init__(self, n, M, K, nnz, eps=1e-8, norm_settings=0, chunk_qubits=0,
                 max_bin_settings=0, validate=True, reg_bits=0, fixed_rounds=-1, phi_cache=-1, precision=0):
        lib = load()
        prm = _Params()
        lib.qst_params_default(ctypes.byref(prm))
        prm.eps, prm.norm_settings, prm.chunk_qubits = float(eps), int(norm_settings), int(chunk_qubits)
        prm.max_bin_settings, prm.validate = int(max_bin_settings), int(bool(validate))
        # fixed_rounds: 12-qubit chunks 2 = two 6-qubit rounds, 1 = three 4-qubit rounds;
        # whole states of 5..9 qubits 3 = a warp per (bin, atom); n = 17..20 4 = 16-qubit
        # chunks on CTA clusters; 0 = per-setting rounds, -1 = automatic (True / False mean 1 / 0)
        prm.reg_bits, prm.fixed_rounds = int(reg_bits), int(fixed_rounds)
        # phi_cache: qst_evaluate's transform cache (two-round plans): 1 on, 0 off, -1 automatic
        prm.phi_cache = int(phi_cache)
        # precision (two-round plans): 0 FP32 butterflies; 1..3 tensor-core group
        # products with the data split into that many BF16 terms
        prm.precision = int(precision)
        h = ctypes.c_void_p()
        _check(lib.qst_plan_create(ctypes.byref(h), int(n), int(M), int(K), int(nnz), ctypes.byref(prm)),
               "qst_plan_create")
        self._h, self.n, self.M, self.K, self.nnz = h, n, M, K, nnz
        self.D = 1 << n

    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                load().qst_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self):
        v = ctypes.c_int64()
        _check(load().qst_plan_workspace_bytes(self._h, ctypes.byref(v)), "workspace_bytes")
        return v.value

    def tangent(self, psi, w, grad_psi, grad_w, out=None):
        """d_k = w_k (I - psi_k psi_k^*) G psi_k from the adjoint's outputs (out may be grad_psi)."""
        _need(psi, torch.complex64, (self.K, self.D), "psi")
        _need(grad_psi, torch.complex64, (self.K, self.D), "grad_psi")
        _need(w, torch.float32, (self.K,), "w")
        _need(grad_w, torch.float32, (self.K,), "grad_w")
        out = torch.empty_like(grad_psi) if out is None else out
        _need(out, torch.complex64, (self.K, self.D), "out")
        _check(load().qst_tangent(self._h, _ptr(psi), _ptr(w), _ptr(grad_psi), _ptr(grad_w), _ptr(out), _stream()),
               "qst_tangent")
        return out

    def geometry(self):
        """dict(chunk_qubits, high_qubits, fixed_rounds) of this plan (fixed_rounds: 4 = 16-qubit
        chunks on CTA clusters, 3 = warp units, 2 = two 6-qubit rounds, 1 = three 4-qubit rounds,
        0 = per-setting rounds)."""
        c, r, fx = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().qst_plan_geometry(self._h, ctypes.byref(c), ctypes.byref(r), ctypes.byref(fx)), "geometry")
        return {"chunk_qubits": c.value, "high_qubits": r.value, "fixed_rounds": fx.value}

    def _data(self, d: Data):
        _need(d.basis, torch.uint8, (self.M, self.n), "basis")
        _need(d.row_ptr, torch.int64, (self.M + 1,), "row_ptr")
        _need(d.outcome, torch.int32, (self.nnz,), "outcome")
        _need(d.count, torch.int32, (self.nnz,), "count")
        _need(d.shots, torch.int32, (self.M,), "shots")

    def forward(self, psi, w, d: Data, p_obs=None, c_obs=None, loss=None, p_dense=None):
        """Runs qst_forward; returns (p_obs, c_obs, loss) (allocated when not given)."""
        _need(psi, torch.complex64, (self.K, self.D), "psi")
        _need(w, torch.float32, (self.K,), "w")
        self._data(d)
        dev = psi.device
        p_obs = torch.empty(self.nnz, dtype=torch.float32, device=dev) if p_obs is None else p_obs
        c_obs = torch.empty(self.nnz, dtype=torch.float32, device=dev) if c_obs is None else c_obs
        loss = torch.empty(1, dtype=torch.float64, device=dev) if loss is None else loss
        if p_dense is not None:
            _need(p_dense, torch.float32, (self.M, self.D), "p_dense")
        rc = load().qst_forward(self._h, _ptr(psi), _ptr(w), _ptr(d.basis), _ptr(d.row_ptr),
                                _ptr(d.outcome), _ptr(d.count), _ptr(d.shots), _ptr(p_obs), _ptr(c_obs),
                                _ptr(loss), _ptr(p_dense), _stream())
        _check(rc, "qst_forward")
        return p_obs, c_obs, loss

    def adjoint(self, psi, w, d: Data, c_obs, grad_psi=None, grad_w=None):
        """Runs qst_adjoint; returns (grad_psi = -w_k G psi_k, grad_w = -h)."""
        _need(psi, torch.complex64, (self.K, self.D), "psi")
        _need(w, torch.float32, (self.K,), "w")
        _need(c_obs, torch.float32, (self.nnz,), "c_obs")
        self._data(d)
        grad_psi = torch.empty_like(psi) if grad_psi is None else grad_psi
        grad_w = torch.empty_like(w) if grad_w is None else grad_w
        rc = load().qst_adjoint(self._h, _ptr(psi), _ptr(w), _ptr(d.basis), _ptr(d.row_ptr),
                                _ptr(d.outcome), _ptr(c_obs), _ptr(grad_psi), _ptr(grad_w), _stream())
        _check(rc, "qst_adjoint")
        return grad_psi, grad_w

    def evaluate(self, psi, w, d: Data, p_obs=None, c_obs=None, loss=None, grad_psi=None, grad_w=None):
        """Runs qst_evaluate (forward, then the adjoint with the forward's c, using the
        plan's transform cache when it has one); returns (p_obs, c_obs, loss, grad_psi, grad_w)."""
        _need(psi, torch.complex64, (self.K, self.D), "psi")
        _need(w, torch.float32, (self.K,), "w")
        self._data(d)
        dev = psi.device
        p_obs = torch.empty(self.nnz, dtype=torch.float32, device=dev) if p_obs is None else p_obs
        c_obs = torch.empty(self.nnz, dtype=torch.float32, device=dev) if c_obs is None else c_obs
        loss = torch.empty(1, dtype=torch.float64, device=dev) if loss is None else loss
        grad_psi = torch.empty_like(psi) if grad_psi is None else grad_psi
        grad_w = torch.empty_like(w) if grad_w is None else grad_w
        _need(p_obs, torch.float32, (self.nnz,), "p_obs")
        _need(c_obs, torch.float32, (self.nnz,), "c_obs")
        _need(loss, torch.float64, (1,), "loss")
        _need(grad_psi, torch.complex64, (self.K, self.D), "grad_psi")
        _need(grad_w, torch.float32, (self.K,), "grad_w")
        rc = load().qst_evaluate(self._h, _ptr(psi), _ptr(w), _ptr(d.basis), _ptr(d.row_ptr), _ptr(d.outcome),
                                 _ptr(d.count), _ptr(d.shots), _ptr(p_obs), _ptr(c_obs), _ptr(loss), _ptr(grad_psi),
                                 _ptr(grad_w), _stream())
        _check(rc, "qst_evaluate")
        return p_obs, c_obs, loss, grad_psi, grad_w

    def evaluate_host(self, psi, w, basis, row_ptr, outcome, count, shots, stream=None):
        """Forward + adjoint from host numpy arrays (copies inside the call).
        Returns (loss, grad_psi complex64 [K][D], grad_w float32 [K])."""
        psi = np.ascontiguousarray(psi, dtype=np.complex64)
        w = np.ascontiguousarray(w, dtype=np.float32)
        arrs = [np.ascontiguousarray(basis, np.uint8), np.ascontiguousarray(row_ptr, np.int64),
                np.ascontiguousarray(outcome, np.uint32), np.ascontiguousarray(count, np.uint32),
                np.ascontiguousarray(shots, np.uint32)]
        return self.evaluate_host_buffers(psi, w, *arrs, stream=stream)

    def evaluate_host_buffers(self, psi, w, basis, row_ptr, outcome, count, shots, out=None, stream=None):
        """Like evaluate_host, for arrays the caller keeps (e.g. pinned), with
        optional preallocated outputs (loss[1] f64, grad_psi, grad_w)."""
        if out is None:
            out = (np.zeros(1, np.float64), np.empty((self.K, self.D), np.complex64), np.empty(self.K, np.float32))
        loss, gp, gw = out

        def hp(a):
            return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else None
        st = ctypes.c_void_p(stream if stream is not None else torch.cuda.current_stream().cuda_stream)
        rc = load().qst_evaluate_host(self._h, hp(psi), hp(w), hp(basis), hp(row_ptr), hp(outcome), hp(count),
                                      hp(shots), hp(loss), hp(gp), hp(gw), None, st)
        _check(rc, "qst_evaluate_host")
        return float(loss[0]), gp, gw

    def refactor(self, psi, w, tau, k_out=None):
        """qst_refactor, in place on psi [K][D] complex64 and w [K] float32; returns
        the device int tensor holding the number of kept atoms."""
        _need(psi, torch.complex64, (self.K, self.D), "psi")
        _need(w, torch.float32, (self.K,), "w")
        k_out = torch.zeros(1, dtype=torch.int32, device=psi.device) if k_out is None else k_out
        _check(load().qst_refactor(self._h, _ptr(psi), _ptr(w), float(tau), _ptr(k_out), _stream()),
               "qst_refactor")
        return k_out

    def step(self, slot, r, psi, w, d: Data, **params):
        """qst_step: one slot of Algorithm 1 (0 = atom r, 1 = coefficients, 2 = refactor,
        3 = spectral step with Lanczos Ritz pairs),
        in place on psi and w.  Returns (J, accepted, eta_used)."""
        _need(psi, torch.complex64, (self.K, self.D), "psi")
        _need(w, torch.float32, (self.K,), "w")
        self._data(d)
        sp = _StepParams()
        load().qst_step_params_default(ctypes.byref(sp))
        for k, v in params.items():
            setattr(sp, k, v)
        J, acc, eta = ctypes.c_double(), ctypes.c_int(), ctypes.c_double()
        _check(load().qst_step(self._h, int(slot), int(r), _ptr(psi), _ptr(w), _ptr(d.basis), _ptr(d.row_ptr),
                               _ptr(d.outcome), _ptr(d.count), _ptr(d.shots), ctypes.byref(sp), ctypes.byref(J),
                               ctypes.byref(acc), ctypes.byref(eta), _stream()), "qst_step")
        return J.value, bool(acc.value), eta.value

    def iterate(self, T, t0, psi, w, d: Data, J_hist=None, accepted=None, T_alpha=5, T_ref=50, delta_window=20,
                delta_tol=1e-4, max_oracle_calls=100000, spectral=False, **step_params):
        """qst_iterate: T iterations of Algorithm 1 from iteration t0, in place on psi
        and w, every decision on the device (one CUDA graph, replayed on later calls
        with the same buffers), with the stopping rules of Table I (delta over the
        last delta_window accepted updates below delta_tol, or max_oracle_calls
        serial-equivalent oracle calls; 0 disables either).  spectral: the T_rho
        slots run the spectral step (qst_step slot 3) between graph segments, the
        host synchronising there.  Returns device tensors (J_hist float64 [T],
        accepted int32 [T]); nothing else is synchronised."""
        _need(psi, torch.complex64, (self.K, self.D), "psi")
        _need(w, torch.float32, (self.K,), "w")
        self._data(d)
        ip = _IterParams()
        load().qst_iter_params_default(ctypes.byref(ip))
        ip.T_alpha, ip.T_ref = int(T_alpha), int(T_ref)
        ip.delta_window, ip.delta_tol, ip.max_oracle_calls = int(delta_window), float(delta_tol), int(max_oracle_calls)
        ip.spectral = int(bool(spectral))
        for k, v in step_params.items():
            setattr(ip.step, k, v)
        J_hist = torch.empty(T, dtype=torch.float64, device="cuda") if J_hist is None else J_hist
        accepted = torch.empty(T, dtype=torch.int32, device="cuda") if accepted is None else accepted
        _check(load().qst_iterate(self._h, int(T), int(t0), _ptr(psi), _ptr(w), _ptr(d.basis), _ptr(d.row_ptr),
                                  _ptr(d.outcome), _ptr(d.count), _ptr(d.shots), ctypes.byref(ip), _ptr(J_hist),
                                  _ptr(accepted), _stream()), "qst_iterate")
        return J_hist, accepted

    def iterate_state(self):
        """qst_iterate_state (synchronises): dict(stopped, oracle_calls, accepted_updates, J)."""
        st, calls, acc, J = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_int(), ctypes.c_double()
        _check(load().qst_iterate_state(self._h, ctypes.byref(st), ctypes.byref(calls), ctypes.byref(acc),
                                        ctypes.byref(J)), "qst_iterate_state")
        return {"stopped": bool(st.value), "oracle_calls": calls.value, "accepted_updates": acc.value, "J": J.value}

    def status(self):
        """Synchronise and return the device status bits (0 = clean)."""
        st = ctypes.c_int()
        rc = load().qst_plan_status(self._h, ctypes.byref(st))
        if rc not in (QST_OK, 5):
            _check(rc, "qst_plan_status")
        return st.value

    def check(self):
        st = self.status()
        if st:
            names = [v for b, v in DEV_BITS.items() if st & b]
            raise QSTError("device-side error: " + ", ".join(names))

    def set_timing(self, on=True):
        _check(load().qst_plan_set_timing(self._h, int(bool(on))), "set_timing")

    def kernel_stats(self):
        n = len(KERNEL_KINDS)
        la = (ctypes.c_int64 * n)()
        ms = (ctypes.c_double * n)()
        _check(load().qst_plan_kernel_stats(self._h, la, ms, n), "kernel_stats")
        return {k: (la[i], ms[i]) for i, k in enumerate(KERNEL_KINDS)}

    def reset_stats(self):
        _check(load().qst_plan_reset_stats(self._h), "reset_stats")

    def launch_count(self):
        v = ctypes.c_int64()
        _check(load().qst_plan_launch_count(self._h, ctypes.byref(v)), "launch_count")
        return v.value


class QSTLoss(torch.autograd.Function):
    """L_eps(psi, w) with the hand-written adjoint as its backward.

    forward(psi complex64 [K][D], w float32 [K], plan, data) -> loss (float64 scalar).
    The rotated amplitudes are recomputed in backward, not saved."""

    @staticmethod
    def forward(ctx, psi, w, plan: Plan, data: Data):
        psi_c, w_c = psi.detach().contiguous(), w.detach().contiguous()
        _, c_obs, loss = plan.forward(psi_c, w_c, data)
        ctx.save_for_backward(psi_c, w_c, c_obs)
        ctx.plan, ctx.data = plan, data
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        psi, w, c_obs = ctx.saved_tensors
        grad_psi, grad_w = ctx.plan.adjoint(psi, w, ctx.data, c_obs)
        g32 = g.to(torch.float32)
        return 2.0 * g32 * grad_psi, g32 * grad_w, None, None


def simplex_project(v, tau, beta=None, keep=None, k_out=None):
    """qst_simplex_project: v float64 [K] CUDA tensor -> (beta [K], keep [K] int32, k_out [1] int32)."""
    if not (isinstance(v, torch.Tensor) and v.is_cuda and v.dtype == torch.float64 and v.dim() == 1):
        raise QSTError("v must be a 1-D float64 CUDA tensor")
    K = v.shape[0]
    beta = torch.empty_like(v) if beta is None else beta
    keep = torch.empty(K, dtype=torch.int32, device=v.device) if keep is None else keep
    k_out = torch.empty(1, dtype=torch.int32, device=v.device) if k_out is None else k_out
    _check(load().qst_simplex_project(_ptr(v.contiguous()), int(K), float(tau), _ptr(beta), _ptr(keep),
                                      _ptr(k_out), _stream()), "qst_simplex_project")
    return beta, keep, k_out


QST_ERR_SCRATCH_TOO_SMALL = 6
NOALLOC_SCRATCH_BYTES = 32 << 20


def _noalloc_args(psi, w, d: Data, c_obs, grad_psi, grad_w, device_status):
    """Every check qst_adjoint_noalloc's arguments need before their pointers reach
    the library: dtypes, shapes and contiguity first (Plan.adjoint's and Data's
    checks), then that every tensor is on the current CUDA device (the library
    takes its scratch and launches on that device).  Returns n."""
    if not isinstance(psi, torch.Tensor) or psi.dim() != 2:
        raise QSTError("psi must be a 2-D complex64 tensor [K][2^n]")
    K, D = psi.shape
    if K < 1 or D < 2 or D & (D - 1):
        raise QSTError(f"psi: expected [K >= 1][2^n], a power of two with n >= 1, got {tuple(psi.shape)}")
    n = D.bit_length() - 1
    if d.n != n:
        raise QSTError(f"data is for n = {d.n} qubits, psi for n = {n}")
    M, nnz = d.basis.shape[0], d.outcome.shape[0]
    named = [(psi, torch.complex64, (K, D), "psi"), (w, torch.float32, (K,), "w"),
             (grad_psi, torch.complex64, (K, D), "grad_psi"), (grad_w, torch.float32, (K,), "grad_w"),
             (c_obs, torch.float32, (nnz,), "c_obs"), (device_status, torch.int32, (1,), "device_status"),
             (d.basis, torch.uint8, (M, n), "basis"), (d.row_ptr, torch.int64, (M + 1,), "row_ptr"),
             (d.outcome, torch.int32, (nnz,), "outcome"), (d.count, torch.int32, (nnz,), "count"),
             (d.shots, torch.int32, (M,), "shots")]
    for t, dt, shape, name in named:
        if not isinstance(t, torch.Tensor):
            raise QSTError(f"{name} must be a tensor")
        if t.dtype != dt or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
            raise QSTError(f"{name}: expected contiguous {dt} {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")
    for t, _, _, name in named:
        if not t.is_cuda:
            raise QSTError(f"{name} must be a CUDA tensor")
        if t.device.index != torch.cuda.current_device():
            raise QSTError(f"{name} is on cuda:{t.device.index}, the current device is "
                           f"cuda:{torch.cuda.current_device()}")
    return n


def adjoint_noalloc(psi, w, d: Data, c_obs, grad_psi, grad_w, device_status, params=None):
    """qst_adjoint_noalloc: the adjoint for callers that cannot allocate device
    memory (their workspace would otherwise come from cudaMalloc).  Every
    argument is a caller-owned CUDA tensor on the current device; device_status
    is an int32 [1] tensor that receives the device-side data-check bits.
    Arguments are checked here (QSTError) before any pointer reaches the
    library.  Returns the status code (QST_ERR_SCRATCH_TOO_SMALL when the
    problem needs more than the library's fixed scratch)."""
    n = _noalloc_args(psi, w, d, c_obs, grad_psi, grad_w, device_status)
    K = psi.shape[0]
    prm = None
    if params is not None:
        prm = _Params()
        load().qst_params_default(ctypes.byref(prm))
        for k, v in params.items():
            setattr(prm, k, v)
    return load().qst_adjoint_noalloc(int(n), int(d.M), int(K), int(d.nnz),
                                      ctypes.byref(prm) if prm is not None else None,
                                      _ptr(psi), _ptr(w), _ptr(d.basis), _ptr(d.row_ptr), _ptr(d.outcome),
                                      _ptr(c_obs), _ptr(grad_psi), _ptr(grad_w), _ptr(device_status), _stream())


class Batch:
    """qst_batch: many independent instances evaluated as one captured CUDA graph."""

    def __init__(self, shapes, eps=1e-8, params=None, **plan_kw):
        """shapes: list of (n, M, K, nnz).  params: None (plan_kw shared by every
        instance, with the library's batch bin rule) or one dict of plan parameters
        per instance (taken as given, e.g. from autotune_batch)."""
        lib = load()
        arr = lambda vals, ct: (ct * len(vals))(*vals)  # noqa: E731
        self.shapes = [tuple(int(x) for x in s) for s in shapes]
        dims = (arr([s[0] for s in shapes], ctypes.c_int), arr([s[1] for s in shapes], ctypes.c_int),
                arr([s[2] for s in shapes], ctypes.c_int), arr([s[3] for s in shapes], ctypes.c_int64))
        h = ctypes.c_void_p()
        if params is None:
            prm = _Params()
            lib.qst_params_default(ctypes.byref(prm))
            prm.eps = float(eps)
            for k, v in plan_kw.items():
                setattr(prm, k, v)
            _check(lib.qst_batch_create(ctypes.byref(h), len(shapes), *dims, ctypes.byref(prm)), "qst_batch_create")
        else:
            if len(params) != len(shapes):
                raise ValueError("params: one dict per instance")
            prms = (_Params * len(shapes))()
            for prm, kw in zip(prms, params):
                lib.qst_params_default(ctypes.byref(prm))
                prm.eps = float(eps)
                for k, v in {**plan_kw, **kw}.items():
                    setattr(prm, k, v)
            _check(lib.qst_batch_create_each(ctypes.byref(h), len(shapes), *dims, prms), "qst_batch_create_each")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().qst_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def plan(self, i):
        """Instance i's plan (owned by the batch: valid while the batch is open)."""
        h = ctypes.c_void_p()
        _check(load().qst_batch_plan(self._h, int(i), ctypes.byref(h)), "qst_batch_plan")
        p = Plan.__new__(Plan)
        p._h, p._owned = h, False
        p.n, p.M, p.K, p.nnz = self.shapes[i]
        p.D = 1 << p.n
        return p

    def evaluate(self, psis, ws, datas, losses, c_obss, grads, grad_ws):
        """All arguments are lists (one entry per instance) of CUDA tensors."""
        cnt = len(self.shapes)
        P = ctypes.c_void_p * cnt
        ptrs = lambda ts: P(*[t.data_ptr() for t in ts])  # noqa: E731
        _check(load().qst_batch_evaluate(self._h, ptrs(psis), ptrs(ws), ptrs([d.basis for d in datas]),
                                         ptrs([d.row_ptr for d in datas]), ptrs([d.outcome for d in datas]),
                                         ptrs([d.count for d in datas]), ptrs([d.shots for d in datas]),
                                         ptrs(losses), ptrs(c_obss), ptrs(grads), ptrs(grad_ws), _stream()),
               "qst_batch_evaluate")

    def iterate(self, T, t0, psis, ws, datas, J_hists=None, accepteds=None, T_alpha=5, T_ref=50, delta_window=20,
                delta_tol=1e-4, max_oracle_calls=100000, **step_params):
        """qst_batch_iterate: T iterations of Algorithm 1 on every instance (lists of
        CUDA tensors, in place on psis and ws), all instances in one CUDA graph.
        Returns the per-instance (J_hist, accepted) device tensors."""
        ip = _IterParams()
        load().qst_iter_params_default(ctypes.byref(ip))
        ip.T_alpha, ip.T_ref = int(T_alpha), int(T_ref)
        ip.delta_window, ip.delta_tol, ip.max_oracle_calls = int(delta_window), float(delta_tol), int(max_oracle_calls)
        for k, v in step_params.items():
            setattr(ip.step, k, v)
        cnt = len(self.shapes)
        for (n, M, K, nnz), p, w in zip(self.shapes, psis, ws):
            _need(p, torch.complex64, (K, 1 << n), "psi")
            _need(w, torch.float32, (K,), "w")
        J_hists = [torch.empty(T, dtype=torch.float64, device="cuda") for _ in range(cnt)] if J_hists is None else J_hists
        accepteds = [torch.empty(T, dtype=torch.int32, device="cuda") for _ in range(cnt)] if accepteds is None \
            else accepteds
        P = ctypes.c_void_p * cnt
        ptrs = lambda ts: P(*[t.data_ptr() for t in ts])  # noqa: E731
        _check(load().qst_batch_iterate(self._h, int(T), int(t0), ptrs(psis), ptrs(ws), ptrs([d.basis for d in datas]),
                                        ptrs([d.row_ptr for d in datas]), ptrs([d.outcome for d in datas]),
                                        ptrs([d.count for d in datas]), ptrs([d.shots for d in datas]),
                                        ctypes.byref(ip), ptrs(J_hists), ptrs(accepteds), _stream()),
               "qst_batch_iterate")
        return J_hists, accepteds


def qst_loss(psi, w, plan: Plan, data: Data):
    return QSTLoss.apply(psi, w, plan, data)


def autotune(psi, w, d: Data, eps=1e-8, candidates=None, warmup=2, reps=3):
    """Pick the fastest plan layout for this problem by timing forward + adjoint
    (CUDA events on the current stream) over candidate (reg_bits, chunk_qubits,
    max_bin_settings, fixed_rounds) choices: 16 or 32 amplitudes per thread and
    round, the default chunk or one bit smaller, automatic or fixed bin sizes,
    and two 6-qubit, three 4-qubit or per-setting rounds (states of 5..10
    qubits up to 9: a warp per unit or per-setting rounds).

    Returns (best params dict, [(params, ms per evaluation), ...])."""
    K, D = psi.shape
    n = D.bit_length() - 1
    M, nnz = d.M, d.nnz
    if candidates is None:
        c0 = n if n <= 12 else (12 if n <= 16 else n - 8)
        chunks = [0] + ([c0 - 1] if 13 <= n <= 16 and c0 - 1 >= n - 4 else [])
        fxs = (3, 0) if 5 <= n <= 9 else (2, 1, 0)
        candidates = [dict(reg_bits=rb, chunk_qubits=c, max_bin_settings=sm, fixed_rounds=fx)
                      for rb in (4, 5) for c in chunks for sm in (0, 32) for fx in fxs
                      if not (fx and rb == 5)]
    results = []
    for prm in candidates:
        try:
            plan = Plan(n, M, K, nnz, eps=eps, **prm)
        except QSTError:
            continue
        _, c_obs, _ = plan.forward(psi, w, d)
        g, gw = plan.adjoint(psi, w, d, c_obs)
        for _ in range(warmup):
            plan.forward(psi, w, d, c_obs=c_obs)
            plan.adjoint(psi, w, d, c_obs, grad_psi=g, grad_w=gw)
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record()
        for _ in range(reps):
            plan.forward(psi, w, d, c_obs=c_obs)
            plan.adjoint(psi, w, d, c_obs, grad_psi=g, grad_w=gw)
        end.record()
        torch.cuda.synchronize()
        results.append((prm, start.elapsed_time(end) / reps))
        plan.close()
    results.sort(key=lambda x: x[1])
    return results[0][0], results


def batch_candidates(n):
    """Plan layouts the batch autotuner tries for instances of n qubits."""
    if 5 <= n <= 9:
        return ([dict(fixed_rounds=3, max_bin_settings=sm) for sm in (0, 8, 32)] +
                [dict(fixed_rounds=0, max_bin_settings=sm) for sm in (0, 32)])
    if 10 <= n <= 11:
        return ([dict(fixed_rounds=2, max_bin_settings=sm) for sm in (0, 32, 64, 96)] +
                [dict(fixed_rounds=0, max_bin_settings=sm, reg_bits=rb) for sm in (0, 32, 96) for rb in (4, 5)])
    if 12 <= n <= 16:
        return [dict(fixed_rounds=fr, max_bin_settings=sm) for fr in (2, 1) for sm in (0, 32, 64, 96)]
    return [dict()]


def autotune_batch(shapes, psis, ws, datas, eps=1e-8, warmup=2, reps=3, candidates=batch_candidates):
    """Pick a plan layout per size class for qst_batch: for the instances of each n,
    time them as one batch (one launch per phase over the class, as in the full
    batch, so they share the GPU as they will) under each layout of candidates(n),
    CUDA events on the current stream, and keep the fastest.  Returns (per-instance
    params, [(n, params, ms per evaluation), ...])."""
    classes = {}
    for i, s in enumerate(shapes):
        classes.setdefault(int(s[0]), []).append(i)
    chosen, table = [dict() for _ in shapes], []
    for n, idx in sorted(classes.items()):
        best, best_ms = dict(), None
        ps, w_, ds = [psis[i] for i in idx], [ws[i] for i in idx], [datas[i] for i in idx]
        losses = [torch.zeros(1, dtype=torch.float64, device=p.device) for p in ps]
        cs = [torch.zeros(d.nnz, dtype=torch.float32, device=p.device) for p, d in zip(ps, ds)]
        gs = [torch.zeros_like(p) for p in ps]
        gws = [torch.zeros_like(x) for x in w_]
        for cand in candidates(n):
            try:
                b = Batch([shapes[i] for i in idx], eps=eps, params=[cand] * len(idx))
            except QSTError:
                continue
            for _ in range(warmup):
                b.evaluate(ps, w_, ds, losses, cs, gs, gws)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                b.evaluate(ps, w_, ds, losses, cs, gs, gws)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            b.close()
            table.append((n, cand, ms))
            if best_ms is None or ms < best_ms:
                best, best_ms = cand, ms
        for i in idx:
            chosen[i] = dict(best)
    return chosen, table
