#!/usr/bin/env python
"""Benchmark: one step = forward + adjoint over one batch of synthetic data
(n = 16 qubits, M = 4096 random Pauli settings, 2000 shots each, K = 16 atoms),
through the C ABI of libqst.so (qst_evaluate: the forward stores the rotated
amplitudes at the observed outcomes and the adjoint applies the inverse
rotations to them; the line also records the adjoint that recomputes them).

Prints ONE JSON line (rank 0).  Timing: W untimed warm-up steps, then K steps
bracketed by a barrier + device synchronisation; each step is timed with CUDA
events on the launching stream, and L2 is flushed (512 MiB write) between
steps, outside the events.  The result is the max over ranks.  With N > 1
ranks every rank runs an independent replica of the same workload (the
measurement partition needs no collective on one GPU per replica).

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (a few settings per step).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+adjoint amplitudes/s (M×K×2^n), s/iteration, % roofline vs plain FP32 path"
WORKLOAD = "n16_m4096_k16"
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--reg-bits", type=int, default=0, help="amplitudes per thread per round = 2^reg_bits (0 = auto)")
    ap.add_argument("--chunk-qubits", type=int, default=0)
    ap.add_argument("--max-bin-settings", type=int, default=0)
    ap.add_argument("--autotune", action="store_true", help="time candidate plan layouts first and use the fastest")
    ap.add_argument("--iterations", type=int, default=10, help="Algorithm 1 iterations timed through qst_iterate")
    ap.add_argument("--no-iterations", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 64-instance batched evaluation (field batched; single rank only)")
    ap.add_argument("--no-wide", action="store_true",
                    help="skip the n = 20, M = 1024, K = 8 evaluation (field n20; default workload, single rank)")
    ap.add_argument("--shard", action="store_true",
                    help="each rank evaluates a contiguous shard of the settings with the global B and the ranks "
                         "all-reduce (loss, grad, grad_w) every step (measurement partition of Sec. III-B); "
                         "the default runs one replica per rank")
    ap.add_argument("--phi-cache", type=int, default=-1, choices=[-1, 0, 1],
                    help="qst_evaluate's transform cache: 1 on, 0 off (the adjoint recomputes the rotations), "
                         "-1 the plan's automatic choice")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1, 2, 3],
                    help="chunk transforms of two-round plans: 0 FP32 butterflies; 1..3 tensor-core products "
                         "over 6-qubit groups with the data split into that many BF16 terms (the line then also "
                         "times the FP32 plan on the same data: field vs_fp32)")
    ap.add_argument("--fixed-rounds", type=int, default=-1, choices=[-1, 0, 1, 2, 3, 4],
                    help="12-qubit chunk kernels: 2 = two 6-qubit rounds, 1 = three 4-qubit rounds, "
                         "0 = rounds chosen per setting; 3 = warp units (5..9 qubits); 4 = 16-qubit chunks on "
                         "CTA clusters (17..20 qubits); -1 = the plan's automatic choice")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled while the timed region
    runs: NVML every 10 ms from a thread (the device matched by PCI bus id), the
    first sample taken before __enter__ returns; nvidia-smi every 200 ms when NVML
    is not available.  Reading only: no setting of the GPU is changed."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.thread = None
        self.samples = []  # (sm_mhz, sm_max_mhz, set of reasons)
        self.lines = []
        self._stop = threading.Event()

    def _nvml(self):
        """Minimal NVML reader over ctypes (read-only queries of nvml.h): returns
        (sm_clock(), max_sm_clock, reasons()) for the device of self.index."""
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit")
        h = ctypes.c_void_p()
        try:
            import torch
            pr = torch.cuda.get_device_properties(self.index)
            bus = b"%08X:%02X:%02X.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
            if lib.nvmlDeviceGetHandleByPciBusId_v2(bus, ctypes.byref(h)) != 0:
                raise RuntimeError("by bus id")
        except Exception:
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(h)) != 0:
                raise RuntimeError("by index")
        NVML_CLOCK_SM = 1
        mx = ctypes.c_uint()
        if lib.nvmlDeviceGetMaxClockInfo(h, NVML_CLOCK_SM, ctypes.byref(mx)) != 0:
            raise RuntimeError("max clock")
        reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons

        def sm_clock():
            v = ctypes.c_uint()
            lib.nvmlDeviceGetClockInfo(h, NVML_CLOCK_SM, ctypes.byref(v))
            return float(v.value)

        def reasons():
            v = ctypes.c_ulonglong()
            reasons_fn(h, ctypes.byref(v))
            # clock-event reason bits of nvml.h
            bits = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
                    "hw_thermal_slowdown": 0x40}
            return {k for k, b in bits.items() if v.value & b}
        return sm_clock, float(mx.value), reasons

    def _poll(self, sm_clock, mx, reasons, first):
        while True:
            self.samples.append((sm_clock(), mx, reasons()))
            first.set()
            if self._stop.wait(0.01):
                break

    def __enter__(self):
        try:
            sm_clock, mx, reasons = self._nvml()
            first = threading.Event()
            self.thread = threading.Thread(target=self._poll, args=(sm_clock, mx, reasons, first), daemon=True)
            self.thread.start()
            first.wait(timeout=2)
            return self
        except Exception:
            self.thread = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        self._stop.set()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        for a, b, r in self.samples:
            sm.append(a)
            mx.append(b)
            reasons |= r
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names[1:], parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvml, 10 ms" if self.samples else "nvidia-smi, 200 ms"}


def kernel_source_hash():
    """sha256 over the CUDA sources (qst.cu and its headers, in name order)."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2607_19577_b300", "csrc")
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh")):
            h.update(name.encode())
            h.update(open(os.path.join(d, name), "rb").read())
    return h.hexdigest()


def algorithmic_ops(basis, K, D):
    """FP32 lane operations (FADD/FMUL/FFMA each 1) of the plain butterfly method,
    per amplitude with m_s = X/Y qubits of setting s: the forward rotation and
    |.|^2 weighting 2 m_s + 4; the adjoint 4 m_s + 8 when it recomputes the
    rotation (2 m_s + 4 for the recomputation, 2 m_s + 4 for the inverse rotation,
    c scaling and accumulation).  Returns (forward, recomputing adjoint, inverse
    part alone), the last being the work of the adjoint that reads the stored
    transforms."""
    m = np.count_nonzero(basis, axis=1).astype(np.float64)
    fwd = float(np.sum(2 * m + 4)) * K * D
    adj = float(np.sum(4 * m + 8)) * K * D
    inv = float(np.sum(2 * m + 4)) * K * D
    return fwd, adj, inv


def cpu_oracle_rate(inst, budget_s, settings_per_call=1, max_settings=None):
    """Time the FP64 oracle (forward + adjoint, all K atoms) on the first settings
    of the workload, one setting at a time, until budget_s is spent."""
    import oracle
    psi = inst.psi.astype(np.complex128)
    w = inst.w.astype(np.float64)
    done, t_total = 0, 0.0
    while (t_total < budget_s or done < 1) and (max_settings is None or done < max_settings):
        lo = done % inst.M
        hi = min(lo + settings_per_call, inst.M)
        rp = inst.row_ptr[lo:hi + 1] - inst.row_ptr[lo]
        a, b = inst.row_ptr[lo], inst.row_ptr[hi]
        t0 = time.perf_counter()
        f = oracle.forward(inst.n, inst.basis[lo:hi], psi, w, rp, inst.outcome[a:b], inst.count[a:b],
                           inst.shots[lo:hi], eps=inst.eps, B=inst.M)
        oracle.adjoint(inst.n, inst.basis[lo:hi], psi, w, rp, inst.outcome[a:b], f["c_obs"], B=inst.M)
        t_total += time.perf_counter() - t0
        done += hi - lo
    return done, t_total


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def cpu_oracle_rate_all_cores(inst, budget_s, rate_1core, threads):
    """Time the FP64 oracle (forward + adjoint, all K atoms) with the settings of a
    sample sharded over `threads` host threads (oracle.forward_sharded /
    adjoint_sharded: contiguous shards with the global B, each shard one call of
    the unchanged C routines, which release the GIL).  The sample is the first S
    settings, S sized from the single-core rate so the run takes about budget_s."""
    import oracle
    psi = inst.psi.astype(np.complex128)
    w = inst.w.astype(np.float64)
    per_setting = inst.K * inst.D
    S = int(max(threads, min(inst.M, budget_s * rate_1core * threads * 0.6 / per_setting)))
    S = min(S, inst.M)
    e = inst.row_ptr[S]
    t0 = time.perf_counter()
    f = oracle.forward_sharded(inst.n, inst.basis[:S], psi, w, inst.row_ptr[:S + 1], inst.outcome[:e],
                               inst.count[:e], inst.shots[:S], eps=inst.eps, B=inst.M, threads=threads)
    oracle.adjoint_sharded(inst.n, inst.basis[:S], psi, w, inst.row_ptr[:S + 1], inst.outcome[:e], f["c_obs"],
                           B=inst.M, threads=threads)
    return S, time.perf_counter() - t0


def batched_eval(flush, reps=10, autotune=False):
    """The batched workload (64 independent instances, n uniform in 6..14, rank
    1..8, K = 2 rank, 200..3000 settings, 500..5000 shots; synth.make_batch(seed=0)):
    one forward + adjoint of every instance per evaluation, through qst.Batch (one
    CUDA graph launch) and, for comparison, through one plan per instance called
    in sequence.  CUDA events on the current stream, L2 flushed before each
    timed evaluation."""
    import torch
    from paper_2607_19577_b300 import qst, synth
    insts = synth.make_batch(seed=0, count=64)
    amps = sum(i.M * i.K * (1 << i.n) for i in insts)
    datas = [qst.Data.from_numpy(i.n, i.basis, i.row_ptr, i.outcome, i.count, i.shots) for i in insts]
    psis = [torch.from_numpy(i.psi).cuda() for i in insts]
    ws_ = [torch.from_numpy(i.w).cuda() for i in insts]
    losses = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in insts]
    cs = [torch.zeros(i.nnz, dtype=torch.float32, device="cuda") for i in insts]
    gs = [torch.zeros_like(p) for p in psis]
    gws = [torch.zeros_like(w) for w in ws_]
    batch = qst.Batch([(i.n, i.M, i.K, i.nnz) for i in insts])
    plans = [qst.Plan(i.n, i.M, i.K, i.nnz, eps=i.eps) for i in insts]

    def graph():
        batch.evaluate(psis, ws_, datas, losses, cs, gs, gws)

    def sequential():
        for p, ps, w, d, l, c, g, gw in zip(plans, psis, ws_, datas, losses, cs, gs, gws):
            p.forward(ps, w, d, c_obs=c, loss=l)
            p.adjoint(ps, w, d, c, grad_psi=g, grad_w=gw)

    def timed(fn):
        for _ in range(3):
            fn()
        total = 0.0
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        return total / reps

    t_graph, t_seq = timed(graph), timed(sequential)
    for p in plans:
        p.close()
    # Algorithm 1 on every instance, one graph (qst_batch_iterate): 10 iterations of the
    # Table I schedule from the evaluation points, capture untimed, then a timed replay
    it_T = 10
    ip_psis, ip_ws = [p.clone() for p in psis], [w.clone() for w in ws_]
    Jh, acc = batch.iterate(it_T, 0, ip_psis, ip_ws, datas)
    for p, w, p0, w0 in zip(ip_psis, ip_ws, psis, ws_):
        p.copy_(p0)
        w.copy_(w0)
    torch.cuda.synchronize()
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    batch.iterate(it_T, 0, ip_psis, ip_ws, datas, J_hists=Jh, accepteds=acc)
    e1.record()
    torch.cuda.synchronize()
    t_it = e0.elapsed_time(e1) / it_T
    n_acc = int(sum(int(a.sum().item()) for a in acc))
    batch.close()
    out = {"workload": "64 instances, synth.make_batch(seed=0)", "amplitudes_per_eval": int(amps),
           "ms_per_eval": t_graph, "value": amps / t_graph * 1e3, "unit": "amplitudes/s",
           "sequential_ms_per_eval": t_seq, "sequential_value": amps / t_seq * 1e3,
           "iterate": {"ms_per_iteration": t_it, "iterations": it_T, "accepted_updates": n_acc,
                       "how": "qst_batch_iterate: every instance's Algorithm 1 sequence (Table I schedule, "
                              "T_alpha = 5) on a forked stream of one captured graph; one timed replay"},
           "how": "qst.Batch: one launch per phase and kernel family over all instances' CTAs, captured in one "
                  "CUDA graph; sequential: one plan per instance, called in order"}
    if autotune:
        shapes = [(i.n, i.M, i.K, i.nnz) for i in insts]
        chosen, table = qst.autotune_batch(shapes, psis, ws_, datas)
        batch = qst.Batch(shapes, params=chosen)
        t_tuned = timed(graph)
        batch.close()
        out["autotuned"] = {"ms_per_eval": t_tuned, "value": amps / t_tuned * 1e3,
                            "choice_per_n": {str(i.n): c for i, c in zip(insts, chosen)},
                            "table": [{"n": n, "params": c, "ms": ms} for n, c, ms in table],
                            "how": "qst.autotune_batch: per size class, the class's instances timed as one batch "
                                   "under each candidate layout; the fastest per class"}
    return out


def wide_eval(flush, reps=3):
    """The n = 20, M = 1024, K = 8 workload (synth.make_instance("n20_m1024_k8",
    seed=0), 10,000 shots a setting): qst_evaluate on the default plan (the wide
    path) with the transform cache (phi_cache = 1) and recomputing the rotated
    amplitudes in the adjoint (phi_cache = 0), CUDA events on the current
    stream, L2 flushed before each timed evaluation, preallocated outputs."""
    import torch
    from paper_2607_19577_b300 import qst, synth
    inst = synth.make_instance("n20_m1024_k8", seed=0)
    n, M, K = inst.n, inst.M, inst.K
    amps = M * K * (1 << n)
    data = qst.Data.from_numpy(n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    psi, w = torch.from_numpy(inst.psi).cuda(), torch.from_numpy(inst.w).cuda()
    outs = (torch.empty(inst.nnz, dtype=torch.float32, device="cuda"),
            torch.empty(inst.nnz, dtype=torch.float32, device="cuda"),
            torch.empty(1, dtype=torch.float64, device="cuda"), torch.empty_like(psi), torch.empty_like(w))
    out = {"workload": "n20_m1024_k8", "amplitudes_per_eval": int(amps), "unit": "amplitudes/s"}
    for name, cache in (("cached", 1), ("recompute", 0)):
        plan = qst.Plan(n, M, K, inst.nnz, eps=inst.eps, phi_cache=cache)
        for _ in range(2):
            plan.evaluate(psi, w, data, *outs)
        total = 0.0
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.evaluate(psi, w, data, *outs)
            e1.record()
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        plan.check()
        out[name] = {"ms_per_eval": total / reps, "value": amps / (total / reps) * 1e3,
                     "geometry": plan.geometry()}
        plan.close()
    out["how"] = (f"qst_evaluate, {reps} timed evaluations after 2 untimed, L2 flushed before each; "
                  "cached: the adjoint reads the forward's transforms at the observed outcomes")
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2607_19577_b300 import synth
    inst = synth.make_instance(args.workload, seed=0)
    cores = host_cores()
    per_step = min(inst.M, cores)  # one setting per host thread and step
    psi = inst.psi.astype(np.complex128)
    w = inst.w.astype(np.float64)

    def one_step(i):
        lo = (i * per_step) % inst.M
        hi = min(lo + per_step, inst.M)
        a, b = inst.row_ptr[lo], inst.row_ptr[hi]
        rp = inst.row_ptr[lo:hi + 1] - a
        f = oracle.forward_sharded(inst.n, inst.basis[lo:hi], psi, w, rp, inst.outcome[a:b], inst.count[a:b],
                                   inst.shots[lo:hi], eps=inst.eps, B=inst.M, threads=cores)
        oracle.adjoint_sharded(inst.n, inst.basis[lo:hi], psi, w, rp, inst.outcome[a:b], f["c_obs"], B=inst.M,
                               threads=cores)
        return hi - lo
    for i in range(args.warmup):
        one_step(i)
    t, done = 0.0, 0
    for i in range(args.steps):
        t0 = time.perf_counter()
        done += one_step(args.warmup + i)
        t += time.perf_counter() - t0
    amps = done * inst.K * inst.D / args.steps
    value = amps * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "amplitudes/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": args.workload, "n": inst.n, "M": inst.M, "K": inst.K,
                       "step": f"{per_step} settings x {inst.K} atoms x 2^{inst.n} outcomes"},
            "cpu_baseline": {"value": value, "unit": "amplitudes/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} of {inst.M} settings per step (one per host thread), "
                                       f"all {inst.K} atoms, forward + adjoint, FP64 C"},
            "e2e": {"value": value, "unit": "amplitudes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def tc_mma_flops(inst, r, T):
    """FLOPs the tensor-core chunk kernels issue per launch (forward or adjoint):
    per setting, high pattern and atom pair, 2 products x T data terms x 8
    K-steps of one M = N = 128, K = 16 MMA (2 M N K FLOPs each)."""
    return float(inst.M) * (1 << r) * ((inst.K + 1) // 2) * 2 * T * 8 * (2 * 128 * 128 * 16)


def tc_roofline(args, inst, geo, stats, ms_step, plain_ops, peaks, peak_alu):
    """Roofline of the tensor-core variant: its dominant kernel's issued MMA
    FLOPs against the measured BF16 tensor peak (cuBLAS burst)."""
    T = args.precision
    flops = tc_mma_flops(inst, geo["high_qubits"], T)
    peak = float(peaks.get("bf16_tflops", 1800.0))
    src = "MEASURED_PEAKS.json bf16_tflops (cuBLAS BF16 GEMM, burst)" if "bf16_tflops" in peaks else \
        "fallback 1.8 PFLOP/s BF16"
    lf, ms_fwd = stats["forward"]
    la, ms_adj = stats["adjoint"]
    f_ms, a_ms = ms_fwd / args.steps, ms_adj / args.steps
    dom_adj = a_ms >= f_ms
    ms_dom = a_ms if dom_adj else f_ms
    part = lambda ms: {"ops_per_launch": flops, "ms_per_launch": ms,  # noqa: E731
                       "achieved": flops / (ms / 1e3) / 1e12, "frac": flops / (ms / 1e3) / 1e12 / peak}
    return {"bound": "tensor", "achieved": flops / (ms_dom / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
            "frac": flops / (ms_dom / 1e3) / 1e12 / peak, "traffic": None,
            "kernel": "k_adjoint_tc" if dom_adj else "k_forward_tc", "peak_source": src,
            "ops_per_launch": flops, "ms_per_launch": ms_dom,
            "ops_definition": f"tcgen05.mma FLOPs issued: 2 group products x {T} BF16 term(s) x 8 K-steps of "
                              "M = N = 128, K = 16 per (setting, high pattern, atom pair)",
            "launches_per_step": la / args.steps,
            "forward": {"kernel": "k_forward_tc", **part(f_ms)},
            "adjoint": {"kernel": "k_adjoint_tc", **part(a_ms)},
            "step_vs_plain_path": {
                "ops_per_step": plain_ops, "ms_per_step": ms_step,
                "frac": plain_ops / (ms_step / 1e3) / 1e12 / peak_alu,
                "definition": "the plain FP32 method's work (6 m_s + 12 lane-ops per amplitude) at the FP32 lane "
                              "peak, over the tensor-core step's time"}}


def tc_against_fp32(args, inst, plan, psi, w, data, flush, ms_tc, grad, grad_w, loss):
    """The FP32 plan on the same data: its evaluation time (same timing rules)
    and the tensor-core result's distance from it at full size."""
    import torch
    from paper_2607_19577_b300 import qst
    fp = qst.Plan(inst.n, inst.M, inst.K, inst.nnz, eps=inst.eps, reg_bits=args.reg_bits,
                  chunk_qubits=args.chunk_qubits, max_bin_settings=args.max_bin_settings,
                  fixed_rounds=args.fixed_rounds, phi_cache=args.phi_cache, precision=0)
    stream = torch.cuda.current_stream()
    p32, c32, l32, g32, gw32 = fp.evaluate(psi, w, data)
    for _ in range(max(args.warmup, 1)):
        flush.zero_()
        fp.evaluate(psi, w, data, p_obs=p32, c_obs=c32, loss=l32, grad_psi=g32, grad_w=gw32)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for e0, e1 in ev:
        flush.zero_()
        e0.record(stream)
        fp.evaluate(psi, w, data, p_obs=p32, c_obs=c32, loss=l32, grad_psi=g32, grad_w=gw32)
        e1.record(stream)
    torch.cuda.synchronize()
    fp.check()
    ms32 = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    amps = inst.M * inst.K * inst.D
    gn = g32.abs().amax(dim=1)
    out = {"ms_per_step_fp32": ms32, "value_fp32": amps / (ms32 / 1e3), "ms_per_step_tc": ms_tc,
           "tc_over_fp32_throughput": ms32 / ms_tc,
           "grad_err_vs_fp32": float(((grad - g32).abs().amax(dim=1) / gn).max().item()),
           "grad_w_err_vs_fp32": float(((grad_w - gw32).abs() / gw32.abs()).max().item()),
           "loss_err_vs_fp32": float(abs(loss.item() - l32.item()) / abs(l32.item())),
           "how": "the FP32 plan (precision 0) evaluated on the same data and stream right after, "
                  f"{args.steps} steps, L2 flushed between steps; errors: per-atom max |d grad| / max |grad|, "
                  "relative h and loss, tensor-core result against the FP32 one"}
    fp.close()
    return out


def run_ours(args):
    import torch
    from paper_2607_19577_b300 import qst, replicas, synth

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    inst = synth.make_instance(args.workload, seed=0)
    M_all = inst.M
    if args.shard:
        # this rank's contiguous range of the settings, evaluated with the global B
        # (the measurement partition of Sec. III-B); the sums are all-reduced per step
        lo, hi = replicas.shard(M_all, rank, ws)
        rp, ea, eb = replicas.shard_rows(inst.row_ptr, lo, hi)
        inst = synth.Instance(name=inst.name, n=inst.n, basis=inst.basis[lo:hi], shots=inst.shots[lo:hi],
                              row_ptr=rp, outcome=inst.outcome[ea:eb], count=inst.count[ea:eb], psi=inst.psi,
                              w=inst.w)
    n, M, K, D = inst.n, inst.M, inst.K, inst.D
    data = qst.Data.from_numpy(n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    psi = torch.from_numpy(inst.psi).cuda()
    w = torch.from_numpy(inst.w).cuda()
    tuned = None
    if args.autotune:
        best, table = qst.autotune(psi, w, data, eps=inst.eps)
        args.reg_bits, args.chunk_qubits, args.max_bin_settings = (best["reg_bits"], best["chunk_qubits"],
                                                                    best["max_bin_settings"])
        args.fixed_rounds = best["fixed_rounds"]
        tuned = [{"params": p, "ms": t} for p, t in table]
    plan = qst.Plan(n, M, K, inst.nnz, eps=inst.eps, reg_bits=args.reg_bits, chunk_qubits=args.chunk_qubits,
                    max_bin_settings=args.max_bin_settings, fixed_rounds=args.fixed_rounds, phi_cache=args.phi_cache,
                    norm_settings=M_all if args.shard else 0, precision=args.precision)
    p_obs = torch.empty(inst.nnz, dtype=torch.float32, device="cuda")
    c_obs = torch.empty_like(p_obs)
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    grad = torch.empty_like(psi)
    grad_w = torch.empty_like(w)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        plan.evaluate(psi, w, data, p_obs=p_obs, c_obs=c_obs, loss=loss, grad_psi=grad, grad_w=grad_w)
        if args.shard:
            replicas.allreduce_evaluation(loss, grad, grad_w, dist)

    for _ in range(max(args.warmup, 0)):
        flush.zero_()  # the first fill also loads torch's kernel (about 0.3 s): keep it out of the timed loop
        step()
    torch.cuda.synchronize()
    plan.check()

    plan.set_timing(True)
    plan.reset_stats()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            step()
            ends[i].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches = plan.launch_count()
    stats = plan.kernel_stats()
    plan.set_timing(False)
    plan.check()
    ms_total = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    amps_step = M * K * D
    # slowest rank's time, every rank's units (each rank runs one replica, or one
    # shard of the settings: then the units add up to the one experiment's M K D)
    ms_total, amps_all = replicas.aggregate(ms_total, amps_step, dist, device="cuda")
    ms_step = ms_total / args.steps
    value = amps_all / (ms_step / 1e3)

    # roofline of the dominant kernel
    fwd_ops, adj_ops, inv_ops = algorithmic_ops(inst.basis, K, D)
    geo = plan.geometry()
    wide = n > 16
    cluster = geo["fixed_rounds"] == 4  # 16-qubit chunks on CTA clusters: the adjoint always reads transforms
    cached = (geo["fixed_rounds"] == 2 and args.phi_cache != 0) or (wide and args.phi_cache == 1) or cluster
    # per-step kernel time (the wide path launches its chunk kernels once per setting group)
    la, ms_adj = stats["adjoint"]
    lf, ms_fwd = stats["forward"]
    adj_ms = ms_adj / args.steps
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    props = torch.cuda.get_device_properties(local)
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    peak_alu = props.multi_processor_count * 128 * sm_max * 1e6 / 1e12  # TFLOP/s, 1 per lane-op
    adj_work = inv_ops if cached else adj_ops  # the adjoint kernel's own algorithmic work
    achieved = adj_work / (adj_ms / 1e3) / 1e12
    if cluster:
        adj_kernel = "k_adjoint_clc"
    elif wide:
        adj_kernel = ("k_adjoint_fx1cp" if cached else "k_adjoint_fx1p") if geo["fixed_rounds"] == 1 else "k_adjoint"
    else:
        adj_kernel = ("k_adjoint_2c" if cached else
                      {2: "k_adjoint_2r", 1: "k_adjoint_fx"}.get(geo["fixed_rounds"], "k_adjoint"))
    traffic = None
    prof = os.path.join(ROOT, "profiles", "adjoint_traffic.json")
    if os.path.exists(prof):
        try:
            rec = json.load(open(prof))
            # counters only count for the kernel source they were taken on
            if (rec.get("source_sha256") == kernel_source_hash() and rec.get("workload") == args.workload
                    and rec.get("kernel") == adj_kernel):
                traffic = rec.get("bytes_per_launch")
        except Exception:
            traffic = None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_alu, "unit": "TFLOP/s",
                "frac": achieved / peak_alu, "traffic": traffic,
                "kernel": adj_kernel,
                "peak_source": f"{props.multi_processor_count} SMs x 128 FP32 lanes x {sm_max:.0f} MHz "
                               "(max SM clock of MEASURED_PEAKS.json)",
                "ops_per_launch": adj_work / max(la / args.steps, 1), "ms_per_launch": adj_ms / max(la / args.steps, 1),
                "ops_definition": ("inverse rotation, c scaling, accumulation: 2 m_s + 4 FP32 lane-ops per "
                                   "amplitude (the adjoint reads the forward's stored transforms)" if cached else
                                   "recomputed rotation + inverse rotation: 4 m_s + 8 FP32 lane-ops per amplitude"),
                "launches_per_step": la / args.steps,
                "forward": {"kernel": ("k_forward_cl" if cluster else "k_forward_fx1p" if wide and geo["fixed_rounds"] == 1 else
                                       {2: "k_forward_2r", 1: "k_forward_fx"}.get(geo["fixed_rounds"], "k_forward")),
                            "ops_per_launch": fwd_ops / max(lf / args.steps, 1),
                            "ms_per_launch": ms_fwd / args.steps / max(lf / args.steps, 1),
                            "launches_per_step": lf / args.steps,
                            "achieved": fwd_ops / (ms_fwd / args.steps / 1e3) / 1e12,
                            "frac": fwd_ops / (ms_fwd / args.steps / 1e3) / 1e12 / peak_alu},
                "step_vs_plain_path": {
                    "ops_per_step": fwd_ops + adj_ops, "ms_per_step": ms_step,
                    "frac": (fwd_ops + adj_ops) / (ms_step / 1e3) / 1e12 / peak_alu,
                    "definition": "the plain FP32 method's work for one forward + recomputing adjoint "
                                  "(6 m_s + 12 lane-ops per amplitude) at the FP32 lane peak, over the whole "
                                  "step's time"}}
    kern = {k: {"launches": v[0], "ms": v[1]} for k, v in stats.items()}
    if args.precision > 0:
        roofline = tc_roofline(args, inst, geo, stats, ms_step, fwd_ops + adj_ops, peaks, peak_alu)
        roofline["vs_fp32"] = tc_against_fp32(args, inst, plan, psi, w, data, flush, ms_step, grad, grad_w, loss)

    # the same evaluation through qst_forward + qst_adjoint, whose adjoint
    # recomputes the rotations (the plain path's structure), for its roofline
    recompute = None
    if cached and not args.shard and not wide and args.precision == 0:
        def sep():
            plan.forward(psi, w, data, p_obs=p_obs, c_obs=c_obs, loss=loss)
            plan.adjoint(psi, w, data, c_obs, grad_psi=grad, grad_w=grad_w)
        for _ in range(2):
            flush.zero_()
            sep()
        torch.cuda.synchronize()
        plan.set_timing(True)
        plan.reset_stats()
        reps = max(3, min(args.steps, 10))
        for _ in range(reps):
            flush.zero_()
            sep()
        torch.cuda.synchronize()
        rs = plan.kernel_stats()
        plan.set_timing(False)
        r_adj = rs["adjoint"][1] / reps
        recompute = {"kernel": "k_adjoint_2r", "ops_per_launch": adj_ops, "ms_per_launch": r_adj,
                     "achieved": adj_ops / (r_adj / 1e3) / 1e12,
                     "frac": adj_ops / (r_adj / 1e3) / 1e12 / peak_alu,
                     "forward_ms": rs["forward"][1] / reps,
                     "ms_per_step": sum(v[1] for v in rs.values()) / reps,
                     "how": "qst_forward + qst_adjoint (the adjoint recomputes V_s psi_k), per-launch events, "
                            f"{reps} steps, L2 flushed between steps"}
        roofline["recompute_path"] = recompute

    # end to end through the host-buffer entry point (copies inside the timed region)
    e2e = None
    if not args.no_e2e and not args.shard:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
        h_psi = torch.from_numpy(inst.psi.view(np.float32)).pin_memory().numpy().view(np.complex64)
        h = [pin(inst.w), pin(inst.basis), pin(inst.row_ptr), pin(inst.outcome), pin(inst.count), pin(inst.shots)]
        outs = (torch.zeros(1, dtype=torch.float64).pin_memory().numpy(),
                torch.empty((K, 2 * D), dtype=torch.float32).pin_memory().numpy().view(np.complex64),
                torch.empty(K, dtype=torch.float32).pin_memory().numpy())
        for _ in range(max(1, min(args.warmup, 3))):
            plan.evaluate_host_buffers(h_psi, *h, out=outs, stream=stream.cuda_stream)
        if dist:
            dist.barrier()
        t_e2e = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan.evaluate_host_buffers(h_psi, *h, out=outs, stream=stream.cuda_stream)
            t_e2e += time.perf_counter() - t0
        t_e2e, _ = replicas.aggregate(t_e2e, amps_step, dist, device="cuda")
        h2d = h_psi.nbytes + sum(a.nbytes for a in h)
        d2h = outs[0].nbytes + outs[1].nbytes + outs[2].nbytes
        e2e = {"value": amps_all / (t_e2e / args.steps), "unit": "amplitudes/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": 1e3 * t_e2e / args.steps}

    # Algorithm 1 iterations on the device (qst_iterate: one CUDA graph, atom /
    # coefficient slots of the Table I schedule), timed with CUDA events
    algo = None
    if not args.no_iterations and not args.shard:
        it_T = args.iterations
        ip_psi, ip_w = psi.clone(), w.clone()
        Jh, acc = plan.iterate(it_T, 0, ip_psi, ip_w, data)  # capture + first run (untimed)
        ip_psi.copy_(psi)
        ip_w.copy_(w)
        torch.cuda.synchronize()
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.iterate(it_T, 0, ip_psi, ip_w, data, J_hist=Jh, accepted=acc)  # graph replay
        e1.record(stream)
        torch.cuda.synchronize()
        plan.check()
        ms_it, _ = replicas.aggregate(e0.elapsed_time(e1), 0, dist, device="cuda")
        jh = Jh.cpu().numpy()
        algo = {"s_per_iteration": ms_it / 1e3 / it_T, "iterations": it_T, "accepted": int(acc.sum().item()),
                "J_first": float(jh[0]), "J_last": float(jh[-1]),
                "how": "qst_iterate replay (one CUDA graph), Table I schedule (T_alpha = 5), step grid 2^-j, "
                       "from the bench state"}

    batched = None
    if ws == 1 and not args.no_batched and not args.shard:
        batched = batched_eval(flush, autotune=args.autotune)
    wide = None
    if ws == 1 and not args.no_wide and not args.shard and args.workload == WORKLOAD:
        wide = wide_eval(flush)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        done, t = cpu_oracle_rate(inst, args.cpu_seconds / 2)
        one = {"value": done * K * D / t, "unit": "amplitudes/s", "cores": 1, "kind": "oracle",
               "sample": f"first {done} of {M} settings of the workload, all {K} atoms, forward + adjoint, "
                         f"{t:.1f} s, single-threaded FP64 C"}
        S, t_all = cpu_oracle_rate_all_cores(inst, args.cpu_seconds / 2, one["value"], cores)
        cpu = {"value": S * K * D / t_all, "unit": "amplitudes/s", "cores": cores, "kind": "oracle",
               "sample": f"first {S} of {M} settings of the workload, all {K} atoms, forward + adjoint, "
                         f"{t_all:.1f} s, FP64 C with the settings sharded over {cores} host threads",
               "one_core": one}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "amplitudes/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "s_per_iteration": ms_step / 1e3,
                "higher_is_better": True, "scaling": "strong" if args.shard else "weak", "vs_baseline": None,
                "dtype": "f32",
                "data": "synthetic (seeded; Pauli strings uniform, Porter-Thomas surrogate counts)",
                "config": {"workload": args.workload, "n": n, "M": M, "K": K, "shots": int(inst.shots[0]),
                           "nnz": int(inst.nnz),
                           "precision_path": "plain FP32" if args.precision == 0 else
                           f"tensor cores: 6-qubit group products on tcgen05.mma kind::f16, the data split into "
                           f"{args.precision} BF16 term(s), operators exact in BF16, FP32 accumulation in TMEM",
                           "step": "qst_evaluate: forward (stores the chunk transforms at the observed outcomes) + "
                                   "adjoint (inverse rotations of c .* the stored transforms)" if cached else
                                   "qst_evaluate: forward + adjoint that recomputes the rotations",
                           "plan": {"reg_bits": args.reg_bits, "chunk_qubits": args.chunk_qubits,
                                    "max_bin_settings": args.max_bin_settings,
                                    "geometry": geo, "autotune": tuned},
                           "l2": "flushed between timed steps (512 MiB write outside the events)",
                           "parallelism": (f"setting shards over {ws} ranks + all-reduce of (loss, grad, grad_w)"
                                           if args.shard else ("replicas" if ws > 1 else "single GPU"))},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
                "algorithm1": algo, "batched": batched, "n20": wide,
                "gpu_launches": launches, "kernels": kern, "wall_ms_per_step": 1e3 * t_wall / args.steps,
                "workspace_bytes": plan.workspace_bytes()}
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
