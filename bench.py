"""Benchmark of the chi0 -> eps -> W hot path on GB300.

Workload: the medium synthetic workload (n_pb = 1500, 64 k-points x 40 occupied x 400
unoccupied = 1,024,000 transition columns, 12 imaginary frequencies, spin factor 2, Philox
inputs). One step = one pass of the whole path: reset, accumulate every k-point (prep +
tensor-core HERK), chi0 readout, eps, FP64 Cholesky inverse and W.

Metric: algorithmic chi0 TFLOP/s, F = 4 K n_pb (n_pb + 1) L per step, over the whole step time
(eps/W included), mixed precision (the default `--prec mixed`). The FP64 form is measured on a
2-k-point sample of the same Z (GB300 FP64 runs at ~1.2 TFLOP/s) and reported beside it.

The default line (one GPU) also carries, each timed on its own after the medium steps, the
largest configuration ("large": n_pb = 4000, 9.2M columns, 16 frequencies, one pass with Z drawn
per k-point on the device) and the batched one ("batched": 24 uneven q-points, q-points/s, tile
plan chosen by the library's autotuner).

`--impl reference` times the FP64 CPU oracle (test infrastructure) on a bounded sample of the
same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synthetic import MEDIUM, coulomb_v, eps_occ, eps_unocc  # noqa: E402

WL = MEDIUM
N_PB, N_K, N_OCC, N_UNOCC, L = WL.n_pb(0), WL.n_k, WL.n_occ, 400, WL.n_omega
K_COLS = N_K * N_OCC * N_UNOCC
F_STEP = 4.0 * K_COLS * N_PB * (N_PB + 1) * L
CONFIG_NAME = "medium chi0+W: n_pb=1500, n_k=64, n_occ=40, n_unocc=400 (K=1,024,000), 12 imaginary frequencies"


# DRAM traffic of one herk_mixed_kernel launch of this workload (one k-point), from the ncu
# capture summarised in profiles/herk_mixed_kernel_medium_one_kpoint.md; valid only for the kernel
# source it was measured on (sha1 prefix), otherwise reported as null.
TRAFFIC_BYTES_PER_LAUNCH = 13.866e9
TRAFFIC_KERNEL_SHA1 = "62b9657a5782"  # the capture ran on aa25a5064d66; this revision adds only the one-frequency prep


def measured_traffic():
    import hashlib
    src = os.path.join(ROOT, "paper_2506_03477_gb300", "csrc", "kernels_mixed.cu")
    try:
        h = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
    except OSError:
        return None
    return TRAFFIC_BYTES_PER_LAUNCH if h == TRAFFIC_KERNEL_SHA1 else None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("bf16_tflops_sustained", 1698.0), d.get("bf16_tflops", 1899.6), d.get("hbm_gbs", 6789.3), "measured"
    return 1700.0, 1900.0, 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # raw samples in the system's temporary directory; the JSON line carries their summary
        self.path = os.path.join(tempfile.gettempdir(), f"qsgw_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        under_load = [s for s, p in zip(sm, power) if p > 0.5 * max(power)] or sm
        return {"sm_mhz": statistics.median(under_load), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, dev_index):
    import torch
    from paper_2506_03477_gb300 import native as N

    torch.cuda.set_device(dev_index)
    dev = torch.device("cuda", dev_index)
    stream = torch.cuda.Stream(dev)
    gen_q = rank  # weak scaling: every rank assembles its own q-point
    prec = N.QSGW_MIXED_F16X3 if args.prec == "mixed" else N.QSGW_FP64

    # inputs resident in HBM (generated on the device, untimed). The mixed path holds Z as
    # complex64: it rounds every element to FP32 before forming digits, so this is bit-identical
    # to complex128 input and moves half the bytes. The FP64 path (and its 2-k-point sample in
    # the mixed run) uses complex128.
    ncol = N_OCC * N_UNOCC
    nk = args.k_points
    mixed = prec == N.QSGW_MIXED_F16X3
    Z = torch.empty((nk, ncol, N_PB), dtype=torch.complex64 if mixed else torch.complex128, device=dev)
    eo = torch.from_numpy(np.stack([eps_occ(WL.seed, gen_q, k, N_OCC) for k in range(N_K)])).to(dev)
    eu = torch.from_numpy(np.stack([eps_unocc(WL.seed, gen_q, k, N_UNOCC) for k in range(N_K)])).to(dev)
    v = torch.from_numpy(coulomb_v(WL.seed, gen_q, N_PB)).to(dev)
    Z128 = {}  # complex128 k-points kept for the FP64 sample
    with torch.cuda.stream(stream):
        for k in range(nk):
            zk = Z[k] if not mixed else torch.empty((ncol, N_PB), dtype=torch.complex128, device=dev)
            N.qsgw_synth_z(WL.seed, gen_q, k, N_PB, N_OCC, N_UNOCC, WL.s_div, zk, N_PB, stream=stream)
            if mixed:
                Z[k].copy_(zk)
                if k < 2 and not args.skip_fp64:
                    Z128[k] = zk
    accumulate = N.qsgw_chi0_accumulate_c64 if mixed else N.qsgw_chi0_accumulate
    chi = torch.empty((L, N_PB, N_PB), dtype=torch.complex128, device=dev)
    W = torch.empty_like(chi)
    torch.cuda.synchronize(dev)

    ctx = N.qsgw_chi0_init([N_PB], WL.omega, WL.spin, prec, stream=stream)
    acc_events = []

    def step(record=False):
        N.qsgw_chi0_reset(ctx, 0)
        for k in range(nk):
            if record:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            accumulate(ctx, 0, Z[k], N_PB, N_OCC, N_UNOCC, eo[k], eu[k], WL.omega)
            if record:
                e1.record(stream)
                acc_events.append((e0, e1))
        N.qsgw_chi0_finalize(ctx, 0, chi)
        N.qsgw_eps_inv(ctx, 0, v, W, n_omega=L)

    launches_per_step = nk * 3 + 1 + 2  # prep_cols, prep_rows, HERK per k; readout; eps + W kernels
    if prec == N.QSGW_FP64:
        launches_per_step = nk * 2 + 3

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    barrier(world)
    with ClockSampler(dev_index) as clk:
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        t0.record(stream)
        for _ in range(args.steps):
            step(record=True)
        t1.record(stream)
        torch.cuda.synchronize(dev)
    ms_total = t0.elapsed_time(t1)
    ms_step = ms_total / args.steps
    ms_step = max_over_ranks(ms_step, world)
    acc_ms = [a.elapsed_time(b) for a, b in acc_events]

    # FP64 form of the same path on a 2-k-point sample (TFLOP/s is intensive)
    fp64 = None
    if args.prec == "mixed" and not args.skip_fp64:
        ctx64 = N.qsgw_chi0_init([N_PB], WL.omega, WL.spin, N.QSGW_FP64, stream=stream)
        ks = [0, 1]
        for k in ks:  # warm-up
            N.qsgw_chi0_accumulate(ctx64, 0, Z128[k], N_PB, N_OCC, N_UNOCC, eo[k], eu[k], WL.omega)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for k in ks:
            N.qsgw_chi0_accumulate(ctx64, 0, Z128[k], N_PB, N_OCC, N_UNOCC, eo[k], eu[k], WL.omega)
        b.record(stream)
        torch.cuda.synchronize(dev)
        N.qsgw_chi0_destroy(ctx64)
        f_s = 4.0 * len(ks) * ncol * N_PB * (N_PB + 1) * L
        fp64_ms = a.elapsed_time(b)
        fp64 = {"tflops": f_s / (fp64_ms * 1e-3) / 1e12, "sample": f"chi0 accumulation of {len(ks)} of 64 k-points",
                "ms": fp64_ms}

    # end to end through the C ABI with host buffers (pinned): Z streamed in by the library
    e2e = None
    if not args.skip_e2e:
        Zh = torch.empty(Z.shape, dtype=Z.dtype, pin_memory=True)
        Zh.copy_(Z)
        eoh, euh = eo.cpu().numpy(), eu.cpu().numpy()
        chi_h = torch.empty(chi.shape, dtype=chi.dtype, pin_memory=True)
        W_h = torch.empty(W.shape, dtype=W.dtype, pin_memory=True)
        del Z
        Z128.clear()
        torch.cuda.empty_cache()

        def e2e_step():
            N.qsgw_chi0_reset(ctx, 0)
            for k in range(nk):
                accumulate(ctx, 0, Zh[k], N_PB, N_OCC, N_UNOCC, eoh[k], euh[k], WL.omega)
            N.qsgw_chi0_finalize(ctx, 0, chi)
            N.qsgw_eps_inv(ctx, 0, v, W, n_omega=L)
            with torch.cuda.stream(stream):
                chi_h.copy_(chi, non_blocking=True)
                W_h.copy_(W, non_blocking=True)
            stream.synchronize()

        e2e_step()
        # the box's own pinned host-to-device rate on one k-point slab (context for the e2e figure:
        # Z crosses the host link once per step, overlapped with the kernels)
        probe = torch.empty(Zh[0].shape, dtype=Zh.dtype, device=dev)
        pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            pa.record(stream)
            for _ in range(4):
                probe.copy_(Zh[0], non_blocking=True)
            pb.record(stream)
        stream.synchronize()
        h2d_gbs = 4 * Zh[0].numel() * Zh.element_size() / (pa.elapsed_time(pb) * 1e-3) / 1e9
        del probe
        barrier(world)
        t = time.perf_counter()
        n_e2e = max(1, min(args.steps, 3))
        for _ in range(n_e2e):
            e2e_step()
        e2e_s = (time.perf_counter() - t) / n_e2e
        e2e_s = max_over_ranks(e2e_s, world)
        h2d = Zh.numel() * Zh.element_size() + (eoh.size + euh.size) * 8
        d2h = 2 * chi.numel() * 16
        e2e = {"value": world * F_STEP * nk / N_K / e2e_s / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1e3, "h2d_gbs_measured": h2d_gbs}
    N.qsgw_chi0_destroy(ctx)

    res = dict(ms_step=ms_step, acc_ms=acc_ms, fp64=fp64, e2e=e2e, clocks=clk.summary(),
               launches=launches_per_step * args.steps, chi=chi)
    return res


# ------------------------------------------------------------------ batched uneven q-points
def run_batched(args, steps=None, warmup=None):
    """24 q-points, n_pb ~ U{900..2200}, 32 k-points with n_unocc ~ U{250..600} per (q, k), 12
    frequencies. Per k-point one qsgw_chi0_accumulate_batch call (24 blocks, one persistent launch,
    the tile plan chosen by qsgw_chi0_autotune on the first k-point's blocks before the warm-up);
    then eps/W for every q. The 24 x 32 blocks of Z (~320 GB) do not fit in HBM together, so each
    k-point's Z is drawn on the device before its batch call, outside the CUDA-event brackets that
    time the library calls. Returns the result as a dict."""
    import torch
    from paper_2506_03477_gb300 import native as N
    from synthetic import BATCHED as B

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    npb = [B.n_pb(q) for q in range(B.n_q)]
    nu = [[B.n_unocc(q, k) for k in range(B.n_k)] for q in range(B.n_q)]
    flops = B.flops()
    ctx = N.qsgw_chi0_init(npb, B.omega, B.spin, N.QSGW_MIXED_F16X3, stream=stream)
    Zq = [torch.empty((B.n_occ * 600, npb[q]), dtype=torch.complex128, device=dev) for q in range(B.n_q)]
    eo = [[torch.from_numpy(eps_occ(B.seed, q, k, B.n_occ)).to(dev) for k in range(B.n_k)] for q in range(B.n_q)]
    eu = [[torch.from_numpy(eps_unocc(B.seed, q, k, nu[q][k])).to(dev) for k in range(B.n_k)] for q in range(B.n_q)]
    vq = [torch.from_numpy(coulomb_v(B.seed, q, npb[q])).to(dev) for q in range(B.n_q)]
    Wq = [torch.empty((B.n_omega, npb[q], npb[q]), dtype=torch.complex128, device=dev) for q in range(B.n_q)]
    events = []
    steps = args.steps if steps is None else steps
    warmup = max(1, min(args.warmup, 1)) if warmup is None else warmup
    # autotune the tile plan on the first k-point's 24 blocks (scratch accumulators; not timed)
    for q in range(B.n_q):
        N.qsgw_synth_z(B.seed, q, 0, npb[q], B.n_occ, nu[q][0], B.s_div, Zq[q], npb[q], stream=stream)
    torch.cuda.synchronize(dev)
    t_tune = time.perf_counter()
    plan, plan_ms = N.qsgw_chi0_autotune(ctx, [(q, Zq[q], npb[q], B.n_occ, nu[q][0], eo[q][0], eu[q][0])
                                              for q in range(B.n_q)], reps=2)
    t_tune = time.perf_counter() - t_tune

    def step(record):
        for q in range(B.n_q):
            N.qsgw_chi0_reset(ctx, q)
        for k in range(B.n_k):
            for q in range(B.n_q):  # input generation, not timed
                N.qsgw_synth_z(B.seed, q, k, npb[q], B.n_occ, nu[q][k], B.s_div, Zq[q], npb[q], stream=stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            N.qsgw_chi0_accumulate_batch(ctx, [(q, Zq[q], npb[q], B.n_occ, nu[q][k], eo[q][k], eu[q][k])
                                               for q in range(B.n_q)])
            e1.record(stream)
            if record:
                events.append(("chi0", e0, e1))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for q in range(B.n_q):
            N.qsgw_eps_inv(ctx, q, vq[q], Wq[q], n_omega=B.n_omega)
        e1.record(stream)
        if record:
            events.append(("epsw", e0, e1))

    for _ in range(warmup):
        step(False)
    torch.cuda.synchronize(dev)
    with ClockSampler(0) as clk:
        for _ in range(steps):
            step(True)
        torch.cuda.synchronize(dev)
    N.qsgw_chi0_destroy(ctx)
    del Zq, Wq
    chi_ms = sum(a.elapsed_time(b) for n, a, b in events if n == "chi0") / steps
    w_ms = sum(a.elapsed_time(b) for n, a, b in events if n == "epsw") / steps
    step_ms = chi_ms + w_ms
    sustained = peaks()[0]
    issued = sum(issued_mma_flops(npb[q], B.n_omega, B.n_occ * nu[q][k], plan[0])
                 for q in range(B.n_q) for k in range(B.n_k))
    out = {"metric": "batched chi0+W: q-points/s (and algorithmic chi0 TFLOP/s)", "workload": B.name,
           "qpoints_per_s": B.n_q / (step_ms * 1e-3), "value": flops / (step_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
           "chi0_only_tflops": flops / (chi_ms * 1e-3) / 1e12, "ms_chi0_per_step": chi_ms, "ms_eps_w_per_step": w_ms,
           "steps": steps, "warmup": warmup, "flops_per_step": flops, "clocks": clk.summary(),
           "tile_plan": {"tile_cols": plan[0], "tail_pieces": plan[1], "ms_per_launch_in_tuning": plan_ms,
                         "tuning_s": t_tune},
           "roofline": {"bound": "tensor", "achieved": flops / (chi_ms * 1e-3) / 1e12, "peak": sustained,
                        "unit": "TFLOP/s", "frac": flops / (chi_ms * 1e-3) / 1e12 / sustained,
                        "tensor_pipe_issued_tflops": issued / (chi_ms * 1e-3) / 1e12,
                        "tensor_pipe_frac": issued / (chi_ms * 1e-3) / 1e12 / sustained},
           "note": "one persistent launch per k-point over all 24 q-points; Z drawn on the device between "
                   "the timed library calls (it does not fit in HBM at once)"}
    return out


def run_large(args):
    """The large streamed workload: n_pb = 4000, 64 k-points x 120 x 1200 (K = 9,216,000), 16
    frequencies (N = 256 per MMA). Z is drawn on the device per k-point inside
    qsgw_chi0_accumulate_synthetic (one call over all 64 k-points; the Philox draw writes and reads
    9.2 GB per k-point, ~0.4 % of the call), then eps/W for all 16 frequencies in FP64."""
    import torch
    from paper_2506_03477_gb300 import native as N
    from synthetic import LARGE as G

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    n, Lg, no, nu = G.n_pb(0), G.n_omega, G.n_occ, G.n_unocc_fixed
    k_cols = G.n_k * no * nu
    flops = 4.0 * k_cols * n * (n + 1) * Lg
    ctx = N.qsgw_chi0_init([n], G.omega, G.spin, N.QSGW_MIXED_F16X3, stream=stream)
    eo = torch.from_numpy(np.concatenate([eps_occ(G.seed, 0, k, no) for k in range(G.n_k)])).to(dev)
    eu = torch.from_numpy(np.concatenate([eps_unocc(G.seed, 0, k, nu) for k in range(G.n_k)])).to(dev)
    v = torch.from_numpy(coulomb_v(G.seed, 0, n)).to(dev)
    W = torch.empty((Lg, n, n), dtype=torch.complex128, device=dev)
    N.qsgw_chi0_accumulate_synthetic(ctx, 0, G.seed, 0, 0, 1, no, [nu], eo, eu, G.s_div)  # warm-up, 1 k-point
    N.qsgw_chi0_sync(ctx)
    N.qsgw_chi0_reset(ctx, 0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize(dev)
    with ClockSampler(0) as clk:
        ev[0].record(stream)
        N.qsgw_chi0_accumulate_synthetic(ctx, 0, G.seed, 0, 0, G.n_k, no, [nu] * G.n_k, eo, eu, G.s_div)
        ev[1].record(stream)
        N.qsgw_eps_inv(ctx, 0, v, W, n_omega=Lg)
        ev[2].record(stream)
        torch.cuda.synchronize(dev)
    N.qsgw_chi0_destroy(ctx)
    del W
    chi_ms, w_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    sustained = peaks()[0]
    issued = issued_mma_flops(n, Lg, no * nu) * G.n_k
    out = {"metric": "large streamed chi0 + W: algorithmic TFLOP/s", "workload": G.name,
           "value": flops / ((chi_ms + w_ms) * 1e-3) / 1e12, "unit": "TFLOP/s",
           "chi0_only_tflops": flops / (chi_ms * 1e-3) / 1e12,
           "ms_chi0": chi_ms, "ms_eps_w": w_ms, "flops": flops, "clocks": clk.summary(),
           "roofline": {"bound": "tensor", "achieved": flops / (chi_ms * 1e-3) / 1e12, "peak": sustained,
                        "unit": "TFLOP/s", "frac": flops / (chi_ms * 1e-3) / 1e12 / sustained,
                        "tensor_pipe_issued_tflops": issued / (chi_ms * 1e-3) / 1e12,
                        "tensor_pipe_frac": issued / (chi_ms * 1e-3) / 1e12 / sustained},
           "eps_inv_tflops": Lg * 4.0 * n ** 3 / (w_ms * 1e-3) / 1e12,
           "note": "one pass (64 k-points after a 1-k-point warm-up); Z drawn on the device inside the call; "
                   "eps_inv_tflops counts 4 n^3 real flops per frequency (Cholesky + inverse from the factor)"}
    return out


def run_sigx(args):
    """Exchange self-energy, Eq. (sigx), at the size of the paper's (InAs)6(GaSb)6 system (its
    Table 2): n_qp = 428 states, 16 k-points x 276 occupied x 3139 product-basis functions
    (K = 13,862,412 columns). Z resident in HBM as complex64 (47 GB; the mixed path rounds Z to
    FP32 anyway); the FP64 path is timed on a 1-k-point sample."""
    import torch
    from paper_2506_03477_gb300 import native as N

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    n_qp, n_pb, seed = 428, 3139, 1
    n_k, n_occ = min(16, args.k_points), args.sigx_occ  # smaller than 16 x 276 only as a profiling aid
    ncol = n_occ * n_pb
    flops = 4.0 * n_k * ncol * n_qp * (n_qp + 1)
    Z = torch.empty((n_k, ncol, n_qp), dtype=torch.complex64, device=dev)
    tmp = torch.empty((ncol, n_qp), dtype=torch.complex128, device=dev)
    v = [torch.from_numpy(coulomb_v(seed, k, n_pb)).to(dev) for k in range(n_k)]
    with torch.cuda.stream(stream):
        for k in range(n_k):
            N.qsgw_synth_z(seed, 7, k, n_qp, n_occ, n_pb, 100.0, tmp, n_qp, stream=stream)
            Z[k].copy_(tmp)
    torch.cuda.synchronize(dev)
    out = torch.empty((n_qp, n_qp), dtype=torch.complex128, device=dev)
    ctx = N.qsgw_sigx_init([n_qp], N.QSGW_MIXED_F16X3, stream=stream)

    def step():
        N.qsgw_chi0_reset(ctx, 0)
        for k in range(n_k):
            N.qsgw_sigx_accumulate_c64(ctx, 0, Z[k], n_qp, n_occ, n_pb, v[k])
        N.qsgw_chi0_finalize(ctx, 0, out)

    for _ in range(max(3, args.warmup)):
        step()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    with ClockSampler(0) as clk:
        a.record(stream)
        for _ in range(args.steps):
            step()
        b.record(stream)
        torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / args.steps
    N.qsgw_chi0_destroy(ctx)
    # FP64 sample: one k-point, complex128 Z
    ctx64 = N.qsgw_sigx_init([n_qp], N.QSGW_FP64, stream=stream)
    with torch.cuda.stream(stream):
        N.qsgw_synth_z(seed, 7, 0, n_qp, n_occ, n_pb, 100.0, tmp, n_qp, stream=stream)
    N.qsgw_sigx_accumulate(ctx64, 0, tmp, n_qp, n_occ, n_pb, v[0])  # warm-up
    N.qsgw_chi0_sync(ctx64)
    a.record(stream)
    N.qsgw_sigx_accumulate(ctx64, 0, tmp, n_qp, n_occ, n_pb, v[0])
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms64 = a.elapsed_time(b)
    N.qsgw_chi0_destroy(ctx64)
    f64 = 4.0 * ncol * n_qp * (n_qp + 1)
    issued = issued_mma_flops(n_qp, 1, ncol) * n_k
    sustained = peaks()[0]
    out_d = {"metric": "exchange self-energy Sigma^x (Eq. sigx): algorithmic TFLOP/s, mixed at <=1e-6",
             "workload": f"sigx n_qp=428, {n_k} k x {n_occ} occ x 3139 pb (K={n_k * ncol / 1e6:.2f}M)"
                         + (", (InAs)6(GaSb)6 sizes" if (n_k, n_occ) == (16, 276) else ", profiling case"),
             "value": flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms, "steps": args.steps,
             "flops_per_step": flops, "fp64_tflops": f64 / (ms64 * 1e-3) / 1e12,
             "mixed_over_fp64": (flops / ms) / (f64 / ms64), "clocks": clk.summary(),
             "roofline": {"bound": "tensor", "achieved": flops / (ms * 1e-3) / 1e12, "peak": sustained,
                          "unit": "TFLOP/s", "frac": flops / (ms * 1e-3) / 1e12 / sustained,
                          "tensor_pipe_issued_tflops": issued / (ms * 1e-3) / 1e12,
                          "tensor_pipe_frac": issued / (ms * 1e-3) / 1e12 / sustained},
             "note": "step = reset + 16 accumulate calls + readout; Z resident (complex64); FP64 on 1 k-point"}
    print(json.dumps(out_d))


def run_realaxis(args):
    """The real-axis route, Eqs. (impolf) and (hilbert), on the medium workload (n_pb = 1500, 64
    k-points x 40 x 400 columns): histogram spectral weights on the log mesh 0.04 * 1.03^j Ry
    (156 bins covering every Delta), then chi0 on the real axis at 12 bin centres. Z resident
    (complex128); one step = reset + 64 accumulate calls + readout of all S_j + real-axis chi0."""
    import torch
    from paper_2506_03477_gb300 import native as N

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    nk = min(args.k_points, N_K)
    ncol = N_OCC * N_UNOCC
    edges = 0.04 * 1.03 ** np.arange(0, 157)
    nb = edges.size - 1
    Z = torch.empty((nk, ncol, N_PB), dtype=torch.complex128, device=dev)
    eo = torch.from_numpy(np.stack([eps_occ(WL.seed, 0, k, N_OCC) for k in range(N_K)])).to(dev)
    eu = torch.from_numpy(np.stack([eps_unocc(WL.seed, 0, k, N_UNOCC) for k in range(N_K)])).to(dev)
    with torch.cuda.stream(stream):
        for k in range(nk):
            N.qsgw_synth_z(WL.seed, 0, k, N_PB, N_OCC, N_UNOCC, WL.s_div, Z[k], N_PB, stream=stream)
    torch.cuda.synchronize(dev)
    S = torch.empty((nb, N_PB, N_PB), dtype=torch.complex128, device=dev)
    bins_out = list(range(20, nb, 12))[:12]
    P = torch.empty((len(bins_out), N_PB, N_PB), dtype=torch.complex128, device=dev)
    ctx = N.qsgw_spectral_init(N_PB, edges, N.QSGW_MIXED_F16X3, stream=stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def step(record):
        for j in range(nb):
            N.qsgw_chi0_reset(ctx, j)
        if record:
            ev[0].record(stream)
        for k in range(nk):
            N.qsgw_spectral_accumulate(ctx, Z[k], N_PB, N_OCC, N_UNOCC, eo[k], eu[k])
        if record:
            ev[1].record(stream)
        N.qsgw_spectral_finalize(ctx, S)
        if record:
            ev[2].record(stream)
        N.qsgw_spectral_real_axis(ctx, S, bins_out, P)
        if record:
            ev[3].record(stream)

    for _ in range(max(1, min(args.warmup, 2))):
        step(False)
    torch.cuda.synchronize(dev)
    with ClockSampler(0) as clk:
        step(True)
        torch.cuda.synchronize(dev)
    N.qsgw_chi0_destroy(ctx)
    acc_ms, fin_ms, re_ms = (ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3]))
    flops = 4.0 * nk * ncol * N_PB * (N_PB + 1)  # every column enters exactly one bin
    # the FP64 form on 2 of the k-points (the FP64 HERK runs near 1 TFLOP/s)
    k64 = min(2, nk)
    ctx64 = N.qsgw_spectral_init(N_PB, edges, N.QSGW_FP64, stream=stream)
    e64 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e64[0].record(stream)
    for k in range(k64):
        N.qsgw_spectral_accumulate(ctx64, Z[k], N_PB, N_OCC, N_UNOCC, eo[k], eu[k])
    N.qsgw_spectral_finalize(ctx64, S)
    e64[1].record(stream)
    torch.cuda.synchronize(dev)
    N.qsgw_chi0_destroy(ctx64)
    fp64_tflops = 4.0 * k64 * ncol * N_PB * (N_PB + 1) / (e64[0].elapsed_time(e64[1]) * 1e-3) / 1e12
    out = {"metric": "real-axis chi0 (Eqs. impolf, hilbert): algorithmic TFLOP/s of the spectral weights S_j",
           "workload": f"medium n_pb={N_PB}, {nk} k x {ncol} columns, {nb} log bins, 12 real-axis outputs",
           "value": flops / ((acc_ms + fin_ms) * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_accumulate": acc_ms,
           "ms_finalize": fin_ms, "ms_real_axis": re_ms, "flops": flops, "clocks": clk.summary(),
           "fp64": {"value": fp64_tflops, "unit": "TFLOP/s", "sample": f"{k64} of {nk} k-points, all bins"},
           "mixed_over_fp64": flops / ((acc_ms + fin_ms) * 1e-3) / 1e12 / fp64_tflops,
           "note": "value counts the accumulate calls and the finalize (the flush of the last staged columns "
                   "and the readout of all S_j); per k-point: bin + stable counting sort + gather into per-bin "
                   "staging; bins are updated 32 per launch when their staging fills"}
    print(json.dumps(out))


def run_sigc(args):
    """The imaginary-axis correlation self-energy, Eq. (sigci), on the medium shapes. W^c(i omega_l)
    of one q-point comes from the library's own chain: chi0 of the medium workload (64 k-points),
    then eps^-1 and W^c (correlation only), 12 frequencies. I^c then runs for 64 target states and
    256 bands (40 occupied, 216 unoccupied) per k-point over 16 k-points, with Z drawn on the device
    (complex128, 6.3 GB resident) and the one W^c standing for every k. One step = reset + 16
    accumulate calls + readout. The FP64 path is timed on 64 bands of one k-point."""
    import torch
    from paper_2506_03477_gb300 import native as N

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    n_qp, n_band, n_k = 64, 256, min(16, args.k_points)
    om = np.asarray(WL.omega, dtype=np.float64)
    # W^c from chi0 -> eps^-1 -> W^c (set-up, not timed)
    ctxc = N.qsgw_chi0_init([N_PB], om, WL.spin, N.QSGW_MIXED_F16X3, stream=stream)
    tmp = torch.empty((N_OCC * N_UNOCC, N_PB), dtype=torch.complex128, device=dev)
    for k in range(N_K):
        eo = torch.from_numpy(eps_occ(WL.seed, 0, k, N_OCC)).to(dev)
        eu = torch.from_numpy(eps_unocc(WL.seed, 0, k, N_UNOCC)).to(dev)
        with torch.cuda.stream(stream):
            N.qsgw_synth_z(WL.seed, 0, k, N_PB, N_OCC, N_UNOCC, WL.s_div, tmp, N_PB, stream=stream)
        N.qsgw_chi0_accumulate(ctxc, 0, tmp, N_PB, N_OCC, N_UNOCC, eo, eu, om)
        N.qsgw_chi0_sync(ctxc)
    del tmp
    v = torch.from_numpy(coulomb_v(WL.seed, 0, N_PB)).to(dev)
    Wc = torch.empty((L, N_PB, N_PB), dtype=torch.complex128, device=dev)
    N.qsgw_eps_inv(ctxc, 0, v, Wc, correlation_only=True, n_omega=L)
    N.qsgw_chi0_destroy(ctxc)
    # inputs of I^c
    rng = np.random.default_rng(WL.seed)
    e_qp = torch.from_numpy(np.sort(rng.uniform(-0.3, 0.4, n_qp))).to(dev)
    e_band = [torch.from_numpy(np.concatenate([eps_occ(WL.seed, 1, k, 40), eps_unocc(WL.seed, 1, k, n_band - 40)]))
              .to(dev) for k in range(n_k)]
    Zs = torch.empty((n_k, n_band * n_qp, N_PB), dtype=torch.complex128, device=dev)
    with torch.cuda.stream(stream):
        for k in range(n_k):
            N.qsgw_synth_z(WL.seed, 5, k, N_PB, n_band, n_qp, WL.s_div, Zs[k], N_PB, stream=stream)
    torch.cuda.synchronize(dev)
    out = torch.empty((n_qp, n_qp), dtype=torch.complex128, device=dev)
    ctx = N.qsgw_sigc_init(n_qp, N_PB, om, N.QSGW_MIXED_F16X3, stream=stream)

    def step(nk, c, nb=n_band):
        N.qsgw_chi0_reset(c, 0)
        for k in range(nk):
            N.qsgw_sigc_accumulate(c, Zs[k], N_PB, nb, e_qp, e_band[k], Wc)
        N.qsgw_sigc_finalize(c, out)

    for _ in range(max(3, args.warmup)):
        step(n_k, ctx)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    with ClockSampler(0) as clk:
        a.record(stream)
        for _ in range(args.steps):
            step(n_k, ctx)
        b.record(stream)
        torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / args.steps
    N.qsgw_chi0_destroy(ctx)

    def flops(nk, nb):  # D = sum_i w_i conj(Z) W^c_i, then D Z^T; 8 real flops per complex MAC
        return nk * 8.0 * (nb * n_qp * N_PB * L * N_PB + n_qp * n_qp * nb * N_PB)

    ctx64 = N.qsgw_sigc_init(n_qp, N_PB, om, N.QSGW_FP64, stream=stream)
    step(1, ctx64, 64)  # warm-up
    a.record(stream)
    step(1, ctx64, 64)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms64 = a.elapsed_time(b)
    N.qsgw_chi0_destroy(ctx64)
    f = flops(n_k, n_band)
    sustained = peaks()[0]
    out_d = {"metric": "imaginary-axis correlation self-energy I^c (Eq. sigci): algorithmic TFLOP/s, mixed",
             "workload": f"sigc n_pb={N_PB}, {L} imaginary frequencies, n_qp={n_qp}, {n_k} k x {n_band} bands; "
                         "W^c from the medium chi0 -> eps^-1 chain",
             "value": f / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms, "flops_per_step": f,
             "fp64": {"value": flops(1, 64) / (ms64 * 1e-3) / 1e12, "unit": "TFLOP/s", "sample": "1 k-point, 64 bands"},
             "frac_of_bf16_sustained_x8": f / (ms * 1e-3) / 1e12 * 8 / sustained if sustained else None,
             "clocks": clk.summary(), "steps": args.steps}
    out_d["mixed_over_fp64"] = out_d["value"] / out_d["fp64"]["value"]
    print(json.dumps(out_d))


# ------------------------------------------------------------------ oracle (CPU) legs
def oracle_inputs(rows):
    """Rows of Z (host generator) and Delta for the sampled chi0 block."""
    import oracle
    from synthetic import z_rows

    ZS = z_rows(WL.seed, 0, rows, N_K, N_OCC, lambda k: N_UNOCC, WL.s_div)
    d = np.concatenate([oracle.delta(eps_occ(WL.seed, 0, k, N_OCC), eps_unocc(WL.seed, 0, k, N_UNOCC))[0]
                        for k in range(N_K)])
    return ZS, d


def oracle_block(ZS, d):
    """Time the FP64 oracle on chi0[rows, rows] over all 1,024,000 columns and 12 frequencies."""
    import oracle

    oracle.build()
    t = time.perf_counter()
    ref = oracle.chi0_rows(ZS, ZS, d, WL.omega, WL.spin)
    sec = time.perf_counter() - t
    flops = 8.0 * K_COLS * L * ZS.shape[0] * ZS.shape[0]
    return ref, sec, flops


def sample_rows(n):
    rng = np.random.default_rng(5)
    return np.unique(np.concatenate([[0, 1499], rng.choice(N_PB, n - 2, replace=False)]))[:n]


def cpu_baseline(chi_gpu=None, n_rows=48):
    rows = sample_rows(n_rows)
    ref, sec, flops = oracle_block(*oracle_inputs(rows))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"value": flops / sec / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
           "sample": f"FP64 oracle chi0 block {len(rows)}x{len(rows)} rows/cols x 1,024,000 columns x 12 frequencies "
                     f"({flops:.3g} algorithmic flops, {sec:.1f} s)"}
    if chi_gpu is not None:
        got = chi_gpu.cpu().numpy().transpose(0, 2, 1)[:, rows][:, :, rows]
        err = max(np.linalg.norm(got[l] - ref[l]) / np.linalg.norm(ref[l]) for l in range(L))
        out["check"] = {"chi0_block_rel_fro_max_over_omega": float(err)}
    return out


# ------------------------------------------------------------------ distributed helpers
_PG = None


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier(group=_PG)


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=_PG)
    return float(t.item())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--sigx-occ", type=int, default=276, help="occupied states per k-point for --workload sigx "
                    "(profiling aid; the workload uses 276)")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-extra", action="store_true", help="leave out the large and batched results of the "
                    "default line")
    ap.add_argument("--workload", default="medium",
                    choices=["medium", "batched", "large", "sigx", "realaxis", "sigc"],
                    help="medium = the benchmark line; batched = the 24-q uneven workload (q-points/s); "
                         "large = n_pb 4000, 9.2M columns, 16 frequencies (one pass); "
                         "sigx = the exchange self-energy at (InAs)6(GaSb)6 sizes; "
                         "realaxis = the histogram / Hilbert route on the medium shapes; "
                         "sigc = the imaginary-axis correlation self-energy on the medium shapes")
    ap.add_argument("--k-points", type=int, default=64,
                    help="k-points per step (profiling aid for small captures; bench lines use all 64)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    global _PG
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo", init_method="env://")
        _PG = dist.group.WORLD

    if args.impl == "reference":
        if rank != 0:
            return
        import oracle  # noqa: F401
        rows = sample_rows(24)
        ZS, d = oracle_inputs(rows)
        secs, flops = [], 0.0
        for _ in range(args.warmup):
            oracle_block(ZS, d)
        for _ in range(args.steps):
            _, s, flops = oracle_block(ZS, d)
            secs.append(s)
        sec = statistics.mean(secs)
        val = flops / sec / 1e12
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        sample = (f"FP64 oracle chi0 block {len(rows)}x{len(rows)} x 1,024,000 columns x 12 frequencies per step "
                  f"({flops:.3g} algorithmic flops)")
        print(json.dumps({"impl": "reference", "metric": metric_name(), "value": val, "unit": "TFLOP/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": config(args),
                          "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                                           "sample": sample},
                          "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    if args.workload in ("batched", "large", "sigx", "realaxis", "sigc"):
        if rank == 0:
            r = {"batched": run_batched, "large": run_large, "sigx": run_sigx, "realaxis": run_realaxis,
                 "sigc": run_sigc}[args.workload](args)
            if r is not None:
                print(json.dumps(r))
        return
    res = run_ours(args, rank, world, local)
    if rank != 0:
        return
    sustained, burst, hbm, src = peaks()
    f_step = F_STEP * args.k_points / N_K
    value = world * f_step / (res["ms_step"] * 1e-3) / 1e12
    acc = res["acc_ms"]
    acc_avg = statistics.mean(acc)
    f_launch = F_STEP / N_K
    achieved = f_launch / (acc_avg * 1e-3) / 1e12
    issued = issued_mma_flops_per_call() if args.prec == "mixed" else None
    roof = {"bound": "tensor" if args.prec == "mixed" else "alu", "kernel": "herk_mixed_kernel (+ prep kernels in the timed call)",
            "achieved": achieved, "peak": sustained, "unit": "TFLOP/s", "frac": achieved / sustained,
            "peak_source": f"{src} bf16 sustained", "traffic": measured_traffic() if args.prec == "mixed" else None,
            "note": "achieved = algorithmic chi0 flops per accumulate call / CUDA-event duration of the call"}
    if issued:
        roof["tensor_pipe_issued_tflops"] = issued / (acc_avg * 1e-3) / 1e12
        roof["tensor_pipe_frac"] = roof["tensor_pipe_issued_tflops"] / sustained
    out = {"metric": metric_name(), "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": res["ms_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f16x3-exact-digit" if args.prec == "mixed" else "f64", "data": "synthetic",
           "config": config(args), "roofline": roof, "gpu_launches": res["launches"], "clocks": res["clocks"],
           "e2e": res["e2e"]}
    if res["fp64"]:
        out["fp64"] = res["fp64"]
        out["mixed_over_fp64"] = achieved / res["fp64"]["tflops"]
    out["chi0_only_tflops"] = achieved
    out["ms_chi0_per_step"] = acc_avg * args.k_points
    out["ms_eps_w_per_step"] = res["ms_step"] - acc_avg * args.k_points
    if args.k_points != N_K:
        out["note"] = f"profiling case: {args.k_points} of {N_K} k-points per step (not a bench line)"
    if not args.skip_cpu and args.k_points == N_K:
        out["cpu_baseline"] = cpu_baseline(res["chi"])
    if world == 1 and not args.skip_extra and args.k_points == N_K:
        # the largest configuration and the batched one, each timed on its own after the medium line
        import torch
        del res
        torch.cuda.empty_cache()
        out["large"] = run_large(args)
        torch.cuda.empty_cache()
        out["batched"] = run_batched(args, steps=1, warmup=1)
    print(json.dumps(out))


def default_tile_width(n_pb, n_omega):
    """The library's default J columns per tile for one block: among the widths t with t * L a multiple
    of 16 and at most 256, from the widest down to 3/4 of it, the one whose J tiles overhang n_pb
    least (the wider on a tie)."""
    ok = [t for t in range(256 // n_omega, 0, -1) if (t * n_omega) % 16 == 0]
    t0 = ok[0]
    return min((t for t in ok if 4 * t >= 3 * t0), key=lambda t: (-(-n_pb // t) * t, -t))


def issued_mma_flops(n_pb, n_omega, k_cols, TJ=None):
    """FP16 MMA flops one accumulate call over k_cols columns issues (same tiling rules as the library;
    TJ = the tile plan's columns per tile, default the library's default width)."""
    if not TJ:
        TJ = default_tile_width(n_pb, n_omega)
    n = TJ * n_omega
    n_pad = (n_pb + 63) // 64 * 64
    n_it, n_jt = n_pad // 64, (n_pb + TJ - 1) // TJ
    tiles = sum(1 for it in range(n_it) for jt in range(n_jt) if jt * TJ + TJ - 1 >= it * 64 and it * 64 < n_pb)
    n_kb = (k_cols + 15) // 16  # 16-column K-blocks (the last chunk stops at the last column)
    return tiles * n_kb * 2 * 6 * (2.0 * 128 * n * 16)  # 2 K-steps x 6 digit products per K-block


def issued_mma_flops_per_call():
    return issued_mma_flops(N_PB, L, N_OCC * N_UNOCC)


def metric_name():
    return "chi0(q,iw) assembly TFLOP/s on 1 GB300: mixed vs FP64 at <=1e-6 rel. err"


def config(args):
    return {"workload": CONFIG_NAME, "precision": args.prec, "n_pb": N_PB, "K": K_COLS, "n_omega": L,
            "flops_per_step": F_STEP, "step": "reset + 64 accumulate calls + chi0 readout + eps + Cholesky inverse + W",
            "l2": ("inputs (12.3 GB of Z) larger than L2; no flush" if args.prec == "mixed"
                   else "inputs (24.6 GB of Z) larger than L2; no flush"), "parallelism": "replicas over q (weak)",
            "z_dtype": "complex64 (mixed: Z is rounded to FP32 before digits; bit-identical to complex128 input)"
            if args.prec == "mixed" else "complex128"}


if __name__ == "__main__":
    main()
