#!/usr/bin/env python
"""Benchmark of the overlap operator's hot path on GB300.

Metric: sgn(gamma5 D_w(mu)) b solves/s at 1e-8 relative error, the mixed
precision batched form (the headline) next to the FP64 form, the single-source
forms and Arnoldi, plus the Wilson stencil's bandwidth against the HBM roof.

Workload (one step = one batch): 12 Gaussian sources b on one 8^4 lattice
(N = 49152), SU(3) links U = exp(i eps H) with eps = 1.0, m_w = -1.5
(kappa = 0.2), mu = 0.3, antiperiodic time, the 20 eigenvalues of A nearest
the imaginary axis deflated (left/right eigenvectors from the library's GPU
eigensolver, set-up untimed); every source gives D_ov(mu) b = b + gamma5 sgn(A) b.
The Krylov size k is the smallest on a grid for which every source of the batch
agrees with a self-converged FP64 solve (k = 1000) to 1e-8.  Inputs are
resident in HBM when the timed region starts; L2 is flushed (a 512 MiB write)
before every timed step and each step is timed on the device with CUDA events.
A second batch, 12 point sources on each of 6^4, 8^4, 12^4 and 16^3 x 8
(mu = 0.2), is timed once as context.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: each rank solves its own batch on its own GPU
(replicas; the path has no data exchange), the max over ranks of the timed
device time sets the aggregate rate.  --impl reference times the FP64 CPU
oracle (scipy sparse matvec) on the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sgn(γ5Dw(μ))b solves/s at 1e-8 rel err, mixed vs FP64; Dw GB/s vs HBM peak"
DIMS = (8, 8, 8, 8)
EPS, SEED_U, SEED_B = 1.0, 1001, 2001
MU, KAPPA = 0.3, 0.2
K_GRID = list(range(300, 1001, 50))
K_REF = 1000
DW_DIMS = (48, 48, 48, 64)  # 7.1M sites: every stencil operand is far larger than L2
NRHS = 12
WORKLOAD = ("8^4 lattice (N=49152), SU(3) exp(i*1.0*H) links, m_w=-1.5, mu=0.3, batches of 12 Gaussian b, "
            "two-sided Lanczos, 20 eigenvalues of smallest |Re lambda| deflated")
MULTI_DIMS = [(6, 6, 6, 6), (8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 8)]
MULTI_MU, MULTI_K, MULTI_M = 0.2, 700, 20
# dram__bytes_read.sum + dram__bytes_write.sum of one k_b_regen launch (12 x 8^4 sequences), steady-state mean
REGEN_DRAM_BYTES_PER_LAUNCH = 30998400


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# FP64 ALU roof: 152 SMs x 2 FP64 FMA / clock / SM x 2 flop x 2.07 GHz = 1.259 TFLOP/s
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# algorithmic work per site: Wilson hopping term 1320 flop, diagonal and
# gamma5 48 flop; FP64 bytes: 4 links (576) + x (192) + y (192)
DW_FLOP_SITE = 1368
DW_BYTES = {"f64": 960, "f32_12": 384, "f32_18": 480}
# two-pass regeneration step (FP64): stencil + recurrence/accumulate epilogue of 12 complex
REGEN_FLOP_SITE = DW_FLOP_SITE + 12 * 30
REGEN_BYTES_SITE = 576 + 192 + 192 + 2 * 192 + 192
# fused FP32 pass-1 step (pair stencil + 2sL recurrence): 12-real links (192) + v_i, w_i (192) +
# v_{i-1}, w_{i-1} (192) + write v_{i+1}, w_{i+1} (192); t, s stay on chip
PASS1_BYTES_SITE = 768
# FP32 operations (add, multiply or fused multiply-add: one each) of one double-float regeneration
# step per site, counted from the arithmetic of df32.cuh in the kernel: per hop the projection
# (12 unnormalised double-float sums x 8), the link product (6 complex outputs x 134: one exact
# product of 4 operations and 11 compensated terms of 12, two renormalisations of 3), the
# coefficient (13 double-float products x 7); per output component the hop sum (16 x 8), the real
# 1/beta_i times a complex number (2 x 7), three complex double-float products (50 each) and three
# complex sums (22 each)
REGEN_DF_OPS_SITE = 8 * (12 * 8 + 6 * 134 + 13 * 7) + 12 * (16 * 8 + 2 * 7 + 3 * 50 + 3 * 22)
# FP32 issue rate: 152 SMs x 128 lanes x 2.07 GHz (one operation per lane and clock)
FP32_OPS_PEAK_T = 152 * 128 * 2.07e9 / 1e12
# FP64 pass-2 step: links (576) + v_i (192) + v_{i-1} (192) + v_{i+1} write (192) + y read/write (384)
PASS2_BYTES_SITE = 1536
M_DEFL = 20


def kernel_roofline(name, ms_per_launch, steps, V, hbm_peak):
    """Algorithmic work of one launch of a kernel class divided by its measured duration."""
    if name == "pass1_persistent":
        return {"bound": "hbm", "achieved": PASS1_BYTES_SITE * V * steps / ms_per_launch / 1e6, "peak": hbm_peak,
                "unit": "GB/s", "algorithmic": f"{PASS1_BYTES_SITE} B/site/step x {V} sites x {steps} steps"}
    if name == "pass2_persistent":
        return {"bound": "alu", "achieved": REGEN_FLOP_SITE * V * steps / ms_per_launch / 1e9,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "algorithmic": f"{REGEN_FLOP_SITE} FP64 flop/site/step x {V} sites x {steps} steps"}
    if name == "dslash_regen":
        return {"bound": "alu", "achieved": REGEN_FLOP_SITE * V / ms_per_launch / 1e9, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "algorithmic": f"{REGEN_FLOP_SITE} FP64 flop/site x {V} sites"}
    if name == "dslash_pair":
        return {"bound": "hbm", "achieved": (2 * 96 * 2 + 192) * V / ms_per_launch / 1e6, "peak": hbm_peak,
                "unit": "GB/s", "algorithmic": f"576 B/site x {V} sites"}
    return None


class Clocks:
    """nvidia-smi samples (200 ms) during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over the ranks of the job (the timing rule: the slowest replica sets the rate)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(total_ms_max: float, world: int, units_per_step: int, steps: int) -> float:
    """Units solved by all replicas per second of the slowest replica's timed device time."""
    return world * units_per_step * steps / (total_ms_max / 1e3)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def make_inputs(torch, n_src, rank):
    from paper_0810_4228_gb300 import synth
    U = synth.gauge_field(DIMS, EPS, SEED_U)
    srcs = synth.gaussian_source(DIMS, SEED_B + 7919 * rank, nrhs=n_src)
    return U, srcs


def calibrate_k(ovl, ctx, torch, b, flags_list, grid=None):
    """Smallest k on K_GRID whose solve agrees with the FP64 k=1000 solve to 1e-8; entries of
    flags_list are (name, flags) for two-sided Lanczos or (name, flags, method)."""
    ref, _ = ctx.sign_krylov(ovl.LANCZOS2, K_REF, MU, KAPPA, b)
    ref = ref.clone()
    nrm = torch.linalg.vector_norm(ref).item()
    out = {}
    for entry in flags_list:
        name, fl = entry[0], entry[1]
        method = entry[2] if len(entry) > 2 else ovl.LANCZOS2
        kg = grid or K_GRID
        chosen, err = kg[-1], None
        for k in kg:
            y, info = ctx.sign_krylov(method, k, MU, KAPPA, b, flags=fl)
            e = torch.linalg.vector_norm(y - ref).item() / nrm
            print(f"[bench] calibrate {name} k={k} err={e:.3e}", file=sys.stderr, flush=True)
            if e <= 1e-8:
                chosen, err = k, e
                break
            err = e
        out[name] = (chosen, err)
    return out


def time_solves(torch, ctx, fn, bufs, warmup, steps, flush):
    """Per-step device time (CUDA events on the library's stream), L2 flushed before each step."""
    st = torch.cuda.current_stream()
    times = []
    for i in range(warmup + steps):
        flush.fill_(i)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn(bufs[i % len(bufs)])
        e1.record(st)
        e1.synchronize()
        if i >= warmup:
            times.append(e0.elapsed_time(e1))
    return times


def dw_bandwidth(torch, ovl, reps=20, dims=DW_DIMS):
    """Stencil GB/s on a lattice far larger than L2 (device-layout vectors)."""
    from paper_0810_4228_gb300 import synth
    V = dims[0] * dims[1] * dims[2] * dims[3]
    ctx = ovl.Context(dims)
    U = synth.gauge_field_torch(dims, EPS, SEED_U, device="cuda")
    ctx.set_gauge(U)
    del U
    torch.cuda.empty_cache()
    res = {}
    st = torch.cuda.current_stream()
    for name, flag, prec in (("f32_12", ovl.F32, 1), ("f32_18", ovl.F32_FULL, 1), ("f64", 0, 0)):
        x = ctx.empty_native(prec)
        if prec == 1:
            x.copy_(torch.randn(ctx.n, dtype=torch.complex64, device="cuda"))
        else:
            x.copy_(torch.randn(ctx.n, dtype=torch.complex128, device="cuda"))
        y = ctx.empty_native(prec)
        for _ in range(3):
            ctx.apply_Dw(MU, KAPPA, x, y, flags=ovl.GAMMA5 | ovl.NATIVE | flag)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            ctx.apply_Dw(MU, KAPPA, x, y, flags=ovl.GAMMA5 | ovl.NATIVE | flag)
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"ms": ms, "GB_s": DW_BYTES[name] * V / ms / 1e6, "GFLOP_s": DW_FLOP_SITE * V / ms / 1e6}
        del x, y
    ctx.close()
    torch.cuda.empty_cache()
    return dims, V, res


def cpu_baseline(k: int, budget_s: float = 30.0):
    """The FP64 oracle's two-sided Lanczos on the same workload, single-threaded, in a child process."""
    code = f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r})
import numpy as np
from oracle import wilson as W, krylov as K
from paper_0810_4228_gb300 import synth
U = synth.gauge_field({DIMS!r}, {EPS}, {SEED_U})
b = synth.gaussian_source({DIMS!r}, {SEED_B})
A = W.a_operator(U, {DIMS!r}, {MU}, {KAPPA})
Ad = A.conj().T.tocsr()
t0 = time.perf_counter()
K.lanczos2(A.dot, Ad.dot, b / np.linalg.norm(b), b / np.linalg.norm(b), 20)
t20 = time.perf_counter() - t0
k = {k}
frac = min(1.0, {budget_s} / max(t20 * k / 20.0, 1e-9))
ks = max(20, int(k * frac))
t0 = time.perf_counter()
y = K.sign_lanczos2(A.dot, Ad.dot, b, ks)
t = time.perf_counter() - t0
print(json.dumps({{"t": t, "ks": ks, "k": k}}))
"""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    d = json.loads(r.stdout.strip().splitlines()[-1])
    per_solve = d["t"] * d["k"] / d["ks"]  # basis cost is linear in k; inner sign is small at this k
    return {"value": 1.0 / per_solve, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": (f"one FP64 oracle two-sided Lanczos solve with {d['ks']} of k={d['k']} steps "
                       f"(scipy CSR matvec + numpy, 1 thread) on the same 8^4 field and source, "
                       f"{d['t']:.1f} s, scaled by k/{d['ks']}")}


def run_reference(args, world, rank):
    if rank != 0:
        return
    k = args.k or 600
    t_all = []
    # each step is a bounded sample: a two-sided Lanczos run of the oracle
    budget = max(2.0, 200.0 / max(args.steps + args.warmup, 1))
    for i in range(args.warmup + args.steps):
        d = cpu_baseline(k, budget_s=budget)
        if i >= args.warmup:
            t_all.append(1.0 / d["value"])
    per = sum(t_all) / len(t_all)
    val = 1.0 / per
    line = {"metric": METRIC, "value": val, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "dims": list(DIMS), "mu": MU, "kappa": KAPPA, "eps": EPS, "k": k},
            "impl": "reference",
            "cpu_baseline": {"value": val, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": d["sample"]},
            "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def batch_launches(nseq, k, m, persistent_pass1=True):
    """Kernels one mixed batched solve launches: per sequence pack, state init, projections (two
    two-stage kernels), split, two FP32 conversions, the Newton fallback (two, they return at once
    when the quadrature settled), start vector, two and one double-float conversions, unpack; then
    pass 1 (one persistent launch, or pair + recurrence per step), the inner sign (prep, six levels
    of solve + sum) and k - 1 regeneration steps.  755 for 12 sequences, k = 550, m = 20 (the ncu
    launch list of one solve counts the same)."""
    per_seq = 1 + 1 + (4 if m > 0 else 0) + 1 + 2 + 2 + 1 + 2 + 1 + 1
    pass1 = 1 if persistent_pass1 else 2 * k - 1
    return nseq * per_seq + pass1 + 1 + 2 * 6 + (k - 1)


def calibrate_batch(torch, bt, srcs, refs, flags, grid):
    """Smallest k on the grid for which every source of the batch is within 1e-8 of its reference."""
    chosen, err = grid[-1], None
    for k in grid:
        outs, _, _ = bt.solve(k, MU, KAPPA, [srcs], flags=flags)
        e = max(torch.linalg.vector_norm(outs[0][r] - refs[r]).item() / torch.linalg.vector_norm(refs[r]).item()
                for r in range(refs.shape[0]))
        print(f"[bench] calibrate batch flags={flags} k={k} err={e:.3e}", file=sys.stderr, flush=True)
        err = e
        if e <= 1e-8:
            chosen = k
            break
    return chosen, err


# row a10: per site of ovl_dw_grad, algorithmic bytes (x 192 + g 192 read, the link force
# 36 complex = 576 written, the temporal link 144 read for d/dmu) and FP64 operations counted
# from the kernel (per direction two projections and 72 complex multiply-adds of the
# spin-traced colour outer products, about 780; the d/dmu term about 460)
DWGRAD_BYTES_SITE = 192 + 192 + 576 + 144
DWGRAD_FLOP_SITE = 4 * 780 + 460


def autograd_timing(torch, ovl, U_np, b, flush, k=800, gdims=(24, 24, 24, 24)):
    """Row a10 on the GPU.  ovl_sign_grad (derivatives of Re <g, sgn(A) b> with respect to the links,
    mu and b, resolvent form: one FP64 two-sided Lanczos process from (b, g)) on the 8^4 workload at
    k = 800 (where the 8^4 gradient test meets central differences to 1e-5), against the FP64
    forward solve at the same k; ovl_dw_grad (adjoint of y = A x: link force and d/dmu) on a lattice
    far larger than L2.  CUDA events on the library's stream around each call (each call ends with
    its own host synchronisation, included).  Failures are reported, not raised."""
    from paper_0810_4228_gb300 import synth
    out = {}

    def timed(fn, reps):
        st = torch.cuda.current_stream()
        ts = []
        for i in range(reps + 1):  # the first call warms up
            flush.fill_(i & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts[1:])

    try:
        lat = ovl.Context(DIMS)
        lat.set_gauge(torch.from_numpy(U_np).cuda())
        g = torch.from_numpy(synth.gaussian_source(DIMS, SEED_B + 600)).cuda()
        bb = b.clone()
        gU = torch.empty((lat.V, 4, 3, 3), dtype=torch.complex128, device="cuda")
        gb, y = torch.empty_like(bb), torch.empty_like(bb)
        t_grad = timed(lambda: lat.sign_grad(k, MU, KAPPA, bb, g, y=y, grad_U=gU, grad_b=gb), 3)
        t_fwd = timed(lambda: lat.sign_krylov(ovl.LANCZOS2, k, MU, KAPPA, bb, y), 3)
        out["sign_grad_8x4"] = {"k": k, "ms": round(t_grad, 3), "forward_fp64_ms": round(t_fwd, 3),
                                "ratio_to_forward": round(t_grad / t_fwd, 2),
                                "outputs": "sgn(A) b, grad_U, grad_mu, grad_b"}
        lat.close()
        del gU, gb, y, g, bb
    except Exception as exc:  # report, keep the rest of the line
        out["sign_grad_8x4"] = {"error": repr(exc)[:200]}
    try:
        V2 = gdims[0] * gdims[1] * gdims[2] * gdims[3]
        lat2 = ovl.Context(gdims)
        U2 = synth.gauge_field_torch(gdims, EPS, SEED_U + 7, device="cuda")
        lat2.set_gauge(U2)
        del U2
        x = torch.randn(V2 * 12, dtype=torch.complex128, device="cuda")
        gg = torch.randn(V2 * 12, dtype=torch.complex128, device="cuda")
        gU2 = torch.empty((V2, 4, 3, 3), dtype=torch.complex128, device="cuda")
        ms = timed(lambda: lat2.dw_grad(MU, KAPPA, x, gg, gU2), 10)
        out["dw_grad"] = {"dims": list(gdims), "sites": V2, "ms": round(ms, 4),
                          "GB_s": round(DWGRAD_BYTES_SITE * V2 / ms / 1e6, 1),
                          "GFLOP_s": round(DWGRAD_FLOP_SITE * V2 / ms / 1e6, 1),
                          "frac_fp64_roof": round(DWGRAD_FLOP_SITE * V2 / ms / 1e9 / FP64_PEAK_TFLOPS, 3),
                          "bytes_per_site": DWGRAD_BYTES_SITE, "flop_per_site": DWGRAD_FLOP_SITE,
                          "bound": "FP64 ALU (3.2 flop/B against 0.19 at the FP64 roof)"}
        lat2.close()
        del x, gg, gU2
        torch.cuda.empty_cache()
    except Exception as exc:  # report, keep the rest of the line
        out["dw_grad"] = {"error": repr(exc)[:200]}
    return out


def multi_lattice_batch(torch, ovl, flush):
    """12 point sources on each of four lattices of different sizes, 20 deflated eigenpairs each,
    mixed vs FP64, timed once."""
    from paper_0810_4228_gb300 import synth
    ctxs, srcs, setup = [], [], []
    for j, d in enumerate(MULTI_DIMS):
        c = ovl.Context(d)
        U = synth.gauge_field_torch(d, EPS, 1003 + j, device="cuda")
        c.set_gauge(U)
        del U
        t0 = time.perf_counter()
        e = c.deflation_eigs(MULTI_MU, KAPPA, MULTI_M)
        setup.append({"m": e["m"], "seconds": round(time.perf_counter() - t0, 2), "max_residual": e["max_residual"]})
        ctxs.append(c)
        srcs.append(torch.from_numpy(synth.point_sources(d, site=0)).cuda())
    bt = ovl.Batch(ctxs, [NRHS] * len(ctxs))
    res = {"lattices": [list(d) for d in MULTI_DIMS], "rhs_per_lattice": NRHS, "mu": MULTI_MU, "k": MULTI_K,
           "deflation": f"{MULTI_M} eigenpairs per lattice (library eigensolver, untimed)", "deflation_setup": setup,
           "sources": "12 spin-colour point sources at site 0"}
    for name, fl in (("mixed", ovl.MIXED), ("fp64", 0)):
        bt.solve(MULTI_K, MULTI_MU, KAPPA, srcs, flags=fl)
        t = time_solves(torch, None, lambda _: bt.solve(MULTI_K, MULTI_MU, KAPPA, srcs, flags=fl), [0], 1, 3, flush)
        ms = statistics.mean(t)
        res[name] = {"ms_per_batch": round(ms, 3), "solves_per_s": round(bt.nseq * 1e3 / ms, 2)}
    # accuracy of the mixed batch against single FP64 k = 1000 solves, one source per lattice
    outs, _, _ = bt.solve(MULTI_K, MULTI_MU, KAPPA, srcs, flags=ovl.MIXED)
    errs = []
    for j, c in enumerate(ctxs):
        ref, _ = c.sign_krylov(ovl.LANCZOS2, K_REF, MULTI_MU, KAPPA, srcs[j][5])
        errs.append(torch.linalg.vector_norm(outs[j][5] - ref).item() / torch.linalg.vector_norm(ref).item())
    res["mixed"]["max_rel_err_vs_k1000_fp64_sampled"] = max(errs)
    bt.close()
    for c in ctxs:
        c.close()
    torch.cuda.empty_cache()
    return res


def run_ours(args, world, rank, local):
    import torch
    from paper_0810_4228_gb300 import ovl, synth

    torch.cuda.set_device(local)
    if args.dw_only:
        ovl.load()
        dims = tuple(int(v) for v in args.dw_dims.split(",")) if args.dw_dims else DW_DIMS
        ddims, dV, dres = dw_bandwidth(torch, ovl, reps=args.steps, dims=dims)
        print(json.dumps({"dw_only": True, "dims": list(ddims), "sites": dV,
                          **{nm: {"ms": r["ms"], "GB_s": r["GB_s"]} for nm, r in dres.items()}}))
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    ovl.load()
    hbm_peak, peak_kind = peaks()
    U = synth.gauge_field(DIMS, EPS, SEED_U)
    srcs_np = synth.gaussian_source(DIMS, SEED_B + 7919 * rank, nrhs=NRHS)
    ctx = ovl.Context(DIMS)
    ctx.set_gauge(torch.from_numpy(U).cuda())
    srcs = torch.from_numpy(srcs_np).cuda()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    V = DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3]

    # ---- deflation set-up: the M_DEFL eigenpairs of A nearest the imaginary axis (untimed, once per field)
    eig = None
    if args.m > 0:
        t0 = time.perf_counter()
        eig = ctx.deflation_eigs(MU, KAPPA, args.m)
        eig["seconds"] = round(time.perf_counter() - t0, 2)
        print(f"[bench] deflation {eig}", file=sys.stderr, flush=True)

    bt = ovl.Batch([ctx], [NRHS])
    fl_mix = ovl.MIXED | ovl.OVERLAP
    fl_64 = ovl.OVERLAP
    # ---- accuracy calibration (untimed): every source against the FP64 k = 1000 solve
    if args.k:
        k_mix = k_64 = k_s = k_s64 = k_arn = k_adf = args.k
        err_mix = err_64 = err_s = err_s64 = err_arn = err_adf = None
    else:
        refs = torch.stack([ctx.sign_krylov(ovl.LANCZOS2, K_REF, MU, KAPPA, srcs[r])[0].clone() for r in range(NRHS)])
        k_mix, err_mix = calibrate_batch(torch, bt, srcs, refs, ovl.MIXED, K_GRID)
        k_64, err_64 = calibrate_batch(torch, bt, srcs, refs, 0, K_GRID)
        cal = calibrate_k(ovl, ctx, torch, srcs[0], [("mixed", ovl.MIXED), ("fp64", 0)])
        (k_s, err_s), (k_s64, err_s64) = cal["mixed"], cal["fp64"]
        # Arnoldi on its own k grid (step 25: it needs a smaller subspace, Sec. 5)
        cal_a = calibrate_k(ovl, ctx, torch, srcs[0], [("arnoldi", 0, ovl.ARNOLDI),
                                                       ("arnoldi_df", ovl.MIXED, ovl.ARNOLDI)],
                            grid=list(range(250, 801, 25)))
        (k_arn, err_arn), (k_adf, err_adf) = cal_a["arnoldi"], cal_a["arnoldi_df"]
    print(f"[bench] batch k mixed={k_mix} ({err_mix}), fp64={k_64} ({err_64}); single k mixed={k_s}, fp64={k_s64}",
          file=sys.stderr, flush=True)

    if args.solves_only:
        if not args.k:
            raise SystemExit("--solves-only needs --k")
        one_method = ovl.ARNOLDI if args.arnoldi else ovl.LANCZOS2
        one_flags = (ovl.OVERLAP | ovl.MIXED) if args.arnoldi else fl_mix
        if args.single or args.arnoldi:
            out1 = torch.empty_like(srcs[0])
            t = time_solves(torch, ctx, lambda b: ctx.sign_krylov(one_method, k_s, MU, KAPPA, b, out1, flags=one_flags),
                            [srcs[r] for r in range(NRHS)], args.warmup, args.steps, flush)
        else:
            t = time_solves(torch, ctx, lambda _: bt.solve(k_mix, MU, KAPPA, [srcs], [srcs.clone()], flags=fl_mix),
                            [0], args.warmup, args.steps, flush)
        if args.profile_one:
            # one more solve between cudaProfilerStart/Stop: `ncu --profile-from-start off` captures
            # exactly the launches of one solve (no effect without a profiler)
            torch.cuda.synchronize()
            torch.cuda.cudart().cudaProfilerStart()
            if args.single or args.arnoldi:
                ctx.sign_krylov(one_method, k_s, MU, KAPPA, srcs[0], out1, flags=one_flags)
            else:
                bt.solve(k_mix, MU, KAPPA, [srcs], [srcs.clone()], flags=fl_mix)
            torch.cuda.synchronize()
            torch.cuda.cudart().cudaProfilerStop()
        print(json.dumps({"solves_only": True, "single": args.single, "arnoldi_doublefloat": args.arnoldi, "k": k_mix,
                          "ms_per_step": statistics.mean(t)}))
        return

    outb = torch.empty_like(srcs)
    # ---- per-phase profile of the batched solve (CUDA events around each phase, eager launches)
    nprof = 3
    bt.profile(reset=True)
    for _ in range(nprof):
        _, pinfo, _ = bt.solve(k_mix, MU, KAPPA, [srcs], [outb], flags=fl_mix | ovl.PROFILE)
    prof, _ = bt.profile(reset=True)
    prof = {kk: v / nprof for kk, v in prof.items()}
    tuned = bt.tuning()
    kused = max(i["k_used"] for i in pinfo)
    print(f"[bench] batch profile {prof}", file=sys.stderr, flush=True)

    # ---- timed region: the mixed batched solve (headline), device-resident inputs
    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_mix = time_solves(torch, ctx, lambda _: bt.solve(k_mix, MU, KAPPA, [srcs], [outb], flags=fl_mix), [0],
                        args.warmup, args.steps, flush)
    torch.cuda.synchronize()
    clk = clocks.stop()
    tot = max_over_ranks(sum(t_mix), world, "cuda")
    if world > 1:
        torch.distributed.barrier()
    value = whole_job_rate(tot, world, NRHS, args.steps)
    print(f"[bench] batched mixed solves/s {value:.2f}, ms/step {statistics.mean(t_mix):.3f}, steps "
          f"{[round(t, 3) for t in t_mix]}", file=sys.stderr, flush=True)

    # ---- FP64 batched, single-source forms and Arnoldi (context, fewer steps)
    nctx = max(3, min(args.steps, 5))
    t_b64 = time_solves(torch, ctx, lambda _: bt.solve(k_64, MU, KAPPA, [srcs], [outb], flags=fl_64), [0], 2, nctx,
                        flush)
    out1 = torch.empty_like(srcs[0])
    bsingle = [srcs[r] for r in range(NRHS)]
    t_s = time_solves(torch, ctx, lambda b: ctx.sign_krylov(ovl.LANCZOS2, k_s, MU, KAPPA, b, out1, flags=fl_mix),
                      bsingle, 2, nctx, flush)
    t_s64 = time_solves(torch, ctx, lambda b: ctx.sign_krylov(ovl.LANCZOS2, k_s64, MU, KAPPA, b, out1, flags=fl_64),
                        bsingle, 2, nctx, flush)
    # the single-source mixed solve by kernel class (rows a1-a8; CUDA events around each class,
    # eager launches), and the optional re-projection of the deflated directions in pass 1 (row a4)
    single_profile, reproj = None, None
    try:
        ctx.profile(reset=True)
        ctx.sign_krylov(ovl.LANCZOS2, k_s, MU, KAPPA, srcs[0], out1, flags=fl_mix | ovl.PROFILE)
        torch.cuda.synchronize()
        single_profile = {kk: round(v["ms"], 4) for kk, v in ctx.profile(reset=True).items() if v.get("launches")}
    except Exception as exc:  # report, keep the rest of the line
        single_profile = {"error": repr(exc)[:200]}
    try:
        t_rp = time_solves(torch, ctx, lambda b: ctx.sign_krylov(ovl.LANCZOS2, k_s, MU, KAPPA, b, out1,
                                                                 flags=fl_mix | ovl.REPROJ), bsingle, 2, nctx, flush)
        reproj = {"k": k_s, "ms": round(statistics.mean(t_rp), 3),
                  "ms_without": round(statistics.mean(t_s), 3), "m": args.m}
        if not args.k:
            yr = ctx.sign_krylov(ovl.LANCZOS2, k_s, MU, KAPPA, srcs[0], flags=ovl.MIXED | ovl.REPROJ)[0]
            reproj["rel_err_vs_k1000_fp64"] = (torch.linalg.vector_norm(yr - refs[0]) /
                                               torch.linalg.vector_norm(refs[0])).item()
    except Exception as exc:  # report, keep the rest of the line
        reproj = {"error": repr(exc)[:200]}
    t_arn = time_solves(torch, ctx, lambda b: ctx.sign_krylov(ovl.ARNOLDI, k_arn, MU, KAPPA, b, out1,
                                                              flags=ovl.OVERLAP), bsingle, 1, 2, flush)
    t_adf = time_solves(torch, ctx, lambda b: ctx.sign_krylov(ovl.ARNOLDI, k_adf, MU, KAPPA, b, out1,
                                                              flags=ovl.OVERLAP | ovl.MIXED), bsingle, 2, nctx, flush)
    # the double-float Gram-Schmidt sweeps against HBM: 4 passes over v_0..v_j at step j, 16 B per
    # complex element (CUDA events around each sweep kernel, eager launches)
    ctx.profile(reset=True)
    ctx.sign_krylov(ovl.ARNOLDI, k_adf, MU, KAPPA, srcs[0], out1, flags=ovl.OVERLAP | ovl.MIXED | ovl.PROFILE)
    torch.cuda.synchronize()
    aprof = ctx.profile(reset=True)
    sweep_ms = sum(aprof.get(kk, {}).get("ms", 0.0) for kk in ("multidot", "multiaxpy"))
    sweep_bytes = 2 * k_adf * (k_adf + 1) * ctx.n * 16
    adf_sweeps = {"bytes_per_solve": sweep_bytes, "ms": round(sweep_ms, 3),
                  "GB_s": round(sweep_bytes / (sweep_ms * 1e6), 1) if sweep_ms else None,
                  "frac_hbm": round(sweep_bytes / (sweep_ms * 1e6) / hbm_peak, 3) if sweep_ms else None,
                  "inner_sign_ms": round(aprof.get("inner_sign", {}).get("ms", 0.0), 3),
                  "stencil_ms": round(aprof.get("dslash", {}).get("ms", 0.0), 3)}

    # ---- end to end through the C ABI with host buffers (copies inside the timed region)
    hsrc = srcs.cpu().pin_memory()
    hout = torch.empty_like(hsrc).pin_memory()
    t_e2e = time_solves(torch, ctx, lambda _: bt.solve(k_mix, MU, KAPPA, [hsrc], [hout], flags=fl_mix), [0],
                        args.warmup, args.steps, flush)
    e2e_val = whole_job_rate(max_over_ranks(sum(t_e2e), world, "cuda"), world, NRHS, args.steps)
    nbytes = srcs.numel() * srcs.element_size()

    # ---- roofline of the dominant phase of the batched solve
    steps2 = max(kused - 1, 1)
    roof_all = {
        "pass1_batched_fp32": {"bound": "hbm", "achieved": PASS1_BYTES_SITE * V * NRHS * kused / prof["pass1"] / 1e6,
                               "peak": hbm_peak, "unit": "GB/s",
                               "algorithmic": f"{PASS1_BYTES_SITE} B/site/step x {V} sites x {NRHS} rhs x {kused} steps",
                               "ms_per_launch_sequence": prof["pass1"]},
        "pass2_batched_doublefloat": {"bound": "alu",
                               "achieved": REGEN_DF_OPS_SITE * V * NRHS * steps2 / prof["pass2_or_combine"] / 1e9,
                               "peak": FP32_OPS_PEAK_T, "unit": "Top/s (FP32 operations)",
                               "algorithmic": f"{REGEN_DF_OPS_SITE} FP32 operations/site/step of the double-float arithmetic "
                                              f"x {V} sites x {NRHS} rhs x {steps2} steps",
                               "fp64_equivalent": {"achieved_tflops": REGEN_FLOP_SITE * V * NRHS * steps2 / prof["pass2_or_combine"] / 1e9,
                                                   "fp64_roof_tflops": FP64_PEAK_TFLOPS,
                                                   "note": f"{REGEN_FLOP_SITE} FP64 flop/site/step: the same step in native FP64"},
                               "ms_per_launch_sequence": prof["pass2_or_combine"]},
    }
    for r_ in roof_all.values():
        r_["frac"] = r_["achieved"] / r_["peak"]
    dname = "pass2_batched_doublefloat" if prof["pass2_or_combine"] >= prof["pass1"] else "pass1_batched_fp32"
    roof = dict(roof_all[dname])
    # DRAM bytes per launch of the dominant kernel from one ncu capture of the same kernel
    # (profiles/regen_dram_8x4_batch12.md); not measured for the pass-1 kernels
    traffic = REGEN_DRAM_BYTES_PER_LAUNCH if dname == "pass2_batched_doublefloat" and NRHS == 12 else None
    roof.update({"kernel": dname, "traffic": traffic,
                 "peak_kind": ("derived FP32 issue rate 152 SM x 128 lanes x 2.07 GHz" if roof["bound"] == "alu"
                               else f"{peak_kind} hbm_gbs")})

    multi = None
    if rank == 0 and not args.no_multi:
        try:
            multi = multi_lattice_batch(torch, ovl, flush)
        except Exception as exc:  # report, keep the headline measurement
            multi = {"error": repr(exc)[:200]}

    # ---- row a10: the gradients (sign function and stencil adjoint)
    grads = None
    if rank == 0 and not args.no_grad:
        try:
            grads = autograd_timing(torch, ovl, U, srcs[0], flush)
        except Exception as exc:  # report, keep the headline measurement
            grads = {"error": repr(exc)[:200]}

    # ---- stencil bandwidth on a lattice far larger than L2
    dw = None
    if rank == 0 and not args.no_dw:
        try:
            ddims, dV, dres = dw_bandwidth(torch, ovl)
        except Exception as exc:  # report, keep the solve measurement
            dres, ddims, dV = {}, DW_DIMS, 0
            dw = {"error": repr(exc)[:200]}
        dw = dw or {"dims": list(ddims), "sites": dV}
        for nm, r in dres.items():
            dw[nm] = {"ms": round(r["ms"], 4), "GB_s": round(r["GB_s"], 1), "frac_hbm": round(r["GB_s"] / hbm_peak, 3),
                      "GFLOP_s": round(r["GFLOP_s"], 1)}
            if nm == "f64":
                dw[nm]["frac_fp64_roof"] = round(r["GFLOP_s"] / (FP64_PEAK_TFLOPS * 1e3), 3)
        dw["hbm_peak_gbs"] = hbm_peak

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(k_mix)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(t_mix),
            "ms_per_step_median": statistics.median(t_mix), "ms_per_step_min": min(t_mix), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "dims": list(DIMS), "mu": MU, "kappa": KAPPA, "eps": EPS,
                       "rhs_per_step": NRHS,
                       "autotuned_shapes": {"pass1_sites_per_block": tuned[0], "regen_blocks_per_sm": tuned[1],
                                            "regen_sequences_per_block": tuned[2]}
                       if tuned else None,
                       "method": "batched two-sided Lanczos, two-pass mixed (FP32 pass 1, FP64 pass 2)",
                       "k": k_mix, "m_deflated": args.m, "deflation_setup": eig,
                       "max_rel_err_vs_k1000_fp64": err_mix,
                       "l2": "flushed (512 MiB write) before every timed step", "parallelism": f"replicas x{world}"},
            "roofline": roof,
            "roofline_phases": roof_all,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "solves/s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes},
            "gpu_launches": batch_launches(NRHS, k_mix, args.m) * args.steps,
            "clocks": clk,
            "fp64_batched": {"solves_per_s": NRHS * 1e3 / statistics.mean(t_b64), "ms_per_batch": statistics.mean(t_b64),
                             "k": k_64, "max_rel_err_vs_k1000_fp64": err_64},
            "mixed_single_source": {"solves_per_s": 1e3 / statistics.mean(t_s), "ms": statistics.mean(t_s), "k": k_s,
                                    "rel_err_vs_k1000_fp64": err_s, "kernels": "persistent passes",
                                    "profile_ms_by_kernel_class": single_profile,
                                    "with_reprojection": reproj},
            "fp64_single_source": {"solves_per_s": 1e3 / statistics.mean(t_s64), "ms": statistics.mean(t_s64),
                                   "k": k_s64, "rel_err_vs_k1000_fp64": err_s64},
            "arnoldi_fp64_single_source": {"solves_per_s": 1e3 / statistics.mean(t_arn), "ms": statistics.mean(t_arn),
                                           "k": k_arn, "rel_err_vs_k1000_fp64": err_arn,
                                           "k_ratio_2sl_over_arnoldi": (k_s64 / k_arn) if k_arn else None},
            "arnoldi_doublefloat_single_source": {"solves_per_s": 1e3 / statistics.mean(t_adf),
                                                  "ms": statistics.mean(t_adf), "k": k_adf,
                                                  "rel_err_vs_k1000_fp64": err_adf,
                                                  "gram_schmidt_sweeps": adf_sweeps},
            "profile_ms_per_batch": {kk: round(v, 4) for kk, v in prof.items()},
            "multi_lattice_batch": multi,
            "dw": dw,
            "autograd": grads,
        }
        print(json.dumps(line))
    bt.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--k", type=int, default=0, help="fix the Krylov size (skip the accuracy calibration)")
    ap.add_argument("--m", type=int, default=M_DEFL, help="deflated eigenpairs (0: none)")
    ap.add_argument("--no-dw", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-multi", action="store_true", help="skip the four-lattice point-source batch")
    ap.add_argument("--no-grad", action="store_true", help="skip the gradient timings")
    ap.add_argument("--single", action="store_true", help="with --solves-only: single-source solves instead of batches")
    ap.add_argument("--dw-only", action="store_true", help="only the stencil bandwidth measurement (--steps repetitions)")
    ap.add_argument("--dw-dims", default="", help="lattice of the stencil bandwidth measurement, e.g. 32,32,32,32")
    ap.add_argument("--arnoldi", action="store_true",
                    help="with --solves-only: single-source double-float Arnoldi solves (D_ov b) instead")
    ap.add_argument("--profile-one", action="store_true",
                    help="with --solves-only: one extra solve inside cudaProfilerStart/Stop (for ncu)")
    ap.add_argument("--solves-only", action="store_true",
                    help="only the timed solves (for profiler captures): needs --k, skips calibration, "
                         "profile, FP64/Arnoldi/e2e legs, the bandwidth lattice and the CPU baseline")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
