#!/usr/bin/env python
"""MG-GCR time-to-solution benchmark (one JSON line on rank 0).

Workload (the mixed-vs-FP64 configuration): an 8^3 x 16 lattice with a seeded
beta = 6.0 Wilson-action heatbath gauge field (200 sweeps, cold start),
Wilson mass swept over m_crit + {0.1, 0.03, 0.01, 0.003} (m_crit of this
field from tests/golden/mcrit.json), two-level adaptive MG with 4^4
aggregates and Nv = 20 null vectors, one Gaussian right-hand side, outer
flexible GCR(50) to a true FP64 relative residual of 1e-10.

One step = the whole hot path for the four masses: one mg_setup at the
lightest mass (null-vector relaxation, block Gram-Schmidt, Galerkin coarse
operator), one mg_retarget_batch to the four masses (the null space is mass
independent since D(m) = D(0) + m 1; coarse operators shifted, the four
coarsest inverses built in shared launches) and one mg_solve per mass, in the
chosen mixed-precision form
(FP16 fine smoother, FP32 Krylov, FP64 reliable updates / Gram-Schmidt /
coarsest refinement).  The
plain-FP64 form of the same step is timed beside it.  `value` is seconds
per step (lower is better) with the gauge field and sources resident on the
device; `e2e` is the same step through the C ABI with host buffers.

Also reported: dslash HBM bandwidth on a 32^3 x 64 lattice (working set
larger than L2) per storage precision, the roofline of the dominant kernel
(CUDA events around each of its launches inside a profiled step), SM clocks
sampled during the timed steps, and the FP64 CPU oracle timed on a bounded
sample (`cpu_baseline`).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0811_4331_gb300 import inputs  # noqa: E402

DIMS = (8, 8, 8, 16)
BETA, HB_SWEEPS, HB_SEED = 6.0, 200, 0
DMASSES = (0.1, 0.03, 0.01, 0.003)
NV, BLOCK, SETUP_SWEEPS = 20, (4, 4, 4, 4), 300
TOL = 1e-10
RHS_SEED = 1
BW_DIMS = (32, 32, 32, 64)
# no commas inside: a reader that splits the line's values at commas keeps the whole string
WORKLOAD = "8^3x16 beta=6.0 heatbath (200 sweeps; seed 0); 2-level MG 4^4 blocks Nv=20 (300 MR setup sweeps); " \
           "mass sweep m_crit + 0.1/0.03/0.01/0.003 (setup at the lightest; one batched retarget to all four); " \
           "1 Gaussian RHS; tol 1e-10"


def bench_config(args):
    """The step's configuration (the same dict in the library's line and the oracle's)."""
    return {"workload": WORKLOAD, "lattice": "8^3x16", "mg": "2 levels; 4^4 blocks; Nv=20",
            "masses": "m_crit + 0.1/0.03/0.01/0.003", "tol": 1e-10,
            "l2": "256 MB buffer written between timed steps (GPU)",
            "sweep": ("the four masses as concurrent handles (retarget batch + mg_solve_many)"
                      if args.sweep == "many" else "one solve with a mass per right-hand side (mg_solve_masses)"),
            "precision": "fine smoother FP16 storage / FP32 math; Krylov FP32; FP64 reliable updates / "
                         "Gram-Schmidt / coarsest solve (the oracle: FP64 throughout)"}


def mcrit():
    key = "%dx%dx%dx%d_beta%.1f_sweeps%d_seed%d" % (*DIMS, BETA, HB_SWEEPS, HB_SEED)
    with open(os.path.join(ROOT, "tests", "golden", "mcrit.json")) as f:
        return json.load(f)[key]["m_crit"]


def make_inputs():
    U = inputs.heatbath_gauge(DIMS, BETA, HB_SWEEPS, HB_SEED)
    b = inputs.gaussian_spinor(DIMS, RHS_SEED)
    return U, b


def params(wm, mixed, smoother=0):
    return wm.mg_default_params(n_levels=2, block=[BLOCK], nv=[NV], setup_sweeps=[SETUP_SWEEPS], mixed=mixed,
                                fine_prec=wm.MG_F16, seed=7, fine_smoother=smoother)


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------- ranks
def max_over_ranks(times, world, device):
    """Per-step times, each the maximum over the ranks of the process group (the slowest replica
    bounds the job); `device` is where the reduction runs ("cuda" under NCCL, "cpu" under gloo)."""
    t = np.asarray(times, dtype=np.float64)
    if world <= 1:
        return t
    import torch
    tt = torch.tensor(t, device=device)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
    return tt.cpu().numpy()


# ---------------------------------------------------------------------------- native arm
def native(args, rank, world, U, b):
    import torch
    from paper_0811_4331_gb300 import wilson_mg as wm

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    mc = mcrit()
    masses = [mc + d for d in DMASSES]
    Ud = torch.from_numpy(U).cuda()
    bd = torch.from_numpy(b).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > L2
    solve_streams = [torch.cuda.Stream() for _ in DMASSES]

    def step(mixed, host=False, stats_out=None, smoother=0):
        """One mass sweep: null-vector setup once at the lightest mass, every other mass
        through mg_retarget (same eigenvectors: D(m) = D(0) + m 1), one solve per mass."""
        p = params(wm, mixed, smoother)
        p.defer_coarsest = 1  # the four coarsest inverses are built together by the batched retarget
        base = wm.mg_setup(U if host else Ud, DIMS, masses[-1], p, stream=stream)
        if args.sweep == "masses" and smoother == 0:  # one solve, a mass per right-hand side
            B4 = np.stack([b] * len(masses)) if host else torch.stack([bd] * len(masses))
            X4 = np.zeros_like(B4) if host else torch.zeros_like(B4)
            _, sts = wm.mg_solve_masses(base, masses, B4, X4, TOL, stream=stream)
            if stats_out is not None:
                for r, m in enumerate(masses):
                    stats_out.append((m, sts[r], X4[r] if host else X4[r].cpu().numpy()))
            wm.mg_destroy(base)
            return
        hs = wm.mg_retarget_batch(base, masses, stream=stream)
        # the four solves side by side, one host thread and stream each
        if host:
            bs = [b] * len(masses)
            xs = [np.zeros_like(b) for _ in masses]
        else:
            bs = [bd] * len(masses)
            xs = [torch.zeros_like(bd) for _ in masses]
            for q in solve_streams:
                q.wait_stream(stream)
        _, sts = wm.mg_solve_many(hs, bs, xs, TOL, streams=solve_streams)
        for m, h, x, st in zip(masses, hs, xs, sts):
            if stats_out is not None:
                stats_out.append((m, st[0], x if host else x.cpu().numpy()))
            wm.mg_destroy(h)
        wm.mg_destroy(base)

    launches = [0]  # library kernel launches inside the timed steps of the last timed() call

    def timed(mixed, K, W, host=False, smoother=0):
        for _ in range(W):
            step(mixed, host, smoother=smoother)
        times = []
        n0 = wm.mg_launch_count()
        for _ in range(K):
            flush.zero_()
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(mixed, host, smoother=smoother)
            e1.record(stream)
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            times.append(e0.elapsed_time(e1) / 1e3)
        launches[0] = wm.mg_launch_count() - n0
        return max_over_ranks(times, world, "cuda")

    clk = ClockSampler(dev)
    if not args.ncu:
        clk.start()
    t_mixed = timed(1, args.steps, args.warmup)
    n_launch = launches[0]
    clocks = clk.stop()
    res = {"mixed_s": t_mixed.tolist()}
    if args.only_timed:
        return {"value": float(np.median(t_mixed)), "mixed_s": res["mixed_s"], "clocks": clocks}
    # correctness of the timed form: the true FP64 residual the library recomputes at exit
    chk = []
    step(1, stats_out=chk)
    per_mass = []
    for m, st, x in chk:
        rel = float(st["true_rel_residual"])
        per_mass.append({"dm": round(m - mc, 4), "iters": st["iters"], "fine_dslash": st["fine_dslash"],
                         "fine_dslash_f64": st["fine_dslash_f64"], "true_rel_residual": rel})
        assert rel <= TOL * 1.0001, ("mixed solve missed the tolerance", m, rel)
    out = {"per_mass_mixed": per_mass}
    # plain FP64 beside it
    if not args.no_plain:
        t_plain = timed(0, max(1, min(args.steps, 2)), 1)
        chk = []
        step(0, stats_out=chk)
        out["fp64_plain"] = {"value": float(np.median(t_plain)), "unit": "s per 4-mass sweep",
                             "per_mass": [{"dm": round(m - mc, 4), "iters": st["iters"],
                                           "fine_dslash": st["fine_dslash"],
                                           "true_rel_residual": st["true_rel_residual"]} for m, st, _ in chk]}
        out["speedup_mixed_vs_fp64"] = float(np.median(t_plain) / np.median(t_mixed))
        out["fp64_plain_s"] = float(np.median(t_plain))
        # plain FP64 MG with the adaptive setup of Sec. 2 (16 of the 20 candidates from two adaptive
        # steps of 64 solver iterations), for the operator-application count against BiCGstab
        pa = wm.mg_default_params(n_levels=2, block=[BLOCK], nv=[NV], setup_sweeps=[SETUP_SWEEPS], mixed=0, seed=7,
                                  adapt_steps=2, adapt_nv=[16], adapt_cycles=64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ha = wm.mg_setup(Ud, DIMS, masses[-1], pa, stream=stream)
        pm = []
        for m in masses:
            hm = wm.mg_retarget(ha, m, stream=stream)
            x = torch.zeros_like(bd)
            _, st = wm.mg_solve(hm, bd, x, TOL, stream=stream)
            pm.append({"dm": round(m - mc, 4), "iters": st[0]["iters"], "fine_dslash": st[0]["fine_dslash"],
                       "true_rel_residual": st[0]["true_rel_residual"]})
            wm.mg_destroy(hm)
        wm.mg_destroy(ha)
        torch.cuda.synchronize()
        out["fp64_adaptive"] = {"value": round(time.perf_counter() - t0, 4), "unit": "s per 4-mass sweep (setup + "
                                "four solves one after another)", "per_mass": pm}
    # the same mixed step with the even-odd fine smoother (MR on the Schur complement; not in the paper)
    if not args.no_plain:
        t_eo = timed(1, max(1, min(args.steps, 3)), 1, smoother=1)
        chk = []
        step(1, stats_out=chk, smoother=1)
        pm = []
        for m, st, x in chk:
            rel = float(st["true_rel_residual"])
            assert rel <= TOL * 1.0001, ("even-odd smoother solve missed the tolerance", m, rel)
            pm.append({"dm": round(m - mc, 4), "iters": st["iters"], "fine_dslash": st["fine_dslash"],
                       "true_rel_residual": rel})
        out["mixed_eo_smoother"] = {"value": float(np.median(t_eo)), "unit": "s per 4-mass sweep", "per_mass": pm,
                                    # mg_solve_masses needs the MR fine smoother, so this row always runs
                                    # the masses as concurrent handles
                                    "sweep": "concurrent handles (retarget batch + mg_solve_many)"}
    # the unpreconditioned baseline the paper compares against (Secs. 4-5): FP64 BiCGstab per mass, on the
    # full system and on its even-odd Schur complement
    if not args.no_plain:
        hk = wm.mg_setup(Ud, DIMS, masses[0], wm.mg_default_params(n_levels=1), stream=stream)
        for key, method in (("bicgstab_fp64", wm.MG_KRYLOV_BICGSTAB), ("bicgstab_eo_fp64", wm.MG_KRYLOV_BICGSTAB_EO)):
            kb = []
            for m in masses:
                hm = wm.mg_retarget(hk, m, stream=stream)
                x = torch.zeros_like(bd)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                status, st = wm.krylov_solve(hm, method, bd, x, TOL, max_iter=40000, stream=stream,
                                             raise_on_noconv=False)
                torch.cuda.synchronize()
                kb.append({"dm": round(m - mc, 4), "iters": st[0]["iters"], "fine_dslash": st[0]["fine_dslash"],
                           "seconds": round(time.perf_counter() - t0, 4), "converged": status == wm.MG_OK,
                           "true_rel_residual": st[0]["true_rel_residual"]})
                wm.mg_destroy(hm)
            out[key] = kb
        wm.mg_destroy(hk)
        # the paper's comparison (Sec. 5): fine-operator applications of BiCGstab over those of plain
        # FP64 MG-GCR, per mass, and the time of each FP64 solve (MG: its share of the sweep)
        if "fp64_plain" in out:
            out["bicgstab_over_mg_fine_dslash"] = [
                {"dm": a["dm"], "ratio": round(b_["fine_dslash"] / a["fine_dslash"], 2),
                 "ratio_eo": round(c["fine_dslash"] / a["fine_dslash"], 2),
                 "ratio_adaptive_mg": round(b_["fine_dslash"] / d["fine_dslash"], 2)}
                for a, b_, c, d in zip(out["fp64_plain"]["per_mass"], out["bicgstab_fp64"], out["bicgstab_eo_fp64"],
                                       out["fp64_adaptive"]["per_mass"])]
    # end to end through the C ABI with host buffers
    t_e2e = timed(1, max(1, min(args.steps, 3)), 1, host=True)
    V = int(np.prod(DIMS))
    h2d = U.nbytes + len(masses) * 2 * b.nbytes
    d2h = len(masses) * b.nbytes
    out["e2e"] = {"value": float(np.median(t_e2e)), "unit": "s per 4-mass sweep", "h2d_bytes_per_step": h2d,
                  "d2h_bytes_per_step": d2h}
    # roofline of the dominant kernel, from events around each of its launches in one profiled step
    out["roofline"], out["kernel_shares"] = profiled_step(wm, torch, Ud, bd, masses, stream)
    out["clocks"] = clocks
    out["mixed_s"] = res["mixed_s"]
    out["value"] = float(np.median(t_mixed))
    # library kernel launches inside the K timed steps (a graph replay counts its kernel nodes)
    out["gpu_launches"] = int(n_launch)
    if not args.no_dslash_hbm and rank == 0:
        out["dslash_hbm"] = dslash_bandwidth(wm, torch, stream)
    return out


def class_profile(wm, handles_run, peaks):
    """Run `handles_run(collect)` with the per-launch event profiler on every kernel class;
    return {(class, prec): [launches, ms, algorithmic bytes]}."""
    tot = {}

    def collect(h):
        for k, nm in enumerate(wm.KERNEL_CLASS_NAMES):
            for prec in range(4):
                n, ms = wm.mg_profile_read(h, k, prec)
                if n:
                    nb = wm.mg_profile_bytes(h, k, prec)
                    a = tot.get((nm, prec), [0, 0.0, 0.0])
                    tot[(nm, prec)] = [a[0] + n, a[1] + ms, a[2] + nb]

    wm.mg_profile(None, (1 << len(wm.KERNEL_CLASS_NAMES)) - 1)
    try:
        handles_run(collect)
    finally:
        wm.mg_profile(None, 0)
    return tot


PREC_NAMES = ["f64", "f32", "f16", "bf16"]


# DRAM bytes per launch (dram__bytes read + write, cold cache) of this step's kernels, from one ncu capture
# (profiles/dslash_small_f16_c2_step.md); valid while those kernels stay as captured.
C2_TRAFFIC = {("dslash", 2): 1232000}


def shares_and_roofline(tot, peaks, galerkin_flops=None, inverse_n=None, traffic=None):
    """Device-time share of every class and the roofline of the dominant one: achieved =
    algorithmic bytes (each operand once per launch) / summed CUDA-event time of its launches.
    traffic: {(class, precision): DRAM bytes per launch from an ncu capture of this workload}."""
    all_ms = sum(v[1] for v in tot.values())
    hbm = peaks.get("hbm_gbs")
    shares = {}
    for k, v in sorted(tot.items(), key=lambda kv: -kv[1][1]):
        e = {"launches": v[0], "ms": round(v[1], 4), "share": round(v[1] / all_ms, 4)}
        if v[2] > 0:
            e["algorithmic_GB"] = round(v[2] / 1e9, 4)
            e["achieved_GBs"] = round(v[2] / (v[1] / 1e3) / 1e9, 1)
        shares["%s/%s" % (k[0], PREC_NAMES[k[1]])] = e
    (top, tprec), (n, ms, nb) = max(tot.items(), key=lambda kv: kv[1][1])
    avg_s = ms / 1e3 / max(n, 1)
    roof = {"kernel": "%s/%s" % (top, PREC_NAMES[tprec]), "launches": n, "avg_us": round(avg_s * 1e6, 3),
            "traffic": (traffic or {}).get((top, tprec))}
    if nb > 0:
        ach = nb / n / avg_s / 1e9
        roof.update(bound="hbm", achieved=round(ach, 1), peak=hbm, unit="GB/s", frac=round(ach / hbm, 4),
                    algorithmic="%.4g B per launch (mean over %d launches; each operand once per launch)" % (nb / n, n))
    elif top == "galerkin" and galerkin_flops:
        ach = galerkin_flops / avg_s / 1e12
        roof.update(bound="alu", achieved=round(ach, 3), peak=1.196, unit="TFLOP/s (FP64)",
                    frac=round(ach / 1.196, 4), algorithmic="%.3g FP64 flop per launch" % galerkin_flops)
    elif top == "inverse" and inverse_n:
        fl = 8.0 * inverse_n ** 3
        pk = 74.6 if tprec == 1 else 1.196
        ach = fl / avg_s / 1e12
        roof.update(bound="alu", achieved=round(ach, 3), peak=pk, unit="TFLOP/s", frac=round(ach / pk, 4),
                    algorithmic="Gauss-Jordan, 8 N^3 flop, N = %d" % inverse_n)
    else:
        roof.update(bound="latency", achieved=None, peak=None, unit=None, frac=None)
    return roof, shares


def profiled_step(wm, torch, Ud, bd, masses, stream):
    """One extra step (setup + solve per mass) with the per-launch event profiler on every kernel class.

    Returns the roofline of the dominant class and the device-time share of every class.
    """
    p = params(wm, 1)
    peaks = measured_peaks()

    def run(collect):
        p.defer_coarsest = 1
        base = wm.mg_setup(Ud, DIMS, masses[-1], p, stream=stream)
        hs = dict(zip(masses, wm.mg_retarget_batch(base, masses, stream=stream)))
        for m in masses:
            h = hs.pop(m)
            x = torch.zeros_like(bd)
            wm.mg_solve(h, bd, x, TOL, stream=stream)
            collect(h)
            wm.mg_destroy(h)
        collect(base)
        wm.mg_destroy(base)

    tot = class_profile(wm, run, peaks)
    V = int(np.prod(DIMS))
    bs = int(np.prod(BLOCK))
    gal = 9 * (bs * 170 + 2 * NV * 6 * bs * 8) * (V // bs) * 2 * NV
    return shares_and_roofline(tot, peaks, galerkin_flops=gal, inverse_n=2 * NV * (V // bs), traffic=C2_TRAFFIC)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


def dslash_bandwidth(wm, torch, stream, dims=BW_DIMS, precs=None):
    """Achieved GB/s of dslash_apply on 32^3 x 64 (inputs + links + output > L2) per storage precision."""
    U = inputs.random_gauge_fast(dims, 5)
    Ud = torch.from_numpy(U).cuda()
    del U
    V = int(np.prod(dims))
    peak = measured_peaks().get("hbm_gbs", 6800.0)
    out = {"dims": list(dims), "peak_gbs": peak}
    # algorithmic bytes per site: spinor in + out (24 complex) + 4 stored links per site
    per_site = {wm.MG_F64: 24 * 16 + 4 * 9 * 16, wm.MG_F32: 24 * 8 + 4 * 6 * 8,
                wm.MG_F16: 24 * 4 + 4 * 6 * 4, wm.MG_BF16: 24 * 4 + 4 * 6 * 4}
    flops_site = 1320 + 48
    for prec, name in ((wm.MG_F16, "f16"), (wm.MG_BF16, "bf16"), (wm.MG_F32, "f32"), (wm.MG_F64, "f64")):
        if precs is not None and name not in precs:
            continue
        p = wm.mg_default_params(n_levels=1, mixed=0 if prec == wm.MG_F64 else 1,
                                 fine_prec=prec if prec != wm.MG_F64 else wm.MG_F16)
        h = wm.mg_setup(Ud, dims, -0.79, p, stream=stream)
        a = wm.internal_empty(h, 0, prec)
        c = wm.internal_empty(h, 0, prec)
        if a.is_complex():
            a.copy_(torch.randn(a.shape, dtype=a.dtype, device="cuda"))
        else:
            a.copy_(torch.randn(a.shape, device="cuda").to(a.dtype))
        for _ in range(3):
            wm.dslash_apply(h, prec, a, c, 1, stream)
        reps = 20 if prec != wm.MG_F64 else 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(reps):
            wm.dslash_apply(h, prec, a if i % 2 == 0 else c, c if i % 2 == 0 else a, 1, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / reps
        gbs = per_site[prec] * V / t / 1e9
        ent = {"us": round(t * 1e6, 2), "bytes_per_site": per_site[prec], "achieved_gbs": round(gbs, 1),
               "frac_of_measured_hbm": round(gbs / peak, 4), "tflops": round(flops_site * V / t / 1e12, 3)}
        if prec == wm.MG_F64:
            ent["bound"] = "alu"
            ent["fp64_peak_tflops"] = 1.196
            ent["frac_of_fp64_peak"] = round(flops_site * V / t / 1e12 / 1.196, 4)
        out[name] = ent
        del h, a, c
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------- tensor-core contractions
def mma_workload(args):
    """The tensor-core contractions alone at the 16^3 x 32 sizes of the batched solve: the level-1
    coarse stencil (BF16 operator, FP32 vectors, 48 x 48 blocks), the FP16 restriction and prolongation
    of 24 right-hand sides (P of Nv = 24 on 4^4 aggregates); CUDA events around `reps` launches each,
    algorithmic bytes as the library's profiler counts them (every operand once per launch)."""
    import torch
    from paper_0811_4331_gb300 import wilson_mg as wm
    stream = torch.cuda.current_stream()
    U = inputs.heatbath_gauge(C3_DIMS, BETA, HB_SWEEPS, HB_SEED)
    Ud = torch.from_numpy(U).cuda()
    p = wm.mg_default_params(n_levels=3, block=[(4, 4, 4, 4), (2, 2, 2, 2)], nv=[24, 24],
                             setup_sweeps=[args.mma_sweeps, args.mma_sweeps], mixed=1, seed=7, coarse_mma=1)
    h = wm.mg_setup(Ud, C3_DIMS, c3_mcrit() + args.c3_dm, p, stream=stream)
    R = args.mma_rhs
    d1, nc1, _ = wm.mg_level_info(h, 1)
    V0, V1 = int(np.prod(C3_DIMS)), int(np.prod(d1))
    fine = wm.internal_empty(h, 0, wm.MG_F16, R)
    fine.copy_(torch.randn(fine.shape, device="cuda").to(fine.dtype))
    c_in = wm.internal_empty(h, 1, wm.MG_F32, R)
    c_in.copy_(torch.randn(c_in.shape, dtype=c_in.dtype, device="cuda"))
    c_out = wm.internal_empty(h, 1, wm.MG_F32, R)
    f_out = wm.internal_empty(h, 0, wm.MG_F16, R)
    nv = 24
    pbytes = V0 * 12 * nv * 4                     # P once, FP16 complex
    fbytes, cbytes = V0 * 12 * 4 * R, V1 * nc1 * 8 * R
    kern = {
        "coarse_mma": (lambda: wm.coarse_apply(h, 1, wm.MG_F32, c_in, c_out, R, stream),
                       9 * nc1 * nc1 * 4 * V1 + 2 * cbytes, 9 * nc1 * nc1 * 8 * V1 * R),
        "restrict_mma": (lambda: wm.restrict_apply(h, 0, wm.MG_F16, fine, c_out, R, stream),
                         pbytes + fbytes + cbytes, 8 * 12 * nv * V0 * R),
        "prolong_mma": (lambda: wm.prolong_apply(h, 0, wm.MG_F16, c_in, f_out, R, stream),
                        pbytes + fbytes + cbytes, 8 * 12 * nv * V0 * R),
    }
    peak = measured_peaks()
    out = {"workload": "16^3x32 beta=6.0 field, 3-level mixed hierarchy (4^4 then 2^4 blocks, Nv=24/24), "
                       "%d right-hand sides" % R, "rhs": R}
    for name, (fn, nbytes, flops) in kern.items():
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.mma_reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / args.mma_reps
        out[name] = {"us": round(t * 1e6, 2), "bytes": int(nbytes), "achieved_gbs": round(nbytes / t / 1e9, 1),
                     "frac_of_measured_hbm": round(nbytes / t / 1e9 / peak.get("hbm_gbs", 6800.0), 4),
                     "tflops": round(flops / t / 1e12, 3)}
    wm.mg_destroy(h)
    return out


# ---------------------------------------------------------------------------- oracle (cpu) arm
# The FP64 numpy oracle runs the bench step (setup at the lightest mass, then
# the four masses) on the host cores: a spawn process pool takes the
# independent units of the step, the NV candidate relaxations and the four
# mass solves (each unit single-threaded, the oracle's code as it stands).
# A sampled step runs every unit, with SWEEPS_SAMPLE of the SETUP_SWEEPS MR
# sweeps and ITERS_SAMPLE outer iterations per mass, and its measured wall
# time is scaled to the whole step by the sweep count and by the oracle's own
# iteration counts (tests/golden/c2_reference.json); --oracle-full times the
# whole step instead (the cross-check of that scaling).
SWEEPS_SAMPLE, ITERS_SAMPLE = 6, 1
ORACLE_SAMPLE = ("FP64 numpy oracle on the same inputs, spawn process pool (one process per candidate "
                 "relaxation, then one per mass): %d of the %d setup MR sweeps of all %d candidates, block QR + "
                 "Galerkin P^+DP + dense LU per mass, %d outer MG-GCR iterations per mass; value = relaxation "
                 "wall x %d/%d + max over the masses of (QR/Galerkin/LU + oracle iteration count from "
                 "tests/golden/c2_reference.json, sweep form, x time per iteration)"
                 % (SWEEPS_SAMPLE, SETUP_SWEEPS, NV, ITERS_SAMPLE, SETUP_SWEEPS, SWEEPS_SAMPLE))

_ORACLE_U = None


def _oracle_init(path):
    global _ORACLE_U
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    _ORACLE_U = np.load(path)


def _oracle_lat():
    return (DIMS[3], DIMS[2], DIMS[1], DIMS[0])


def _oracle_apply(m):
    from oracle import dirac
    lat = _oracle_lat()
    return lambda y: dirac.wilson_dirac(_ORACLE_U, y.reshape(lat + (4, 3)), m).reshape(lat + (12,))


def _oracle_relax(job):
    """Candidate k after `sweeps` MR steps on A x = 0 (Sec. 2), seed-7 start vectors."""
    from oracle import multigrid as mg
    k, sweeps, m = job
    lat = _oracle_lat()
    n = int(np.prod(lat)) * 12
    start = inputs.counter_gaussian(7, n, offset=k * n).reshape(lat + (12,))  # start vector k of stream 7
    return mg.relax_null_vectors(_oracle_apply(m), [start], sweeps)[0]


def _oracle_mass(job):
    """One mass: P from the candidates, A_c = P^+ A P, dense LU, then MG-GCR to TOL (iters None) or
    `iters` outer iterations; returns (prep seconds, solve seconds, iterations, true residual)."""
    import scipy.linalg
    from oracle import dirac
    from oracle import multigrid as mg
    cands, m, iters = job
    lat = _oracle_lat()
    t0 = time.perf_counter()
    blk = mg.Blocking(lat, BLOCK, 12)
    P = mg.block_orthonormalize(list(cands), blk)
    Ac = mg.coarse_stencil(dirac.wilson_stencil(_ORACLE_U, m), P, blk)
    lu = scipy.linalg.lu_factor(mg.dense_from_stencil(Ac))
    apply = _oracle_apply(m)
    fine = mg.Level(apply, lat, 12)
    fine.P, fine.blk = P, blk
    coarse = mg.Level(lambda y: dirac.stencil_apply(Ac, y), blk.coarse, 2 * NV)
    coarse.stencil, coarse.lu = Ac, lu
    hier = [fine, coarse]
    b = inputs.gaussian_spinor(DIMS, RHS_SEED).reshape(lat + (12,))
    t1 = time.perf_counter()
    if iters is None:
        x, info = mg.fgcr(apply, b, lambda r: mg.vcycle(hier, 0, r), tol=TOL, restart=50)
        n, rel = info["iters"], info["true_rel_residual"]
    else:
        try:
            mg.fgcr(apply, b, lambda r: mg.vcycle(hier, 0, r), tol=1e-300, restart=iters, max_restarts=1)
        except ArithmeticError:
            pass
        n, rel = iters, None
    return t1 - t0, time.perf_counter() - t1, n, rel


def oracle_iters():
    """The oracle's own MG-GCR iteration counts of the step's form (setup at the lightest mass)."""
    with open(os.path.join(ROOT, "tests", "golden", "c2_reference.json")) as f:
        ref = json.load(f)
    return [m["iters"] for m in ref["sweep"]["masses"]]


def oracle_step(pool, nproc, full=False):
    """One oracle step on the pool; returns (wall seconds measured, seconds of the whole step, parts)."""
    mc = mcrit()
    masses = [mc + d for d in DMASSES]
    sweeps = SETUP_SWEEPS if full else SWEEPS_SAMPLE
    t0 = time.perf_counter()
    cands = pool.map(_oracle_relax, [(k, sweeps, masses[-1]) for k in range(NV)])
    t1 = time.perf_counter()
    res = pool.map(_oracle_mass, [(cands, m, None if full else ITERS_SAMPLE) for m in masses])
    t2 = time.perf_counter()
    parts = {"relax_wall_s": round(t1 - t0, 3), "masses_wall_s": round(t2 - t1, 3), "processes": nproc,
             "prep_s": [round(r[0], 3) for r in res], "solve_s": [round(r[1], 3) for r in res],
             "iters": [r[2] for r in res]}
    if full:
        parts["true_rel_residual"] = [r[3] for r in res]
        return t2 - t0, t2 - t0, parts
    whole = (t1 - t0) * SETUP_SWEEPS / SWEEPS_SAMPLE + max(
        r[0] + it * r[1] / ITERS_SAMPLE for r, it in zip(res, oracle_iters()))
    return t2 - t0, whole, parts


def oracle_pool(U):
    """(spawn pool with the gauge field loaded in every worker, process count, temp dir)."""
    import multiprocessing
    import tempfile
    td = tempfile.mkdtemp()
    path = os.path.join(td, "gauge.npy")
    np.save(path, U)
    nproc = max(1, min(os.cpu_count() or 1, NV))
    pool = multiprocessing.get_context("spawn").Pool(nproc, initializer=_oracle_init, initargs=(path,))
    return pool, nproc, td


def cpu_baseline_subprocess(U):
    """One sampled oracle step in a child process (no GPU), scaled to the whole step."""
    import tempfile
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "gauge.npy")
        np.save(path, U)
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", path], env=env,
                           capture_output=True, text=True)
    if r.returncode != 0:
        return {"error": r.stderr[-500:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": round(d["seconds"], 3), "unit": "s per 4-mass sweep", "cores": d["processes"],
            "kind": "oracle", "sample": ORACLE_SAMPLE, "sample_wall_s": round(d["wall"], 3), "parts": d["parts"]}


def oracle_sample_main(path, full=False):
    import shutil
    U = np.load(path)
    pool, nproc, td = oracle_pool(U)
    try:
        wall, whole, parts = oracle_step(pool, nproc, full=full)
    finally:
        pool.close()
        pool.join()
        shutil.rmtree(td, ignore_errors=True)
    print(json.dumps({"seconds": whole, "wall": wall, "processes": nproc, "parts": parts}))


def reference_arm(args, rank, world):
    """--impl reference: the oracle as it stands, on the host cores, same metric and unit.  Each step
    is one sampled oracle step (measured: ms_per_step); value scales it to the whole 4-mass sweep."""
    if rank != 0:
        return None
    import shutil
    U, _ = make_inputs()
    pool, nproc, td = oracle_pool(U)
    try:
        for _ in range(args.warmup):
            oracle_step(pool, nproc)
        walls, wholes, parts = [], [], None
        for _ in range(args.steps):
            w, v, parts = oracle_step(pool, nproc)
            walls.append(w)
            wholes.append(v)
    finally:
        pool.close()
        pool.join()
        shutil.rmtree(td, ignore_errors=True)
    v = float(np.median(wholes))
    return {"impl": "reference", "metric": "MG-GCR time-to-solution @1e-10 rel residual, mixed vs FP64; "
                                          "dslash HBM GB/s",
            "value": round(v, 3), "unit": "s per 4-mass sweep (setup + solve)", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(float(np.median(walls)) * 1e3, 1),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded beta=6.0 heatbath gauge field, Gaussian source)",
            "config": bench_config(args),
            "cpu_baseline": {"value": round(v, 3), "unit": "s per 4-mass sweep", "cores": nproc, "kind": "oracle",
                             "sample": ORACLE_SAMPLE, "parts": parts},
            "e2e": {"value": round(v, 3), "unit": "s per 4-mass sweep", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------------------- multi-RHS workload
C3_DIMS = (16, 16, 16, 32)


# Setup of the 16^3 x 32 hierarchy (Nv = 24/24): 4 + 16 candidates of each level from 300 MR sweeps, the
# rest from two adaptive steps of 64 solver iterations each (Sec. 2).  At m_crit + 0.02 the mixed solve
# needs 100 iterations this way, against 250 with 1000/300 relaxation sweeps alone and 450 with 300/100.
C3_SWEEPS = (300, 300)
C3_ADAPT = dict(adapt_steps=2, adapt_nv=[20, 8], adapt_cycles=64)


def c3_params(wm, mixed):
    return wm.mg_default_params(n_levels=3, block=[(4, 4, 4, 4), (2, 2, 2, 2)], nv=[24, 24],
                                setup_sweeps=list(C3_SWEEPS), mixed=mixed, seed=7, coarse_mma=mixed, **C3_ADAPT)


def c3_mcrit():
    """m_crit of the 16^3 x 32 beta = 6.0 field: minus the smallest real part of the spectrum of D(m = 0),
    from the oracle's Arnoldi run (tests/golden/mcrit.json)."""
    key = "%dx%dx%dx%d_beta%.1f_sweeps%d_seed%d" % (*C3_DIMS, BETA, HB_SWEEPS, HB_SEED)
    with open(os.path.join(ROOT, "tests", "golden", "mcrit.json")) as f:
        return json.load(f)[key]["m_crit"]


def c3_workload(args):
    """16^3 x 32 beta = 6.0: 12 point sources (one per spin x colour) + 12 Gaussian sources in one
    mixed-precision three-level solve, against 24 single-source plain FP64 solves (same hierarchy shape)."""
    import torch
    from paper_0811_4331_gb300 import wilson_mg as wm
    stream = torch.cuda.current_stream()
    U = inputs.heatbath_gauge(C3_DIMS, BETA, HB_SWEEPS, HB_SEED)
    Ud = torch.from_numpy(U).cuda()
    srcs = [inputs.point_source(C3_DIMS, s, c) for s in range(4) for c in range(3)]
    srcs += [inputs.gaussian_spinor(C3_DIMS, 100 + r) for r in range(12)]
    B = torch.from_numpy(np.stack(srcs)).cuda()
    mass = c3_mcrit() + args.c3_dm
    out = {"workload": "16^3x32 beta=6.0 heatbath (200 sweeps, seed 0), 3-level MG 4^4 then 2^4 blocks, Nv=24/24, "
                       "setup %d/%d MR sweeps + 2 adaptive steps (20/8 of the candidates, 64 solver iterations each), "
                       "m = m_crit + %g (m_crit = %.4f from Arnoldi), 12 point + 12 Gaussian sources, tol 1e-10"
                       % (C3_SWEEPS[0], C3_SWEEPS[1], args.c3_dm, c3_mcrit())}
    res = {}
    for mixed in ((1,) if args.no_plain else (1, 0)):
        # the mixed form applies the level-1 stencil to all right-hand sides on tensor cores
        p = c3_params(wm, mixed)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = wm.mg_setup(Ud, C3_DIMS, mass, p, stream=stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        X = torch.zeros_like(B)
        if mixed:
            _, st = wm.mg_solve(h, B, X, TOL, stream=stream)
            its = [s["iters"] for s in st]
            rel = [s["true_rel_residual"] for s in st]
        else:
            its, rel = [], []
            for r in range(B.shape[0]):
                xr = torch.zeros_like(B[r])
                _, st = wm.mg_solve(h, B[r].contiguous(), xr, TOL, stream=stream)
                X[r] = xr
                its.append(st[0]["iters"])
                rel.append(st[0]["true_rel_residual"])
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        res["mixed_multi_rhs" if mixed else "fp64_single_rhs"] = {
            "setup_s": round(t1 - t0, 4), "solve_s": round(t2 - t1, 4), "iters": its,
            "max_true_rel_residual": max(rel)}
        del h
    out.update(res)
    if "fp64_single_rhs" in res:
        out["speedup_solve"] = round(res["fp64_single_rhs"]["solve_s"] / res["mixed_multi_rhs"]["solve_s"], 3)
    # class shares and the dominant class's roofline of the mixed multi-RHS solve (one profiled run)
    p = c3_params(wm, 1)

    def run(collect):
        h = wm.mg_setup(Ud, C3_DIMS, mass, p, stream=stream)
        X = torch.zeros_like(B)
        wm.mg_solve(h, B, X, TOL, stream=stream)
        collect(h)
        wm.mg_destroy(h)

    tot = class_profile(wm, run, measured_peaks())
    out["roofline"], out["kernel_shares"] = shares_and_roofline(tot, measured_peaks())
    return out


# ---------------------------------------------------------------------------- large lattice
C5_DIMS = (32, 32, 32, 64)


# the 16^3 x 32 setup's adaptive steps, on the first two of the three coarsenings
C5_ADAPT = dict(adapt_steps=2, adapt_nv=[20, 8, 0], adapt_cycles=64)


def tile_gauge(U, reps):
    """A periodic field on the lattice reps times larger per direction: the same links repeated
    (still a periodic SU(3) configuration with the source's plaquette; its Dirac spectrum contains the
    source's, so it keeps a comparable critical mass)."""
    lat = U.shape[1:5]  # (Lt, Lz, Ly, Lx)
    out = U
    for ax, r in zip(range(1, 5), reversed(reps)):
        out = np.concatenate([out] * r, axis=ax)
    assert out.shape[1:5] == tuple(l * r for l, r in zip(lat, reversed(reps)))
    return np.ascontiguousarray(out)


def c5_workload(args):
    """32^3 x 64: MG with 4^4 then 2^4 blocks (Nv = 24/32) and a fourth level (2^4, Nv = 24) for an exact
    coarsest solve, 12 Gaussian sources, the mixed multi-RHS solve against 12 single-RHS plain FP64
    solves, at masses above the m_crit of the 16^3 x 32 field it tiles (the tiled lattice holds that
    field's spectrum and more momenta, so its own m_crit lies at or below it: the dm are kept >= 0.03)."""
    import torch
    from paper_0811_4331_gb300 import wilson_mg as wm
    stream = torch.cuda.current_stream()
    U = tile_gauge(inputs.heatbath_gauge(C3_DIMS, BETA, HB_SWEEPS, HB_SEED), (2, 2, 2, 2))
    Ud = torch.from_numpy(U).cuda()
    del U
    nrhs = args.c5_rhs
    B = torch.from_numpy(np.stack([inputs.gaussian_spinor(C5_DIMS, 200 + r) for r in range(nrhs)])).cuda()
    out = {"workload": "32^3x64: the 16^3x32 beta=6.0 heatbath field (200 sweeps, seed 0) tiled 2x2x2x2, "
                       "4-level MG 4^4, 2^4, 2^4 blocks, Nv=24/32/24, setup 300 MR sweeps + 2 adaptive steps "
                       "(20/8 candidates of the first two levels, 64 solver iterations each), %d Gaussian sources, "
                       "tol 1e-10, GCR(%d)"
                       % (nrhs, args.c5_restart), "masses": []}
    for dm in args.c5_dm:
        mass = c3_mcrit() + dm
        row = {"m": round(mass, 4)}
        for mixed in ((1,) if args.no_plain else (1, 0)):
            # the third level (4^3 x 8 sites x 64 components = 32768 unknowns) is too large for the
            # exact dense coarsest solve, so a fourth level (2^4 blocks, Nv = 24: 1536 unknowns) takes it
            p = wm.mg_default_params(n_levels=4, block=[(4, 4, 4, 4), (2, 2, 2, 2), (2, 2, 2, 2)], nv=[24, 32, 24],
                                     setup_sweeps=[300, 300, 300], mixed=mixed, seed=7, coarse_mma=mixed,
                                     gcr_restart=args.c5_restart, max_iter=4000, **C5_ADAPT)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = wm.mg_setup(Ud, C5_DIMS, mass, p, stream=stream)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            X = torch.zeros_like(B)
            if mixed:
                _, st = wm.mg_solve(h, B, X, TOL, stream=stream)
            else:
                st = []
                for r in range(nrhs):
                    xr = torch.zeros_like(B[r])
                    _, s1 = wm.mg_solve(h, B[r].contiguous(), xr, TOL, stream=stream)
                    st += s1
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            row["mixed_multi_rhs" if mixed else "fp64_single_rhs"] = {
                "setup_s": round(t1 - t0, 3), "solve_s": round(t2 - t1, 3), "iters": [s["iters"] for s in st],
                "max_true_rel_residual": max(s["true_rel_residual"] for s in st)}
            wm.mg_destroy(h)
        if "fp64_single_rhs" in row:
            row["speedup_solve"] = round(row["fp64_single_rhs"]["solve_s"] / row["mixed_multi_rhs"]["solve_s"], 3)
        out["masses"].append(row)
    return out


# ---------------------------------------------------------------------------- serving workload
def serve_workload(args):
    """Poisson stream of solve requests over three beta = 6.0 fields (8^4, 12^4, 16^3 x 32): masses
    uniform in [m_crit + 0.005, m_crit + 0.1], 1-12 Gaussian right-hand sides each, hierarchies cached per
    field (setup at the lightest mass, retargeted per request), HBM-budget admission, 4 workers."""
    import torch
    from paper_0811_4331_gb300 import serve
    from paper_0811_4331_gb300 import wilson_mg as wm
    with open(os.path.join(ROOT, "tests", "golden", "mcrit.json")) as f:
        mc = json.load(f)
    # m_crit of each field from the oracle's Arnoldi run (tests/golden/mcrit.json)
    def crit_of(dims):
        key = "%dx%dx%dx%d_beta6.0_sweeps200_seed0" % dims
        return mc[key]["m_crit"], 0.005

    crit = {d: crit_of(d) for d in ((8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 32))}
    two = wm.mg_default_params(n_levels=2, block=[(4, 4, 4, 4)], nv=[20], setup_sweeps=[300], mixed=1, seed=7)
    three = c3_params(wm, 1)
    fields = {}
    for dims, p in (((8, 8, 8, 8), two), ((12, 12, 12, 12), two), ((16, 16, 16, 32), three)):
        U = inputs.heatbath_gauge(dims, BETA, HB_SWEEPS, HB_SEED)
        fields["x".join(map(str, dims))] = (U, dims, crit[dims][0] + crit[dims][1], p)
    names = sorted(fields)
    budget = int(0.5 * torch.cuda.get_device_properties(0).total_memory)
    rng = np.random.default_rng(4)
    out = {"workload": "serving: Poisson arrivals, fields 8^4 / 12^4 / 16^3x32 (beta=6.0 heatbath), masses "
                       "U[m_crit+0.005, m_crit+0.1] (m_crit of each field from the oracle's Arnoldi run), "
                       "1-12 Gaussian RHS, tol 1e-10, 4 workers, waiting requests of a field merged into one "
                       "solve of up to 64 RHS (a mass per RHS), half of HBM as budget (resident hierarchies "
                       "included)",
           "m_crit": {"x".join(map(str, d)): v[0] for d, v in crit.items()},
           "rates": []}
    srv = serve.SolveServer(fields, None, budget, workers=4, keep_results=False)
    for name in names:  # warm the per-field hierarchies (setup once per field)
        srv.base(name)
    n_per_rate = args.serve_requests // len(args.serve_rates)
    for rate in args.serve_rates:
        reqs = []
        for i in range(n_per_rate):
            f = names[int(rng.integers(0, len(names)))]
            dims = fields[f][1]
            nrhs = int(rng.integers(1, 13))
            seed = int(rng.integers(1 << 30))
            m = crit[dims][0] + float(rng.uniform(crit[dims][1], 0.1))

            def make(i=i, f=f, dims=dims, nrhs=nrhs, seed=seed, m=m):
                # the right-hand sides are drawn when the request arrives: a 16^3 x 32 request holds up
                # to 300 MB, too much to keep a whole stream of them in host memory
                g = np.random.default_rng(seed)
                shp = (nrhs,) + (dims[3], dims[2], dims[1], dims[0], 4, 3)
                return serve.Request(i, f, m, g.standard_normal(shp) + 1j * g.standard_normal(shp), TOL, 0.0)

            reqs.append(make)
        nb0 = len(srv.batches)
        st = serve.run_stream(srv, reqs, serve.poisson_arrivals(rate, len(reqs), int(rng.integers(1 << 30))))
        bt = srv.batches[nb0:]
        st["rate_per_s"] = rate
        st["max_inflight"] = srv.max_inflight
        st["batches"] = len(bt)
        st["mean_requests_per_batch"] = round(float(np.mean([n for n, _ in bt])), 2) if bt else None
        st["mean_rhs_per_batch"] = round(float(np.mean([k for _, k in bt])), 2) if bt else None
        out["rates"].append(st)
    out["resident_hierarchy_bytes"] = int(srv.resident_bytes)
    best = max(out["rates"], key=lambda r: r["solves_per_s"])
    out["saturation"] = {"solves_per_s": round(best["solves_per_s"], 2), "rhs_per_s": round(best["rhs_per_s"], 1),
                         "at_rate_per_s": best["rate_per_s"]}
    srv.close()
    return out


# ---------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-dslash-hbm", action="store_true")
    ap.add_argument("--only-timed", action="store_true", help="time the mixed step only (for profiler runs)")
    ap.add_argument("--ncu", action="store_true",
                    help="profiler run: the timed mixed step only, no clock sampling (no child processes)")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-full", action="store_true",
                    help="time the whole oracle step (setup + four mass solves to 1e-10) on the host cores and exit")
    ap.add_argument("--workload", choices=["c2", "c3", "c5", "serve", "dslash", "mma"], default="c2",
                    help="c2: the mass-sweep step (default bench line); c3: 24-source batched solve; serve: stream; "
                         "dslash: the fine stencil alone (--dslash-dims, --dslash-prec); mma: the tensor-core "
                         "contractions alone at the 16^3x32 sizes")
    ap.add_argument("--sweep", choices=["many", "masses"], default="many",
                    help="c2 step: the four masses as concurrent handles (mg_solve_many) or as one solve with a "
                         "mass per right-hand side (mg_solve_masses)")
    ap.add_argument("--dslash-dims", type=int, nargs=4, default=list(BW_DIMS))
    ap.add_argument("--dslash-prec", nargs="+", choices=["f16", "bf16", "f32", "f64"], default=None)
    ap.add_argument("--c3-dm", type=float, default=0.02)
    ap.add_argument("--mma-rhs", type=int, default=24)
    ap.add_argument("--mma-reps", type=int, default=20)
    ap.add_argument("--mma-sweeps", type=int, default=20, help="setup sweeps of the mma workload's hierarchy")
    ap.add_argument("--c5-dm", type=float, nargs="+", default=[0.06, 0.03])
    ap.add_argument("--c5-rhs", type=int, default=12)
    ap.add_argument("--c5-restart", type=int, default=16)
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[10.0, 20.0, 40.0, 80.0])
    args = ap.parse_args()
    if args.ncu:
        args.only_timed = True
    if args.oracle_sample:
        oracle_sample_main(args.oracle_sample)
        return
    if args.oracle_full:
        import tempfile
        with tempfile.TemporaryDirectory() as td:
            path = os.path.join(td, "gauge.npy")
            np.save(path, make_inputs()[0])
            oracle_sample_main(path, full=True)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        out = reference_arm(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    import torch
    if args.workload == "c3":
        print(json.dumps(c3_workload(args)))
        return
    if args.workload == "c5":
        print(json.dumps(c5_workload(args)))
        return
    if args.workload == "serve":
        print(json.dumps(serve_workload(args)))
        return
    if args.workload == "mma":
        print(json.dumps(mma_workload(args)))
        return
    if args.workload == "dslash":
        st = torch.cuda.Stream()
        from paper_0811_4331_gb300 import wilson_mg as wm
        print(json.dumps(dslash_bandwidth(wm, torch, st, tuple(args.dslash_dims), args.dslash_prec)))
        return
    if world > 1:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group("nccl")
    U, b = make_inputs()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.only_timed:
        cpu = cpu_baseline_subprocess(U)
    r = native(args, rank, world, U, b)
    if rank == 0:
        v = r.pop("value")
        line = {"metric": "MG-GCR time-to-solution @1e-10 rel residual, mixed vs FP64; dslash HBM GB/s",
                "value": round(v, 5), "unit": "s per 4-mass sweep (setup + solve)", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v * 1e3, 3),
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded beta=6.0 heatbath gauge field, Gaussian source)",
                "config": bench_config(args),
                "solves_per_s": round(world * len(DMASSES) / v, 3)}
        line.update(r)
        line["cpu_baseline"] = cpu
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
