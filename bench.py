#!/usr/bin/env python
"""Benchmark of the MEM hot path on GB300.

Headline: cell-solves/s of the batched standalone maximal-entropy solve
(Algorithm 1 on 2^20 independent 35-moment cells, tensor Gauss-Hermite 8^3,
cold start beta = 0), tuned (fused) back-end, inputs resident in HBM.  One
step = one mem_solve over the whole batch.  Reported beside it: the same
metric end to end through the C ABI from pinned host buffers (e2e), the plain
FP32 back-end, the 12^3 rule, the Mach-10 shock (4096 cells, graph-captured
Algorithm 2 step) in cell-updates/s, the roofline of the fused kernel, and the
FP64 oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tuned|reference]
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MEM cell-solves/s & cell-updates/s at Ma10, tuned vs plain FP32; p99 latency"
UNIT = "cell-solves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tuned", choices=["tuned", "reference"])
    ap.add_argument("--cells", type=int, default=1 << 20)
    ap.add_argument("--order", type=int, default=8)
    ap.add_argument("--no-extras", action="store_true", help="headline only (used for profiler runs)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--case", nargs="+", default=None, metavar=("NAME", "N"),
                    help="kernel-focused run for profilers instead of the benchmark: "
                         "solve|mixed|plain [cells] | ensemble|mach10|mach10flic|mach10nine|mach10flicnine|config4 [steps]")
    return ap.parse_args()


# ---------------------------------------------------------------- helpers
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.p is None:
            return out
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        os.unlink(self.f.name)
        return out


def fused_flops_per_pass(n):
    """Algorithmic FP32 flops of one Newton pass of the fused kernel for one
    cell (FMA = 2): two sum-factorised exponent evaluations, one line-search
    trial, the three moment stages, Hessian assembly from the Hermite
    linearisation, Cholesky and two triangular solves."""
    expo = n * n * 49 + n ** 3 * 5
    trial = n ** 3 * 2
    stages = n ** 3 * 9 + 45 * n * n + 165 * n
    terms = 0
    idx = [(a, b, d - a - b) for d in range(5) for a in range(d, -1, -1) for b in range(d - a, -1, -1)]
    for i in range(1, 35):
        for j in range(1, i + 1):
            t = 1
            for x, y in zip(idx[i], idx[j]):
                t *= min(x, y) + 1
            terms += t
    hess = terms + 595
    chol = sum((34 - k - 1) * (34 - k) // 2 + (34 - k - 1) for k in range(34))
    trsv = 34 * 34
    fma = 2 * expo + trial + stages + hess + chol + trsv
    return 2 * fma


# dram__bytes_read.sum + dram__bytes_write.sum of one k_fused_solve<8> launch
# on the headline workload (2^20 cells) from one ncu capture, keyed to the
# SHA-256 of the kernel's sources at that capture: a changed kernel reports
# traffic None until it is captured again.
TRAFFIC = {"kernel": "k_fused_solve<8>", "bytes": 403.26e6,
           "sources": ("fused.cu", "sumfact.cuh", "common.cuh"),
           "sha256": "17529a48b205143caa83dd964397463e180df315021dec3483a84bcb09c5aab7"}


def kernel_sources_sha(names):
    import hashlib
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2303_02898_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def traffic_bytes():
    sha = kernel_sources_sha(TRAFFIC["sources"])
    return TRAFFIC["bytes"] if sha == TRAFFIC["sha256"] else None


def measured_peaks(mem):
    """The library's micro-benchmarks on this GPU (one launch each, CUDA
    events): FP32 FMA and TF32 / BF16 tensor-core flop/s, exp2 evaluations/s."""
    out = {}
    for key, kind, iters in (("fp32_tflops", mem.PEAK_FMA, 4000), ("exp2_tera_per_s", mem.PEAK_EXP2, 2000),
                             ("bf16_tc_tflops", mem.PEAK_TC_BF16, 20000), ("tf32_tc_tflops", mem.PEAK_TC_TF32, 20000)):
        best = 0.0
        for _ in range(3):
            sec, work = mem.bench_peak(kind, iters)
            best = max(best, work / sec / 1e12)
        out[key] = best
    out["how"] = ("mem_bench_peak: FP32 FMA chains / ex2.approx chains on 152 x 4 blocks of 512 threads; "
                  "tcgen05.mma 128x256 (K 16 BF16 / 8 TF32) back to back from SMEM into TMEM, one CTA per SM; "
                  "best of 3 launches")
    return out

SHOCK_MACH = 3.0   # largest Mach the 8^3 Gauss-Hermite Hermite-gauge rule keeps stable from a step


def run_ensemble(mem, ctx, torch, np, nsteps=10):
    """256 packed shock problems (ncells logU[256, 16384], Mach U[1.2, 3]) advanced
    together; cell-updates/s of the graph-captured fused step vs the plain one."""
    from paper_2303_02898_gb300 import workloads
    probs = workloads.ensemble_problems(256, seed=1, mach_hi=SHOCK_MACH)
    cells = sum(p.ncells for p in probs)
    out = {}
    for impl, graph, tag, n in ((mem.IMPL_FUSED, 1, "tuned", nsteps), (mem.IMPL_PLAIN, 0, "plain", 3)):
        sh = mem.Shock(ctx, problems=[dict(mach=p.mach, ncells=p.ncells, xl=p.xl, xr=p.xr) for p in probs],
                       impl=impl, graph=graph)
        sh.step(2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sh.step(n)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        fin = all(np.isfinite(sh.problem(i)["rho"]).all() for i in (0, 100, 255))
        sh.close()
        out["ensemble_%s" % tag] = {"value": cells * n / dt, "unit": "cell-updates/s", "problems": len(probs),
                                    "cells": cells, "steps": n, "ms_per_step": 1e3 * dt / n, "finite": fin}
    out["ensemble_tuned_over_plain"] = out["ensemble_tuned"]["value"] / out["ensemble_plain"]["value"]
    return out


def _mach10_paper_mesh(mem, torch, np, vctx, scheme, nsteps, stats=35):
    """One Mach-10 problem on the paper's mesh: cell-updates/s of the
    graph-captured step, then steps and wall time to the steady metric."""
    sh = mem.Shock(vctx, mach=10.0, ncells=150, xl=-47.1, xr=47.1, ic=1, graph=1, scheme=scheme, stats=stats)
    sh.step(3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sh.step(nsteps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    rec = {"value": 150 * nsteps / dt, "unit": "cell-updates/s", "cells": 150, "domain": [-47.1, 47.1],
           "steps": nsteps, "ms_per_step": 1e3 * dt / nsteps, "rule": "velocity-space 6x4 blocks x 8 GL, K=12",
           "scheme": {0: "local Lax-Friedrichs", 1: "Lax-Wendroff", 2: "FLIC"}[scheme],
           "statistics": "the paper's nine (u_x, u_r) statistics" if stats == 9 else "35 Hermite products"}
    done, d = 3 + nsteps, None
    t1 = time.perf_counter()
    while done < 20000:
        d = sh.step(500, steady=True)
        done += 500
        if not np.isfinite(d) or d < 1e-6:
            break
    torch.cuda.synchronize()
    prof = sh.get()
    rec.update({"steady_steps": done, "steady_metric": float(d), "steady_wall_s": time.perf_counter() - t1 + dt,
                "sim_time": prof["t"], "T_max_over_T_down": float(np.max(prof["T"]) / 32.1233),
                "rho_max_over_rho_down": float(np.max(prof["rho"]) / 3.88386),
                "finite": bool(np.isfinite(prof["M"]).all())})
    sh.close()
    return rec


def run_mach10(mem, torch, np, nsteps=400):
    """Mach-10 shocks on the velocity-space rule (6 x 4 blocks of 8-point
    Gauss-Legendre in (u_x, u_r), 12 azimuths; domain from the
    Rankine-Hugoniot states, n = 5):
      - the paper's Mach-10 mesh, 150 cells on [-47.1, 47.1], tanh start:
        cell-updates/s of the graph-captured step, then the steps and wall
        time to steady state (max |d rho| / (rho_+ - rho_-) < 1e-6 per step,
        at most 20000 steps);
      - a packed ensemble of 256 such problems, Mach U[1.2, 10];
      - 4096 cells on [-50, 50] (cell width 0.024): over-refined by 25x
        relative to the paper's mesh; reported as far as it stays finite."""
    from paper_2303_02898_gb300 import workloads
    out = {}
    vctx = mem.Context.velocity(mem.shock_domain(mach=10.0))
    for stats, sfx in ((35, ""), (9, "_nine")):
        out["shock_mach10_paper_mesh" + sfx] = _mach10_paper_mesh(mem, torch, np, vctx, mem.SCHEME_LF, nsteps, stats)
        # the paper's own Mach-10 scheme (Section 4): FLIC, one more Newton solve per interface
        out["shock_mach10_paper_mesh_flic" + sfx] = _mach10_paper_mesh(mem, torch, np, vctx, mem.SCHEME_FLIC, nsteps,
                                                                       stats)
    rng = np.random.default_rng(7)
    machs = rng.uniform(1.2, 10.0, 256)
    probs = [dict(mach=float(m), ncells=150, xl=-47.1, xr=47.1) for m in machs]
    for key, scheme, stats in (("ensemble_mach10_paper_mesh", mem.SCHEME_LF, 35),
                               ("ensemble_mach10_paper_mesh_flic", mem.SCHEME_FLIC, 35),
                               ("ensemble_mach10_paper_mesh_nine", mem.SCHEME_LF, 9),
                               ("ensemble_mach10_paper_mesh_flic_nine", mem.SCHEME_FLIC, 9)):
        sh = mem.Shock(vctx, problems=probs, ic=1, graph=1, scheme=scheme, stats=stats)
        sh.step(3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sh.step(50)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        fin = all(np.isfinite(sh.problem(i)["rho"]).all() for i in range(0, 256, 15))
        # Newton passes of the last step (every cell): the solve kernel's roofline
        passes = int(sh.device_tensors()[4].sum().item())
        sh.close()
        cells = 256 * 150
        out[key] = {"value": cells * 50 / dt, "unit": "cell-updates/s", "problems": 256, "cells": cells,
                    "mach": [1.2, 10.0], "steps": 50, "ms_per_step": 1e3 * dt / 50, "finite": fin,
                    "scheme": "FLIC" if scheme == mem.SCHEME_FLIC else "local Lax-Friedrichs",
                    "statistics": stats}
        if scheme == mem.SCHEME_LF:
            rule = vctx.velocity_rule()[0]
            nx, nr = rule[0] * rule[2], rule[1] * rule[2]
            fpp = vel_flops_per_pass(nx, nr * rule[3]) if stats == 35 else axi_flops_per_pass(nx, nr)
            peak = measured_peaks(mem)["fp32_tflops"]
            ach = passes * fpp / (dt / 50) / 1e12
            out[key]["roofline_" + ("k_vel" if stats == 35 else "k_axi")] = {
                "bound": "alu", "unit": "TFLOP/s", "achieved": ach, "peak": peak, "frac": ach / peak,
                "passes_per_step": passes, "flops_per_pass": fpp,
                "note": "of measured FP32 FMA rate; whole step time (the solve kernel is most of it, "
                        "profiles/launches_mach10_ensemble_*.md) in the denominator"}
    out.update(run_mach10_4096(mem, torch, np, vctx))
    vctx.close()
    return out


def run_mach10_4096(mem, torch, np, vctx, nsteps=2000, chunk=200):
    """The Mach-10 mesh of 4096 cells on [-50, 50] (cell width 0.024, 25x
    finer than the paper's), tanh start, graph-captured step, warm-started
    Newton: cell-updates/s over nsteps steps in chunks, and whether (and
    when) the FP32 state stops being finite.  Both statistics systems."""
    out = {}
    for stats, key in ((35, "shock_mach10_4096_pm50"), (9, "shock_mach10_4096_pm50_nine")):
        sh = mem.Shock(vctx, mach=10.0, ncells=4096, xl=-50.0, xr=50.0, ic=1, graph=1, stats=stats)
        sh.step(3)
        torch.cuda.synchronize()
        bad_at, done, metric = None, 0, None
        t0 = time.perf_counter()
        while done < nsteps:
            metric = sh.step(chunk, steady=True)
            done += chunk
            if not np.isfinite(metric) or not np.isfinite(sh.get()["M"]).all():
                bad_at = done
                break
        dt = time.perf_counter() - t0
        prof = sh.get()
        sh.close()
        out[key] = {"value": 4096 * done / dt, "unit": "cell-updates/s", "cells": 4096, "domain": [-50.0, 50.0],
                    "steps": done, "ms_per_step": 1e3 * dt / done, "finite": bad_at is None,
                    "non_finite_by_step": bad_at, "steady_metric_last": float(metric), "sim_time": prof["t"],
                    "statistics": stats,
                    "note": "cell width 0.024 vs the paper's 0.628; the paper reports Mach-10 FP32 runs failing "
                            "beyond 160 cells on [-47.1, 47.1] (Fig. 7)"}
    return out


def axi_flops_per_pass(nx, nr):
    """Algorithmic FP32 flops of one Newton pass of the nine-statistic kernel
    for one cell (FMA = 2): one sweep over the nx x nr nodes (5 FMA of
    exponent, 10 of x stage), the s stage (50 moments over nr nodes), the
    linearisation terms of the 8 x 8 Hessian (about 200), the 8 x 8 Cholesky
    and two triangular solves."""
    return 2 * (nx * nr * 15 + 50 * nr + 200 + 8 ** 3 // 6 + 2 * 64)


def vel_flops_per_pass(nx, npt):
    """Algorithmic FP32 flops of one Newton pass of the 35-statistic
    velocity-rule kernel (k_vel) for one cell (FMA = 2): on each of the
    nx x npt nodes 5 FMA of exponent and 9 of x stage; on each of the npt
    plane points the 35 terms of P_a and the 165 moments of degree <= 8 plus
    about 60 products he_b(y) he_c(z); the 1670 linearisation terms of the
    34 x 34 Hessian, its Cholesky (34^3 / 6) and two triangular solves."""
    return 2 * (nx * npt * 14 + npt * 260 + 1670 + 34 ** 3 // 6 + 2 * 34 * 34)


def run_ensemble_config4(mem, torch, np, nsteps=40):
    """The batched ensemble as stated: 256 problems, ncells logU[256, 16384],
    Mach U[1.2, 10] (seed 1), cell width 0.628, each problem on its own
    Rankine-Hugoniot box of the velocity-space rule, tanh start, all packed
    in one batch whose graph-captured step runs one persistent Newton launch
    (the paper's nine-statistic system: solve, flux and speed) over every
    cell of every problem.  Per-problem outcome after nsteps steps (finite or
    failed in FP32; the paper's Mach-10 runs fail above 160 cells on its
    domain, Fig. 7), and cell-updates/s."""
    from paper_2303_02898_gb300 import workloads
    probs = workloads.ensemble_problems(256, seed=1)
    cells = sum(p.ncells for p in probs)
    vctx = mem.Context.velocity(mem.shock_domain(mach=10.0))
    sh = mem.Shock(vctx, problems=[dict(mach=p.mach, ncells=p.ncells, xl=p.xl, xr=p.xr) for p in probs], ic=1,
                   graph=0, stats=9)
    sh.step(3)
    # launch shape of the nine-statistic kernel from the autotuner, timed on
    # the batch's own state (first 2^17 cells)
    Md, bd, gd = sh.device_tensors()[:3]
    nt = min(Md.shape[0], 1 << 17)
    rep = vctx.tune(mem.TUNE_AXI, Md[:nt], bd[:nt].clone(), gd[:nt], reps=2)
    bw, bb, bms = rep["candidates"][rep["best"]]
    sh.close()
    sh = mem.Shock(vctx, problems=[dict(mach=p.mach, ncells=p.ncells, xl=p.xl, xr=p.xr) for p in probs], ic=1,
                   graph=1, stats=9)
    sh.step(3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sh.step(nsteps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    fin = np.array([bool(np.isfinite(sh.problem(i)["rho"]).all()) for i in range(len(probs))])
    mach = np.array([p.mach for p in probs])
    nc = np.array([p.ncells for p in probs])
    # Newton passes of the last step (every cell), for the kernel's roofline
    passes = int(sh.device_tensors()[4].sum().item())
    rule = vctx.velocity_rule()[0]
    nx, nr = rule[0] * rule[2], rule[1] * rule[2]
    fpp = axi_flops_per_pass(nx, nr)
    peak = measured_peaks(mem)["fp32_tflops"]
    ach = passes * fpp / (dt / nsteps) / 1e12
    sh.close()
    vctx.close()
    return {"ensemble_config4": {"value": cells * nsteps / dt, "unit": "cell-updates/s", "problems": len(probs),
                                 "cells": int(cells), "steps": nsteps, "ms_per_step": 1e3 * dt / nsteps,
                                 "mach": [1.2, 10.0], "ncells": [256, 16384],
                                 "finite_problems": int(fin.sum()),
                                 "failed": [{"mach": round(float(m), 2), "ncells": int(n)}
                                            for m, n, f in zip(mach, nc, fin) if not f],
                                 "statistics": 9, "rule": "velocity-space 6x4 blocks x 8 GL per problem box",
                                 "roofline_k_axi": {"bound": "alu", "unit": "TFLOP/s", "achieved": ach, "peak": peak,
                                                    "frac": ach / peak, "passes_per_step": passes,
                                                    "flops_per_pass": fpp,
                                                    "note": "of measured FP32 FMA rate; whole step time (k_axi is "
                                                            "95 % of it) in the denominator"},
                                 "autotune": {"kernel": "k_axi", "chosen": {"warps": bw, "blocks_per_sm": bb},
                                              "candidates": [{"warps": w, "blocks_per_sm": b, "ms": round(ms, 3)}
                                                             for w, b, ms in rep["candidates"]],
                                              "gain_over_default": rep["default_ms"] / bms}}}


def run_serving_config5(mem, torch, np, nreq=24, max_steps=3000, chunk=50):
    """Serving as stated: Poisson arrivals at 200/s (seed 2), Mach U[1.5, 10],
    ncells logU[128, 32768], cell width 0.628, velocity-space rule with the
    nine-statistic system, tanh start; each request runs until its steady
    metric (max |d rho| / (rho_+ - rho_-) per step) is below 1e-6 or it
    reaches max_steps; continuous batching with graph-captured steps.
    p50/p99 latency, cell-updates/s, and the same requests one at a time."""
    from paper_2303_02898_gb300 import workloads
    t_arr, probs = workloads.serving_trace(nreq, seed=2)
    vctx = mem.Context.velocity(mem.shock_domain(mach=10.0))
    sv = mem.Server(vctx, hbm_budget_bytes=64 << 30, max_cells=1 << 21, steady_tol=1e-6, max_steps=max_steps)
    ids, nxt = [], 0
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        while nxt < nreq and t_arr[nxt] <= now:
            p = probs[nxt]
            ids.append((sv.submit(mach=p.mach, ncells=p.ncells, xl=p.xl, xr=p.xr, ic=1, stats=9), p))
            nxt += 1
        sv.progress(chunk)
        st = sv.stats()
        if nxt == nreq and st["completed"] == nreq:
            break
        if st["resident"] == 0 and st["queued"] == 0 and nxt < nreq:
            time.sleep(max(0.0, t_arr[nxt] - (time.perf_counter() - t0)))
    wall = time.perf_counter() - t0
    res = [(sv.poll(i, ncells=p.ncells), p) for i, p in ids]
    sv.close()
    lat = np.array([r["latency_s"] for r, _ in res])
    upd = sum(r["steps"] * p.ncells for r, p in res)
    # one at a time, the same number of steps each
    t1 = time.perf_counter()
    for r, p in res:
        sh = mem.Shock(vctx, mach=p.mach, ncells=p.ncells, xl=p.xl, xr=p.xr, ic=1, graph=1, stats=9)
        sh.step(r["steps"])
        sh.close()
    torch.cuda.synchronize()
    seq = time.perf_counter() - t1
    vctx.close()
    return {"serving_config5": {"requests": nreq, "rate_per_s": 200.0, "mach": [1.5, 10.0], "ncells": [128, 32768],
                                "max_steps": max_steps, "steady_tol": 1e-6,
                                "steady_requests": int(sum(r["steady"] for r, _ in res)),
                                "finite_requests": int(sum(bool(np.isfinite(r["rho"]).all()) for r, _ in res)),
                                "p50_latency_s": float(np.percentile(lat, 50)),
                                "p99_latency_s": float(np.percentile(lat, 99)),
                                "throughput": upd / wall, "unit": "cell-updates/s", "wall_s": wall,
                                "one_at_a_time_throughput": upd / seq, "one_at_a_time_wall_s": seq,
                                "statistics": 9, "graph": "each packed batch's step captured once and replayed"}}


def run_serving_mach10(mem, torch, np, nreq=32, max_steps=100, chunk=10):
    """Poisson trace (200 req/s, Mach U[1.5, 10]) on the velocity-space rule,
    each request capped at max_steps time steps.  Sizes follow the paper's
    Mach-10 mesh (cell width 0.628, ncells logU[128, 160]): longer Mach-10
    meshes fail in FP32.  Continuous batching vs the same requests one at a
    time on the same back-end (the plain back-end has no velocity-space form)."""
    from paper_2303_02898_gb300 import workloads
    t_arr, probs = workloads.serving_trace(nreq, seed=3, lo=128, hi=160, mach_lo=1.5, mach_hi=10.0)
    vctx = mem.Context.velocity(mem.shock_domain(mach=10.0))
    sv = mem.Server(vctx, hbm_budget_bytes=8 << 30, max_cells=1 << 16, steady_tol=1e-6, max_steps=max_steps)
    ids, nxt = [], 0
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        while nxt < nreq and t_arr[nxt] <= now:
            p = probs[nxt]
            ids.append((sv.submit(mach=p.mach, ncells=p.ncells, xl=p.xl, xr=p.xr, ic=1), p))
            nxt += 1
        sv.progress(chunk)
        st = sv.stats()
        if nxt == nreq and st["completed"] == nreq:
            break
        if st["resident"] == 0 and st["queued"] == 0 and nxt < nreq:
            time.sleep(max(0.0, t_arr[nxt] - (time.perf_counter() - t0)))
    wall = time.perf_counter() - t0
    res = [(sv.poll(i, ncells=p.ncells), p) for i, p in ids]
    lat = np.array([r["latency_s"] for r, _ in res])
    upd = sum(r["steps"] * p.ncells for r, p in res)
    sv.close()
    t1 = time.perf_counter()
    for r, p in res:
        sh = mem.Shock(vctx, mach=p.mach, ncells=p.ncells, xl=p.xl, xr=p.xr, ic=1, graph=0)
        sh.step(r["steps"])
        sh.close()
    torch.cuda.synchronize()
    seq = time.perf_counter() - t1
    vctx.close()
    return {"serving_mach10": {"requests": nreq, "rate_per_s": 200.0, "max_steps": max_steps, "mach": [1.5, 10.0],
                               "ncells": [128, 160], "rule": "velocity-space 6x4 blocks x 8 GL, K=12",
                               "p50_latency_s": float(np.percentile(lat, 50)),
                               "p99_latency_s": float(np.percentile(lat, 99)),
                               "throughput": upd / wall, "unit": "cell-updates/s", "wall_s": wall,
                               "one_at_a_time_throughput": upd / seq, "one_at_a_time_wall_s": seq,
                               "all_finite": bool(all(np.isfinite(r["rho"]).all() for r, _ in res))}}


def _serving_steady(mem, torch, np, nreq, max_steps, chunk, steady_tol):
    """Requests served to steady state: the Poisson trace of serving_mach10
    (200 req/s, Mach U[1.5, 10], the paper's Mach-10 cell width, ncells
    logU[128, 160]) with the nine-statistic system, each request running
    until max |d rho| / (rho_+ - rho_-) < steady_tol per step (or
    max_steps); continuous batching with graph-captured batch steps.  p50 /
    p99 latency from arrival to completion, and how many requests reached
    the tolerance."""
    from paper_2303_02898_gb300 import workloads
    t_arr, probs = workloads.serving_trace(nreq, seed=3, lo=128, hi=160, mach_lo=1.5, mach_hi=10.0)
    vctx = mem.Context.velocity(mem.shock_domain(mach=10.0))
    sv = mem.Server(vctx, hbm_budget_bytes=8 << 30, max_cells=1 << 16, steady_tol=steady_tol, max_steps=max_steps)
    ids, nxt = [], 0
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        while nxt < nreq and t_arr[nxt] <= now:
            p = probs[nxt]
            ids.append((sv.submit(mach=p.mach, ncells=p.ncells, xl=p.xl, xr=p.xr, ic=1, stats=9), p))
            nxt += 1
        sv.progress(chunk)
        st = sv.stats()
        if nxt == nreq and st["completed"] == nreq:
            break
        if st["resident"] == 0 and st["queued"] == 0 and nxt < nreq:
            time.sleep(max(0.0, t_arr[nxt] - (time.perf_counter() - t0)))
    wall = time.perf_counter() - t0
    res = [(sv.poll(i, ncells=p.ncells), p) for i, p in ids]
    sv.close()
    vctx.close()
    lat = np.array([r["latency_s"] for r, _ in res])
    steps = np.array([r["steps"] for r, _ in res])
    upd = sum(r["steps"] * p.ncells for r, p in res)
    return {
        "requests": nreq, "rate_per_s": 200.0, "mach": [1.5, 10.0], "ncells": [128, 160],
        "max_steps": max_steps, "steady_tol": steady_tol, "statistics": 9,
        "steady_requests": int(sum(r["steady"] for r, _ in res)),
        "steps_to_steady": {"min": int(steps.min()), "median": float(np.median(steps)), "max": int(steps.max())},
        "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
        "throughput": upd / wall, "unit": "cell-updates/s", "wall_s": wall,
        "all_finite": bool(all(np.isfinite(r["rho"]).all() for r, _ in res)),
        "graph": "each packed batch's step captured once and replayed"}


def run_serving_steady(mem, torch, np, nreq=32, max_steps=40000, chunk=200):
    """The steady-state serving trace at the stated tolerance (1e-6) and at
    2e-5: in FP32 the metric levels off between 1e-5 and 7e-5 per step on the
    paper's Mach-10 mesh, so few requests reach 1e-6."""
    return {"serving_steady_mach10_nine": {"tol_1e-06": _serving_steady(mem, torch, np, nreq, max_steps, chunk, 1e-6),
                                           "tol_2e-05": _serving_steady(mem, torch, np, nreq, max_steps, chunk, 2e-5)}}


def run_condition_study(mem, torch, np, steps=200, every=10):
    """Section 4, Fig. 7 analogue: the largest pivot-ratio estimate of
    cond(H) met over a run, against the number of cells, at Mach 4 (domain
    [-16.3, 16.3]) and Mach 10 ([-47.1, 47.1]); velocity-space rule, tanh
    start, sampled every `every` steps."""
    out = {}
    for mach, L in ((4.0, 16.3), (10.0, 47.1)):
        vctx = mem.Context.velocity(mem.shock_domain(mach=mach))
        rows = []
        for n in (32, 64, 100, 150, 200, 300):
            sh = mem.Shock(vctx, mach=mach, ncells=n, xl=-L, xr=L, ic=1, graph=1)
            worst, done, fin = 0.0, 0, True
            while done < steps:
                sh.step(every)
                done += every
                worst = max(worst, sh.condition(0))
                if not np.isfinite(sh.problem(0)["rho"]).all():
                    fin = False
                    break
            sh.close()
            rows.append({"cells": n, "max_cond": worst, "steps": done, "finite": fin})
        vctx.close()
        out["mach%g" % mach] = rows
    return {"condition_vs_cells": out}


GAUGE_BOX = (-30.7, 37.3, 34.0)  # Section 4: (u_x, u_r) in [-30.7, 37.3] x [0, 34.0]


def _status_letters(st):
    """One letter per cell: c converged (res <= tol), s stagnated (alpha <=
    alpha_min), m maxI reached, f stopped (Cholesky / non-finite)."""
    out = []
    for v in st:
        v = int(v)
        out.append("c" if v & 1 else "s" if v & 2 else "m" if v & 4 else "f")
    return "".join(out)


def _golden_beta(name):
    """FP64 parameters stored by tests/golden/make_gauge_study.py (oracle)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "gauge_study.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f).get(name)


def _log_mse(beta, ref, np):
    """log10 of the mean-square parameter error per cell (beta_1..34)."""
    d = beta[:, 1:].astype(np.float64) - np.asarray(ref, dtype=np.float64)[:, 1:]
    return [round(float(np.log10(max((r * r).mean(), 1e-300))), 2) for r in d]


def gauge_study_inputs(mem, torch, machs, gamma=5.0 / 3.0):
    """Upstream Maxwellians (n = 1, T = 1, v = sqrt(gamma) Mach) in their
    Hermite gauge (moments e_0) and in the trivial gauge (0, 1) (moments
    T(g0, gH) e_0, by mem_gauge_transform), each started from the uniform
    density: beta = 1/sqrt(2) on the three he_2 statistics cancels the
    gauge's Gaussian.  Returns (M, beta0, g) for [Hermite cells | trivial cells]."""
    dev = torch.device("cuda", torch.cuda.current_device())
    B = len(machs)
    gH = torch.zeros(B, 6, device=dev)
    gH[:, 0] = torch.tensor([gamma ** 0.5 * m for m in machs], device=dev)
    gH[:, 3:] = 1.0
    g0 = torch.zeros(B, 6, device=dev)
    g0[:, 3:] = 1.0
    eH = torch.zeros(B, 35, device=dev)
    eH[:, 0] = 1.0
    M0 = torch.zeros(B, 35, device=dev)
    ctx = mem.Context(8)
    ctx.gauge_transform(g0, gH, eH, M0)
    ctx.close()
    M = torch.cat([eH, M0]).contiguous()
    g = torch.cat([gH, g0]).contiguous()
    beta0 = torch.zeros(2 * B, 35, device=dev)
    beta0[:, 0] = 1.0
    beta0[:, 4] = beta0[:, 7] = beta0[:, 9] = 0.5 ** 0.5  # he_2 statistics (2,0,0), (0,2,0), (0,0,2)
    return M, beta0, g


def run_gauge_study(mem, torch, np):
    """Section 4, Fig. 3 analogue on the 35 statistics: Newton passes from
    the uniform density to the upstream Maxwellians of Mach 2-12, trivial
    gauge vs Hermite gauge, FP32, tol 1e-6 and 1e-9, maxI 500; and the
    log mean-square error of the FP32 parameters against FP64 ones (oracle,
    stored).  Velocity-space rule on the paper's box, 16 x 12 blocks of
    8-point Gauss-Legendre, 10 azimuths.  The solves return their solution
    (final_step = 1) so that the comparison with the exact FP64 parameters
    measures rounding, not the unapplied last Newton direction."""
    machs = list(range(2, 13))
    B = len(machs)
    vctx = mem.Context.velocity(GAUGE_BOX, nbx=16, nbr=12, ng=8, K=10)
    M, beta0, g = gauge_study_inputs(mem, torch, machs)
    ref_h, ref_t = _golden_beta("beta64_hermite"), _golden_beta("beta64_trivial")
    out = {"mach": machs}
    for tol in (1e-6, 1e-9):
        beta = beta0.clone()
        st = torch.zeros(M.shape[0], dtype=torch.int32, device=M.device)
        it = torch.zeros_like(st)
        vctx.solve_gauge(M, beta, g, st, it, tol=tol, maxI=500, final_step=1)
        torch.cuda.synchronize()
        itn, stn, bn = it.cpu().numpy(), st.cpu().numpy(), beta.cpu().numpy()
        row = {"passes_hermite": itn[:B].tolist(), "passes_trivial": itn[B:].tolist(),
               "status_hermite": _status_letters(stn[:B]), "status_trivial": _status_letters(stn[B:])}
        if ref_h is not None and ref_t is not None:
            row["log_mse_hermite"] = _log_mse(bn[:B], ref_h, np)
            row["log_mse_trivial"] = _log_mse(bn[B:], ref_t, np)
        out["tol_%g" % tol] = row
    vctx.close()
    return {"gauge_study": out}


def run_newton_study(mem, torch, np, n=26):
    """Section 4, Fig. 2 analogue: the he_3(u_x) moment M_(3,0,0) raised from
    0 to 0.5 on top of the equilibrium (n = 1, v = 0, T = 1) in the trivial
    gauge, solved in FP32 from beta = 0 by the modified Newton method
    (lambda I retries) and by plain Newton (no retries: a failed Cholesky
    stops the solve); tol 1e-8, maxI 500, the paper's box as above.  Then
    both methods on the gauge study's trivial-gauge cells at tol 1e-9."""
    dev = torch.device("cuda", torch.cuda.current_device())
    m4 = np.linspace(0.0, 0.5, n)
    vctx = mem.Context.velocity(GAUGE_BOX, nbx=16, nbr=12, ng=8, K=10)
    M = torch.zeros(n, 35, device=dev)
    M[:, 0] = 1.0
    M[:, 10] = torch.tensor(m4, dtype=torch.float32, device=dev)  # statistic (3,0,0)
    g = torch.zeros(n, 6, device=dev)
    g[:, 3:] = 1.0
    ref = _golden_beta("beta64_m4_sweep")
    out = {"m4": [round(float(x), 3) for x in m4]}
    for name, ml in (("modified", 20), ("plain", 0)):
        beta = torch.zeros(n, 35, device=dev)
        beta[:, 0] = 1.0
        st = torch.zeros(n, dtype=torch.int32, device=dev)
        it = torch.zeros_like(st)
        vctx.solve_gauge(M, beta, g, st, it, tol=1e-8, maxI=500, max_lambda=ml, final_step=1)
        torch.cuda.synchronize()
        bn = beta.cpu().numpy()
        row = {"passes": it.cpu().numpy().tolist(), "status": _status_letters(st.cpu().numpy()),
               "beta_300": [round(float(x), 6) for x in bn[:, 10]]}
        if ref is not None:
            row["log_mse"] = _log_mse(bn, ref, np)
        out[name] = row
    # The same comparison on the gauge study's trivial-gauge cells (Mach
    # 2-12, uniform start, tol 1e-9), where FP32 Hessians turn indefinite.
    machs = list(range(2, 13))
    B = len(machs)
    M, beta0, g = gauge_study_inputs(mem, torch, machs)
    M, beta0, g = M[B:].contiguous(), beta0[B:].contiguous(), g[B:].contiguous()
    row = {"mach": machs}
    for name, ml in (("modified", 20), ("plain", 0)):
        beta = beta0.clone()
        st = torch.zeros(B, dtype=torch.int32, device=dev)
        it = torch.zeros_like(st)
        vctx.solve_gauge(M, beta, g, st, it, tol=1e-9, maxI=500, max_lambda=ml, final_step=1)
        torch.cuda.synchronize()
        stn = st.cpu().numpy()
        row[name] = {"passes": it.cpu().numpy().tolist(), "status": _status_letters(stn),
                     "lambda_retries": int(((stn & 16) != 0).sum())}
    out["trivial_gauge_tol_1e-9"] = row
    vctx.close()
    return {"newton_study": out}


def run_convergence_study(mem, torch, np, t_end=4.0, Ns=(32, 64, 128, 256, 512, 1024, 2048)):
    """Section 4, Fig. 6 analogue: the Mach-4 shock on x in [-16.3, 16.3]
    (tanh start, thickness 5.44; velocity-space rule of 6 x 4 blocks of
    8-point Gauss-Legendre on the Rankine-Hugoniot box with (n_a, n_b, n_r)
    = (10, 6, 6), the paper's [-22.7, 16.1] x [0, 14.5]; tol 1e-9), solved
    with FLIC and with local Lax-Friedrichs on N cells, all N in one packed
    batch, each stopped at simulated time t_end.  L1 distance of sigma_xx
    from the finest mesh that stayed finite, averaged onto N cells.  FLIC is
    run again with the paper's own nine-statistic system (flic_nine), with
    the two other readings of its limiter (one phi per interface: the
    smallest of the nine statistics', or the density's), and on smaller
    velocity boxes (the mitigation the paper names for the ill-conditioning
    of over-refined meshes: (n_a, n_b, n_r) = (8, 5, 5) and (6, 4, 4))."""
    kw = dict(mach=4.0, xl=-16.3, xr=16.3, ic=1, thickness=5.44, tol=1e-9, na=10.0, nb=6.0, nr=6.0, t_end=t_end)
    vctx = mem.Context.velocity(mem.shock_domain(**kw), nbx=6, nbr=4, ng=8, K=12)
    L = kw["xr"] - kw["xl"]
    out = {"t_end": t_end}
    for name, scheme, stats, fl, box in (("flic", mem.SCHEME_FLIC, 35, 0, None), ("lf", mem.SCHEME_LF, 35, 0, None),
                                         ("flic_nine", mem.SCHEME_FLIC, 9, 0, None),
                                         ("flic_smallest_limiter", mem.SCHEME_FLIC, 9, 1, None),
                                         ("flic_density_limiter", mem.SCHEME_FLIC, 9, 2, None),
                                         ("flic_box_8_5_5", mem.SCHEME_FLIC, 35, 0, (8.0, 5.0, 5.0)),
                                         ("flic_nine_box_8_5_5", mem.SCHEME_FLIC, 9, 0, (8.0, 5.0, 5.0)),
                                         ("flic_nine_box_6_4_4", mem.SCHEME_FLIC, 9, 0, (6.0, 4.0, 4.0))):
        pkw = dict(kw)
        if box is not None:
            pkw.update(na=box[0], nb=box[1], nr=box[2])
        sh = mem.Shock(vctx, problems=[dict(ncells=N) for N in Ns], graph=1, scheme=scheme, stats=stats,
                       flic_limiter=fl, **pkw)
        t0 = time.time()
        # the finest mesh needs about t_end / (cfl dx / 10) steps
        max_steps = int(3 * t_end * 10.0 * Ns[-1] / (0.5 * L)) + 1000
        steps = 0
        while steps < max_steps:
            sh.step(200)
            steps += 200
            P = [sh.problem(i) for i in range(len(Ns))]
            if all(p["t"] >= t_end or not np.isfinite(p["rho"]).all() for p in P):
                break
        sh.close()
        fin = [bool(np.isfinite(p["sxx"]).all()) for p in P]
        r = max(i for i in range(len(Ns)) if fin[i]) if any(fin) else None
        row = {"cells": list(Ns), "finite": fin, "steps": steps, "wall_s": round(time.time() - t0, 1)}
        if box is not None:
            row["box"] = {"n_a_b_r": list(box), "domain": [round(x, 3) for x in mem.shock_domain(**pkw)]}
        if r is not None and r > 0:
            ref = P[r]["sxx"].astype(np.float64)
            err = []
            for i in range(r):
                proj = ref.reshape(Ns[i], len(ref) // Ns[i]).mean(1)
                err.append(float(np.abs(P[i]["sxx"].astype(np.float64) - proj).sum() * L / Ns[i]))
            row.update({"reference_cells": Ns[r], "l1_sxx": err,
                        "order": [round(float(np.log2(err[k] / err[k + 1])), 2) for k in range(len(err) - 1)]})
        out[name] = row
    vctx.close()
    return {"convergence_mach4": out}


def _serve_trace(mem, ctx, np, t_arr, probs, max_steps, chunk):
    """Replay a trace through the continuous-batching server; returns the
    per-request results, the wall time and the cell-updates done."""
    nreq = len(probs)
    sv = mem.Server(ctx, hbm_budget_bytes=40 << 30, max_cells=1 << 20, steady_tol=1e-6, max_steps=max_steps)
    ids, nxt = [], 0
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        while nxt < nreq and t_arr[nxt] <= now:
            p = probs[nxt]
            ids.append((sv.submit(mach=p.mach, ncells=p.ncells, xl=p.xl, xr=p.xr), p))
            nxt += 1
        sv.progress(chunk)
        st = sv.stats()
        if nxt == nreq and st["completed"] == nreq:
            break
        if st["resident"] == 0 and st["queued"] == 0 and nxt < nreq:
            time.sleep(max(0.0, t_arr[nxt] - (time.perf_counter() - t0)))
    wall = time.perf_counter() - t0
    res = [(sv.poll(i), p) for i, p in ids]
    sv.close()
    return res, wall, sum(r["steps"] * p.ncells for r, p in res)


def run_serving(mem, ctx, torch, np, nreq=32, max_steps=100, chunk=10):
    """Poisson trace (200 req/s, ncells logU[128, 32768], Mach U[1.5, 3]),
    each request capped at max_steps time steps: continuous batching (fused
    back-end) vs the same requests one at a time on the plain FP32 back-end.
    The offered load exceeds the GPU's capacity, so the trace is replayed a
    second time with its arrival times stretched to 0.8 x the capacity the
    first replay measured (requests/s = throughput / mean updates per request)."""
    from paper_2303_02898_gb300 import workloads
    t_arr, probs = workloads.serving_trace(nreq, seed=2, mach_hi=SHOCK_MACH)
    res, wall, upd = _serve_trace(mem, ctx, np, t_arr, probs, max_steps, chunk)
    lat = np.array([r["latency_s"] for r, _ in res])
    capacity = (upd / wall) / (upd / nreq)
    rate2 = 0.8 * capacity
    res2, wall2, upd2 = _serve_trace(mem, ctx, np, np.asarray(t_arr) * (200.0 / rate2), probs, max_steps, chunk)
    lat2 = np.array([r["latency_s"] for r, _ in res2])
    # one at a time: each request alone, back to back, same number of steps
    t1 = time.perf_counter()
    for r, p in res:
        sh = mem.Shock(ctx, mach=p.mach, ncells=p.ncells, xl=p.xl, xr=p.xr, graph=0, impl=mem.IMPL_PLAIN)
        sh.step(r["steps"])
        sh.close()
    torch.cuda.synchronize()
    seq = time.perf_counter() - t1
    return {"serving": {"requests": nreq, "rate_per_s": 200.0, "max_steps": max_steps,
                        "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                        "throughput": upd / wall, "unit": "cell-updates/s", "wall_s": wall,
                        "one_at_a_time_throughput": upd / seq, "one_at_a_time_wall_s": seq,
                        "capacity_req_per_s": capacity,
                        "at_0.8_capacity": {"rate_per_s": rate2, "p50_latency_s": float(np.percentile(lat2, 50)),
                                            "p99_latency_s": float(np.percentile(lat2, 99)),
                                            "throughput": upd2 / wall2, "wall_s": wall2}}}


def residual_stats(ctx, torch, np, M, beta, n=65536):
    """FP64 relative moment residuals (mem_residual64 on the GPU) of the first
    n cells: the acceptance quantity (<= 1e-5), per result."""
    n = min(n, M.shape[0])
    res = torch.zeros(n, dtype=torch.float64, device=M.device)
    ctx.residual64(M[:n], beta[:n].contiguous(), res)
    r = res.cpu().numpy()
    return {"cells": n, "max": float(r.max()), "median": float(np.median(r)), "p99": float(np.percentile(r, 99)),
            "above_1e-5": int((r > 1e-5).sum())}


def run_as_drawn(mem, ctx, torch, np, opts, B=1 << 18):
    """The standalone workload as stated, without the redraw of the (a, b)
    that give a density a second mode: how many cells are bimodal, and how
    the solve ends on them and on the rest (FP64 residual by mem_residual64)."""
    from paper_2303_02898_gb300 import workloads
    dev = torch.device("cuda", torch.cuda.current_device())
    t = workloads.solve_targets(B, seed=0, redraw=False)
    T32 = lambda a: torch.tensor(a, dtype=torch.float32, device=dev).contiguous()  # noqa: E731
    M = torch.zeros(B, 35, device=dev)
    g = torch.zeros(B, 6, device=dev)
    ctx.targets(T32(t.v), T32(t.T), T32(t.a), T32(t.b), M, g, gen_order=24)
    beta = torch.zeros_like(M)
    st = torch.zeros(B, dtype=torch.int32, device=dev)
    ctx.solve(M, beta, st, None, opts=opts)
    res = torch.zeros(B, dtype=torch.float64, device=dev)
    ctx.residual64(M, beta, res)
    r, s = res.cpu().numpy(), st.cpu().numpy()
    bi = t.bimodal
    conv = (s & 3) != 0
    out = {"cells": B, "bimodal_cells": int(bi.sum()),
           "converged_unimodal": float(conv[~bi].mean()), "converged_bimodal": float(conv[bi].mean()) if bi.any() else None,
           "residual_above_1e-5_unimodal": int((r[~bi] > 1e-5).sum()),
           "residual_above_1e-5_bimodal": int((r[bi] > 1e-5).sum()),
           "residual_max_bimodal": float(np.nanmax(r[bi])) if bi.any() else None,
           "note": "the moments of a bimodal cell come from a 24^3 Gauss-Hermite rule centred on the density's "
                   "main mode, which misses a far second mode"}
    return {"solve_as_drawn": out}


def run_mixed(mem, ctx, torch, np, M, beta, st, it, plain_value, B):
    """The mixed-precision back-end (tensor-core contraction: split TF32
    moments, TF32 Hessian; FP64 residual of failed cells) on the headline
    batch, against the plain FP32 back-end."""
    opts = mem.default_opts(impl=mem.IMPL_MIXED, final_step=1)
    beta.zero_()
    ctx.solve(M, beta, st, it, opts=opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n = 2
    for _ in range(n):
        beta.zero_()
        ctx.solve(M, beta, st, it, opts=opts)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / n
    stn, itn = st.cpu().numpy(), it.cpu().numpy()
    v = B / (ms * 1e-3)
    return {"mixed_tc": {"value": v, "unit": "cell-solves/s", "ms_per_step": ms,
                         "mean_passes": float(itn.mean()),
                         "converged": float(np.mean((stn & 3) != 0)),
                         "fp64_ok_cells": int(((stn & mem.ST_FP64_OK) != 0).sum()),
                         "residual_fp64": residual_stats(ctx, torch, np, M, beta),
                         "precision": "moments split TF32 (3 products), Hessian 1 TF32 product, FP32 accumulation "
                                      "on tcgen05; line search, Cholesky and solves FP32"},
            "mixed_over_plain_fp32": v / plain_value}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------- CPU oracle
def cpu_baseline(order, sample, seed=0):
    from oracle import oracle as O
    from paper_2303_02898_gb300 import workloads
    t = workloads.solve_targets(sample, seed=seed)
    M, _ = O.target_batch(24, t.v, t.T, t.a, t.b)
    t0 = time.perf_counter()
    O.solve_batch(order, M, final_step=True)
    dt = time.perf_counter() - t0
    return {"value": sample / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": "first %d cells of the same workload (seed %d), FP64 Algorithm 1, Q=%d^3, OpenMP" % (sample, seed, order),
            "seconds": dt}


def run_reference(args, rank):
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2303_02898_gb300 import workloads
    sample = 2048
    t = workloads.solve_targets(sample, seed=0)
    M, _ = O.target_batch(24, t.v, t.T, t.a, t.b)
    for _ in range(args.warmup):
        O.solve_batch(args.order, M, final_step=True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.solve_batch(args.order, M, final_step=True)
    dt = time.perf_counter() - t0
    value = sample * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, sample),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": "%d cells of the workload per step (seed 0)" % sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(args, cells):
    return {"workload": "batched standalone max-entropy solves: 35 moments (degree <= 4 in 3D velocity), "
                        "targets from seeded polynomial log-densities (v~N(0,3^2), T~logU[0.5,20], cubic~N(0,0.05^2), "
                        "quartic~-U(0.01,0.1)), cold start beta=0",
            "cells_per_gpu": cells, "quadrature": "Gauss-Hermite %d^3 in the Hermite gauge" % args.order,
            "algorithm": "Algorithm 1 (paper constants, tol 1e-8, maxI 500) plus its final Newton step "
                         "(final_step=1, library extension)",
            "moments": 35, "l2": "inputs larger than L2 (M 147 MB read, beta 147 MB written per step)"}


# ---------------------------------------------------------------- profiler cases
def _timed_ms(torch, fn, n):
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(n):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / n


def run_case(name, n):
    """Kernel-focused runs for profilers and quick timing: inputs built on the
    device (seeded, synthetic), two warm-up iterations, then the timed ones;
    one line with the mean time per iteration (CUDA events).
      solve [cells]       mem_solve, fused back-end, 8^3 rule (default 2^20 cells)
      mixed [cells]       the same with the mixed (tensor-core) back-end
      plain [cells]       the same with the plain FP32 back-end
      ensemble [steps]    256-problem shock batch, 8^3 rule (Mach <= 3)
      mach10 [steps]      256-problem Mach 1.2-10 batch, velocity-space rule
      mach10flic [steps]  the same batch with FLIC interface fluxes
      mach10nine, mach10flicnine [steps]  the same with the nine-statistic system
      config4 [steps]     the stated 256-problem ensemble (970k cells), nine statistics"""
    import numpy as np
    import torch
    from paper_2303_02898_gb300 import mem, workloads
    dev = torch.device("cuda:0")
    if name in ("solve", "mixed", "plain"):
        impl = {"solve": mem.IMPL_FUSED, "mixed": mem.IMPL_MIXED, "plain": mem.IMPL_PLAIN}[name]
        cells = n or (1 << 20)
        ctx = mem.Context(8)
        t = workloads.solve_targets(cells, seed=0)
        T32 = lambda a: torch.tensor(a, dtype=torch.float32, device=dev).contiguous()  # noqa: E731
        M = torch.zeros(cells, 35, device=dev)
        g = torch.zeros(cells, 6, device=dev)
        ctx.targets(T32(t.v), T32(t.T), T32(t.a), T32(t.b), M, g, gen_order=24)
        beta = torch.zeros(cells, 35, device=dev)
        st = torch.zeros(cells, dtype=torch.int32, device=dev)

        def run():
            beta.zero_()
            ctx.solve(M, beta, st, impl=impl, final_step=1)
        for _ in range(2):
            run()
        ms = _timed_ms(torch, run, 2)
        print("%s cells=%d ms=%.3f cell-solves/s=%.4g" % (name, cells, ms, cells / ms * 1e3))
        ctx.close()
    elif name == "ensemble":
        ctx = mem.Context(8)
        probs = workloads.ensemble_problems(256, seed=1, mach_hi=3.0)
        sh = mem.Shock(ctx, problems=[dict(mach=p.mach, ncells=p.ncells, xl=p.xl, xr=p.xr) for p in probs], graph=1)
        sh.step(2)
        cells = sum(p.ncells for p in probs)
        ms = _timed_ms(torch, lambda: sh.step(1), n or 3)
        print("ensemble cells=%d ms/step=%.3f cell-updates/s=%.4g" % (cells, ms, cells / ms * 1e3))
        sh.close()
        ctx.close()
    elif name == "config4":
        vctx = mem.Context.velocity(mem.shock_domain(mach=10.0))
        probs = workloads.ensemble_problems(256, seed=1)
        sh = mem.Shock(vctx, problems=[dict(mach=p.mach, ncells=p.ncells, xl=p.xl, xr=p.xr) for p in probs], ic=1,
                       graph=1, stats=9)
        sh.step(2)
        cells = sum(p.ncells for p in probs)
        ms = _timed_ms(torch, lambda: sh.step(1), n or 3)
        print("%s cells=%d ms/step=%.3f cell-updates/s=%.4g" % (name, cells, ms, cells / ms * 1e3))
        sh.close()
        vctx.close()
    elif name in ("mach10", "mach10flic", "mach10nine", "mach10flicnine"):
        scheme = mem.SCHEME_FLIC if "flic" in name else mem.SCHEME_LF
        vctx = mem.Context.velocity(mem.shock_domain(mach=10.0))
        rng = np.random.default_rng(7)
        probs = [dict(mach=float(m), ncells=150, xl=-47.1, xr=47.1) for m in rng.uniform(1.2, 10.0, 256)]
        sh = mem.Shock(vctx, problems=probs, ic=1, graph=1, scheme=scheme, stats=9 if "nine" in name else 35)
        sh.step(2)
        cells = 150 * len(probs)
        ms = _timed_ms(torch, lambda: sh.step(1), n or 3)
        print("%s cells=%d ms/step=%.3f cell-updates/s=%.4g" % (name, cells, ms, cells / ms * 1e3))
        sh.close()
        vctx.close()
    else:
        raise SystemExit("unknown case %r" % name)


# ---------------------------------------------------------------- GPU arm
def whole_job(dist, ms_local, cells_local, device):
    """Weak scaling: every rank solves its own shard (its own seed), so the
    job's step time is the slowest rank's and its work the sum of the shards.
    Returns (max ms over ranks, total cells); no reduction without dist."""
    import torch
    if dist is None:
        return ms_local, cells_local
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(cells_local)], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(c.item()))


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.case:
        return run_case(args.case[0], int(args.case[1]) if len(args.case) > 1 else 0)

    import numpy as np
    import torch
    from paper_2303_02898_gb300 import mem, workloads
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    B = args.cells
    ctx = mem.Context(args.order)
    t = workloads.solve_targets(B, seed=rank)
    T32 = lambda a: torch.tensor(a, dtype=torch.float32, device=dev).contiguous()  # noqa: E731
    M = torch.zeros(B, 35, device=dev)
    g = torch.zeros(B, 6, device=dev)
    ctx.targets(T32(t.v), T32(t.T), T32(t.a), T32(t.b), M, g, gen_order=24)
    beta = torch.zeros_like(M)
    st = torch.zeros(B, dtype=torch.int32, device=dev)
    it = torch.zeros(B, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    # Algorithm 1 plus its final Newton step (final_step = 1, a library
    # extension): the 1e-5 residual bar is on the solution, not on the
    # iterate one direction behind it; the literal order is reported beside.
    opts = mem.default_opts(impl=mem.IMPL_FUSED, final_step=1)
    # launch shape of the persistent solve kernel from the autotuner, timed
    # on the first 2^18 cells of this batch (set-up, not timed)
    nt = min(B, 1 << 18)
    tuning = ctx.tune(mem.TUNE_FUSED, M[:nt], torch.zeros(nt, 35, device=dev), reps=2, opts=opts)
    bw, bb, bms = tuning["candidates"][tuning["best"]]
    tuning = {"kernel": "k_fused_solve<%d, warps>" % args.order, "cells": nt,
              "candidates": [{"warps": w, "blocks_per_sm": b, "ms": round(ms, 3)} for w, b, ms in tuning["candidates"]],
              "chosen": {"warps": bw, "blocks_per_sm": bb}, "gain_over_default": tuning["default_ms"] / bms}

    def step():
        beta.zero_()
        ctx.solve(M, beta, st, it, opts=opts)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        beta.zero_()
        ev[k][0].record(stream)
        ctx.solve(M, beta, st, it, opts=opts)
        ev[k][1].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    ms_total, cells_total = whole_job(dist, e0.elapsed_time(e1), B, dev)
    ms = ms_total / args.steps
    kern_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    value = cells_total / (ms * 1e-3)
    itn = it.cpu().numpy()
    stn = st.cpu().numpy()
    passes = int(itn.sum())
    flops = passes * fused_flops_per_pass(args.order)
    peaks = measured_peaks(mem)
    peak_fp32 = peaks["fp32_tflops"]
    achieved = flops / (kern_ms * 1e-3) / 1e12
    # the dense contraction the method defines (exponent 2 x 35 Q per
    # evaluation, moments + packed Hessian 2 Q 665, Cholesky and solves):
    # 0.77 MFLOP per cell-iteration at Q = 512, against the TF32 tensor rate
    Q = args.order ** 3
    dense_per_pass = 2 * 35 * Q * 2 + 2 * Q * 665 + 34 ** 3 / 3 + 2 * 34 * 34
    dense_achieved = passes * dense_per_pass / (kern_ms * 1e-3) / 1e12
    conv = float(np.mean((stn & (mem.ST_CONVERGED | mem.ST_STAGNATED)) != 0))
    solve_stats = {"converged_fraction": conv, "mean_passes": passes / B, "max_passes": int(itn.max()),
                   "order": "final Newton step applied (final_step=1)",
                   "residual_fp64": residual_stats(ctx, torch, np, M, beta)}
    # Algorithm 1's own order (the last direction not applied), same batch
    lit = mem.default_opts(impl=mem.IMPL_FUSED, final_step=0)
    beta.zero_()
    ctx.solve(M, beta, st, it, opts=lit)
    solve_stats["literal_order"] = {"order": "Algorithm 1 as printed (final_step=0)",
                                    "residual_fp64": residual_stats(ctx, torch, np, M, beta),
                                    "mean_passes": float(it.float().mean())}

    # ---- end to end through the C ABI from pinned host buffers: mem_solve_host
    # streams the batch through the device in chunks, the host <-> device
    # copies of one chunk overlapping the solve of the next (cold start:
    # beta from 0, as in the device-resident step)
    M_h = M.cpu().pin_memory()
    beta_h = torch.zeros(B, 35).pin_memory()
    st_h = torch.zeros(B, dtype=torch.int32).pin_memory()

    def e2e_step():
        ctx.solve_host(M_h, beta_h, st_h, None, warm=False, opts=opts, stream=stream)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    a1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = max_over_ranks(a0.elapsed_time(a1)) / args.steps
    e2e = {"value": B * world / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": B * 35 * 4,
           "d2h_bytes_per_step": B * 35 * 4 + B * 4}

    extras = {}
    if not args.no_extras:
        # plain FP32 back-end (separate kernels, host loop) on the same batch
        popts = mem.default_opts(impl=mem.IMPL_PLAIN)
        beta.zero_()
        ctx.solve(M, beta, st, it, opts=popts)
        torch.cuda.synchronize()
        p0 = time.perf_counter()
        nplain = 2
        for _ in range(nplain):
            beta.zero_()
            ctx.solve(M, beta, st, it, opts=popts)
        torch.cuda.synchronize()
        pms = (time.perf_counter() - p0) * 1e3 / nplain
        extras["plain_fp32"] = {"value": B / (pms * 1e-3), "unit": UNIT, "ms_per_step": pms,
                                "converged": float(np.mean((st.cpu().numpy() & 3) != 0))}
        extras["tuned_over_plain"] = value / world / extras["plain_fp32"]["value"]
        extras.update(run_mixed(mem, ctx, torch, np, M, beta, st, it, extras["plain_fp32"]["value"], B))
        extras.update(run_as_drawn(mem, ctx, torch, np, opts))
        # 12^3 rule, tuned
        ctx12 = mem.Context(12)
        M12 = torch.zeros(B, 35, device=dev)
        g12 = torch.zeros(B, 6, device=dev)
        ctx12.targets(T32(t.v), T32(t.T), T32(t.a), T32(t.b), M12, g12, gen_order=24)
        for _ in range(2):
            beta.zero_()
            ctx12.solve(M12, beta, st, it, opts=opts)
        torch.cuda.synchronize()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for _ in range(3):
            beta.zero_()
            ctx12.solve(M12, beta, st, it, opts=opts)
        q1.record(stream)
        torch.cuda.synchronize()
        extras["tuned_q12"] = {"value": B / (q0.elapsed_time(q1) / 3 * 1e-3), "unit": UNIT,
                               "mean_passes": float(it.float().mean())}
        ctx12.close()
        del M12, g12
        extras.update(run_mach10(mem, torch, np))
        # Mach 3 from a step on the Gauss-Hermite rule: 4096 cells at the
        # paper's cell width 0.628, graph-captured fused step vs plain
        for impl, graph, nst in ((mem.IMPL_FUSED, 1, 200), (mem.IMPL_PLAIN, 0, 10)):
            L = 0.5 * 4096 * 0.628
            sh = mem.Shock(ctx, mach=SHOCK_MACH, ncells=4096, xl=-L, xr=L, impl=impl, graph=graph, ic=0)
            sh.step(3)
            torch.cuda.synchronize()
            s0 = time.perf_counter()
            sh.step(nst)
            torch.cuda.synchronize()
            sdt = time.perf_counter() - s0
            d = sh.get()
            key = "shock_mach%g_%s" % (SHOCK_MACH, "tuned" if impl == mem.IMPL_FUSED else "plain")
            extras[key] = {"value": 4096 * nst / sdt, "unit": "cell-updates/s", "steps": nst,
                           "ms_per_step": 1e3 * sdt / nst, "sim_time": d["t"], "ic": "step", "cells": 4096,
                           "domain": [-L, L], "finite": bool(np.isfinite(d["M"]).all())}
            sh.close()
        extras.update(run_ensemble(mem, ctx, torch, np))
        extras.update(run_serving(mem, ctx, torch, np))
        extras.update(run_serving_mach10(mem, torch, np))
        extras.update(run_ensemble_config4(mem, torch, np))
        extras.update(run_serving_config5(mem, torch, np))
        extras.update(run_serving_steady(mem, torch, np))
        extras.update(run_condition_study(mem, torch, np))
        extras.update(run_gauge_study(mem, torch, np))
        extras.update(run_newton_study(mem, torch, np))
        extras.update(run_convergence_study(mem, torch, np))

    cfg = workload_config(args, B)
    cfg["redrawn_cells"] = int(t.redrawn)
    cfg["redraw_note"] = ("cells whose first (a, b) draw gives the density a second mode are redrawn "
                          "(solve_as_drawn reports the workload without it)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": cfg,
            "e2e": e2e, "gpu_launches": args.steps,
            "clocks": clocks,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_fp32, "unit": "TFLOP/s",
                         "frac": achieved / peak_fp32, "traffic": traffic_bytes(),
                         "kernel": "k_fused_solve<%d>" % args.order, "kernel_ms": kern_ms,
                         "flops_per_launch": flops, "newton_passes": passes,
                         "peak_note": "of measured: FP32 FMA rate of mem_bench_peak on this GPU (CUDA events); "
                                      "flops = the sum-factorised kernel's own count per Newton pass",
                         "dense_equivalent": {"flops_per_pass": dense_per_pass, "achieved": dense_achieved,
                                              "peak": peaks["tf32_tc_tflops"],
                                              "frac": dense_achieved / peaks["tf32_tc_tflops"],
                                              "note": "the dense contraction's algorithmic flops (0.77 MFLOP per "
                                                      "cell-iteration at Q=512) over the measured TF32 tensor rate"}},
            "measured_peaks": peaks, "autotune": tuning,
            "solve_stats": solve_stats}
    line.update(extras)
    if rank == 0 and world == 1 and not args.no_cpu:
        # about 13 s of FP64 solves on the GPU host's 16 cores (~9.8k cells/s)
        line["cpu_baseline"] = cpu_baseline(args.order, 131072)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
