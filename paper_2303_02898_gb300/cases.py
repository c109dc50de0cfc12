"""Kernel-focused runs of the library, for profilers and quick timing.

    python -m paper_2303_02898_gb300.cases solve [cells]       # mem_solve, fused back-end, 8^3 rule
    python -m paper_2303_02898_gb300.cases ensemble [steps]    # 256-problem shock batch, 8^3 rule (Mach <= 3)
    python -m paper_2303_02898_gb300.cases mach10 [steps]      # 256-problem Mach 1.2-10 batch, velocity-space rule
    python -m paper_2303_02898_gb300.cases mach10flic [steps]  # the same batch with FLIC interface fluxes

Each case builds its inputs on the device (seeded, synthetic), runs a few
warm-up iterations and then the timed ones, and prints one line with the
mean time per iteration (CUDA events).  Nothing here reads the oracle.
"""
import sys

import numpy as np
import torch

from . import mem, workloads


def _timed(fn, n):
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(n):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / n


def solve(cells=1 << 20, iters=2):
    dev = torch.device("cuda:0")
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
        ctx.solve(M, beta, st)
    for _ in range(2):
        run()
    ms = _timed(run, iters)
    print("solve cells=%d ms=%.3f cell-solves/s=%.4g" % (cells, ms, cells / ms * 1e3))
    ctx.close()


def ensemble(steps=3):
    ctx = mem.Context(8)
    probs = workloads.ensemble_problems(256, seed=1, mach_hi=3.0)
    sh = mem.Shock(ctx, problems=[dict(mach=p.mach, ncells=p.ncells, xl=p.xl, xr=p.xr) for p in probs], graph=1)
    sh.step(2)
    cells = sum(p.ncells for p in probs)
    ms = _timed(lambda: sh.step(1), steps)
    print("ensemble cells=%d ms/step=%.3f cell-updates/s=%.4g" % (cells, ms, cells / ms * 1e3))
    sh.close()
    ctx.close()


def mach10(steps=3, scheme=mem.SCHEME_LF):
    vctx = mem.Context.velocity(mem.shock_domain(mach=10.0))
    rng = np.random.default_rng(7)
    probs = [dict(mach=float(m), ncells=150, xl=-47.1, xr=47.1) for m in rng.uniform(1.2, 10.0, 256)]
    sh = mem.Shock(vctx, problems=probs, ic=1, graph=1, scheme=scheme)
    sh.step(2)
    cells = 150 * len(probs)
    ms = _timed(lambda: sh.step(1), steps)
    print("mach10 scheme=%d cells=%d ms/step=%.3f cell-updates/s=%.4g" % (scheme, cells, ms, cells / ms * 1e3))
    sh.close()
    vctx.close()


if __name__ == "__main__":
    case = sys.argv[1] if len(sys.argv) > 1 else "solve"
    arg = [int(a) for a in sys.argv[2:3]]
    {"solve": solve, "ensemble": ensemble, "mach10": mach10,
     "mach10flic": lambda *a: mach10(*a, scheme=mem.SCHEME_FLIC)}[case](*arg)
