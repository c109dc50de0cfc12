"""GPU parity for the gauge and modified-Newton studies of Section 4 (the
Fig. 3 and Fig. 2 setups, on the 35 statistics) against the FP64 oracle.

Velocity-space rule on the paper's box (u_x, u_r) in [-30.7, 37.3] x
[0, 34.0], 16 x 12 blocks of 8-point Gauss-Legendre, 10 azimuths, as stored
with the FP64 solutions in tests/golden/gauge_study.json.

- Hermite gauge, upstream Maxwellians of Mach 2-12 from the uniform density:
  every cell converges at tol 1e-6 and 1e-9 in the oracle's FP64 number of
  passes, +-1 (in exact arithmetic the pass count is gauge-invariant, so the
  FP64 count is the target for both gauges), and meets the relative-residual
  bar of the velocity tests (1e-5, or 4x the residual of the FP64 solution
  rounded to FP32) plus 1.1x the residual the oracle's own solve leaves at
  the same tolerance (0.1-0.2 at tol 1e-6, ~1e-9 at tol 1e-9).
- Trivial gauge: the same problems; at tol 1e-9 FP32 needs more passes than
  the Hermite gauge (the paper's Fig. 3 finding) -- checked on the total.
- M_(3,0,0) sweep 0 -> 0.5 in the trivial gauge: the modified Newton method
  converges everywhere and meets the residual bar; plain Newton (no lambda I
  retries) is bit-identical to it on every cell where no retry happened.
"""
import json
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RES_TOL = 1e-5


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def mem(dev):
    from paper_2303_02898_gb300 import mem as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def gold(O):
    d = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "gauge_study.json")))
    r = d["rule"]
    O.set_velocity_rule(r["rule_id"], r["ax"], r["bx"], r["nbx"], r["br"], r["nbr"], r["ng"], r["K"])
    return d


@pytest.fixture(scope="module")
def vctx(mem, gold):
    r = gold["rule"]
    c = mem.Context.velocity((r["ax"], r["bx"], r["br"]), nbx=r["nbx"], nbr=r["nbr"], ng=r["ng"], K=r["K"])
    yield c
    c.close()


def T32(a, dev):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device=dev).contiguous()


def np64(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def uniform_beta(O, B):
    b = np.zeros((B, 35))
    b[:, 0] = 1.0
    for a, bb, c in ((2, 0, 0), (0, 2, 0), (0, 0, 2)):
        b[:, O.index_of(a, bb, c)] = 1.0 / math.sqrt(2.0)
    return b


@pytest.fixture(scope="module")
def problems(O, gold):
    """(M, g) of the Hermite-gauge cells, then the trivial-gauge cells."""
    machs = gold["mach"]
    B = len(machs)
    g0 = np.tile([0.0, 0.0, 0.0, 1.0, 1.0, 1.0], (B, 1))
    gH = g0.copy()
    gH[:, 0] = [math.sqrt(5.0 / 3.0) * m for m in machs]
    e0 = np.zeros((B, 35))
    e0[:, 0] = 1.0
    Mt = np.array([O.transform_M(g0[i], gH[i], e0[i]) for i in range(B)])
    return np.concatenate([e0, Mt]), np.concatenate([gH, g0])


def solve(vctx, M, g, beta0, dev, **kw):
    B = M.shape[0]
    Mt, gt, bt = T32(M, dev), T32(g, dev), T32(beta0, dev)
    st = torch.zeros(B, dtype=torch.int32, device=dev)
    it = torch.zeros(B, dtype=torch.int32, device=dev)
    # The studies compare FP32 parameters with exact FP64 ones, so the solve
    # returns its solution (final_step = 1): in Algorithm 1's own order the
    # unapplied last direction (about sqrt(2 tol)) would hide the rounding.
    kw.setdefault("final_step", 1)
    vctx.solve_gauge(Mt, bt, gt, st, it, maxI=500, **kw)
    return np64(bt), np64(st).astype(int), np64(it).astype(int), np64(Mt), np64(gt)


def residual_ok(O, rule, beta, M, g, beta64, res_same_tol=0.0):
    """Residual bar; res_same_tol is the residual of the oracle's own solve at
    the same tolerance and start.  At tol 1e-6 Algorithm 1 stops on the
    Newton decrement while the density is still wider than the Maxwellian
    (H is large there), leaving a relative moment residual of 0.1-0.2 in FP64
    too; where the FP32 path stops depends on its rounding, so that residual
    is matched to 10%."""
    res = O.residual(rule, beta, M, g)
    floor = O.residual(rule, np.asarray(beta64).astype(np.float32).astype(np.float64), M, g)
    return res <= max(RES_TOL, 4.0 * floor) + 1.1 * res_same_tol, (res, floor, res_same_tol)


@pytest.mark.parametrize("tol", [1e-6, 1e-9])
def test_hermite_gauge_passes_match_fp64(O, vctx, gold, problems, dev, tol):
    M, g = problems
    B = len(gold["mach"])
    beta, st, it, Mf, gf = solve(vctx, M, g, uniform_beta(O, 2 * B), dev, tol=tol)
    ref = np.array(gold["passes64_hermite_tol_%g" % tol])
    assert np.array_equal(ref, np.array(gold["passes64_trivial_tol_%g" % tol]))
    assert np.all(st[:B] & 1), st[:B]
    assert np.abs(it[:B] - ref).max() <= 1, (it[:B], ref)
    rule = gold["rule"]["rule_id"]
    bo, sto, ito = O.solve_batch(rule, Mf[:B], beta0=uniform_beta(O, B), tol=tol, g=gf[:B], final_step=True)
    assert np.abs(ito - ref).max() <= 1, (ito, ref)
    for c in range(B):
        ok, info = residual_ok(O, rule, beta[c], Mf[c], gf[c], gold["beta64_hermite"][c],
                               O.residual(rule, bo[c], Mf[c], gf[c]))
        assert ok, (gold["mach"][c], info)
    if tol == 1e-9:
        assert it[B:].sum() > it[:B].sum(), (it[B:], it[:B])
    assert np.all(st & 8 == 0), st


def test_m4_sweep_modified_and_plain_newton(O, vctx, gold, dev):
    m4 = np.array(gold["m4"])
    n = len(m4)
    M = np.zeros((n, 35))
    M[:, 0] = 1.0
    M[:, O.index_of(3, 0, 0)] = m4
    g = np.tile([0.0, 0.0, 0.0, 1.0, 1.0, 1.0], (n, 1))
    b0 = np.zeros((n, 35))
    b0[:, 0] = 1.0
    bm, stm, itm, Mf, gf = solve(vctx, M, g, b0, dev, tol=1e-8)
    bp, stp, itp, _, _ = solve(vctx, M, g, b0, dev, tol=1e-8, max_lambda=0)
    assert np.all(stm & 1), stm
    rule = gold["rule"]["rule_id"]
    for c in range(n):
        ok, info = residual_ok(O, rule, bm[c], Mf[c], gf[c], gold["beta64_m4_sweep"][c])
        assert ok, (m4[c], info)
    same = (stm & 16) == 0
    assert np.array_equal(bm[same], bp[same])
    assert np.array_equal(itm[same], itp[same])
    # plain Newton stops (lambda cap) exactly where the modified method retried
    assert np.all((stp[~same] & 32) != 0)


def test_trivial_gauge_needs_lambda_retries(O, vctx, gold, problems, dev):
    """Trivial gauge, tol 1e-9: near convergence FP32 rounding leaves the
    Hessians of the faster Maxwellians (cond ~1e7 in this gauge) numerically
    indefinite, so the modified method retries with lambda I and still
    converges, while plain Newton stops (lambda cap) at the first such pass;
    the Hermite gauge never needs a retry.  Cells without a retry are
    bit-identical under both methods."""
    M, g = problems
    B = len(gold["mach"])
    u0 = uniform_beta(O, 2 * B)
    bm, stm, itm, _, _ = solve(vctx, M, g, u0, dev, tol=1e-9)
    bp, stp, itp, _, _ = solve(vctx, M, g, u0, dev, tol=1e-9, max_lambda=0)
    assert np.all(stm & 1), stm
    assert np.all(stm[:B] & 16 == 0), stm[:B]
    lam = (stm & 16) != 0
    assert lam[B:].any(), stm[B:]
    assert np.all(stp[lam] & 32), stp
    assert np.all(itp[lam] <= itm[lam]), (itp, itm)
    assert np.array_equal(bm[~lam], bp[~lam])
    assert np.array_equal(itm[~lam], itp[~lam])
