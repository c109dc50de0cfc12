"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances: the acceptance test of the solve is the relative moment residual
||E phi(beta) - M/n|| / ||M/n|| <= 1e-5, evaluated by the oracle in FP64 at
the same quadrature; shock profiles rho, u_x, T agree within 1e-3 in L-inf
after normalisation by the upstream-downstream jump.  Other quantities are
compared at FP32-rounding level, with bounds stated per test.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RES_TOL = 1e-5
PROFILE_TOL = 1e-3
# Algorithm 1 returns beta one Newton direction behind its last pass (the
# default on both sides); final_step = 1 applies that direction, which the
# 1e-5 residual bar needs (the FP64 oracle leaves up to 2.5e-4 on the
# standalone targets in the literal order).  Acceptance tests use the
# extension on both sides; the literal order has its own tests below.
EXT = dict(final_step=1)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def mem():
    from paper_2303_02898_gb300 import mem as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def ctx8(mem, dev):
    c = mem.Context(8)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx12(mem, dev):
    c = mem.Context(12)
    yield c
    c.close()


def T32(a, dev):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device=dev).contiguous()


def np64(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def random_gauges(rng, B):
    w = rng.normal(0, 2.0, (B, 3))
    s = np.exp(rng.uniform(np.log(0.5), np.log(3.0), (B, 3)))
    return np.concatenate([w, s], axis=1)


# ------------------------------------------------------------------ gauge
def test_gauge_transform_matches_oracle(O, mem, ctx8, dev):
    rng = np.random.default_rng(20)
    B = 67
    g1, g2 = random_gauges(rng, B), random_gauges(rng, B)
    g1[:, 3:] = g2[:, 3:] * np.exp(rng.uniform(-0.3, 0.3, (B, 3)))
    g1[:, :3] = g2[:, :3] + rng.normal(0, 0.5, (B, 3)) * g2[:, 3:]
    M = np.zeros((B, 35))
    M[:, 0] = 1.0
    M[:, 1:] = rng.normal(0, 0.1, (B, 34))
    out = torch.zeros(B, 35, device=dev)
    ctx8.gauge_transform(T32(g1, dev), T32(g2, dev), T32(M, dev), out)
    got = np64(out)
    Mf = np64(T32(M, dev))
    g1f, g2f = np64(T32(g1, dev)), np64(T32(g2, dev))
    for c in range(B):
        ref = O.gauge_T(g1f[c], g2f[c]) @ Mf[c]
        scale = np.abs(O.gauge_T(g1f[c], g2f[c])).max() * np.abs(Mf[c]).max()
        assert np.abs(got[c] - ref).max() <= 2e-6 * scale, c


@pytest.mark.parametrize("axisym", [False, True])
def test_hermite_gauge_and_beta_transport(O, mem, ctx8, dev, axisym):
    rng = np.random.default_rng(21 + axisym)
    B = 45
    g = random_gauges(rng, B)
    if axisym:
        g[:, 1:3] = 0.0
        g[:, 5] = g[:, 4]
    M = np.zeros((B, 35))
    M[:, 0] = np.exp(rng.uniform(-1, 1, B))
    M[:, 1:] = rng.normal(0, 0.08, (B, 34)) * M[:, :1]
    beta = np.zeros((B, 35))
    beta[:, 0] = M[:, 0]
    beta[:, 1:] = rng.normal(0, 0.02, (B, 34))
    Mt, gt, bt = T32(M, dev), T32(g, dev), T32(beta, dev)
    Mf, gf, bf = np64(Mt), np64(gt), np64(bt)
    gout = torch.zeros(B, 6, device=dev)
    Mout = torch.zeros(B, 35, device=dev)
    ctx8.gauge_hermite(Mt, gt, gout, Mout, bt, axisym=axisym)
    go, Mo, bo = np64(gout), np64(Mout), np64(bt)
    for c in range(B):
        gH = O.hermite_gauge(Mf[c], gf[c], axisym=axisym)
        assert np.abs(go[c] - gH).max() <= 1e-5 * (1 + np.abs(gH).max()), c
        MH = O.transform_M(gH, gf[c], Mf[c])
        assert np.abs(Mo[c] - MH).max() <= 2e-5 * np.abs(Mf[c]).max() * 10, c
        bH = O.transform_beta(gH, gf[c], bf[c])
        assert np.abs(bo[c] - bH).max() <= 2e-5 * (1 + np.abs(bH).max()) * 10, c


# ------------------------------------------------------------------ solve
def _solve(mem, ctx, M, dev, impl, beta0=None, **kw):
    Mt = M if torch.is_tensor(M) else T32(M, dev)
    B = Mt.shape[0]
    beta = torch.zeros_like(Mt) if beta0 is None else T32(beta0, dev)
    st = torch.full((B,), -1, dtype=torch.int32, device=dev)
    it = torch.full((B,), -1, dtype=torch.int32, device=dev)
    ctx.solve(Mt, beta, st, it, impl=impl, **kw)
    torch.cuda.synchronize()
    return np64(Mt), np64(beta), st.cpu().numpy(), it.cpu().numpy()


@pytest.mark.parametrize("impl", [0, 1])
def test_solve_perturbed_moments(O, mem, ctx8, dev, impl):
    from paper_2303_02898_gb300 import workloads
    M = workloads.perturbed_hermite_moments(1003, seed=3, scale=0.04)   # ragged: not a multiple of 4 or 32
    Mf, b, st, it = _solve(mem, ctx8, M, dev, impl, **EXT)
    ok = (st & (mem.ST_CONVERGED | mem.ST_STAGNATED)) != 0
    assert ok.all(), np.unique(st, return_counts=True)
    assert (it >= 1).all() and (it <= 20).all()
    assert np.all(b[:, 0] == Mf[:, 0])
    bo, sto, ito = O.solve_batch(8, Mf, final_step=True)
    res = O.residual_batch(8, b, Mf)
    assert res.max() <= RES_TOL, res.max()
    assert np.abs(b[:, 1:] - bo[:, 1:]).max() <= 1e-4
    # same path through Algorithm 1: iteration counts agree except on a few
    assert np.mean(np.abs(it - ito) <= 1) > 0.95


@pytest.mark.parametrize("order", [8, 12])
def test_targets_and_solve_match_oracle(O, mem, dev, order, ctx8, ctx12):
    from paper_2303_02898_gb300 import workloads
    ctx = ctx8 if order == 8 else ctx12
    t = workloads.solve_targets(333, seed=5)
    B = len(t.T)
    Mg = torch.zeros(B, 35, device=dev)
    gg = torch.zeros(B, 6, device=dev)
    ctx.targets(T32(t.v, dev), T32(t.T, dev), T32(t.a, dev), T32(t.b, dev), Mg, gg, gen_order=24)
    Mo, go = O.target_batch(24, t.v, t.T, t.a, t.b)
    Mgn, ggn = np64(Mg), np64(gg)
    assert np.abs(Mgn - Mo).max() <= 2e-5, np.abs(Mgn - Mo).max()
    assert np.abs(ggn - go).max() <= 2e-5 * (1 + np.abs(go).max())
    for impl in (0, 1):
        _, b, st, it = _solve(mem, ctx, Mg, dev, impl, **EXT)
        ok = (st & (mem.ST_CONVERGED | mem.ST_STAGNATED)) != 0
        assert ok.all(), (impl, np.unique(st, return_counts=True))
        res = O.residual_batch(order, b, Mgn)
        assert res.max() <= RES_TOL, (impl, res.max(), np.argmax(res))
        bo, _, _ = O.solve_batch(order, Mgn, final_step=True)
        assert np.abs(b[:, 1:] - bo[:, 1:]).max() <= 5e-3, (impl, np.abs(b[:, 1:] - bo[:, 1:]).max())


def test_solve_edge_cases(O, mem, ctx8, dev):
    # empty batch is a no-op
    e = torch.zeros(0, 35, device=dev)
    ctx8.solve(e, e.clone())
    # invalid inputs are flagged per cell, valid neighbours still solve
    M = np.zeros((5, 35))
    M[:, 0] = [1.0, -1.0, 0.0, 1.0, 2.0]
    M[3, 7] = np.nan
    M[4, 10] = 0.02
    _, b, st, it = _solve(mem, ctx8, M, dev, 1)
    assert st[1] == mem.ST_BADINPUT and st[2] == mem.ST_BADINPUT and st[3] == mem.ST_BADINPUT
    assert it[1] == 0 and st[0] & mem.ST_CONVERGED and st[4] & mem.ST_CONVERGED
    assert np.abs(b[0, 1:]).max() < 1e-6 and it[0] == 1
    # warm start at the solution takes one pass
    from paper_2303_02898_gb300 import workloads
    Mw = workloads.perturbed_hermite_moments(64, seed=9, scale=0.03)
    Mf, b1, _, _ = _solve(mem, ctx8, Mw, dev, 1, **EXT)
    _, b2, st2, it2 = _solve(mem, ctx8, Mf, dev, 1, beta0=b1, **EXT)
    assert (it2 <= 2).all() and np.abs(b2 - b1).max() < 1e-4
    # the default is the literal order of Algorithm 1 (no final step): the
    # same passes, beta one Newton direction behind
    _, b3, st3, it3 = _solve(mem, ctx8, Mf, dev, 1)
    _, b4, st4, it4 = _solve(mem, ctx8, Mf, dev, 1, **EXT)
    assert (st3 & mem.ST_CONVERGED).all() and np.array_equal(it3, it4)
    assert 0.0 < np.abs(b3 - b4).max() < 1e-3


@pytest.mark.parametrize("impl", [0, 1])
@pytest.mark.parametrize("order", [8, 12])
@pytest.mark.parametrize("workload", ["perturbed", "targets"])
def test_literal_order_matches_oracle(O, mem, dev, ctx8, ctx12, impl, order, workload):
    """Algorithm 1 as printed (beta returned without the last direction), on
    both sides.  Where the GPU and the oracle take the same number of passes
    they return the same iterate, so beta agrees element-wise; the moment
    residual of that iterate, evaluated by the oracle in FP64, is one Newton
    step's worth and matches the oracle's own literal-order residual."""
    from paper_2303_02898_gb300 import workloads
    ctx = ctx8 if order == 8 else ctx12
    if workload == "perturbed":
        M = workloads.perturbed_hermite_moments(517, seed=31, scale=0.04)
        Mt = T32(M, dev)
    else:
        t = workloads.solve_targets(257, seed=13)
        Mt = torch.zeros(len(t.T), 35, device=dev)
        gg = torch.zeros(len(t.T), 6, device=dev)
        ctx.targets(T32(t.v, dev), T32(t.T, dev), T32(t.a, dev), T32(t.b, dev), Mt, gg, gen_order=24)
    Mf, b, st, it = _solve(mem, ctx, Mt, dev, impl, final_step=0)
    assert ((st & (mem.ST_CONVERGED | mem.ST_STAGNATED)) != 0).all()
    bo, sto, ito = O.solve_batch(order, Mf, final_step=False)
    same = it == ito
    assert same.mean() > 0.85, same.mean()
    scale = 1.0 + np.abs(bo[:, 1:]).max(axis=1)
    err = np.abs(b[:, 1:] - bo[:, 1:]).max(axis=1) / scale
    assert err[same].max() <= (1e-4 if workload == "perturbed" else 5e-3), err[same].max()
    res, res_o = O.residual_batch(order, b, Mf), O.residual_batch(order, bo, Mf)
    # the literal order's residual is set by the last direction, the same
    # on both sides where the pass counts agree
    assert np.all(res[same] <= 1.5 * res_o[same] + RES_TOL), np.max(res[same] - 1.5 * res_o[same])
    print("literal order %s q%d impl %d: passes equal on %.3f; residual median %.2e p99 %.2e max %.2e "
          "(oracle max %.2e); cells above 1e-5: %d of %d" % (
              workload, order, impl, same.mean(), np.median(res), np.percentile(res, 99), res.max(), res_o.max(),
              int((res > RES_TOL).sum()), len(res)))


def test_plain_and_fused_agree(O, mem, ctx8, dev):
    from paper_2303_02898_gb300 import workloads
    M = workloads.perturbed_hermite_moments(513, seed=11, scale=0.05)
    _, bp, stp, itp = _solve(mem, ctx8, M, dev, 0)
    _, bf, stf, itf = _solve(mem, ctx8, M, dev, 1)
    assert np.abs(bp - bf).max() < 1e-4
    assert np.mean(itp == itf) > 0.9


# ------------------------------------------------------------------ flux
@pytest.mark.parametrize("order", [8, 12])
def test_flux_and_speed_match_oracle(O, mem, dev, order, ctx8, ctx12):
    ctx = ctx8 if order == 8 else ctx12
    rng = np.random.default_rng(30 + order)
    B = 70
    deg = O.basis_index().sum(1)
    # FP32 speeds lose ~1e-7 cond(E[phi phi^T]) relative accuracy; the
    # degree-3/4 parameters are scaled so that cond stays below ~1e5 (on the
    # outer nodes of the 12-point rule he_4 reaches ~60, so 12^3 takes 0.3x).
    f = 1.0 if order == 8 else 0.3
    scale = np.where(deg <= 2, 0.1, np.where(deg == 3, 0.03 * f, 0.01 * f))
    beta = rng.normal(0, 1, (B, 35)) * scale
    beta[:, 0] = np.exp(rng.uniform(-0.5, 0.5, B))
    M = np.zeros((B, 35))
    M[:, 0] = beta[:, 0]
    g = random_gauges(rng, B)
    Mt, bt, gt = T32(M, dev), T32(beta, dev), T32(g, dev)
    F = torch.zeros(B, 35, device=dev)
    sp = torch.zeros(B, device=dev)
    ctx.flux(Mt, bt, gt, F, sp)
    Fg, spg = np64(F), np64(sp)
    bf, gf, Mf = np64(bt), np64(gt), np64(Mt)
    for c in range(B):
        Fo, so, lo, hi = O.flux(order, bf[c], gf[c], Mf[c, 0])
        assert np.abs(Fg[c] - Fo).max() <= 2e-5 * np.abs(Fo).max(), c
        assert spg[c] == pytest.approx(so, rel=2e-5), (c, spg[c], so)
    # Maxwellian: |w_x| + sqrt(5 + sqrt 10) s_x
    Mx = torch.zeros(4, 35, device=dev)
    Mx[:, 0] = 1.0
    gx = T32([[0.0, 0, 0, 1, 1, 1], [2.0, 0, 0, 0.5, 1, 1], [-3.0, 0, 0, 2.0, 1, 1], [12.9, 0, 0, 1.0, 1, 1]], dev)
    spx = torch.zeros(4, device=dev)
    ctx.flux(Mx, Mx.clone(), gx, None, spx)
    r = math.sqrt(5 + math.sqrt(10))
    exp = [r, 2 + 0.5 * r, 3 + 2 * r, 12.9 + r]
    assert np.allclose(np64(spx), exp, rtol=1e-5)


@pytest.mark.parametrize("order", [8, 12])
def test_axisym_flux_matches_full_pencil(O, mem, dev, order, ctx8, ctx12):
    """mem_flux_axisym on cells symmetric in u_y and u_z: the largest speed
    over the parity blocks of (b mod 2, c mod 2) is the full-pencil speed
    (Eq. "The lax F"), against mem_flux and the FP64 oracle."""
    ctx = ctx8 if order == 8 else ctx12
    rng = np.random.default_rng(50 + order)
    B = 70
    idx = O.basis_index()
    deg = idx.sum(1)
    odd = (idx[:, 1] % 2 == 1) | (idx[:, 2] % 2 == 1)
    f = 1.0 if order == 8 else 0.3
    scale = np.where(deg <= 2, 0.1, np.where(deg == 3, 0.03 * f, 0.01 * f))
    beta = rng.normal(0, 1, (B, 35)) * scale
    beta[:, odd] = 0.0
    beta[:, 0] = np.exp(rng.uniform(-0.5, 0.5, B))
    M = np.zeros((B, 35))
    M[:, 0] = beta[:, 0]
    g = random_gauges(rng, B)
    g[:, 1:3] = 0.0
    Mt, bt, gt = T32(M, dev), T32(beta, dev), T32(g, dev)
    F1, F2 = torch.zeros(B, 35, device=dev), torch.zeros(B, 35, device=dev)
    s1, s2 = torch.zeros(B, device=dev), torch.zeros(B, device=dev)
    ctx.flux(Mt, bt, gt, F1, s1)
    ctx.flux_axisym(Mt, bt, gt, F2, s2)
    F1, F2, s1, s2 = np64(F1), np64(F2), np64(s1), np64(s2)
    assert np.abs(F1 - F2).max() <= 1e-6 * np.abs(F1).max()
    assert np.allclose(s2, s1, rtol=2e-5, atol=0)
    bf, gf = np64(bt), np64(gt)
    for c in range(B):
        _, so, _, _ = O.flux(order, bf[c], gf[c], M[c, 0])
        assert s2[c] == pytest.approx(so, rel=2e-5), (c, s2[c], so)


def test_axisym_flux_on_shock_states(mem, ctx8, dev):
    """States of a Mach-3 shock (tanh initial state, 5 steps; odd-parity
    parameters are zero only to solver rounding): parity-block and
    full-pencil speeds agree."""
    sh = mem.Shock(ctx8, mach=3.0, ncells=48, xl=-15.0, xr=15.0, ic=1, graph=0)
    sh.step(5)
    st = sh.get()
    sh.close()
    Mt, bt, gt = T32(st["M"], dev), T32(st["beta"], dev), T32(st["g"], dev)
    B = Mt.shape[0]
    s1, s2 = torch.zeros(B, device=dev), torch.zeros(B, device=dev)
    ctx8.flux(Mt, bt, gt, None, s1)
    ctx8.flux_axisym(Mt, bt, gt, None, s2)
    assert np.allclose(np64(s2), np64(s1), rtol=2e-5, atol=0)


# ------------------------------------------------------------------ shock
def _norm(q, a, b):
    return (q - a) / (b - a)


@pytest.mark.parametrize("impl,graph", [(1, 1), (1, 0), (0, 0)])
def test_shock_mach15_matches_oracle(O, mem, ctx8, dev, impl, graph):
    """Mach 1.5, 64 cells on [-20, 20], step initial state, 20 steps, CFL 0.5."""
    sh = mem.Shock(ctx8, mach=1.5, ncells=64, xl=-20.0, xr=20.0, impl=impl, graph=graph)
    sh.step(20)
    out = sh.get()
    sh.close()
    so = O.Shock(1.5, 64, -20.0, 20.0)
    for _ in range(20):
        so.step()
    rho, ux, T = so.profile()
    assert out["t"] == pytest.approx(so.t, rel=1e-5)
    for name, g_, o_, a, b in (("rho", out["rho"], rho, so.n_up, so.n_dn), ("ux", out["ux"], ux, so.v_up, so.v_dn),
                               ("T", out["T"], T, so.T_up, so.T_dn)):
        err = np.abs(_norm(g_, a, b) - _norm(o_, a, b)).max()
        assert err <= PROFILE_TOL, (name, err)
    assert np.abs(out["M"] - so.M).max() <= 1e-3 * np.abs(so.M).max()


def test_shock_conserves_on_gpu(O, mem, ctx8, dev):
    sh = mem.Shock(ctx8, mach=1.5, ncells=64, xl=-20.0, xr=20.0)
    d0 = sh.get()
    sh.step(10)
    d1 = sh.get()
    sh.close()

    def totals(d):
        tot = np.zeros(3)
        for c in range(1, 65):
            n, v, T, _ = O.macro(d["M"][c].astype(np.float64), d["g"][c].astype(np.float64))
            tot += [n, n * v[0], 0.5 * n * (v @ v + 3 * T)]
        return tot

    t0, t1 = totals(d0), totals(d1)
    assert np.abs(t1 - t0).max() <= 2e-5 * np.abs(t0).max()


def test_shock_uniform_state_steady(mem, ctx8, dev):
    sh = mem.Shock(ctx8, mach=2.0, ncells=32, xl=1.0, xr=33.0)
    d0 = sh.get()
    metric = sh.step(3, steady=True)
    d1 = sh.get()
    sh.close()
    assert np.abs(d1["M"] - d0["M"]).max() < 1e-5 and metric < 1e-5


# ------------------------------------------------------------------ full size
def test_full_size_solve_sampled(O, mem, ctx8, dev):
    """2^20 cells, the standalone-solve workload, in the launch configuration
    the benchmark times; residuals of a seeded sample checked by the oracle."""
    from paper_2303_02898_gb300 import workloads
    B = 1 << 20
    t = workloads.solve_targets(B, seed=0)
    Mg = torch.zeros(B, 35, device=dev)
    gg = torch.zeros(B, 6, device=dev)
    ctx8.targets(T32(t.v, dev), T32(t.T, dev), T32(t.a, dev), T32(t.b, dev), Mg, gg, gen_order=24)
    beta = torch.zeros_like(Mg)
    st = torch.zeros(B, dtype=torch.int32, device=dev)
    it = torch.zeros(B, dtype=torch.int32, device=dev)
    ctx8.solve(Mg, beta, st, it, **EXT)
    torch.cuda.synchronize()
    stn = st.cpu().numpy()
    conv = (stn & (mem.ST_CONVERGED | mem.ST_STAGNATED)) != 0
    assert conv.mean() > 0.999, np.unique(stn, return_counts=True)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(B, 256, replace=False))
    idx = np.concatenate([idx, [0, B - 1]])
    b = beta[idx].double().cpu().numpy()
    M = Mg[idx].double().cpu().numpy()
    res = O.residual_batch(8, b, M)
    ok = conv[idx]
    assert res[ok].max() <= RES_TOL, res.max()


@pytest.mark.parametrize("order", [8, 12])
def test_solve_host_matches_device(O, mem, dev, order, ctx8, ctx12):
    """mem_solve_host streams host arrays through the device in chunks of
    262,144 cells with the copies overlapped: more than one chunk and a
    ragged tail here.  Same kernel per cell, so beta, status and iters equal
    mem_solve's bit for bit, cold (beta from 0) and warm (beta_host read);
    a sample meets the oracle's residual bar."""
    from paper_2303_02898_gb300 import workloads
    ctx = ctx8 if order == 8 else ctx12
    B = 300_001 if order == 8 else 270_000
    t = workloads.solve_targets(B, seed=5)
    Mg = torch.zeros(B, 35, device=dev)
    gg = torch.zeros(B, 6, device=dev)
    ctx.targets(T32(t.v, dev), T32(t.T, dev), T32(t.a, dev), T32(t.b, dev), Mg, gg, gen_order=24)
    beta_d = torch.zeros_like(Mg)
    st_d = torch.zeros(B, dtype=torch.int32, device=dev)
    it_d = torch.zeros(B, dtype=torch.int32, device=dev)
    ctx.solve(Mg, beta_d, st_d, it_d, **EXT)
    M_h = Mg.cpu().pin_memory()
    beta_h = torch.full((B, 35), float("nan")).pin_memory()   # cold start: never read
    st_h = torch.zeros(B, dtype=torch.int32).pin_memory()
    it_h = torch.zeros(B, dtype=torch.int32).pin_memory()
    ctx.solve_host(M_h, beta_h, st_h, it_h, warm=False, **EXT)
    torch.cuda.synchronize()
    assert torch.equal(beta_h, beta_d.cpu())
    assert torch.equal(st_h, st_d.cpu()) and torch.equal(it_h, it_d.cpu())
    # warm start from a perturbed solution, against mem_solve from the same start
    start = beta_d.clone()
    start[:, 1:] *= 0.9
    beta_w = start.clone()
    ctx.solve(Mg, beta_w, st_d, it_d, **EXT)
    beta_hw = start.cpu().pin_memory()
    ctx.solve_host(M_h, beta_hw, st_h, it_h, warm=True, **EXT)
    torch.cuda.synchronize()
    assert torch.equal(beta_hw, beta_w.cpu())
    assert torch.equal(st_h, st_d.cpu()) and torch.equal(it_h, it_d.cpu())
    idx = np.concatenate([np.random.default_rng(1).choice(B, 48, replace=False), [0, B - 1]])
    conv = (st_h.numpy()[idx] & mem.ST_CONVERGED) != 0
    res = O.residual_batch(order, beta_h[idx].double().numpy(), M_h[idx].double().numpy())
    assert conv.all() and res.max() <= RES_TOL, res.max()
    # a single cell (one chunk of one), and the plain back-end, which uses the
    # scratch itself: refused
    b1 = torch.zeros(1, 35).pin_memory()
    ctx.solve_host(M_h[:1].clone().pin_memory(), b1, **EXT)
    torch.cuda.synchronize()
    assert torch.equal(b1, beta_h[:1])
    with pytest.raises(RuntimeError):
        ctx.solve_host(M_h[:8], beta_h[:8], impl=mem.IMPL_PLAIN)


def test_context_scratch_ordered_across_streams(O, mem, dev):
    """The dense flux path (and the plain back-end) share the context's
    scratch.  Calls made on two streams of one context are ordered on the GPU
    by the context's event, so each result equals the same call made alone."""
    from paper_2303_02898_gb300 import workloads
    ctx = mem.Context(10)   # no fused kernel at order 10: the flux uses the scratch
    rng = np.random.default_rng(43)
    Ms, bs, gs = [], [], []
    for k, B in enumerate((3000, 2000, 2500)):
        M = workloads.perturbed_hermite_moments(B, seed=44 + k, scale=0.04)
        Mt = T32(M, dev)
        b = torch.zeros_like(Mt)
        ctx.solve(Mt, b, impl=mem.IMPL_PLAIN)
        Ms.append(Mt)
        bs.append(b)
        gs.append(T32(np.concatenate([rng.normal(0, 1.0, (B, 3)), np.exp(rng.uniform(-0.5, 0.5, (B, 3)))], 1), dev))
    torch.cuda.synchronize()

    def run(streams):
        outs = [(torch.zeros_like(M), torch.zeros(M.shape[0], device=dev)) for M in Ms]
        for s in streams:
            s.wait_stream(torch.cuda.current_stream())
        for k in range(3):   # flux 0 and 2 on the first stream, flux 1 on the second
            st = streams[k % 2]
            with torch.cuda.stream(st):
                ctx.flux(Ms[k], bs[k], gs[k], outs[k][0], outs[k][1], stream=st)
        torch.cuda.synchronize()
        return [np64(x) for o in outs for x in o]

    s0 = torch.cuda.current_stream()
    alone = run([s0, s0])
    both = run([torch.cuda.Stream(), torch.cuda.Stream()])
    for x, y in zip(alone, both):
        assert np.array_equal(x, y)
    ctx.close()
