"""GPU parity for the velocity-space quadrature (block Gauss-Legendre in
u_x and u_r, equispaced azimuths; the rule of the paper's shock runs, Section
3.1 and Appendix D) against the FP64 oracle with the same rule.

Tolerances: the solve is accepted on the relative moment residual
||E phi(beta) - M/n|| / ||M/n|| <= 1e-5 (FP64, same rule), or, where the
exact solution rounded to FP32 already exceeds that (ill-conditioned cells),
within 4x of that rounding floor; fluxes agree to
2e-5 of max |F|; shock profiles to 1e-3 after normalisation by the jump.
Characteristic speeds of strongly non-equilibrium cells are
ill-conditioned generalised eigenvalues (FP32 loses ~1e-7 cond(E[phi phi^T])),
so they are compared at 1e-3 relative.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MACH = 10.0
RULE = 210   # oracle rule id of the velocity-space rule
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
def dom(O):
    d = O.shock_domain(MACH)
    O.set_velocity_rule(RULE, d[0], d[1], 6, d[2], 4, 8, 12)
    return d


@pytest.fixture(scope="module")
def vctx(mem, dom):
    c = mem.Context.velocity(dom, nbx=6, nbr=4, ng=8, K=12)
    yield c
    c.close()


@pytest.fixture(scope="module")
def states(O, dom):
    """Interior cells of the oracle's Mach-10 tanh initial state (two-Maxwellian
    mixtures in their Hermite gauges) with their FP64 parameters."""
    so = O.Shock(MACH, 24, -15.0, 15.0, order=RULE, ic="tanh", thickness=15.7, final_step=True)
    return so.M[1:-1].copy(), so.g[1:-1].copy(), so.beta[1:-1].copy()


def T32(a, dev):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device=dev).contiguous()


def np64(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def test_velocity_rule_shape(vctx, dom):
    shape, d = vctx.velocity_rule()
    assert shape == (6, 4, 8, 12)
    assert d == pytest.approx(dom, rel=1e-12)


def test_velocity_solve_matches_oracle(O, mem, vctx, states, dev):
    M, g, _ = states
    B = M.shape[0]
    Mt, gt = T32(M, dev), T32(g, dev)
    beta = torch.zeros(B, 35, device=dev)
    st = torch.zeros(B, dtype=torch.int32, device=dev)
    it = torch.zeros(B, dtype=torch.int32, device=dev)
    # the acceptance bar is on the solution: the final Newton step applied
    vctx.solve_gauge(Mt, beta, gt, st, it, final_step=1)
    stn, bn = np64(st).astype(int), np64(beta)
    assert np.all(stn & 3), stn
    assert np.all(stn & 8 == 0)
    Mf, gf = np64(Mt), np64(gt)
    _, _, beta_o = states
    relaxed = 0
    for c in range(B):
        res = O.residual(RULE, bn[c], Mf[c], gf[c])
        # Storing the exact (FP64) solution in FP32 already leaves this
        # residual; for the stiffest mixed cells (cond(H) ~ 4e5) it exceeds
        # 1e-5, so no FP32 beta can meet 1e-5 there.
        floor = O.residual(RULE, beta_o[c].astype(np.float32).astype(np.float64), Mf[c], gf[c])
        assert res <= max(RES_TOL, 4.0 * floor), (c, res, floor)
        relaxed += int(res > RES_TOL)
    # cells that needed the relaxed bar (above 1e-5, below 4x the floor)
    print("velocity solve: %d of %d cells above 1e-5 (within 4x their FP32 floor)" % (relaxed, B))
    assert relaxed <= B // 4, relaxed


def test_velocity_solve_rejects_plain_entry(mem, vctx, dev):
    M = torch.zeros(2, 35, device=dev)
    M[:, 0] = 1.0
    with pytest.raises(RuntimeError):
        vctx.solve(M, torch.zeros(2, 35, device=dev))


@pytest.mark.parametrize("axisym", [True, False])
def test_velocity_flux_matches_oracle(O, mem, vctx, states, dev, axisym):
    M, g, beta = states
    B = M.shape[0]
    Mt, bt, gt = T32(M, dev), T32(beta, dev), T32(g, dev)
    F = torch.zeros(B, 35, device=dev)
    sp = torch.zeros(B, device=dev)
    (vctx.flux_axisym if axisym else vctx.flux)(Mt, bt, gt, F, sp)
    Fg, spg = np64(F), np64(sp)
    bf, gf, Mf = np64(bt), np64(gt), np64(Mt)
    for c in range(B):
        Fo, so, _, _ = O.flux(RULE, bf[c], gf[c], Mf[c, 0])
        assert np.abs(Fg[c] - Fo).max() <= 2e-5 * np.abs(Fo).max(), c
        assert spg[c] == pytest.approx(so, rel=1e-3), (c, spg[c], so)


def _norm(q, a, b):
    return (q - a) / (b - a)


def test_velocity_shock_mach10_matches_oracle(O, mem, vctx, dom):
    """Mach 10, 40 cells on [-12.5, 12.5] (cell width 0.625, the paper's
    Mach-10 mesh spacing), tanh initial state, 10 steps, CFL 0.5."""
    sh = mem.Shock(vctx, mach=MACH, ncells=40, xl=-12.5, xr=12.5, ic=1, graph=1)
    sh.step(10)
    out = sh.get()
    sh.close()
    so = O.Shock(MACH, 40, -12.5, 12.5, order=RULE, ic="tanh", thickness=15.7)
    for _ in range(10):
        so.step()
    rho, ux, T = so.profile()
    assert out["t"] == pytest.approx(so.t, rel=1e-4)
    for name, g_, o_, a, b in (("rho", out["rho"], rho, so.n_up, so.n_dn), ("ux", out["ux"], ux, so.v_up, so.v_dn),
                               ("T", out["T"], T, so.T_up, so.T_dn)):
        err = np.abs(_norm(g_, a, b) - _norm(o_, a, b)).max()
        assert err <= 1e-3, (name, err)
    assert np.isfinite(out["M"]).all()


def test_velocity_shock_batch_alone_equals_mix(mem, vctx):
    """Problems of different Mach numbers (each with its own domain) packed in
    one batch give the profiles they give alone."""
    probs = [dict(mach=10.0, ncells=30, xl=-9.4, xr=9.4), dict(mach=4.0, ncells=24, xl=-8.0, xr=8.0)]
    sh = mem.Shock(vctx, problems=probs, ic=1, graph=0)
    sh.step(6)
    for i, pr in enumerate(probs):
        mix = sh.problem(i)
        a = mem.Shock(vctx, ic=1, graph=0, **pr)
        a.step(6)
        alone = a.problem(0)
        a.close()
        for k in ("rho", "ux", "T"):
            assert np.abs(alone[k] - mix[k]).max() <= 1e-6 * np.abs(alone[k]).max(), (i, k)
    sh.close()


def test_velocity_shock_condition_matches_oracle(O, mem, vctx, dom):
    """Fig. 7 diagnostic (Section 4): the largest pivot-ratio estimate of
    cond(H) over a Mach-10 problem's cells after each of four steps.  GPU: the
    FP32 factorisation of the last Newton pass; oracle: FP64 at its converged
    beta.  They agree to the FP32 accuracy of the smallest pivot (relative
    error up to ~1e-7 cond(H), about 1e-2 here) plus the size of the final
    Newton step; the bar is 10 %."""
    sh = mem.Shock(vctx, mach=MACH, ncells=40, xl=-12.5, xr=12.5, ic=1, graph=0)
    so = O.Shock(MACH, 40, -12.5, 12.5, order=RULE, ic="tanh", thickness=15.7)
    so.track_cond = True
    for k in range(4):
        sh.step(1)
        so.step()
        cg, co = sh.condition(0), float(so.cond[1:-1].max())
        assert co > 10.0
        assert cg == pytest.approx(co, rel=0.1), (k, cg, co)
    sh.close()


@pytest.mark.parametrize("scheme", ["lf", "flic"])
@pytest.mark.parametrize("stats", [35, 9])
def test_paper_mesh_mach10_matches_oracle(mem, scheme, stats):
    """The paper's Mach-10 run (Section 4): 150 cells on [-47.1, 47.1], tanh
    start, velocity-space rule on the Rankine-Hugoniot box; 100 local
    Lax-Friedrichs steps or 60 FLIC steps against the FP64 oracle's profiles
    (tests/golden/mach10_paper_mesh.json, written by make_mach10_paper_mesh.py
    from the oracle only), in both statistics systems."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "mach10_paper_mesh.json")))
    g = gold[scheme]
    vctx = mem.Context.velocity(gold["rule"]["box"], nbx=6, nbr=4, ng=8, K=12)
    sh = mem.Shock(vctx, mach=10.0, ncells=150, xl=-47.1, xr=47.1, ic=1, thickness=15.7, graph=1, stats=stats,
                   scheme=mem.SCHEME_FLIC if scheme == "flic" else mem.SCHEME_LF)
    sh.step(g["steps"])
    out = sh.get()
    sh.close()
    vctx.close()
    assert out["t"] == pytest.approx(g["t"], rel=1e-4)
    for k, i in (("rho", 0), ("ux", 1), ("T", 2)):
        a, b = g["up"][i], g["down"][i]
        err = np.abs(_norm(out[k], a, b) - _norm(np.array(g[k]), a, b)).max()
        assert err <= 1e-3, (k, err)
