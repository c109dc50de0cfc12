"""The paper's nine-statistic system on the GPU (mem_solve_axi and shock
problems with stats = 9) against the FP64 oracle's own nine-statistic solve
(or_solve_axi / or_flux_axi, Appendix B) and its 35-statistic shock.

Tolerances: the solve's acceptance bar is the 35-statistic relative moment
residual (the nine-statistic solution is the 35-statistic one for an
axisymmetric cell), 1e-5, or 4 x the FP32 floor of the exact solution for
the stiffest Mach-10 cells (as for the 35-statistic velocity-space solve);
fluxes within 2e-5 of max |F|; speeds within 1e-3 (generalised eigenvalues of
FP32 pencils); shock profiles within 1e-3 after normalisation.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MACH = 10.0
RULE35, RULE9 = 202, 203   # oracle rule ids: 12 azimuths / 1 azimuth, same (u_x, u_r) blocks
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
    O.set_velocity_rule(RULE35, d[0], d[1], 6, d[2], 4, 8, 12)
    O.set_velocity_rule(RULE9, d[0], d[1], 6, d[2], 4, 8, 1)
    return d


@pytest.fixture(scope="module")
def vctx(mem, dom):
    c = mem.Context.velocity(dom, nbx=6, nbr=4, ng=8, K=12)
    yield c
    c.close()


@pytest.fixture(scope="module")
def states(O, dom):
    """Interior cells of the oracle's Mach-10 tanh initial state, exact FP64
    parameters (final step applied)."""
    so = O.Shock(MACH, 24, -15.0, 15.0, order=RULE35, ic="tanh", thickness=15.7, final_step=True)
    return so.M[1:-1].copy(), so.g[1:-1].copy(), so.beta[1:-1].copy()


def T32(a, dev):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device=dev).contiguous()


def np64(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def test_axi_solve_matches_oracle(O, mem, vctx, states, dev):
    M, g, beta_exact = states
    B = M.shape[0]
    V = O.flic_basis()
    Mt, gt = T32(M, dev), T32(g, dev)
    beta = torch.zeros(B, 35, device=dev)
    st = torch.zeros(B, dtype=torch.int32, device=dev)
    it = torch.zeros(B, dtype=torch.int32, device=dev)
    vctx.solve_axi(Mt, beta, gt, st, it, final_step=1)
    stn, bn, itn = np64(st).astype(int), np64(beta), np64(it).astype(int)
    assert np.all(stn & 3), stn
    Mf, gf = np64(Mt), np64(gt)
    # the solution lies in the span of the nine statistics
    proj = (bn[:, 1:] @ V[:, 1:].T) @ V[:, 1:]
    assert np.abs(bn[:, 1:] - proj).max() <= 1e-6 * (1 + np.abs(bn).max())
    relaxed = 0
    for c in range(B):
        a_o, st_o, it_o, _ = O.solve_axi(RULE9, V @ Mf[c], g=gf[c], final_step=True)
        assert st_o & 1
        b_o = a_o @ V
        # the nine-statistic solution is the 35-statistic one: its residual
        # on the 12-azimuth rule meets the 35-statistic bar
        res = O.residual(RULE35, bn[c], Mf[c], gf[c])
        floor = O.residual(RULE35, beta_exact[c].astype(np.float32).astype(np.float64), Mf[c], gf[c])
        assert res <= max(RES_TOL, 4.0 * floor), (c, res, floor)
        relaxed += int(res > RES_TOL)
        scale = 1.0 + np.abs(b_o[1:]).max()
        assert np.abs(bn[c, 1:] - b_o[1:]).max() <= 5e-3 * scale, (c, np.abs(bn[c, 1:] - b_o[1:]).max())
        assert abs(itn[c] - it_o) <= 2, (c, itn[c], it_o)
    print("nine-statistic solve: %d of %d cells above 1e-5 (within 4x their FP32 floor); mean passes %.2f"
          % (relaxed, B, itn.mean()))


def test_axi_flux_and_speed_match_oracle(O, mem, vctx, states, dev):
    M, g, beta = states
    B = M.shape[0]
    V = O.flic_basis()
    Mt, bt, gt = T32(M, dev), T32(beta, dev), T32(g, dev)
    F = torch.zeros(B, 35, device=dev)
    sp = torch.zeros(B, device=dev)
    # maxI = 0, tol = inf: the start is kept (one pass, no step taken)
    vctx.solve_axi(Mt, bt, gt, None, None, F, sp, maxI=0, tol=float("inf"))
    Fg, spg, bf, gf, Mf = np64(F), np64(sp), np64(bt), np64(gt), np64(Mt)
    for c in range(B):
        a = V @ bf[c]
        a[0] = Mf[c, 0]
        F9, s9 = O.flux_axi(RULE9, a, gf[c], Mf[c, 0])
        assert np.abs(V @ Fg[c] - F9).max() <= 2e-5 * np.abs(F9).max(), c
        assert spg[c] == pytest.approx(s9, rel=1e-3), (c, spg[c], s9)
        # the nine-moment flux is the 35-moment flux of an axisymmetric cell
        F35, s35, _, _ = O.flux(RULE35, bf[c], gf[c], Mf[c, 0])
        assert np.abs(Fg[c] - F35).max() <= 2e-5 * np.abs(F35).max(), c


def _norm(q, a, b):
    return (q - a) / (b - a)


@pytest.mark.parametrize("scheme", ["lf", "flic"])
def test_axi_shock_mach10_matches_oracle(O, mem, vctx, dom, scheme):
    """Mach 10, 40 cells on [-12.5, 12.5], tanh start, the nine-statistic
    system in every cell (and interface): the oracle's 35-statistic shock
    within 1e-3 in the normalised profiles."""
    code = mem.SCHEME_FLIC if scheme == "flic" else mem.SCHEME_LF
    nsteps = 8 if scheme == "flic" else 10
    sh = mem.Shock(vctx, mach=MACH, ncells=40, xl=-12.5, xr=12.5, ic=1, graph=1, stats=9, scheme=code)
    sh.step(nsteps)
    out = sh.get()
    sh.close()
    so = O.Shock(MACH, 40, -12.5, 12.5, order=RULE35, ic="tanh", thickness=15.7, scheme=scheme)
    for _ in range(nsteps):
        so.step()
    rho, ux, T = so.profile()
    assert out["t"] == pytest.approx(so.t, rel=1e-4)
    for name, g_, o_, a, b in (("rho", out["rho"], rho, so.n_up, so.n_dn), ("ux", out["ux"], ux, so.v_up, so.v_dn),
                               ("T", out["T"], T, so.T_up, so.T_dn)):
        err = np.abs(_norm(g_, a, b) - _norm(o_, a, b)).max()
        assert err <= 1e-3, (name, err)
    assert np.isfinite(out["M"]).all()


def test_axi_shock_paper_mesh_equals_35(mem, vctx):
    """The paper's Mach-10 mesh (150 cells on [-47.1, 47.1]), 200 steps: the
    nine-statistic step and the 35-statistic step give the same profiles to
    rounding (normalised difference below 1e-4)."""
    out = {}
    for stats in (35, 9):
        sh = mem.Shock(vctx, mach=MACH, ncells=150, xl=-47.1, xr=47.1, ic=1, graph=1, stats=stats)
        sh.step(200)
        out[stats] = sh.get()
        sh.close()
    a, b = out[35], out[9]
    assert b["t"] == pytest.approx(a["t"], rel=1e-4)
    for k, lo, hi in (("rho", 1.0, 3.883495), ("ux", 12.909944, 3.324311), ("T", 1.0, 32.123125)):
        err = np.abs(_norm(a[k], lo, hi) - _norm(b[k], lo, hi)).max()
        assert err <= 1e-4, (k, err)


def test_axi_batch_alone_equals_mix(mem, vctx):
    probs = [dict(mach=10.0, ncells=30, xl=-9.4, xr=9.4), dict(mach=4.0, ncells=24, xl=-8.0, xr=8.0)]
    sh = mem.Shock(vctx, problems=probs, ic=1, graph=0, stats=9)
    sh.step(6)
    for i, pr in enumerate(probs):
        mix = sh.problem(i)
        a = mem.Shock(vctx, ic=1, graph=0, stats=9, **pr)
        a.step(6)
        alone = a.problem(0)
        a.close()
        for k in ("rho", "ux", "T"):
            assert np.array_equal(alone[k], mix[k]), (i, k)
    sh.close()
