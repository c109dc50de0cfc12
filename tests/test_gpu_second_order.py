"""GPU parity for the second-order interface fluxes of the shock step:
two-step Lax-Wendroff (Eq. "The lax W") and FLIC with the van Leer limiter
(Eq. "The FLIC"), against the FP64 oracle.

The oracle follows the paper literally: each cell evaluates both of its
interface fluxes in its own gauge, solving the Lax-Wendroff interface
moments there (twice per interface, once from each side).  The library
solves each interface once, in the Hermite gauge of its moments, and moves
the flux to both neighbours: the same density in exact arithmetic.

Bars: normalised rho, u_x, T within 1e-3 of the oracle (as for the local
Lax-Friedrichs shock tests); a packed batch mixing schemes gives each
problem's profile alone.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PROFILE_TOL = 1e-3
MACH10_RULE = 211  # oracle rule id of the velocity-space rule below


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
def ctx8(mem):
    c = mem.Context(8)
    yield c
    c.close()


def _norm(q, a, b):
    return (q - a) / (b - a)


def _compare(out, so, tol=PROFILE_TOL):
    rho, ux, T = so.profile()
    assert out["t"] == pytest.approx(so.t, rel=1e-4)
    for name, g_, o_, a, b in (("rho", out["rho"], rho, so.n_up, so.n_dn), ("ux", out["ux"], ux, so.v_up, so.v_dn),
                               ("T", out["T"], T, so.T_up, so.T_dn)):
        err = np.abs(_norm(g_, a, b) - _norm(o_, a, b)).max()
        assert err <= tol, (name, err)


@pytest.mark.parametrize("scheme,impl,graph", [("lw", 1, 1), ("flic", 1, 1), ("flic", 1, 0), ("flic", 0, 0)])
def test_shock_mach15_second_order_matches_oracle(O, mem, ctx8, scheme, impl, graph):
    """Mach 1.5, 64 cells on [-20, 20], step start, 20 steps, 8^3 rule."""
    code = {"lw": mem.SCHEME_LW, "flic": mem.SCHEME_FLIC}[scheme]
    sh = mem.Shock(ctx8, mach=1.5, ncells=64, xl=-20.0, xr=20.0, impl=impl, graph=graph, scheme=code)
    sh.step(20)
    out = sh.get()
    sh.close()
    so = O.Shock(1.5, 64, -20.0, 20.0, scheme=scheme)
    for _ in range(20):
        so.step()
    _compare(out, so)
    assert np.abs(out["M"] - so.M).max() <= 1e-3 * np.abs(so.M).max()


@pytest.mark.parametrize("mode", [1, 2])
def test_flic_limiter_readings_match_oracle(O, mem, ctx8, mode):
    """The other readings of the FLIC limiter (one phi per interface: the
    smallest of the nine statistics' in the interface's gauge, or the
    density's), Mach 1.5, 64 cells, 20 steps, against the oracle's same
    reading."""
    sh = mem.Shock(ctx8, mach=1.5, ncells=64, xl=-20.0, xr=20.0, graph=1, scheme=mem.SCHEME_FLIC, flic_limiter=mode)
    sh.step(20)
    out = sh.get()
    sh.close()
    so = O.Shock(1.5, 64, -20.0, 20.0, scheme="flic", flic_limiter=mode)
    for _ in range(20):
        so.step()
    _compare(out, so)


def test_shock_mach12_lax_wendroff_paper_setup(O, mem):
    """Section 4's Mach-1.2 run (Lax-Wendroff): 25 cells on [-47.7, 47.7],
    tanh start with thickness 15.9, on a velocity-space rule of 2 x 2 blocks
    over the Rankine-Hugoniot box with 6 thermal speeds each way (the paper's
    box is [-5.4, 7.8] x [0, 6.6]); 20 steps."""
    dom = O.shock_domain(1.2, 6.0, 6.0, 6.0)
    O.set_velocity_rule(212, dom[0], dom[1], 2, dom[2], 2, 8, 12)
    vctx = mem.Context.velocity(dom, nbx=2, nbr=2, ng=8, K=12)
    sh = mem.Shock(vctx, mach=1.2, ncells=25, xl=-47.7, xr=47.7, ic=1, thickness=15.9, scheme=mem.SCHEME_LW,
                   na=6.0, nb=6.0, nr=6.0, graph=1)
    sh.step(20)
    out = sh.get()
    sh.close()
    vctx.close()
    so = O.Shock(1.2, 25, -47.7, 47.7, order=212, ic="tanh", thickness=15.9, scheme="lw")
    for _ in range(20):
        so.step()
    _compare(out, so)


def test_shock_mach10_flic_velocity_rule(O, mem):
    """Mach 10, FLIC (the paper's Mach-10 scheme), 40 cells of width 0.625,
    tanh start, 8 steps, on the 6 x 4-block velocity-space rule."""
    dom = O.shock_domain(10.0)
    O.set_velocity_rule(MACH10_RULE, dom[0], dom[1], 6, dom[2], 4, 8, 12)
    vctx = mem.Context.velocity(dom, nbx=6, nbr=4, ng=8, K=12)
    sh = mem.Shock(vctx, mach=10.0, ncells=40, xl=-12.5, xr=12.5, ic=1, scheme=mem.SCHEME_FLIC, graph=1)
    sh.step(8)
    out = sh.get()
    sh.close()
    vctx.close()
    so = O.Shock(10.0, 40, -12.5, 12.5, order=MACH10_RULE, ic="tanh", thickness=15.7, scheme="flic")
    for _ in range(8):
        so.step()
    _compare(out, so)
    assert np.isfinite(out["M"]).all()


def test_mixed_scheme_batch_alone_equals_mix(mem, ctx8):
    """LF, LW and FLIC problems packed in one batch give the profiles they
    give alone (per-problem scheme, interfaces never cross problems)."""
    probs = [dict(mach=1.5, ncells=40, xl=-15.0, xr=15.0, scheme=mem.SCHEME_FLIC),
             dict(mach=2.0, ncells=24, xl=-10.0, xr=10.0, scheme=mem.SCHEME_LF),
             dict(mach=1.8, ncells=33, xl=-12.0, xr=12.0, scheme=mem.SCHEME_LW)]
    sh = mem.Shock(ctx8, problems=probs, graph=0)
    sh.step(8)
    for i, pr in enumerate(probs):
        mix = sh.problem(i)
        a = mem.Shock(ctx8, graph=0, **pr)
        a.step(8)
        alone = a.problem(0)
        a.close()
        for k in ("rho", "ux", "T"):
            assert np.array_equal(alone[k], mix[k]), (i, k)
    sh.close()


def test_interface_state_converges_and_is_readable(mem):
    """mem_shock_get_interfaces: after a few FLIC steps on the Mach-10 mesh,
    every interface of the problem has a converged solve with its Hermite
    gauge (positive s) and finite flux; warm starts keep the passes low."""
    dom = mem.shock_domain(mach=10.0)
    vctx = mem.Context.velocity(dom, nbx=6, nbr=4, ng=8, K=12)
    sh = mem.Shock(vctx, mach=10.0, ncells=150, xl=-47.1, xr=47.1, ic=1, scheme=mem.SCHEME_FLIC, graph=1)
    sh.step(20)
    I = sh.interfaces()
    sh.close()
    vctx.close()
    sl = slice(1, 152)  # interfaces between cells 0..151
    assert np.all(I["status"][sl] & 3), I["status"][sl]
    assert np.all(I["g"][sl, 3:] > 0)
    assert np.isfinite(I["F"][sl]).all()
    assert I["iters"][sl].mean() < 4.0


def test_t_end_cuts_the_last_step(mem, ctx8):
    """mem_shock_params.t_end: the step that would pass t_end ends there and
    later steps leave the problem as it is (dt = 0)."""
    sh = mem.Shock(ctx8, mach=1.5, ncells=32, xl=-10.0, xr=10.0, t_end=0.5, graph=0)
    sh.step(200)
    a = sh.problem(0)
    sh.step(5)
    b = sh.problem(0)
    sh.close()
    assert a["t"] == 0.5 and b["t"] == 0.5
    for k in ("rho", "ux", "T"):
        assert np.allclose(a[k], b[k], rtol=1e-6, atol=0), k


def test_second_order_convergence_on_gpu(mem, ctx8):
    """The oracle's convergence pin on the library: smooth Mach-1.5 tanh
    profile (thickness 12 on [-20, 20], Kn = 100), N = 32, 64, 128 in one
    batch stopped at t = 2 by t_end; e(N) = L1 distance of the density from
    the 2N mesh averaged onto N cells.  LF first order, LW and FLIC second."""
    Ns = (32, 64, 128)
    for scheme, lo, hi in ((mem.SCHEME_LF, 1.5, 2.3), (mem.SCHEME_LW, 3.0, 4.6), (mem.SCHEME_FLIC, 3.0, 4.6)):
        sh = mem.Shock(ctx8, problems=[dict(ncells=N) for N in Ns], mach=1.5, xl=-20.0, xr=20.0, ic=1,
                       thickness=12.0, kn=100.0, t_end=2.0, scheme=scheme, graph=1)
        sh.step(400)
        P = [sh.problem(i) for i in range(len(Ns))]
        sh.close()
        assert all(p["t"] == 2.0 for p in P)
        r = {N: p["rho"].astype(np.float64) for N, p in zip(Ns, P)}
        e = [np.abs(r[N] - r[2 * N].reshape(-1, 2).mean(1)).mean() for N in (32, 64)]
        assert lo < e[0] / e[1] < hi, (scheme, e)
