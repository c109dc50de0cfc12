"""Packed batches of shock problems and the serving loop (GPU).

A problem's result must not depend on the company it keeps: every kernel
works per cell and every reduction per problem, so the profiles of a problem
run alone and inside a batch (or inside the server's continuously repacked
batch) agree to FP32 rounding (tolerance 1e-6 relative, normally bit-equal).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PROBLEMS = [dict(mach=1.5, ncells=64, xl=-20.0, xr=20.0),
            dict(mach=3.0, ncells=48, xl=-15.0, xr=15.0),
            dict(mach=2.0, ncells=33, xl=-10.0, xr=12.0)]


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_02898_gb300 import mem
    ctx = mem.Context(8)
    yield mem, ctx
    ctx.close()


def _alone(mem, ctx, pr, steps):
    sh = mem.Shock(ctx, graph=0, **pr)
    sh.step(steps)
    out = sh.problem(0)
    sh.close()
    return out


@pytest.mark.parametrize("graph", [0, 1])
def test_batch_alone_equals_mix(env, graph):
    mem, ctx = env
    steps = 12
    sh = mem.Shock(ctx, problems=PROBLEMS, graph=graph)
    assert mem.lib().mem_shock_num_problems(sh.h) == 3
    sh.step(steps)
    for i, pr in enumerate(PROBLEMS):
        mix = sh.problem(i)
        alone = _alone(mem, ctx, pr, steps)
        assert mix["steps"] == steps and alone["steps"] == steps
        assert mix["t"] == pytest.approx(alone["t"], rel=1e-12)
        for k in ("rho", "ux", "T", "sxx", "qx"):
            a, b = alone[k], mix[k]
            assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max(), (i, k)
    sh.close()


def test_batch_matches_oracle(O, env):
    mem, ctx = env
    sh = mem.Shock(ctx, problems=PROBLEMS, graph=1)
    sh.step(10)
    for i, pr in enumerate(PROBLEMS):
        g = sh.problem(i)
        so = O.Shock(pr["mach"], pr["ncells"], pr["xl"], pr["xr"])
        for _ in range(10):
            so.step()
        rho, ux, T = so.profile()
        for gv, ov, a, b in ((g["rho"], rho, so.n_up, so.n_dn), (g["ux"], ux, so.v_up, so.v_dn), (g["T"], T, so.T_up, so.T_dn)):
            assert np.abs((gv - ov) / (b - a)).max() <= 1e-3, i
    sh.close()


def test_tanh_initial_state_matches_oracle(O, env):
    """Appendix D, Eq. "Mx ini": tanh blend of the RH states (thickness 15.7)."""
    mem, ctx = env
    sh = mem.Shock(ctx, mach=1.5, ncells=40, xl=-20.0, xr=20.0, ic=1, graph=0)
    d0 = sh.problem(0)
    so = O.Shock(1.5, 40, -20.0, 20.0, ic="tanh", thickness=15.7)
    rho0, _, T0 = so.profile()
    assert np.abs(d0["rho"] - rho0).max() <= 1e-5 * so.n_dn
    assert np.abs(d0["T"] - T0).max() <= 1e-5 * so.T_dn
    sh.step(8)
    d = sh.problem(0)
    for _ in range(8):
        so.step()
    rho, ux, T = so.profile()
    assert np.abs((d["rho"] - rho) / (so.n_dn - so.n_up)).max() <= 1e-3
    assert np.abs((d["T"] - T) / (so.T_dn - so.T_up)).max() <= 1e-3
    sh.close()


def test_server_continuous_batching(env):
    """Requests arrive while others run; each completes after max_steps (or
    steady state) with exactly the profile it has when run alone."""
    mem, ctx = env
    max_steps = 15
    sv = mem.Server(ctx, hbm_budget_bytes=1 << 30, max_cells=130, steady_tol=1e-12, max_steps=max_steps)
    ids = []
    ids.append((sv.submit(**PROBLEMS[0]), PROBLEMS[0]))
    sv.progress(4)                       # first request running alone
    ids.append((sv.submit(**PROBLEMS[1]), PROBLEMS[1]))
    ids.append((sv.submit(**PROBLEMS[2]), PROBLEMS[2]))  # does not fit yet: 66 + 50 + 35 > 130
    st = sv.stats()
    assert st["queued"] == 2 and st["resident"] == 1
    sv.progress(3)                       # admits the second, third waits
    st = sv.stats()
    assert st["resident"] == 2 and st["queued"] == 1
    assert sv.poll(ids[0][0]) is None
    for _ in range(20):
        sv.progress(5)
        if sv.stats()["completed"] == 3:
            break
    assert sv.stats()["completed"] == 3
    for rid, pr in ids:
        res = sv.poll(rid, ncells=pr["ncells"])
        assert res is not None and res["steps"] == max_steps and res["latency_s"] > 0
        alone = _alone(mem, ctx, pr, max_steps)
        for k in ("rho", "ux", "T"):
            assert np.abs(res[k] - alone[k]).max() <= 1e-6 * np.abs(alone[k]).max(), (rid, k)
    # a request larger than the cell budget is refused at submission
    assert sv.submit(mach=2.0, ncells=500, xl=-10.0, xr=10.0) is None
    with pytest.raises(KeyError):
        sv.poll(12345)
    sv.close()


def test_server_flic_request_equals_alone(env):
    """A FLIC request keeps its interface solves' warm starts when the server
    rebuilds its batch to admit another request, so it ends with the profile
    it has alone (mixed schemes in one batch)."""
    mem, ctx = env
    max_steps = 12
    sv = mem.Server(ctx, hbm_budget_bytes=1 << 30, max_cells=200, steady_tol=1e-12, max_steps=max_steps)
    p1 = dict(mach=1.5, ncells=48, xl=-15.0, xr=15.0, scheme=mem.SCHEME_FLIC)
    p2 = dict(mach=2.0, ncells=30, xl=-10.0, xr=10.0, scheme=mem.SCHEME_LF)
    r1 = sv.submit(**p1)
    sv.progress(3)
    r2 = sv.submit(**p2)  # admitted by a rebuild while the FLIC request is resident
    for _ in range(20):
        sv.progress(3)
        if sv.stats()["completed"] == 2:
            break
    assert sv.stats()["completed"] == 2
    for rid, pr in ((r1, p1), (r2, p2)):
        res = sv.poll(rid, ncells=pr["ncells"])
        assert res is not None and res["steps"] == max_steps
        alone = _alone(mem, ctx, pr, max_steps)
        for k in ("rho", "ux", "T"):
            assert np.abs(res[k] - alone[k]).max() <= 1e-6 * np.abs(alone[k]).max(), (rid, k)
    sv.close()
