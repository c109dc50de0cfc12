"""The autotuner of the launch shapes (mem_tune): it times every candidate,
keeps the fastest, and the kept shape changes the time only -- the solution
of every cell is bit-for-bit the one of the default shape."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_02898_gb300 import mem as m
    m.lib()
    return m


def _check_report(rep):
    c = rep["candidates"]
    assert len(c) >= 3 and c[0][:2] == (4, 0)
    assert all(ms > 0 for _, _, ms in c)
    assert rep["best"] == int(np.argmin([ms for _, _, ms in c]))
    assert rep["default_ms"] == c[0][2]


def test_tune_fused_solve(mem):
    from paper_2303_02898_gb300 import workloads
    dev = torch.device("cuda:0")
    ctx = mem.Context(8)
    B = 1 << 14
    t = workloads.solve_targets(B, seed=3)
    f = lambda a: torch.tensor(a, dtype=torch.float32, device=dev).contiguous()  # noqa: E731
    M = torch.zeros(B, 35, device=dev)
    g = torch.zeros(B, 6, device=dev)
    ctx.targets(f(t.v), f(t.T), f(t.a), f(t.b), M, g, gen_order=24)
    beta0 = torch.zeros_like(M)
    b_def = beta0.clone()
    st_def = torch.zeros(B, dtype=torch.int32, device=dev)
    ctx.solve(M, b_def, st_def)
    rep = ctx.tune(mem.TUNE_FUSED, M, beta0, reps=2)
    _check_report(rep)
    w, bps = rep["candidates"][rep["best"]][:2]
    assert ctx.get_launch(mem.TUNE_FUSED) == (w, bps)
    assert torch.equal(beta0, torch.zeros_like(M))   # the start is not modified
    for cw, cb, _ in rep["candidates"]:
        ctx.set_launch(mem.TUNE_FUSED, cw, cb)
        b = beta0.clone()
        st = torch.zeros(B, dtype=torch.int32, device=dev)
        ctx.solve(M, b, st)
        assert torch.equal(b, b_def) and torch.equal(st, st_def), (cw, cb)
    ctx.close()


def test_tune_nine_statistic_solve(O, mem):
    dev = torch.device("cuda:0")
    dom = O.shock_domain(10.0)
    O.set_velocity_rule(205, dom[0], dom[1], 6, dom[2], 4, 8, 12)
    so = O.Shock(10.0, 40, -12.5, 12.5, order=205, ic="tanh", thickness=15.7)
    reps = 64
    M = torch.tensor(np.tile(so.M, (reps, 1)), dtype=torch.float32, device=dev).contiguous()
    g = torch.tensor(np.tile(so.g, (reps, 1)), dtype=torch.float32, device=dev).contiguous()
    vctx = mem.Context.velocity(dom)
    beta0 = torch.zeros_like(M)
    beta0[:, 0] = M[:, 0]
    b_def = beta0.clone()
    vctx.solve_axi(M, b_def, g)
    rep = vctx.tune(mem.TUNE_AXI, M, beta0, g, reps=2)
    _check_report(rep)
    for cw, cb, _ in rep["candidates"]:
        vctx.set_launch(mem.TUNE_AXI, cw, cb)
        b = beta0.clone()
        vctx.solve_axi(M, b, g)
        assert torch.equal(b, b_def), (cw, cb)
    vctx.close()


def test_tuning_table_round_trip(mem, tmp_path, monkeypatch):
    """mem_tune_save / mem_tune_load: the shape kept for this GPU, rule and
    kernel comes back in a new context, also through MEM_TUNE_TABLE at
    context creation; other rules and kernels keep their defaults."""
    path = str(tmp_path / "tune.tsv")
    c8 = mem.Context(8)
    c8.set_launch(mem.TUNE_FUSED, 8, 2)
    c8.tune_save(path)
    c8.set_launch(mem.TUNE_FUSED, 2, 6)
    c8.tune_save(path)                      # replaces the line with the same key
    c8.close()
    lines = open(path).read().strip().splitlines()
    assert len(lines) == 1 and lines[0].split("\t")[2:] == ["0", "2", "6"]
    v = mem.Context.velocity(mem.shock_domain(mach=10.0))
    v.set_launch(mem.TUNE_AXI, 2, 10)
    v.tune_save(path)
    v.close()
    assert len(open(path).read().strip().splitlines()) == 2
    n8 = mem.Context(8)
    assert n8.get_launch(mem.TUNE_FUSED) == (4, 0)
    assert n8.tune_load(path) and n8.get_launch(mem.TUNE_FUSED) == (2, 6)
    n8.close()
    n12 = mem.Context(12)
    assert not n12.tune_load(path) and n12.get_launch(mem.TUNE_FUSED) == (4, 0)
    n12.close()
    monkeypatch.setenv("MEM_TUNE_TABLE", path)
    a8 = mem.Context(8)
    av = mem.Context.velocity(mem.shock_domain(mach=10.0))
    assert a8.get_launch(mem.TUNE_FUSED) == (2, 6) and av.get_launch(mem.TUNE_AXI) == (2, 10)
    a8.close()
    av.close()
