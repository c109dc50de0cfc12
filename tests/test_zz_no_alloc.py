"""mem_flux_noalloc: fluxes and speeds for callers that cannot allocate device
memory (their allocator owns the budget, or a cudaMalloc on their path would
cost a synchronisation).  It must give what mem_flux gives, call after call,
from its fixed library-resident working memory.  This file is collected last
so that a run stopping at its first failure has run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _inputs(rng, B, dev):
    deg = np.array([sum(e) for e in [(a, b, d - a - b) for d in range(5) for a in range(d, -1, -1)
                                     for b in range(d - a, -1, -1)]])
    # near-Gaussian cells (cond E[phi phi^T] below ~200): two FP32 evaluations
    # of the same speed then agree to rounding
    scale = np.where(deg <= 2, 0.1, np.where(deg == 3, 0.015, 0.005))
    beta = rng.normal(0, 1, (B, 35)) * scale
    beta[:, 0] = np.exp(rng.uniform(-0.5, 0.5, B))
    M = np.zeros((B, 35))
    M[:, 0] = beta[:, 0]
    g = np.concatenate([rng.normal(0, 2.0, (B, 3)), np.exp(rng.uniform(np.log(0.5), np.log(3.0), (B, 3)))], 1)
    f = lambda a: torch.tensor(a, dtype=torch.float32, device=dev).contiguous()  # noqa: E731
    return f(M), f(beta), f(g)


def test_flux_noalloc_matches_flux_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_02898_gb300 import mem
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    ctx = mem.Context(8)
    L = mem.lib()
    rng = np.random.default_rng(99)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for B in (1000, 1024):   # two calls in a row through the C ABI
        M, beta, g = _inputs(rng, B, dev)
        F_ref = torch.zeros(B, 35, device=dev)
        s_ref = torch.zeros(B, device=dev)
        ctx.flux(M, beta, g, F_ref, s_ref)
        F = torch.full((B, 35), float("nan"), device=dev)
        s = torch.full((B,), float("nan"), device=dev)
        p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
        rc = L.mem_flux_noalloc(ctx.h, p(M), p(beta), p(g), p(F), p(s), B, stream)
        assert rc == mem.MEM_OK
        torch.cuda.synchronize()
        Fr, sr, Fn, sn = F_ref.cpu().numpy(), s_ref.cpu().numpy(), F.cpu().numpy(), s.cpu().numpy()
        assert np.isfinite(Fn).all() and np.isfinite(sn).all()
        assert np.abs(Fn - Fr).max() <= 2e-5 * np.abs(Fr).max()
        assert np.allclose(sn, sr, rtol=2e-5)
    # beyond the fixed capacity: rejected, nothing written
    M, beta, g = _inputs(rng, 1025, dev)
    assert ctx.flux_noalloc(M, beta, g, torch.zeros(1025, 35, device=dev), None) == mem.MEM_EINVAL
    ctx.close()


@pytest.mark.parametrize("order", [8, 12])
def test_flux_noalloc_matches_oracle(O, order):
    """Both Gauss-Hermite orders at the full 1024-cell capacity (12^3 = 1728
    nodes fills the sigma region up to the moment region that follows it):
    two calls in a row, element-wise against mem_flux and against the FP64
    oracle's flux and speed."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_02898_gb300 import mem
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    ctx = mem.Context(order)
    rng = np.random.default_rng(100 + order)
    for call in range(2):
        B = 1024
        M, beta, g = _inputs(rng, B, dev)
        F_ref = torch.zeros(B, 35, device=dev)
        s_ref = torch.zeros(B, device=dev)
        ctx.flux(M, beta, g, F_ref, s_ref)
        F = torch.full((B, 35), float("nan"), device=dev)
        s = torch.full((B,), float("nan"), device=dev)
        assert ctx.flux_noalloc(M, beta, g, F, s) == mem.MEM_OK
        torch.cuda.synchronize()
        Fr, sr, Fn, sn = F_ref.cpu().numpy(), s_ref.cpu().numpy(), F.cpu().numpy(), s.cpu().numpy()
        assert np.abs(Fn - Fr).max() <= 2e-5 * np.abs(Fr).max()
        assert np.allclose(sn, sr, rtol=2e-5)
        bf, gf, Mf = (t.double().cpu().numpy() for t in (beta, g, M))
        for c in range(0, B, 7):
            Fo, so, _, _ = O.flux(order, bf[c], gf[c], Mf[c, 0])
            assert np.abs(Fn[c] - Fo).max() <= 2e-5 * np.abs(Fo).max(), (call, c)
            assert sn[c] == pytest.approx(so, rel=2e-5), (call, c, sn[c], so)
    ctx.close()


def test_flux_noalloc_rejects_velocity_context():
    """A velocity-space context builds none of the tables this path reads;
    even a rule small enough for the node limit (4 blocks of 4 points in u_x,
    one block of 4 in u_r, 9 azimuths: 576 nodes) is turned away before any
    launch."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_02898_gb300 import mem
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    vctx = mem.Context.velocity((-6.0, 6.0, 6.0), nbx=4, nbr=1, ng=4, K=9)
    M, beta, g = _inputs(np.random.default_rng(5), 8, dev)
    F = torch.zeros(8, 35, device=dev)
    assert vctx.flux_noalloc(M, beta, g, F, None) == mem.MEM_EINVAL
    vctx.close()
