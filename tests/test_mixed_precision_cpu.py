"""The premise of the mixed-precision back-end, checked on the CPU with the
oracle's quadrature and statistics: Algorithm 1 only uses the Hessian as the
Newton model, so forming E[phi phi^T] from TF32- or BF16-rounded sigma and
phi_i phi_j (the tensor-core inputs) leaves the Newton passes unchanged and
the final moment residual (exact moments, final step applied) below the
1e-5 bar.  A plain numpy restatement of Algorithm 1 with the paper's
constants; the FP64 column of the same code is the control."""
import numpy as np
import pytest


def _round(x, keep_mask, half):
    x = np.asarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    u = ((u + half) & keep_mask).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def tf32(x):
    return _round(x, 0xffffe000, 0x1000)


def bf16(x):
    return _round(x, 0xffff0000, 0x8000)


def _solve(Phi, lw, M, rnd, tol=1e-8, maxI=500):
    n = M[0]
    mt = M / n
    b = np.zeros(35)
    P2 = np.einsum("qi,qj->qij", Phi[:, 1:], Phi[:, 1:])
    P2r = rnd(P2) if rnd else P2

    def ev(b):
        e = lw + Phi[:, 1:] @ b[1:]
        mx = e.max()
        w = np.exp(e - mx)
        return mx + np.log(w.sum()), w / w.sum()
    L, sig = ev(b)
    L -= b[1:] @ mt[1:]
    d = np.zeros(35)
    G = np.zeros(35)
    it, alpha = 0, 1.0
    while True:
        if it > 0:
            gd = G[1:] @ d[1:]
            alpha = 2.0
            for _ in range(26):
                alpha *= 0.5
                bt = b + alpha * d
                Lt, sg = ev(bt)
                Lt -= bt[1:] @ mt[1:]
                LD = L - Lt
                if LD + 5e-4 * alpha * gd >= -(5e-6 + 5e-5 * abs(LD)):
                    break
            b, L, sig = bt, Lt, sg
        m = sig @ Phi
        G = m - mt
        G[0] = 0.0
        S = np.einsum("q,qij->ij", rnd(sig) if rnd else sig, P2r)
        H = S - np.outer(m[1:], m[1:])
        x = -np.linalg.solve(H, G[1:])
        d = np.concatenate([[0.0], x])
        res = 0.5 * abs(x @ G[1:])
        it += 1
        if res <= tol or alpha <= 1e-6 or it > maxI:
            if res <= tol:
                b = b + d
            return b, it


@pytest.mark.parametrize("workload", ["targets", "perturbed"])
def test_low_precision_hessian_keeps_newton_passes(O, workload):
    from paper_2303_02898_gb300 import workloads
    if workload == "targets":
        t = workloads.solve_targets(24, seed=5)
        M, _ = O.target_batch(24, t.v, t.T, t.a, t.b)
    else:
        M = workloads.perturbed_hermite_moments(24, seed=17, scale=0.04)
    nodes, lw = O.rule_nodes(8)
    Phi = np.array([O.phi(u) for u in nodes])
    for c in range(M.shape[0]):
        b64, it64 = _solve(Phi, lw, M[c], None)
        # the restatement is Algorithm 1: same passes as the oracle
        bo, _, ito, _, _ = O.solve(8, M[c], final_step=True)
        assert it64 == ito, (c, it64, ito)
        for rnd in (tf32, bf16):
            b, it = _solve(Phi, lw, M[c], rnd)
            assert abs(it - it64) <= 1, (c, rnd.__name__, it, it64)
            assert O.residual(8, b, M[c]) <= max(1e-5, 1.5 * O.residual(8, b64, M[c])), (c, rnd.__name__)
