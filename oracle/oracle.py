"""ctypes binding of the FP64 oracle (oracle/mem_oracle.c).

TEST INFRASTRUCTURE ONLY.  Each wrapper states the paper passage it follows;
the arithmetic lives in the C file.  Arrays are float64 numpy arrays in the
same layouts as the CUDA library: moments/parameters [B, 35], gauges [B, 6]
= (w_x, w_y, w_z, s_x, s_y, s_z).
"""
import ctypes
import os

import numpy as np

from . import build as _build

NP = 35
ST_CONVERGED, ST_STAGNATED, ST_MAXITER, ST_NONFINITE = 1, 2, 4, 8
ST_LAMBDA, ST_LAMBDA_CAP, ST_BADINPUT = 16, 32, 64

_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.or_objective.restype = ctypes.c_double
        L.or_residual.restype = ctypes.c_double
        L.or_index_of.restype = ctypes.c_int
        L.or_num_threads.restype = ctypes.c_int
        L.or_pivot_ratio.restype = ctypes.c_double
        L.or_cond_estimate.restype = ctypes.c_double
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _i(a):
    return a.ctypes.data_as(_I)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def num_threads():
    return lib().or_num_threads()


def basis_index():
    """(a, b, c) exponents of the 35 statistics, in library order."""
    out = np.zeros((NP, 3), dtype=np.int32)
    lib().or_basis_index(_i(out))
    return out


def index_of(a, b, c):
    return lib().or_index_of(int(a), int(b), int(c))


def set_box_rule(rule_id, nbx, nbr, ng, Lx, Lr):
    """Register block Gauss-Legendre tensor rule `rule_id` (100..115) on
    [-Lx, Lx] x [-Lr, Lr]^2 in the gauge frame; returns the node count."""
    q = lib().or_set_box_rule(rule_id, nbx, nbr, ng, ctypes.c_double(Lx), ctypes.c_double(Lr))
    if q <= 0:
        raise ValueError("bad box rule")
    return q


def set_velocity_rule(rule_id, ax, bx, nbx, br, nbr, ng=8, K=12):
    """Register velocity-space rule `rule_id` (200..215): block Gauss-Legendre
    in u_x on [ax, bx] and in u_r on [0, br] (polar weight), K azimuthal
    angles.  Returns the node count."""
    q = lib().or_set_velocity_rule(rule_id, ctypes.c_double(ax), ctypes.c_double(bx), nbx, ctypes.c_double(br), nbr,
                                   ng, K)
    if q < 0:
        raise ValueError("bad velocity rule")
    return q


def shock_domain(mach, na=5.0, nb=5.0, nr=5.0, gamma=5.0 / 3.0):
    """Integration domain (a_x, b_x, b_r) of Appendix D from the
    Rankine-Hugoniot states: n_a, n_b, n_r thermal speeds beyond the up- and
    downstream Maxwellians."""
    r, t = rh(mach, gamma)
    v_up, v_dn, c_up, c_dn = np.sqrt(gamma) * mach, np.sqrt(gamma) * mach / r, 1.0, np.sqrt(t)
    ax = min(v_dn - na * c_dn, v_up - na * c_up)
    bx = max(v_up + nb * c_up, v_dn + nb * c_dn)
    br = max(nr * c_up, nr * c_dn)
    return ax, bx, br


def gh_rule(n):
    """Probabilists' Gauss-Hermite nodes/weights (Golub-Welsch), weights sum to 1."""
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().or_gh_rule(n, _d(x), _d(w)) != 0:
        raise ValueError("unsupported order")
    return x, w


def phi(u):
    """The 35 orthonormal Hermite-product statistics at ubar (Appendix B, 3D)."""
    u = _f64(u, (3,))
    out = np.zeros(NP)
    lib().or_phi(_d(u), _d(out))
    return out


def rule_nodes(order):
    Q = order ** 3
    u = np.zeros((Q, 3))
    lw = np.zeros(Q)
    lib().or_rule_nodes(order, _d(u), _d(lw))
    return u, lw


def _g(g):
    """Gauge argument: None (gauge-frame rules ignore it) or a 6-vector."""
    return None if g is None else _d(_f64(g, (6,)))


def expect(order, beta, g=None):
    """logZ, E phi, E phi phi^T, E ubar_x phi, E ubar_x phi phi^T (Section 3.1).
    g: the cell's gauge, needed by velocity-space rules only."""
    beta = _f64(beta, (NP,))
    lz = ctypes.c_double()
    m = np.zeros(NP)
    S = np.zeros((NP, NP))
    X = np.zeros(NP)
    XS = np.zeros((NP, NP))
    lib().or_expect(order, _g(g), _d(beta), ctypes.byref(lz), _d(m), _d(S), _d(X), _d(XS))
    return lz.value, m, S, X, XS


def objective(order, beta, M, g=None):
    """Appendix C objective L(beta; M) with beta_0 = n."""
    return lib().or_objective(order, _g(g), _d(_f64(beta, (NP,))), _d(_f64(M, (NP,))))


def residual(order, beta, M, g=None):
    """Relative moment residual ||E phi(beta) - M/n|| / ||M/n||."""
    return lib().or_residual(order, _g(g), _d(_f64(beta, (NP,))), _d(_f64(M, (NP,))))


def residual_batch(order, beta, M, g=None):
    beta = _f64(beta).reshape(-1, NP)
    M = _f64(M).reshape(-1, NP)
    if g is None:
        return np.array([residual(order, b, m) for b, m in zip(beta, M)])
    g = _f64(g).reshape(-1, 6)
    return np.array([residual(order, b, m, gg) for b, m, gg in zip(beta, M, g)])


def solve(order, M, beta0=None, tol=1e-8, maxI=500, final_step=False, g=None):
    """Algorithm 1 on one cell.  Returns (beta, status, iters, res, max_lambda)."""
    M = _f64(M, (NP,))
    beta = np.zeros(NP) if beta0 is None else _f64(beta0, (NP,)).copy()
    opts = np.array([tol, float(maxI), float(bool(final_step))])
    it = ctypes.c_int()
    res = ctypes.c_double()
    lam = ctypes.c_double()
    st = lib().or_solve(order, _g(g), _d(M), _d(beta), _d(opts), ctypes.byref(it), ctypes.byref(res), ctypes.byref(lam))
    return beta, st, it.value, res.value, lam.value


def solve_batch(order, M, beta0=None, tol=1e-8, maxI=500, nthreads=0, final_step=False, g=None):
    """Algorithm 1 over a batch of cells (OpenMP).  Returns (beta, status, iters)."""
    M = _f64(M).reshape(-1, NP)
    B = M.shape[0]
    beta = np.zeros((B, NP)) if beta0 is None else _f64(beta0).reshape(B, NP).copy()
    st = np.zeros(B, dtype=np.int32)
    it = np.zeros(B, dtype=np.int32)
    opts = np.array([tol, float(maxI), float(bool(final_step))])
    gg = None if g is None else _d(_f64(g).reshape(B, 6))
    lib().or_solve_batch(order, ctypes.c_int64(B), gg, _d(M), _d(beta), _i(st), _i(it), _d(opts), nthreads)
    return beta, st, it


def pivot_ratio(A):
    """Largest / smallest Cholesky pivot of the SPD matrix A (-1 if not SPD)."""
    A = _f64(A)
    n = A.shape[0]
    return lib().or_pivot_ratio(n, _d(np.ascontiguousarray(A)))


def cond_estimate(order, beta, g=None):
    """Pivot-ratio estimate of cond(H) at beta (Section 4, Fig. 7)."""
    return lib().or_cond_estimate(order, _g(g), _d(_f64(beta, (NP,))))


def set_flic_limiter(mode):
    """Which ratio sets the FLIC limiter: 0 one per statistic of the nine
    (default); 1 one per interface, the smallest of the nine statistics'
    limiters, in the interface's Hermite gauge; 2 one per interface from the
    density."""
    lib().or_set_flic_limiter(int(mode))


def set_shock_stats(stats):
    """Which system or_shock_step solves: 35 the Hermite products (default),
    9 the paper's nine statistics of axisymmetric flow through or_solve_axi /
    or_flux_axi (the state stays the 35 moments, in the span of the nine)."""
    lib().or_set_shock_stats(int(stats))


def flic_basis():
    """The nine statistics of the paper's 1D system (Eq. "Sufficient 35") as
    unit vectors over the 3D Hermite products [9, 35] (the FLIC limiter's
    statistics)."""
    v = np.zeros((9, NP))
    lib().or_flic_basis(_d(v))
    return v


def interface_flux(order, scheme, c, side, M, F, g, speed, dtdx, tol=1e-10, maxI=500, final_step=False,
                   flic_limiter=0):
    """Interface flux between cells c - 1 + side and c + side, in the gauge of
    cell c (Eqs. "The lax F", "The lax W", "The FLIC"): scheme lf, lw, flic."""
    M = _f64(M).reshape(-1, NP)
    F = _f64(F).reshape(-1, NP)
    g = _f64(g).reshape(-1, 6)
    speed = _f64(speed).reshape(-1)
    out = np.zeros(NP)
    opts = np.array([tol, float(maxI), float(bool(final_step))])
    set_flic_limiter(flic_limiter)
    st = lib().or_interface_flux(order, {"lf": 0, "lw": 1, "flic": 2}[scheme], c, side, _d(M), _d(F), _d(g),
                                 _d(speed), ctypes.c_double(dtdx), _d(opts), _d(out))
    return out, st


def solve_axi(order, M9, alpha0=None, tol=1e-8, maxI=500, final_step=False, g=None):
    """Algorithm 1 on the paper's nine 1D statistics (psi_j = v_j . phi,
    flic_basis); M9 = (n, psi moments).  Returns (alpha, status, iters, res)."""
    M9 = _f64(M9, (9,))
    a = np.zeros(9) if alpha0 is None else _f64(alpha0, (9,)).copy()
    opts = np.array([tol, float(maxI), float(bool(final_step))])
    it = ctypes.c_int()
    res = ctypes.c_double()
    st = lib().or_solve_axi(order, _g(g), _d(M9), _d(a), _d(opts), ctypes.byref(it), ctypes.byref(res))
    return a, st, it.value, res.value


def flux_axi(order, alpha, g, n):
    """Flux of the nine moments and the speed of the nine-statistic system."""
    F = np.zeros(9)
    sp = ctypes.c_double()
    lib().or_flux_axi(order, _d(_f64(alpha, (9,))), _d(_f64(g, (6,))), ctypes.c_double(n), _d(F), ctypes.byref(sp))
    return F, sp.value


def gauge_T(g_to, g_from):
    """T(g', g) of Eq. "Change gauge M F": M(g') = T M(g)."""
    T = np.zeros((NP, NP))
    lib().or_gauge_T(_d(_f64(g_to, (6,))), _d(_f64(g_from, (6,))), _d(T))
    return T


def hermite_gauge(M, g, axisym=False):
    """Hermite gauge parameters from moments in gauge g (Eq. "Hermite parameters")."""
    gH = np.zeros(6)
    lib().or_hermite_gauge(_d(_f64(M, (NP,))), _d(_f64(g, (6,))), int(bool(axisym)), _d(gH))
    return gH


def transform_M(g_to, g_from, M):
    out = np.zeros(NP)
    lib().or_transform_M(_d(_f64(g_to, (6,))), _d(_f64(g_from, (6,))), _d(_f64(M, (NP,))), _d(out))
    return out


def transform_beta(g_to, g_from, beta):
    out = np.zeros(NP)
    lib().or_transform_beta(_d(_f64(g_to, (6,))), _d(_f64(g_from, (6,))), _d(_f64(beta, (NP,))), _d(out))
    return out


def flux(order, beta, g, n):
    """F = n (w_x E phi + s_x E ubar_x phi) and the spectral radius of dF/dM."""
    F = np.zeros(NP)
    sp, lo, hi = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().or_flux(order, _d(_f64(beta, (NP,))), _d(_f64(g, (6,))), ctypes.c_double(n), _d(F),
                  ctypes.byref(sp), ctypes.byref(lo), ctypes.byref(hi))
    return F, sp.value, lo.value, hi.value


def flux_batch(order, M, beta, g, nthreads=0):
    M = _f64(M).reshape(-1, NP)
    B = M.shape[0]
    beta = _f64(beta).reshape(B, NP)
    g = _f64(g).reshape(B, 6)
    F = np.zeros((B, NP))
    sp = np.zeros(B)
    lib().or_flux_batch(order, ctypes.c_int64(B), _d(M), _d(beta), _d(g), _d(F), _d(sp), nthreads)
    return F, sp


def macro(M, g):
    """(n, v[3], T, P/n[3x3]) from moments in gauge g (Appendix A definitions)."""
    out = np.zeros(14)
    lib().or_macro(_d(_f64(M, (NP,))), _d(_f64(g, (6,))), _d(out))
    return out[0], out[1:4].copy(), out[4], out[5:].reshape(3, 3).copy()


def gaussian_moments(mean_bar, cov_bar, n):
    out = np.zeros(NP)
    lib().or_gaussian_moments(_d(_f64(mean_bar, (3,))), _d(_f64(cov_bar, (3, 3))), ctypes.c_double(n), _d(out))
    return out


def esbgk(M, g, Pr=2.0 / 3.0):
    """ES-BGK target moments in gauge g (Appendix A, Eq. "The ES BGK model")."""
    out = np.zeros(NP)
    lib().or_esbgk(_d(_f64(M, (NP,))), _d(_f64(g, (6,))), ctypes.c_double(Pr), _d(out))
    return out


def rh(mach, gamma=5.0 / 3.0):
    """Rankine-Hugoniot density and temperature ratios (Appendix D)."""
    r, t = ctypes.c_double(), ctypes.c_double()
    lib().or_rh(ctypes.c_double(mach), ctypes.c_double(gamma), ctypes.byref(r), ctypes.byref(t))
    return r.value, t.value


def target_moments(order, v, T, a, b):
    """Moments (own Hermite gauge) of exp(-|c|^2/2 + cubic(a) - quartic(b))."""
    M = np.zeros(NP)
    gH = np.zeros(6)
    lib().or_target_moments(order, _d(_f64(v, (3,))), ctypes.c_double(T), _d(_f64(a, (10,))),
                            _d(_f64(b, (6,))), _d(M), _d(gH))
    return M, gH


def target_batch(order, v, T, a, b, nthreads=0):
    v = _f64(v).reshape(-1, 3)
    B = v.shape[0]
    T = _f64(T).reshape(B)
    a = _f64(a).reshape(B, 10)
    b = _f64(b).reshape(B, 6)
    M = np.zeros((B, NP))
    gH = np.zeros((B, 6))
    lib().or_target_batch(order, ctypes.c_int64(B), _d(v), _d(T), _d(a), _d(b), _d(M), _d(gH), nthreads)
    return M, gH


# --------------------------------------------------------------------------
# Algorithm 2 on a 1D normal shock (Appendix D set-up).

RELAX_KN1 = float(np.sqrt(2.0 / np.pi))  # mu = sqrt(2/pi) T at Kn = 1; tau = coef/(Pr n)


class Shock:
    """FP64 shock-tube state: N interior cells + 2 Dirichlet ghost cells."""

    def __init__(self, mach, ncells, xl, xr, order=8, cfl=0.5, Pr=2.0 / 3.0, gamma=5.0 / 3.0,
                 kn=1.0, tol=1e-8, maxI=500, nthreads=0, ic="step", thickness=15.7, scheme="lf",
                 final_step=False, flic_limiter=0, stats=35):
        self.order, self.N, self.cfl, self.Pr = order, ncells, cfl, Pr
        # 35: the Hermite products; 9: the paper's nine statistics of
        # axisymmetric flow (Appendix B), see set_shock_stats
        if stats not in (9, 35):
            raise ValueError("stats must be 9 or 35")
        self.stats = stats
        # interface flux: Eq. "The lax F" (lf), "The lax W" (lw), "The FLIC" (flic)
        self.scheme = {"lf": 0, "lw": 1, "flic": 2}[scheme]
        self.flic_limiter = flic_limiter  # see set_flic_limiter
        self.dx = (xr - xl) / ncells
        self.x = xl + (np.arange(ncells) + 0.5) * self.dx
        self.relax = kn * RELAX_KN1 / Pr
        self.opts = np.array([tol, float(maxI), float(bool(final_step))])
        self.nthreads = nthreads
        r, t = rh(mach, gamma)
        self.n_up, self.T_up, self.v_up = 1.0, 1.0, np.sqrt(gamma) * mach
        self.n_dn, self.T_dn, self.v_dn = r, t, np.sqrt(gamma) * mach / r
        NT = ncells + 2
        self.M = np.zeros((NT, NP))
        self.beta = np.zeros((NT, NP))
        self.g = np.zeros((NT, 6))
        xs = np.concatenate([[xl - 0.5 * self.dx], self.x, [xr + 0.5 * self.dx]])
        g_up = np.array([self.v_up, 0, 0, 1.0, 1.0, 1.0]) * np.array([1, 1, 1, np.sqrt(self.T_up)] + [np.sqrt(self.T_up)] * 2)
        g_dn = np.array([self.v_dn, 0, 0] + [np.sqrt(self.T_dn)] * 3)
        for c in range(NT):
            if ic == "step" or c == 0 or c == NT - 1:
                up = xs[c] < 0.0
                n = self.n_up if up else self.n_dn
                self.M[c, 0] = n
                self.beta[c, 0] = n
                self.g[c] = g_up if up else g_dn
            else:
                # Appendix D, Eq. "Mx ini": moments blended with a tanh profile
                # of thickness parameter T (the two Maxwellians' moments are
                # blended in one gauge, then moved to the Hermite gauge).
                h = thickness / 2.0
                w = (np.tanh(xs[c] / h) - np.tanh(xl / h)) / (np.tanh(xr / h) - np.tanh(xl / h))
                Mu = np.zeros(NP)
                Mu[0] = self.n_up
                Md = transform_M(g_up, g_dn, np.r_[self.n_dn, np.zeros(NP - 1)])
                Mb = (1 - w) * Mu + w * Md
                gH = hermite_gauge(Mb, g_up, axisym=True)
                self.M[c] = transform_M(gH, g_up, Mb)
                self.g[c] = gH
                self.beta[c, 0] = self.M[c, 0]
        if stats == 9:
            v = flic_basis()
            if ic != "step":
                for c in range(1, NT - 1):
                    a, _, _, _ = solve_axi(order, v @ self.M[c], v @ self.beta[c], tol, maxI, final_step, self.g[c])
                    self.beta[c] = a @ v
            self.speed = np.array([flux_axi(order, v @ self.beta[c], self.g[c], self.M[c, 0])[1] for c in range(NT)])
        else:
            if ic != "step":
                b, st, it = solve_batch(order, self.M[1:-1], None, tol, maxI, nthreads, final_step=final_step,
                                        g=self.g[1:-1])
                self.beta[1:-1] = b
            _, self.speed = flux_batch(order, self.M, self.beta, self.g, nthreads)
        self.status = np.zeros(NT, dtype=np.int32)
        self.iters = np.zeros(NT, dtype=np.int32)
        # pivot-ratio condition estimate of each cell's last solve (Fig. 7), on request
        self.track_cond = False
        self.cond = np.zeros(NT)
        # status bits of the interface solves (Lax-Wendroff / FLIC), OR-ed per cell
        self.iface_status = np.zeros(NT, dtype=np.int32)
        self.t = 0.0
        self.steps = 0

    def step(self):
        out = np.zeros(3)
        set_flic_limiter(self.flic_limiter)
        set_shock_stats(self.stats)
        lib().or_shock_step(self.order, self.N, ctypes.c_double(self.dx), ctypes.c_double(self.cfl),
                            ctypes.c_double(self.Pr), ctypes.c_double(self.relax), _d(self.M), _d(self.beta),
                            _d(self.g), _d(self.speed), _i(self.status), _i(self.iters), _d(self.opts),
                            self.nthreads, _d(out), _d(self.cond) if self.track_cond else None, self.scheme,
                            _i(self.iface_status))
        self.t += out[0]
        self.steps += 1
        return out  # dt, max speed, max |d rho|

    def profile(self):
        """rho, u_x, T for the interior cells."""
        rho = np.zeros(self.N)
        ux = np.zeros(self.N)
        T = np.zeros(self.N)
        for i in range(self.N):
            n, v, Tc, _ = macro(self.M[i + 1], self.g[i + 1])
            rho[i], ux[i], T[i] = n, v[0], Tc
        return rho, ux, T
