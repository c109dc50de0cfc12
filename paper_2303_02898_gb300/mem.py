"""Thin Python binding of the C ABI in include/mem.h (argument marshalling only).

Every function here passes device pointers of torch tensors (and the current
torch CUDA stream) to libmem_gb300.so; all arithmetic of the method runs in
the library's CUDA kernels.  Importing this module without the built library
raises immediately: there is no fallback path.
"""
import ctypes
import os
import re

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmem_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "mem.h")

NP = 35
MEM_OK, MEM_PENDING = 0, 1
MEM_EINVAL, MEM_ENOMEM, MEM_ECUDA, MEM_EBUSY, MEM_ENOTFOUND = -1, -2, -3, -4, -5
ST_CONVERGED, ST_STAGNATED, ST_MAXITER, ST_NONFINITE = 1, 2, 4, 8
ST_LAMBDA, ST_LAMBDA_CAP, ST_BADINPUT, ST_FP64_OK = 16, 32, 64, 128
IMPL_PLAIN, IMPL_FUSED, IMPL_MIXED = 0, 1, 2


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_float), ("maxI", ctypes.c_int32), ("lambda0", ctypes.c_float),
                ("lambda_mul", ctypes.c_float), ("max_lambda", ctypes.c_int32), ("c_armijo", ctypes.c_float),
                ("atol", ctypes.c_float), ("rtol", ctypes.c_float), ("maxT", ctypes.c_int32),
                ("alpha_min", ctypes.c_float), ("final_step", ctypes.c_int32), ("impl", ctypes.c_int32)]


class ShockParams(ctypes.Structure):
    _fields_ = [("mach", ctypes.c_double), ("ncells", ctypes.c_int32), ("xl", ctypes.c_double),
                ("xr", ctypes.c_double), ("cfl", ctypes.c_double), ("Pr", ctypes.c_double),
                ("gamma", ctypes.c_double), ("kn", ctypes.c_double), ("ic", ctypes.c_int32),
                ("impl", ctypes.c_int32), ("graph", ctypes.c_int32), ("tol", ctypes.c_float),
                ("maxI", ctypes.c_int32), ("na", ctypes.c_double), ("nb", ctypes.c_double),
                ("nr", ctypes.c_double), ("scheme", ctypes.c_int32), ("thickness", ctypes.c_double),
                ("t_end", ctypes.c_double), ("stats", ctypes.c_int32), ("flic_limiter", ctypes.c_int32)]


SCHEME_LF, SCHEME_LW, SCHEME_FLIC = 0, 1, 2


class TuneReport(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("warps", ctypes.c_int32 * 16), ("blocks_per_sm", ctypes.c_int32 * 16),
                ("ms", ctypes.c_float * 16), ("best", ctypes.c_int32), ("default_ms", ctypes.c_float)]


TUNE_FUSED, TUNE_AXI = 0, 1


class ShockResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("steps", ctypes.c_int32), ("ncells", ctypes.c_int32),
                ("steady", ctypes.c_int32), ("sim_time", ctypes.c_double), ("latency_s", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p


def lib():
    """Load libmem_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmem_gb300.so is not built (run __graft_entry__.build()); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        L.mem_version.restype = ctypes.c_char_p
        for name in ("mem_init", "mem_solve", "mem_flux", "mem_gauge_hermite", "mem_gauge_transform",
                     "mem_targets", "mem_shock_init", "mem_shock_step", "mem_shock_get",
                     "mem_shock_device_state", "mem_quad_order", "mem_shock_init_batch",
                     "mem_shock_num_problems", "mem_shock_get_problem", "mem_serve_create", "mem_serve_submit",
                     "mem_shock_get_interfaces",
                     "mem_serve_progress", "mem_serve_poll", "mem_serve_stats"):
            getattr(L, name).restype = ctypes.c_int
        L.mem_solve.argtypes = [_P, _P, _P, _P, _P, ctypes.c_int64, ctypes.POINTER(SolveOpts), _P]
        L.mem_solve_host.restype = ctypes.c_int
        L.mem_solve_host.argtypes = [_P, _P, _P, _P, _P, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(SolveOpts), _P]
        L.mem_solve_gauge.restype = ctypes.c_int
        L.mem_solve_gauge.argtypes = [_P, _P, _P, _P, _P, _P, ctypes.c_int64, ctypes.POINTER(SolveOpts), _P]
        L.mem_init_velocity.restype = ctypes.c_int
        L.mem_init_velocity.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double, _P]
        L.mem_shock_domain.restype = ctypes.c_int
        L.mem_shock_condition.restype = ctypes.c_int
        L.mem_shock_condition.argtypes = [_P, ctypes.c_int, _P]
        L.mem_velocity_rule.restype = ctypes.c_int
        L.mem_velocity_rule.argtypes = [_P, _P, _P]
        L.mem_flux.argtypes = [_P, _P, _P, _P, _P, _P, ctypes.c_int64, _P]
        L.mem_flux_axisym.restype = ctypes.c_int
        L.mem_flux_axisym.argtypes = [_P, _P, _P, _P, _P, _P, ctypes.c_int64, _P]
        L.mem_flux_noalloc.restype = ctypes.c_int
        L.mem_flux_noalloc.argtypes = [_P, _P, _P, _P, _P, _P, ctypes.c_int64, _P]
        L.mem_gauge_hermite.argtypes = [_P, _P, _P, _P, _P, _P, ctypes.c_int64, ctypes.c_int, _P]
        L.mem_gauge_transform.argtypes = [_P, _P, _P, _P, _P, ctypes.c_int64, _P]
        L.mem_targets.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P, ctypes.c_int64, _P]
        L.mem_shock_step.argtypes = [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _P]
        L.mem_destroy.argtypes = [_P]
        L.mem_shock_free.argtypes = [_P]
        L.mem_serve_destroy.argtypes = [_P]
        L.mem_serve_create.argtypes = [_P, ctypes.c_size_t, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, _P]
        L.mem_serve_progress.argtypes = [_P, ctypes.c_int, _P]
        L.mem_serve_poll.argtypes = [_P, ctypes.c_uint64, _P, _P, _P, _P]
        L.mem_solve_axi.restype = ctypes.c_int
        L.mem_solve_axi.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int64, ctypes.POINTER(SolveOpts), _P]
        L.mem_tune.restype = ctypes.c_int
        L.mem_tune.argtypes = [_P, ctypes.c_int, _P, _P, _P, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(SolveOpts),
                               ctypes.POINTER(TuneReport), _P]
        L.mem_set_launch.restype = ctypes.c_int
        L.mem_set_launch.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.mem_get_launch.restype = ctypes.c_int
        L.mem_get_launch.argtypes = [_P, ctypes.c_int, _P, _P]
        L.mem_tune_save.restype = ctypes.c_int
        L.mem_tune_save.argtypes = [_P, ctypes.c_char_p]
        L.mem_tune_load.restype = ctypes.c_int
        L.mem_tune_load.argtypes = [_P, ctypes.c_char_p]
        L.mem_residual64.restype = ctypes.c_int
        L.mem_residual64.argtypes = [_P, _P, _P, _P, ctypes.c_int32, _P, _P, ctypes.c_double, ctypes.c_int64, _P]
        L.mem_bench_peak.restype = ctypes.c_int
        L.mem_bench_peak.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]
        L.mem_tc_selftest.restype = ctypes.c_int
        L.mem_tc_selftest.argtypes = [ctypes.c_int, ctypes.c_int, _P, _P, _P]
        _lib = L
    return _lib


def declared_functions():
    """Names of the functions include/mem.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mem_[a-z_0-9]+)\s*\(", txt)))


def _hptr(t):
    """Address of a contiguous CPU tensor (host buffers of mem_solve_host)."""
    if t is None:
        return None
    if t.is_cuda:
        raise ValueError("expected a host tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(rc, what):
    if rc != MEM_OK:
        raise RuntimeError("%s failed with code %d" % (what, rc))


def default_opts(**kw):
    o = SolveOpts()
    lib().mem_solve_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Context:
    """mem_init / mem_destroy: quadrature and statistics tables on the device.
    Context.velocity(...) builds a context with a velocity-space rule
    (mem_init_velocity)."""

    def __init__(self, quad_order=8, degree=4, _handle=None):
        if _handle is None:
            h = ctypes.c_void_p()
            _check(lib().mem_init(degree, quad_order, ctypes.byref(h)), "mem_init")
            _handle = h
        self.h = _handle
        self.quad_order = quad_order

    @classmethod
    def velocity(cls, domain, nbx=6, nbr=4, ng=8, K=12, degree=4):
        """Velocity-space block Gauss-Legendre rule on domain (a_x, b_x, b_r)."""
        h = ctypes.c_void_p()
        ax, bx, br = (float(v) for v in domain)
        _check(lib().mem_init_velocity(degree, nbx, nbr, ng, K, ax, bx, br, ctypes.byref(h)), "mem_init_velocity")
        return cls(quad_order=0, _handle=h)

    def velocity_rule(self):
        """((nbx, nbr, ng, K), (a_x, b_x, b_r)) of a velocity-space context."""
        shape = (ctypes.c_int32 * 4)()
        dom = (ctypes.c_double * 3)()
        _check(lib().mem_velocity_rule(self.h, shape, dom), "mem_velocity_rule")
        return tuple(shape), tuple(dom)

    def close(self):
        if self.h:
            lib().mem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- solve
    def solve(self, M, beta, status=None, iters=None, opts=None, stream=None, **kw):
        """mem_solve: Algorithm 1 on every row of M (in place on beta)."""
        B = M.shape[0]
        o = opts if opts is not None else default_opts(**kw)
        rc = lib().mem_solve(self.h, _ptr(M), _ptr(beta), _ptr(status), _ptr(iters), B, ctypes.byref(o),
                             _stream(stream))
        _check(rc, "mem_solve")

    def solve_host(self, M, beta, status=None, iters=None, warm=False, opts=None, stream=None, **kw):
        """mem_solve_host: Algorithm 1 on host (CPU, ideally pinned) tensors,
        streamed through the device in chunks with the copies overlapped.
        Asynchronous on `stream`: synchronise before reading beta / status."""
        B = M.shape[0]
        o = opts if opts is not None else default_opts(**kw)
        rc = lib().mem_solve_host(self.h, _hptr(M), _hptr(beta), _hptr(status), _hptr(iters), B, int(bool(warm)),
                                  ctypes.byref(o), _stream(stream))
        _check(rc, "mem_solve_host")

    def solve_gauge(self, M, beta, gauge, status=None, iters=None, opts=None, stream=None, **kw):
        """mem_solve_gauge: Algorithm 1 with the cells' gauges (velocity-space rules)."""
        B = M.shape[0]
        o = opts if opts is not None else default_opts(**kw)
        rc = lib().mem_solve_gauge(self.h, _ptr(M), _ptr(beta), _ptr(gauge), _ptr(status), _ptr(iters), B,
                                   ctypes.byref(o), _stream(stream))
        _check(rc, "mem_solve_gauge")

    def solve_axi(self, M, beta, gauge, status=None, iters=None, F=None, speed=None, opts=None, stream=None, **kw):
        """mem_solve_axi: the paper's nine-statistic system (velocity-space rules):
        Algorithm 1, flux and speed per axisymmetric cell."""
        o = opts if opts is not None else default_opts(**kw)
        rc = lib().mem_solve_axi(self.h, _ptr(M), _ptr(beta), _ptr(gauge), _ptr(status), _ptr(iters), _ptr(F),
                                 _ptr(speed), M.shape[0], ctypes.byref(o), _stream(stream))
        _check(rc, "mem_solve_axi")

    def tune(self, kernel, M, beta0, gauge=None, reps=2, opts=None, stream=None, **kw):
        """mem_tune: time every launch shape of `kernel` on this batch, keep the
        fastest; returns the list of (warps, blocks_per_sm, ms), the kept index
        and the default's time."""
        o = opts if opts is not None else default_opts(**kw)
        r = TuneReport()
        _check(lib().mem_tune(self.h, kernel, _ptr(M), _ptr(beta0), _ptr(gauge), M.shape[0], reps, ctypes.byref(o),
                              ctypes.byref(r), _stream(stream)), "mem_tune")
        cands = [(r.warps[i], r.blocks_per_sm[i], r.ms[i]) for i in range(r.n)]
        return {"candidates": cands, "best": r.best, "default_ms": r.default_ms}

    def set_launch(self, kernel, warps, blocks_per_sm):
        _check(lib().mem_set_launch(self.h, kernel, warps, blocks_per_sm), "mem_set_launch")

    def get_launch(self, kernel):
        w, b = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().mem_get_launch(self.h, kernel, ctypes.byref(w), ctypes.byref(b)), "mem_get_launch")
        return w.value, b.value

    def tune_save(self, path):
        """mem_tune_save: write this context's launch shape to the tuning table."""
        _check(lib().mem_tune_save(self.h, os.fsencode(path)), "mem_tune_save")

    def tune_load(self, path):
        """mem_tune_load: apply the table's entry for this GPU, rule and kernel;
        False when the table has none."""
        rc = lib().mem_tune_load(self.h, os.fsencode(path))
        if rc == MEM_ENOTFOUND:
            return False
        _check(rc, "mem_tune_load")
        return True

    def residual64(self, M, beta, res, status=None, mask=0, status_out=None, accept=1e-5, stream=None):
        """mem_residual64: FP64 relative moment residual per cell (res: float64
        CUDA tensor), for the cells with status & mask (all if mask == 0)."""
        rc = lib().mem_residual64(self.h, _ptr(M), _ptr(beta), _ptr(status), int(mask), _ptr(res), _ptr(status_out),
                                  float(accept), M.shape[0], _stream(stream))
        _check(rc, "mem_residual64")

    def flux(self, M, beta, gauge, F=None, speed=None, stream=None):
        rc = lib().mem_flux(self.h, _ptr(M), _ptr(beta), _ptr(gauge), _ptr(F), _ptr(speed), M.shape[0],
                            _stream(stream))
        _check(rc, "mem_flux")

    def flux_axisym(self, M, beta, gauge, F=None, speed=None, stream=None):
        """mem_flux_axisym: flux() for cells symmetric in u_y and u_z."""
        rc = lib().mem_flux_axisym(self.h, _ptr(M), _ptr(beta), _ptr(gauge), _ptr(F), _ptr(speed), M.shape[0],
                                   _stream(stream))
        _check(rc, "mem_flux_axisym")

    def flux_noalloc(self, M, beta, gauge, F=None, speed=None, stream=None):
        """mem_flux_noalloc: as flux(), with library-resident working memory
        (at most 1024 cells per call); returns the C return code."""
        return lib().mem_flux_noalloc(self.h, _ptr(M), _ptr(beta), _ptr(gauge), _ptr(F), _ptr(speed),
                                      M.shape[0], _stream(stream))

    def gauge_hermite(self, M_in, g_in, g_out, M_out, beta=None, axisym=False, stream=None):
        rc = lib().mem_gauge_hermite(self.h, _ptr(M_in), _ptr(g_in), _ptr(g_out), _ptr(M_out), _ptr(beta),
                                     M_in.shape[0], int(bool(axisym)), _stream(stream))
        _check(rc, "mem_gauge_hermite")

    def gauge_transform(self, g_to, g_from, M_in, M_out, stream=None):
        rc = lib().mem_gauge_transform(self.h, _ptr(g_to), _ptr(g_from), _ptr(M_in), _ptr(M_out),
                                       M_in.shape[0], _stream(stream))
        _check(rc, "mem_gauge_transform")

    def targets(self, v, T, a, b, M_out, g_out, gen_order=24, stream=None):
        rc = lib().mem_targets(self.h, gen_order, _ptr(v), _ptr(T), _ptr(a), _ptr(b), _ptr(M_out), _ptr(g_out),
                               v.shape[0], _stream(stream))
        _check(rc, "mem_targets")


def default_shock_params(**kw):
    p = ShockParams()
    lib().mem_shock_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def shock_domain(**kw):
    """mem_shock_domain: the velocity-space integration domain (a_x, b_x, b_r)
    of a shock problem with these parameters."""
    p = default_shock_params(**kw)
    d = (ctypes.c_double * 3)()
    _check(lib().mem_shock_domain(ctypes.byref(p), d), "mem_shock_domain")
    return tuple(d)


class Shock:
    """mem_shock_init / step / get / free; with `problems` (a list of dicts of
    parameters) a packed batch through mem_shock_init_batch."""

    def __init__(self, ctx, problems=None, **kw):
        self.ctx = ctx
        h = ctypes.c_void_p()
        if problems is None:
            self.p = default_shock_params(**kw)
            _check(lib().mem_shock_init(ctx.h, ctypes.byref(self.p), ctypes.byref(h)), "mem_shock_init")
            self.ps = [self.p]
        else:
            self.ps = [default_shock_params(**dict(kw, **pr)) for pr in problems]
            arr = (ShockParams * len(self.ps))(*self.ps)
            _check(lib().mem_shock_init_batch(ctx.h, arr, len(self.ps), ctypes.byref(h)), "mem_shock_init_batch")
            self.p = self.ps[0]
        self.h = h
        self.N = self.p.ncells

    def step(self, nsteps=1, steady=False, stream=None):
        d = ctypes.c_double(0.0)
        rc = lib().mem_shock_step(self.h, nsteps, ctypes.byref(d) if steady else None, _stream(stream))
        _check(rc, "mem_shock_step")
        return d.value if steady else None

    def get(self):
        import numpy as np
        NT = self.N + 2
        M = np.zeros((NT, NP), np.float32)
        g = np.zeros((NT, 6), np.float32)
        b = np.zeros((NT, NP), np.float32)
        prof = [np.zeros(self.N, np.float32) for _ in range(5)]
        t = ctypes.c_double()
        f = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        rc = lib().mem_shock_get(self.h, f(M), f(g), f(b), *[f(x) for x in prof], ctypes.byref(t))
        _check(rc, "mem_shock_get")
        return dict(M=M, g=g, beta=b, rho=prof[0], ux=prof[1], T=prof[2], sxx=prof[3], qx=prof[4], t=t.value)

    def problem(self, i):
        """Profiles (rho, u_x, T, sigma_xx, q_x), time and steps of problem i."""
        import numpy as np
        n = self.ps[i].ncells
        prof = [np.zeros(n, np.float32) for _ in range(5)]
        t = ctypes.c_double()
        st = ctypes.c_int32()
        f = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        _check(lib().mem_shock_get_problem(self.h, i, *[f(x) for x in prof], ctypes.byref(t), ctypes.byref(st)),
               "mem_shock_get_problem")
        return dict(rho=prof[0], ux=prof[1], T=prof[2], sxx=prof[3], qx=prof[4], t=t.value, steps=st.value)

    def condition(self, i=0):
        """mem_shock_condition: largest pivot-ratio condition estimate over
        problem i's cells in the last step (velocity-space contexts)."""
        c = ctypes.c_double()
        _check(lib().mem_shock_condition(self.h, i, ctypes.byref(c)), "mem_shock_condition")
        return c.value

    def interfaces(self):
        """mem_shock_get_interfaces: host copy of the Lax-Wendroff / FLIC
        interface state, packed like the cells (entry c: between cells c - 1
        and c)."""
        import numpy as np
        NT = sum(p.ncells + 2 for p in self.ps)
        MI = np.zeros((NT, NP), np.float32)
        b = np.zeros((NT, NP), np.float32)
        g = np.zeros((NT, 6), np.float32)
        F = np.zeros((NT, NP), np.float32)
        st = np.zeros(NT, np.int32)
        it = np.zeros(NT, np.int32)
        f = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        _check(lib().mem_shock_get_interfaces(self.h, f(MI), f(b), f(g), f(F), f(st), f(it)),
               "mem_shock_get_interfaces")
        return dict(M=MI, beta=b, g=g, F=F, status=st, iters=it)

    def device_state(self):
        ptrs = [ctypes.c_void_p() for _ in range(6)]
        _check(lib().mem_shock_device_state(self.h, *[ctypes.byref(p) for p in ptrs]), "mem_shock_device_state")
        return [p.value for p in ptrs]

    def device_tensors(self):
        """Zero-copy views (M, beta, gauge, status, iters) of the packed device
        state, ghost cells included (valid while the shock lives)."""
        NT = sum(p.ncells + 2 for p in self.ps)
        M, beta, g, _, status, iters = self.device_state()

        class _View:
            def __init__(self, ptr, shape, typestr="<f4"):
                self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False),
                                                 "version": 2}
        dev = torch.device("cuda", torch.cuda.current_device())
        views = [torch.as_tensor(_View(p, (NT, n)), device=dev) for p, n in ((M, NP), (beta, NP), (g, 6))]
        views += [torch.as_tensor(_View(p, (NT,), "<i4"), device=dev) for p in (status, iters)]
        return tuple(views)

    def close(self):
        if self.h:
            lib().mem_shock_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """mem_serve_*: continuous batching of shock solves."""

    def __init__(self, ctx, hbm_budget_bytes=8 << 30, max_cells=1 << 20, steady_tol=1e-6, max_steps=100000):
        self.ctx = ctx
        h = ctypes.c_void_p()
        _check(lib().mem_serve_create(ctx.h, hbm_budget_bytes, max_cells, steady_tol, max_steps, ctypes.byref(h)),
               "mem_serve_create")
        self.h = h

    def submit(self, **kw):
        p = default_shock_params(**kw)
        rid = ctypes.c_uint64()
        rc = lib().mem_serve_submit(self.h, ctypes.byref(p), ctypes.byref(rid))
        if rc == MEM_EBUSY:
            return None
        _check(rc, "mem_serve_submit")
        return rid.value

    def progress(self, iters=1, stream=None):
        _check(lib().mem_serve_progress(self.h, iters, _stream(stream)), "mem_serve_progress")

    def poll(self, rid, ncells=None):
        import numpy as np
        r = ShockResult()
        if ncells:
            prof = [np.zeros(ncells, np.float32) for _ in range(3)]
            ptrs = [p.ctypes.data_as(ctypes.c_void_p) for p in prof]
        else:
            prof, ptrs = None, [None, None, None]
        rc = lib().mem_serve_poll(self.h, rid, ctypes.byref(r), *ptrs)
        if rc == MEM_OK:
            out = dict(steps=r.steps, ncells=r.ncells, steady=bool(r.steady), sim_time=r.sim_time,
                       latency_s=r.latency_s)
            if prof:
                out.update(rho=prof[0], ux=prof[1], T=prof[2])
            return out
        if rc == MEM_PENDING:
            return None
        raise KeyError(rid)

    def stats(self):
        v = [ctypes.c_int32() for _ in range(4)]
        _check(lib().mem_serve_stats(self.h, *[ctypes.byref(x) for x in v]), "mem_serve_stats")
        return dict(queued=v[0].value, resident=v[1].value, resident_cells=v[2].value, completed=v[3].value)

    def close(self):
        if self.h:
            lib().mem_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PEAK_FMA, PEAK_EXP2, PEAK_TC_BF16, PEAK_TC_TF32 = 0, 1, 2, 3


def bench_peak(kind, iters):
    """mem_bench_peak: (seconds, work) of one timed micro-benchmark launch on
    the current device (work = flops, or exp2 evaluations for PEAK_EXP2)."""
    sec, work = ctypes.c_double(), ctypes.c_double()
    _check(lib().mem_bench_peak(kind, iters, ctypes.byref(sec), ctypes.byref(work)), "mem_bench_peak")
    return sec.value, work.value


def tc_selftest(kind, A, B):
    """mem_tc_selftest: D = A B^T through the tensor cores (kind 1 = BF16,
    2 = TF32 operands); A [128][64], B [N][64] float32 host arrays."""
    import numpy as np
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    N = B.shape[0]
    D = np.zeros((128, N), dtype=np.float32)
    _check(lib().mem_tc_selftest(kind, N, A.ctypes.data, B.ctypes.data, D.ctypes.data), "mem_tc_selftest")
    return D
