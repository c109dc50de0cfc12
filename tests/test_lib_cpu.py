"""CPU-side checks of the CUDA library: it builds for sm_103a, loads, and
exports every entry point include/mem.h declares (no compute without a GPU)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest


def test_library_builds_and_exports_header_symbols():
    from paper_2303_02898_gb300 import build as libbuild
    path = libbuild.build()
    assert os.path.exists(path)
    from paper_2303_02898_gb300 import mem
    L = mem.lib()
    names = mem.declared_functions()
    assert len(names) >= 15, names
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert L.mem_version().startswith(b"mem-gb300")


def test_opts_defaults_are_the_papers():
    from paper_2303_02898_gb300 import mem
    o = mem.default_opts()
    assert o.tol == pytest.approx(1e-8) and o.maxI == 500 and o.maxT == 25
    assert o.c_armijo == pytest.approx(5e-4) and o.atol == pytest.approx(5e-6) and o.rtol == pytest.approx(5e-5)
    assert o.lambda0 == pytest.approx(1e-3) and o.lambda_mul == 10 and o.alpha_min == pytest.approx(1e-6)
    # Algorithm 1 returns beta without the direction of its last pass
    assert o.final_step == 0
    p = mem.default_shock_params()
    assert p.cfl == 0.5 and p.Pr == pytest.approx(2 / 3) and p.gamma == pytest.approx(5 / 3)


def test_invalid_arguments_rejected_without_gpu():
    from paper_2303_02898_gb300 import mem
    L = mem.lib()
    h = ctypes.c_void_p()
    assert L.mem_init(3, 8, ctypes.byref(h)) == mem.MEM_EINVAL
    assert L.mem_init(4, 40, ctypes.byref(h)) == mem.MEM_EINVAL
    assert L.mem_solve(None, None, None, None, None, 0, None, None) == mem.MEM_EINVAL
    assert L.mem_solve_host(None, None, None, None, None, 0, 0, None, None) == mem.MEM_EINVAL
    assert L.mem_tune_save(None, None) == mem.MEM_EINVAL
    assert L.mem_tune_load(None, b"/nonexistent") == mem.MEM_EINVAL


def test_oracle_and_library_share_no_code():
    """The oracle and the CUDA library are independent: no include, import or
    source path crosses between them."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    csrc = os.path.join(root, "paper_2303_02898_gb300", "csrc")
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read()
        assert "oracle" not in txt.lower(), f
    for f in ("mem.py", "build.py", "workloads.py", "__init__.py"):
        txt = open(os.path.join(root, "paper_2303_02898_gb300", f)).read()
        assert "import oracle" not in txt and "from oracle" not in txt, f
    otxt = open(os.path.join(root, "oracle", "mem_oracle.c")).read()
    assert "#include \"" not in otxt


def test_shock_params_defaults_and_validation_without_gpu():
    """Host logic of the shock parameters (no device work): defaults of the
    interface scheme, tanh thickness and t_end, and the validation that
    mem_shock_domain shares with mem_shock_init."""
    from paper_2303_02898_gb300 import mem
    p = mem.default_shock_params()
    assert p.scheme == mem.SCHEME_LF and p.thickness == pytest.approx(15.7) and p.t_end == 0.0
    assert len(mem.shock_domain(mach=4.0, scheme=mem.SCHEME_FLIC, ic=1, thickness=5.44, t_end=4.0)) == 3
    L = mem.lib()
    d = (ctypes.c_double * 3)()
    for bad in (dict(scheme=3), dict(scheme=-1), dict(ic=1, thickness=0.0), dict(t_end=-1.0), dict(mach=0.5)):
        q = mem.default_shock_params(**bad)
        assert L.mem_shock_domain(ctypes.byref(q), d) == mem.MEM_EINVAL, bad


def test_shock_domain_matches_oracle_without_gpu(O):
    """The library's integration box (host code, Appendix D) equals the
    oracle's for the paper's Mach-4 (10, 6, 6) and Mach-10 (5, 5, 5) choices."""
    from paper_2303_02898_gb300 import mem
    for mach, n in ((4.0, (10.0, 6.0, 6.0)), (10.0, (5.0, 5.0, 5.0)), (1.2, (6.0, 6.0, 6.0))):
        lib_box = mem.shock_domain(mach=mach, na=n[0], nb=n[1], nr=n[2])
        assert np.allclose(lib_box, O.shock_domain(mach, *n), rtol=1e-12, atol=1e-12)
