"""CPU-side checks of the CUDA library: it builds for sm_103a, loads, and
exports every entry point include/mem.h declares (no compute without a GPU)."""
import ctypes
import os
import subprocess

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
    p = mem.default_shock_params()
    assert p.cfl == 0.5 and p.Pr == pytest.approx(2 / 3) and p.gamma == pytest.approx(5 / 3)


def test_invalid_arguments_rejected_without_gpu():
    from paper_2303_02898_gb300 import mem
    L = mem.lib()
    h = ctypes.c_void_p()
    assert L.mem_init(3, 8, ctypes.byref(h)) == mem.MEM_EINVAL
    assert L.mem_init(4, 40, ctypes.byref(h)) == mem.MEM_EINVAL
    assert L.mem_solve(None, None, None, None, None, 0, None, None) == mem.MEM_EINVAL


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
