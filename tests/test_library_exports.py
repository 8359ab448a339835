"""CPU checks of the boundary: the library builds for sm_103a, loads, and
exports every entry point declared in include/rfm.h (no GPU calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rfm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rfm_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("rfm_problem_create", "rfm_assemble", "rfm_ipn_solve", "rfm_amipn_solve", "rfm_eval"):
        assert must in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    from paper_2510_04170_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2510_04170_gb300 import rfm
    assert set(rfm.EXPORTS) <= set(_declared())


def test_default_opts_are_the_papers_settings():
    from paper_2510_04170_gb300 import build, rfm
    build.build()
    o = rfm.SolveOpts()
    rfm.load().rfm_default_opts(ctypes.byref(o))
    assert (o.gamma, o.eta, o.eps, o.m_max, o.tau_rel, o.row_scale_c) == (3.0, 1e-6, 1e-10, 3, 1e-3, 100.0)
