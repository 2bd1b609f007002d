"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point declared in include/liblyap.h (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "liblyap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lyap_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = header_functions()
    for must in ("lyap_ctx_create", "lyap_ctx_destroy", "lyap_opts_default", "lyap_sign_solve", "lyap_solve_ir"):
        assert must in names


def test_library_exports_header_symbols():
    from paper_2510_02126_gb300 import build_lib
    path = build_lib.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2510_02126_gb300 import lyap as liblyap
    assert set(header_functions()) <= set(liblyap.exported_symbols())


def test_struct_layout_matches_header():
    # sizes of the option / info structs as laid out by the C compiler
    from paper_2510_02126_gb300 import lyap as liblyap
    assert ctypes.sizeof(liblyap.LyapOpts) == 4 * 2 + 8 + 4 * 3 + 8 * 3 + 4 * 2 + 8 * 4 + 4 * 2 + 4 * 8 + 4
    assert ctypes.sizeof(liblyap.LyapInfo) == 4 * 10 + 8 + 8 * 64 * 2 + 8 + 8 + 8 * 12 * 3


def test_opts_default_without_gpu():
    from paper_2510_02126_gb300 import lyap as liblyap
    o = liblyap.make_opts()
    assert o.rho == 0.1 and o.imax == 50 and o.kmax == 50 and o.eta_r == 1e-4 and o.stop_after == 2
