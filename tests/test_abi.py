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
    # u_s, scaling | tau_newton | newton_norm_fro, stop_after, delta_rule (+pad) | scale_off, rank_tol,
    # rho | kmax, imax | tau_ir, eta_r, eta_s, stag_theta | stag_count, project_psd, profile,
    # ckpt_every | mem_budget | fp64_products, u, u_r, u_c, inner, adi_shifts, adi_maxit (+pad) | adi_tol | eksm_maxit, reserved2
    assert ctypes.sizeof(liblyap.LyapOpts) == 4 * 2 + 8 + 4 * 4 + 8 * 3 + 4 * 2 + 8 * 4 + 4 * 4 + 8 + 4 * 8 + 8 + 4 * 2
    assert ctypes.sizeof(liblyap.LyapInfo) == 4 * 10 + 8 + 8 * 64 * 2 + 8 + 8 + 8 * 12 * 3


def test_opts_default_without_gpu():
    from paper_2510_02126_gb300 import lyap as liblyap
    o = liblyap.make_opts()
    assert o.rho == 0.1 and o.imax == 50 and o.kmax == 50 and o.eta_r == 1e-4 and o.stop_after == 2
    # the options beyond the paper's: sign-Newton inner solver, FP64 working precision
    assert o.inner == liblyap.INNER_SIGN and o.adi_shifts == 8 and o.adi_maxit == 200 and o.eksm_maxit == 60
    assert o.u == o.u_r == o.u_c == liblyap.FP64 and o.scaling == liblyap.SCALE_FROB


def test_opts_names_map_to_enum_values():
    from paper_2510_02126_gb300 import lyap as liblyap
    o = liblyap.make_opts("bf16", inner="eksm", scaling="spectral", adi_tol=1e-9)
    assert (o.u_s, o.inner, o.scaling, o.adi_tol) == (liblyap.BF16, 2, 4, 1e-9)
    o = liblyap.make_opts("fp32", inner="adi", scaling="norm2")
    assert (o.u_s, o.inner, o.scaling) == (liblyap.FP32, 1, 3)
    header = open(os.path.join(ROOT, "include", "liblyap.h")).read()
    for name, value in (("LYAP_INNER_ADI", 1), ("LYAP_INNER_EKSM", 2), ("LYAP_SCALE_NORM2", 3),
                        ("LYAP_SCALE_SPECTRAL", 4)):
        assert re.search(rf"\b{name} = {value}\b", header), name


def test_field_offsets_match_c_compiler(tmp_path):
    # every field of the option and info structs sits where the C compiler puts it
    import shutil
    import subprocess
    import pytest
    from paper_2510_02126_gb300 import lyap as liblyap
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "liblyap.h"', "int main(void) {"]
    for cname, st in (("lyap_opts_t", liblyap.LyapOpts), ("lyap_info_t", liblyap.LyapInfo)):
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                          check=True).stdout.split("\n") if l)
    for cname, st in (("lyap_opts_t", liblyap.LyapOpts), ("lyap_info_t", liblyap.LyapInfo)):
        assert int(out[cname]) == ctypes.sizeof(st), cname
        for f, _ in st._fields_:
            assert int(out[f"{cname}.{f}"]) == getattr(st, f).offset, (cname, f)
