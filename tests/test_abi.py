"""CPU checks of the C ABI boundary: the library builds, loads, and exports every symbol
that include/wcipm.h declares, with ctypes structures whose layout matches the header."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wcipm.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sdp_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2407_14013_gb300 import build, _native
    build.build()
    return _native.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("sdp_setup", "sdp_newton_solve", "sdp_newton_solve_host", "sdp_destroy", "sdp_last_error",
                 "sdp_default_options"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2407_14013_gb300 import _native
    so = _native.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (sdp_[a-z_]+)", out))
    for name in declared_functions():
        assert name in exported, f"{name} declared in wcipm.h but not exported"
        assert name in _native.EXPORTS, f"{name} has no binding"


def test_checked_build_exports_the_same_symbols_and_registers_its_checks(lib):
    """libwcipm_checked.so (the sparse operator's gathers and scatters compiled with
    -DSDP_CHECK_BOUNDS) exports the same boundary; in it the bounds records exist, so
    sdp_bounds_report reaches the device (SDP_ECUDA without one) instead of answering
    SDP_EUNSUPPORTED as the default build does.  The default build answers SDP_EUNSUPPORTED
    before any CUDA call."""
    from paper_2407_14013_gb300 import _native
    out = subprocess.run(["nm", "-D", "--defined-only", _native.LIB_CHECKED_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (sdp_[a-z_]+)", out))
    for name in declared_functions():
        assert name in exported, f"{name} not exported by the checked build"
    assert _native.sdp_bounds_report() == (_native.SDP_EUNSUPPORTED, 0, 0)
    assert _native.sdp_bounds_selftest(0, -1, 10) == _native.SDP_EUNSUPPORTED
    code = ("from paper_2407_14013_gb300 import _native as n; n.load(n.LIB_CHECKED_PATH); "
            "import torch; g = torch.cuda.is_available(); st, f, c = n.sdp_bounds_report(); "
            "assert st == (n.SDP_OK if g else n.SDP_ECUDA) and f == c == 0, st; "
            "assert n.sdp_bounds_selftest(0, 1, -1) == n.SDP_EINVAL; print('ok')")
    res = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0 and res.stdout.strip().endswith("ok"), res.stderr[-2000:]


def test_struct_layout_matches_header(lib):
    """Compile a tiny C program against the header and compare sizeof/offsetof with ctypes."""
    from paper_2407_14013_gb300 import _native
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "wcipm.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(sdp_problem), offsetof(sdp_problem, a_dense), sizeof(sdp_options),
         offsetof(sdp_options, newton_rtol));
  printf("%zu %zu %zu\n", sizeof(sdp_newton_info), offsetof(sdp_newton_info, s_A),
         offsetof(sdp_newton_info, prof_A32_launches));
  printf("%zu\n", offsetof(sdp_options, inner_rtol));
  printf("%zu %zu %zu\n", offsetof(sdp_options, pcg_start), sizeof(sdp_ipm_info), offsetof(sdp_ipm_info, total_ms));
  printf("%zu %zu %zu\n", offsetof(sdp_options, tc_products), offsetof(sdp_options, krylov),
         offsetof(sdp_options, int_passes));
  return 0;
}
'''
    tmpd = os.path.join(ROOT, "paper_2407_14013_gb300", "_build")
    os.makedirs(tmpd, exist_ok=True)
    c = os.path.join(tmpd, "layout.c")
    exe = os.path.join(tmpd, "layout")
    open(c, "w").write(src)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
    vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(_native.sdp_problem)
    assert vals[1] == _native.sdp_problem.a_dense.offset
    assert vals[2] == ctypes.sizeof(_native.sdp_options)
    assert vals[3] == _native.sdp_options.newton_rtol.offset
    assert vals[4] == ctypes.sizeof(_native.sdp_newton_info)
    assert vals[5] == _native.sdp_newton_info.s_A.offset
    assert vals[6] == _native.sdp_newton_info.prof_A32_launches.offset
    assert vals[7] == _native.sdp_options.inner_rtol.offset
    assert vals[8] == _native.sdp_options.pcg_start.offset
    assert vals[9] == ctypes.sizeof(_native.sdp_ipm_info)
    assert vals[10] == _native.sdp_ipm_info.total_ms.offset
    assert vals[11] == _native.sdp_options.tc_products.offset
    assert vals[12] == _native.sdp_options.krylov.offset
    assert vals[13] == _native.sdp_options.int_passes.offset


def test_default_options_and_setup_errors(lib):
    """Host-side validation needs no GPU: bad shapes are rejected before any CUDA call."""
    from paper_2407_14013_gb300 import _native
    o = _native.sdp_default_options()
    assert o.r_hat == 10 and o.max_pcg == 2000 and o.newton_rtol == 1e-12 and o.int_passes == 1
    p = _native.sdp_problem()
    p.n, p.m, p.kind = 1, 1, _native.SDP_A_DIAG
    with pytest.raises(_native.SdpError) as e:
        _native.sdp_setup(p, o, 0)
    assert e.value.status == _native.SDP_EINVAL
    p.n, p.m, p.kind = 4, 3, _native.SDP_A_DIAG
    with pytest.raises(_native.SdpError) as e:
        _native.sdp_setup(p, o, 0)
    assert e.value.status == _native.SDP_EINVAL
    p.n, p.m, p.kind = 4, 4, _native.SDP_A_DENSE_SVEC
    with pytest.raises(_native.SdpError) as e:
        _native.sdp_setup(p, o, 0)                        # a_dense is NULL
    assert e.value.status == _native.SDP_EINVAL
    p.kind = _native.SDP_A_SPARSE_COO                     # no entries
    with pytest.raises(_native.SdpError) as e:
        _native.sdp_setup(p, o, 0)
    assert e.value.status == _native.SDP_EINVAL
    p.nnz = 1
    p.a_con = p.a_row = p.a_col = p.a_val = 8            # never read: the mixed form is refused first
    o.precision = _native.SDP_MIXED_FP32
    with pytest.raises(_native.SdpError) as e:
        _native.sdp_setup(p, o, 0)
    assert e.value.status == _native.SDP_EUNSUPPORTED
    o.precision = _native.SDP_FP64
    p.nnz, p.a_con, p.a_row, p.a_col, p.a_val = 0, 0, 0, 0, 0
    p.kind = _native.SDP_A_DIAG
    for field, bad in (("int_passes", 2), ("tc_products", -1), ("krylov", 3), ("pcg_start", 2)):
        o2 = _native.sdp_default_options()
        setattr(o2, field, bad)
        with pytest.raises(_native.SdpError) as e:
            _native.sdp_setup(p, o2, 0)
        assert e.value.status == _native.SDP_EINVAL and field in str(e.value), field
    o.r_fixed = 4                                        # r must be < n
    with pytest.raises(_native.SdpError) as e:
        _native.sdp_setup(p, o, 0)
    assert e.value.status == _native.SDP_EINVAL


def test_product_path_does_not_touch_the_oracle():
    """The package never imports the oracle, and fails loudly without its CUDA library."""
    pkg = os.path.join(ROOT, "paper_2407_14013_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert not re.search(r"^\s*(import|from)\s+oracle", src, flags=re.M), f
    for d in ("oracle", "workloads"):                  # neither side reaches into the other
        for f in os.listdir(os.path.join(ROOT, d)):
            if f.endswith(".py"):
                src = open(os.path.join(ROOT, d, f)).read()
                assert "paper_2407_14013_gb300" not in src, f
                if d == "workloads":
                    assert not re.search(r"^\s*(import|from)\s+oracle", src, flags=re.M), f
    from paper_2407_14013_gb300 import _native
    saved = _native._lib
    try:
        _native._lib = None
        with pytest.raises(RuntimeError):
            _native.load(os.path.join(ROOT, "does_not_exist.so"))
    finally:
        _native._lib = saved


def test_batch_argument_errors_without_gpu():
    """sdp_solve_batch validates its arguments before any CUDA call: an empty batch is a no-op,
    a NULL handle or a repeated handle is SDP_EINVAL with nothing solved."""
    from paper_2407_14013_gb300 import _native
    st, infos = _native.sdp_solve_batch([], [], [], [], [], [], 1e-8, 10)
    assert st == [] and infos == []
    with pytest.raises(_native.SdpError) as e:
        _native.sdp_solve_batch([0, 0], [8, 8], [8, 8], [8, 8], [8, 8], [8, 8], 1e-8, 10)
    assert e.value.status == _native.SDP_EINVAL and "NULL handle" in str(e.value)
    with pytest.raises(_native.SdpError) as e:
        _native.sdp_solve_batch([16, 16], [8, 8], [8, 8], [8, 8], [8, 8], [8, 8], 1e-8, 10)   # never dereferenced
    assert e.value.status == _native.SDP_EINVAL and "twice" in str(e.value)
    with pytest.raises(_native.SdpError):
        _native.sdp_solve_batch([16], [8], [8], [8], [8], [8], -1.0, 10)


def test_linear_block_setter_validates_without_gpu():
    """sdp_set_linear_diag refuses a NULL handle before any CUDA call."""
    from paper_2407_14013_gb300 import _native
    with pytest.raises(_native.SdpError) as e:
        _native.sdp_set_linear_diag(0, 8)
    assert e.value.status == _native.SDP_EINVAL and "NULL handle" in str(e.value)


def test_slack_solve_validates_without_gpu():
    """sdp_solve_slack refuses a NULL handle before any CUDA call."""
    from paper_2407_14013_gb300 import _native
    info = _native.sdp_ipm_info()
    with pytest.raises(_native.SdpError) as e:
        _native.sdp_solve_slack(0, [8] * 11, 1e-8, 10, info)
    assert e.value.status == _native.SDP_EINVAL and "NULL handle" in str(e.value)


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++17")])
def test_header_is_strict_c_and_cpp(lang, std, tmp_path):
    """include/wcipm.h is a plain C interface: it compiles alone, warning-free, as pedantic C99
    and as C++17 (no CUDA or torch types in the signatures)."""
    src = tmp_path / "h.c"
    src.write_text('#include "wcipm.h"\nint main(void) { return 0; }\n')
    cc = "gcc" if lang == "c" else "g++"
    r = subprocess.run([cc, std, "-Wall", "-Wextra", "-Werror", "-pedantic", "-x", lang, "-I",
                        os.path.join(ROOT, "include"), str(src), "-o", str(tmp_path / "h")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
