"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/jqcd.h declares, and its structs have the layout the
Python binding assumes (checked by compiling the header with gcc)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "jqcd.h")


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"JQCD_API\s+[\w\s\*]*?\b(jqcd_\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("jqcd_gauge_upload", "jqcd_dslash_eo", "jqcd_mdagm", "jqcd_cg_solve"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2409_03030_gb300 import jqcd
    lib = ctypes.CDLL(jqcd.LIB_PATH)
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert set(jqcd.exported_symbols()) == set(declared_functions())
    assert jqcd.jqcd_abi_version() == 1


def test_spinor_bytes_host_only():
    from paper_2409_03030_gb300 import jqcd
    vh = 24 * 24 * 24 * 48 // 2
    assert jqcd.spinor_bytes((24, 24, 24, 48), jqcd.PREC_DW) == vh * 192
    assert jqcd.spinor_bytes((24, 24, 24, 48), jqcd.PREC_F64) == vh * 192
    assert jqcd.spinor_bytes((24, 24, 24, 48), jqcd.PREC_F32) == vh * 96
    assert jqcd.spinor_bytes((24, 24, 24, 48), jqcd.PREC_F16N) == vh * 52
    with pytest.raises(jqcd.JqcdError):
        jqcd.spinor_bytes((3, 4, 4, 4), jqcd.PREC_DW)
    with pytest.raises(jqcd.JqcdError):
        jqcd.spinor_bytes((4, 4, 4, 4), 7)


def test_struct_layout_matches_c(tmp_path):
    from paper_2409_03030_gb300 import jqcd
    src = tmp_path / "layout.c"
    src.write_text('#include "jqcd.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(jqcd_lattice),'
                   ' sizeof(jqcd_solve_params), sizeof(jqcd_solve_info),'
                   ' offsetof(jqcd_solve_params, delta), offsetof(jqcd_solve_info, true_rel_resid),'
                   ' offsetof(jqcd_solve_info, hop_count)); printf("%zu %zu %zu\\n",'
                   ' sizeof(jqcd_request), sizeof(jqcd_serve_stats), offsetof(jqcd_request, x));'
                   ' return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [ctypes.sizeof(jqcd.jqcd_lattice), ctypes.sizeof(jqcd.jqcd_solve_params),
            ctypes.sizeof(jqcd.jqcd_solve_info), jqcd.jqcd_solve_params.delta.offset,
            jqcd.jqcd_solve_info.true_rel_resid.offset, jqcd.jqcd_solve_info.hop_count.offset,
            ctypes.sizeof(jqcd.jqcd_request), ctypes.sizeof(jqcd.jqcd_serve_stats),
            jqcd.jqcd_request.x.offset]
    assert got == want


def test_constants_match_header(tmp_path):
    """Status codes, precisions, solver modes and the allocation-free limit of
    the binding equal the header's values (compiled with gcc)."""
    from paper_2409_03030_gb300 import jqcd
    names = ["JQCD_OK", "JQCD_EINVAL", "JQCD_ENOMEM", "JQCD_ECUDA", "JQCD_ENOCONV", "JQCD_EBUSY",
             "JQCD_ETIMEOUT", "JQCD_ENOTFOUND", "JQCD_EBREAKDOWN", "JQCD_PENDING", "JQCD_PREC_DW",
             "JQCD_PREC_F32", "JQCD_PREC_F16N", "JQCD_PREC_F64", "JQCD_CG_DW", "JQCD_CG_F64",
             "JQCD_CG_MIXED_F32", "JQCD_CG_MIXED_F16", "JQCD_NOALLOC_MAX_SITES_PER_PARITY"]
    src = tmp_path / "consts.c"
    src.write_text('#include "jqcd.h"\n#include <stdio.h>\nint main(void){'
                   + "".join(f'printf("%ld\\n", (long)({n}));' for n in names) + "return 0;}\n")
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [jqcd.OK, jqcd.EINVAL, jqcd.ENOMEM, jqcd.ECUDA, jqcd.ENOCONV, jqcd.EBUSY, jqcd.ETIMEOUT,
            jqcd.ENOTFOUND, jqcd.EBREAKDOWN, jqcd.PENDING, jqcd.PREC_DW, jqcd.PREC_F32,
            jqcd.PREC_F16N, jqcd.PREC_F64, jqcd.CG_DW, jqcd.CG_F64, jqcd.CG_MIXED_F32,
            jqcd.CG_MIXED_F16, jqcd.NOALLOC_MAX_SITES_PER_PARITY]
    assert got == want


def test_init_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2409_03030_gb300 import jqcd
    h = ctypes.c_void_p()
    assert jqcd.jqcd_init(0, ctypes.byref(h)) == jqcd.ECUDA
    assert not h.value
