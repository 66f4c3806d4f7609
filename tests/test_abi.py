"""CPU-side checks of the boundary: the library builds for sm_103a, loads,
and exports every symbol include/lbmd.h declares (no compute call without a
GPU); the ctypes structures match the header's layout."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1610_02733_gb300 import build_lib, lbmd
    build_lib.build()
    return lbmd.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "lbmd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbmd_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    from paper_1610_02733_gb300 import lbmd
    declared = _declared()
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(lbmd.EXPORTS) == declared


def test_params_struct_layout():
    from paper_1610_02733_gb300 import lbmd
    P = lbmd.LbmdParams
    # six int32, then doubles from offset 24
    assert P.rho0.offset == 24
    assert P.body_force.offset == 24 + 6 * 8
    assert P.seed.offset == 24 + 9 * 8
    assert P.stream.offset == 24 + 12 * 8
    assert P.integrator.offset == 24 + 13 * 8
    assert P.spread.offset == 24 + 13 * 8 + 4 and P.noise.offset == 24 + 14 * 8
    assert ct.sizeof(P) == 24 + 15 * 8  # three int32 at the end, padded to 8 bytes
    O = lbmd.LbmdObservables
    assert O.lb_step.offset == 9 * 8 and ct.sizeof(O) == 11 * 8


def test_status_strings_without_gpu(lib):
    for s in (0, -1, -2, -3, -4, -5, -6, -7):
        assert lib.lbmd_status_string(s)


def test_product_package_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_1610_02733_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                for bad in ("import oracle", "from oracle", "lbmd_oracle", "orc_"):
                    assert bad not in text, (f, bad)


def test_params_layout_matches_the_c_compiler(tmp_path):
    # every field offset of the ctypes mirror equals the C compiler's offsetof
    import os
    import subprocess
    from paper_1610_02733_gb300 import lbmd
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    names = [f[0] for f in lbmd.LbmdParams._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbmd.h"\nint main(void) {\n' +
                   "".join('printf("%%zu\\n", offsetof(lbmd_params, %s));\n' % n for n in names) +
                   'printf("%zu\\n", sizeof(lbmd_params));\nreturn 0;\n}\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", inc, str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [getattr(lbmd.LbmdParams, n).offset for n in names] + [ct.sizeof(lbmd.LbmdParams)]
    assert got == want

