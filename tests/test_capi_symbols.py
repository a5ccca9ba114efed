"""The C-ABI library builds, loads and exports every entry point of include/lspr.h
(no compute call: these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lspr.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"LSPR_API\s+(?:const\s+)?\w+\s*\*?\s*(lspr_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    from paper_1812_10722_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for required in ("lspr_create", "lspr_destroy", "lspr_mesh_upload", "lspr_tree_build", "lspr_matvec",
                     "lspr_solve", "lspr_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(_declared()) <= exported
    # nothing but the C ABI is exported
    assert {e for e in exported if not e.startswith("lspr_")} <= {"_init", "_fini"}


def test_status_strings(built):
    from paper_1812_10722_gb300 import lspr
    L = lspr.lib()
    for code in range(8):
        assert L.lspr_status_string(code)
    assert L.lspr_status_string(99) == b"unknown status"
    assert b"sm_103a" in L.lspr_version()


def test_no_gpu_fails_loudly(built):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1812_10722_gb300 import lspr
    with pytest.raises(lspr.LsprError):
        lspr.Context(0)


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "lspr.h"\nint main(void) { lspr_quad_opts q = {4, 19, 9, 0.5}; (void)q; return 0; }\n')
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-c",
                        str(src), "-o", str(tmp_path / "t.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_binding_structs_match_header(tmp_path):
    # the ctypes mirrors of the option/result structs have the header's layout
    from paper_1812_10722_gb300 import lspr
    names = {"lspr_quad_opts": lspr.QuadOpts, "lspr_solve_opts": lspr.SolveOpts,
             "lspr_solve_stats": lspr.SolveStats, "lspr_tune_opts": lspr.TuneOpts,
             "lspr_tune_result": lspr.TuneResult}
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "lspr.h"\nint main(void) {\n' +
                   "".join(f'    printf("{n} %zu\\n", sizeof({n}));\n' for n in names) + "    return 0;\n}\n")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    for line in out.split("\n"):
        if line:
            n, size = line.split()
            assert ctypes.sizeof(names[n]) == int(size), n
    r = lspr.SolveResult(None, None, None, None, None, 0.0, 0)   # a plain record
    assert r.seconds == 0.0
