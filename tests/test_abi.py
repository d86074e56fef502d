"""The C ABI: the library loads, exports every function include/ikr.h declares,
and the ctypes structures match the C layout.  No GPU needed."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ikr.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_02319_gb300 import ikr
    return ikr


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ikr_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ikr_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    cdll = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert getattr(cdll, n) is not None


def test_struct_layouts_match_the_header(lib, tmp_path):
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "ikr.h"\nint main(void){'
                   'printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(ikr_system), sizeof(ikr_eigenpairs),'
                   ' sizeof(ikr_report), sizeof(ikr_solve_opts), offsetof(ikr_report, history),'
                   ' offsetof(ikr_solve_opts, timeout_s)); return 0;}\n')
    exe = tmp_path / "sizes"
    cuda_inc = "/usr/local/cuda/include"
    r = subprocess.run(["gcc", str(src), f"-I{ROOT}/include", f"-I{cuda_inc}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    vals = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()))
    assert vals == [ctypes.sizeof(lib.System), ctypes.sizeof(lib.Eigenpairs), ctypes.sizeof(lib.Report),
                    ctypes.sizeof(lib.SolveOpts), lib.Report.history.offset, lib.SolveOpts.timeout_s.offset]


def test_host_only_calls(lib):
    o = lib.default_opts()
    assert o.tau == 1e-8 and o.m == 20 and o.strategy == lib.STRATEGIES["bal"] and o.s0 == 1.0
    assert lib._status_name(lib.IKR_ERR_NOGAP) == "IKR_ERR_NOGAP"
    assert "sm_103a" in lib.version()
    o = lib.default_opts(strategy="D10n", precision="mixed", tau=1e-6)
    assert o.strategy == 5 and o.precision == lib.MIXED and o.tau == 1e-6


def test_null_arguments_are_rejected(lib):
    h = ctypes.c_void_p()
    assert lib._LIB.ikr_setup_groundstate(None, None, None, ctypes.byref(h)) == lib.IKR_ERR_ARG
    assert not h.value
    assert lib._LIB.ikr_solve_response(None, 1, None, None, None, None, None) == lib.IKR_ERR_ARG
    assert lib._LIB.ikr_basis_size(None, 0, None) == lib.IKR_ERR_ARG
    assert lib._LIB.ikr_set_schur(None, 1) == lib.IKR_ERR_ARG
    assert lib._LIB.ikr_set_tensor_cores(None, 1) == lib.IKR_ERR_ARG
    assert lib._LIB.ikr_projection_coefficients(None, 0, 1, None, 1, None, None) == lib.IKR_ERR_ARG
    assert lib._LIB.ikr_project_out(None, 0, 1, None, 1, None) == lib.IKR_ERR_ARG
