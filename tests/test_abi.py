"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/lbm.h declares, validates parameters before touching a
device, and the product path shares nothing with the oracle."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_1503_08406_gb300 import build
    build.build()
    import paper_1503_08406_gb300 as P
    P.load()
    return P


def test_every_declared_symbol_is_exported(P):
    names = P.declared_functions()
    assert len(names) >= 14
    lib = ctypes.CDLL(P.lbm.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", P.lbm.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lbm_\w+)", out))
    assert set(names) <= exported
    assert not any("ora_" in s for s in exported)


def test_params_struct_matches_header(P):
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} lbm_params;", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        typ, rest = decl.split(None, 1)
        for name in rest.split(","):
            fields.append(re.sub(r"\[.*\]", "", name).strip())
    assert fields == [f for f, _ in P.lbm_params._fields_]


def test_invalid_parameters_rejected_without_device(P):
    lib = P.load()
    cases = [
        dict(nx=2, ny=8),                                                   # too small
        dict(nx=8, ny=8, bc=("periodic", "dirichlet", "adiabatic", "adiabatic")),  # unpaired
        dict(nx=8, ny=8, bc=(7, 1, 2, 2)),                                  # unknown bc
        dict(nx=8, ny=8, storage=3),                                        # unknown storage
        dict(nx=8, ny=8, kernel_variant=3),                                 # unknown kernel
    ]
    for c in cases:
        nx, ny = c.pop("nx"), c.pop("ny")
        p = P.make_params(nx, ny, **c)
        n = ctypes.c_size_t()
        assert lib.lbm_workspace_bytes(ctypes.byref(p), ctypes.byref(n)) == -1
        h = ctypes.c_void_p()
        assert lib.lbm_create(ctypes.byref(p), None, None, 0, ctypes.byref(h)) == -1
        assert not h.value
    bad = [dict(flow=1, Ra=0.0, Pr=1.0, tau_nu=-1.0),          # nothing to derive tau_nu from
           dict(flow=0, tau_T=-1.0),                            # conduction needs tau_T
           dict(flow=0, tau_T=0.5),                             # tau_T must exceed 1/2
           dict(flow=0, tau_T=0.8, varpi=-4.0),                 # -4 < varpi < 1
           dict(flow=0, tau_T=0.8, T_s=0.1, T_l=0.0),           # T_l >= T_s
           dict(flow=0, tau_T=0.8, St=0.0)]
    for c in bad:
        p = P.make_params(16, 16, **c)
        h = ctypes.c_void_p()
        assert lib.lbm_create(ctypes.byref(p), None, None, 0, ctypes.byref(h)) == -1, c


def test_workspace_size_and_error_strings(P):
    p = P.make_params(2048, 2048, Ra=1e6, Pr=1.0)
    nbytes = P.lbm_workspace_bytes(p)
    n = 2048 * 2048
    # 14 population planes + f_l + phi + K + scratch pair + staging planes
    assert 25 * 4 * n <= nbytes < 32 * 4 * n
    # 16-bit storage halves the 14 population planes
    half = P.lbm_workspace_bytes(P.make_params(2048, 2048, Ra=1e6, Pr=1.0, storage="fp16"))
    assert nbytes - half == 14 * 2 * n
    assert P.lbm_workspace_bytes(P.make_params(2048, 2048, Ra=1e6, Pr=1.0, storage="bf16")) == half
    assert P.lbm_error_string(-4) == "inner enthalpy iteration hit its cap"
    assert P.lbm_error_string(-7) == "a bounded device-side wait timed out"
    assert P.lbm_error_string(0) == "ok"


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1503_08406_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b|lbm_oracle|\bora_\w+\(", text,
                                     re.M), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert not re.search(r"^\s*(import|from)\s+paper_1503_08406_gb300|#include\s+.lbm\.h",
                                 text, re.M), f
