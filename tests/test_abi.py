"""CPU checks of the C ABI: the library builds, loads, exports every entry point
declared in include/biot_pint.h, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_2310_10430_gb300 import biot
from paper_2310_10430_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "biot_pint.h")


@pytest.fixture(scope="module")
def L():
    B.build()
    return biot.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(biot_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("biot_mesh_create", "biot_assemble", "biot_precond_setup", "biot_pint_solve",
                     "biot_get_solution", "biot_destroy", "biot_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name
    out = os.popen(f"nm -D --defined-only {biot.LIB_PATH}").read()
    for name in declared_functions():
        assert re.search(rf"\bT {name}\b", out), name


def test_binding_covers_the_header():
    assert set(declared_functions()) <= set(biot._SIGNATURES)


def test_struct_layouts_match_header():
    # 8-byte aligned doubles/pointers, int32 members as declared
    assert ctypes.sizeof(biot.BiotParams) == 8 * 6 + 4 * 3 + 4 + 8 + 4 * 4
    # ... + inner, gmg_levels (int32) and the two power-method estimates (double)
    assert ctypes.sizeof(biot.BiotInfo) == 4 * 3 + 4 + 8 + 4 * 8 + 8 + 8 + 4 * 2 + 8 * 2
    # ... + spmm_variant (int32, padded to 8) and the two SpMM times
    assert ctypes.sizeof(biot.BiotTuning) == 4 * 8 + 8 * 4 + 4 * 2 + 4 * 2 + 8 * 2 + 8 + 8 * 2


def test_invalid_arguments_rejected_on_host(L):
    with pytest.raises(biot.BiotError) as e:
        biot.biot_mesh_create(0)
    assert e.value.status == biot.BIOT_E_INVALID
    with pytest.raises(biot.BiotError):
        biot.biot_mesh_create(5000)
    with pytest.raises(biot.BiotError):
        biot.biot_mesh_create(4, -1.0, 1.0)
    assert "n = 5000" in biot.biot_last_error(None) or "domain" in biot.biot_last_error(None)
    assert L.biot_get_info(None, None) == biot.BIOT_E_INVALID
    assert L.biot_sweep(None, 1, 1, None) == biot.BIOT_E_INVALID
    L.biot_destroy(None)
    assert biot.biot_launch_count() >= 0
