"""CPU checks of the C ABI: the library loads, exports every symbol include/*.h declares, and rejects
invalid arguments before touching a device."""
import ctypes

import pytest

from paper_1811_03510_gb300 import build_ext, ccs


@pytest.fixture(scope="module")
def L():
    build_ext.build()
    return ccs.lib()


def test_exports_every_declared_symbol(L):
    names = ccs.declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n


def test_rejects_null_out_and_null_scene(L):
    assert L.ccs_scene_create(None, None, None, None, None, 0, 0, None) == ccs.CCS_ERR_INVALID_ARG
    assert b"out" in L.ccs_last_error()
    assert L.ccs_scene_info(None, None, None) == ccs.CCS_ERR_INVALID_ARG
    assert L.ccs_intersect(None, None, 0, None, None, None) == ccs.CCS_ERR_INVALID_ARG
    assert L.ccs_bvh_refit(None, None) == ccs.CCS_ERR_INVALID_ARG
    assert L.ccs_scene_destroy(None) == ccs.CCS_OK


def test_rejects_too_many_patches(L):
    h = ctypes.c_void_p()
    assert L.ccs_scene_create(ctypes.byref(h), None, None, None, None, (1 << 26) + 1, 0, None) == ccs.CCS_ERR_INVALID_ARG


def test_binding_raises_with_message(L):
    with pytest.raises(ccs.CcsError) as e:
        ccs._check(ccs.CCS_ERR_INVALID_ARG)
    assert "CCS_ERR_INVALID_ARG" in str(e.value)
