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


def test_binding_structs_and_constants_match_the_header(tmp_path):
    """The ctypes mirrors of the option, ray, hit and trial structs have the C layout of include/ccs.h,
    and the binding's constants equal the header's (checked with the host C compiler)."""
    import os
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    fields = [f[0] for f in ccs.ccs_trace_opts._fields_]
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "ccs.h"', "int main(void) {",
           'printf("opts %zu\\n", sizeof(ccs_trace_opts));',
           'printf("rays %zu\\n", sizeof(ccs_rays));', 'printf("hits %zu\\n", sizeof(ccs_hits));',
           'printf("trial %zu\\n", sizeof(ccs_autotune_trial));',
           'printf("NUM_COUNTERS %d\\n", CCS_NUM_COUNTERS);', 'printf("TRACE_COUNT %u\\n", CCS_TRACE_COUNT);',
           'printf("TRACE_ORDER %u\\n", CCS_TRACE_ORDER);', 'printf("CACHE_DEFAULT %u\\n", CCS_CACHE_DEFAULT);',
           'printf("TRACE_HOST_MAPPED %u\\n", CCS_TRACE_HOST_MAPPED);',
           'printf("TRACE_PAIRS %u\\n", CCS_TRACE_PAIRS);']
    src += [f'printf("off_{f} %zu\\n", offsetof(ccs_trace_opts, {f}));' for f in fields]
    src += ["return 0; }"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", inc, str(c), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    assert int(got["opts"]) == ctypes.sizeof(ccs.ccs_trace_opts)
    assert int(got["rays"]) == ctypes.sizeof(ccs.ccs_rays)
    assert int(got["hits"]) == ctypes.sizeof(ccs.ccs_hits)
    assert int(got["trial"]) == ctypes.sizeof(ccs.ccs_autotune_trial)
    for f in fields:
        assert int(got["off_" + f]) == getattr(ccs.ccs_trace_opts, f).offset, f
    assert int(got["NUM_COUNTERS"]) == ccs.CCS_NUM_COUNTERS == len(ccs.COUNTER_NAMES)
    assert int(got["TRACE_COUNT"]) == ccs.CCS_TRACE_COUNT
    assert int(got["TRACE_ORDER"]) == ccs.CCS_TRACE_ORDER
    assert int(got["TRACE_HOST_MAPPED"]) == ccs.CCS_TRACE_HOST_MAPPED
    assert int(got["TRACE_PAIRS"]) == ccs.CCS_TRACE_PAIRS
    assert int(got["CACHE_DEFAULT"]) == ccs.CCS_CACHE_DEFAULT
