"""The C ABI library: it builds, loads without a GPU, exports every function that
include/fb.h declares, and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

import paper_2311_09265_b300 as fbp
from paper_2311_09265_b300 import _build

HEADER = os.path.join(ROOT, "include", "fb.h")


@pytest.fixture(scope="module")
def libfb():
    _build.build()
    return fbp.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(fb_[a-z_0-9]+)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_hot_path_entry_points():
    names = declared_functions()
    for want in ("fb_nnf", "fb_remap", "fb_blend_window", "fb_interpolate"):
        assert want in names
    assert set(names) == set(fbp.HEADER_FUNCTIONS)


def test_library_exports_every_declared_symbol(libfb):
    missing = [n for n in declared_functions() if not hasattr(libfb, n)]
    assert not missing, missing


@pytest.mark.parametrize("variant", ["build_debug", "build_checked"])
def test_diagnostic_variants_export_every_declared_symbol(variant):
    """libfb_debug.so (candidate counter) and libfb_checked.so (device-side checks) are
    the same sources under a define: same ABI."""
    path = getattr(_build, variant)()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_product_library_reports_no_checks_without_touching_the_device(libfb):
    v = ctypes.c_uint64()
    assert libfb.fb_check_status(ctypes.byref(v), ctypes.byref(v), ctypes.byref(v), 0) == fbp.FB_ERR_UNSUPPORTED


def test_nnf_step_rejects_a_null_context(libfb):
    p = fbp.Params.make(5, 1)
    rc = libfb.fb_nnf_step(None, None, None, 16, 16, ctypes.byref(p), 0, None, None, None, None, None)
    assert rc == fbp.FB_ERR_ARG and b"ctx" in libfb.fb_last_error(None)


def test_library_is_built_for_sm_103a_only():
    out = os.popen(f"cuobjdump --list-elf {_build.LIB_PATH} 2>/dev/null").read()
    if not out:
        pytest.skip("cuobjdump unavailable")
    archs = set(re.findall(r"sm_(\d+a?)", out))
    assert archs == {"103a"}, archs


def test_pair_tag_packs_source_and_target(libfb):
    assert fbp.fb_pair_tag(3, 7) == (3 << 16) | 7
    assert fbp.fb_pair_tag(0, 0) == 0
    assert fbp.fb_pair_tag(65535, 65534) == 0xFFFFFFFE


def test_status_strings(libfb):
    assert libfb.fb_status_string(0) == b"FB_OK"
    assert libfb.fb_status_string(1) == b"FB_ERR_ARG"
    assert libfb.fb_status_string(4) == b"FB_ERR_TIMEOUT"


def test_null_context_is_rejected_before_any_device_work(libfb):
    p = fbp.Params.make(5, 4)
    rc = libfb.fb_nnf(None, None, None, 16, 16, ctypes.byref(p), None, None, None, None)
    assert rc == fbp.FB_ERR_ARG
    assert b"ctx" in libfb.fb_last_error(None)
    rc = libfb.fb_blend_window(None, None, None, 4, 16, 16, 3, ctypes.byref(p), None, None)
    assert rc == fbp.FB_ERR_ARG
    keys = (ctypes.c_int32 * 1)(0)
    rc = libfb.fb_interpolate(None, None, 4, 16, 16, ctypes.cast(keys, ctypes.c_void_p), None, 1,
                              ctypes.byref(p), None, None)
    assert rc == fbp.FB_ERR_ARG
    rc = libfb.fb_remap(None, None, None, 16, 16, 5, None, None)
    assert rc == fbp.FB_ERR_ARG
    assert libfb.fb_ctx_launches(None) == 0
    assert libfb.fb_ctx_destroy(None) == fbp.FB_OK


def test_params_struct_matches_header_layout():
    text = open(HEADER).read()
    body = re.search(r"typedef struct fb_params \{(.*?)\} fb_params;", text, re.S).group(1)
    fields = re.findall(r"(u?int\d+_t)\s+([a-z_0-9]+);", body)
    assert [f for _, f in fields] == [f for f, _ in fbp.Params._fields_]
    assert ctypes.sizeof(fbp.Params) == 40   # 36 bytes of fields, 8-byte aligned (seed)
