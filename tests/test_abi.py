"""The C ABI library loads and exports every entry point include/ckpp.h
declares; host-only calls behave as documented (no GPU needed)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ckpp.h")


def declared_functions():
    text = open(HEADER).read()  # the method's ABI (ckpp_workload.h is checked separately)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ckpp_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def K():
    from paper_1712_09624_gb300 import build
    build.build()
    from paper_1712_09624_gb300 import _ckpp
    return _ckpp


def test_workload_library_exports(K):
    from paper_1712_09624_gb300 import build
    text = open(os.path.join(ROOT, "include", "ckpp_workload.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = sorted(set(re.findall(r"\b(ckpp_wl_[a-z_0-9]+)\s*\(", text)))
    assert names == ["ckpp_wl_fill_keys", "ckpp_wl_host_io", "ckpp_wl_keys_at", "ckpp_wl_l2_read",
                     "ckpp_wl_lookup_batch"]
    lib = ctypes.CDLL(build.WL_LIB)
    for name in names:
        assert hasattr(lib, name)


def test_serve_runtime_exports(K):
    """include/ckpp_serve.h (the served form's host runtime) is exported by
    libckpp.so and bound by name."""
    text = open(os.path.join(ROOT, "include", "ckpp_serve.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = sorted(set(re.findall(r"\b(ckpp_[a-z_0-9]+)\s*\(", text)))
    assert set(K.SERVE_EXPORTED) == set(names) and len(names) == 9
    lib = ctypes.CDLL(K.LIB_PATH)
    for name in names:
        assert hasattr(lib, name)


def test_every_declared_symbol_is_exported(K):
    names = declared_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(K.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), f"{name} declared in ckpp.h but not exported"
    assert set(K.EXPORTED) == set(names)


def test_host_only_calls(K):
    assert K.ckpp_abi_version() == 3
    g = K.geometry(1 << 24)
    assert K.ckpp_required_bytes(g) == 256 + (1 << 24) * 256  # 256-byte buckets, entries inside
    gt = K.geometry(1 << 24, timers=True)
    assert K.ckpp_required_bytes(gt) == 256 + (1 << 24) * 256
    for bad in (K.geometry(1), K.geometry(0), K.geometry(1 << 32)):
        assert K.ckpp_required_bytes(bad) == 0
    wrong_slots = K.ckpp_geometry(1024, 4, 0, 0)
    assert K.ckpp_required_bytes(wrong_slots) == 0
    assert K.ckpp_workspace_bytes(0) > 0
    # the dedup set: 8 bytes per position, 8 positions per key up to 2^17 keys, 4 above
    assert K.ckpp_workspace_bytes(1 << 20) >= 8 * (4 << 20) + 8 * (1 << 20)
    assert K.ckpp_workspace_bytes(1 << 12) >= 8 * (8 << 12) + 8 * (1 << 12)
    assert K.ckpp_workspace_bytes(1 << 30) >= 8 * (4 << 30)
    assert K.ckpp_workspace_bytes((1 << 30) + 1) == 0
    lib = K.library()
    assert lib.ckpp_error_string(-3).decode().startswith("more than 64512")
    # argument checks return before touching the device
    h = ctypes.c_void_p()
    assert lib.ckpp_create(ctypes.byref(h), ctypes.byref(g), None, 0, None) == K.CKPP_EINVAL
    assert lib.ckpp_destroy(None) == K.CKPP_EINVAL
    assert lib.ckpp_bulk_lookup(None, None, 0, None, None, 0, 0, None) == K.CKPP_EINVAL


def test_insert_launch_mode_is_host_state(K):
    """The insert launch mode is a host-side setting: unknown modes are
    rejected and a set returns the previous mode (no GPU needed)."""
    prev = K.ckpp_set_insert_launch(K.INSERT_LAUNCH_CHAIN)
    try:
        assert K.ckpp_set_insert_launch(K.INSERT_LAUNCH_SINGLE) == K.INSERT_LAUNCH_CHAIN
        assert K.library().ckpp_set_insert_launch(7) == K.CKPP_EINVAL
        assert K.ckpp_set_insert_launch(K.INSERT_LAUNCH_CHAIN) == K.INSERT_LAUNCH_SINGLE
    finally:
        K.ckpp_set_insert_launch(prev)
