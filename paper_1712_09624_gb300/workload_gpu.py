"""Device-side twin of ``workload``: the same seeded keys, lookup batches and
expected answers, drawn directly in device memory by libckpp_workload.so
(include/ckpp_workload.h). Used where a workload is too large to draw on the
host (billions of keys); tests check it against ``workload`` bit for bit."""

from __future__ import annotations

import ctypes as C
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libckpp_workload.so")


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1712_09624_gb300.build`")
    L = C.CDLL(LIB_PATH)
    u64, vp = C.c_uint64, C.c_void_p
    L.ckpp_wl_fill_keys.restype = C.c_int
    L.ckpp_wl_fill_keys.argtypes = [u64, u64, u64, vp, vp, vp]
    L.ckpp_wl_lookup_batch.restype = C.c_int
    L.ckpp_wl_lookup_batch.argtypes = [u64, u64, u64, u64, C.c_double, vp, vp, vp, vp]
    L.ckpp_wl_keys_at.restype = C.c_int
    L.ckpp_wl_keys_at.argtypes = [u64, vp, u64, vp, vp]
    L.ckpp_wl_l2_read.restype = C.c_int
    L.ckpp_wl_l2_read.argtypes = [vp, u64, C.c_uint32, vp, vp]
    L.ckpp_wl_host_io.restype = C.c_int
    L.ckpp_wl_host_io.argtypes = [vp, u64, vp, vp, vp]
    return L


_lib = _load()


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def fill_keys(seed: int, first: int, n: int, device, stream=None, with_values: bool = True):
    """Keys [first, first+n) of workload.fill(seed, .) and their values."""
    keys = torch.empty((n, 16), dtype=torch.uint8, device=device)
    vals = torch.empty(n, dtype=torch.int64, device=device) if with_values else None
    rc = _lib.ckpp_wl_fill_keys(seed & (2**64 - 1), first, n, keys.data_ptr() if n else None,
                                vals.data_ptr() if (vals is not None and n) else None, _stream(stream))
    if rc:
        raise RuntimeError(f"ckpp_wl_fill_keys failed ({rc})")
    return keys, vals


def keys_at(seed: int, idx: torch.Tensor, stream=None) -> torch.Tensor:
    """Keys idx[i] of workload.fill(seed, .) for a device int64 index tensor."""
    n = idx.shape[0]
    keys = torch.empty((n, 16), dtype=torch.uint8, device=idx.device)
    rc = _lib.ckpp_wl_keys_at(seed & (2**64 - 1), idx.data_ptr() if n else None, n,
                              keys.data_ptr() if n else None, _stream(stream))
    if rc:
        raise RuntimeError(f"ckpp_wl_keys_at failed ({rc})")
    return keys


def lookup_batch(seed: int, n: int, n_inserted: int, neg_rate: float, batch_id: int = 0, device=None, stream=None):
    """workload.lookup_batch(seed, n, workload.fill(seed, n_inserted), neg_rate, batch_id) on the device:
    (keys, expect_found uint8, expect_value int64)."""
    keys = torch.empty((n, 16), dtype=torch.uint8, device=device)
    found = torch.empty(n, dtype=torch.uint8, device=device)
    value = torch.empty(n, dtype=torch.int64, device=device)
    rc = _lib.ckpp_wl_lookup_batch(seed & (2**64 - 1), batch_id, n, n_inserted, float(neg_rate),
                                   keys.data_ptr() if n else None, found.data_ptr() if n else None,
                                   value.data_ptr() if n else None, _stream(stream))
    if rc:
        raise RuntimeError(f"ckpp_wl_lookup_batch failed ({rc})")
    return keys, found, value


def l2_read(buf: torch.Tensor, passes: int, sink: torch.Tensor, stream=None):
    """Stream buf (a uint8 CUDA tensor, size a multiple of 16) passes times
    through the L2 read probe (ckpp_wl_l2_read)."""
    rc = _lib.ckpp_wl_l2_read(buf.data_ptr(), buf.numel(), passes, sink.data_ptr(), _stream(stream))
    if rc != 0:
        raise RuntimeError(f"ckpp_wl_l2_read failed ({rc})")


def host_io(keys: torch.Tensor, out_vals: torch.Tensor, out_found: torch.Tensor, stream=None):
    """The host I/O of a lookup without the table (see ckpp_wl_host_io): keys
    [n, 16] uint8, out_vals [n] int64, out_found [n] uint8 or bool, each pinned
    host or device memory."""
    n = keys.shape[0]
    rc = _lib.ckpp_wl_host_io(keys.data_ptr() if n else None, n, out_vals.data_ptr() if n else None,
                              out_found.data_ptr() if n else None, _stream(stream))
    if rc != 0:
        raise RuntimeError(f"ckpp_wl_host_io failed ({rc})")
