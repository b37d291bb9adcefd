"""ctypes binding of libckpp.so: argument marshalling only.

Every function here has the name of the C entry point it calls
(include/ckpp.h) and takes torch CUDA tensors in place of device pointers; all
work happens in the library's kernels. If the library is missing the import of
this module fails with a RuntimeError naming the build step: there is no
fallback.
"""

from __future__ import annotations

import ctypes as C
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libckpp.so")

CKPP_OK, CKPP_EINVAL, CKPP_ECUDA, CKPP_ESTALE, CKPP_EBUSY = 0, -1, -2, -3, -4
ST_INSERTED, ST_UPDATED, ST_FULL, ST_DELETED, ST_NOT_FOUND, ST_BUSY, ST_NO_TABLE = 1, 2, 3, 4, 5, 6, 7
CKPP_TIMERS = 1
SLOTS = 8


class ckpp_geometry(C.Structure):
    _fields_ = [("n_buckets", C.c_uint64), ("slots_per_bucket", C.c_uint32), ("flags", C.c_uint32),
                ("seed", C.c_uint64)]


class ckpp_stats(C.Structure):
    _fields_ = [("n_buckets", C.c_uint64), ("n_slots", C.c_uint64), ("n_occupied", C.c_uint64),
                ("n_live", C.c_uint64), ("n_in_secondary", C.c_uint64), ("n_moved_zero", C.c_uint64),
                ("moved_sum", C.c_uint64), ("bloom_bits_set", C.c_uint64), ("bloom_pop_sq", C.c_uint64),
                ("moved_hist", C.c_uint64 * 16)]


class ckpp_lookup_job(C.Structure):
    _fields_ = [("keys", C.c_void_p), ("out_vals", C.c_void_p), ("out_found", C.c_void_p), ("n", C.c_uint32),
                ("table", C.c_uint32)]


class ckpp_batch_tuning(C.Structure):
    _fields_ = [("threads_per_key", C.c_uint32), ("group_depth", C.c_uint32), ("blocks_per_sm", C.c_uint32),
                ("keys_per_warp", C.c_uint32)]


class ckpp_plan_config(C.Structure):
    _fields_ = [("insert_flush_s", C.c_double), ("lookup_hold_s", C.c_double), ("insert_flush_keys", C.c_uint64),
                ("footprint_bytes", C.c_uint64), ("bytes_per_key", C.c_uint64), ("max_jobs", C.c_uint32),
                ("overlap", C.c_uint32)]


class ckpp_turn(C.Structure):
    _fields_ = [("action", C.c_int32), ("pad", C.c_int32), ("wake", C.c_double), ("admitted_lo", C.c_int64),
                ("admitted_hi", C.c_int64), ("n_lookups", C.c_int64), ("n_inserts", C.c_int64),
                ("n_after", C.c_int64), ("insert_first", C.c_int64), ("insert_keys", C.c_int64),
                ("nbytes", C.c_int64), ("n_trailing", C.c_int64), ("nbytes_b", C.c_int64)]


class ckpp_serve_buffers(C.Structure):
    _fields_ = [("pool_keys", C.c_void_p), ("pool_vals", C.c_void_p), ("pool_found", C.c_void_p),
                ("n_tables", C.c_uint32), ("max_jobs", C.c_uint32), ("ins_keys", C.c_void_p),
                ("ins_tables", C.c_void_p), ("ins_vals", C.c_void_p), ("ins_status", C.c_void_p),
                ("ins_workspace", C.c_void_p), ("ins_workspace_bytes", C.c_size_t), ("d_jobs", C.c_void_p),
                ("h_jobs", C.c_void_p), ("ring_slots", C.c_uint32), ("max_inflight", C.c_uint32),
                ("batch_b", C.c_void_p)]


class ckpp_serve_stats(C.Structure):
    _fields_ = [("wall_s", C.c_double), ("gpu_busy_s", C.c_double), ("turns", C.c_uint64),
                ("launches", C.c_uint64), ("flushes", C.c_uint64), ("held", C.c_uint64), ("admitted", C.c_uint64),
                ("gpu_busy_b_s", C.c_double), ("trailing", C.c_uint64)]


LOOKUP_BLOOM, LOOKUP_OPTIMISTIC, LOOKUP_PESSIMISTIC = 0, 1, 2
PLAN_IDLE, PLAN_BLOCK, PLAN_NONE, PLAN_LAUNCH = 0, 1, 2, 3
BATCH_MAX_JOBS = 8192
JOB_BYTES = C.sizeof(ckpp_lookup_job)


class CkppError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {_lib.ckpp_error_string(code).decode()} ({code})")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1712_09624_gb300.build` "
                           "(or __graft_entry__.build()); there is no CPU fallback")
    L = C.CDLL(LIB_PATH)
    vp, u64, u32, u16, sz = C.c_void_p, C.c_uint64, C.c_uint32, C.c_uint16, C.c_size_t
    gp = C.POINTER(ckpp_geometry)
    sigs = {
        "ckpp_required_bytes": (sz, [gp]),
        "ckpp_workspace_bytes": (sz, [u64]),
        "ckpp_create": (C.c_int, [C.POINTER(vp), gp, vp, sz, vp]),
        "ckpp_destroy": (C.c_int, [vp]),
        "ckpp_attach": (C.c_int, [C.POINTER(vp), vp, sz, u32, vp]),
        "ckpp_bulk_lookup": (C.c_int, [vp, vp, u64, vp, vp, u32, u16, vp]),
        "ckpp_bulk_insert": (C.c_int, [vp, vp, vp, u64, u32, u16, vp, vp, sz, vp]),
        "ckpp_bulk_delete": (C.c_int, [vp, vp, u64, u32, vp, vp, sz, vp]),
        "ckpp_bulk_insert_noalloc": (C.c_int, [vp, vp, vp, u64, u32, u16, vp, vp]),
        "ckpp_expire": (C.c_int, [vp, u32, vp, vp]),
        "ckpp_stats_get": (C.c_int, [vp, u32, C.POINTER(ckpp_stats), vp]),
        "ckpp_lookup_probe_counts": (C.c_int, [vp, vp, u64, u32, C.c_int, vp, vp]),
        "ckpp_bulk_lookup_variant": (C.c_int, [vp, vp, u64, vp, vp, u32, u16, C.c_int, vp]),
        "ckpp_batch_bytes": (sz, [u32]),
        "ckpp_batch_create": (C.c_int, [C.POINTER(vp), C.POINTER(vp), u32, vp, sz, vp]),
        "ckpp_batch_destroy": (C.c_int, [vp]),
        "ckpp_batch_lookup": (C.c_int, [vp, vp, u32, vp, u32, C.POINTER(ckpp_batch_tuning), vp]),
        "ckpp_batch_insert": (C.c_int, [vp, vp, vp, vp, u64, u32, u16, vp, vp, sz, vp]),
        "ckpp_batch_delete": (C.c_int, [vp, vp, vp, u64, u32, vp, vp, sz, vp]),
        "ckpp_sync_status": (C.c_int, [vp, vp]),
        "ckpp_get_geometry": (C.c_int, [vp, gp]),
        "ckpp_get_last_scan": (C.c_int, [vp, C.POINTER(C.c_uint32), C.POINTER(C.c_int)]),
        "ckpp_shard_workspace_bytes": (sz, [u64, u32]),
        "ckpp_shard_partition": (C.c_int, [vp, vp, u64, u64, u32, vp, vp, vp, vp, vp, sz, vp]),
        "ckpp_shard_unpermute": (C.c_int, [vp, u64, vp, vp, vp, vp, vp]),
        "ckpp_set_insert_launch": (C.c_int, [C.c_int]),
        # include/ckpp_serve.h (host code)
        "ckpp_plan_create": (C.c_int, [vp, vp, vp, vp, vp, C.c_int64, C.POINTER(ckpp_plan_config), C.POINTER(vp)]),
        "ckpp_plan_destroy": (C.c_int, [vp]),
        "ckpp_plan_next": (C.c_int, [vp, C.c_double, C.c_int, C.POINTER(ckpp_turn), vp, vp, vp, vp, C.c_int64]),
        "ckpp_plan_complete": (C.c_int, [vp, C.c_int64]),
        "ckpp_plan_complete_b": (C.c_int, [vp, C.c_int64, C.c_int]),
        "ckpp_plan_state": (C.c_int, [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
        "ckpp_serve_stage_jobs": (C.c_int, [vp, C.c_int64, vp, vp, vp, vp, vp, vp, vp]),
        "ckpp_serve_run": (C.c_int, [vp, vp, C.POINTER(ckpp_serve_buffers), C.POINTER(ckpp_batch_tuning), vp, vp,
                                     C.POINTER(ckpp_serve_stats)]),
        "ckpp_serve_run_plain": (C.c_int, [vp, vp, C.POINTER(ckpp_serve_buffers), vp, vp,
                                           C.POINTER(ckpp_serve_stats)]),
        "ckpp_error_string": (C.c_char_p, [C.c_int]),
        "ckpp_abi_version": (C.c_int, []),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


_lib = _load()
EXPORTED = ("ckpp_required_bytes", "ckpp_workspace_bytes", "ckpp_create", "ckpp_destroy", "ckpp_bulk_lookup",
            "ckpp_bulk_insert", "ckpp_bulk_delete", "ckpp_expire", "ckpp_stats_get", "ckpp_lookup_probe_counts",
            "ckpp_sync_status", "ckpp_get_geometry", "ckpp_get_last_scan", "ckpp_error_string",
            "ckpp_abi_version", "ckpp_bulk_insert_noalloc", "ckpp_bulk_lookup_variant", "ckpp_batch_bytes",
            "ckpp_batch_create", "ckpp_batch_destroy", "ckpp_batch_lookup", "ckpp_batch_insert",
            "ckpp_batch_delete", "ckpp_shard_workspace_bytes", "ckpp_shard_partition", "ckpp_shard_unpermute",
            "ckpp_set_insert_launch", "ckpp_attach")
SERVE_EXPORTED = ("ckpp_plan_create", "ckpp_plan_destroy", "ckpp_plan_next", "ckpp_plan_complete",
                  "ckpp_plan_complete_b", "ckpp_plan_state", "ckpp_serve_stage_jobs", "ckpp_serve_run",
                  "ckpp_serve_run_plain")
INSERT_LAUNCH_CHAIN, INSERT_LAUNCH_SINGLE = 0, 1
NOALLOC_MAX_KEYS = 65536
MAX_SHARDS = 64


def library():
    return _lib


def _check(rc: int, what: str):
    if rc != CKPP_OK:
        raise CkppError(rc, what)


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: torch.Tensor | None):
    return None if t is None else t.data_ptr()


def _dev(t: torch.Tensor, name: str, dtype=None):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype not in (dtype if isinstance(dtype, tuple) else (dtype,)):
        raise TypeError(f"{name} has dtype {t.dtype}, expected {dtype}")
    return t


def geometry(n_buckets: int, timers: bool = False, seed: int = 0) -> ckpp_geometry:
    return ckpp_geometry(n_buckets, SLOTS, CKPP_TIMERS if timers else 0, seed)


def ckpp_required_bytes(geo: ckpp_geometry) -> int:
    return int(_lib.ckpp_required_bytes(C.byref(geo)))


def ckpp_workspace_bytes(n: int) -> int:
    return int(_lib.ckpp_workspace_bytes(n))


def ckpp_create(geo: ckpp_geometry, buf: torch.Tensor, stream=None) -> int:
    _dev(buf, "buf", torch.uint8)
    h = C.c_void_p()
    _check(_lib.ckpp_create(C.byref(h), C.byref(geo), _ptr(buf), buf.numel(), _stream(stream)), "ckpp_create")
    return h.value


def ckpp_destroy(handle: int):
    _check(_lib.ckpp_destroy(handle), "ckpp_destroy")


def _dev_or_pinned(t: torch.Tensor, name: str, dtype):
    if t.is_cuda:
        return _dev(t, name, dtype)
    if not t.is_pinned():
        raise ValueError(f"{name} must be a CUDA tensor or pinned host memory")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.dtype not in (dtype if isinstance(dtype, tuple) else (dtype,)):
        raise TypeError(f"{name} has dtype {t.dtype}, expected {dtype}")
    return t


def ckpp_bulk_lookup(handle: int, keys: torch.Tensor, out_vals: torch.Tensor, out_found: torch.Tensor,
                     now: int = 0, refresh_ttl: int = 0, stream=None):
    """Device tensors, or pinned host tensors read/written in place by the kernel."""
    n = keys.shape[0]
    _dev_or_pinned(keys, "keys", torch.uint8)
    _dev_or_pinned(out_vals, "out_vals", (torch.int64, torch.uint64))
    _dev_or_pinned(out_found, "out_found", (torch.uint8, torch.bool))
    _check(_lib.ckpp_bulk_lookup(handle, _ptr(keys), n, _ptr(out_vals), _ptr(out_found), now, refresh_ttl,
                                 _stream(stream)), "ckpp_bulk_lookup")


def ckpp_bulk_insert(handle: int, keys: torch.Tensor, vals: torch.Tensor, status: torch.Tensor,
                     workspace: torch.Tensor, now: int = 0, ttl: int = 0, stream=None):
    n = keys.shape[0]
    _dev(keys, "keys", torch.uint8)
    _dev(vals, "vals", (torch.int64, torch.uint64))
    _dev(status, "status", torch.uint8)
    _dev(workspace, "workspace", torch.uint8)
    _check(_lib.ckpp_bulk_insert(handle, _ptr(keys), _ptr(vals), n, now, ttl, _ptr(status), _ptr(workspace),
                                 workspace.numel(), _stream(stream)), "ckpp_bulk_insert")


def ckpp_bulk_insert_noalloc(handle: int, keys: torch.Tensor, vals: torch.Tensor, status: torch.Tensor,
                             now: int = 0, ttl: int = 0, stream=None):
    """Insert without a workspace, for callers that cannot allocate device
    memory: the library's built-in scratch array (at most NOALLOC_MAX_KEYS keys
    per call; calls that overlap on the GPU must not share it)."""
    n = keys.shape[0]
    _dev(keys, "keys", torch.uint8)
    _dev(vals, "vals", (torch.int64, torch.uint64))
    _dev(status, "status", torch.uint8)
    _check(_lib.ckpp_bulk_insert_noalloc(handle, _ptr(keys), _ptr(vals), n, now, ttl, _ptr(status),
                                         _stream(stream)), "ckpp_bulk_insert_noalloc")


def ckpp_bulk_delete(handle: int, keys: torch.Tensor, status: torch.Tensor, workspace: torch.Tensor,
                     now: int = 0, stream=None):
    n = keys.shape[0]
    _dev(keys, "keys", torch.uint8)
    _dev(status, "status", torch.uint8)
    _dev(workspace, "workspace", torch.uint8)
    _check(_lib.ckpp_bulk_delete(handle, _ptr(keys), n, now, _ptr(status), _ptr(workspace), workspace.numel(),
                                 _stream(stream)), "ckpp_bulk_delete")


def ckpp_expire(handle: int, now: int, d_n_expired: torch.Tensor | None = None, stream=None):
    if d_n_expired is not None:
        _dev(d_n_expired, "d_n_expired", (torch.int64, torch.uint64))
    _check(_lib.ckpp_expire(handle, now, _ptr(d_n_expired), _stream(stream)), "ckpp_expire")


def ckpp_stats_get(handle: int, now: int = 0, stream=None) -> dict:
    s = ckpp_stats()
    _check(_lib.ckpp_stats_get(handle, now, C.byref(s), _stream(stream)), "ckpp_stats_get")
    out = {name: getattr(s, name) for name, _ in ckpp_stats._fields_ if name != "moved_hist"}
    out["moved_hist"] = list(s.moved_hist)
    return out


def ckpp_lookup_probe_counts(handle: int, keys: torch.Tensor, d_counts: torch.Tensor, now: int = 0,
                             variant: int = LOOKUP_BLOOM, stream=None):
    _dev(keys, "keys", torch.uint8)
    _dev(d_counts, "d_counts", (torch.int64, torch.uint64))
    if d_counts.numel() < 4:
        raise ValueError("d_counts needs 4 elements")
    _check(_lib.ckpp_lookup_probe_counts(handle, _ptr(keys), keys.shape[0], now, variant, _ptr(d_counts),
                                         _stream(stream)), "ckpp_lookup_probe_counts")


def ckpp_bulk_lookup_variant(handle: int, keys: torch.Tensor, out_vals: torch.Tensor, out_found: torch.Tensor,
                             now: int = 0, refresh_ttl: int = 0, variant: int = LOOKUP_BLOOM, stream=None):
    _dev(keys, "keys", torch.uint8)
    _dev(out_vals, "out_vals", (torch.int64, torch.uint64))
    _dev(out_found, "out_found", (torch.uint8, torch.bool))
    _check(_lib.ckpp_bulk_lookup_variant(handle, _ptr(keys), keys.shape[0], _ptr(out_vals), _ptr(out_found), now,
                                         refresh_ttl, variant, _stream(stream)), "ckpp_bulk_lookup_variant")


def ckpp_batch_bytes(n_tables: int) -> int:
    return int(_lib.ckpp_batch_bytes(n_tables))


def ckpp_batch_create(handles, buf: torch.Tensor, stream=None) -> int:
    _dev(buf, "buf", torch.uint8)
    arr = (C.c_void_p * len(handles))(*handles)
    h = C.c_void_p()
    _check(_lib.ckpp_batch_create(C.byref(h), arr, len(handles), _ptr(buf), buf.numel(), _stream(stream)),
           "ckpp_batch_create")
    return h.value


def ckpp_batch_destroy(handle: int):
    _check(_lib.ckpp_batch_destroy(handle), "ckpp_batch_destroy")


def ckpp_batch_insert(handle: int, keys: torch.Tensor, table_ids: torch.Tensor, vals: torch.Tensor,
                      status: torch.Tensor, workspace: torch.Tensor, now: int = 0, ttl: int = 0, stream=None):
    n = keys.shape[0]
    _dev(keys, "keys", torch.uint8)
    _dev(table_ids, "table_ids", (torch.int32, torch.uint32))
    _dev(vals, "vals", (torch.int64, torch.uint64))
    _dev(status, "status", torch.uint8)
    _dev(workspace, "workspace", torch.uint8)
    _check(_lib.ckpp_batch_insert(handle, _ptr(keys), _ptr(table_ids), _ptr(vals), n, now, ttl, _ptr(status),
                                  _ptr(workspace), workspace.numel(), _stream(stream)), "ckpp_batch_insert")


def ckpp_batch_delete(handle: int, keys: torch.Tensor, table_ids: torch.Tensor, status: torch.Tensor,
                      workspace: torch.Tensor, now: int = 0, stream=None):
    n = keys.shape[0]
    _dev(keys, "keys", torch.uint8)
    _dev(table_ids, "table_ids", (torch.int32, torch.uint32))
    _dev(status, "status", torch.uint8)
    _dev(workspace, "workspace", torch.uint8)
    _check(_lib.ckpp_batch_delete(handle, _ptr(keys), _ptr(table_ids), n, now, _ptr(status), _ptr(workspace),
                                  workspace.numel(), _stream(stream)), "ckpp_batch_delete")


def ckpp_batch_lookup(handle: int, d_jobs: torch.Tensor, max_jobs: int, d_n_jobs: torch.Tensor | None = None,
                      now: int = 0, tuning: tuple | None = None, stream=None):
    """d_jobs: device uint8 tensor holding max_jobs ckpp_lookup_job records.
    tuning: (threads_per_key, group_depth, blocks_per_sm[, keys_per_warp]); threads_per_key 1, 2 or 4,
    keys_per_warp 0 or 32 / threads_per_key."""
    _dev(d_jobs, "d_jobs", torch.uint8)
    if d_jobs.numel() < max_jobs * JOB_BYTES:
        raise ValueError("d_jobs holds fewer than max_jobs jobs")
    if d_n_jobs is not None:
        _dev(d_n_jobs, "d_n_jobs", (torch.int32, torch.uint32))
    tn = None if tuning is None else C.byref(
        ckpp_batch_tuning(tuning[0], tuning[1], tuning[2], tuning[3] if len(tuning) > 3 else 0))
    _check(_lib.ckpp_batch_lookup(handle, _ptr(d_jobs), max_jobs, _ptr(d_n_jobs), now, tn, _stream(stream)),
           "ckpp_batch_lookup")


def ckpp_sync_status(handle: int, stream=None) -> int:
    rc = _lib.ckpp_sync_status(handle, _stream(stream))
    if rc not in (CKPP_OK, CKPP_EBUSY):
        _check(rc, "ckpp_sync_status")
    return rc


def ckpp_get_last_scan(handle: int) -> tuple[int, bool]:
    t = C.c_uint32()
    e = C.c_int()
    _check(_lib.ckpp_get_last_scan(handle, C.byref(t), C.byref(e)), "ckpp_get_last_scan")
    return t.value, bool(e.value)


def ckpp_abi_version() -> int:
    return int(_lib.ckpp_abi_version())


def ckpp_shard_workspace_bytes(n: int, n_shards: int) -> int:
    return int(_lib.ckpp_shard_workspace_bytes(n, n_shards))


def ckpp_shard_partition(keys: torch.Tensor, vals: torch.Tensor | None, seed: int, n_shards: int,
                         out_pos: torch.Tensor, out_keys: torch.Tensor, out_vals: torch.Tensor | None,
                         out_counts: torch.Tensor, workspace: torch.Tensor, stream=None):
    n = keys.shape[0]
    _dev(keys, "keys", torch.uint8)
    _dev(out_pos, "out_pos", (torch.int32, torch.uint32))
    _dev(out_keys, "out_keys", torch.uint8)
    _dev(out_counts, "out_counts", (torch.int64, torch.uint64))
    _dev(workspace, "workspace", torch.uint8)
    for t, name in ((vals, "vals"), (out_vals, "out_vals")):
        if t is not None:
            _dev(t, name, (torch.int64, torch.uint64))
    _check(_lib.ckpp_shard_partition(_ptr(keys), _ptr(vals), n, seed & (2**64 - 1), n_shards, _ptr(out_pos),
                                     _ptr(out_keys), _ptr(out_vals), _ptr(out_counts), _ptr(workspace),
                                     workspace.numel(), _stream(stream)), "ckpp_shard_partition")


def ckpp_shard_unpermute(pos: torch.Tensor, in_u64: torch.Tensor | None, in_u8: torch.Tensor | None,
                         out_u64: torch.Tensor | None, out_u8: torch.Tensor | None, stream=None):
    n = pos.shape[0]
    _dev(pos, "pos", (torch.int32, torch.uint32))
    for t, name in ((in_u64, "in_u64"), (out_u64, "out_u64"), (in_u8, "in_u8"), (out_u8, "out_u8")):
        if t is not None:
            _dev(t, name)
    _check(_lib.ckpp_shard_unpermute(_ptr(pos), n, _ptr(in_u64), _ptr(in_u8), _ptr(out_u64), _ptr(out_u8),
                                     _stream(stream)), "ckpp_shard_unpermute")


def ckpp_set_insert_launch(mode: int) -> int:
    """Process-wide launch mode of insert calls (INSERT_LAUNCH_*); returns the previous one."""
    rc = _lib.ckpp_set_insert_launch(mode)
    if rc < 0:
        raise CkppError(rc, "ckpp_set_insert_launch")
    return rc


def ckpp_attach(buf: torch.Tensor, now: int = 0, stream=None) -> int:
    """Handle over a table whose bytes already sit in buf (a uint8 CUDA tensor):
    checkpoint and resume, see include/ckpp.h."""
    _dev(buf, "buf", torch.uint8)
    h = C.c_void_p()
    _check(_lib.ckpp_attach(C.byref(h), _ptr(buf), buf.numel(), now, _stream(stream)), "ckpp_attach")
    return h.value
