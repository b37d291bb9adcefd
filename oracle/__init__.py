"""Cuckoo++ CPU oracle (test infrastructure).

This package is the checker, not the product: only the tests, the smoke check
and the bench's CPU-baseline leg import it. It holds

* ``ckpp_oracle.c`` -- the method step by step (Sec. 2, 4.1, 4.2 and 4.3 of the
  paper) as a plain single-threaded C table, loaded here through ctypes;
* ``odef.py``       -- the plain definition every lookup/insert/delete result must
  equal: a Python dict from key to (value, expiry).

Neither shares code with the CUDA library. The C file is compiled with gcc on
first use (or by ``build()``) into ``libckpp_oracle.so`` beside it.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ckpp_oracle.c")
_LIB = os.path.join(_HERE, "libckpp_oracle.so")

INSERTED, UPDATED, FULL, DELETED, NOT_FOUND = 1, 2, 3, 4, 5
OK, EINVAL, ESTALE = 0, -1, -3
SEED2_XOR = 0x9E3779B97F4A7C15

_lib = None


def build(force: bool = False, out: str | None = None, mutant: int = 0) -> str:
    """Compile the oracle with gcc (plain -O2, no target-specific flags).

    ``mutant`` > 0 builds a copy with one planted mistake (for the tests that
    check the pins catch it) into ``out``."""
    target = out or _LIB
    if mutant or out or force or not os.path.exists(target) or os.path.getmtime(target) < os.path.getmtime(_SRC):
        tmp = target + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-shared", "-fPIC",
                               f"-DOC_MUTANT={int(mutant)}", "-o", tmp, _SRC])
        os.replace(tmp, target)
    return target


def _u8p(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint8))


def _u16p(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint16))


def _u32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint32))


def _u64p(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint64))


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def load(path: str):
    """Load an oracle shared library and declare its signatures."""
    L = C.CDLL(path)
    vp, u8p, u16p, u32p, u64p = (C.c_void_p, C.POINTER(C.c_uint8), C.POINTER(C.c_uint16),
                                 C.POINTER(C.c_uint32), C.POINTER(C.c_uint64))
    L.oc_mix64.restype = C.c_uint64
    L.oc_mix64.argtypes = [C.c_uint64]
    L.oc_hash.restype = C.c_uint64
    L.oc_hash.argtypes = [u8p, C.c_uint64]
    L.oc_alive.restype = C.c_int
    L.oc_alive.argtypes = [C.c_uint16, C.c_uint32]
    L.oc_address_batch.restype = None
    L.oc_address_batch.argtypes = [C.c_uint64, C.c_uint64, u8p, C.c_uint64, u64p, u64p, u64p, u64p,
                                   u16p, u8p, u8p]
    L.oc_create.restype = vp
    L.oc_create.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64]
    L.oc_destroy.restype = None
    L.oc_destroy.argtypes = [vp]
    L.oc_insert.restype = C.c_int
    L.oc_insert.argtypes = [vp, u8p, u64p, C.c_uint64, C.c_uint32, C.c_uint32, u8p]
    L.oc_lookup.restype = C.c_int
    L.oc_lookup.argtypes = [vp, u8p, C.c_uint64, C.c_uint32, C.c_uint32, u64p, u8p]
    L.oc_delete.restype = C.c_int
    L.oc_delete.argtypes = [vp, u8p, C.c_uint64, C.c_uint32, u8p]
    L.oc_expire.restype = C.c_int64
    L.oc_expire.argtypes = [vp, C.c_uint32]
    L.oc_size.restype = C.c_uint64
    L.oc_size.argtypes = [vp]
    L.oc_dump.restype = C.c_uint64
    L.oc_dump.argtypes = [vp, u8p, u64p, u16p, u64p, u8p, u8p]
    L.oc_meta_dump.restype = None
    L.oc_meta_dump.argtypes = [vp, u64p, u32p]
    L.oc_lookup_probe_counts.restype = None
    L.oc_lookup_probe_counts.argtypes = [vp, u8p, C.c_uint64, C.c_uint32, u64p, u64p]
    L.oc_check_invariants.restype = C.c_int
    L.oc_check_invariants.argtypes = [vp, C.c_int, u64p]
    L.oc_nb.restype = C.c_uint64
    L.oc_nb.argtypes = [vp]
    L.oc_slots.restype = C.c_uint32
    L.oc_slots.argtypes = [vp]
    return L


def _keys(keys) -> np.ndarray:
    k = np.ascontiguousarray(keys, dtype=np.uint8)
    if k.ndim != 2 or k.shape[1] != 16:
        k = k.reshape(-1, 16)
    return k


def mix64(z: int) -> int:
    return int(lib().oc_mix64(z))


def hash_key(key, seed: int) -> int:
    k = _keys(key)
    return int(lib().oc_hash(_u8p(k), seed))


def alive(expiry: int, now: int, library=None) -> bool:
    return bool((library or lib()).oc_alive(expiry & 0xFFFF, now & 0xFFFFFFFF))


def address(keys, nb: int, seed: int, library=None) -> dict:
    """H1, H2, b1, b2, tag, bloom bit indices of every key (C1-C4 readings)."""
    k = _keys(keys)
    n = k.shape[0]
    out = {name: np.zeros(n, dt) for name, dt in (("h1", np.uint64), ("h2", np.uint64), ("b1", np.uint64),
                                                  ("b2", np.uint64), ("tag", np.uint16), ("bit1", np.uint8),
                                                  ("bit2", np.uint8))}
    (library or lib()).oc_address_batch(nb, seed, _u8p(k), n, _u64p(out["h1"]), _u64p(out["h2"]), _u64p(out["b1"]),
                           _u64p(out["b2"]), _u16p(out["tag"]), _u8p(out["bit1"]), _u8p(out["bit2"]))
    return out


class OracleError(RuntimeError):
    pass


class Table:
    """One O-ckpp table (the method, sequentially)."""

    def __init__(self, n_buckets: int, slots: int = 8, timers: bool = False, seed: int = 0, library=None):
        self.L = library or lib()
        self._h = self.L.oc_create(n_buckets, slots, 1 if timers else 0, seed)
        if not self._h:
            raise OracleError(f"bad geometry nb={n_buckets} slots={slots}")
        self.n_buckets, self.slots, self.timers, self.seed = n_buckets, slots, timers, seed

    def close(self):
        if self._h:
            self.L.oc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _rc(rc):
        if rc < 0:
            raise OracleError({EINVAL: "EINVAL", ESTALE: "ESTALE"}.get(rc, str(rc)))
        return rc

    def insert(self, keys, values, now: int = 0, ttl: int = 0) -> np.ndarray:
        k = _keys(keys)
        v = np.ascontiguousarray(values, dtype=np.uint64)
        st = np.zeros(k.shape[0], np.uint8)
        self._rc(self.L.oc_insert(self._h, _u8p(k), _u64p(v), k.shape[0], now, ttl, _u8p(st)))
        return st

    def lookup(self, keys, now: int = 0, refresh_ttl: int = 0):
        k = _keys(keys)
        vals = np.zeros(k.shape[0], np.uint64)
        found = np.zeros(k.shape[0], np.uint8)
        self._rc(self.L.oc_lookup(self._h, _u8p(k), k.shape[0], now, refresh_ttl, _u64p(vals), _u8p(found)))
        return vals, found

    def delete(self, keys, now: int = 0) -> np.ndarray:
        k = _keys(keys)
        st = np.zeros(k.shape[0], np.uint8)
        self._rc(self.L.oc_delete(self._h, _u8p(k), k.shape[0], now, _u8p(st)))
        return st

    def expire(self, now: int) -> int:
        return self._rc(int(self.L.oc_expire(self._h, now)))

    def size(self) -> int:
        return int(self.L.oc_size(self._h))

    def dump(self) -> dict:
        n = self.size()
        d = {"key": np.zeros((n, 16), np.uint8), "value": np.zeros(n, np.uint64), "expiry": np.zeros(n, np.uint16),
             "bucket": np.zeros(n, np.uint64), "slot": np.zeros(n, np.uint8), "in_secondary": np.zeros(n, np.uint8)}
        self.L.oc_dump(self._h, _u8p(d["key"]), _u64p(d["value"]), _u16p(d["expiry"]), _u64p(d["bucket"]),
                      _u8p(d["slot"]), _u8p(d["in_secondary"]))
        return d

    def meta(self):
        bloom = np.zeros(self.n_buckets, np.uint64)
        moved = np.zeros(self.n_buckets, np.uint32)
        self.L.oc_meta_dump(self._h, _u64p(bloom), _u32p(moved))
        return bloom, moved

    def probe_counts(self, keys, now: int = 0):
        """(secondary-bucket reads, key/value record reads) a lookup of keys makes."""
        k = _keys(keys)
        sec = np.zeros(1, np.uint64)
        rec = np.zeros(1, np.uint64)
        self.L.oc_lookup_probe_counts(self._h, _u8p(k), k.shape[0], now, _u64p(sec), _u64p(rec))
        return int(sec[0]), int(rec[0])

    def check(self, check_reset: bool = True) -> int:
        bad = np.zeros(1, np.uint64)
        return int(self.L.oc_check_invariants(self._h, 1 if check_reset else 0, _u64p(bad)))
