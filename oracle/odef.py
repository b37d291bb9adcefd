"""O-def: the plain definition of a flow table with expiring entries.

Test infrastructure only. A Cuckoo++ table answers exactly like a map from key
to (value, expiry): the filter of Sec. 4.1 only prunes reads and never hides a
stored key, and the timers of Sec. 4.2 make an entry count only while
``(uint16)(expiry - now) < 1024``. This module is that map, written out with a
Python dict, so every lookup result and every insert/delete status of the
method can be checked against it exactly.

Sequential semantics within a batch: keys are applied in index order.
"""

from __future__ import annotations

import numpy as np

INSERTED, UPDATED, DELETED, NOT_FOUND = 1, 2, 4, 5
ALIVE_WINDOW = 1024


def alive(expiry: int, now: int) -> bool:
    """Sec. 4.2: alive iff the unsigned 16-bit difference is below 1024."""
    return ((expiry - now) & 0xFFFF) < ALIVE_WINDOW


class MapTable:
    def __init__(self, timers: bool = False):
        self.timers = timers
        self.d: dict[bytes, list] = {}

    def _alive(self, rec, now):
        return (not self.timers) or alive(rec[1], now)

    def insert(self, keys, values, now=0, ttl=0):
        keys = np.asarray(keys, np.uint8).reshape(-1, 16)
        st = np.zeros(len(keys), np.uint8)
        for i, k in enumerate(keys):
            kb = k.tobytes()
            rec = self.d.get(kb)
            st[i] = UPDATED if (rec is not None and self._alive(rec, now)) else INSERTED
            self.d[kb] = [int(values[i]), (now + ttl) & 0xFFFF if self.timers else 0]
        return st

    def lookup(self, keys, now=0, refresh_ttl=0):
        keys = np.asarray(keys, np.uint8).reshape(-1, 16)
        vals = np.zeros(len(keys), np.uint64)
        found = np.zeros(len(keys), np.uint8)
        for i, k in enumerate(keys):
            rec = self.d.get(k.tobytes())
            if rec is not None and self._alive(rec, now):
                vals[i] = rec[0]
                found[i] = 1
                if self.timers and refresh_ttl:
                    rec[1] = (now + refresh_ttl) & 0xFFFF
        return vals, found

    def delete(self, keys, now=0):
        keys = np.asarray(keys, np.uint8).reshape(-1, 16)
        st = np.zeros(len(keys), np.uint8)
        for i, k in enumerate(keys):
            kb = k.tobytes()
            rec = self.d.pop(kb, None)
            st[i] = DELETED if (rec is not None and self._alive(rec, now)) else NOT_FOUND
        return st

    def expire(self, now):
        dead = [k for k, rec in self.d.items() if not self._alive(rec, now)]
        for k in dead:
            del self.d[k]
        return len(dead)

    def live(self, now=0) -> dict[bytes, tuple[int, int]]:
        """Key -> (value, expiry) of every live entry."""
        return {k: (rec[0], rec[1]) for k, rec in self.d.items() if self._alive(rec, now)}
