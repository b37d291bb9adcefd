"""Host policy of the served form: the request stream and the turn planner.

Host code only, so that the admission and write-coalescing rules can be
checked without a GPU: the stream is drawn with numpy and the planner is the
native one of include/ckpp_serve.h (compiled into libckpp.so, no CUDA call);
``serve.py`` runs the planned turns on the device.

Request stream: packet bursts arrive from many ports (Poisson arrivals,
uniform burst sizes); each burst targets one table and is either a lookup of
flows or an insert of new flows.

Turn planner, called whenever the loop is free to launch:

* admission: every burst that has arrived, in arrival order, while the staging
  footprint (keys in, results out) of the work admitted and not yet completed
  stays within a budget; a burst that does not fit waits, and a single burst
  larger than the whole budget is admitted alone once nothing else is
  outstanding;
* lookups: the admitted lookup bursts go out in the same turn (one batched
  lookup launch);
* write coalescing: admitted insert bursts wait and go out together (one
  multi-table insert call over a contiguous range of the insert pool) once
  ``insert_flush_keys`` keys wait, the oldest has waited ``insert_flush_s``,
  a lookup held behind them has waited ``lookup_hold_s``, the stream has
  ended, or waiting inserts hold the footprint budget that a newly arrived
  burst needs;
* per-table arrival order: on every table, lookups and inserts take effect in
  the order they arrived, so each lookup sees exactly the inserts of its table
  that arrived before it (what it would see if every burst ran alone, one
  after the other). A turn launches up to three steps on one stream, in this
  order: the lookups whose table has no waiting insert; the flush of the
  waiting inserts; the lookups that arrived while an insert of their table was
  waiting (held until that flush). An insert that arrives for a table with a
  held lookup ends the turn's admission and forces the flush, so that the held
  lookup cannot see it; it starts the next group of waiting inserts.
* overlap (the default): flushes run on a second stream, beside later turns'
  lookups; a lookup whose table has a flush in flight trails it on that
  stream (include/ckpp_serve.h).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

KEY_BYTES_IO = 16 + 8 + 1  # key in, value and flag out


@dataclass
class ServeConfig:
    n_tables: int = 256
    total_slots: int = 500_000_000
    warm_lf: float = 0.8
    ports: int = 64
    min_burst: int = 32
    max_burst: int = 4096
    offered_lookups_per_s: float = 2e9
    insert_fraction: float = 0.10
    neg_rate: float = 0.2
    duration_s: float = 0.2
    footprint_bytes: int = 256 << 20
    insert_flush_keys: int = 32768    # coalesced inserts go out once this many keys wait ...
    insert_flush_s: float = 100e-6    # ... or the oldest has waited this long
    lookup_hold_s: float = 100e-6     # ... or a lookup held behind them has waited this long
    raw_fraction: float = 0.2         # share of lookup keys naming flows inserted earlier in the run
    max_inflight: int = 1             # turns queued on the device at most (0: no limit)
    overlap: bool = True              # flushes on a second stream, beside later turns' lookups
    seed: int = 7


@dataclass
class Stream:
    """Pre-drawn request stream (arrival order)."""
    arrival: np.ndarray    # seconds since start
    table: np.ndarray      # target table
    size: np.ndarray       # keys in the burst
    insert: np.ndarray     # True: insert of new flows
    offset: np.ndarray     # lookups: offset in the table's lookup pool; inserts: offset in the insert pool
    # lookup keys that name flows inserted earlier in the run (read-after-write): key raw_pos of
    # table raw_table's lookup pool is key raw_src of the insert pool, whose insert burst arrived
    # before the lookup burst; sorted by table
    raw_table: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    raw_pos: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    raw_src: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))


def draw_stream(cfg: ServeConfig) -> Stream:
    rng = np.random.default_rng(cfg.seed)
    mean_burst = (cfg.min_burst + cfg.max_burst) / 2
    rate_per_port = cfg.offered_lookups_per_s / (cfg.ports * mean_burst)
    per_port = []
    for _ in range(cfg.ports):
        n = int(rate_per_port * cfg.duration_s * 1.2) + 16
        t = np.cumsum(rng.exponential(1.0 / rate_per_port, n))
        per_port.append(t[t < cfg.duration_s])
    arrival = np.sort(np.concatenate(per_port))
    nb = arrival.shape[0]
    table = rng.integers(0, cfg.n_tables, nb)
    size = rng.integers(cfg.min_burst, cfg.max_burst + 1, nb)
    insert = rng.random(nb) < cfg.insert_fraction
    offset = np.zeros(nb, np.int64)
    ins_sizes = np.where(insert, size, 0)
    offset[insert] = (np.cumsum(ins_sizes) - ins_sizes)[insert]
    look = ~insert
    for t in range(cfg.n_tables):
        sel = look & (table == t)
        s = size[sel]
        offset[sel] = np.cumsum(s) - s
    raw = draw_read_after_write(cfg, rng, table, size, insert, offset)
    return Stream(arrival, table, size, insert, offset, *raw)


def draw_read_after_write(cfg: ServeConfig, rng, table, size, insert, offset):
    """Each key of a lookup burst, with probability raw_fraction, names a flow
    that an insert burst of the same table inserted earlier in the run
    (uniform over all such flows so far); keys of a burst with no earlier
    insert on its table are left as drawn. Returns (raw_table, raw_pos,
    raw_src): the table, the position in that table's lookup pool and the
    insert-pool index of every such key."""
    out_t, out_p, out_s = [], [], []
    if cfg.raw_fraction <= 0:
        return (np.zeros(0, np.int64),) * 3
    for t in range(cfg.n_tables):
        bursts = np.flatnonzero(table == t)  # arrival order
        starts, lens = [], []                # insert-pool ranges of the table's inserts so far
        cum = np.zeros(1, np.int64)
        for b in bursts:
            if insert[b]:
                starts.append(int(offset[b]))
                lens.append(int(size[b]))
                cum = np.concatenate([cum, [cum[-1] + int(size[b])]])
                continue
            if not starts:
                continue
            m = int(rng.binomial(int(size[b]), cfg.raw_fraction))
            if m == 0:
                continue
            pos = offset[b] + rng.choice(int(size[b]), m, replace=False)
            u = rng.integers(0, int(cum[-1]), m)
            r = np.searchsorted(cum, u, side="right") - 1
            src = np.asarray(starts, np.int64)[r] + (u - cum[r])
            out_t.append(np.full(m, t, np.int64))
            out_p.append(pos.astype(np.int64))
            out_s.append(src.astype(np.int64))
    if not out_t:
        return (np.zeros(0, np.int64),) * 3
    return np.concatenate(out_t), np.concatenate(out_p), np.concatenate(out_s)


@dataclass
class Turn:
    """What one turn launches, in this order: ``lookups``, then the flush of
    ``inserts``, then ``lookups_after``. With overlap, ``lookups`` go to the
    first stream and the rest to the second, after ``trailing`` (lookups
    behind a flush in flight)."""
    admitted: slice                 # bursts admitted this turn (arrival order)
    lookups: np.ndarray             # lookup bursts whose table has no waiting insert (nor flush in flight)
    inserts: list = field(default_factory=list)  # insert bursts to launch now, in arrival order
    insert_first: int = 0           # insert-pool offset of inserts[0]
    insert_keys: int = 0            # keys in inserts (a contiguous range of the insert pool)
    lookups_after: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))  # held behind inserts
    nbytes: int = 0                 # staging footprint the turn's bursts release when it completes
    trailing: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))  # overlap: behind a flush in flight
    nbytes_b: int = 0               # overlap: footprint of the second-stream part

    @property
    def done(self) -> np.ndarray:
        """The bursts that complete with this turn."""
        return np.concatenate([self.lookups, self.trailing, np.asarray(self.inserts, np.int64), self.lookups_after])

    @property
    def part_b(self) -> np.ndarray:
        """Overlap: the bursts of the second-stream part."""
        return np.concatenate([self.trailing, np.asarray(self.inserts, np.int64), self.lookups_after])


class TurnPlanner:
    """The served form's turn planner over a pre-drawn stream: the native
    planner of include/ckpp_serve.h (host code, no GPU needed), whose rules the
    module doc states. ``plan`` returns one of
      ("idle", None, wake)  nothing to do before host time ``wake``;
      ("block", None, 0)    the budget is full: wait for the oldest launch;
      ("none", None, 0)     bursts were admitted, nothing to launch yet;
      ("launch", turn, 0)   launch ``turn``.
    The caller reports each completed turn with ``complete(turn)``."""

    def __init__(self, stream: Stream, cfg: ServeConfig, max_jobs: int):
        import ctypes as C

        from . import _ckpp as K
        self.K, self.C, self.lib = K, C, K.library()
        self.st, self.cfg, self.max_jobs = stream, cfg, max_jobs
        self.n = n = stream.arrival.shape[0]
        # the planner borrows these arrays: they live as long as it does
        self._arrays = (np.ascontiguousarray(stream.arrival, np.float64),
                        np.ascontiguousarray(stream.table, np.uint32),
                        np.ascontiguousarray(stream.size, np.uint32),
                        np.ascontiguousarray(stream.insert, np.uint8),
                        np.ascontiguousarray(stream.offset, np.int64))
        conf = K.ckpp_plan_config(cfg.insert_flush_s, cfg.lookup_hold_s, cfg.insert_flush_keys,
                                  cfg.footprint_bytes, KEY_BYTES_IO, max_jobs, 1 if cfg.overlap else 0)
        self._h = C.c_void_p()
        K._check(self.lib.ckpp_plan_create(*(a.ctypes.data for a in self._arrays), n, C.byref(conf),
                                           C.byref(self._h)), "ckpp_plan_create")
        self._out = np.empty((4, max(n, 1)), np.int64)
        self._ptrs = tuple(int(self._out[i].ctypes.data) for i in range(4))
        self._turn = K.ckpp_turn()
        self._turn_ref = C.byref(self._turn)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self.lib.ckpp_plan_destroy(h)
            self._h = None

    def _state(self):
        C = self.C
        pk, fb, fin = C.c_int64(), C.c_int64(), C.c_int()
        self.K._check(self.lib.ckpp_plan_state(self._h, C.byref(pk), C.byref(fb), C.byref(fin)), "ckpp_plan_state")
        return pk.value, fb.value, bool(fin.value)

    @property
    def pending_keys(self) -> int:
        """Insert keys admitted and waiting for a flush."""
        return self._state()[0]

    @property
    def flight_bytes(self) -> int:
        """Footprint admitted and not yet completed."""
        return self._state()[1]

    def finished(self) -> bool:
        """Every burst admitted and launched."""
        return self._state()[2]

    def plan(self, now: float, outstanding: bool):
        K, t = self.K, self._turn
        rc = self.lib.ckpp_plan_next(self._h, now, 1 if outstanding else 0, self._turn_ref, *self._ptrs,
                                     self._out.shape[1])
        if rc != K.CKPP_OK:
            K._check(rc, "ckpp_plan_next")
        a = t.action
        if a == K.PLAN_IDLE:
            return "idle", None, t.wake
        if a == K.PLAN_BLOCK:
            return "block", None, 0.0
        if a == K.PLAN_NONE:
            return "none", None, 0.0
        out = self._out
        turn = Turn(admitted=slice(t.admitted_lo, t.admitted_hi), lookups=out[0, :t.n_lookups].copy(),
                    trailing=out[1, :t.n_trailing].copy(), inserts=out[2, :t.n_inserts].tolist(),
                    insert_first=t.insert_first, insert_keys=t.insert_keys,
                    lookups_after=out[3, :t.n_after].copy(), nbytes=t.nbytes, nbytes_b=t.nbytes_b)
        return "launch", turn, 0.0

    def complete(self, turn: Turn):
        """The turn (with overlap: its first-stream part) completed."""
        self.K._check(self.lib.ckpp_plan_complete(self._h, turn.nbytes), "ckpp_plan_complete")

    def complete_b(self, turn: Turn):
        """Overlap: the turn's second-stream part completed."""
        self.K._check(self.lib.ckpp_plan_complete_b(self._h, turn.nbytes_b, 1 if turn.inserts else 0),
                      "ckpp_plan_complete_b")
