"""Host policy of the served form: the request stream and the turn planner.

Pure host code (numpy only), so that the admission and write-coalescing rules
can be checked without a GPU; ``serve.py`` runs the planned turns on the
device.

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
  the stream has ended, or waiting inserts hold the footprint budget that a
  newly arrived burst needs.
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
    insert_flush_s: float = 300e-6    # ... or the oldest has waited this long
    seed: int = 7


@dataclass
class Stream:
    """Pre-drawn request stream (arrival order)."""
    arrival: np.ndarray    # seconds since start
    table: np.ndarray      # target table
    size: np.ndarray       # keys in the burst
    insert: np.ndarray     # True: insert of new flows
    offset: np.ndarray     # lookups: offset in the table's lookup pool; inserts: offset in the insert pool


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
    return Stream(arrival, table, size, insert, offset)


@dataclass
class Turn:
    """What one turn launches."""
    admitted: slice                 # bursts admitted this turn (arrival order)
    lookups: np.ndarray             # lookup bursts to launch now
    inserts: list = field(default_factory=list)  # insert bursts to launch now, in arrival order
    insert_first: int = 0           # insert-pool offset of inserts[0]
    insert_keys: int = 0            # keys in inserts (a contiguous range of the insert pool)
    nbytes: int = 0                 # staging footprint the turn's bursts release when it completes

    @property
    def done(self) -> np.ndarray:
        """The bursts that complete with this turn."""
        return np.concatenate([self.lookups, np.asarray(self.inserts, np.int64)])


class TurnPlanner:
    """Admission and write coalescing over a pre-drawn stream (module doc).
    ``plan`` returns one of
      ("idle", None, wake)  nothing to do before host time ``wake``;
      ("block", None, 0)    the budget is full: wait for the oldest launch;
      ("none", None, 0)     bursts were admitted, nothing to launch yet;
      ("launch", turn, 0)   launch ``turn``.
    The caller reports each completed turn with ``complete(turn)``."""

    def __init__(self, stream: Stream, cfg: ServeConfig, max_jobs: int):
        self.st, self.cfg, self.max_jobs = stream, cfg, max_jobs
        self.n = stream.arrival.shape[0]
        self.foot = stream.size.astype(np.int64) * KEY_BYTES_IO
        self.nxt = 0               # first burst not yet admitted
        self.pending: list = []    # admitted insert bursts not yet launched
        self.pending_keys = 0
        self.flight_bytes = 0      # footprint admitted and not yet completed

    def finished(self) -> bool:
        """Every burst admitted and launched."""
        return self.nxt >= self.n and not self.pending

    def _flush_due(self, now: float) -> bool:
        st, cfg = self.st, self.cfg
        return bool(self.pending) and (self.pending_keys >= cfg.insert_flush_keys or self.nxt >= self.n or
                                       now - st.arrival[self.pending[0]] >= cfg.insert_flush_s)

    def plan(self, now: float, outstanding: bool):
        st, cfg = self.st, self.cfg
        arrived = self.nxt < self.n and st.arrival[self.nxt] <= now
        flush = self._flush_due(now)
        if not arrived and not flush:
            wake = st.arrival[self.nxt] if self.nxt < self.n else now
            if self.pending:
                wake = min(wake, st.arrival[self.pending[0]] + cfg.insert_flush_s)
            return "idle", None, float(wake)
        sel = slice(self.nxt, self.nxt)
        if arrived:
            hi = int(np.searchsorted(st.arrival, now, side="right"))
            hi = min(hi, self.nxt + self.max_jobs)
            room = cfg.footprint_bytes - self.flight_bytes
            fit = int(np.searchsorted(np.cumsum(self.foot[self.nxt:hi]), room, side="right"))
            if fit == 0:
                if self.pending:
                    flush = True  # waiting inserts hold the budget: send them
                elif outstanding:
                    return "block", None, 0.0
                else:
                    fit = 1  # a burst larger than the budget goes alone
            sel = slice(self.nxt, self.nxt + fit)
            self.flight_bytes += int(self.foot[sel].sum())
        idx = np.arange(sel.start, sel.stop)
        lookups = idx[~st.insert[sel]]
        for b in idx[st.insert[sel]]:
            self.pending.append(int(b))
            self.pending_keys += int(st.size[b])
        self.nxt = sel.stop
        flush = bool(self.pending) and (flush or self._flush_due(now))
        if not lookups.shape[0] and not flush:
            return "none", None, 0.0
        turn = Turn(admitted=sel, lookups=lookups)
        if flush:
            turn.inserts = self.pending
            turn.insert_first = int(st.offset[self.pending[0]])
            turn.insert_keys = self.pending_keys
            self.pending, self.pending_keys = [], 0
        turn.nbytes = int(self.foot[turn.done].sum())
        return "launch", turn, 0.0

    def complete(self, turn: Turn):
        self.flight_bytes -= turn.nbytes
