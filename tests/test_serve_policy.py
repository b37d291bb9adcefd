"""The served form's host policy (admission within the footprint budget, write
coalescing, per-table arrival order) on CPU: the native turn planner
(include/ckpp_serve.h, host code) is driven by a simulated clock and a
simulated in-order device, every turn it plans is checked, and it plans the
same turns as the rules written out in plain Python."""

from collections import deque
from dataclasses import replace

import numpy as np
import pytest

from paper_1712_09624_gb300.serve_policy import KEY_BYTES_IO, ServeConfig, Turn, TurnPlanner, draw_stream

@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_1712_09624_gb300 import build
    build.build()  # the planner is host code in libckpp.so


SMALL = ServeConfig(n_tables=8, ports=8, min_burst=32, max_burst=1024, offered_lookups_per_s=50e6,
                    insert_fraction=0.2, duration_s=0.02, footprint_bytes=4 << 20, insert_flush_keys=8192,
                    insert_flush_s=200e-6, seed=3, overlap=False)  # one stream; overlap mode is tested below


def simulate(cfg, host_s=10e-6, dev_fixed_s=5e-6, dev_per_key_s=0.2e-9, max_jobs=4096, planner=TurnPlanner):
    """Runs the planner to the end. The host spends host_s per launched turn;
    the device runs turns in launch order, each taking dev_fixed_s plus
    dev_per_key_s per key. Returns the stream, the launched turns as (launch
    time, turn, insert keys waiting before the planning call, footprint
    outstanding after it) and the largest footprint ever outstanding."""
    st = draw_stream(cfg)
    pl = planner(st, cfg, max_jobs)
    now, dev_free = 0.0, 0.0
    outstanding = deque()  # (finish time, turn)
    launched, max_flight = [], 0
    for _ in range(10_000_000):
        if pl.finished() and not outstanding:
            break
        while outstanding and outstanding[0][0] <= now:
            pl.complete(outstanding.popleft()[1])
        pend_keys = pl.pending_keys
        action, turn, wake = pl.plan(now, bool(outstanding))
        max_flight = max(max_flight, pl.flight_bytes)
        if action == "idle":
            times = [w for w in (wake,) if w > now] + ([outstanding[0][0]] if outstanding else [])
            now = min(times) if times else now + 1e-6
            continue
        if action == "block":
            now = max(now, outstanding[0][0])
            continue
        if action == "none":
            continue
        keys = int(st.size[turn.done].sum())
        dev_free = max(now, dev_free) + dev_fixed_s + dev_per_key_s * keys
        outstanding.append((dev_free, turn))
        launched.append((now, turn, pend_keys, pl.flight_bytes))
        now += host_s
    else:
        raise AssertionError("planner did not finish")
    return st, launched, max_flight


def execution_order(launched):
    """Bursts in the order the device applies them: turn by turn, the turn's
    lookups, then its inserts, then the lookups held behind them."""
    order = []
    for _, turn, _, _ in launched:
        order.extend(int(b) for b in turn.lookups)
        order.extend(int(b) for b in turn.inserts)
        order.extend(int(b) for b in turn.lookups_after)
    return order


def check_table_order(st, launched):
    """Per table, every lookup sees exactly the inserts of its table that
    arrived before it: the inserts applied before it equal those that arrived
    before it (read-after-write and write-after-read across turns)."""
    applied = {}
    for b in execution_order(launched):
        t = int(st.table[b])
        if st.insert[b]:
            applied.setdefault(t, set()).add(b)
        else:
            arrived_before = {i for i in np.flatnonzero(st.insert & (st.table == t)) if i < b}
            assert applied.get(t, set()) == arrived_before, f"lookup {b} of table {t} sees the wrong inserts"


def check_common(st, launched):
    n = st.arrival.shape[0]
    seen = np.zeros(n, np.int64)
    last_insert_end = 0
    ins_order = []
    for t, turn, _, _ in launched:
        done = turn.done
        seen[done] += 1
        assert (st.arrival[done] <= t + 1e-12).all(), "a burst launched before it arrived"
        for look in (turn.lookups, turn.lookups_after):
            assert not st.insert[look].any() and (np.diff(look) > 0).all()
        if turn.lookups_after.shape[0]:
            assert turn.inserts, "lookups held behind inserts go out only with their flush"
        if turn.inserts:
            ins = np.asarray(turn.inserts)
            assert st.insert[ins].all() and (np.diff(ins) > 0).all()
            ins_order.extend(turn.inserts)
            # one contiguous range of the insert pool, following the previous flush
            assert turn.insert_first == st.offset[ins[0]] == last_insert_end
            assert turn.insert_keys == int(st.size[ins].sum())
            assert (st.offset[ins[1:]] == st.offset[ins[:-1]] + st.size[ins[:-1]]).all()
            last_insert_end = turn.insert_first + turn.insert_keys
        assert turn.nbytes == int(st.size[done].sum()) * KEY_BYTES_IO
    assert (seen == 1).all(), "every burst is launched exactly once"
    assert ins_order == list(np.flatnonzero(st.insert)), "inserts flushed in arrival order"
    check_table_order(st, launched)


def flush_reasons(st, cfg, launched, host_s=10e-6):
    """For every flush, which of the planner's triggers held at its launch:
    keys (enough keys wait), age (the oldest insert waited long enough), hold
    (a held lookup waited long enough), end (the stream ended), conflict (the
    next burst is an insert on a table with a held lookup)."""
    out = []
    end = st.arrival[-1]
    for t, turn, _, _ in launched:
        if not turn.inserts:
            continue
        r = set()
        if turn.insert_keys >= cfg.insert_flush_keys:
            r.add("keys")
        if t - st.arrival[turn.inserts[0]] >= cfg.insert_flush_s - 1e-12:
            r.add("age")
        if turn.lookups_after.shape[0] and t - st.arrival[turn.lookups_after[0]] >= cfg.lookup_hold_s - 1e-12:
            r.add("hold")
        if t >= end:
            r.add("end")
        nxt = turn.admitted.stop
        held_tables = set(st.table[turn.lookups_after].tolist())
        if nxt < st.arrival.shape[0] and st.insert[nxt] and int(st.table[nxt]) in held_tables:
            r.add("conflict")
        out.append((t, turn, r))
    return out


def test_every_burst_once_in_order_with_contiguous_flushes():
    st, launched, max_flight = simulate(SMALL)
    check_common(st, launched)
    assert max_flight <= SMALL.footprint_bytes
    flushes = [x for x in launched if x[1].inserts]
    assert len(flushes) > 5 and len(launched) > 50


def test_flush_triggers():
    """Each flush happens because enough keys wait, the oldest insert or held
    lookup waited long enough, the stream ended, or an insert arrived for a
    table with a held lookup; none is early, and none waits much beyond the
    age limits while the device keeps up."""
    cfg = SMALL
    st, launched, _ = simulate(cfg)
    host_s = 10e-6
    reasons = flush_reasons(st, cfg, launched)
    assert reasons
    for t, turn, r in reasons:
        assert r, (t, turn.insert_keys)
        assert t - st.arrival[turn.inserts[0]] <= cfg.insert_flush_s + 2 * host_s + 1e-9
        if turn.lookups_after.shape[0]:
            assert t - st.arrival[turn.lookups_after[0]] <= cfg.lookup_hold_s + 2 * host_s + 1e-9
    # without the age limits, every flush but the last carries the key threshold or is forced by a
    # conflict, and no planning call starts with the threshold already reached (no late flush)
    cfg = replace(cfg, insert_flush_s=10.0, lookup_hold_s=10.0)
    st, launched, _ = simulate(cfg)
    reasons = flush_reasons(st, cfg, launched)
    assert all(r & {"keys", "conflict"} for _, _, r in reasons[:-1])
    assert any("conflict" in r for _, _, r in reasons)
    assert all(pend_before < cfg.insert_flush_keys for _, _, pend_before, _ in launched)
    check_common(st, launched)
    # with many tables conflicts are rare and the key threshold sends most flushes
    cfg = replace(cfg, n_tables=1024)
    st, launched, _ = simulate(cfg)
    reasons = flush_reasons(st, cfg, launched)
    assert all(r & {"keys", "conflict"} for _, _, r in reasons[:-1])
    assert sum("keys" in r for _, _, r in reasons) > len(reasons) // 2
    check_common(st, launched)


def test_table_order_under_heavy_conflict():
    """Two tables, half the bursts inserts: held lookups and forced flushes on
    almost every turn; every lookup still sees exactly the earlier inserts of
    its table."""
    cfg = replace(SMALL, n_tables=2, insert_fraction=0.5, insert_flush_keys=1 << 20, insert_flush_s=1e-3,
                  lookup_hold_s=5e-4)
    st, launched, _ = simulate(cfg)
    check_common(st, launched)
    assert sum(1 for x in launched if x[1].lookups_after.shape[0]) > 5


def test_read_after_write_keys_name_earlier_inserts():
    """The stream's read-after-write lookup keys name flows of the same table
    whose insert burst arrived before the lookup burst, and make up about
    raw_fraction of the lookup keys that have such flows to name."""
    st = draw_stream(SMALL)
    assert st.raw_pos.shape[0] > 1000
    ins = np.flatnonzero(st.insert)
    ins_end = st.offset[ins] + st.size[ins]
    for t, pos, src in zip(st.raw_table[:2000], st.raw_pos[:2000], st.raw_src[:2000]):
        look = np.flatnonzero(~st.insert & (st.table == t))
        b = look[np.searchsorted(st.offset[look], pos, side="right") - 1]
        assert st.offset[b] <= pos < st.offset[b] + st.size[b]
        i = ins[np.searchsorted(st.offset[ins], src, side="right") - 1]
        assert st.offset[i] <= src < ins_end[ins == i][0]
        assert st.table[i] == t and i < b
    assert (np.diff(st.raw_table) >= 0).all(), "sorted by table"
    # positions are distinct within a table
    for t in range(SMALL.n_tables):
        p = st.raw_pos[st.raw_table == t]
        assert np.unique(p).shape[0] == p.shape[0]
    eligible = 0
    for t in range(SMALL.n_tables):
        first_ins = np.flatnonzero(st.insert & (st.table == t))
        if first_ins.shape[0]:
            eligible += int(st.size[~st.insert & (st.table == t) & (np.arange(st.size.shape[0]) > first_ins[0])].sum())
    assert abs(st.raw_pos.shape[0] / eligible - SMALL.raw_fraction) < 0.01


@pytest.mark.parametrize("insert_fraction", [0.0, 1.0])
def test_all_lookups_or_all_inserts(insert_fraction):
    cfg = replace(SMALL, insert_fraction=insert_fraction)
    st, launched, _ = simulate(cfg)
    check_common(st, launched)
    n_flush = sum(1 for x in launched if x[1].inserts)
    if insert_fraction == 0.0:
        assert n_flush == 0
    else:
        assert all(x[1].lookups.shape[0] == 0 and x[1].lookups_after.shape[0] == 0 for x in launched)
        assert n_flush >= 1


def test_budget_smaller_than_one_burst_still_serves_everything():
    """A budget below one burst's footprint admits one burst at a time, each
    once nothing else is outstanding, and waiting inserts are flushed to free
    it."""
    cfg = replace(SMALL, footprint_bytes=100, duration_s=0.005)
    st, launched, _ = simulate(cfg)
    check_common(st, launched)
    for _, turn, _, _ in launched:
        assert turn.admitted.stop - turn.admitted.start <= 1


def test_saturated_device_blocks_on_the_budget():
    """When the device is slower than the arrivals, admission stops at the
    budget (apart from inserts flushed to free it) and waits for completions."""
    cfg = replace(SMALL, footprint_bytes=1 << 20)
    st, launched, max_flight = simulate(cfg, dev_per_key_s=50e-9)  # 20M keys/s against 50M offered
    check_common(st, launched)
    assert max_flight <= cfg.footprint_bytes
    # the device, not the arrivals, sets the pace: the last launch comes well after the last arrival
    assert launched[-1][0] > st.arrival[-1] + 10e-3


def test_order_check_catches_lookups_run_before_their_inserts():
    """Planted mistake: launching the held lookups with the turn's first
    lookups (before the flush, as a planner without holding would) breaks
    read-after-write, and the order check says so."""
    from dataclasses import replace as dc_replace
    cfg = replace(SMALL, n_tables=2, insert_fraction=0.5)
    st, launched, _ = simulate(cfg)
    check_table_order(st, launched)
    moved = [(t, dc_replace(turn, lookups=np.sort(np.concatenate([turn.lookups, turn.lookups_after])),
                            lookups_after=np.zeros(0, np.int64)), a, b) for t, turn, a, b in launched]
    with pytest.raises(AssertionError):
        check_table_order(st, moved)


class RefPlanner:
    """The planner's rules written in plain Python, one burst at a time, as
    the served form's host policy states them: the native planner must plan
    the same turns."""

    def __init__(self, stream, cfg, max_jobs):
        self.st, self.cfg, self.max_jobs = stream, cfg, max_jobs
        self.n = stream.arrival.shape[0]
        self.foot = stream.size.astype(np.int64) * KEY_BYTES_IO
        self.nxt = 0
        self.pending, self.pending_keys, self.pending_tables = [], 0, set()
        self.held, self.held_tables = [], set()
        self.flight_bytes = 0
        self.flight_cnt, self.flushes = {}, []  # overlap: flushes in flight per table, their tables in order

    def finished(self):
        return self.nxt >= self.n and not self.pending and not self.held

    def _flush_due(self, now):
        st, cfg = self.st, self.cfg
        return bool(self.pending) and (self.pending_keys >= cfg.insert_flush_keys or self.nxt >= self.n or
                                       now - st.arrival[self.pending[0]] >= cfg.insert_flush_s or
                                       (bool(self.held) and now - st.arrival[self.held[0]] >= cfg.lookup_hold_s))

    def _wake(self, now):
        st, cfg = self.st, self.cfg
        wake = st.arrival[self.nxt] if self.nxt < self.n else now
        if self.pending:
            wake = min(wake, st.arrival[self.pending[0]] + cfg.insert_flush_s)
        if self.held:
            wake = min(wake, st.arrival[self.held[0]] + cfg.lookup_hold_s)
        return float(wake)

    def plan(self, now, outstanding):
        st, cfg = self.st, self.cfg
        arrived = self.nxt < self.n and st.arrival[self.nxt] <= now
        flush = self._flush_due(now)
        if not arrived and not flush:
            return "idle", None, self._wake(now)
        lo = stop = self.nxt
        lookups, trailing = [], []
        if arrived:
            hi = lo
            while hi < self.n and st.arrival[hi] <= now:
                hi += 1
            room = cfg.footprint_bytes - self.flight_bytes
            fit, acc = 0, 0
            while lo + fit < hi and acc + self.foot[lo + fit] <= room:
                acc += self.foot[lo + fit]
                fit += 1
            if fit == 0:
                if self.pending:
                    flush = True
                elif outstanding:
                    return "block", None, 0.0
                else:
                    fit = 1
            for b in range(lo, lo + fit):
                t = int(st.table[b])
                if st.insert[b]:
                    if t in self.held_tables:
                        flush = True
                        break
                    self.pending.append(b)
                    self.pending_keys += int(st.size[b])
                    self.pending_tables.add(t)
                else:
                    if len(lookups) + len(trailing) + len(self.held) >= self.max_jobs:
                        flush = True
                        break
                    if t in self.pending_tables:
                        self.held.append(b)
                        self.held_tables.add(t)
                    elif self.flight_cnt.get(t, 0):
                        trailing.append(b)
                    else:
                        lookups.append(b)
                stop = b + 1
            self.flight_bytes += int(self.foot[lo:stop].sum())
            self.nxt = stop
        flush = bool(self.pending) and (flush or self._flush_due(now))
        if not lookups and not trailing and not flush:
            return "none", None, 0.0
        turn = Turn(admitted=slice(lo, stop), lookups=np.asarray(lookups, np.int64),
                    trailing=np.asarray(trailing, np.int64))
        if flush:
            turn.inserts, turn.insert_first = self.pending, int(st.offset[self.pending[0]])
            turn.insert_keys, turn.lookups_after = self.pending_keys, np.asarray(self.held, np.int64)
            if cfg.overlap:
                tables = list(dict.fromkeys(int(st.table[b]) for b in self.pending))
                for t in tables:
                    self.flight_cnt[t] = self.flight_cnt.get(t, 0) + 1
                self.flushes.append(tables)
            self.pending, self.pending_keys, self.pending_tables = [], 0, set()
            self.held, self.held_tables = [], set()
        if cfg.overlap:
            turn.nbytes = int(self.foot[turn.lookups].sum())
            turn.nbytes_b = int(self.foot[turn.part_b].sum())
        else:
            turn.nbytes = int(self.foot[turn.done].sum())
        return "launch", turn, 0.0

    def complete(self, turn):
        self.flight_bytes -= turn.nbytes

    def complete_b(self, turn):
        self.flight_bytes -= turn.nbytes_b
        if turn.inserts:
            for t in self.flushes.pop(0):
                self.flight_cnt[t] -= 1


@pytest.mark.parametrize("variant", ["small", "two_tables", "few_jobs", "tiny_budget", "many_tables"])
def test_native_planner_equals_plain_rules(variant):
    cfg = {"small": SMALL,
           "two_tables": replace(SMALL, n_tables=2, insert_fraction=0.5, lookup_hold_s=5e-4),
           "few_jobs": SMALL,
           "tiny_budget": replace(SMALL, footprint_bytes=60_000, duration_s=0.005),
           "many_tables": replace(SMALL, n_tables=1024)}[variant]
    max_jobs = 3 if variant == "few_jobs" else 4096
    runs = [simulate(cfg, max_jobs=max_jobs, planner=cls) for cls in (TurnPlanner, RefPlanner)]
    (st, a, _), (_, b, _) = runs
    assert len(a) == len(b)
    for (ta, x, pa, fa), (tb, y, pb, fb) in zip(a, b):
        assert ta == tb and pa == pb and fa == fb
        assert x.admitted == y.admitted and x.inserts == y.inserts
        assert np.array_equal(x.lookups, y.lookups) and np.array_equal(x.lookups_after, y.lookups_after)
        assert x.insert_first == y.insert_first and x.insert_keys == y.insert_keys and x.nbytes == y.nbytes
    check_common(st, a)


def test_native_planner_argument_errors():
    """Unsorted arrivals and a table index out of range are refused at
    creation; an output room too small for the turn is refused without
    changing the planner's state."""
    import ctypes as C

    from paper_1712_09624_gb300 import _ckpp as K
    lib = K.library()
    conf = K.ckpp_plan_config(1e-3, 1e-3, 100, 1 << 20, KEY_BYTES_IO, 16)
    arrival = np.array([0.0, 2e-6, 1e-6])
    table = np.array([0, 1, 2], np.uint32)
    size = np.array([10, 10, 10], np.uint32)
    insert = np.array([0, 1, 0], np.uint8)
    offset = np.zeros(3, np.int64)
    h = C.c_void_p()
    args = lambda arr, tb: (arr.ctypes.data, tb.ctypes.data, size.ctypes.data, insert.ctypes.data,
                            offset.ctypes.data, 3, C.byref(conf), C.byref(h))
    assert lib.ckpp_plan_create(*args(arrival, table)) == K.CKPP_EINVAL
    arrival = np.sort(arrival)
    assert lib.ckpp_plan_create(*args(arrival, np.array([0, 1 << 20, 2], np.uint32))) == K.CKPP_EINVAL
    assert lib.ckpp_plan_create(*args(arrival, table)) == K.CKPP_OK
    try:
        out = np.zeros((4, 3), np.int64)
        turn = K.ckpp_turn()
        ptrs = [out[i].ctypes.data for i in range(4)]
        assert lib.ckpp_plan_next(h, 1.0, 0, C.byref(turn), *ptrs, 2) == K.CKPP_EINVAL  # three bursts arrived
        assert lib.ckpp_plan_next(h, 1.0, 0, C.byref(turn), *ptrs, 3) == K.CKPP_OK
        assert turn.action == K.PLAN_LAUNCH and (turn.admitted_lo, turn.admitted_hi) == (0, 3)
        assert turn.n_lookups == 2 and turn.n_inserts == 1 and turn.insert_keys == 10  # the stream ended
        assert lib.ckpp_plan_complete(h, turn.nbytes + 1) == K.CKPP_EINVAL
        assert lib.ckpp_plan_complete(h, turn.nbytes) == K.CKPP_OK
        fin = C.c_int()
        assert lib.ckpp_plan_state(h, None, None, C.byref(fin)) == K.CKPP_OK and fin.value == 1
    finally:
        lib.ckpp_plan_destroy(h)


def test_stage_jobs_writes_one_job_record_per_burst():
    """ckpp_serve_stage_jobs (host code) turns burst indices into the batched
    lookup's job records: each job's key, value and flag pointers are its
    table's pool addresses advanced to the burst's offset, with its size and
    table."""
    from paper_1712_09624_gb300 import _ckpp as K
    lib = K.library()
    rng = np.random.default_rng(5)
    n_b, n_t = 500, 7
    table = rng.integers(0, n_t, n_b).astype(np.uint32)
    offset = rng.integers(0, 1 << 30, n_b).astype(np.int64)
    size = rng.integers(0, 5000, n_b).astype(np.uint32)
    pools = [rng.integers(1 << 40, 1 << 41, n_t).astype(np.uint64) * np.uint64(256) for _ in range(3)]
    bursts = np.sort(rng.choice(n_b, 200, replace=False)).astype(np.int64)
    jobs = np.zeros(bursts.shape[0], np.dtype([("keys", "<u8"), ("out_vals", "<u8"), ("out_found", "<u8"),
                                                ("n", "<u4"), ("table", "<u4")]))
    assert jobs.itemsize == K.JOB_BYTES
    args = [a.ctypes.data for a in (table, offset, size, *pools)]
    assert lib.ckpp_serve_stage_jobs(bursts.ctypes.data, bursts.shape[0], *args, jobs.ctypes.data) == K.CKPP_OK
    t = table[bursts]
    off = offset[bursts].astype(np.uint64)
    assert (jobs["keys"] == pools[0][t] + np.uint64(16) * off).all()
    assert (jobs["out_vals"] == pools[1][t] + np.uint64(8) * off).all()
    assert (jobs["out_found"] == pools[2][t] + off).all()
    assert (jobs["n"] == size[bursts]).all() and (jobs["table"] == t).all()
    assert lib.ckpp_serve_stage_jobs(None, 0, *args, None) == K.CKPP_OK  # nothing to stage
    assert lib.ckpp_serve_stage_jobs(bursts.ctypes.data, -1, *args, jobs.ctypes.data) == K.CKPP_EINVAL
    assert lib.ckpp_serve_stage_jobs(bursts.ctypes.data, 1, *args[:-1], None, jobs.ctypes.data) == K.CKPP_EINVAL


def test_serving_loops_refuse_bad_arguments_without_a_gpu():
    """The native serving loops check their arguments before any CUDA call:
    missing pointers and a buffer set whose tables do not cover the stream
    are refused with CKPP_EINVAL."""
    import ctypes as C

    from paper_1712_09624_gb300 import _ckpp as K
    lib = K.library()
    stats = K.ckpp_serve_stats()
    assert lib.ckpp_serve_run(None, None, None, None, None, None, C.byref(stats)) == K.CKPP_EINVAL
    assert lib.ckpp_serve_run_plain(None, None, None, None, None, C.byref(stats)) == K.CKPP_EINVAL
    st = draw_stream(replace(SMALL, duration_s=0.002))
    pl = TurnPlanner(st, SMALL, 64)
    pools = np.zeros(SMALL.n_tables, np.uint64)
    done = np.zeros(st.arrival.shape[0])
    # fewer tables than the stream names, and no job buffers
    buf = K.ckpp_serve_buffers(pools.ctypes.data, pools.ctypes.data, pools.ctypes.data, 1, 64)
    handles = (C.c_void_p * SMALL.n_tables)(*([1] * SMALL.n_tables))
    assert lib.ckpp_serve_run_plain(pl._h, handles, C.byref(buf), None, done.ctypes.data,
                                    C.byref(stats)) == K.CKPP_EINVAL
    assert lib.ckpp_serve_run(pl._h, C.c_void_p(1), C.byref(buf), None, None, done.ctypes.data,
                              C.byref(stats)) == K.CKPP_EINVAL


# ---------------------------------------------------------------- overlap mode

def simulate_overlap(cfg, host_s=10e-6, dev_fixed_s=5e-6, dev_per_key_s=0.2e-9, max_jobs=4096,
                     planner=TurnPlanner):
    """Runs the planner in overlap mode against a simulated device with two
    in-order streams: a turn's first-stream part (its free lookups) runs in
    order on stream A; its second-stream part (trailing lookups, flush, held
    lookups) on stream B, after A's part of the same turn. Completions are
    reported when the clock passes them, before the next planning call.
    Returns the stream and the turns as (launch time, turn, A end, B end or
    None)."""
    st = draw_stream(cfg)
    pl = planner(st, cfg, max_jobs)
    now, a_free, b_free = 0.0, 0.0, 0.0
    out_a, out_b, launched = deque(), deque(), []
    for _ in range(10_000_000):
        if pl.finished() and not out_a and not out_b:
            break
        while out_a and out_a[0][0] <= now:
            pl.complete(out_a.popleft()[1])
        while out_b and out_b[0][0] <= now:
            pl.complete_b(out_b.popleft()[1])
        action, turn, wake = pl.plan(now, bool(out_a or out_b))
        if action == "idle":
            times = [w for w in (wake,) if w > now] + [q[0][0] for q in (out_a, out_b) if q]
            now = min(times) if times else now + 1e-6
            continue
        if action == "block":
            now = max(now, min(q[0][0] for q in (out_a, out_b) if q))
            continue
        if action == "none":
            continue
        keys_a = int(st.size[turn.lookups].sum())
        a_end = max(now, a_free) + (dev_fixed_s + dev_per_key_s * keys_a if keys_a else 0.0)
        a_free = a_end
        out_a.append((a_end, turn))
        b_end = None
        if turn.part_b.shape[0]:
            b_end = max(now, b_free, a_end) + dev_fixed_s + dev_per_key_s * int(st.size[turn.part_b].sum())
            b_free = b_end
            out_b.append((b_end, turn))
        launched.append((now, turn, a_end, b_end))
        now += host_s
    else:
        raise AssertionError("planner did not finish")
    return st, launched


def check_overlap_order(st, launched):
    """Every burst is launched once; per table, each lookup and each insert
    are ordered as they arrived, by the device's dependencies alone: the same
    stream's order, a second-stream part waiting for its turn's first-stream
    part (and so for every earlier one), and a second-stream part reported
    complete before a later turn was planned."""
    n = st.arrival.shape[0]
    seen = np.zeros(n, np.int64)
    where = {}  # burst -> (stream, turn index, phase)
    launch_t, b_end = [], []
    for k, (t, turn, a_end, be) in enumerate(launched):
        launch_t.append(t)
        b_end.append(be)
        for b in turn.lookups:
            where[int(b)] = ("A", k, 0)
        for ph, arr in ((0, turn.trailing), (1, np.asarray(turn.inserts, np.int64)), (2, turn.lookups_after)):
            for b in arr:
                where[int(b)] = ("B", k, ph)
        seen[turn.done] += 1
    assert (seen == 1).all(), "every burst is launched exactly once"

    def before(x, y):  # x happens before y
        (sx, kx, px), (sy, ky, py) = where[x], where[y]
        if sx == sy:
            return (kx, px) < (ky, py)
        if sx == "A":  # y on B waits for its turn's first-stream part, which follows x's
            return kx <= ky
        return b_end[kx] is not None and b_end[kx] <= launch_t[ky]  # reported complete before y's turn
    for t in np.unique(st.table):
        idx = np.flatnonzero(st.table == t)
        ins = [int(b) for b in idx if st.insert[b]]
        for lk in (int(b) for b in idx if not st.insert[b]):
            for i in ins:
                if i < lk:
                    assert before(i, lk), f"lookup {lk} of table {t} runs before the earlier insert {i}"
                else:
                    assert before(lk, i), f"insert {i} of table {t} is applied before the earlier lookup {lk}"


OVERLAP = replace(SMALL, overlap=True)


@pytest.mark.parametrize("variant", ["small", "two_tables", "few_jobs", "many_tables", "slow_device"])
def test_overlap_orders_every_table_and_matches_plain_rules(variant):
    cfg = {"small": OVERLAP, "few_jobs": OVERLAP, "slow_device": OVERLAP,
           "two_tables": replace(OVERLAP, n_tables=2, insert_fraction=0.5, lookup_hold_s=5e-4),
           "many_tables": replace(OVERLAP, n_tables=1024)}[variant]
    kw = {"max_jobs": 3} if variant == "few_jobs" else {}
    if variant == "slow_device":
        kw.update(dev_per_key_s=20e-9)  # flushes long enough that many turns meet one in flight
    runs = [simulate_overlap(cfg, planner=cls, **kw) for cls in (TurnPlanner, RefPlanner)]
    (st, a), (_, b) = runs
    assert len(a) == len(b)
    for (ta, x, _, _), (tb, y, _, _) in zip(a, b):
        assert ta == tb and x.admitted == y.admitted and x.inserts == y.inserts
        for f in ("lookups", "trailing", "lookups_after"):
            assert np.array_equal(getattr(x, f), getattr(y, f)), f
        assert (x.insert_first, x.insert_keys, x.nbytes, x.nbytes_b) == (y.insert_first, y.insert_keys, y.nbytes,
                                                                         y.nbytes_b)
    check_overlap_order(st, a)
    if variant in ("small", "slow_device"):
        assert sum(x.trailing.shape[0] for _, x, _, _ in a) > 0, "no lookup trailed a flush in flight"


def test_overlap_order_check_catches_trailing_lookups_on_the_first_stream():
    """Planted mistake: trailing lookups launched with the free lookups (on
    the first stream, not behind the flush in flight) can run before an
    earlier insert of their table, and the check says so."""
    from dataclasses import replace as dc_replace
    st, launched = simulate_overlap(replace(OVERLAP, n_tables=2, insert_fraction=0.5), dev_per_key_s=20e-9)
    check_overlap_order(st, launched)
    moved = [(t, dc_replace(turn, lookups=np.sort(np.concatenate([turn.lookups, turn.trailing])),
                            trailing=np.zeros(0, np.int64)), a, b) for t, turn, a, b in launched]
    with pytest.raises(AssertionError):
        check_overlap_order(st, moved)
