"""The served form's host policy (admission within the footprint budget, write
coalescing, per-table arrival order) on CPU: the turn planner is driven by a
simulated clock and a simulated in-order device, and every turn it plans is
checked."""

from collections import deque
from dataclasses import replace

import numpy as np
import pytest

from paper_1712_09624_gb300.serve_policy import KEY_BYTES_IO, ServeConfig, TurnPlanner, draw_stream

SMALL = ServeConfig(n_tables=8, ports=8, min_burst=32, max_burst=1024, offered_lookups_per_s=50e6,
                    insert_fraction=0.2, duration_s=0.02, footprint_bytes=4 << 20, insert_flush_keys=8192,
                    insert_flush_s=200e-6, seed=3)


def simulate(cfg, host_s=10e-6, dev_fixed_s=5e-6, dev_per_key_s=0.2e-9, max_jobs=4096):
    """Runs the planner to the end. The host spends host_s per launched turn;
    the device runs turns in launch order, each taking dev_fixed_s plus
    dev_per_key_s per key. Returns the stream, the launched turns as (launch
    time, turn, insert keys waiting before the planning call, footprint
    outstanding after it) and the largest footprint ever outstanding."""
    st = draw_stream(cfg)
    pl = TurnPlanner(st, cfg, max_jobs)
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
