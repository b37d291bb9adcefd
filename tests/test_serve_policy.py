"""The served form's host policy (admission within the footprint budget, write
coalescing) on CPU: the turn planner is driven by a simulated clock and a
simulated in-order device, and every turn it plans is checked."""

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


def check_common(st, launched):
    n = st.arrival.shape[0]
    seen = np.zeros(n, np.int64)
    last_lookup, last_insert_end = -1, 0
    ins_order = []
    for t, turn, _, _ in launched:
        done = turn.done
        seen[done] += 1
        assert (st.arrival[done] <= t + 1e-12).all(), "a burst launched before it arrived"
        look = turn.lookups
        assert not st.insert[look].any() and (np.diff(look) > 0).all()
        if look.shape[0]:
            assert look[0] > last_lookup, "lookups out of arrival order"
            last_lookup = look[-1]
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


def test_every_burst_once_in_order_with_contiguous_flushes():
    st, launched, max_flight = simulate(SMALL)
    check_common(st, launched)
    assert max_flight <= SMALL.footprint_bytes
    flushes = [x for x in launched if x[1].inserts]
    assert len(flushes) > 5 and len(launched) > 50


def test_flush_triggers():
    """Each flush happens because enough keys wait, the oldest waited long
    enough, or the stream ended; none is early, and none waits much beyond
    the age limit while the device keeps up."""
    cfg = SMALL
    st, launched, _ = simulate(cfg)
    flushes = [x for x in launched if x[1].inserts]
    end = st.arrival[-1]
    host_s = 10e-6
    for t, turn, _, _ in flushes:
        oldest = st.arrival[turn.inserts[0]]
        keys_ok = turn.insert_keys >= cfg.insert_flush_keys
        age_ok = t - oldest >= cfg.insert_flush_s - 1e-12
        end_ok = t >= end
        assert keys_ok or age_ok or end_ok, (t, turn.insert_keys, t - oldest)
        assert t - oldest <= cfg.insert_flush_s + 2 * host_s + 1e-9
    # without the age limit, every flush but the last carries the key threshold,
    # and no planning call starts with the threshold already reached (no late flush)
    st, launched, _ = simulate(replace(cfg, insert_flush_s=10.0))
    flushes = [x[1] for x in launched if x[1].inserts]
    assert all(f.insert_keys >= cfg.insert_flush_keys for f in flushes[:-1])
    assert all(pend_before < cfg.insert_flush_keys for _, _, pend_before, _ in launched)


@pytest.mark.parametrize("insert_fraction", [0.0, 1.0])
def test_all_lookups_or_all_inserts(insert_fraction):
    cfg = replace(SMALL, insert_fraction=insert_fraction)
    st, launched, _ = simulate(cfg)
    check_common(st, launched)
    n_flush = sum(1 for x in launched if x[1].inserts)
    if insert_fraction == 0.0:
        assert n_flush == 0
    else:
        assert all(x[1].lookups.shape[0] == 0 for x in launched) and n_flush >= 1


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
