"""Served form: continuous batching gives every burst the result it gets
alone (needs a GB300). A fifth of the lookup keys name flows that earlier
insert bursts of the same table add during the run, so a lookup launched
before an earlier insert of its table, or after a later one, would show."""

import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("max_inflight,overlap", [(1, False), (0, False), (3, False), (1, True), (2, True)])
def test_served_results_equal_alone_results(max_inflight, overlap):
    from paper_1712_09624_gb300.serve import ServeConfig, Service
    # 8 tables of 64K slots at LF 0.6; ~60K new flows arrive (10% of 0.6 M keys offered), well within capacity;
    # the pacing of the loop (turns queued on the device) changes the turns, never the results
    cfg = ServeConfig(n_tables=8, total_slots=1 << 19, warm_lf=0.6, ports=4, min_burst=32, max_burst=512,
                      offered_lookups_per_s=20e6, insert_fraction=0.1, neg_rate=0.2, duration_s=0.03,
                      footprint_bytes=1 << 20, seed=11, max_inflight=max_inflight, overlap=overlap)
    mixed = Service(cfg)
    alone = Service(cfg)
    rm = mixed.run("batched")
    ra = alone.run("plain")
    assert rm["bursts"] == ra["bursts"] > 50
    assert rm["read_after_write_keys"] > 1000
    assert rm["held_lookup_bursts"] > 0, "no lookup waited for an insert: the ordering rule went unexercised"
    if overlap:
        assert rm["trailing_lookup_bursts"] > 0, "no lookup trailed a flush in flight"
    assert mixed.check() == {"lookups_match_map": True, "inserts_all_inserted": True}
    assert alone.check() == {"lookups_match_map": True, "inserts_all_inserted": True}
    for pm, pa in zip(mixed.pools, alone.pools):
        assert torch.equal(pm["vals"], pa["vals"]) and torch.equal(pm["found"], pa["found"])
    assert torch.equal(mixed.ins_status, alone.ins_status)
    # the inserted flows are in their tables afterwards
    import numpy as np
    st = mixed.stream
    ins_tables = np.repeat(st.table[st.insert], st.size[st.insert])
    for t in range(cfg.n_tables):
        sel = torch.from_numpy(np.nonzero(ins_tables == t)[0]).cuda()
        if sel.numel() == 0:
            continue
        v, f = mixed.tables[t].lookup(mixed.ins_keys[sel])
        assert bool(f.all()) and torch.equal(v, mixed.ins_vals[sel])
    # the read-after-write keys are hits, in both arms
    for t, p in enumerate(mixed.pools):
        pos = torch.from_numpy(st.raw_pos[st.raw_table == t]).cuda()
        assert bool(p["found"][pos].all()) and bool(alone.pools[t]["found"][pos].all())
    assert rm["latency_us"]["p50"] > 0
