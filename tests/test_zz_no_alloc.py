"""ckpp_bulk_insert_noalloc against ckpp_bulk_insert (needs a GB300).

The no-alloc entry point is for callers that cannot allocate device memory
when they insert (a data-plane thread held to a fixed memory budget, a plugin
whose host framework owns all device memory): it uses a scratch array built
into the library instead of a caller workspace. Two calls in a row through the
C ABI must give the same statuses, lookups and live set as the workspace
entry point on an identical table; the array keeps the previous call's
contents, so the second call also checks that the entry point clears it.
This file is collected last on purpose.
"""

import numpy as np
import pytest
import torch

from paper_1712_09624_gb300 import workload as W

pytestmark = pytest.mark.gpu


def test_noalloc_matches_workspace_insert_two_calls():
    from gpu_layout import download
    from paper_1712_09624_gb300 import _ckpp as K
    from paper_1712_09624_gb300.table import FlowTable

    nb = 1 << 13
    a = FlowTable(nb, timers=True, seed=77)
    b = FlowTable(nb, timers=True, seed=77)
    first = W.make_keys(77, 70, 40000)
    second = np.concatenate([W.make_keys(77, 71, 20000), first[:15000], first[:3000]])
    batches = [(first, 10, 500), (second, 20, 700)]
    for call, (keys_np, now, ttl) in enumerate(batches):
        keys = torch.from_numpy(keys_np).cuda()
        vals = torch.arange(keys.shape[0], dtype=torch.int64, device="cuda") + 1000 * call
        st_ws = torch.empty(keys.shape[0], dtype=torch.uint8, device="cuda")
        st_na = torch.empty(keys.shape[0], dtype=torch.uint8, device="cuda")
        K.ckpp_bulk_insert(a.handle, keys, vals, st_ws, a.workspace(keys.shape[0]), now, ttl)
        K.ckpp_bulk_insert_noalloc(b.handle, keys, vals, st_na, now, ttl)
        assert torch.equal(st_ws, st_na), f"call {call}: statuses differ"
        assert set(np.unique(st_na.cpu().numpy())) <= {K.ST_INSERTED, K.ST_UPDATED}
        va, fa = a.lookup(keys, now)
        vb, fb = b.lookup(keys, now)
        assert torch.equal(fa, fb) and torch.equal(va, vb), f"call {call}: lookups differ"
    da, db = download(a), download(b)
    assert db.check() == []
    assert da.live(20) == db.live(20)
    assert a.sync_status() == 0 and b.sync_status() == 0


def test_noalloc_full_size_batch_near_capacity():
    """A call of exactly CKPP_NOALLOC_MAX_KEYS keys fills the scratch array to
    its last byte (the largest duplicate-key set, lists and fixup list). It
    takes a timers table from 58K live entries plus 40K dead ones to load
    factor 0.9, so the batch reuses dead slots (moved-counter upkeep and the
    deferred filter resets) and needs cuckoo paths; 5,536 of its keys repeat
    earlier keys of the batch. The no-alloc call must match the workspace call
    on a table built the same way."""
    from gpu_layout import download
    from paper_1712_09624_gb300 import _ckpp as K
    from paper_1712_09624_gb300.table import FlowTable

    nb = 1 << 14
    n_max = K.NOALLOC_MAX_KEYS
    live = int(0.9 * nb * 8) - 60000
    a = FlowTable(nb, timers=True, seed=79)
    b = FlowTable(nb, timers=True, seed=79)
    pre_dead = W.make_keys(79, 73, 40000)
    pre_live = W.make_keys(79, 74, live)
    fresh = W.make_keys(79, 75, 60000)
    rng = np.random.default_rng(79)
    big = np.concatenate([fresh, fresh[rng.integers(0, 60000, n_max - 60000)]])
    big = big[rng.permutation(n_max)]
    assert big.shape[0] == n_max
    for t in (a, b):
        assert (t.insert(pre_dead, np.arange(40000), 10, 5).cpu().numpy() == K.ST_INSERTED).all()
        assert (t.insert(pre_live, np.arange(live), 10, 1000).cpu().numpy() == K.ST_INSERTED).all()
    keys = torch.from_numpy(big).cuda()
    vals = torch.arange(n_max, dtype=torch.int64, device="cuda") + 7
    st_ws = torch.empty(n_max, dtype=torch.uint8, device="cuda")
    st_na = torch.empty(n_max, dtype=torch.uint8, device="cuda")
    ws = a.workspace(n_max)
    K.ckpp_bulk_insert(a.handle, keys, vals, st_ws, ws, 20, 900)
    K.ckpp_bulk_insert_noalloc(b.handle, keys, vals, st_na, 20, 900)
    torch.cuda.synchronize()
    diag = ws[:32].cpu().numpy().view(np.uint32)
    assert diag[0] > 0, "no key needed a cuckoo path: the case does not reach the displacement passes"
    assert torch.equal(st_ws, st_na)
    assert set(np.unique(st_na.cpu().numpy())) == {K.ST_INSERTED, K.ST_UPDATED}
    assert int((st_na == K.ST_INSERTED).sum()) == 60000
    va, fa = a.lookup(keys, 20)
    vb, fb = b.lookup(keys, 20)
    assert bool(fb.all()) and torch.equal(fa, fb) and torch.equal(va, vb)
    da, db = download(a), download(b)
    assert db.check() == [] and da.check() == []
    assert da.live(20) == db.live(20)
    assert len(db.live(20)) == live + 60000
    assert a.sync_status() == 0 and b.sync_status() == 0


def test_noalloc_rejects_oversized_batch():
    from paper_1712_09624_gb300 import _ckpp as K
    from paper_1712_09624_gb300.table import FlowTable

    t = FlowTable(1 << 12, seed=78)
    n = K.NOALLOC_MAX_KEYS + 1
    keys = torch.from_numpy(W.make_keys(78, 72, n)).cuda()
    vals = torch.zeros(n, dtype=torch.int64, device="cuda")
    st = torch.empty(n, dtype=torch.uint8, device="cuda")
    with pytest.raises(K.CkppError) as e:
        K.ckpp_bulk_insert_noalloc(t.handle, keys, vals, st, 0, 0)
    assert e.value.code == K.CKPP_EINVAL
