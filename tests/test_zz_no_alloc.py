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
