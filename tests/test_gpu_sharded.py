"""The sharding kernels (ckpp_shard_partition, ckpp_shard_unpermute) against a
host restatement of the shard rule and a stable sort, and a single-rank
ShardedTable against a plain table (needs a GB300). More ranks than one run
only on CPU here (tests/test_sharded.py): one GPU cannot host ranks whose
collectives wait on one another."""

import numpy as np
import pytest
import torch

from paper_1712_09624_gb300 import workload as W

pytestmark = pytest.mark.gpu


def expected_shards(keys: np.ndarray, seed: int, n_shards: int) -> np.ndarray:
    import oracle
    h1 = oracle.address(keys, 2, seed)["h1"]
    return ((((h1 >> np.uint64(16)) & np.uint64(0xFFFF)) * np.uint64(n_shards)) >> np.uint64(16)).astype(np.int64)


@pytest.mark.parametrize("n,n_shards", [(100_003, 1), (100_003, 3), (257, 8), (1 << 18, 64), (1, 5),
                                         (3_000_017, 13), ((1 << 22) + 5, 64)])
def test_partition_is_a_stable_sort_by_shard(n, n_shards):
    from paper_1712_09624_gb300 import _ckpp as K
    seed = 17
    keys_np = W.make_keys(seed, 80, n)
    keys_np[: n // 10] = keys_np[n // 10: 2 * (n // 10)]  # duplicates keep their batch order
    vals_np = np.arange(n, dtype=np.int64) * 3 + 1
    keys = torch.from_numpy(keys_np).cuda()
    vals = torch.from_numpy(vals_np).cuda()
    pos = torch.empty(n, dtype=torch.int32, device="cuda")
    ks = torch.empty_like(keys)
    vs = torch.empty_like(vals)
    counts = torch.empty(n_shards, dtype=torch.int64, device="cuda")
    ws = torch.empty(K.ckpp_shard_workspace_bytes(n, n_shards), dtype=torch.uint8, device="cuda")
    K.ckpp_shard_partition(keys, vals, seed, n_shards, pos, ks, vs, counts, ws)
    shard = expected_shards(keys_np, seed, n_shards)
    want = np.argsort(shard, kind="stable")
    assert (pos.cpu().numpy()[want] == np.arange(n)).all()  # key want[j] sits at sorted position j
    assert (ks.cpu().numpy() == keys_np[want]).all() and (vs.cpu().numpy() == vals_np[want]).all()
    assert (counts.cpu().numpy() == np.bincount(shard, minlength=n_shards)).all()
    # unpermute: results in sorted order go back to the caller's order
    back64 = torch.empty_like(vs)
    back8 = torch.empty(n, dtype=torch.uint8, device="cuda")
    K.ckpp_shard_unpermute(pos, vs, (vs & 0xFF).to(torch.uint8), back64, back8)
    assert torch.equal(back64, vals) and torch.equal(back8, (vals & 0xFF).to(torch.uint8))


def test_partition_edges():
    from paper_1712_09624_gb300 import _ckpp as K
    ws = torch.empty(K.ckpp_shard_workspace_bytes(16, 4), dtype=torch.uint8, device="cuda")
    empty = torch.empty((0, 16), dtype=torch.uint8, device="cuda")
    counts = torch.full((4,), 7, dtype=torch.int64, device="cuda")
    o = torch.empty(0, dtype=torch.int32, device="cuda")
    K.ckpp_shard_partition(empty, None, 1, 4, o, empty, None, counts, ws)
    assert counts.cpu().tolist() == [0, 0, 0, 0]
    assert K.ckpp_shard_workspace_bytes(16, 0) == 0 and K.ckpp_shard_workspace_bytes(16, K.MAX_SHARDS + 1) == 0
    keys = torch.from_numpy(W.make_keys(1, 81, 16)).cuda()
    for bad in (0, K.MAX_SHARDS + 1):
        with pytest.raises(K.CkppError):
            K.ckpp_shard_partition(keys, None, 1, bad, torch.empty(16, dtype=torch.int32, device="cuda"),
                                   torch.empty_like(keys), None, torch.empty(max(bad, 1), dtype=torch.int64,
                                                                             device="cuda"), ws)


def test_single_rank_sharded_table_equals_plain_table():
    """Without torch.distributed the shard table is the only shard: its calls
    (through the partition and unpermute kernels) equal a plain table's."""
    from paper_1712_09624_gb300.sharded import ShardedTable
    from paper_1712_09624_gb300.table import FlowTable
    nb, seed = 1 << 12, 23
    st = ShardedTable(nb, timers=True, seed=seed)
    ft = FlowTable(nb, timers=True, seed=seed)
    f = W.fill(seed, int(0.8 * nb * 8))
    keys = torch.from_numpy(f.keys).cuda()
    vals = torch.from_numpy(f.values.view(np.int64)).cuda()
    a = st.insert(keys, vals, 5, 100)
    b = ft.insert(keys, vals, 5, 100)
    assert torch.equal(a, b)
    q = torch.from_numpy(W.lookup_batch(seed, 20000, f, 0.4).keys).cuda()
    va, fa = st.lookup(q, 6)
    vb, fb = ft.lookup(q, 6)
    assert torch.equal(fa, fb) and torch.equal(va, vb)
    assert torch.equal(st.delete(q[:5000], 7), ft.delete(q[:5000], 7))
