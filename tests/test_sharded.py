"""A table split over ranks by hash (paper_1712_09624_gb300/sharded.py), on CPU:
gloo ranks, each owning one oracle table as its shard. Inserts, lookups and
deletes routed through the two all-to-alls must give every rank exactly what
one oracle table gives for the ranks' batches concatenated in rank order
(duplicate keys across ranks included)."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

SEED = 5


def shard_of(keys: np.ndarray, n_shards: int) -> np.ndarray:
    """The shard rule stated in include/ckpp.h: bits 16-31 of the primary hash
    (from the oracle's H1), multiply-shift reduced to n_shards."""
    import oracle
    h1 = oracle.address(keys, 2, SEED)["h1"]
    return (((h1 >> np.uint64(16)) & np.uint64(0xFFFF)) * np.uint64(n_shards)) >> np.uint64(16)


class OraclePartitioner:
    """Stable partition by shard on the host (numpy), the CPU stand-in for the
    library's partition kernels."""

    def partition(self, keys, vals, n_shards):
        k = keys.numpy()
        s = shard_of(k, n_shards).astype(np.int64)
        order = np.argsort(s, kind="stable")
        counts = np.bincount(s, minlength=n_shards)
        vs = None if vals is None else torch.from_numpy(vals.numpy()[order].copy())
        return (torch.from_numpy(order.astype(np.int32)), torch.from_numpy(k[order].copy()), vs,
                torch.from_numpy(counts.astype(np.int64)))

    def unpermute(self, order, sorted_results):
        out = []
        for r in sorted_results:
            o = torch.empty_like(r)
            o[order.long()] = r
            out.append(o)
        return out


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def batches(world: int, n: int = 700):
    """Each rank's insert batch (with in-batch duplicates, and keys that
    another rank also inserts) and lookup / delete batches."""
    from paper_1712_09624_gb300 import workload as W
    out = []
    common = W.make_keys(SEED, 90, 50)
    for r in range(world):
        own = W.make_keys(SEED + r, 91, n)
        ins = np.concatenate([own, own[:40], common])
        rng = np.random.default_rng(r)
        ins = ins[rng.permutation(ins.shape[0])]
        vals = (np.arange(ins.shape[0], dtype=np.uint64) + 10_000 * r)
        fresh = W.make_keys(SEED + r, 92, 200)
        look = np.concatenate([own[:300], common[:20], fresh])
        dele = np.concatenate([own[300:400], common[20:30], fresh[:5]])
        out.append((ins, vals, look, dele))
    return out


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1712_09624_gb300.sharded import ShardRouter
    local = oracle.Table(512, 8, True, SEED)
    router = ShardRouter(OraclePartitioner())
    ins, vals, look, dele = batches(world)[rank]
    res = {}
    r = router.send(torch.from_numpy(ins), torch.from_numpy(vals.view(np.int64)))
    st = local.insert(r.keys.numpy(), r.vals.numpy().view(np.uint64), 100, 500)
    res["insert"] = router.back(r, [torch.from_numpy(st)])[0].numpy()
    res["recv_order_ok"] = True
    r = router.send(torch.from_numpy(look))
    v, f = local.lookup(r.keys.numpy(), 120)
    bv, bf = router.back(r, [torch.from_numpy(v.view(np.int64)), torch.from_numpy(f)])
    res["lookup"] = (bv.numpy().view(np.uint64), bf.numpy())
    r = router.send(torch.from_numpy(dele))
    st = local.delete(r.keys.numpy(), 130)
    res["delete"] = router.back(r, [torch.from_numpy(st)])[0].numpy()
    r = router.send(torch.from_numpy(look))
    v, f = local.lookup(r.keys.numpy(), 140)
    bv, bf = router.back(r, [torch.from_numpy(v.view(np.int64)), torch.from_numpy(f)])
    res["lookup_after_delete"] = (bv.numpy().view(np.uint64), bf.numpy())
    res["owned_ok"] = bool((shard_of(local.dump()["key"], world) == rank).all()) and local.check() == 0
    out[rank] = res
    torch.distributed.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_calls_equal_one_table(world):
    import oracle
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    bs = batches(world)
    ref = oracle.Table(512 * world, 8, True, SEED)
    st = ref.insert(np.concatenate([b[0] for b in bs]), np.concatenate([b[1] for b in bs]), 100, 500)
    seg = np.cumsum([0] + [b[0].shape[0] for b in bs])
    assert set(np.unique(st)) == {oracle.INSERTED, oracle.UPDATED}
    lookups = [ref.lookup(b[2], 120) for b in bs]
    dst = ref.delete(np.concatenate([b[3] for b in bs]), 130)
    dseg = np.cumsum([0] + [b[3].shape[0] for b in bs])
    after = [ref.lookup(b[2], 140) for b in bs]
    for r in range(world):
        assert (res[r]["insert"] == st[seg[r]:seg[r + 1]]).all(), f"rank {r}: insert statuses"
        for name, want in (("lookup", lookups[r]), ("lookup_after_delete", after[r])):
            v, f = res[r][name]
            assert (f == want[1]).all() and (v == want[0]).all(), f"rank {r}: {name}"
        assert (res[r]["delete"] == dst[dseg[r]:dseg[r + 1]]).all(), f"rank {r}: delete statuses"
        assert res[r]["owned_ok"], f"rank {r} holds a key of another shard, or its table is inconsistent"
    # keys every rank inserted resolve in rank order: the last rank's value wins (values of rank r's
    # batch are its indices plus 10000 r); look[300:320] are such keys, looked up before the deletes
    v, f = res[0]["lookup"]
    assert f[300:320].all() and (v[300:320] >= 10_000 * (world - 1)).all()


def test_single_rank_router_is_a_pass_through():
    """Without torch.distributed the router sends every key to itself."""
    from paper_1712_09624_gb300.sharded import ShardRouter
    from paper_1712_09624_gb300 import workload as W
    keys = torch.from_numpy(W.make_keys(SEED, 93, 64))
    vals = torch.arange(64, dtype=torch.int64)
    router = ShardRouter(OraclePartitioner())
    r = router.send(keys, vals)
    assert r.send_counts == r.recv_counts == [64]
    assert torch.equal(r.keys, keys) and torch.equal(r.vals, vals)
    back = router.back(r, [vals * 2])[0]
    assert torch.equal(back, vals * 2)
