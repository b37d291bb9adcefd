"""Lookup strategies and the batched form against the plain lookup and the
oracle (needs a GB300)."""

import numpy as np
import pytest
import torch

import oracle
from paper_1712_09624_gb300 import workload as W

pytestmark = pytest.mark.gpu


def FT(*a, **kw):
    from paper_1712_09624_gb300.table import FlowTable
    return FlowTable(*a, **kw)


def test_lookup_strategies_agree_and_count_reads():
    """Sec. 3 / Sec. 4.1: optimistic, pessimistic and Cuckoo++ lookups return the
    same answers; they differ only in secondary-bucket reads, whose counts match
    those implied by the table the kernels built, read back bucket by bucket."""
    from paper_1712_09624_gb300 import _ckpp as K
    from gpu_layout import download, expected_probe_counts
    nb = 1 << 14
    f = W.fill(51, int(0.9 * nb * 8))
    g = FT(nb, seed=51)
    o = oracle.Table(nb, 8, False, 51)
    g.insert(f.keys, f.values)
    o.insert(f.keys, f.values)
    d = download(g)
    assert d.check() == []
    q = W.lookup_batch(51, 100003, f, 0.5)
    ov, of = o.lookup(q.keys)
    counts = {}
    for variant in (K.LOOKUP_BLOOM, K.LOOKUP_OPTIMISTIC, K.LOOKUP_PESSIMISTIC):
        v, fd = g.lookup_variant(q.keys, variant)
        assert (fd.cpu().numpy() == of).all() and (v.cpu().numpy().view(np.uint64) == ov).all()
        counts[variant] = g.probe_counts(q.keys, variant=variant).cpu().numpy()
        assert tuple(int(c) for c in counts[variant]) == expected_probe_counts(d, q.keys, variant)
    n = q.keys.shape[0]
    misses_in_primary = counts[K.LOOKUP_OPTIMISTIC][1]
    assert counts[K.LOOKUP_PESSIMISTIC][1] == n
    assert counts[K.LOOKUP_BLOOM][1] < misses_in_primary < n
    # every variant reads the same records for keys it finds; negatives add only tag false matches
    assert counts[K.LOOKUP_PESSIMISTIC][2] >= counts[K.LOOKUP_BLOOM][2]


def make_tables(n_tables, seed):
    rng = np.random.default_rng(seed)
    tables, fills = [], []
    for i in range(n_tables):
        nb = int(rng.choice([2, 3, 17, 256, 1000, 4099, 20000]))
        timers = bool(rng.random() < 0.3)
        m = int(0.85 * nb * 8)
        f = W.fill(seed * 1000 + i, m)
        t = FT(nb, timers=timers, seed=seed * 1000 + i)
        st = t.insert(f.keys, f.values, 10, 900 if timers else 0).cpu().numpy()
        assert (st == 1).all()
        tables.append(t)
        fills.append(f)
    return tables, fills


def plain_results(tables, qs):
    out = []
    for ti, keys in qs:
        v, fd = tables[ti].lookup(keys, 20)
        out.append((v.clone(), fd.to(torch.uint8).clone()))
    return out


@pytest.fixture(scope="module")
def batch_setup():
    from paper_1712_09624_gb300.batched import BatchedLookup
    tables, fills = make_tables(40, 52)
    rng = np.random.default_rng(53)
    qs = []
    for ti in range(len(tables)):
        n = int(rng.choice([0, 1, 31, 32, 33, 1000, 4097]))
        q = W.lookup_batch(52 * 1000 + ti, n, fills[ti], 0.3, batch_id=1)
        qs.append((ti, torch.from_numpy(q.keys).cuda()))
    qs.append((7, torch.from_numpy(W.lookup_batch(9, 500, fills[7], 0.3).keys).cuda()))  # a second job on one table
    return BatchedLookup(tables, max_jobs=64), tables, qs


@pytest.mark.parametrize("tuning", [(1, 1, 2, 32), (1, 2, 1, 32), (4, 2, 2, 8), (2, 1, 3, 16), (4, 1, 1, 0)])
def test_batched_equals_plain_per_table(batch_setup, tuning):
    batch, tables, qs = batch_setup
    ref = plain_results(tables, qs)
    outs = [(torch.full((k.shape[0],), -7, dtype=torch.int64, device="cuda"),
             torch.full((k.shape[0],), 9, dtype=torch.uint8, device="cuda")) for _, k in qs]
    batch.set_jobs([(ti, k, ov, of) for (ti, k), (ov, of) in zip(qs, outs)])
    batch.launch(20, tuning)
    torch.cuda.synchronize()
    for (rv, rf), (ov, of) in zip(ref, outs):
        assert torch.equal(rv, ov) and torch.equal(rf, of)


def test_batched_rejects_inconsistent_tuning(batch_setup):
    """threads_per_key is 1, 2 or 4 lanes per key; keys_per_warp, when given,
    must be 32 / threads_per_key."""
    from paper_1712_09624_gb300 import _ckpp as K
    batch, _, _ = batch_setup
    for bad in [(3, 1, 2, 0), (4, 1, 2, 32), (1, 1, 2, 8), (1, 3, 2, 0), (1, 1, 5, 0), (8, 1, 2, 4)]:
        with pytest.raises(K.CkppError) as e:
            batch.launch(20, bad)
        assert e.value.code == K.CKPP_EINVAL, bad


def test_autotune_searches_threads_per_key(batch_setup):
    """The autotuner times every (threads per key, group depth, blocks per SM)
    and keeps the fastest; the kept tuning still gives the plain results."""
    from paper_1712_09624_gb300.batched import autotune
    batch, tables, qs = batch_setup
    outs = [(torch.zeros(k.shape[0], dtype=torch.int64, device="cuda"),
             torch.zeros(k.shape[0], dtype=torch.uint8, device="cuda")) for _, k in qs]
    batch.set_jobs([(ti, k, ov, of) for (ti, k), (ov, of) in zip(qs, outs)])
    best, results = autotune(batch, sum(k.shape[0] for _, k in qs), now=20, reps=1)
    assert {c[0] for c in results} == {1, 2, 4} and len(results) == 3 * 2 * 4
    assert all(c[3] * c[0] == 32 for c in results) and best == min(results, key=results.get)
    ref = plain_results(tables, qs)
    for ov, of in outs:
        ov.zero_()
        of.zero_()
    batch.launch(20)
    torch.cuda.synchronize()
    for (rv, rf), (ov, of) in zip(ref, outs):
        assert torch.equal(rv, ov) and torch.equal(rf, of)


def test_batched_skips_jobs_without_table_and_replays_graph(batch_setup):
    batch, tables, qs = batch_setup
    ref = plain_results(tables, qs)
    outs = [(torch.full((k.shape[0],), -7, dtype=torch.int64, device="cuda"),
             torch.full((k.shape[0],), 9, dtype=torch.uint8, device="cuda")) for _, k in qs]
    jobs = [(ti, k, ov, of) for (ti, k), (ov, of) in zip(qs, outs)]
    bad_keys = qs[5][1]
    bad_out = (torch.full((bad_keys.shape[0],), -7, dtype=torch.int64, device="cuda"),
               torch.full((bad_keys.shape[0],), 9, dtype=torch.uint8, device="cuda"))
    batch.set_jobs(jobs[:10] + [(len(tables) + 3, bad_keys, *bad_out)])
    batch.capture(20)
    batch.replay()
    torch.cuda.synchronize()
    for (rv, rf), (ov, of) in zip(ref[:10], outs[:10]):
        assert torch.equal(rv, ov) and torch.equal(rf, of)
    assert bool((bad_out[0] == -7).all()) and bool((bad_out[1] == 9).all())
    # rewrite the jobs, replay the same graph
    outs2 = [(torch.zeros(k.shape[0], dtype=torch.int64, device="cuda"),
              torch.zeros(k.shape[0], dtype=torch.uint8, device="cuda")) for _, k in qs]
    batch.set_jobs([(ti, k, ov, of) for (ti, k), (ov, of) in zip(qs, outs2)])
    batch.replay()
    torch.cuda.synchronize()
    for (rv, rf), (ov, of) in zip(ref, outs2):
        assert torch.equal(rv, ov) and torch.equal(rf, of)


def test_batched_max_jobs_mostly_tiny_and_empty():
    """8192 jobs (the maximum), most with 0-2 keys and a few large, in random
    order: a lane's key often lies many jobs past its previous key's job, so
    the job search gallops far and crosses runs of empty jobs. Every output
    equals the plain per-table lookup."""
    from paper_1712_09624_gb300 import _ckpp as K
    from paper_1712_09624_gb300.batched import BatchedLookup
    tables, fills = make_tables(12, 54)
    rng = np.random.default_rng(55)
    pools = [torch.from_numpy(W.lookup_batch(54 * 1000 + ti, 20000, fills[ti], 0.3, batch_id=2).keys).cuda()
             for ti in range(len(tables))]
    n_jobs = K.BATCH_MAX_JOBS
    sizes = rng.choice([0, 0, 0, 1, 1, 2, 33, 2000], size=n_jobs, p=[0.3, 0.1, 0.1, 0.2, 0.1, 0.1, 0.07, 0.03])
    qs = []
    for j in range(n_jobs):
        ti = int(rng.integers(0, len(tables)))
        lo = int(rng.integers(0, 20000 - int(sizes[j])))
        qs.append((ti, pools[ti][lo:lo + int(sizes[j])]))
    ref = plain_results(tables, qs)
    outs = [(torch.full((k.shape[0],), -7, dtype=torch.int64, device="cuda"),
             torch.full((k.shape[0],), 9, dtype=torch.uint8, device="cuda")) for _, k in qs]
    batch = BatchedLookup(tables, max_jobs=n_jobs)
    batch.set_jobs([(ti, k, ov, of) for (ti, k), (ov, of) in zip(qs, outs)])
    for tuning in [(1, 1, 2, 32), (4, 2, 1, 8)]:
        for ov, of in outs:
            ov.fill_(-7)
            of.fill_(9)
        batch.launch(20, tuning)
        torch.cuda.synchronize()
        for (rv, rf), (ov, of) in zip(ref, outs):
            assert torch.equal(rv, ov) and torch.equal(rf, of)


def test_batched_matches_oracle_small():
    """Batched results against the oracle on a few small tables."""
    from paper_1712_09624_gb300.batched import BatchedLookup
    tables, fills, ors = [], [], []
    for i, nb in enumerate((5, 300, 2048)):
        f = W.fill(60 + i, int(0.9 * nb * 8))
        t = FT(nb, seed=60 + i)
        t.insert(f.keys, f.values)
        o = oracle.Table(nb, 8, False, 60 + i)
        o.insert(f.keys, f.values)
        tables.append(t), fills.append(f), ors.append(o)
    b = BatchedLookup(tables)
    qs = [W.lookup_batch(70 + i, 3000, fills[i], 0.3) for i in range(3)]
    outs = [(torch.empty(3000, dtype=torch.int64, device="cuda"), torch.empty(3000, dtype=torch.uint8, device="cuda"))
            for _ in range(3)]
    b.set_jobs([(i, torch.from_numpy(qs[i].keys).cuda(), *outs[i]) for i in range(3)])
    b.launch()
    torch.cuda.synchronize()
    for i in range(3):
        ov, of = ors[i].lookup(qs[i].keys)
        assert (outs[i][1].cpu().numpy() == of).all()
        assert (outs[i][0].cpu().numpy().view(np.uint64) == ov).all()


def test_batch_insert_and_delete_across_tables_match_per_table_calls():
    """ckpp_batch_insert / ckpp_batch_delete (one call, keys bound for many
    tables) give the statuses and tables of one ckpp_bulk_insert /
    ckpp_bulk_delete per table, and the oracle's."""
    from paper_1712_09624_gb300 import _ckpp as K
    from paper_1712_09624_gb300.batched import BatchedLookup
    from gpu_layout import download, oracle_live
    rng = np.random.default_rng(80)
    sizes = [3, 64, 500, 2000]
    multi = [FT(nb, timers=(i % 2 == 1), seed=80 + i) for i, nb in enumerate(sizes)]
    single = [FT(nb, timers=(i % 2 == 1), seed=80 + i) for i, nb in enumerate(sizes)]
    ors = [oracle.Table(nb, 8, i % 2 == 1, 80 + i) for i, nb in enumerate(sizes)]
    batch = BatchedLookup(multi)
    pools = [W.make_keys(80 + i, 81, int(1.1 * nb * 8)) for i, nb in enumerate(sizes)]
    now = 10
    for step in range(6):
        tids, keys, vals = [], [], []
        for i, nb in enumerate(sizes):
            cap = int(0.85 * nb * 8) - ors[i].size()
            n = int(rng.integers(0, max(1, min(cap, 400)) + 1))
            pick = pools[i][rng.integers(0, pools[i].shape[0], n)]
            tids.append(np.full(n, i, np.int32)), keys.append(pick)
            vals.append(rng.integers(0, 2**62, n, dtype=np.int64).astype(np.uint64))
        order = rng.permutation(sum(len(t) for t in tids))  # keys of all tables interleaved
        T = np.concatenate(tids)[order]
        Kk = np.concatenate(keys)[order]
        V = np.concatenate(vals)[order]
        bad = np.array([len(sizes) + 5], np.int32)  # one key naming no table
        T = np.concatenate([T, bad]); Kk = np.concatenate([Kk, pools[0][:1]]); V = np.concatenate([V, [7]]).astype(np.uint64)
        kd = torch.from_numpy(Kk).cuda(); td = torch.from_numpy(T).cuda()
        vd = torch.from_numpy(V.view(np.int64)).cuda(); st = torch.empty(len(T), dtype=torch.uint8, device="cuda")
        ws = torch.empty(K.ckpp_workspace_bytes(len(T)), dtype=torch.uint8, device="cuda")
        K.ckpp_batch_insert(batch.handle, kd, td, vd, st, ws, now, 500)
        st = st.cpu().numpy()
        assert st[-1] == K.ST_NO_TABLE
        for i in range(len(sizes)):
            sel = np.nonzero(T[:-1] == i)[0]
            ref = single[i].insert(Kk[sel], V[sel], now, 500).cpu().numpy()
            assert (st[sel] == ref).all()
            assert (st[sel] == ors[i].insert(Kk[sel], V[sel], now, 500)).all()
        # delete a few keys of every table in one call
        dsel = rng.choice(len(T) - 1, size=min(200, len(T) - 1), replace=False)
        dst = torch.empty(len(dsel), dtype=torch.uint8, device="cuda")
        K.ckpp_batch_delete(batch.handle, torch.from_numpy(Kk[dsel]).cuda(), torch.from_numpy(T[dsel]).cuda(),
                            dst, ws, now)
        dst = dst.cpu().numpy()
        for i in range(len(sizes)):
            sel = np.nonzero(T[dsel] == i)[0]
            assert (dst[sel] == ors[i].delete(Kk[dsel][sel], now)).all()
            single[i].delete(Kk[dsel][sel], now)
        now += 7
    for i in range(len(sizes)):
        d = download(multi[i])
        assert d.check() == []
        assert d.live(now) == oracle_live(ors[i], now)
