"""Pins of the CPU oracle against things other than itself.

Each ``check_*`` function runs one family of pins against an oracle library
handle and returns a list of failure messages (empty = all pins hold). The
oracle tests assert the lists are empty; the mutation tests build oracles with
one planted mistake each and assert that some list is not.

Pins used (none re-types the oracle's own formulas):
  * published SplitMix64 outputs for seed 0 (the mixer's constants);
  * the timer arithmetic of Sec. 4.2 (golden rows);
  * properties the hash readings must have: b1 != b2, bucket and tag
    uniformity, independence of tag and filter bits, avalanche;
  * a brute-force linear-scan list map replaying random operation streams on
    tiny tables (exact: statuses, lookup results, live sets);
  * the structural invariants of Sec. 2 and Sec. 4.1 after every batch;
  * lazy deletion (Sec. 4.2): a table full of dead entries takes new keys;
  * the fill statistics (share of entries in their secondary, moved-counter
    histogram) against a fluid-limit model of the insertion rule of Sec. 2
    and the counter rule of Sec. 4.1 (``fill_model.py``).
"""

from __future__ import annotations

import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
GOLDEN_RATIO = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def read_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ----------------------------------------------------------------- hashing

def check_splitmix_vectors(L) -> list[str]:
    bad = []
    for k, hexout in read_rows("splitmix64_seed0.txt"):
        got = int(L.oc_mix64((int(k) * GOLDEN_RATIO) & M64))
        if got != int(hexout, 16):
            bad.append(f"splitmix output {k}: {got:016x} != {hexout}")
    return bad


def check_address_properties(L, n=40000, seed=11) -> list[str]:
    """b1 != b2 for every key and bucket count; b1, b2 and tag uniform; tag
    independent of the filter bits; filter bits independent of each other."""
    from paper_1712_09624_gb300 import workload as W
    bad = []
    keys = W.make_keys(seed, 9, n)
    for nb in (2, 3, 5, 1024):
        a = oracle.address(keys, nb, seed, library=L)
        if (a["b1"] >= nb).any() or (a["b2"] >= nb).any():
            bad.append(f"bucket out of range nb={nb}")
        if (a["b1"] == a["b2"]).any():
            bad.append(f"b1 == b2 for some key, nb={nb}")
    a = oracle.address(keys, 1024, seed, library=L)
    # chi-square of b1 over 1024 buckets (df 1023): mean 1023, sd ~45
    for name in ("b1",):
        cnt = np.bincount(a[name].astype(np.int64), minlength=1024)
        exp = n / 1024
        chi = ((cnt - exp) ** 2 / exp).sum()
        if not 1023 - 6 * 45 < chi < 1023 + 6 * 45:
            bad.append(f"{name} not uniform: chi2={chi:.0f}")
    tag_lo = (a["tag"] & 63).astype(np.int64)
    # P(tag low bits == bit1) is 1/64 for independent values
    same = (tag_lo == a["bit1"].astype(np.int64)).mean()
    if not 0.5 / 64 < same < 2.0 / 64:
        bad.append(f"tag and bloom bit correlated: {same:.4f}")
    same12 = (a["bit1"] == a["bit2"]).mean()
    if not 0.5 / 64 < same12 < 2.0 / 64:
        bad.append(f"bloom bits correlated: {same12:.4f}")
    tb = np.bincount(a["tag"].astype(np.int64) >> 10, minlength=64)
    chi = ((tb - n / 64) ** 2 / (n / 64)).sum()
    if not chi < 63 + 6 * 11.2:
        bad.append(f"tag not uniform: chi2={chi:.0f}")
    # The tag must not repeat bucket-index bits (Sec. 4.3 takes it from the main
    # hash, and a tag that the bucket fixes would stop telling apart the keys
    # sharing that bucket): chi-square of 64 x 64 contingency tables between
    # b1 (and b2) over 64 buckets and the tag's low and high six bits.
    a64 = oracle.address(keys, 64, seed, library=L)
    df = 63 * 63
    for bname in ("b1", "b2"):
        for tname, tb6 in (("tag low bits", a64["tag"].astype(np.int64) & 63),
                           ("tag high bits", a64["tag"].astype(np.int64) >> 10)):
            table = np.zeros((64, 64))
            np.add.at(table, (a64[bname].astype(np.int64), tb6), 1)
            expect = np.outer(table.sum(1), table.sum(0)) / n
            chi = ((table - expect) ** 2 / np.maximum(expect, 1e-12)).sum()
            if not chi < df + 6 * (2 * df) ** 0.5:
                bad.append(f"{bname} and {tname} dependent: chi2={chi:.0f} (df {df})")
    return bad


def check_avalanche(L, n=300, seed=5) -> list[str]:
    """Flipping any one of the 128 key bits flips each bit of H1 with odds near 1/2."""
    from paper_1712_09624_gb300 import workload as W
    keys = W.make_keys(seed, 8, n)
    base = oracle.address(keys, 2, seed, library=L)["h1"]
    flips = np.zeros(64)
    for bit in range(128):
        k2 = keys.copy()
        k2[:, bit // 8] ^= np.uint8(1 << (bit % 8))
        h = oracle.address(k2, 2, seed, library=L)["h1"]
        x = base ^ h
        flips += np.unpackbits(x.view(np.uint8)).reshape(n, 64).sum(0)
    p = flips / (128 * n)
    bad = []
    if not (np.abs(p - 0.5) < 0.03).all():
        bad.append(f"avalanche off: min {p.min():.3f} max {p.max():.3f}")
    return bad


# ------------------------------------------------------------------ timers

def check_timer_golden(L) -> list[str]:
    bad = []
    for e, now, want in read_rows("timers_sec4_2.txt"):
        got = int(L.oc_alive(int(e) & 0xFFFF, int(now)))
        if got != int(want):
            bad.append(f"alive({e},{now}) = {got}, paper says {want}")
    return bad


# -------------------------------------------------- brute force replay

class ListMap:
    """Linear-scan list of [key, value, expiry]: the brute-force reference."""

    def __init__(self, timers):
        self.timers = timers
        self.rows: list[list] = []

    def alive(self, exp, now):
        return (not self.timers) or ((exp - now) & 0xFFFF) < 1024

    def find(self, kb):
        for r in self.rows:
            if r[0] == kb:
                return r
        return None

    def live(self, now):
        return sorted((r[0], r[1], r[2] if self.timers else 0) for r in self.rows if self.alive(r[2], now))


def _live_of(t: oracle.Table, now: int):
    d = t.dump()
    out = []
    for i in range(d["value"].shape[0]):
        exp = int(d["expiry"][i])
        if (not t.timers) or ((exp - now) & 0xFFFF) < 1024:
            out.append((d["key"][i].tobytes(), int(d["value"][i]), exp if t.timers else 0))
    return sorted(out)


def _free_or_dead(t: oracle.Table, bucket: int, now: int) -> bool:
    d = t.dump()
    sel = d["bucket"] == bucket
    if sel.sum() < t.slots:
        return True
    if not t.timers:
        return False
    return any(((int(e) - now) & 0xFFFF) >= 1024 for e in d["expiry"][sel])


def replay(L, seed, nb, slots, timers, n_ops, pool_factor=3.0, stop_at_first=True) -> list[str]:
    """Random insert/lookup/delete/expire stream on a tiny table, compared with
    the brute-force list after every batch."""
    rng = np.random.default_rng(seed)
    from paper_1712_09624_gb300 import workload as W
    cap = nb * slots
    pool = W.make_keys(seed, 21, max(4, int(pool_factor * cap)))
    t = oracle.Table(nb, slots, timers, seed, library=L)
    ref = ListMap(timers)
    now = 1000
    last_scan = now
    bad: list[str] = []

    def fail(msg):
        bad.append(f"[seed={seed} nb={nb} S={slots} timers={timers}] {msg}")

    for step in range(n_ops):
        if bad and stop_at_first:
            break
        r = rng.random()
        if timers and r < 0.12:
            now += int(rng.integers(0, 700)) if rng.random() < 0.8 else int(rng.integers(1000, 3000))
            continue
        if timers and (r < 0.17 or now - last_scan > 60000):
            last_scan = now
            t.expire(now)
            ref.rows = [x for x in ref.rows if ref.alive(x[2], now)]
            d = t.dump()
            if any(((int(e) - now) & 0xFFFF) >= 1024 for e in d["expiry"]):
                fail(f"step {step}: dead entry left after expire")
            continue
        m = int(rng.integers(1, 7))
        idx = rng.integers(0, pool.shape[0], m)
        keys = pool[idx]
        if r < 0.55:
            vals = rng.integers(0, 2**63, m, dtype=np.int64).astype(np.uint64)
            ttl = int(rng.integers(0, 1024))
            st = t.insert(keys, vals, now, ttl)
            for i in range(m):
                kb = keys[i].tobytes()
                row = ref.find(kb)
                if st[i] == oracle.FULL:
                    a = oracle.address(keys[i:i + 1], nb, seed, library=L)
                    stored = any(k.tobytes() == kb for k in t.dump()["key"])
                    if stored:
                        fail(f"step {step}: FULL for a key already stored")
                    elif _free_or_dead(t, int(a["b1"][0]), now) or _free_or_dead(t, int(a["b2"][0]), now):
                        fail(f"step {step}: FULL while a bucket of the key has a free or dead slot")
                    continue
                want = oracle.UPDATED if (row is not None and ref.alive(row[2], now)) else oracle.INSERTED
                if st[i] != want:
                    fail(f"step {step}: insert status {st[i]} != {want}")
                if row is None:
                    row = [kb, 0, 0]
                    ref.rows.append(row)
                row[1] = int(vals[i])
                row[2] = (now + ttl) & 0xFFFF if timers else 0
        elif r < 0.85:
            refresh = int(rng.integers(0, 1024)) if (timers and rng.random() < 0.3) else 0
            vals, found = t.lookup(keys, now, refresh)
            for i in range(m):
                row = ref.find(keys[i].tobytes())
                ok = row is not None and ref.alive(row[2], now)
                if found[i] != ok or (ok and vals[i] != row[1]) or (not ok and vals[i] != 0):
                    fail(f"step {step}: lookup ({found[i]},{vals[i]}) != ({int(ok)},{row[1] if ok else 0})")
                if ok and refresh:
                    row[2] = (now + refresh) & 0xFFFF
        else:
            st = t.delete(keys, now)
            for i in range(m):
                kb = keys[i].tobytes()
                row = ref.find(kb)
                want = oracle.DELETED if (row is not None and ref.alive(row[2], now)) else oracle.NOT_FOUND
                if st[i] != want:
                    fail(f"step {step}: delete status {st[i]} != {want}")
                if row is not None:
                    ref.rows.remove(row)
        rc = t.check(True)
        if rc:
            fail(f"step {step}: invariant {rc} violated")
        if _live_of(t, now) != ref.live(now):
            fail(f"step {step}: live set differs from the brute-force list")
    t.close()
    return bad


REPLAY_CONFIGS = [
    # (seed, nb, slots, timers, n_ops, pool_factor)
    (1, 2, 2, False, 250, 3.0),
    (2, 3, 4, False, 250, 2.0),
    (3, 4, 8, False, 300, 1.6),
    (4, 16, 8, False, 300, 1.3),
    (5, 2, 8, True, 300, 2.0),
    (6, 5, 4, True, 300, 2.0),
    (7, 16, 8, True, 400, 1.4),
    (8, 8, 2, True, 300, 1.5),
]


def check_replays(L, configs=REPLAY_CONFIGS) -> list[str]:
    bad = []
    for cfg in configs:
        bad += replay(L, *cfg)
    return bad


def check_lazy_reuse(L) -> list[str]:
    """Sec. 4.2: inserting over dead entries works like inserting into free slots."""
    from paper_1712_09624_gb300 import workload as W
    bad = []
    nb, slots = 2, 2
    t = oracle.Table(nb, slots, True, 3, library=L)
    k1 = W.make_keys(3, 31, 64)
    placed = 0
    for i in range(64):
        if placed == nb * slots:
            break
        st = t.insert(k1[i:i + 1], np.array([i], np.uint64), 10, 1)
        placed += int(st[0] == oracle.INSERTED)
    if t.size() != nb * slots:
        bad.append("could not fill the tiny table")
    k2 = W.make_keys(3, 32, 4)
    st = t.insert(k2, np.arange(4, dtype=np.uint64), 20, 5)  # every old entry is dead at now=20
    if not (st == oracle.INSERTED).all():
        bad.append(f"dead slots not reused: {st}")
    _, found = t.lookup(k2, 20)
    if not found.all():
        bad.append("keys inserted over dead slots not found")
    t.close()
    return bad


# ------------------------------------------- fill statistics vs a model

def fill_statistics(L, nb, load_factors, seed):
    """Fill an nb x 8 table in key order and record, at each load factor, the
    share of entries in their secondary bucket, the share of zero moved
    counters, the counter histogram and the exact filter pass rate of a
    negative key (mean over buckets of P(both query bits set))."""
    from paper_1712_09624_gb300 import workload as W
    cap = nb * 8
    t = oracle.Table(nb, 8, False, seed, library=L)
    f = W.fill(seed, int(max(load_factors) * cap))
    out, done = {}, 0
    for lf in sorted(load_factors):
        m = int(lf * cap)
        st = t.insert(f.keys[done:m], f.values[done:m])
        done = m
        bloom, moved = t.meta()
        bits = np.unpackbits(bloom.view(np.uint8)).reshape(-1, 64).sum(1).astype(np.float64)
        out[lf] = dict(
            all_inserted=bool((st == oracle.INSERTED).all()),
            f_sec=float(t.dump()["in_secondary"].mean()),
            moved_zero=float((moved == 0).mean()),
            hist=np.bincount(moved) / nb,
            fpr_exact=float(((bits / 64.0) ** 2).mean()),
            table=t,
        )
    return out


def check_fill_model(L, nb=1 << 16, seed=3) -> list[str]:
    """Sec. 2 (primary if it has room, else secondary) and Sec. 4.1 (counter per
    displaced key) against the fluid-limit model of that rule
    (``fill_model.py``), at load factors where keys with both buckets full are
    rare enough for the model to be exact. Bands are five standard deviations
    of the table-to-table spread at this size (measured over seeds)."""
    import fill_model
    model = fill_model.fill_model([0.6, 0.7, 0.8])
    got = fill_statistics(L, nb, [0.6, 0.7, 0.8], seed)
    bad = []
    for lf in (0.6, 0.7, 0.8):
        g, m = got[lf], model[lf]
        if not g["all_inserted"]:
            bad.append(f"fill to LF {lf} left keys not INSERTED")
        if abs(g["f_sec"] - m["f_sec"]) > 0.0015:
            bad.append(f"LF {lf}: secondary share {g['f_sec']:.4f}, model {m['f_sec']:.4f}")
        if abs(g["moved_zero"] - m["moved_zero"]) > 0.005:
            bad.append(f"LF {lf}: zero-counter share {g['moved_zero']:.4f}, model {m['moved_zero']:.4f}")
        k = max(len(g["hist"]), 16)
        gh = np.pad(g["hist"], (0, k - len(g["hist"])))
        tv = 0.5 * np.abs(gh - m["hist"][:k]).sum() + 0.5 * m["hist"][k:].sum()
        if tv > 0.008:
            bad.append(f"LF {lf}: counter histogram off the model by {tv:.4f} (total variation)")
    for v in got.values():
        v["table"].close()
    return bad


ALL_CHECKS = [check_splitmix_vectors, check_timer_golden, check_address_properties, check_avalanche,
              check_lazy_reuse, check_replays, check_fill_model]
