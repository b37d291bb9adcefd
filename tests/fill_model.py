"""Fluid-limit model of filling a two-choice bucketized cuckoo table.

An independent prediction of the statistics the paper plots for a table filled
with random keys (Sec. 3 / Fig. 2: fraction of entries in their secondary
bucket; Sec. 4.1 / Fig. 5: moved counters; Sec. 4.1 / Table 2: filter false
positives). It follows the insertion rule of Sec. 2 and the counter rule of
Sec. 4.1 only, and shares nothing with the oracle's code, so the oracle's fill
statistics can be checked against it.

The rule: a new key goes into its primary bucket if that bucket has a free
slot. Otherwise the key (or, through a cuckoo path, an entry the primary
gives up) ends up in its secondary bucket, which sets two bits of the
primary's filter and increments the primary's moved counter.

Model (t = keys inserted per bucket, so load factor = t / S; the number of
buckets is taken to infinity):
  n_i(t)  fraction of buckets holding i < S entries;
  m_c(t)  fraction of full buckets whose moved counter is c;
  f = sum_c m_c, the fraction of full buckets.
Each key has a uniform primary. While its primary has room (probability 1-f)
the key lands there; when it is full (probability f) one entry is displaced
and the full primary's counter goes up by one. Every key adds one entry to
some bucket that has room; primaries are uniform and secondaries are uniform,
so a bucket with room gains entries at rate 1/(1-f) (rate 1 in total spread
over the fraction 1-f). Hence

  dn_0/dt = -r n_0,   dn_i/dt = r (n_{i-1} - n_i),   r = 1 / (1 - f),
  dm_0/dt = r n_{S-1} - m_0,   dm_c/dt = m_{c-1} - m_c.

The fraction of entries in their secondary bucket is sum_c c m_c / t, and the
fraction of zero counters is sum_i n_i + m_0. The model is exact as the
bucket count grows while keys whose two buckets are both full stay rare. Once
they are common (load factor 0.9 and up with 8 slots) a cuckoo path can
displace more than one entry, which the model does not count, so there it is
a lower bound on the secondary fraction, and an upper bound on the share of
zero counters, for a breadth-first path search.

Filter pass rate (Table 2's false-positive rate): a counter of c means c keys
each set two independent uniform bits of 64. A negative key tests two
independent uniform bits; it passes with probability
  q1/64 + (63/64) q2,  q1 = 1 - (63/64)^(2c),  q2 = 1 - 2 (63/64)^(2c) + (62/64)^(2c),
where q1 is the chance a given bit is set and q2 the chance two given distinct
bits both are (inclusion-exclusion). Averaged over the counter histogram of a
freshly filled table (no deletions, so no stale bits) this is the expected
share of negative lookups that read the secondary bucket.
"""

from __future__ import annotations

import numpy as np


def _rhs(n, m, S):
    f = m.sum()
    r = 1.0 / (1.0 - f)
    dn = np.empty_like(n)
    dn[0] = -r * n[0]
    dn[1:] = r * (n[:-1] - n[1:])
    dm = np.empty_like(m)
    dm[0] = r * n[S - 1] - m[0]
    dm[1:] = m[:-1] - m[1:]
    return dn, dm


def fill_model(load_factors, slots: int = 8, dt: float = 2e-3, cmax: int = 96) -> dict:
    """Model statistics at each load factor (ascending), integrated with RK4.

    Returns {lf: {"f_sec", "moved_zero", "hist" (counter -> fraction of buckets),
    "full", "fpr"}}."""
    S = slots
    n = np.zeros(S)
    n[0] = 1.0
    m = np.zeros(cmax)
    t = 0.0
    out = {}
    for lf in sorted(load_factors):
        T = lf * S
        while t < T - 1e-12:
            h = min(dt, T - t)
            k1 = _rhs(n, m, S)
            k2 = _rhs(n + 0.5 * h * k1[0], m + 0.5 * h * k1[1], S)
            k3 = _rhs(n + 0.5 * h * k2[0], m + 0.5 * h * k2[1], S)
            k4 = _rhs(n + h * k3[0], m + h * k3[1], S)
            n = n + h / 6.0 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
            m = m + h / 6.0 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
            t += h
        hist = m.copy()
        hist[0] += n.sum()
        c = np.arange(cmax)
        out[lf] = {
            "f_sec": float((c * m).sum() / T),
            "moved_zero": float(hist[0]),
            "hist": hist,
            "full": float(m.sum()),
            "fpr": float((hist * pass_rate(c)).sum()),
        }
    return out


def pass_rate(c):
    """Chance that a negative key passes a 64-bit filter holding c keys (two
    independent uniform bit indices per key and per query)."""
    c = np.asarray(c, dtype=np.float64)
    a = (63.0 / 64.0) ** (2 * c)
    b = (62.0 / 64.0) ** (2 * c)
    q1 = 1.0 - a
    q2 = 1.0 - 2.0 * a + b
    return q1 / 64.0 + (63.0 / 64.0) * q2
