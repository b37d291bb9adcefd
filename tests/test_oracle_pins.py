"""The CPU oracle against its pins (no GPU).

The oracle is what the CUDA path is checked against, so it is itself pinned
to things other than itself: published SplitMix64 outputs, the timer arithmetic
of Sec. 4.2, properties of the hash readings, a brute-force list map on tiny
tables, the structural invariants of Sec. 2 / Sec. 4.1, a fluid-limit model of
the insertion rule, and the statistics the paper prints (Fig. 2, Fig. 5,
Table 2). A mutation test plants known mistakes in the oracle and checks that
these pins catch every one.
"""

import os

import numpy as np
import pytest

import oracle
import fill_model
import oracle_pins as P
from oracle.odef import MapTable
from paper_1712_09624_gb300 import workload as W


@pytest.fixture(scope="module")
def L():
    return oracle.lib()


@pytest.mark.parametrize("check", P.ALL_CHECKS, ids=lambda c: c.__name__)
def test_pin(L, check):
    assert check(L) == []


# mutant id -> planted mistake (see OC_MUTANT in the oracle source)
MUTANTS = {
    1: "filter insertion sets only one of the two bits",
    2: "filter never reset when the moved counter reaches zero",
    3: "tag taken from the secondary hash",
    4: "both filter bit indices taken from the same six hash bits",
    5: "alive test uses <= 1024",
    6: "in_secondary flag not updated on a cuckoo move",
    7: "removal forgets the moved counter",
    8: "lookup filter test inverted",
    9: "dead slots not reused by insertion",
    10: "upsert always reports UPDATED",
    11: "b2 may equal b1",
    12: "lookup returns dead entries",
    13: "the expire scan removes dead entries without the moved-counter upkeep",
    14: "a cuckoo move out of a secondary bucket keeps the primary's moved counter",
    15: "an update in place keeps the old expiry",
    16: "b1 taken from the low bits of H1, which the tag also uses",
    17: "the cuckoo-path search starts from the secondary bucket",
    18: "insertion tries the secondary bucket before the primary",
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS), ids=lambda m: f"m{m}")
def test_pins_catch_planted_mistake(tmp_path, mutant):
    Lm = oracle.load(oracle.build(out=str(tmp_path / f"mut{mutant}.so"), mutant=mutant))
    failures = []
    for check in P.ALL_CHECKS:
        failures += check(Lm)
    assert failures, f"no pin caught mutant {mutant}: {MUTANTS[mutant]}"


def test_odef_matches_oracle_on_fill_and_mixed_ops(L):
    """O-ckpp against the plain dict definition on a few thousand keys."""
    nb = 512
    t = oracle.Table(nb, 8, True, 9)
    d = MapTable(timers=True)
    f = W.fill(9, int(0.93 * nb * 8))
    now = 50
    for lo in range(0, f.keys.shape[0], 700):
        k, v = f.keys[lo:lo + 700], f.values[lo:lo + 700]
        assert (t.insert(k, v, now, 300) == d.insert(k, v, now, 300)).all()
        now += 40
        q = W.lookup_batch(9, 500, f, 0.3, batch_id=lo).keys
        a, b = t.lookup(q, now, 0), d.lookup(q, now, 0)
        assert (a[0] == b[0]).all() and (a[1] == b[1]).all()
        dk = f.keys[lo:lo + 50]
        assert (t.delete(dk, now) == d.delete(dk, now)).all()
        assert t.check() == 0
    dump = t.dump()
    live_t = {bytes(k): int(v) for k, v, e in zip(dump["key"], dump["value"], dump["expiry"])
              if oracle.alive(int(e), now)}
    live_d = {k: v for k, (v, e) in d.live(now).items()}
    assert live_t == live_d


def test_estale_window(L):
    """Sec. 4.2: the table must be scanned at least every 64512 units."""
    t = oracle.Table(4, 8, True, 1)
    k = W.make_keys(1, 40, 2)
    t.insert(k[:1], np.array([1], np.uint64), 100, 10)       # first timed call sets the epoch
    t.lookup(k, 100 + 64512)                                  # exactly at the bound: allowed
    with pytest.raises(oracle.OracleError, match="ESTALE"):
        t.lookup(k, 100 + 64513)
    assert t.expire(100 + 64000) == 1                         # scan deletes the dead entry
    t.lookup(k, 100 + 64000 + 64512)
    with pytest.raises(oracle.OracleError, match="ESTALE"):
        t.insert(k[1:], np.array([2], np.uint64), 100 + 64000 + 64513, 1)


def test_no_timers_ignores_time(L):
    t = oracle.Table(4, 8, False, 1)
    k = W.make_keys(1, 41, 3)
    t.insert(k, np.arange(3, dtype=np.uint64), 0, 0)
    v, f = t.lookup(k, 10**9)
    assert f.all() and (v == np.arange(3)).all()


def test_bad_geometry_rejected(L):
    for nb, s in ((1, 8), (0, 8), (4, 3), (4, 16), (2**32, 8)):
        with pytest.raises(oracle.OracleError):
            oracle.Table(nb, s)


# ---------------------------------------------------- paper statistics

@pytest.fixture(scope="module")
def fill_stats(L):
    """Fill a 2^17 x 8 table step by step and record the statistics the paper
    plots (Fig. 2: fraction in secondary; Fig. 5: moved counters; Table 2: FPR)."""
    nb = 1 << 17
    stats = P.fill_statistics(L, nb, [0.45, 0.6, 0.7, 0.8, 0.95], 7)
    neg = W.make_keys(7, W.STREAM_NEGATIVE_KEYS, 200000)
    # the table holds the 0.95 fill; the negative-lookup counts are taken there
    t = stats[0.95]["table"]
    for lf, s in stats.items():
        assert s["all_inserted"], lf
        s["fpr_closed"] = float((s["hist"] * fill_model.pass_rate(np.arange(len(s["hist"])))).sum())
    sec_reads, _ = t.probe_counts(neg)
    stats[0.95]["fpr_measured"] = sec_reads / neg.shape[0]
    assert t.check() == 0
    for s in stats.values():
        s.pop("table").close()
    return stats


@pytest.fixture(scope="module")
def model():
    return fill_model.fill_model([0.45, 0.6, 0.7, 0.8, 0.95])


def paper_statistics():
    """Rows of tests/golden/paper_statistics.txt: (quantity, LF) -> (paper, lo, hi),
    lo and hi None where the row reads "model"."""
    rows = {}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_statistics.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                q, lf, paper, lo, hi = line.split()
                band = (None, None) if lo == "model" else (float(lo), float(hi))
                rows[(q, float(lf))] = (float(paper),) + band
    return rows


def test_fig2_fraction_in_secondary(fill_stats, model):
    """Sec. 3 / Fig. 2 (8 slots): almost none below LF 0.5, 6% at 0.7, 16% at 0.95.

    Below 0.5 and at 0.95 the oracle sits in a band around the paper's value.
    At 0.7 the paper's 6% is beyond the insertion rule of Sec. 2 with a uniform
    hash: the rule's fluid limit, which is exact at this load factor, gives
    4.38%. The oracle must equal the model there, and the paper's value must be
    above both: the gap belongs to the rule, not to this oracle."""
    rows = {lf: v for (q, lf), v in paper_statistics().items() if q == "secondary_fraction"}
    assert sorted(rows) == [0.45, 0.7, 0.95]
    for lf, (paper, lo, hi) in rows.items():
        got = fill_stats[lf]["f_sec"]
        if lo is None:
            assert abs(got - model[lf]["f_sec"]) < 0.0015, (lf, got, model[lf]["f_sec"])
            assert model[lf]["f_sec"] < paper - 0.01
        else:
            assert lo <= got < hi, (lf, got)


def test_fill_matches_rule_model(fill_stats, model):
    """The whole fill against the fluid limit of the insertion rule (Sec. 2) and
    the counter rule (Sec. 4.1). Exact while keys with both buckets full are
    rare (LF <= 0.8); at 0.95 a cuckoo path can displace more than one entry,
    which only raises the secondary share and lowers the zero-counter share."""
    for lf in (0.45, 0.6, 0.7, 0.8):
        assert abs(fill_stats[lf]["f_sec"] - model[lf]["f_sec"]) < 0.0015, lf
        assert abs(fill_stats[lf]["moved_zero"] - model[lf]["moved_zero"]) < 0.004, lf
    g, m = fill_stats[0.95], model[0.95]
    assert m["f_sec"] - 0.001 < g["f_sec"] < m["f_sec"] + 0.015, (g["f_sec"], m["f_sec"])
    assert m["moved_zero"] - 0.03 < g["moved_zero"] < m["moved_zero"] + 0.002, (g["moved_zero"], m["moved_zero"])


def test_table2_bloom_false_positive_rate(fill_stats, model):
    """Table 2: FPR 0.0002 / 0.001 / 0.003 at LF 0.6 / 0.8 / 0.95, within x1.6 of
    the paper; and within 8% of the rate the model's counter histogram gives
    (exact bit-collision formula, ``fill_model.pass_rate``), 15% at 0.95 where
    the model undercounts displaced keys."""
    rows = {lf: v for (q, lf), v in paper_statistics().items() if q == "bloom_fpr"}
    assert sorted(rows) == [0.6, 0.8, 0.95]
    for lf, (paper, lo, hi) in rows.items():
        assert abs(lo - paper / 1.6) < 1e-9 and abs(hi - paper * 1.6) < 1e-9
        got = fill_stats[lf]["fpr_exact"]
        assert lo < got < hi, (lf, got)
        assert lo < model[lf]["fpr"] < hi, (lf, model[lf]["fpr"])
        rel = 0.15 if lf > 0.9 else 0.08
        assert abs(got / model[lf]["fpr"] - 1) < rel, (lf, got, model[lf]["fpr"])


def test_fpr_closed_form_and_measured_pass_rate(fill_stats):
    """The negative-lookup filter pass rate equals mean((popcount/64)^2) (two
    independent uniform bit indices), and that equals the rate the counter
    histogram gives through the bit-collision formula."""
    for lf, s in fill_stats.items():
        exp = s["fpr_exact"]
        assert abs(s["fpr_closed"] - exp) <= 0.05 * exp + 1e-6, (lf, s["fpr_closed"], exp)
    s = fill_stats[0.95]
    sd = (s["fpr_exact"] / 200000) ** 0.5
    assert abs(s["fpr_measured"] - s["fpr_exact"]) < 4.5 * sd + 1e-6


def test_fig5_moved_counter_zero(fill_stats, model):
    """Sec. 4.1 / Fig. 5: the paper says more than 50% of buckets have a zero
    moved counter at LF 0.95. The rule's fluid limit gives 48.7% (one counter
    step per key whose primary is full), and cuckoo paths that displace more
    than one entry only lower it, so the printed value is beyond the rule with
    a uniform hash. The oracle must sit between the model less 3 points and
    the model, and the share must fall as the table fills."""
    paper, lo, hi = paper_statistics()[("moved_zero_fraction", 0.95)]
    assert lo is None and model[0.95]["moved_zero"] < paper
    got = fill_stats[0.95]["moved_zero"]
    assert model[0.95]["moved_zero"] - 0.03 < got < model[0.95]["moved_zero"] + 0.002, got
    zs = [fill_stats[lf]["moved_zero"] for lf in (0.45, 0.6, 0.7, 0.8, 0.95)]
    assert zs == sorted(zs, reverse=True)
