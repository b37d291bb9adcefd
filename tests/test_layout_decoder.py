"""The host-side decoder of the GPU layout and its read-count replay, checked
against the oracle on the CPU (an oracle table written out in the GPU byte
layout must decode to the same entries and the same lookup read counts)."""

import numpy as np

import oracle
from gpu_layout import Decoded, encode_oracle, expected_probe_counts, oracle_live
from paper_1712_09624_gb300 import workload as W


def test_decoder_round_trip_and_read_counts():
    for timers in (False, True):
        nb, seed = 2000, 91 + timers
        f = W.fill(seed, int(0.93 * nb * 8))
        o = oracle.Table(nb, 8, timers, seed)
        o.insert(f.keys, f.values, 5, 800 if timers else 0)
        d = Decoded(encode_oracle(o), nb, timers, seed)
        assert d.check() == []
        assert d.live(20) == oracle_live(o, 20)
        q = W.lookup_batch(seed, 20000, f, 0.5)
        n, sec, rec, l1 = expected_probe_counts(d, q.keys, 0, 20)
        assert n == q.keys.shape[0] and (sec, rec) == o.probe_counts(q.keys, 20)
        _, sec_opt, rec_opt, l1_opt = expected_probe_counts(d, q.keys, 1, 20)
        _, sec_pes, rec_pes, l1_pes = expected_probe_counts(d, q.keys, 2, 20)
        assert sec < sec_opt < sec_pes == n
        assert rec <= rec_opt == rec_pes
        assert l1 <= l1_opt == l1_pes
        # a second line is read only for a tag match among the second line's slots
        assert 0 < l1 < n


def test_decoder_flags_a_broken_filter():
    """A displaced key whose bits are cleared from its primary's filter is
    reported, and the replayed Bloom lookup then skips its secondary."""
    nb, seed = 500, 93
    f = W.fill(seed, int(0.95 * nb * 8))
    o = oracle.Table(nb, 8, False, seed)
    o.insert(f.keys, f.values)
    d = Decoded(encode_oracle(o), nb, False, seed)
    b = int(np.nonzero(d.moved)[0][0])
    d.bloom[b] = np.uint64(0)
    assert "a displaced key's bits are missing from its primary's filter" in d.check()
