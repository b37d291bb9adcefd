"""Seeded synthetic 5-tuple flow traffic.

This module only draws inputs; it holds none of the table's arithmetic, so the
CUDA path and the CPU oracle can both be fed from it.

Random numbers come from the Philox4x64-10 counter-based generator (Salmon et
al., SC'11) through numpy's ``Philox`` bit generator, whose raw 64-bit output
stream for a given 128-bit key is fixed by that algorithm. Every draw uses a
distinct key ``(seed, stream)``, so each quantity is reproducible on its own.

Key layout (16 bytes, little endian): src_ip u32 | dst_ip u32 | src_port u16 |
dst_port u16 | proto u8 in {6, 17} | 3 zero pad bytes. The paper draws random
keys (Sec. 5, common parameters); IPs and ports are uniform here, the protocol
is TCP or UDP with equal odds.
"""

from __future__ import annotations

import sys
from dataclasses import dataclass

import numpy as np

assert sys.byteorder == "little", "keys are laid out little endian"

# stream identifiers (second word of the Philox key)
STREAM_INSERT_KEYS = 1
STREAM_NEGATIVE_KEYS = 2
STREAM_NEG_MASK = 3
STREAM_POS_PICK = 4
STREAM_VALUES = 5
STREAM_MISC = 6


def raw64(seed: int, stream: int, n: int) -> np.ndarray:
    """The first n raw 64-bit outputs of Philox4x64-10 keyed by (seed, stream)."""
    bg = np.random.Philox(key=np.array([seed & (2**64 - 1), stream & (2**64 - 1)], dtype=np.uint64))
    return np.asarray(bg.random_raw(n), dtype=np.uint64)


def make_keys(seed: int, stream: int, n: int) -> np.ndarray:
    """n random 5-tuple keys as a uint8 [n, 16] array."""
    r = raw64(seed, stream, 2 * n).reshape(n, 2) if n else np.zeros((0, 2), np.uint64)
    words = np.empty((n, 2), np.uint64)
    words[:, 0] = r[:, 0]  # src_ip | dst_ip << 32
    proto = np.where((r[:, 1] >> np.uint64(32)) & np.uint64(1), np.uint64(17), np.uint64(6))
    words[:, 1] = (r[:, 1] & np.uint64(0xFFFFFFFF)) | (proto << np.uint64(32))
    return words.view(np.uint8).reshape(n, 16)


def uniform_index(r: np.ndarray, n: int) -> np.ndarray:
    """Map raw 64-bit draws to [0, n) by multiply-high on their top 32 bits."""
    return ((r >> np.uint64(32)) * np.uint64(n)) >> np.uint64(32)


@dataclass
class LookupBatch:
    keys: np.ndarray          # uint8 [n, 16]
    expect_found: np.ndarray  # uint8 [n]
    expect_value: np.ndarray  # uint64 [n] (0 where not found)


@dataclass
class FillWorkload:
    keys: np.ndarray    # uint8 [m, 16], inserted in index order
    values: np.ndarray  # uint64 [m], value = insertion index


def fill(seed: int, n_keys: int) -> FillWorkload:
    """Keys to insert, value = index (the table is filled in index order)."""
    return FillWorkload(make_keys(seed, STREAM_INSERT_KEYS, n_keys), np.arange(n_keys, dtype=np.uint64))


def lookup_batch(seed: int, n: int, inserted: FillWorkload, neg_rate: float, batch_id: int = 0) -> LookupBatch:
    """A lookup batch: each key is negative with probability neg_rate (Bernoulli,
    so the count and positions vary as in the paper's Sec. 5); positives are drawn
    uniformly with replacement from the inserted keys, negatives are fresh keys."""
    sub = (seed << 20) ^ batch_id
    m = inserted.keys.shape[0]
    u = raw64(sub, STREAM_NEG_MASK, n)
    neg = (u >> np.uint64(11)).astype(np.float64) * (1.0 / 2**53) < neg_rate if m else np.ones(n, bool)
    pick = uniform_index(raw64(sub, STREAM_POS_PICK, n), max(m, 1))
    fresh = make_keys(sub, STREAM_NEGATIVE_KEYS, n)
    keys = np.where(neg[:, None], fresh, inserted.keys[pick] if m else fresh)
    found = (~neg).astype(np.uint8)
    value = np.where(neg, np.uint64(0), inserted.values[pick] if m else np.uint64(0)).astype(np.uint64)
    return LookupBatch(np.ascontiguousarray(keys), found, value)
