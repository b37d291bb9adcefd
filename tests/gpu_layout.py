"""Host-side decoder of the GPU table layout, for checking a downloaded table.

Test code: it reads the bytes of a table buffer (the layout documented in
include/ckpp.h and the CUDA sources) into numpy arrays and checks them with the
oracle's hash (``oracle.address``), so the structural invariants of Sec. 2 and
Sec. 4.1 are verified on what the kernels actually wrote.
"""

from __future__ import annotations

import numpy as np

import oracle

HEADER = 256
SLOTS = 8
BUCKET = 256


def first_hi_slot(timers: bool) -> int:
    """The first slot whose entry lives in the bucket's second line."""
    return 3 if timers else 4


EXPIRY_OFF = 32  # timers: expiry[8] in line 0, right after the 32-byte header


def key_offsets(timers: bool) -> np.ndarray:
    """Byte offset of each slot's key in a bucket: the first slots in line 0
    after the 32-byte header (and, with timers, the 16 bytes of expiries), the
    others from the start of line 1."""
    h = first_hi_slot(timers)
    s = np.arange(SLOTS)
    first = 48 if timers else 32
    return np.where(s < h, first + 16 * s, 128 + 16 * (s - h))


def value_offsets(timers: bool) -> np.ndarray:
    """Byte offset of each slot's value: the first line's values from byte 96
    (after keys 0-3, or after the expiries and keys 0-2 with timers), the second
    line's after its keys."""
    s = np.arange(SLOTS)
    if timers:
        return np.where(s < 3, 96 + 8 * s, 208 + 8 * (s - 3))
    return np.where(s < 4, 96 + 8 * s, 192 + 8 * (s - 4))


def reserved_ranges(timers: bool) -> list[tuple[int, int]]:
    return [(120, 128), (248, 256)] if timers else [(224, 256)]


class Decoded:
    def __init__(self, buf: np.ndarray, n_buckets: int, timers: bool, seed: int):
        self.nb, self.timers, self.seed = n_buckets, timers, seed
        hdr = buf[:HEADER]
        self.magic = int(hdr[0:4].view(np.uint32)[0])
        self.abi = int(hdr[4:8].view(np.uint32)[0])
        self.err = int(hdr[32:36].view(np.uint32)[0])
        bk = buf[HEADER:HEADER + n_buckets * BUCKET].reshape(n_buckets, BUCKET)
        self.tags = np.ascontiguousarray(bk[:, 0:16]).view(np.uint16).reshape(n_buckets, 8)
        self.bloom = np.ascontiguousarray(bk[:, 16:24]).view(np.uint64).reshape(n_buckets)
        self.ctrl = np.ascontiguousarray(bk[:, 24:28]).view(np.uint32).reshape(n_buckets)
        self.moved = np.ascontiguousarray(bk[:, 28:32]).view(np.uint32).reshape(n_buckets)
        if timers:
            self.expiry = np.ascontiguousarray(bk[:, EXPIRY_OFF:EXPIRY_OFF + 16]).view(np.uint16).reshape(n_buckets, 8)
        else:
            self.expiry = np.zeros((n_buckets, 8), np.uint16)
        self.bucket_reserved = np.concatenate([bk[:, a:b] for a, b in reserved_ranges(timers)], axis=1)
        ko = key_offsets(timers)
        keys = np.stack([bk[:, o:o + 16] for o in ko], axis=1)  # [nb, 8, 16]
        self.rec_key = np.ascontiguousarray(keys.reshape(n_buckets * SLOTS, 16))
        vo = value_offsets(timers)
        vals = np.stack([np.ascontiguousarray(bk[:, o:o + 8]).view(np.uint64).reshape(-1) for o in vo], axis=1)
        self.rec_value = np.ascontiguousarray(vals.reshape(-1))
        bits = np.arange(8, dtype=np.uint32)
        self.busy = ((self.ctrl[:, None] >> bits) & 1).astype(bool)
        self.insec = ((self.ctrl[:, None] >> (bits + 8)) & 1).astype(bool)

    def occupied(self):
        """Flat slot indices (bucket * 8 + slot) of busy slots."""
        return np.nonzero(self.busy.reshape(-1))[0]

    def alive(self, now: int) -> np.ndarray:
        if not self.timers:
            return np.ones((self.nb, 8), bool)
        d = (self.expiry.astype(np.int64) - (now & 0xFFFF)) & 0xFFFF
        return d < 1024

    def live(self, now: int) -> dict:
        """key bytes -> (value, expiry) of every live entry."""
        idx = np.nonzero((self.busy & self.alive(now)).reshape(-1))[0]
        exp = self.expiry.reshape(-1)
        return {self.rec_key[i].tobytes(): (int(self.rec_value[i]), int(exp[i]) if self.timers else 0) for i in idx}

    def check(self, check_reset: bool = True, bucket_sample: np.ndarray | None = None) -> list[str]:
        """Structural invariants; returns failure messages (empty = all hold)."""
        bad = []
        if self.magic != 0x50504B43:
            bad.append("bad magic")
        if (self.ctrl & 0x7FFF0000).any() or (self.ctrl & 0x80000000).any():
            bad.append("lock bit, claimed bits or unused ctrl bits set")
        if (self.insec & ~self.busy).any():
            bad.append("in_secondary set on an empty slot")
        occ = self.occupied()
        if bucket_sample is not None:
            sel = np.isin(occ // SLOTS, bucket_sample)
            occ = occ[sel]
        keys = self.rec_key[occ]
        a = oracle.address(keys, self.nb, self.seed)
        b = occ // SLOTS
        s = occ % SLOTS
        if not ((b == a["b1"]) | (b == a["b2"])).all():
            bad.append("an entry sits in neither of its buckets")
        insec = self.insec[b, s]
        if not (insec == (b == a["b2"])).all():
            bad.append("in_secondary flag disagrees with the bucket")
        if not (self.tags[b, s] == a["tag"]).all():
            bad.append("stored tag differs from the key's tag")
        if self.bucket_reserved.any():
            bad.append("reserved bucket bytes not zero")
        bits = (np.uint64(1) << a["bit1"].astype(np.uint64)) | (np.uint64(1) << a["bit2"].astype(np.uint64))
        p = a["b1"][insec]
        if not ((self.bloom[p] & bits[insec]) == bits[insec]).all():
            bad.append("a displaced key's bits are missing from its primary's filter")
        if bucket_sample is None:
            cnt = np.bincount(p.astype(np.int64), minlength=self.nb)
            if not (cnt == self.moved).all():
                bad.append("moved counter differs from the number of displaced keys")
            kv = np.ascontiguousarray(keys).view(np.dtype((np.void, 16))).reshape(-1)
            if np.unique(kv).shape[0] != kv.shape[0]:
                bad.append("a key is stored twice")
            if check_reset and ((self.moved == 0) & (self.bloom != 0)).any():
                bad.append("zero moved counter with a non-empty filter")
        return bad


def download(table) -> Decoded:
    import torch
    torch.cuda.synchronize()
    return Decoded(table.buf.cpu().numpy(), table.n_buckets, table.timers, table.seed)


def oracle_live(t: "oracle.Table", now: int) -> dict:
    d = t.dump()
    out = {}
    for i in range(d["value"].shape[0]):
        e = int(d["expiry"][i])
        if (not t.timers) or ((e - now) & 0xFFFF) < 1024:
            out[d["key"][i].tobytes()] = (int(d["value"][i]), e if t.timers else 0)
    return out


def expected_probe_counts(d: Decoded, keys: np.ndarray, variant: int,
                          now: int = 0) -> tuple[int, int, int, int]:
    # `now` does not change the counts: a key met in a dead entry ends the
    # search like a live one (Sec. 4.2), and no read depends on liveness.
    """(keys, secondary-bucket reads, record reads, second-line reads) that a
    lookup of ``keys`` with strategy ``variant`` (0 Bloom, 1 optimistic,
    2 pessimistic) makes on the decoded table: candidates are busy slots whose
    tag matches, confirmed in slot order until the key is met (Sec. 2); the
    secondary is read after a primary miss when both filter bits are set
    (Bloom, Sec. 4.1), after every primary miss (optimistic) or always
    (pessimistic, Sec. 3). A bucket's second line is read when the key is not
    among the first line's slots and a tag of the second line's slots matches;
    a pessimistic read of the secondary after a primary hit reads its first
    line only."""
    a = oracle.address(keys, d.nb, d.seed)
    kv = np.ascontiguousarray(keys).view(np.dtype((np.void, 16))).reshape(-1)
    rk = np.ascontiguousarray(d.rec_key).view(np.dtype((np.void, 16))).reshape(-1)
    slots = np.arange(SLOTS)

    def bucket_reads(b):
        cand = (d.tags[b] == a["tag"][:, None]) & d.busy[b]
        hit = cand & (rk[(b[:, None] * SLOTS + slots).reshape(-1)].reshape(-1, SLOTS) == kv[:, None])
        found = hit.any(axis=1)
        first = np.where(found, hit.argmax(axis=1), SLOTS)
        upto = cand & (slots[None, :] <= first[:, None])
        h = first_hi_slot(d.timers)
        line1 = ~(found & (first < h)) & cand[:, h:].any(axis=1)
        return found, upto.sum(axis=1), line1

    f1, r1, l1 = bucket_reads(a["b1"].astype(np.int64))
    _, r2, l2 = bucket_reads(a["b2"].astype(np.int64))
    bits = (np.uint64(1) << a["bit1"].astype(np.uint64)) | (np.uint64(1) << a["bit2"].astype(np.uint64))
    if variant == 0:
        read2 = ~f1 & ((d.bloom[a["b1"]] & bits) == bits)
        sec = int(read2.sum())
    elif variant == 1:
        read2 = ~f1
        sec = int(read2.sum())
    else:
        read2 = ~f1
        sec = keys.shape[0]
    rec = int(r1.sum() + r2[read2].sum())
    line1 = int(l1.sum() + l2[read2].sum())
    return keys.shape[0], sec, rec, line1


def encode_oracle(t: "oracle.Table") -> np.ndarray:
    """The oracle table's entries written out in the GPU byte layout (header,
    then 256-byte buckets), so the decoder and the helpers above can be checked
    on the CPU against the oracle's own answers."""
    nb, timers = t.n_buckets, t.timers
    buf = np.zeros(HEADER + nb * BUCKET, np.uint8)
    buf[0:4] = np.frombuffer(np.uint32(0x50504B43).tobytes(), np.uint8)
    buf[4:8] = np.frombuffer(np.uint32(2).tobytes(), np.uint8)
    d = t.dump()
    bloom, moved = t.meta()
    bk = buf[HEADER:].reshape(nb, BUCKET)
    bk[:, 16:24] = bloom.view(np.uint8).reshape(nb, 8)
    bk[:, 28:32] = moved.view(np.uint8).reshape(nb, 4)
    ctrl = np.zeros(nb, np.uint32)
    a = oracle.address(d["key"], nb, t.seed)
    ko, vo = key_offsets(timers), value_offsets(timers)
    for i in range(d["value"].shape[0]):
        b, s = int(d["bucket"][i]), int(d["slot"][i])
        ctrl[b] |= np.uint32(1 << s) | np.uint32(int(d["in_secondary"][i]) << (8 + s))
        bk[b, 2 * s:2 * s + 2] = np.frombuffer(np.uint16(a["tag"][i]).tobytes(), np.uint8)
        bk[b, ko[s]:ko[s] + 16] = d["key"][i]
        bk[b, vo[s]:vo[s] + 8] = np.frombuffer(np.uint64(d["value"][i]).tobytes(), np.uint8)
        if timers:
            e = np.uint16(d["expiry"][i]).tobytes()
            bk[b, EXPIRY_OFF + 2 * s:EXPIRY_OFF + 2 * s + 2] = np.frombuffer(e, np.uint8)
    bk[:, 24:28] = ctrl.view(np.uint8).reshape(nb, 4)
    return buf
