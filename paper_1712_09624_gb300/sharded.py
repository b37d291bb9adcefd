"""A flow table split over several GPUs by hash (one shard per rank).

The paper gives every core a private table (Sec. 2 and Sec. 5.3). The same
share-nothing tables can serve one logical table when the keys are
partitioned by hash: rank r owns the keys whose shard is r (the shard is bits
16-31 of the primary hash, see ``ckpp_shard_partition`` in include/ckpp.h), in
an ordinary table of its own. A bulk call that every rank makes together with
its own batch goes:

1. partition the batch by owner (stable: each owner's keys stay in batch
   order);
2. all-to-all of the per-owner key counts, then of the keys (and values);
3. each owner runs its ordinary bulk call on the keys it received, ordered by
   source rank, then batch index;
4. all-to-all of the results back (the reverse splits);
5. the results land in the caller's order.

The owner sees the ranks' batches concatenated in rank order, so the call has
the result of one batch made of rank 0's keys, then rank 1's, and so on (for
insert and delete: duplicate keys resolve in that order, Sec. 2). The only
collectives are the two all-to-alls (plus the count exchange); there is no
other communication.

``ShardRouter`` is the exchange itself and works on any tensors
``torch.distributed`` can move (gloo on CPU in the tests, NCCL on GPUs). The
partition and the local table are supplied by the caller: on GPUs,
``DevicePartitioner`` (the library's partition kernels) and a ``FlowTable``,
combined in ``ShardedTable``.
"""

from __future__ import annotations

from dataclasses import dataclass

import torch
import torch.distributed as dist


@dataclass
class Routed:
    """One batch after the exchange: what the owner received, and what the
    way back needs."""
    keys: torch.Tensor          # [m, 16] keys this rank owns, by source rank then batch index
    vals: torch.Tensor | None   # [m] values with them (inserts)
    order: torch.Tensor         # [n] the partition's record of the caller's batch, for the way back
    send_counts: list           # keys sent to each rank
    recv_counts: list           # keys received from each rank


class ShardRouter:
    """The two all-to-alls of a sharded bulk call (module doc). partitioner:
    ``partition(keys, vals, n_shards) -> (order, keys_sorted, vals_sorted,
    counts)`` and ``unpermute(order, sorted_results) -> results`` (a list of
    1-D tensors, each in the caller's order); ``order`` is whatever record of
    the permutation the partitioner hands back to its own unpermute."""

    def __init__(self, partitioner, group=None):
        self.part = partitioner
        self.group = group
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0

    def _a2a(self, out: torch.Tensor, inp: torch.Tensor, out_splits: list, in_splits: list):
        if self.world == 1:
            out.copy_(inp)
        else:
            dist.all_to_all_single(out, inp, out_splits, in_splits, group=self.group)

    def send(self, keys: torch.Tensor, vals: torch.Tensor | None = None) -> Routed:
        order, keys_s, vals_s, counts = self.part.partition(keys, vals, self.world)
        counts = counts.to(torch.int64)
        recv = torch.empty_like(counts)
        self._a2a(recv, counts, [1] * self.world, [1] * self.world)
        send_counts = [int(c) for c in counts.tolist()]
        recv_counts = [int(c) for c in recv.tolist()]
        m = sum(recv_counts)
        rk = torch.empty((m, 16), dtype=torch.uint8, device=keys.device)
        self._a2a(rk, keys_s, recv_counts, send_counts)
        rv = None
        if vals is not None:
            rv = torch.empty(m, dtype=vals.dtype, device=vals.device)
            self._a2a(rv, vals_s, recv_counts, send_counts)
        return Routed(rk, rv, order, send_counts, recv_counts)

    def back(self, routed: Routed, results: list) -> list:
        """results: 1-D tensors of the owner's results for routed.keys; returns
        them for the caller's own batch, in its order."""
        n = sum(routed.send_counts)
        sorted_back = []
        for r in results:
            out = torch.empty(n, dtype=r.dtype, device=r.device)
            self._a2a(out, r, routed.send_counts, routed.recv_counts)
            sorted_back.append(out)
        return self.part.unpermute(routed.order, sorted_back)


class DevicePartitioner:
    """Partition and unpermute with the library's kernels
    (``ckpp_shard_partition``, ``ckpp_shard_unpermute``)."""

    def __init__(self, seed: int, stream=None):
        from . import _ckpp
        self.K = _ckpp
        self.seed, self.stream = seed, stream
        self._ws = None

    def partition(self, keys: torch.Tensor, vals: torch.Tensor | None, n_shards: int):
        K = self.K
        n, dev = keys.shape[0], keys.device
        need = K.ckpp_shard_workspace_bytes(n, n_shards)
        if need == 0:
            raise ValueError(f"cannot partition {n} keys into {n_shards} shards")
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=dev)
        pos = torch.empty(n, dtype=torch.int32, device=dev)  # each key's sorted position
        keys_s = torch.empty((n, 16), dtype=torch.uint8, device=dev)
        vals_s = None if vals is None else torch.empty(n, dtype=vals.dtype, device=dev)
        counts = torch.empty(n_shards, dtype=torch.int64, device=dev)
        K.ckpp_shard_partition(keys, vals, self.seed, n_shards, pos, keys_s, vals_s, counts, self._ws, self.stream)
        return pos, keys_s, vals_s, counts

    def unpermute(self, pos: torch.Tensor, sorted_results: list) -> list:
        K = self.K
        out = []
        for r in sorted_results:
            o = torch.empty_like(r)
            if r.element_size() == 8:
                K.ckpp_shard_unpermute(pos, r, None, o, None, self.stream)
            elif r.element_size() == 1:
                K.ckpp_shard_unpermute(pos, None, r, None, o, self.stream)
            else:
                raise TypeError(f"results of {r.element_size()}-byte elements cannot be unpermuted")
            out.append(o)
        return out


class ShardedTable:
    """This rank's shard of a table split over the ranks of ``group``, on its
    current GPU. Every rank must make each call, with its own batch (possibly
    empty); calls return the results of the caller's keys in its order."""

    def __init__(self, n_buckets_per_shard: int, timers: bool = False, seed: int = 0, group=None, device=None,
                 stream=None):
        from .table import FlowTable
        self.local = FlowTable(n_buckets_per_shard, timers=timers, seed=seed, device=device, stream=stream)
        self.router = ShardRouter(DevicePartitioner(seed, stream), group)
        self.stream = stream

    def lookup(self, keys: torch.Tensor, now: int = 0, refresh_ttl: int = 0):
        r = self.router.send(keys)
        vals, found = self.local.lookup(r.keys, now, refresh_ttl, self.stream)
        v, f = self.router.back(r, [vals, found.to(torch.uint8)])
        return v, f.to(torch.bool)

    def insert(self, keys: torch.Tensor, vals: torch.Tensor, now: int = 0, ttl: int = 0) -> torch.Tensor:
        r = self.router.send(keys, vals)
        return self.router.back(r, [self.local.insert(r.keys, r.vals, now, ttl, self.stream)])[0]

    def delete(self, keys: torch.Tensor, now: int = 0) -> torch.Tensor:
        r = self.router.send(keys)
        return self.router.back(r, [self.local.delete(r.keys, now, self.stream)])[0]
