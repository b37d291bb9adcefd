"""The device-side traffic generator draws exactly what workload.py draws."""

import numpy as np
import pytest

from paper_1712_09624_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,first,n", [(1, 0, 1), (1, 0, 1001), (7, 3, 4097), (2**40 + 5, 12345, 777)])
def test_fill_keys_match_host(seed, first, n):
    from paper_1712_09624_gb300 import workload_gpu as WG
    k, v = WG.fill_keys(seed, first, n, "cuda")
    ref = W.fill(seed, first + n)
    assert (k.cpu().numpy() == ref.keys[first:]).all()
    assert (v.cpu().numpy().view(np.uint64) == ref.values[first:]).all()


@pytest.mark.parametrize("seed,n,m,neg,bid", [(1, 5000, 3000, 0.5, 0), (3, 4097, 100, 0.3, 7), (4, 999, 0, 0.2, 1),
                                             (5, 2048, 70000, 0.0, 2), (6, 2048, 70000, 1.0, 3)])
def test_lookup_batch_matches_host(seed, n, m, neg, bid):
    from paper_1712_09624_gb300 import workload_gpu as WG
    k, f, v = WG.lookup_batch(seed, n, m, neg, bid, device="cuda")
    ref = W.lookup_batch(seed, n, W.fill(seed, m), neg, batch_id=bid)
    assert (k.cpu().numpy() == ref.keys).all()
    assert (f.cpu().numpy() == ref.expect_found).all()
    assert (v.cpu().numpy().view(np.uint64) == ref.expect_value).all()


def test_keys_at_match_host():
    import torch
    from paper_1712_09624_gb300 import workload_gpu as WG
    idx = np.array([0, 5, 3, 1000, 77, 77, 2], np.int64)
    k = WG.keys_at(9, torch.from_numpy(idx).cuda())
    ref = W.fill(9, 1001).keys[idx]
    assert (k.cpu().numpy() == ref).all()


@pytest.mark.parametrize("n,host,offset", [(1, True, 0), (4099, True, 0), (4096, False, 0), (1000, True, 1)])
def test_host_io_probe_outputs(n, host, offset):
    """The host-link probe writes k0 ^ (k1 << 1) and k1 & 1 for every key,
    through the vector path (aligned outputs) and the per-lane path (outputs
    offset by one element, and the ragged last warp)."""
    import torch
    from paper_1712_09624_gb300 import workload_gpu as WG
    keys_np = W.make_keys(31, 5, n)
    words = keys_np.view(np.uint64).reshape(n, 2)
    want_v = words[:, 0] ^ (words[:, 1] << np.uint64(1))
    want_f = (words[:, 1] & np.uint64(1)).astype(np.uint8)
    keys = torch.from_numpy(keys_np)
    vals = torch.zeros(n + offset, dtype=torch.int64)
    found = torch.full((n + offset,), 7, dtype=torch.uint8)
    if host:
        keys, vals, found = keys.pin_memory(), vals.pin_memory(), found.pin_memory()
    else:
        keys, vals, found = keys.cuda(), vals.cuda(), found.cuda()
    WG.host_io(keys, vals[offset:], found[offset:])
    torch.cuda.synchronize()
    assert (vals[offset:].cpu().numpy().view(np.uint64) == want_v).all()
    assert (found[offset:].cpu().numpy() == want_f).all()
