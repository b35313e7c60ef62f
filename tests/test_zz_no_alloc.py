"""The sort entry point that allocates no device memory, checked against the
allocating one (rg_radix_sort_pairs) through the C ABI.

Some callers cannot allocate device memory while they sort -- code whose
device memory belongs to a caching allocator that already holds what the
GPU has free, frame loops that may not stall on an allocation -- so librg
offers a variant whose temporaries live in a fixed device array.  Integer work: results must be
identical.  Two calls in a row, with different data, show that whatever the
first call leaves in the shared array does not leak into the second."""
import numpy as np
import pytest
import torch

import paper_2001_09792_gb300 as rg

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("librg")]


def keys_for(n, key_bits, seed):
    rng = np.random.default_rng(seed)
    if key_bits == 32:
        k = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
        k[: n // 3] = rng.integers(0, 50, size=n // 3).astype(np.uint32)  # duplicates: stability matters
        return torch.from_numpy(k.view(np.int32)).cuda()
    k = rng.integers(0, 2 ** 63, size=n, dtype=np.uint64) | (rng.integers(0, 2, size=n, dtype=np.uint64) << np.uint64(63))
    k[: n // 3] = rng.integers(0, 50, size=n // 3).astype(np.uint64)
    return torch.from_numpy(k.view(np.int64)).cuda()


@pytest.mark.parametrize("key_bits", [32, 64])
def test_noalloc_sort_matches_allocating_sort_on_two_calls(key_bits):
    for call, n in enumerate([rg.RG_NOALLOC_SORT_MAX_PAIRS, 100_003]):
        keys = keys_for(n, key_bits, seed=10 * call + key_bits)
        vals = torch.randperm(n, device="cuda").to(torch.int32)
        want_k, want_v = rg.rg_radix_sort_pairs(keys, vals)
        got_k, got_v = rg.rg_radix_sort_pairs_noalloc(keys, vals)
        torch.cuda.synchronize()
        assert torch.equal(got_k, want_k) and torch.equal(got_v, want_v), f"call {call}"


def test_noalloc_sort_rejects_more_than_the_fixed_array_holds():
    n = rg.RG_NOALLOC_SORT_MAX_PAIRS + 1
    keys = torch.zeros(n, dtype=torch.int32, device="cuda")
    vals = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(rg.RgError) as e:
        rg.rg_radix_sort_pairs_noalloc(keys, vals)
    assert e.value.status == rg.RG_ERR_INVALID_ARG
    assert "RG_NOALLOC_SORT_MAX_PAIRS" in str(e.value)
