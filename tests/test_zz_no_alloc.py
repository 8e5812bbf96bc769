"""fgs_sort_pairs_static: the radix sort for callers that cannot allocate.

Callers such as a framework that owns every device allocation through its
own memory pool, or latency-critical code that cannot pay for the
synchronisation cudaMalloc implies, cannot hand the sort a scratch buffer.
This entry point sorts in place using a fixed array the library owns.  The
test checks it against the allocating fgs_sort_pairs, key for key and value
for value, on two calls in a row (the second call reuses the array the first
one left behind), and that an oversized request is refused.  It lives in a
file of its own that pytest collects last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_09999_gb300 import binding as B  # noqa: E402


def _keys(n, bits, seed):
    rng = np.random.default_rng(seed)
    hi = rng.integers(0, 1 << (bits - 32), n, dtype=np.uint64)
    lo = rng.integers(0, 1 << 32, n, dtype=np.uint64)
    keys = (hi << np.uint64(32)) | lo
    keys[::5] = keys[1]  # many equal keys: stability matters
    return keys


def _allocating_sort(keys, vals, bits):
    n = keys.size
    k = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    v = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    k2, v2 = torch.empty_like(k), torch.empty_like(v)
    nb = B.fgs_sort_scratch_bytes(n)
    scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
    alt = B.fgs_sort_pairs(k.data_ptr(), v.data_ptr(), k2.data_ptr(), v2.data_ptr(), n, bits,
                           scratch.data_ptr(), nb, torch.cuda.current_stream().cuda_stream)
    return (k2, v2) if alt else (k, v)


def test_static_sort_matches_allocating_sort_twice():
    stream = torch.cuda.current_stream().cuda_stream
    # 44 bits: 6 passes (result in the first buffer pair); 40 bits: 5 passes
    # (result copied back from the library's array); the second call is the
    # largest size the array holds.
    for call, (n, bits, seed) in enumerate([(300_001, 44, 1), (B.FGS_STATIC_SORT_MAX_PAIRS, 40, 2)]):
        keys = _keys(n, bits, seed)
        vals = np.arange(n, dtype=np.uint32)[::-1].copy()
        ref_k, ref_v = _allocating_sort(keys, vals, bits)
        k = torch.from_numpy(keys.view(np.int64).copy()).cuda()
        v = torch.from_numpy(vals.view(np.int32).copy()).cuda()
        B.fgs_sort_pairs_static(k.data_ptr(), v.data_ptr(), n, bits, stream)
        torch.cuda.synchronize()
        assert torch.equal(k, ref_k), call
        assert torch.equal(v, ref_v), call
        order = np.argsort(keys & np.uint64((1 << bits) - 1), kind="stable")
        np.testing.assert_array_equal(v.cpu().numpy().view(np.uint32), vals[order])


def test_static_sort_refuses_more_than_it_holds():
    k = torch.zeros(1, dtype=torch.int64, device="cuda")
    v = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(B.FGSError) as e:
        B.fgs_sort_pairs_static(k.data_ptr(), v.data_ptr(), B.FGS_STATIC_SORT_MAX_PAIRS + 1, 40,
                                torch.cuda.current_stream().cuda_stream)
    assert e.value.code == -10
