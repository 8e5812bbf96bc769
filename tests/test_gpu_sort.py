"""Radix sort (fgs_sort_pairs) against numpy's stable sort: bit-exact keys
and values on seeded keys, across sizes that span several CTA tiles, a
ragged tail, the empty case and every bit width class."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_09999_gb300 import binding as B  # noqa: E402


def _sort_gpu(keys, vals, bits):
    n = keys.size
    # at least one element so that the device pointers are not NULL
    k = torch.from_numpy(np.concatenate([keys, np.zeros(1, np.uint64)]).view(np.int64)).cuda()
    v = torch.from_numpy(np.concatenate([vals, np.zeros(1, np.uint32)]).view(np.int32)).cuda()
    k2 = torch.empty_like(k)
    v2 = torch.empty_like(v)
    nb = B.fgs_sort_scratch_bytes(n)
    scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
    alt = B.fgs_sort_pairs(k.data_ptr(), v.data_ptr(), k2.data_ptr(), v2.data_ptr(), n, bits,
                           scratch.data_ptr(), nb, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    ko, vo = (k2, v2) if alt else (k, v)
    return ko[:n].cpu().numpy().view(np.uint64), vo[:n].cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("n,bits", [(0, 40), (1, 40), (4095, 44), (4096, 44), (4097, 44),
                                    (100_003, 44), (250_000, 32), (70_001, 64), (33_333, 8),
                                    (20_000, 1), (1_000_000, 47)])
def test_sort_matches_numpy_stable(n, bits):
    rng = np.random.default_rng(n + bits)
    if bits > 32:
        hi = rng.integers(0, 1 << (bits - 32), n, dtype=np.uint64)
        lo = rng.integers(0, 1 << 32, n, dtype=np.uint64)
        keys = (hi << np.uint64(32)) | lo
    else:
        keys = rng.integers(0, 1 << bits, n, dtype=np.uint64)
    # plant many equal keys to exercise stability
    if n > 10:
        keys[::7] = keys[0]
    vals = np.arange(n, dtype=np.uint32)
    ks, vs = _sort_gpu(keys.copy(), vals.copy(), bits)
    mask = np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    order = np.argsort(keys & mask, kind="stable")
    np.testing.assert_array_equal(vs, vals[order])
    np.testing.assert_array_equal(ks, keys[order])


def test_sort_ignores_bits_above_width():
    """Only the low `bits` bits order the keys; higher bits ride along."""
    rng = np.random.default_rng(9)
    n = 50_000
    keys = rng.integers(0, 1 << 63, n, dtype=np.uint64)
    vals = np.arange(n, dtype=np.uint32)
    ks, vs = _sort_gpu(keys.copy(), vals.copy(), 20)
    order = np.argsort(keys & np.uint64((1 << 20) - 1), kind="stable")
    np.testing.assert_array_equal(vs, vals[order])
