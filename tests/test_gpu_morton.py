"""The locality-preserving order on the GPU (Sec. 3.3 "Locality-preserving
densification"), through the C ABI, against the oracle: z-order codes and
the permutation bit for bit (integer results; the quantisation is decided in
float32 on both sides), from one Gaussian to the 3M-Gaussian bench scene;
the gather of every parameter and moment group bit for bit; and the
invariance it must keep -- a reordered scene renders the same image bit for
bit and the same gradients, permuted."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from gpu_util import gpu_forward, gpu_grads, rel_l2  # noqa: E402
from paper_2602_09999_gb300 import binding as B  # noqa: E402
from paper_2602_09999_gb300 import scenes  # noqa: E402
from paper_2602_09999_gb300 import train as T  # noqa: E402


def _gpu_order(means):
    m = torch.from_numpy(np.ascontiguousarray(means, np.float32)).cuda()
    n = m.shape[0]
    order = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    codes = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    sb = B.fgs_morton_scratch_bytes(n)
    scratch = torch.empty(max(sb, 256), dtype=torch.uint8, device="cuda")
    B.fgs_morton_order(m.data_ptr(), n, order.data_ptr(), codes.data_ptr(), scratch.data_ptr(), sb,
                       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return (order[:n].cpu().numpy().view(np.uint32), codes[:n].cpu().numpy().view(np.uint32))


def _check(means):
    order, codes = _gpu_order(means)
    want_codes = oracle.morton_codes(means)
    want_order = oracle.morton_order(means)
    np.testing.assert_array_equal(order, want_order)
    np.testing.assert_array_equal(codes, want_codes[want_order])


@pytest.mark.parametrize("n", [1, 7, 4097, 100_003])
def test_codes_and_order_bit_exact(n):
    rng = np.random.default_rng(n)
    means = (rng.standard_normal((n, 3)) * [3.0, 0.5, 10.0] + [1.0, -2.0, 0.0]).astype(np.float32)
    _check(means)


def test_codes_and_order_bit_exact_bench_scene():
    """The 3M-Gaussian outdoor scene the bench times (several sort tiles,
    many equal codes in its dense clusters)."""
    _check(scenes.outdoor_scene(3_000_000, seed=0)["means"])


def test_degenerate_boxes():
    same = np.tile(np.float32([0.5, -1.0, 2.0]), (5000, 1))
    order, codes = _gpu_order(same)
    np.testing.assert_array_equal(order, np.arange(5000))
    assert not codes.any()
    rng = np.random.default_rng(4)
    flat = rng.uniform(-1, 1, (3000, 3)).astype(np.float32)
    flat[:, 1] = 0.25
    _check(flat)
    # many exact duplicates: ties keep index order
    dup = np.repeat(rng.uniform(0, 1, (50, 3)).astype(np.float32), 40, axis=0)
    rng.shuffle(dup)
    _check(dup)
    assert _gpu_order(np.zeros((0, 3), np.float32))[0].size == 0


def _dev(params, sh_dtype=torch.float32):
    return T.to_device_params(params, sh_dtype=sh_dtype)


@pytest.mark.parametrize("sh_dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("dynamic", [False, True])
def test_permute_every_group_bit_exact(sh_dtype, dynamic):
    n = 20_011
    p = scenes.dynamic_scene(n, seed=8) if dynamic else scenes.outdoor_scene(n, seed=8)
    src = _dev(p, sh_dtype)
    groups = T.groups_of(src)
    dst = {k: torch.empty_like(src[k]) for k in groups}
    order = np.random.default_rng(9).permutation(n).astype(np.int32)
    o = torch.from_numpy(order).cuda()
    s = torch.cuda.current_stream().cuda_stream
    B.fgs_permute_params(T.params_struct(src), T.params_struct(dst), o.data_ptr(), s)
    copy = {k: torch.empty_like(src[k]) for k in groups}
    B.fgs_permute_params(T.params_struct(src), T.params_struct(copy), None, s)
    torch.cuda.synchronize()
    for k in groups:
        assert torch.equal(dst[k].cpu(), src[k].cpu()[torch.from_numpy(order).long()]), k
        assert torch.equal(copy[k], src[k]), k


def test_reordered_scene_renders_the_same():
    """The oracle's z-order applied to a scene (numpy gather): the GPU image
    of the reordered scene equals the original bit for bit, and its
    gradients are the original's, permuted (up to atomic-add order)."""
    p = scenes.outdoor_scene(40_000, seed=2)
    cams = scenes.orbit_cameras(2, 203, 131, radius=6.0, seed=5)
    order = oracle.morton_order(p["means"]).astype(np.int64)
    q = {k: np.ascontiguousarray(v[order]) for k, v in p.items()}
    *_, img_p = gpu_forward(p, cams)
    *_, img_q = gpu_forward(q, cams)
    assert torch.equal(img_p, img_q)
    targets = [scenes.target_image(203, 131, view=i) for i in range(2)]
    Lp, gp, _ = gpu_grads(p, cams, targets)
    Lq, gq, _ = gpu_grads(q, cams, targets)
    assert Lp == Lq
    for k in T.GROUPS:
        assert rel_l2(gq[k], gp[k][order]) < 1e-5, k


def test_trainer_reorder_keeps_the_step():
    """Trainer.reorder on seeded parameters and seeded moments: the order is
    the oracle's for the seeded means; parameters and both moments are the
    same rows permuted; the buffers keep their addresses, so a graph
    captured before the reorder still runs, and its forward renders the
    same images and loss as before the reorder."""
    p = scenes.outdoor_scene(30_000, seed=4)
    cams = scenes.orbit_cameras(2, 160, 120, radius=6.0, seed=6)
    targets = [scenes.target_image(160, 120, view=i) for i in range(2)]
    warm = T.Trainer(p, cams, k_max=2_000_000)  # loads every kernel before the capture
    warm.set_targets(targets)
    warm.step()
    tr = T.Trainer(p, cams, k_max=2_000_000)
    tr.set_targets(targets)
    rng = np.random.default_rng(10)
    for d in (tr.exp_avg, tr.exp_avg_sq):
        for k in tr.groups:
            d[k].copy_(torch.from_numpy(rng.uniform(0.0, 1.0, tuple(d[k].shape)).astype(np.float32)))
    tr.forward_only()
    tr.rast.loss(tr.images, tr.targets, tr.lam, tr.loss, tr.dl)
    torch.cuda.synchronize()
    img0, loss0 = tr.images.clone(), tr.loss.clone()
    before = {name: {k: d[k].cpu().clone() for k in tr.groups}
              for name, d in (("p", tr.params), ("m", tr.exp_avg), ("v", tr.exp_avg_sq))}
    ptrs = [d[k].data_ptr() for d in (tr.params, tr.exp_avg, tr.exp_avg_sq) for k in tr.groups]
    tr.capture(warmup=0)                     # recorded, not run
    order = tr.reorder()
    torch.cuda.synchronize()
    o = order.cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(o, oracle.morton_order(p["means"]))
    for name, d in (("p", tr.params), ("m", tr.exp_avg), ("v", tr.exp_avg_sq)):
        for k in tr.groups:
            assert torch.equal(d[k].cpu(), before[name][k][o]), (name, k)
    assert ptrs == [d[k].data_ptr() for d in (tr.params, tr.exp_avg, tr.exp_avg_sq)
                    for k in tr.groups]
    tr.replay()                              # forward of the reordered scene, then the update
    torch.cuda.synchronize()
    assert torch.equal(tr.images, img0)
    assert torch.equal(tr.loss, loss0)
