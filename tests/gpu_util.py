"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
the FP64 oracle on the same seeded inputs, and compare what is unique."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

import oracle
from paper_2602_09999_gb300 import binding as B
from paper_2602_09999_gb300 import train as T
from paper_2602_09999_gb300 import tune

IMAGE_TOL = 2e-4          # max abs image error (fixed by the hot-path target)
GRAD_REL_L2 = 1e-3        # relative L2 error per gradient tensor (same source)


def gpu_forward(params, cams, k_max=None, sh_degree=3, bg=(0.0, 0.0, 0.0), sh_dtype=torch.float32,
                tuning=None, per_gaussian=False):
    n = params["means"].shape[0]
    views = T.Views(cams)
    if k_max is None:
        k_max = max(4096, 64 * n * len(cams))
    rast = T.Rasterizer(n, views, k_max, per_gaussian=per_gaussian)
    if tuning is not None:
        tune.apply(rast.layout, tuning)
    t = T.to_device_params(params, sh_dtype=sh_dtype)
    images = torch.zeros(3 * views.total_pixels, device="cuda")
    rast.forward(T.params_struct(t), sh_degree, bg, images)
    torch.cuda.synchronize()
    return rast, views, t, images


def gpu_lists(rast, view_tile_off):
    """Per global tile: the sorted Gaussian ids (numpy)."""
    flags, inst = rast.error()
    K = min(inst, rast.k_max)
    keys, vals, ranges = rast.sorted_lists()
    vals = vals[:K].cpu().numpy().astype(np.int64)
    keys = keys[:K].cpu().numpy()
    ranges = ranges.cpu().numpy().astype(np.int64)
    return keys, vals, ranges, flags, inst


def compare_lists(rast, views, pre_list, lists_list):
    """Bit-exact comparison of the tile lists, after removing the instances
    whose keep decision float32 may take either way.  Returns the number of
    compared tiles and the number of excluded instances."""
    keys, vals, ranges, flags, inst = gpu_lists(rast, None)
    assert flags == 0
    tile_off = 0
    compared = excluded = 0
    for v, (pre, lists) in enumerate(zip(pre_list, lists_list)):
        ntiles = lists["ranges"].shape[0]
        marg = (lists["flags"] & oracle.IMARGINAL) != 0
        marginal_pairs = set(zip(lists["tile"][marg].tolist(), lists["gid"][marg].tolist()))
        excluded += len(marginal_pairs)
        for t in range(ntiles):
            a, b = lists["ranges"][t]
            sel = slice(a, b)
            o_g = lists["gid"][sel]
            o_keep = (lists["flags"][sel] & oracle.KEEP) != 0
            o_marg = (lists["flags"][sel] & oracle.IMARGINAL) != 0
            want = o_g[o_keep & ~o_marg].tolist()
            ga, gb = ranges[tile_off + t]
            got_all = vals[ga:gb].tolist()
            got = [g for g in got_all if (t, g) not in marginal_pairs]
            if got != want:
                # equal depths within float32 resolution may be ordered either way
                assert sorted(got) == sorted(want), (v, t)
                d = pre["depth"]
                for x, y in zip(got, want):
                    if x != y:
                        assert abs(d[x] - d[y]) <= 2e-6 * abs(d[x]), (v, t, x, y)
            # the tile-sort keys are the global tile ids
            if gb > ga:
                assert np.all(keys[ga:gb] == tile_off + t)
            compared += 1
        tile_off += ntiles
    return compared, excluded


def oracle_forward(params, cams, sh_degree=3, bg=(0.0, 0.0, 0.0), margins=oracle.FP32_MARGINS):
    pres, lists, outs = [], [], []
    for cam in cams:
        pre, li, out = oracle.render(cam, params, sh_degree, bg, margins)
        pres.append(pre)
        lists.append(li)
        outs.append(out)
    return pres, lists, outs


T_TOL = 5e-5              # final transmittance, where its decisions are those of a path


def gpu_pixel_state(rast, views):
    """Per view: the GPU's final transmittance T[H,W] and last blended
    Gaussian [H,W] (-1 for none), read from the workspace of the last
    forward (n_contrib is the 1-based list position of the last blended
    entry in the pixel's tile list)."""
    Tg, ncg = rast.per_pixel()
    Tg, ncg = Tg.cpu().numpy(), ncg.cpu().numpy().astype(np.int64)
    _, vals, ranges = rast.sorted_lists()
    vals = vals.cpu().numpy().astype(np.int64)
    ranges = ranges.cpu().numpy().astype(np.int64)
    out, tile_off = [], 0
    for v, (W, H) in enumerate(views.sizes):
        a, b = int(views.pix_off[v]), int(views.pix_off[v + 1])
        nc = ncg[a:b].reshape(H, W)
        tx, ty = (W + 15) // 16, (H + 15) // 16
        uu, vv = np.meshgrid(np.arange(W), np.arange(H))
        start = ranges[tile_off + (vv // 16) * tx + (uu // 16), 0]
        last = np.where(nc > 0, vals[np.maximum(start + nc - 1, 0)], -1)
        out.append((Tg[a:b].reshape(H, W), last))
        tile_off += tx * ty
    return out


@dataclass
class ImageCheck:
    """Outcome of image_check.  bad: pixels that fail their check;
    exact_pixels / exact_max: pixels whose every float32 decision is
    determined and their max abs error; path_pixels / path_max: pixels
    checked against the admissible results of the oracle's decision paths
    and the largest error to the nearest admissible result; allowance_pixels
    / allowance_excess: pixels whose paths overflowed, held to tol plus the
    oracle's summed allowance, and their largest excess over that bound;
    excluded: pixels with no bound at all (none in any test scene)."""
    bad: int
    exact_pixels: int
    exact_max: float
    path_pixels: int
    path_max: float
    allowance_pixels: int
    allowance_excess: float
    excluded: int

    @property
    def pixels(self):
        return self.exact_pixels + self.path_pixels + self.allowance_pixels + self.excluded

    def summary(self):
        return (f"{self.path_pixels} px checked against an admissible path (max err to the nearest "
                f"{self.path_max:.2e}), {self.allowance_pixels} px on allowance, {self.excluded} "
                f"excluded, max err on {self.exact_pixels} exact px {self.exact_max:.2e}")


def image_check(img, out, tol=IMAGE_TOL, T=None, last=None, t_tol=T_TOL):
    """GPU image [3,H,W] (and optionally its final transmittance T[H,W] and
    last blended Gaussian last[H,W], -1 for none) against the oracle.
    Every pixel whose float32 decisions are all determined (path status 0)
    must be within tol of the oracle (T within t_tol, the same last
    Gaussian).  A pixel with decisions float32 may take either way (status
    1) must be within tol of one of the FP64 results of its admissible
    decision paths, jointly in colour, T and last Gaussian.  Only pixels
    whose paths overflowed (status 2) fall back to tol plus the oracle's
    summed first-order allowance; pixels without a bound at all (hard) are
    excluded and counted."""
    img = np.asarray(img, np.float64)
    H, W = img.shape[1:]
    err = np.abs(img - out["image"]).max(axis=0)
    status = out["status"]
    hard = out["hard"].astype(bool) & (status == 2)
    exact = status == 0
    bad = exact & (err > tol)
    if T is not None:
        bad |= exact & (np.abs(np.asarray(T, np.float64) - out["T_final"]) > t_tol)
    if last is not None:
        bad |= exact & (np.asarray(last) != out["last_gid"])
    # several admissible results: the nearest one, all fields at once
    pix, val = out["path_pix"], out["path_val"]
    flat = img.reshape(3, -1)
    d = np.abs(val[:, :3] - flat[:, pix].T).max(axis=1)
    fits = d <= tol
    if T is not None:
        fits &= np.abs(val[:, 3] - np.asarray(T, np.float64).reshape(-1)[pix]) <= t_tol
    if last is not None:
        fits &= val[:, 4] == np.asarray(last).reshape(-1)[pix]
    any_fit = np.zeros(H * W, bool)
    np.logical_or.at(any_fit, pix, fits)
    nearest = np.full(H * W, np.inf)
    np.minimum.at(nearest, pix, d)
    multi = (status == 1).reshape(-1)
    bad |= (multi & ~any_fit).reshape(H, W)
    # overflowed enumerations: the allowance bound
    over = (status == 2) & ~hard
    excess = (err - tol - out["allowance"])[over]
    bad |= over & (err > tol + out["allowance"])
    return ImageCheck(bad=int(bad.sum()), exact_pixels=int(exact.sum()),
                      exact_max=float(err[exact].max(initial=0.0)), path_pixels=int(multi.sum()),
                      path_max=float(nearest[multi].max(initial=0.0)),
                      allowance_pixels=int(over.sum()),
                      allowance_excess=float(excess.max(initial=-np.inf)), excluded=int(hard.sum()))


def dilate_mask(m, r):
    """Pixels within r (Chebyshev distance) of a set pixel."""
    m = np.asarray(m, bool)
    if not r or not m.any():
        return m
    pad = np.pad(m, r)
    acc = np.zeros_like(m)
    H, W = m.shape
    for dy in range(2 * r + 1):
        for dx in range(2 * r + 1):
            acc |= pad[dy:dy + H, dx:dx + W]
    return acc


def gradient_mask(out, target=None, tol=IMAGE_TOL, dilate=0):
    """Pixels whose dL/dC the gradient comparison zeroes on both sides: those
    with a decision float32 may take the other way whose effect on the value
    is unbounded (overflow of the oracle's event lists) or, summed, above the
    image tolerance.  Elsewhere GPU and oracle values differ by at most the
    tolerance plus a smaller allowance, which moves the smooth part of dL/dC
    -- here and in the SSIM window around -- too little for the gradient bar,
    so no dilation is needed.  The L1 term is not smooth: its derivative is
    the sign of (C - target), a decision float32 may take the other way
    where |C - target| is within that bound; given the target, those pixels
    are masked too (one flipped sign moves the gradients of the few Gaussians
    on that pixel by several percent)."""
    allow = out["allowance"]
    m = out["hard"].astype(bool) | (allow > tol)
    if target is not None:
        near = np.abs(out["image"] - np.asarray(target, np.float64)) <= tol + allow[None]
        m |= near.any(axis=0)
    return dilate_mask(m, dilate)


def ambiguity_masks(cams, params, sh_degree=3, bg=(0.0, 0.0, 0.0), dilate=0, targets=None):
    """gradient_mask of the oracle's render of every view (with the L1 sign
    decisions when the targets are given)."""
    masks = []
    for v, cam in enumerate(cams):
        _, _, out = oracle.render(cam, params, sh_degree, bg, oracle.FP32_MARGINS)
        masks.append(gradient_mask(out, None if targets is None else targets[v], dilate=dilate))
    return masks


def ill_conditioned(cams, params, factor=4.0):
    """Gaussians whose footprint half-extent exceeds `factor` times the larger
    image side in some view (near-plane or grazing splats): their gradient
    sums thousands of cancelling per-pixel terms, which float32 accumulation
    in any order cannot resolve to 1e-3."""
    bad = np.zeros(np.asarray(params["means"]).shape[0], bool)
    for cam in cams:
        pre = oracle.preprocess(cam, params)
        ext = pre["aux"][:, 5:7].max(axis=1)
        bad |= pre["visible"] & (ext > factor * max(cam.width, cam.height))
    return bad


def oracle_grads(cams, params, targets, masks=None, lam=0.2, bg=(0.0, 0.0, 0.0), sh_degree=3):
    """Oracle loss (batch mean) and parameter gradients, with dL/dC zeroed on
    the masked pixels of each view."""
    grads = oracle.zero_grads(params)
    B = len(cams)
    total = 0.0
    for v, (cam, tgt) in enumerate(zip(cams, targets)):
        pre, lists, out = oracle.render(cam, params, sh_degree, bg)
        L, dL = oracle.loss(out["image"], tgt, lam, grad_scale=1.0 / B)
        total += L / B
        if masks is not None:
            dL[:, masks[v]] = 0.0
        sg = oracle.blend_backward(cam, pre, lists, dL, bg)
        oracle.preprocess_backward(cam, params, sg, sh_degree, grads)
    return total, grads


def gpu_grads(params, cams, targets, masks=None, lam=0.2, bg=(0.0, 0.0, 0.0), sh_degree=3,
              sh_dtype=torch.float32, tuning=None, k_max=None, per_gaussian=False):
    """GPU loss and gradients through the C ABI, with dL/dC zeroed on the
    masked pixels of each view."""
    rast, views, t, images = gpu_forward(params, cams, k_max=k_max, bg=bg, sh_degree=sh_degree,
                                         sh_dtype=sh_dtype, tuning=tuning, per_gaussian=per_gaussian)
    tg = views.concat([torch.from_numpy(np.asarray(x, np.float32)) for x in targets]).cuda()
    loss = torch.zeros(1, device="cuda")
    dl = torch.zeros_like(images)
    rast.loss(images, tg, lam, loss, dl)
    if masks is not None:
        for v, m in enumerate(masks):
            view = views.split(dl)[v]
            view[:, torch.from_numpy(m).cuda()] = 0.0
    grads = {k: torch.zeros(t[k].shape, device="cuda") for k in T.groups_of(t)}
    rast.backward(T.params_struct(t), sh_degree, bg, dl, T.params_struct(grads))
    torch.cuda.synchronize()
    return float(loss.item()), {k: v.cpu().numpy() for k, v in grads.items()}, rast


def grad_errors(gg, go, exclude=None):
    """Relative L2 error per tensor over the Gaussians not excluded (every
    group both sides hold: six, or eight for dynamic Gaussians)."""
    out = {}
    for k in [k for k in T.GROUPS + T.MOTION_GROUPS if k in gg and k in go]:
        a, b = np.asarray(gg[k], np.float64), np.asarray(go[k], np.float64)
        if exclude is not None and exclude.any():
            a, b = a[~exclude], b[~exclude]
        out[k] = rel_l2(a, b) if np.any(b) else float(np.abs(a).max(initial=0.0))
    return out


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a))
