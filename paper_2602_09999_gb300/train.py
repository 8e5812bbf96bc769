"""PyTorch-facing training step built on libfastergs.

PyTorch provides device memory, streams and CUDA-graph capture only; every
step of the path runs in the library's kernels through :mod:`.binding`.

  Views        cameras of one batch: the host array (view sizes) and a
               device copy the kernels read, so poses can change between
               graph replays.
  Rasterizer   owns the workspace (one uint8 tensor carved by the
               library's layout) and calls forward / loss / backward.
  RasterizeFn  torch.autograd.Function: images from the Gaussian
               parameters, backward through the hand-written adjoint.
  Trainer      parameters, gradients and Adam moments; one call of
               ``step()`` is forward + loss + backward + Adam (Suppl. A:
               the optimiser runs right after the backward, Suppl. B.1);
               ``capture()`` records that step as a CUDA graph.
"""
from __future__ import annotations

import ctypes
import math
from typing import Dict, Sequence

import numpy as np
import torch

from . import binding as B

GROUPS = ("means", "log_scales", "quats", "opacity", "sh_dc", "sh_rest")
# dynamic Gaussians add a velocity and a temporal centre (and a scalar sigma_t)
MOTION_GROUPS = ("velocity", "t0")
WIDTH = {"means": (3,), "log_scales": (3,), "quats": (4,), "opacity": (), "sh_dc": (3,),
         "sh_rest": (15, 3), "velocity": (3,), "t0": ()}
# Suppl. A learning rates (means at its initial value)
DEFAULT_LR = (1.6e-4, 5e-3, 1e-3, 2.5e-2, 2.5e-3, 1.25e-4)
# velocity and temporal centre (no value in the paper: the means' rate and 1e-3)
MOTION_LR = (1.6e-4, 1e-3)
ADAM_BETAS = (0.9, 0.999)
ADAM_EPS = 1e-15
_DTYPE = {torch.float32: B.FGS_F32, torch.bfloat16: B.FGS_BF16, torch.float16: B.FGS_F16}


def current_stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def groups_of(t) -> tuple:
    """Parameter groups a dict holds: the six static ones, plus velocity and
    t0 for dynamic Gaussians."""
    return GROUPS + MOTION_GROUPS if "velocity" in t else GROUPS


def params_struct(t: Dict[str, torch.Tensor]) -> B.fgs_params:
    """fgs_params over the tensors of t (and its scalar sigma_t, if any)."""
    n = t["means"].shape[0]
    gs = groups_of(t)
    for k in gs:
        x = t[k]
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError(f"{k} must be a contiguous CUDA tensor")
        if tuple(x.shape) != (n,) + WIDTH[k]:
            raise ValueError(f"{k} has shape {tuple(x.shape)}, expected {(n,) + WIDTH[k]}")
    return B.params_struct(n, [t[k].data_ptr() for k in gs], [_DTYPE[t[k].dtype] for k in gs],
                           float(t.get("sigma_t", 0.0)))


class Views:
    """Cameras of one batch (at most 16 views)."""

    def __init__(self, cams: Sequence, device="cuda"):
        self.cams = list(cams)
        self.n = len(self.cams)
        self.host = B.camera_array(self.cams)
        self.nbytes = ctypes.sizeof(self.host)
        self.device = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        self._staging = torch.empty(self.nbytes, dtype=torch.uint8, pin_memory=True)
        self.sizes = [(int(c.width), int(c.height)) for c in self.cams]
        self.pix_off = np.concatenate([[0], np.cumsum([w * h for w, h in self.sizes])]).astype(np.int64)
        self.total_pixels = int(self.pix_off[-1])
        self.set_poses(self.cams)

    def set_poses(self, cams: Sequence):
        """New poses for the same view sizes (asynchronous on the current stream)."""
        if [(int(c.width), int(c.height)) for c in cams] != self.sizes:
            raise ValueError("view sizes are fixed for a Views object")
        self.cams = list(cams)
        self.host = B.camera_array(self.cams)
        torch.cuda.current_stream().synchronize()  # staging buffer may still be in flight
        ctypes.memmove(self._staging.data_ptr(), ctypes.addressof(self.host), self.nbytes)
        self.device.copy_(self._staging, non_blocking=True)

    def split(self, flat: torch.Tensor):
        """Per-view [3, H, W] views of a concatenated image buffer."""
        out = []
        for v, (w, h) in enumerate(self.sizes):
            a = 3 * int(self.pix_off[v])
            out.append(flat[a:a + 3 * w * h].view(3, h, w))
        return out

    def concat(self, images) -> torch.Tensor:
        return torch.cat([torch.as_tensor(im).reshape(-1) for im in images])


class Rasterizer:
    """Workspace and the forward / loss / backward calls of one batch shape."""

    def __init__(self, n: int, views: Views, k_max: int, device="cuda", per_gaussian=False):
        """per_gaussian: reserve the buffers of the per-Gaussian blend
        backward and select it (fgs_tuning.blend_backward)."""
        self.n = int(n)
        self.views = views
        flags = B.FGS_WS_PER_GAUSSIAN if per_gaussian else 0
        self.layout = B.fgs_workspace_size_ex(self.n, views.host, views.n, int(k_max), flags)
        if per_gaussian:
            self.layout.tuning.blend_backward = B.FGS_BACKWARD_PER_GAUSSIAN
        self.ws = torch.zeros(self.layout.total_bytes, dtype=torch.uint8, device=device)
        if self.ws.data_ptr() % 256:
            raise RuntimeError("workspace is not 256-byte aligned")

    @property
    def k_max(self) -> int:
        return int(self.layout.k_max)

    def slot(self, s: int, dtype=torch.uint8) -> torch.Tensor:
        off, nb = int(self.layout.offset[s]), int(self.layout.bytes[s])
        return self.ws[off:off + nb].view(dtype)

    def forward(self, params: B.fgs_params, sh_degree: int, bg, images: torch.Tensor):
        B.fgs_render_forward(self.ws.data_ptr(), self.layout, params, sh_degree, self.views.host,
                             self.views.device.data_ptr(), bg, images.data_ptr(), current_stream())

    def loss(self, images, targets, lam, loss_out, dl):
        B.fgs_loss_l1_dssim(self.ws.data_ptr(), self.layout, self.views.host, images.data_ptr(),
                            targets.data_ptr(), lam, loss_out.data_ptr(), dl.data_ptr(),
                            current_stream())

    def backward_adam(self, params: B.fgs_params, sh_degree: int, bg, dl: torch.Tensor,
                      exp_avg: B.fgs_params, exp_avg_sq: B.fgs_params, adam_state: int,
                      grads=None):
        """Backward fused with the Adam step (params updated in place);
        grads (optional) receives the gradients used."""
        B.fgs_render_backward_adam(self.ws.data_ptr(), self.layout, params, sh_degree,
                                   self.views.host, self.views.device.data_ptr(), bg,
                                   dl.data_ptr(), exp_avg, exp_avg_sq, adam_state, grads,
                                   current_stream())

    def backward(self, params: B.fgs_params, sh_degree: int, bg, dl: torch.Tensor,
                 grads: B.fgs_params):
        B.fgs_render_backward(self.ws.data_ptr(), self.layout, params, sh_degree, self.views.host,
                              self.views.device.data_ptr(), bg, dl.data_ptr(), grads,
                              current_stream())

    def error(self, clear=False):
        """(flags, instances) of the last forward; synchronises."""
        return B.fgs_get_error(self.ws.data_ptr(), clear, current_stream())

    # read-only views of forward state, for tests and diagnostics
    def sorted_lists(self):
        alt = bool(self.layout.sorted_in_alt)
        keys = self.slot(B.FGS_WS_KEYS_ALT if alt else B.FGS_WS_KEYS, torch.int32)  # tile ids
        vals = self.slot(B.FGS_WS_VALS_ALT if alt else B.FGS_WS_VALS, torch.int32)
        ranges = self.slot(B.FGS_WS_RANGES, torch.int32).view(-1, 2)
        return keys, vals, ranges

    def screen(self):
        """Screen records [views, n, 12]; valid where rendered() is true."""
        return self.slot(B.FGS_WS_SCREEN, torch.float32).view(self.views.n, self.n, 12)

    def rendered(self):
        """[views, n] bool: the pairs the last forward rendered (kept tiles > 0)."""
        return self.slot(B.FGS_WS_RECT, torch.int32).view(self.views.n, self.n, 4)[:, :, 3] > 0

    def per_pixel(self):
        return (self.slot(B.FGS_WS_T_FINAL, torch.float32),
                self.slot(B.FGS_WS_N_CONTRIB, torch.int32))

    def fragment_counts(self):
        """(list positions evaluated up to each pixel's last contributor,
        fragments blended), summed over all pixels of the last forward."""
        nc = self.slot(B.FGS_WS_N_CONTRIB, torch.int32).to(torch.int64).sum().item()
        nb = self.slot(B.FGS_WS_N_BLENDED, torch.int32).to(torch.int64).sum().item()
        return int(nc), int(nb)


class RasterizeFn(torch.autograd.Function):
    """images = render(means, log_scales, quats, opacity, sh_dc, sh_rest)."""

    @staticmethod
    def forward(ctx, rast: Rasterizer, sh_degree: int, bg, means, log_scales, quats, opacity,
                sh_dc, sh_rest):
        t = dict(zip(GROUPS, (means, log_scales, quats, opacity, sh_dc, sh_rest)))
        t = {k: v.contiguous() for k, v in t.items()}
        images = torch.empty(3 * rast.views.total_pixels, device=means.device, dtype=torch.float32)
        rast.forward(params_struct(t), sh_degree, bg, images)
        ctx.rast, ctx.sh_degree, ctx.bg = rast, sh_degree, bg
        ctx.save_for_backward(*[t[k] for k in GROUPS])
        return images

    @staticmethod
    def backward(ctx, dl):
        saved = dict(zip(GROUPS, ctx.saved_tensors))
        grads = {k: torch.empty(saved[k].shape, device=dl.device, dtype=torch.float32) for k in GROUPS}
        ctx.rast.backward(params_struct(saved), ctx.sh_degree, ctx.bg, dl.contiguous(),
                          params_struct(grads))
        return (None, None, None) + tuple(grads[k] for k in GROUPS)


def to_device_params(params, device="cuda", sh_dtype=torch.float32):
    out = {}
    for k in groups_of(params):
        x = torch.as_tensor(np.ascontiguousarray(params[k])) if isinstance(params[k], np.ndarray) \
            else params[k]
        dt = sh_dtype if k in ("sh_dc", "sh_rest") else torch.float32
        out[k] = x.to(device=device, dtype=dt).contiguous()
    if "sigma_t" in params:
        out["sigma_t"] = float(params["sigma_t"])
    return out


# (SH dtype, moment dtype) pairs the fused backward + Adam supports
FUSED_PAIRS = {(torch.float32, torch.float32), (torch.bfloat16, torch.float32),
               (torch.bfloat16, torch.bfloat16), (torch.float16, torch.float32),
               (torch.float16, torch.float16)}


class Trainer:
    """Parameters, gradients, Adam moments and the per-step buffers of one
    batch shape.  ``step()`` runs forward, loss, backward and Adam on the
    current stream without host synchronisation; ``capture()`` records it
    as a CUDA graph that ``replay()`` re-launches.  With ``fused_adam`` (the
    default where the storage pair allows it) the backward and the Adam
    step are one call and the gradients are stored only if ``store_grads``."""

    def __init__(self, params, cams: Sequence, k_max: int, sh_degree=3, lam=0.2,
                 bg=(0.0, 0.0, 0.0), lr=DEFAULT_LR, sh_dtype=torch.float32,
                 moment_dtype=torch.float32, lr_means_final=0.0, decay_steps=0, device="cuda",
                 fused_adam=True, store_grads=False, per_gaussian=False):
        self.device = device
        self.fused_adam = bool(fused_adam) and (sh_dtype, moment_dtype) in FUSED_PAIRS
        self.store_grads = bool(store_grads)
        self.params = to_device_params(params, device, sh_dtype)
        self.n = self.params["means"].shape[0]
        self.groups = groups_of(self.params)
        self.grads = {k: torch.zeros(self.params[k].shape, device=device) for k in self.groups}
        self.exp_avg = {k: torch.zeros(self.params[k].shape, device=device, dtype=moment_dtype)
                        for k in self.groups}
        self.exp_avg_sq = {k: torch.zeros(self.params[k].shape, device=device, dtype=moment_dtype)
                           for k in self.groups}
        self.views = Views(cams, device)
        self.rast = Rasterizer(self.n, self.views, k_max, device, per_gaussian=per_gaussian)
        P = self.views.total_pixels
        self.images = torch.zeros(3 * P, device=device)
        self.targets = torch.zeros(3 * P, device=device)
        self.dl = torch.zeros(3 * P, device=device)
        self.loss = torch.zeros(1, device=device)
        self.sh_degree, self.lam, self.bg = int(sh_degree), float(lam), tuple(float(b) for b in bg)
        st = B.fgs_adam_state()
        lr = tuple(lr) + (MOTION_LR if len(lr) == len(GROUPS) else ())
        for g in range(len(lr)):
            st.lr[g] = float(lr[g])
        st.lr_means_final = float(lr_means_final)
        st.decay_steps = int(decay_steps)
        st.beta1, st.beta2, st.eps = ADAM_BETAS[0], ADAM_BETAS[1], ADAM_EPS
        st.step = 0
        host = torch.frombuffer(bytearray(ctypes.string_at(ctypes.addressof(st), ctypes.sizeof(st))),
                                dtype=torch.uint8)
        self.adam_state = host.to(device)
        self._structs()
        self.graph = None

    def _structs(self):
        self.p_s = params_struct(self.params)
        self.g_s = params_struct(self.grads)
        self.m_s = params_struct(self.exp_avg)
        self.v_s = params_struct(self.exp_avg_sq)

    def set_targets(self, targets):
        flat = self.views.concat([torch.as_tensor(t) for t in targets]).to(self.device)
        self.targets.copy_(flat)

    def step(self):
        s = current_stream()
        self.rast.forward(self.p_s, self.sh_degree, self.bg, self.images)
        self.rast.loss(self.images, self.targets, self.lam, self.loss, self.dl)
        if self.fused_adam:
            self.rast.backward_adam(self.p_s, self.sh_degree, self.bg, self.dl, self.m_s, self.v_s,
                                    self.adam_state.data_ptr(),
                                    self.g_s if self.store_grads else None)
            return
        self.rast.backward(self.p_s, self.sh_degree, self.bg, self.dl, self.g_s)
        B.fgs_adam_step_device(self.p_s, self.g_s, self.m_s, self.v_s, self.adam_state.data_ptr(), s)

    def forward_only(self):
        self.rast.forward(self.p_s, self.sh_degree, self.bg, self.images)

    def forward_backward(self):
        """Forward, loss and backward without the optimiser step."""
        self.rast.forward(self.p_s, self.sh_degree, self.bg, self.images)
        self.rast.loss(self.images, self.targets, self.lam, self.loss, self.dl)
        self.rast.backward(self.p_s, self.sh_degree, self.bg, self.dl, self.g_s)

    def reorder(self) -> torch.Tensor:
        """Puts the Gaussians in z-order (Sec. 3.3 "Locality-preserving
        densification"; the paper repeats it every few thousand steps):
        parameters, both Adam moments and the gradient buffers are permuted
        in place, through a temporary and back, so every buffer keeps its
        address and a captured graph stays valid.  Returns the order
        (device int32): order[i] is the previous index of the Gaussian now
        at i."""
        s = current_stream()
        n = self.n
        order = torch.empty(n, dtype=torch.int32, device=self.device)
        sb = B.fgs_morton_scratch_bytes(n)
        scratch = torch.empty(sb, dtype=torch.uint8, device=self.device)
        B.fgs_morton_order(self.params["means"].data_ptr(), n, order.data_ptr(), None,
                           scratch.data_ptr(), sb, s)
        for d in (self.params, self.exp_avg, self.exp_avg_sq, self.grads):
            tmp = {k: torch.empty_like(d[k]) for k in self.groups}
            B.fgs_permute_params(params_struct(d), params_struct(tmp), order.data_ptr(), s)
            B.fgs_permute_params(params_struct(tmp), params_struct(d), None, s)
        return order

    def adam_step_count(self) -> int:
        st = B.fgs_adam_state.from_buffer_copy(bytes(self.adam_state.cpu().numpy()))
        return int(st.step)

    def capture(self, warmup=1):
        """Records step() as a CUDA graph (after `warmup` eager steps on a
        side stream, which do update the parameters)."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(warmup):
                self.step()
        torch.cuda.current_stream().wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step()
        return self.graph

    def replay(self):
        self.graph.replay()
