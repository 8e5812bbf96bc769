"""FP64 CPU oracle for one Faster-GS (arXiv 2602.09999) optimisation step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path (``paper_2602_09999_gb300``) and imports nothing
from it; the two meet only through the seeded inputs of
``paper_2602_09999_gb300.scenes``, which hold none of the method's
arithmetic.

The arithmetic lives in ``fgs_oracle.c`` (plain C, double precision).  This
module compiles it with gcc, loads it with ctypes and composes the stages of
one step in the paper's order:

  preprocess (Eq. 1, Eq. 2, Sec. 2.1 activations, Sec. 3.2 bounds and tile
  culling, Suppl. B.1 degeneracy tests)  ->  instance lists sorted by
  (tile, depth) (Sec. 3.2 "Sorting"; numpy's stable sort is the library
  sort step)  ->  blending (Eq. 3, Eq. 4)  ->  loss (Suppl. A)  ->  exact
  adjoint of the blend and of the preprocessing  ->  Adam (Suppl. A).

Parity pins for every function are in ``tests/test_oracle_*.py``.  Parity
unpinned: the sign convention of the real SH basis beyond what the scipy
comparison fixes is self-consistent only; the synthetic-scene constants are
recorded, not derived from the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fgs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

TILE = 16
PARAM_NAMES = ("means", "log_scales", "quats", "opacity", "sh_dc", "sh_rest")
VISIBLE = 1
MARGINAL = 2
KEEP = 1
IMARGINAL = 2


def build(force: bool = False) -> str:
    """Compile fgs_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("near_plane", ctypes.c_double), ("cam_pos", ctypes.c_double * 3),
                ("time", ctypes.c_double)]


class _Motion(ctypes.Structure):
    _fields_ = [("velocity", ctypes.c_void_p), ("t0", ctypes.c_void_p),
                ("sigma_t", ctypes.c_double)]


class _Margins(ctypes.Structure):
    _fields_ = [("rel", ctypes.c_double), ("q_rel", ctypes.c_double),
                ("pos_rel", ctypes.c_double), ("px", ctypes.c_double),
                ("t_rel", ctypes.c_double), ("depth_rel", ctypes.c_double),
                ("value_tol", ctypes.c_double), ("tile_culling", ctypes.c_int32)]


@dataclass
class Margins:
    """Decision margins inside which float32 may decide a threshold test the
    other way (zero = pure FP64 decisions), and the tile-culling switch.

    rel: scalar thresholds (depth vs near plane, |q|, det, opacity, k);
    q_rel: rounding of a quadratic form relative to the sum of its |terms|;
    pos_rel: error of mu2D relative to max(1, |mu2D|) in pixels, which moves
    the quadratic form by about 2 |C d| pos_err; px: rectangle edges;
    t_rel: transmittance stop test; depth_rel: depth ties; value_tol: a
    pixel is flagged only where taking such a decision the other way can move
    its value by more than this (blend or skip an entry: alpha T (c - R), R
    the normalised colour behind it; swap tied entries: T a1 a2 (c1 - c2);
    0 flags every such decision)."""
    rel: float = 0.0
    q_rel: float = 0.0
    pos_rel: float = 0.0
    px: float = 0.0
    t_rel: float = 0.0
    depth_rel: float = 0.0
    value_tol: float = 0.0
    tile_culling: int = 1


# margins used when the oracle is compared with a float32 implementation:
# roughly 10-30 float32 ulps of each quantity the decision depends on
FP32_MARGINS = Margins(rel=2e-6, q_rel=1e-6, pos_rel=5e-7, px=2e-3, t_rel=1e-4,
                       depth_rel=2e-6, value_tol=5e-5)
NO_MARGINS = Margins()


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _cam_struct(cam) -> _Camera:
    c = _Camera()
    R = np.asarray(cam.R, dtype=np.float32).astype(np.float64).reshape(9)
    t = np.asarray(cam.t, dtype=np.float32).astype(np.float64)
    pos = np.asarray(cam.cam_pos, dtype=np.float32).astype(np.float64)
    for i in range(9):
        c.R[i] = R[i]
    for i in range(3):
        c.t[i] = t[i]
        c.cam_pos[i] = pos[i]
    c.fx = float(np.float32(cam.fx))
    c.fy = float(np.float32(cam.fy))
    c.cx = float(np.float32(cam.cx))
    c.cy = float(np.float32(cam.cy))
    c.time = float(np.float32(getattr(cam, "time", 0.0)))
    c.width = int(cam.width)
    c.height = int(cam.height)
    c.near_plane = float(np.float32(cam.near))
    return c


def _mg_struct(m: Margins) -> _Margins:
    return _Margins(m.rel, m.q_rel, m.pos_rel, m.px, m.t_rel, m.depth_rel, m.value_tol,
                    int(m.tile_culling))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


MOTION_NAMES = ("velocity", "t0")


def is_dynamic(params) -> bool:
    """Dynamic Gaussians carry a velocity, a temporal centre and sigma_t."""
    return "velocity" in params


def names_of(params):
    return PARAM_NAMES + MOTION_NAMES if is_dynamic(params) else PARAM_NAMES


class _MotionArrays:
    """The orc_motion struct of params (a NULL pointer for static ones),
    keeping its float64 arrays alive."""

    def __init__(self, params):
        self.arrays = None
        if is_dynamic(params):
            n = np.shape(params["means"])[0]
            self.arrays = (_f64(params["velocity"]).reshape(n, 3), _f64(params["t0"]).reshape(n))
            self.struct = _Motion(self.arrays[0].ctypes.data, self.arrays[1].ctypes.data,
                                  float(np.float32(params["sigma_t"])))

    def ref(self):
        return ctypes.byref(self.struct) if self.arrays is not None else None


def _param_arrays(params):
    """Parameters as float64 (float32 inputs are promoted exactly)."""
    arrs = tuple(_f64(params[k]) for k in PARAM_NAMES)
    n = arrs[0].shape[0]
    shapes = ((n, 3), (n, 3), (n, 4), (n,), (n, 3), (n, 15, 3))
    for a, shp in zip(arrs, shapes):
        if a.shape != shp:
            raise ValueError(f"parameter shape {a.shape} != {shp}")
    return arrs


def sh_basis(direction, degree=3, with_grad=False):
    """Real SH basis Y[16] (and dY[16,3]) at a unit direction."""
    lib = _lib_handle()
    d = np.ascontiguousarray(direction, dtype=np.float64)
    Y = np.zeros(16)
    dY = np.zeros(48) if with_grad else None
    lib.orc_sh_basis(_p(d), ctypes.c_int(degree), _p(Y), _p(dY) if with_grad else None)
    return (Y, dY.reshape(16, 3)) if with_grad else Y


def preprocess(cam, params, sh_degree=3, margins: Margins = NO_MARGINS):
    """Per-Gaussian screen state for one camera (see orc_preprocess)."""
    lib = _lib_handle()
    arrs = _param_arrays(params)
    n = arrs[0].shape[0]
    out = dict(xy=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n),
               rgb=np.zeros((n, 3)), clamped=np.zeros((n, 3), np.uint8), depth=np.zeros(n),
               rect=np.zeros((n, 4), np.int32), status=np.zeros(n, np.int32),
               aux=np.zeros((n, 8)))
    c, m, mo = _cam_struct(cam), _mg_struct(margins), _MotionArrays(params)
    rc = lib.orc_preprocess(ctypes.byref(c), ctypes.c_int64(n), ctypes.c_int(sh_degree),
                            *[_p(a) for a in arrs], mo.ref(), ctypes.byref(m),
                            _p(out["xy"]), _p(out["conic"]), _p(out["opacity"]), _p(out["rgb"]),
                            _p(out["clamped"]), _p(out["depth"]), _p(out["rect"]),
                            _p(out["status"]), _p(out["aux"]))
    if rc != 0:
        raise ValueError(f"orc_preprocess failed ({rc})")
    out["visible"] = (out["status"] & VISIBLE) != 0
    out["marginal"] = (out["status"] & MARGINAL) != 0
    return out


def tile_grid(cam):
    return (cam.width + TILE - 1) // TILE, (cam.height + TILE - 1) // TILE


def build_lists(cam, params, pre, sh_degree=3, margins: Margins = NO_MARGINS):
    """Instance lists for one camera.

    Candidates are emitted in ascending Gaussian id, tiles row-major inside
    each rectangle, then ordered by (tile id, depth) with a stable sort, so
    equal depths keep Gaussian-id order.  Returns tile, gid, flags (KEEP /
    IMARGINAL) per sorted entry and ranges[n_tiles, 2].
    """
    lib = _lib_handle()
    arrs = _param_arrays(params)
    n = arrs[0].shape[0]
    c, m, mo = _cam_struct(cam), _mg_struct(margins), _MotionArrays(params)
    counts = np.zeros(n, np.int64)
    lib.orc_count_instances(ctypes.byref(c), ctypes.c_int64(n), ctypes.c_int(sh_degree),
                            *[_p(a) for a in arrs], mo.ref(), ctypes.byref(m), _p(counts))
    offsets = np.zeros(n, np.int64)
    if n > 1:
        offsets[1:] = np.cumsum(counts)[:-1]
    total = int(counts.sum())
    tile = np.zeros(max(total, 1), np.int32)
    gid = np.zeros(max(total, 1), np.int32)
    flags = np.zeros(max(total, 1), np.uint8)
    lib.orc_emit_instances(ctypes.byref(c), ctypes.c_int64(n), ctypes.c_int(sh_degree),
                           *[_p(a) for a in arrs], mo.ref(), ctypes.byref(m), _p(offsets),
                           _p(tile), _p(gid), _p(flags))
    tile, gid, flags = tile[:total], gid[:total], flags[:total]
    depth = pre["depth"][gid]
    order = np.argsort(depth, kind="stable")
    order = order[np.argsort(tile[order], kind="stable")]
    tile, gid, flags = tile[order], gid[order], flags[order]
    tx, ty = tile_grid(cam)
    ids = np.arange(tx * ty)
    ranges = np.stack([np.searchsorted(tile, ids, "left"),
                       np.searchsorted(tile, ids, "right")], axis=1).astype(np.int64)
    return dict(tile=tile, gid=gid, flags=flags, ranges=np.ascontiguousarray(ranges),
                counts=counts)


def blend_forward(cam, pre, lists, bg=(0.0, 0.0, 0.0), margins: Margins = NO_MARGINS):
    lib = _lib_handle()
    W, H = cam.width, cam.height
    bg = np.asarray(bg, np.float64)
    out = dict(image=np.zeros((3, H, W)), T_final=np.zeros((H, W)),
               n_contrib=np.zeros((H, W), np.int32), last_gid=np.zeros((H, W), np.int32),
               ambiguous=np.zeros((H, W), np.uint8), hard=np.zeros((H, W), np.uint8),
               allowance=np.zeros((H, W)))
    m = _mg_struct(margins)
    lib.orc_blend_forward(ctypes.c_int32(W), ctypes.c_int32(H), _p(lists["ranges"]),
                          _p(lists["gid"]), _p(lists["flags"]), _p(pre["xy"]), _p(pre["conic"]),
                          _p(pre["opacity"]), _p(pre["rgb"]), _p(pre["depth"]), _p(bg),
                          ctypes.byref(m), _p(out["image"]), _p(out["T_final"]),
                          _p(out["n_contrib"]), _p(out["last_gid"]), _p(out["ambiguous"]),
                          _p(out["hard"]), _p(out["allowance"]))
    return out


MAX_PATHS = 64


def blend_paths(cam, pre, lists, bg=(0.0, 0.0, 0.0), margins: Margins = NO_MARGINS,
                max_paths=MAX_PATHS):
    """Admissible results of every pixel (see orc_blend_paths): the results a
    float32 evaluation may reach when it takes the decisions within the
    margins either way.  Returns status[H,W] (0: one result, the FP64 one;
    1: several; 2: more than max_paths, bounded only by the allowance) and,
    for the status-1 pixels, path_pix[M] (pixel index v W + u, ascending)
    with path_val[M, 5] = (C + T bg, T, last blended Gaussian or -1)."""
    lib = _lib_handle()
    W, H = cam.width, cam.height
    bg = np.asarray(bg, np.float64)
    m = _mg_struct(margins)
    status = np.zeros((H, W), np.uint8)
    cap = max(1024, 2 * W * H)
    while True:
        pix = np.zeros(cap, np.int64)
        val = np.zeros((cap, 5))
        n_out = ctypes.c_int64(0)
        rc = lib.orc_blend_paths(ctypes.c_int32(W), ctypes.c_int32(H), _p(lists["ranges"]),
                                 _p(lists["gid"]), _p(lists["flags"]), _p(pre["xy"]),
                                 _p(pre["conic"]), _p(pre["opacity"]), _p(pre["rgb"]),
                                 _p(pre["depth"]), _p(bg), ctypes.byref(m), ctypes.c_int32(max_paths),
                                 ctypes.c_int64(cap), _p(status), ctypes.byref(n_out), _p(pix),
                                 _p(val))
        if rc != 0:
            raise MemoryError("orc_blend_paths failed")
        if n_out.value <= cap:
            break
        cap = int(n_out.value)
    k = int(n_out.value)
    order = np.argsort(pix[:k], kind="stable")
    return dict(status=status, path_pix=pix[:k][order], path_val=val[:k][order])


def blend_brute(cam, pre, bg=(0.0, 0.0, 0.0)):
    """Tile-free twin: every pixel walks all visible Gaussians in (depth, id)
    order."""
    lib = _lib_handle()
    W, H = cam.width, cam.height
    vis = np.nonzero(pre["visible"])[0]
    order = vis[np.argsort(pre["depth"][vis], kind="stable")].astype(np.int32)
    bg = np.asarray(bg, np.float64)
    image = np.zeros((3, H, W))
    T = np.zeros((H, W))
    last = np.zeros((H, W), np.int32)
    lib.orc_blend_brute(ctypes.c_int32(W), ctypes.c_int32(H), ctypes.c_int64(order.size),
                        _p(order), _p(pre["xy"]), _p(pre["conic"]), _p(pre["opacity"]),
                        _p(pre["rgb"]), _p(pre["depth"]), _p(bg), _p(image), _p(T), _p(last))
    return dict(image=image, T_final=T, last_gid=last)


def blend_backward(cam, pre, lists, dL_dimage, bg=(0.0, 0.0, 0.0)):
    """Screen-space gradients (mu2D, conic, opacity, rgb) per Gaussian."""
    lib = _lib_handle()
    n = pre["xy"].shape[0]
    W, H = cam.width, cam.height
    g = dict(xy=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n),
             rgb=np.zeros((n, 3)))
    dL = np.ascontiguousarray(dL_dimage, dtype=np.float64)
    bg = np.asarray(bg, np.float64)
    rc = lib.orc_blend_backward(ctypes.c_int32(W), ctypes.c_int32(H),
                                ctypes.c_int64(lists["gid"].size), _p(lists["ranges"]),
                                _p(lists["gid"]), _p(lists["flags"]), _p(pre["xy"]),
                                _p(pre["conic"]), _p(pre["opacity"]), _p(pre["rgb"]), _p(bg),
                                _p(dL), _p(g["xy"]), _p(g["conic"]), _p(g["opacity"]),
                                _p(g["rgb"]))
    if rc != 0:
        raise MemoryError("orc_blend_backward failed")
    return g


def zero_grads(params):
    return {k: np.zeros(np.shape(params[k]), np.float64) for k in names_of(params)}


def preprocess_backward(cam, params, screen_grads, sh_degree=3, grads=None):
    """Accumulates parameter gradients from screen-space gradients."""
    lib = _lib_handle()
    arrs = _param_arrays(params)
    n = arrs[0].shape[0]
    if grads is None:
        grads = zero_grads(params)
    c, mo = _cam_struct(cam), _MotionArrays(params)
    dyn = is_dynamic(params)
    lib.orc_preprocess_backward(ctypes.byref(c), ctypes.c_int64(n), ctypes.c_int(sh_degree),
                                *[_p(a) for a in arrs], _p(screen_grads["xy"]),
                                _p(screen_grads["conic"]), _p(screen_grads["opacity"]),
                                _p(screen_grads["rgb"]),
                                *[_p(grads[k]) for k in PARAM_NAMES], mo.ref(),
                                _p(grads["velocity"]) if dyn else None,
                                _p(grads["t0"]) if dyn else None)
    return grads


def loss(image, target, lam=0.2, grad_scale=1.0):
    """(1 - lam) L1 + lam (1 - SSIM) and dL/dimage for one [3,H,W] image,
    both images read as float64."""
    lib = _lib_handle()
    img = np.ascontiguousarray(image, dtype=np.float64)
    tgt = np.ascontiguousarray(target, dtype=np.float64)
    _, H, W = img.shape
    dL = np.zeros((3, H, W))
    out = ctypes.c_double(0.0)
    rc = lib.orc_loss(ctypes.c_int32(H), ctypes.c_int32(W), _p(img), _p(tgt),
                      ctypes.c_double(lam), ctypes.c_double(grad_scale), ctypes.byref(out), _p(dL))
    if rc != 0:
        raise MemoryError("orc_loss failed")
    return out.value, dL


def adam(p, g, m, v, lr, step, b1=0.9, b2=0.999, eps=1e-15):
    """In-place FP64 Adam on float64 arrays."""
    lib = _lib_handle()
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    rc = lib.orc_adam(ctypes.c_int64(p.size), _p(p), _p(g), _p(m), _p(v), ctypes.c_double(lr),
                      ctypes.c_double(b1), ctypes.c_double(b2), ctypes.c_double(eps),
                      ctypes.c_int32(step))
    if rc != 0:
        raise ValueError("orc_adam failed")


# learning rates of Suppl. A in the order of PARAM_NAMES (means at its
# initial value; the decay and scene-scale factor are host scalars), then
# velocity and temporal centre of dynamic Gaussians (not given in the paper:
# the means' rate and 1e-3)
DEFAULT_LR = (1.6e-4, 5e-3, 1e-3, 2.5e-2, 2.5e-3, 1.25e-4, 1.6e-4, 1e-3)


def render(cam, params, sh_degree=3, bg=(0.0, 0.0, 0.0), margins: Margins = NO_MARGINS,
           paths=None):
    """Forward for one camera: preprocess, lists, blend.  With paths (by
    default whenever the margins are not all zero) `out` also holds the
    admissible results of blend_paths."""
    pre = preprocess(cam, params, sh_degree, margins)
    lists = build_lists(cam, params, pre, sh_degree, margins)
    out = blend_forward(cam, pre, lists, bg, margins)
    if paths is None:
        paths = margins.t_rel > 0.0 or margins.rel > 0.0
    if paths:
        out.update(blend_paths(cam, pre, lists, bg, margins))
    return pre, lists, out


def train_step(cams, params, targets, moments=None, step=1, sh_degree=3, lam=0.2,
               bg=(0.0, 0.0, 0.0), lr=DEFAULT_LR):
    """One optimisation step over a batch of views: mean of the per-view
    losses, gradients summed over views, one Adam update (FP64 state).

    ``moments`` is (m, v) dicts of float64 arrays or None (zeros).  Returns
    (loss, images, grads, new_params, (m, v))."""
    B = len(cams)
    grads = zero_grads(params)
    images, total = [], 0.0
    for cam, tgt in zip(cams, targets):
        pre, lists, out = render(cam, params, sh_degree, bg)
        L, dL = loss(out["image"], tgt, lam, grad_scale=1.0 / B)
        total += L / B
        sg = blend_backward(cam, pre, lists, dL, bg)
        preprocess_backward(cam, params, sg, sh_degree, grads)
        images.append(out["image"])
    if moments is None:
        moments = (zero_grads(params), zero_grads(params))
    m, v = moments
    new = {}
    for k, lr_k in zip(names_of(params), lr):
        p = np.asarray(params[k], np.float64).copy()
        adam(p, grads[k], m[k], v[k], lr_k, step)
        new[k] = p
    if is_dynamic(params):
        new["sigma_t"] = params["sigma_t"]
    return total, images, grads, new, (m, v)


# ---------------------------------------------------------------------------
# Locality-preserving order (Sec. 3.3 "Locality-preserving densification"):
# the z-order (Morton) permutation of the Gaussians' means.  An integer
# result decided in floating point: the quantisation is taken in float32,
# one rounding per operation, the precision the kernel decides it in (the
# paper fixes none).  The means must be finite.
# ---------------------------------------------------------------------------
MORTON_BITS = 10


def morton_quantise(means):
    """Per axis a: q_a = min(1023, floor((x_a - lo_a) * s_a)) with
    s_a = 1024 / (hi_a - lo_a) (0 when the box is flat along a), lo and hi
    the bounding box of the means; every operation in float32."""
    m = np.asarray(means, np.float32).reshape(-1, 3)
    q = np.zeros(m.shape, np.int64)
    if m.shape[0] == 0:
        return q
    top = (1 << MORTON_BITS) - 1
    for a in range(3):
        lo, hi = np.float32(m[:, a].min()), np.float32(m[:, a].max())
        ext = np.float32(hi - lo)
        s = np.float32(np.float32(1 << MORTON_BITS) / ext) if ext > 0 else np.float32(0.0)
        v = (m[:, a] - lo) * s                         # float32 difference, then product
        q[:, a] = np.clip(np.floor(v.astype(np.float64)), 0, top).astype(np.int64)
    return q


def morton_codes(means):
    """The z-order code: bit b of q_x, q_y, q_z goes to bit 3b, 3b + 1 and
    3b + 2 of the code (30 bits)."""
    q = morton_quantise(means)
    code = np.zeros(q.shape[0], np.int64)
    for b in range(MORTON_BITS):
        for a in range(3):
            code |= ((q[:, a] >> b) & 1) << (3 * b + a)
    return code.astype(np.uint32)


def morton_order(means):
    """Indices of the Gaussians in z-order; equal codes keep index order
    (numpy's stable sort is the library sort step)."""
    return np.argsort(morton_codes(means), kind="stable").astype(np.uint32)
