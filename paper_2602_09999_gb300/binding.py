"""ctypes binding of libfastergs.so (include/fastergs.h).

Argument marshalling only: every function here has the name of the C entry
point it calls, turns a non-zero status into :class:`FGSError`, and does no
computation of its own.  Device buffers are passed as integer addresses
(``tensor.data_ptr()``); streams as integer ``cudaStream_t`` handles.

Loading fails loudly (RuntimeError) when the library has not been built:
there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build_lib

FGS_TILE = 16
FGS_MAX_VIEWS = 16
FGS_NUM_GROUPS = 8
FGS_F32, FGS_BF16, FGS_F16 = 0, 1, 2
FGS_FLAG_CAPACITY = 1
FGS_FLAG_NONFINITE = 2

(FGS_WS_HEADER, FGS_WS_SCREEN, FGS_WS_RECT, FGS_WS_LOCAL_OFF, FGS_WS_BLOCK_SUM, FGS_WS_KEYS,
 FGS_WS_VALS, FGS_WS_KEYS_ALT, FGS_WS_VALS_ALT, FGS_WS_SORT_HIST, FGS_WS_RANGES, FGS_WS_T_FINAL,
 FGS_WS_N_CONTRIB, FGS_WS_SCREEN_GRAD, FGS_WS_LOSS_MAPS, FGS_WS_LOSS_PART, FGS_WS_N_BLENDED,
 FGS_WS_TILE_QUEUE, FGS_WS_DEPTH_KEYS, FGS_WS_DEPTH_VALS, FGS_WS_DEPTH_KEYS_ALT,
 FGS_WS_DEPTH_VALS_ALT, FGS_WS_SORTED_OFF, FGS_WS_SORTED_BLOCK, FGS_WS_BUCKET_OFF,
 FGS_WS_BUCKET_TILE, FGS_WS_BUCKET_STATE, FGS_WS_PIXEL_FINAL, FGS_WS_NUM_SLOTS) = range(29)
FGS_WS_PER_GAUSSIAN = 1

STATUS = {0: "FGS_OK", -1: "FGS_ERR_NULL", -2: "FGS_ERR_SHAPE", -3: "FGS_ERR_SH_DEGREE",
          -4: "FGS_ERR_WORKSPACE", -5: "FGS_ERR_DTYPE", -6: "FGS_ERR_CUDA", -7: "FGS_ERR_VIEWS",
          -8: "FGS_ERR_ALIGN", -9: "FGS_ERR_ARG", -10: "FGS_ERR_TOO_LARGE"}
FGS_STATIC_SORT_MAX_PAIRS = 1 << 20

EXPORTED = ("fgs_workspace_size", "fgs_workspace_size_ex", "fgs_render_forward", "fgs_loss_l1_dssim",
            "fgs_render_backward", "fgs_render_backward_adam", "fgs_adam_step",
            "fgs_adam_step_device",
            "fgs_sort_scratch_bytes", "fgs_sort_pairs", "fgs_sort_pairs_static",
            "fgs_morton_scratch_bytes", "fgs_morton_order", "fgs_permute_params",
            "fgs_peak_fma", "fgs_peak_ex2", "fgs_peak_l2_read", "fgs_get_error",
            "fgs_profile_attach",
            "fgs_profile_count", "fgs_strerror", "fgs_flag_string")


class FGSError(RuntimeError):
    def __init__(self, func, code):
        self.code = code
        super().__init__(f"{func} -> {STATUS.get(code, code)}: {fgs_strerror(code)}")


class fgs_camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("near_plane", ctypes.c_float), ("cam_pos", ctypes.c_float * 3),
                ("time", ctypes.c_float)]


class fgs_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("data", ctypes.c_void_p * FGS_NUM_GROUPS),
                ("dtype", ctypes.c_int32 * FGS_NUM_GROUPS), ("sigma_t", ctypes.c_float)]


class fgs_tuning(ctypes.Structure):
    _fields_ = [("blend_pixels_per_thread", ctypes.c_int32), ("blend_batch", ctypes.c_int32),
                ("blend_schedule", ctypes.c_int32), ("blend_backward", ctypes.c_int32),
                ("backward_pixels_per_thread", ctypes.c_int32), ("backward_batch", ctypes.c_int32),
                ("depth_sort_digit_bits", ctypes.c_int32), ("tile_sort_digit_bits", ctypes.c_int32),
                ("duplicate_order", ctypes.c_int32)]


BLEND_CONFIGS = ((1, 256), (2, 128), (2, 256), (4, 64), (4, 128), (4, 256))
SORT_DIGIT_BITS = (8, 11)   # radix digit widths of the render path's two sorts
FGS_SCHEDULE_QUEUE, FGS_SCHEDULE_GRID = 0, 1
BLEND_SCHEDULES = (FGS_SCHEDULE_QUEUE, FGS_SCHEDULE_GRID)
FGS_BACKWARD_PER_PIXEL, FGS_BACKWARD_PER_GAUSSIAN = 0, 1
FGS_DUPLICATE_STRIDED, FGS_DUPLICATE_SPLIT = 0, 1
DUPLICATE_ORDERS = (FGS_DUPLICATE_STRIDED, FGS_DUPLICATE_SPLIT)


class fgs_workspace_layout(ctypes.Structure):
    _fields_ = [("total_bytes", ctypes.c_size_t),
                ("offset", ctypes.c_size_t * FGS_WS_NUM_SLOTS),
                ("bytes", ctypes.c_size_t * FGS_WS_NUM_SLOTS),
                ("n", ctypes.c_int64), ("k_max", ctypes.c_int64),
                ("n_views", ctypes.c_int32), ("total_tiles", ctypes.c_int32),
                ("total_pixels", ctypes.c_int64), ("sort_bits", ctypes.c_int32),
                ("sorted_in_alt", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("tuning", fgs_tuning)]


class fgs_adam_state(ctypes.Structure):
    _fields_ = [("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
                ("lr", ctypes.c_float * FGS_NUM_GROUPS), ("lr_means_final", ctypes.c_float),
                ("decay_steps", ctypes.c_int32), ("step", ctypes.c_int32),
                ("step_size", ctypes.c_float * FGS_NUM_GROUPS), ("inv_bc2_sqrt", ctypes.c_float),
                ("beta1_f", ctypes.c_float), ("beta2_f", ctypes.c_float),
                ("one_minus_beta1_f", ctypes.c_float), ("one_minus_beta2_f", ctypes.c_float),
                ("eps_f", ctypes.c_float)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return build_lib.LIB


def lib():
    """The loaded library; raises when it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(
                    f"libfastergs.so not found at {path}: build it first "
                    "(python -c 'import __graft_entry__ as g; g.build()')")
            L = ctypes.CDLL(path)
            P, I32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
            L.fgs_workspace_size.argtypes = [I64, P, I32, I64, P]
            L.fgs_workspace_size_ex.argtypes = [I64, P, I32, I64, I32, P]
            L.fgs_render_forward.argtypes = [P, P, P, I32, P, P, P, P, P]
            L.fgs_loss_l1_dssim.argtypes = [P, P, P, P, P, ctypes.c_float, P, P, P]
            L.fgs_render_backward.argtypes = [P, P, P, I32, P, P, P, P, P, P]
            L.fgs_render_backward_adam.argtypes = [P, P, P, I32, P, P, P, P, P, P, P, P, P]
            L.fgs_adam_step.argtypes = [P, P, P, P, P, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, I32, P]
            L.fgs_adam_step_device.argtypes = [P, P, P, P, P, P]
            L.fgs_sort_scratch_bytes.argtypes = [I64]
            L.fgs_sort_scratch_bytes.restype = SZ
            L.fgs_sort_pairs.argtypes = [P, P, P, P, I64, I32, P, SZ, P, P]
            L.fgs_sort_pairs_static.argtypes = [P, P, I64, I32, P]
            L.fgs_morton_scratch_bytes.argtypes = [I64]
            L.fgs_morton_scratch_bytes.restype = SZ
            L.fgs_morton_order.argtypes = [P, I64, P, P, P, SZ, P]
            L.fgs_permute_params.argtypes = [P, P, P, P]
            L.fgs_peak_fma.argtypes = [I32, P, P, P]
            L.fgs_peak_ex2.argtypes = [I32, P, P, P]
            L.fgs_peak_l2_read.argtypes = [P, I64, I32, P, P, P]
            L.fgs_get_error.argtypes = [P, P, P, I32, P]
            L.fgs_profile_attach.argtypes = [P, P, I32]
            L.fgs_profile_count.argtypes = []
            L.fgs_strerror.argtypes = [ctypes.c_int]
            L.fgs_strerror.restype = ctypes.c_char_p
            L.fgs_flag_string.argtypes = [ctypes.c_uint32]
            L.fgs_flag_string.restype = ctypes.c_char_p
            for name in EXPORTED:
                if name not in ("fgs_sort_scratch_bytes", "fgs_morton_scratch_bytes",
                                "fgs_strerror", "fgs_flag_string"):
                    getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def _check(func, rc):
    if rc != 0:
        raise FGSError(func, rc)


def _ref(x):
    return ctypes.byref(x) if x is not None else None


def _float3(v):
    return (ctypes.c_float * 3)(*[float(a) for a in v])


def fgs_profile_attach(events, labels, capacity):
    """events: ctypes array of cudaEvent_t handles (c_void_p); labels:
    ctypes array of c_char_p of the same length (filled by the library)."""
    _check("fgs_profile_attach", lib().fgs_profile_attach(events, labels, int(capacity)))


def fgs_profile_count() -> int:
    return int(lib().fgs_profile_count())


def fgs_strerror(code: int) -> str:
    return lib().fgs_strerror(int(code)).decode()


def fgs_flag_string(flag: int) -> str:
    return lib().fgs_flag_string(int(flag)).decode()


def fgs_workspace_size(n, cams_host, n_views, k_max) -> fgs_workspace_layout:
    out = fgs_workspace_layout()
    _check("fgs_workspace_size",
           lib().fgs_workspace_size(int(n), cams_host, int(n_views), int(k_max), ctypes.byref(out)))
    return out


def fgs_workspace_size_ex(n, cams_host, n_views, k_max, flags) -> fgs_workspace_layout:
    out = fgs_workspace_layout()
    _check("fgs_workspace_size_ex",
           lib().fgs_workspace_size_ex(int(n), cams_host, int(n_views), int(k_max), int(flags),
                                       ctypes.byref(out)))
    return out


def fgs_render_forward(ws, layout, params, sh_degree, cams_host, cams_device, bg, images, stream):
    _check("fgs_render_forward",
           lib().fgs_render_forward(ws, ctypes.byref(layout), ctypes.byref(params), int(sh_degree),
                                    cams_host, cams_device, _float3(bg), images, stream))


def fgs_loss_l1_dssim(ws, layout, cams_host, images, targets, lam, loss_out, dl_dimages, stream):
    _check("fgs_loss_l1_dssim",
           lib().fgs_loss_l1_dssim(ws, ctypes.byref(layout), cams_host, images, targets,
                                   float(lam), loss_out, dl_dimages, stream))


def fgs_render_backward(ws, layout, params, sh_degree, cams_host, cams_device, bg, dl_dimages,
                        grads, stream):
    _check("fgs_render_backward",
           lib().fgs_render_backward(ws, ctypes.byref(layout), ctypes.byref(params),
                                     int(sh_degree), cams_host, cams_device, _float3(bg),
                                     dl_dimages, ctypes.byref(grads), stream))


def fgs_render_backward_adam(ws, layout, params, sh_degree, cams_host, cams_device, bg, dl_dimages,
                             exp_avg, exp_avg_sq, state_device, grads, stream):
    """grads: an fgs_params or None (the gradients are then not stored)."""
    _check("fgs_render_backward_adam",
           lib().fgs_render_backward_adam(ws, ctypes.byref(layout), ctypes.byref(params),
                                          int(sh_degree), cams_host, cams_device, _float3(bg),
                                          dl_dimages, ctypes.byref(exp_avg),
                                          ctypes.byref(exp_avg_sq), state_device,
                                          ctypes.byref(grads) if grads is not None else None,
                                          stream))


def fgs_adam_step(params, grads, exp_avg, exp_avg_sq, lr, beta1, beta2, eps, step, stream):
    lr = [float(a) for a in lr][:FGS_NUM_GROUPS]
    lr_arr = (ctypes.c_float * FGS_NUM_GROUPS)(*(lr + [0.0] * (FGS_NUM_GROUPS - len(lr))))
    _check("fgs_adam_step",
           lib().fgs_adam_step(ctypes.byref(params), ctypes.byref(grads), ctypes.byref(exp_avg),
                               ctypes.byref(exp_avg_sq), lr_arr, float(beta1), float(beta2),
                               float(eps), int(step), stream))


def fgs_adam_step_device(params, grads, exp_avg, exp_avg_sq, state_device, stream):
    _check("fgs_adam_step_device",
           lib().fgs_adam_step_device(ctypes.byref(params), ctypes.byref(grads),
                                      ctypes.byref(exp_avg), ctypes.byref(exp_avg_sq),
                                      state_device, stream))


def fgs_sort_scratch_bytes(n) -> int:
    return int(lib().fgs_sort_scratch_bytes(int(n)))


def fgs_sort_pairs(keys, vals, keys_alt, vals_alt, n, bits, scratch, scratch_bytes, stream) -> int:
    """Returns 1 when the sorted result is in the *_alt buffers."""
    alt = ctypes.c_int32(0)
    _check("fgs_sort_pairs",
           lib().fgs_sort_pairs(keys, vals, keys_alt, vals_alt, int(n), int(bits), scratch,
                                int(scratch_bytes), ctypes.byref(alt), stream))
    return int(alt.value)


def fgs_sort_pairs_static(keys, vals, n, bits, stream):
    """In-place sort with the library's own scratch (no allocation)."""
    _check("fgs_sort_pairs_static",
           lib().fgs_sort_pairs_static(keys, vals, int(n), int(bits), stream))


def fgs_morton_scratch_bytes(n) -> int:
    return int(lib().fgs_morton_scratch_bytes(int(n)))


def fgs_morton_order(means, n, order, codes, scratch, scratch_bytes, stream):
    """z-order permutation of the means into `order` (and the sorted codes
    into `codes`, unless it is None)."""
    _check("fgs_morton_order",
           lib().fgs_morton_order(means, int(n), order, codes, scratch, int(scratch_bytes), stream))


def fgs_permute_params(src, dst, order, stream):
    """dst rows = src rows taken in `order` (None: a plain copy)."""
    _check("fgs_permute_params",
           lib().fgs_permute_params(_ref(src), _ref(dst), order, stream))


def fgs_peak_fma(iters, out, stream) -> int:
    """Launches the FP32 FMA microbenchmark; returns its grid (CTAs of 256)."""
    grid = ctypes.c_int32(0)
    _check("fgs_peak_fma", lib().fgs_peak_fma(int(iters), out, ctypes.byref(grid), stream))
    return int(grid.value)


def fgs_peak_ex2(iters, out, stream) -> int:
    grid = ctypes.c_int32(0)
    _check("fgs_peak_ex2", lib().fgs_peak_ex2(int(iters), out, ctypes.byref(grid), stream))
    return int(grid.value)


def fgs_peak_l2_read(buf, n4, reps, out, stream) -> int:
    grid = ctypes.c_int32(0)
    _check("fgs_peak_l2_read",
           lib().fgs_peak_l2_read(buf, int(n4), int(reps), out, ctypes.byref(grid), stream))
    return int(grid.value)


def fgs_get_error(ws, clear=False, stream=None):
    """Synchronises; returns (flags, instances)."""
    flags = ctypes.c_uint32(0)
    inst = ctypes.c_uint64(0)
    _check("fgs_get_error", lib().fgs_get_error(ws, ctypes.byref(flags), ctypes.byref(inst),
                                                1 if clear else 0, stream))
    return int(flags.value), int(inst.value)


def camera_array(cams):
    """Host array of fgs_camera from objects with R, t, fx, fy, cx, cy,
    width, height, near, cam_pos (e.g. scenes.Camera)."""
    arr = (fgs_camera * len(cams))()
    for a, c in zip(arr, cams):
        R = [float(x) for x in list(c.R.reshape(9))]
        for i in range(9):
            a.R[i] = R[i]
        for i in range(3):
            a.t[i] = float(c.t[i])
            a.cam_pos[i] = float(c.cam_pos[i])
        a.fx, a.fy, a.cx, a.cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        a.width, a.height = int(c.width), int(c.height)
        a.near_plane = float(c.near)
        a.time = float(getattr(c, "time", 0.0))
    return arr


def params_struct(n, ptrs, dtypes, sigma_t=0.0) -> fgs_params:
    """6 groups (static Gaussians) or 8 (dynamic: velocity and t0 too)."""
    p = fgs_params()
    p.n = int(n)
    for g in range(len(ptrs)):
        p.data[g] = int(ptrs[g])
        p.dtype[g] = int(dtypes[g])
    p.sigma_t = float(sigma_t)
    return p
