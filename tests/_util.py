"""Small helpers shared by the tests (no method arithmetic)."""
import numpy as np

from paper_2602_09999_gb300 import scenes


def axis_camera(W=33, H=33, f=50.0):
    """Camera at the world origin looking down +z (R = I, t = 0)."""
    return scenes.Camera(R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32), fx=f, fy=f,
                         cx=W / 2.0, cy=H / 2.0, width=W, height=H, near=0.2,
                         cam_pos=np.zeros(3, np.float32))


def make_params(means, log_scales, quats, logits, dc, rest=None, dtype=np.float32):
    means = np.asarray(means, dtype).reshape(-1, 3)
    n = means.shape[0]
    rest = np.zeros((n, 15, 3), dtype) if rest is None else np.asarray(rest, dtype)
    return dict(means=means, log_scales=np.asarray(log_scales, dtype).reshape(n, 3),
                quats=np.asarray(quats, dtype).reshape(n, 4),
                opacity=np.asarray(logits, dtype).reshape(n),
                sh_dc=np.asarray(dc, dtype).reshape(n, 3), sh_rest=rest.reshape(n, 15, 3))


def iso_gaussians(depths, sigmas, opacities, colours, offsets=None):
    """Isotropic Gaussians on (or near) the optical axis of axis_camera."""
    n = len(depths)
    offsets = np.zeros((n, 2)) if offsets is None else np.asarray(offsets, np.float64)
    means = np.stack([offsets[:, 0], offsets[:, 1], np.asarray(depths, np.float64)], 1)
    ls = np.repeat(np.log(np.asarray(sigmas, np.float64))[:, None], 3, 1)
    q = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    o = np.asarray(opacities, np.float64)
    logits = np.log(o / (1.0 - o))
    return make_params(means, ls, q, logits, colours, dtype=np.float64)


Y00 = 0.5 / np.sqrt(np.pi)
