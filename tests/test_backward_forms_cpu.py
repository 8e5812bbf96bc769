"""The forms in which the CUDA blend backwards evaluate dC/dalpha (Eq. 4's
adjoint) agree with its plain definition in exact (FP64) arithmetic, so they
differ from it by float32 rounding only.  Per pixel, with fragments i front
to back, T_1 = 1, T_{i+1} = T_i (1 - alpha_i) and
C = sum_i alpha_i T_i c_i + T_{m+1} bg, the definition is
dC/dalpha_i = T_i c_i - S_i / (1 - alpha_i), S_i the colour of everything
behind i, weighted as blended (S_i = sum_{j>i} alpha_j T_j c_j + T_{m+1} bg).
The kernels use:
- back to front, T recovered by division from the final T and the colour
  behind A (A = bg behind the last, A <- alpha c + (1 - alpha) A):
  dC/dalpha_i = T_i (c_i - A_i);
- the same with only g . A kept, g = dL/dC of the pixel: a scalar recursion;
- front to back from the final colour (the per-Gaussian order):
  A_i = (C - C_{<=i}) / T_{i+1}.
A central difference of C in each alpha_i checks the definition itself."""
import numpy as np
import pytest


def _pixel(rng, m):
    alpha = rng.uniform(1.0 / 255.0, 0.99, m)
    c = rng.uniform(0.0, 1.0, (m, 3))
    bg = rng.uniform(0.0, 1.0, 3)
    g = rng.normal(size=3)
    return alpha, c, bg, g


def _colour(alpha, c, bg):
    T, C = 1.0, np.zeros(3)
    for a, ci in zip(alpha, c):
        C = C + a * T * ci
        T = T * (1.0 - a)
    return C + T * bg, T


def _definition(alpha, c, bg):
    m = len(alpha)
    T = np.cumprod(np.r_[1.0, 1.0 - alpha])       # T_1 .. T_{m+1}
    out = np.zeros((m, 3))
    for i in range(m):
        S = sum(alpha[j] * T[j] * c[j] for j in range(i + 1, m)) + T[m] * bg
        out[i] = T[i] * c[i] - S / (1.0 - alpha[i])
    return out


def _back_to_front(alpha, c, bg, T_final):
    m = len(alpha)
    out = np.zeros((m, 3))
    T, A = T_final, bg.copy()
    for i in range(m - 1, -1, -1):
        Ti = T / (1.0 - alpha[i])                   # T in front of fragment i
        out[i] = Ti * (c[i] - A)
        A = A + alpha[i] * (c[i] - A)
        T = Ti
    return out


def _back_to_front_scalar(alpha, c, bg, g, T_final):
    m = len(alpha)
    out = np.zeros(m)
    T, s = T_final, float(g @ bg)
    for i in range(m - 1, -1, -1):
        Ti = T / (1.0 - alpha[i])
        gc = float(g @ c[i]) - s
        out[i] = Ti * gc
        s = s + alpha[i] * gc
        T = Ti
    return out


def _front_to_back(alpha, c, C_final):
    m = len(alpha)
    out = np.zeros((m, 3))
    T, C = 1.0, np.zeros(3)
    for i in range(m):
        C = C + alpha[i] * T * c[i]
        Tn = T * (1.0 - alpha[i])
        R = (C_final - C) / Tn
        out[i] = T * (c[i] - R)
        T = Tn
    return out


@pytest.mark.parametrize("m", [1, 2, 7, 40])
def test_backward_forms_equal_the_definition(m):
    rng = np.random.default_rng(100 + m)
    for _ in range(20):
        alpha, c, bg, g = _pixel(rng, m)
        C, T_final = _colour(alpha, c, bg)
        ref = _definition(alpha, c, bg)
        scale = np.abs(ref).max() + 1.0
        np.testing.assert_allclose(_back_to_front(alpha, c, bg, T_final), ref, rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(_back_to_front_scalar(alpha, c, bg, g, T_final), ref @ g, rtol=0,
                                   atol=1e-12 * scale * np.abs(g).sum())
        np.testing.assert_allclose(_front_to_back(alpha, c, C), ref, rtol=0, atol=1e-9 * scale)


def test_definition_against_central_differences():
    rng = np.random.default_rng(7)
    alpha, c, bg, _ = _pixel(rng, 6)
    ref = _definition(alpha, c, bg)
    h = 1e-6
    for i in range(len(alpha)):
        up, dn = alpha.copy(), alpha.copy()
        up[i] += h
        dn[i] -= h
        fd = (_colour(up, c, bg)[0] - _colour(dn, c, bg)[0]) / (2 * h)
        np.testing.assert_allclose(fd, ref[i], rtol=1e-7, atol=1e-9)


def test_a_dropped_term_is_caught():
    """Leaving the background out of the colour behind (a plausible slip)
    breaks the agreement."""
    rng = np.random.default_rng(9)
    alpha, c, bg, _ = _pixel(rng, 5)
    _, T_final = _colour(alpha, c, bg)
    wrong = _back_to_front(alpha, c, np.zeros(3), T_final)
    assert np.abs(wrong - _definition(alpha, c, bg)).max() > 1e-3


# ---------------------------------------------------------------------------
# float32 evaluation near the early stop
# ---------------------------------------------------------------------------
F32 = np.float32
U32 = 2.0 ** -24        # unit roundoff of float32


def _near_stop_pixel(rng, m):
    """m fragments whose final T lies in [1e-4, 2e-4] (the stop keeps T >=
    1e-4), alphas in [1/255, 0.99], as float32."""
    while True:
        target = rng.uniform(1e-4, 2e-4)
        a = rng.uniform(0.05, 0.9, m - 1)
        ln = np.log1p(-a)
        ln *= np.log(target * rng.uniform(2.0, 90.0)) / ln.sum()
        a = np.clip(-np.expm1(ln), 1.0 / 255.0, 0.99)
        last = 1.0 - target / np.prod(1.0 - a)
        if 1.0 / 255.0 <= last <= 0.99:
            alpha = np.r_[a, last].astype(F32)
            return (alpha, rng.uniform(0.0, 1.0, (m, 3)).astype(F32),
                    rng.uniform(0.0, 1.0, 3).astype(F32), rng.normal(size=3).astype(F32))


def _colour32(alpha, c, bg):
    T, C = F32(1.0), np.zeros(3, F32)
    for a, ci in zip(alpha, c):
        C = (C + (a * T) * ci).astype(F32)
        T = F32(T * (F32(1.0) - a))
    return (C + T * bg).astype(F32), T


def _front_to_back32(alpha, c, C_final):
    out = np.zeros((len(alpha), 3))
    T, C = F32(1.0), np.zeros(3, F32)
    for i in range(len(alpha)):
        C = (C + (alpha[i] * T) * c[i]).astype(F32)
        Tn = F32(T * (F32(1.0) - alpha[i]))
        R = ((C_final - C) / Tn).astype(F32)
        out[i] = (T * (c[i] - R)).astype(F32)
        T = Tn
    return out


def _back_to_front_scalar32(alpha, c, bg, g, T_final):
    out = np.zeros(len(alpha))
    T, s = F32(T_final), F32(g @ bg)
    for i in range(len(alpha) - 1, -1, -1):
        Ti = F32(T / (F32(1.0) - alpha[i]))
        gc = F32(F32(g @ c[i]) - s)
        out[i] = F32(Ti * gc)
        s = F32(s + alpha[i] * gc)
        T = Ti
    return out


@pytest.mark.parametrize("m", [2, 9, 30, 60])
def test_float32_forms_near_the_stop(m):
    """The two forms in float32 on pixels driven to T near 1e-4, against the
    FP64 definition of the same float32 inputs.  The front-to-back form
    divides C - C_<=i by T_{i+1} >= 1e-4, so its rounding of C is amplified;
    fragment i's error stays within 2 m u (1 + max c + max bg) / (1 -
    alpha_i) (u = 2^-24), the scalar back-to-front form's within
    2 m u (1 + max c + max bg) |g|_1.  Over one pixel's fragments the
    relative L2 error stays below 5e-4 for the front-to-back form (reached
    with two or three near-opaque fragments, where every derivative is
    small) and 1e-4 for the back-to-front one: under the 1e-3 bar either
    backward order's gradients, sums over many pixels, are held to."""
    rng = np.random.default_rng(500 + m)
    for _ in range(200):
        alpha, c, bg, g = _near_stop_pixel(rng, m)
        A, C, BG, G = (x.astype(np.float64) for x in (alpha, c, bg, g))
        ref = _definition(A, C, BG)
        Cf, Tf = _colour32(alpha, c, bg)
        assert 0.9e-4 <= Tf <= 2.1e-4
        scale = m * U32 * (1.0 + C.max() + BG.max())
        f2b = _front_to_back32(alpha, c, Cf)
        err = np.abs(f2b - ref).max(axis=1)
        assert np.all(err <= 2.0 * scale / (1.0 - A)), (err * (1.0 - A) / scale).max()
        b2f = _back_to_front_scalar32(alpha, c, bg, g, Tf)
        assert np.all(np.abs(b2f - ref @ G) <= 2.0 * scale * np.abs(G).sum())
        assert np.linalg.norm(f2b - ref) <= 5e-4 * np.linalg.norm(ref)
        assert np.linalg.norm(b2f - ref @ G) <= 1e-4 * np.linalg.norm(ref @ G)
