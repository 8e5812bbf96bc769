// fgs_common.cuh -- definitions shared by the sm_103a kernels of libfastergs.
//
// Threshold constants of Faster-GS (arXiv 2602.09999):
//   tau_alpha = 1/255 (Sec. 3.2 "Splat Bounding"), alpha clamp 0.99 and
//   early-stop transmittance 1e-4 (Suppl. B.1), degenerate quaternion norm
//   1e-4 and 2D-covariance determinant 1e-6 (Suppl. B.1), 2D dilation 0.3
//   (Suppl. C, Eq. original_2dfilter), 16x16 tiles (Sec. 3.1).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fastergs.h"

namespace fgs {

constexpr int kTile = FGS_TILE;
constexpr int kTilePixels = kTile * kTile;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kQNormMin = 1e-4f;
constexpr float kDetMin = 1e-6f;
constexpr float kDilation = 0.3f;
constexpr int kPreBlock = 128;  // Gaussians per preprocess CTA (scan granularity)

// Per-view sizes and prefix offsets, passed to kernels by value.  Sizes are
// fixed for the lifetime of a captured graph; poses come from device memory.
struct ViewTable {
    int32_t n_views;
    int32_t total_tiles;
    int64_t total_pixels;
    int32_t width[FGS_MAX_VIEWS];
    int32_t height[FGS_MAX_VIEWS];
    int32_t tiles_x[FGS_MAX_VIEWS];
    int32_t tile_off[FGS_MAX_VIEWS + 1];
    int64_t pix_off[FGS_MAX_VIEWS + 1];
};

// Screen-space state of one (view, Gaussian): 48 bytes, read by the blend
// kernels as three 16-byte loads.  The conic is stored in eigen form (see
// EigenConic below).
struct alignas(16) Screen {
    float4 q0;  // mu2D.x, mu2D.y, conic eigenvalues lb >= ls
    float4 q1;  // major-axis direction (cos, sin), opacity, depth
    float4 q2;  // rgb, bits: clamp mask (bits 0..2) | visible (bit 3)
};

// Tile set of one (view, Gaussian): its tile rectangle (inclusive; x0 > x1
// when it is not rendered), for rectangles of at most 32 tiles the tiles
// that survive culling (bit t = row-major tile t of the rectangle), so the
// duplication pass need not test them again, and the number of kept tiles.
struct alignas(16) TileRect {
    ushort4 r;
    uint32_t keep;
    uint32_t count;
};

// Opacity-aware extent (Sec. 3.2): alpha = o G reaches 1/255 where
// d^T conic d <= k = 2 ln(255 o).  Preprocess, duplication and the blend
// masks all derive k from the stored opacity with this one expression, so
// their tile decisions agree bit for bit.
// Dynamic Gaussians (Sec. 3.4, linear-velocity form of the conditional
// Gaussian): at time t the mean is mu + v (t - t0) and the opacity is
// scaled by the temporal marginal exp(-(t - t0)^2 / (2 sigma_t^2)).
struct Motion {
    const float* vel;  // [n,3] or nullptr (static Gaussians)
    const float* t0;   // [n]
    float inv_var;     // 1 / sigma_t^2
};

__device__ __forceinline__ float temporal_weight(float dt, float inv_var)
{
    return expf(-0.5f * dt * dt * inv_var);
}

__device__ __forceinline__ float opacity_k(float o)
{
    return fmaxf(2.0f * __logf(255.0f * o), 0.0f);
}

// Screen-space gradient accumulators of one (view, Gaussian): dL/dmu2D,
// dL/dSigma2D as the full symmetric matrix [[H00, H01], [H01, H11]] (the
// conic gradient mapped through d conic = -conic dSigma conic), dL/do and
// dL/drgb.
struct alignas(16) ScreenGrad {
    float4 g0;  // d mu.x, d mu.y, H00, H01
    float4 g1;  // H11, d o, d r, d g
    float4 g2;  // d b(lue), unused x3
};

struct WsHeader {
    uint32_t flags;
    uint32_t reserved;
    unsigned long long instances;  // total (Gaussian, tile) instances of the last forward
    uint32_t counters[4];
};

__host__ __device__ inline int view_of_tile(const ViewTable& vt, int tile)
{
    int v = 0;
    while (v + 1 < vt.n_views && tile >= vt.tile_off[v + 1]) ++v;
    return v;
}

struct Cam {
    float R[9], t[3], fx, fy, cx, cy, near_plane, pos[3], time;
    int width, height;
};

__device__ inline Cam load_cam(const fgs_camera* cams, int v)
{
    const fgs_camera* c = cams + v;
    Cam k;
#pragma unroll
    for (int i = 0; i < 9; ++i) k.R[i] = __ldg(&c->R[i]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        k.t[i] = __ldg(&c->t[i]);
        k.pos[i] = __ldg(&c->cam_pos[i]);
    }
    k.fx = __ldg(&c->fx);
    k.fy = __ldg(&c->fy);
    k.cx = __ldg(&c->cx);
    k.cy = __ldg(&c->cy);
    k.near_plane = __ldg(&c->near_plane);
    k.time = __ldg(&c->time);
    k.width = __ldg(&c->width);
    k.height = __ldg(&c->height);
    return k;
}

// ---------------------------------------------------------------------------
// Storage-type helpers (SH and Adam moments may be bf16 / fp16)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float to_f32(__half x) { return __half2float(x); }
template <typename T> __device__ __forceinline__ T from_f32(float x);
template <> __device__ __forceinline__ float from_f32<float>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ __half from_f32<__half>(float x) { return __float2half_rn(x); }

// ---------------------------------------------------------------------------
// Decisions that two kernels must take bit-identically are written with
// explicit round-to-nearest intrinsics, so no FMA contraction choice of the
// compiler can make them differ between call sites.
// ---------------------------------------------------------------------------

// The conic (inverse dilated 2D covariance) is kept in eigen form: the two
// eigenvalues (lb >= ls) and the unit eigenvector (c, s) of the small one,
// i.e. the major axis of the splat.  With e = (c, s),
//   q(d) = d^T conic d = ls (e . d)^2 + lb (e_perp . d)^2,
// a sum of two non-negative terms.  Storing (a, b, c) instead loses the small
// eigenvalue of needle-like splats (a c - b^2 cancels), which moves q by
// percents at pixels far along the needle; the eigen form is computed from
// the covariance itself (lmax by a sum of non-negative terms, lmin = det /
// lmax with the Cauchy-Binet determinant), so it stays accurate.
struct EigenConic {
    float lb, ls, c, s;  // eigenvalues and the major-axis direction
};

__device__ __forceinline__ EigenConic eigen_from_stored(float lb, float ls, float c, float s)
{
    EigenConic e;
    e.lb = lb;
    e.ls = ls;
    e.c = c;
    e.s = s;
    return e;
}

__device__ __forceinline__ float eigen_q(const EigenConic& e, float dx, float dy)
{
    const float u = __fmaf_rn(e.c, dx, __fmul_rn(e.s, dy));    // along the major axis
    const float w = __fmaf_rn(e.c, dy, -__fmul_rn(e.s, dx));   // across it
    return __fmaf_rn(__fmul_rn(e.ls, u), u, __fmul_rn(__fmul_rn(e.lb, w), w));
}

// Tile culling of Sec. 3.2 (the per-tile maximum of the Gaussian): minimum
// of the quadratic form over the box of the tile's pixel centres (offsets
// from the mean); keep the tile iff it is <= k.  The minimum of a convex
// quadratic over a box is 0 when the mean is inside, else it lies on an edge,
// where the 1D minimiser is clamped to the edge.  With the conic entries
// a = ls c^2 + lb s^2, b = (ls - lb) s c, cc = ls s^2 + lb c^2, the minimiser
// on the edge x = X lies at y = ry X (ry = -b / cc) and on the edge y = Y at
// x = rx Y (rx = -b / a); these slopes are per Gaussian (make_cull), so the
// per-tile test is multiplications, clamps and four evaluations of the form.
struct TileCull {
    float mx, my, k, rx, ry;
    EigenConic e;
};

__device__ __forceinline__ TileCull make_cull(float mx, float my, const EigenConic& e, float k)
{
    TileCull c;
    c.mx = mx;
    c.my = my;
    c.k = k;
    c.e = e;
    const float a = __fmaf_rn(e.ls, __fmul_rn(e.c, e.c), __fmul_rn(e.lb, __fmul_rn(e.s, e.s)));
    const float b = __fmul_rn(__fsub_rn(e.ls, e.lb), __fmul_rn(e.s, e.c));
    const float cc = __fmaf_rn(e.ls, __fmul_rn(e.s, e.s), __fmul_rn(e.lb, __fmul_rn(e.c, e.c)));
    c.ry = __fdiv_rn(-b, cc);
    c.rx = __fdiv_rn(-b, a);
    return c;
}

__device__ __forceinline__ bool tile_keep(const TileCull& c, int tx, int ty, int width, int height)
{
    const float x_lo = __fadd_rn((float)(tx * kTile), 0.5f);
    const float x_hi = fminf(__fadd_rn((float)(tx * kTile + kTile - 1), 0.5f), __fadd_rn((float)width, -0.5f));
    const float y_lo = __fadd_rn((float)(ty * kTile), 0.5f);
    const float y_hi = fminf(__fadd_rn((float)(ty * kTile + kTile - 1), 0.5f), __fadd_rn((float)height, -0.5f));
    const float x0 = __fsub_rn(x_lo, c.mx), x1 = __fsub_rn(x_hi, c.mx);
    const float y0 = __fsub_rn(y_lo, c.my), y1 = __fsub_rn(y_hi, c.my);
    if (x0 <= 0.0f && 0.0f <= x1 && y0 <= 0.0f && 0.0f <= y1) return true;
    float best = eigen_q(c.e, x0, fminf(fmaxf(__fmul_rn(c.ry, x0), y0), y1));
    best = fminf(best, eigen_q(c.e, x1, fminf(fmaxf(__fmul_rn(c.ry, x1), y0), y1)));
    best = fminf(best, eigen_q(c.e, fminf(fmaxf(__fmul_rn(c.rx, y0), x0), x1), y0));
    best = fminf(best, eigen_q(c.e, fminf(fmaxf(__fmul_rn(c.rx, y1), x0), x1), y1));
    return best <= c.k;
}

// One evaluated fragment: alpha = min(0.99, o G), G = exp(power) and
// whether the clamp is active.
struct Frag {
    float alpha, G;
    bool clamped;
};

// ---------------------------------------------------------------------------
// Real SH basis (Condon-Shortley phase, orthonormal), degree <= 3, at a unit
// direction; coefficient k = l*l + l + m.
// ---------------------------------------------------------------------------
struct SHC {
    static constexpr float c0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
    static constexpr float c1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
    static constexpr float c2a = 1.0925484305920792f;   // sqrt(15/pi)/2
    static constexpr float c2b = 0.31539156525252005f;  // sqrt(5/pi)/4
    static constexpr float c2c = 0.5462742152960396f;   // sqrt(15/pi)/4
    static constexpr float c3a = 0.5900435899266435f;   // sqrt(35/(2 pi))/4
    static constexpr float c3b = 2.890611442640554f;    // sqrt(105/pi)/2
    static constexpr float c3c = 0.4570457994644658f;   // sqrt(21/(2 pi))/4
    static constexpr float c3d = 0.3731763325901154f;   // sqrt(7/pi)/4
    static constexpr float c3e = 1.445305721320277f;    // sqrt(105/pi)/4
};

__device__ __forceinline__ void sh_basis(float x, float y, float z, int degree, float Y[16])
{
    Y[0] = SHC::c0;
#pragma unroll
    for (int k = 1; k < 16; ++k) Y[k] = 0.0f;
    if (degree < 1) return;
    Y[1] = -SHC::c1 * y;
    Y[2] = SHC::c1 * z;
    Y[3] = -SHC::c1 * x;
    if (degree < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = SHC::c2a * x * y;
    Y[5] = -SHC::c2a * y * z;
    Y[6] = SHC::c2b * (2.0f * zz - xx - yy);
    Y[7] = -SHC::c2a * x * z;
    Y[8] = SHC::c2c * (xx - yy);
    if (degree < 3) return;
    Y[9] = -SHC::c3a * y * (3.0f * xx - yy);
    Y[10] = SHC::c3b * x * y * z;
    Y[11] = -SHC::c3c * y * (4.0f * zz - xx - yy);
    Y[12] = SHC::c3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = -SHC::c3c * x * (4.0f * zz - xx - yy);
    Y[14] = SHC::c3e * z * (xx - yy);
    Y[15] = -SHC::c3a * x * (xx - 3.0f * yy);
}

// sh_basis with every rounding explicit (see quat_to_rot_rn).
__device__ __forceinline__ void sh_basis_rn(float x, float y, float z, int degree, float Y[16])
{
    Y[0] = SHC::c0;
#pragma unroll
    for (int k = 1; k < 16; ++k) Y[k] = 0.0f;
    if (degree < 1) return;
    Y[1] = __fmul_rn(-SHC::c1, y);
    Y[2] = __fmul_rn(SHC::c1, z);
    Y[3] = __fmul_rn(-SHC::c1, x);
    if (degree < 2) return;
    const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    const float xmy = __fsub_rn(xx, yy);                                     // x^2 - y^2
    const float r2 = __fsub_rn(__fsub_rn(__fmul_rn(2.0f, zz), xx), yy);      // 2 z^2 - x^2 - y^2
    const float r4 = __fsub_rn(__fsub_rn(__fmul_rn(4.0f, zz), xx), yy);      // 4 z^2 - x^2 - y^2
    Y[4] = __fmul_rn(__fmul_rn(SHC::c2a, x), y);
    Y[5] = __fmul_rn(__fmul_rn(-SHC::c2a, y), z);
    Y[6] = __fmul_rn(SHC::c2b, r2);
    Y[7] = __fmul_rn(__fmul_rn(-SHC::c2a, x), z);
    Y[8] = __fmul_rn(SHC::c2c, xmy);
    if (degree < 3) return;
    Y[9] = __fmul_rn(__fmul_rn(-SHC::c3a, y), __fmaf_rn(3.0f, xx, -yy));
    Y[10] = __fmul_rn(__fmul_rn(__fmul_rn(SHC::c3b, x), y), z);
    Y[11] = __fmul_rn(__fmul_rn(-SHC::c3c, y), r4);
    Y[12] = __fmul_rn(__fmul_rn(SHC::c3d, z), __fmaf_rn(-3.0f, yy, __fmaf_rn(-3.0f, xx, __fmul_rn(2.0f, zz))));
    Y[13] = __fmul_rn(__fmul_rn(-SHC::c3c, x), r4);
    Y[14] = __fmul_rn(__fmul_rn(SHC::c3e, z), xmy);
    Y[15] = __fmul_rn(__fmul_rn(-SHC::c3a, x), __fmaf_rn(-3.0f, yy, xx));
}

// d/d(x, y, z) of sum_k coef[k] Y_k for the polynomial forms above.
__device__ __forceinline__ void sh_dir_grad(float x, float y, float z, int degree,
                                            const float coef[16], float g[3])
{
    g[0] = g[1] = g[2] = 0.0f;
    if (degree < 1) return;
    g[0] += -SHC::c1 * coef[3];
    g[1] += -SHC::c1 * coef[1];
    g[2] += SHC::c1 * coef[2];
    if (degree < 2) return;
    g[0] += SHC::c2a * y * coef[4] - SHC::c2a * z * coef[7] - 2.0f * SHC::c2b * x * coef[6] +
            2.0f * SHC::c2c * x * coef[8];
    g[1] += SHC::c2a * x * coef[4] - SHC::c2a * z * coef[5] - 2.0f * SHC::c2b * y * coef[6] -
            2.0f * SHC::c2c * y * coef[8];
    g[2] += -SHC::c2a * y * coef[5] + 4.0f * SHC::c2b * z * coef[6] - SHC::c2a * x * coef[7];
    if (degree < 3) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    g[0] += -SHC::c3a * 6.0f * x * y * coef[9] + SHC::c3b * y * z * coef[10] +
            SHC::c3c * 2.0f * x * y * coef[11] - SHC::c3d * 6.0f * x * z * coef[12] -
            SHC::c3c * (4.0f * zz - 3.0f * xx - yy) * coef[13] + SHC::c3e * 2.0f * x * z * coef[14] -
            SHC::c3a * (3.0f * xx - 3.0f * yy) * coef[15];
    g[1] += -SHC::c3a * (3.0f * xx - 3.0f * yy) * coef[9] + SHC::c3b * x * z * coef[10] -
            SHC::c3c * (4.0f * zz - xx - 3.0f * yy) * coef[11] - SHC::c3d * 6.0f * y * z * coef[12] +
            SHC::c3c * 2.0f * x * y * coef[13] - SHC::c3e * 2.0f * y * z * coef[14] +
            SHC::c3a * 6.0f * x * y * coef[15];
    g[2] += SHC::c3b * x * y * coef[10] - SHC::c3c * 8.0f * y * z * coef[11] +
            SHC::c3d * (6.0f * zz - 3.0f * xx - 3.0f * yy) * coef[12] -
            SHC::c3c * 8.0f * x * z * coef[13] + SHC::c3e * (xx - yy) * coef[14];
}

// Rotation matrix of a unit quaternion (w, x, y, z), Hamilton convention.
__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float R[9])
{
    R[0] = 1.0f - 2.0f * (y * y + z * z);
    R[1] = 2.0f * (x * y - w * z);
    R[2] = 2.0f * (x * z + w * y);
    R[3] = 2.0f * (x * y + w * z);
    R[4] = 1.0f - 2.0f * (x * x + z * z);
    R[5] = 2.0f * (y * z - w * x);
    R[6] = 2.0f * (x * z - w * y);
    R[7] = 2.0f * (y * z + w * x);
    R[8] = 1.0f - 2.0f * (x * x + y * y);
}

// The same rotation with every rounding explicit.  The forward preprocess
// uses the _rn forms (this, sh_basis_rn, and explicit roundings in its
// projection and colour), so its static and motion instantiations, inlined
// into different kernels, compute the same screen state bit for bit whatever
// the compiler contracts around them.  The backward keeps the plain forms.
__device__ __forceinline__ void quat_to_rot_rn(float w, float x, float y, float z, float R[9])
{
    R[0] = __fmaf_rn(-2.0f, __fmaf_rn(y, y, __fmul_rn(z, z)), 1.0f);
    R[1] = __fmul_rn(2.0f, __fmaf_rn(x, y, -__fmul_rn(w, z)));
    R[2] = __fmul_rn(2.0f, __fmaf_rn(x, z, __fmul_rn(w, y)));
    R[3] = __fmul_rn(2.0f, __fmaf_rn(x, y, __fmul_rn(w, z)));
    R[4] = __fmaf_rn(-2.0f, __fmaf_rn(x, x, __fmul_rn(z, z)), 1.0f);
    R[5] = __fmul_rn(2.0f, __fmaf_rn(y, z, -__fmul_rn(w, x)));
    R[6] = __fmul_rn(2.0f, __fmaf_rn(x, z, -__fmul_rn(w, y)));
    R[7] = __fmul_rn(2.0f, __fmaf_rn(y, z, __fmul_rn(w, x)));
    R[8] = __fmaf_rn(-2.0f, __fmaf_rn(x, x, __fmul_rn(y, y)), 1.0f);
}

__device__ __forceinline__ void set_flag(WsHeader* h, uint32_t bit) { atomicOr(&h->flags, bit); }

// Records the next attached profiling event (no-op unless attached).
void profile_mark(cudaStream_t st, const char* label);

}  // namespace fgs
