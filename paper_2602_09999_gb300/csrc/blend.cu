// blend.cu -- per-tile alpha blending and its backward (sm_103a).
//
// Forward (Eq. 3-4, Sec. 3.1 16x16 tiles, Suppl. B.1 rules): one CTA per
// tile of any view, one thread per pixel.  The CTA streams its sorted list
// in batches of 256 entries staged in shared memory; each pixel blends front
// to back, skips alpha < 1/255, clamps alpha at 0.99 and stops before an
// entry that would take T below 1e-4.  It stores C + T bg, the final T and
// the list position of the last blended entry, so the backward recomputes
// the blend instead of storing per-fragment state.
//
// Backward (Sec. 3.2 "Per-Gaussian Backward" discusses the cost of the
// atomics this design reduces): the CTA walks the same list back to front
// from the largest last-contributor position of its pixels; each pixel
// recovers T_i = T_{i+1} / (1 - alpha_i) and the colour behind it,
// A_i = alpha_{i+1} c_{i+1} + (1 - alpha_{i+1}) A_{i+1} (A = bg behind the
// last), so dC/dalpha_i = T_i (c_i - A_i) and dC/dc_i = alpha_i T_i.  The 9
// per-fragment gradients are summed over the warp with shuffles, over the
// CTA with shared-memory atomics, and leave the CTA as one set of global
// vector atomics per (instance, CTA).
#include "fgs_common.cuh"

namespace fgs {

constexpr int kBlendThreads = kTilePixels;  // 256

struct TilePix {
    int v, tile_local, px, py, W, H;
    bool inside;
};

__device__ __forceinline__ TilePix tile_pixel(const ViewTable& vt, int tile)
{
    TilePix t;
    t.v = view_of_tile(vt, tile);
    t.tile_local = tile - vt.tile_off[t.v];
    const int tx = t.tile_local % vt.tiles_x[t.v], ty = t.tile_local / vt.tiles_x[t.v];
    t.px = tx * kTile + (threadIdx.x % kTile);
    t.py = ty * kTile + (threadIdx.x / kTile);
    t.W = vt.width[t.v];
    t.H = vt.height[t.v];
    t.inside = t.px < t.W && t.py < t.H;
    return t;
}

__global__ void __launch_bounds__(kBlendThreads)
blend_fwd_kernel(ViewTable vt, int64_t n, const uint2* __restrict__ ranges,
                 const uint32_t* __restrict__ gids, const Screen* __restrict__ screen, float bg0,
                 float bg1, float bg2, float* __restrict__ images, float* __restrict__ T_final,
                 uint32_t* __restrict__ n_contrib)
{
    __shared__ float4 s_q0[kBlendThreads];
    __shared__ float2 s_co[kBlendThreads];
    __shared__ float4 s_rgb[kBlendThreads];
    const int tile = blockIdx.x;
    const TilePix tp = tile_pixel(vt, tile);
    const uint2 range = ranges[tile];
    const float fx = (float)tp.px + 0.5f, fy = (float)tp.py + 0.5f;
    const Screen* scr = screen + (int64_t)tp.v * n;
    float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0;
    bool done = !tp.inside;
    for (uint32_t start = range.x; start < range.y; start += kBlendThreads) {
        if (__syncthreads_count(done) == kBlendThreads) break;
        const uint32_t j = start + threadIdx.x;
        if (j < range.y) {
            const Screen rec = scr[gids[j]];
            s_q0[threadIdx.x] = rec.q0;
            s_co[threadIdx.x] = make_float2(rec.q1.x, rec.q1.y);
            s_rgb[threadIdx.x] = rec.q2;
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)kBlendThreads, range.y - start);
        for (int jj = 0; !done && jj < cnt; ++jj) {
            Frag f;
            const float2 co = s_co[jj];
            if (!eval_fragment(fx, fy, s_q0[jj], co.x, co.y, f)) continue;
            const float test = T * (1.0f - f.alpha);
            if (test < kTMin) {
                done = true;
                break;
            }
            const float w = f.alpha * T;
            const float4 c = s_rgb[jj];
            C0 += w * c.x;
            C1 += w * c.y;
            C2 += w * c.z;
            T = test;
            last = start + jj - range.x + 1;
        }
    }
    if (tp.inside) {
        const int64_t P = (int64_t)tp.W * tp.H;
        const int64_t pix = (int64_t)tp.py * tp.W + tp.px;
        float* img = images + 3 * vt.pix_off[tp.v];
        img[pix] = C0 + T * bg0;
        img[P + pix] = C1 + T * bg1;
        img[2 * P + pix] = C2 + T * bg2;
        T_final[vt.pix_off[tp.v] + pix] = T;
        n_contrib[vt.pix_off[tp.v] + pix] = last;
    }
}

__device__ __forceinline__ float warp_sum(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Sums eight per-lane values over the warp with 9 shuffles (reduce-scatter:
// each butterfly step sends half of the remaining values).  Afterwards lane
// l holds the total of value ((l >> 2) & 7) -- lanes 0, 4, ..., 28 hold
// values 0..7.
__device__ __forceinline__ float warp_sum8_scatter(const float v[8], int lane)
{
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
    float a[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float send = h16 ? v[j] : v[j + 4];
        const float keep = h16 ? v[j + 4] : v[j];
        a[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float b[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float send = h8 ? a[j] : a[j + 2];
        const float keep = h8 ? a[j + 2] : a[j];
        b[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float c = (h4 ? b[1] : b[0]) + __shfl_xor_sync(0xffffffffu, h4 ? b[0] : b[1], 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

__global__ void __launch_bounds__(kBlendThreads)
blend_bwd_kernel(ViewTable vt, int64_t n, const uint2* __restrict__ ranges,
                 const uint32_t* __restrict__ gids, const Screen* __restrict__ screen, float bg0,
                 float bg1, float bg2, const float* __restrict__ dL_dimg,
                 const float* __restrict__ T_final, const uint32_t* __restrict__ n_contrib,
                 ScreenGrad* __restrict__ sgrad)
{
    __shared__ float4 s_q0[kBlendThreads];
    __shared__ float2 s_co[kBlendThreads];
    __shared__ float4 s_rgb[kBlendThreads];
    __shared__ uint32_t s_gid[kBlendThreads];
    __shared__ float s_acc[9][kBlendThreads];
    __shared__ uint32_t s_max;
    const int tile = blockIdx.x;
    const TilePix tp = tile_pixel(vt, tile);
    const uint2 range = ranges[tile];
    const float fx = (float)tp.px + 0.5f, fy = (float)tp.py + 0.5f;
    const Screen* scr = screen + (int64_t)tp.v * n;
    ScreenGrad* sg = sgrad + (int64_t)tp.v * n;
    const int lane = threadIdx.x & 31;

    float T = 1.0f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    uint32_t last = 0;
    if (tp.inside) {
        const int64_t P = (int64_t)tp.W * tp.H;
        const int64_t pix = (int64_t)tp.py * tp.W + tp.px;
        const float* dl = dL_dimg + 3 * vt.pix_off[tp.v];
        g0 = dl[pix];
        g1 = dl[P + pix];
        g2 = dl[2 * P + pix];
        T = T_final[vt.pix_off[tp.v] + pix];
        last = n_contrib[vt.pix_off[tp.v] + pix];
    }
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    if (last) atomicMax(&s_max, last);
    __syncthreads();
    const uint32_t end = range.x + s_max;
    float A0 = bg0, A1 = bg1, A2 = bg2;  // colour behind, normalised by T after the entry

    for (uint32_t bend = end; bend > range.x;) {
        const uint32_t bstart = bend > range.x + kBlendThreads ? bend - kBlendThreads : range.x;
        const int cnt = (int)(bend - bstart);
        __syncthreads();
        if (threadIdx.x < cnt) {
            const uint32_t j = bend - 1 - threadIdx.x;  // slot 0 is the back-most entry
            const uint32_t g = gids[j];
            const Screen rec = scr[g];
            s_gid[threadIdx.x] = g;
            s_q0[threadIdx.x] = rec.q0;
            s_co[threadIdx.x] = make_float2(rec.q1.x, rec.q1.y);
            s_rgb[threadIdx.x] = rec.q2;
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) s_acc[k][threadIdx.x] = 0.f;
        __syncthreads();
        for (int jj = 0; jj < cnt; ++jj) {
            const uint32_t pos = bend - jj - range.x;  // 1-based list position
            Frag f;
            const float4 q0 = s_q0[jj];
            const float2 co = s_co[jj];
            bool contrib = pos <= last && eval_fragment(fx, fy, q0, co.x, co.y, f);
            float d[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) d[k] = 0.f;
            if (contrib) {
                const float4 c = s_rgb[jj];
                const float Ti = T / (1.0f - f.alpha);
                const float dalpha = Ti * (g0 * (c.x - A0) + g1 * (c.y - A1) + g2 * (c.z - A2));
                const float wT = f.alpha * Ti;
                d[6] = wT * g0;
                d[7] = wT * g1;
                d[8] = wT * g2;
                A0 = f.alpha * c.x + (1.0f - f.alpha) * A0;
                A1 = f.alpha * c.y + (1.0f - f.alpha) * A1;
                A2 = f.alpha * c.z + (1.0f - f.alpha) * A2;
                T = Ti;
                if (!f.clamped) {
                    const float dpow = dalpha * f.alpha;  // alpha = o G here
                    d[5] = dalpha * f.G;
                    d[2] = -0.5f * f.dx * f.dx * dpow;
                    d[3] = -f.dx * f.dy * dpow;
                    d[4] = -0.5f * f.dy * f.dy * dpow;
                    d[0] = dpow * (q0.z * f.dx + q0.w * f.dy);
                    d[1] = dpow * (q0.w * f.dx + co.x * f.dy);
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
                // value index of lane l after the scatter: (l >> 2) & 7
                const float part = warp_sum8_scatter(d, lane);
                const float last_v = warp_sum(d[8]);
                if ((lane & 3) == 0) atomicAdd(&s_acc[(lane >> 2) & 7][jj], part);
                if (lane == 1) atomicAdd(&s_acc[8][jj], last_v);
            }
        }
        __syncthreads();
        if (threadIdx.x < cnt) {
            const int s = threadIdx.x;
            const float4 a = make_float4(s_acc[0][s], s_acc[1][s], s_acc[2][s], s_acc[3][s]);
            const float4 b = make_float4(s_acc[4][s], s_acc[5][s], s_acc[6][s], s_acc[7][s]);
            const float e = s_acc[8][s];
            if (a.x != 0.f || a.y != 0.f || a.z != 0.f || a.w != 0.f || b.x != 0.f || b.y != 0.f ||
                b.z != 0.f || b.w != 0.f || e != 0.f) {
                ScreenGrad* dst = sg + s_gid[s];
                atomicAdd(&dst->g0, a);
                atomicAdd(&dst->g1, b);
                atomicAdd(&dst->g2.x, e);
            }
        }
        bend = bstart;
    }
}

cudaError_t launch_blend_fwd(const ViewTable& vt, int64_t n, const uint2* ranges, const uint32_t* gids,
                             const Screen* screen, const float bg[3], float* images, float* T_final,
                             uint32_t* n_contrib, cudaStream_t st)
{
    if (vt.total_tiles <= 0) return cudaSuccess;
    blend_fwd_kernel<<<vt.total_tiles, kBlendThreads, 0, st>>>(vt, n, ranges, gids, screen, bg[0], bg[1],
                                                               bg[2], images, T_final, n_contrib);
    profile_mark(st, "blend_fwd");
    return cudaGetLastError();
}

cudaError_t launch_blend_bwd(const ViewTable& vt, int64_t n, const uint2* ranges, const uint32_t* gids,
                             const Screen* screen, const float bg[3], const float* dL_dimg,
                             const float* T_final, const uint32_t* n_contrib, ScreenGrad* sgrad,
                             cudaStream_t st)
{
    if (vt.total_tiles <= 0) return cudaSuccess;
    blend_bwd_kernel<<<vt.total_tiles, kBlendThreads, 0, st>>>(vt, n, ranges, gids, screen, bg[0], bg[1],
                                                               bg[2], dL_dimg, T_final, n_contrib, sgrad);
    profile_mark(st, "blend_bwd");
    return cudaGetLastError();
}

}  // namespace fgs
