// preprocess.cu -- per-Gaussian kernels of the training step (sm_103a).
//
//  preprocess_fwd : Eq. 1-2 projection, Sec. 2.1 activations (fused, Sec. 3.2
//                   "Rasterization Kernel Fusion"), Suppl. B.1 degeneracy
//                   tests, Suppl. C dilation, Sec. 3.2 opacity-aware
//                   rectangle and per-tile culling, SH colour.  One thread
//                   per Gaussian loops over all views, so the parameters
//                   are read once per batch.  A CTA-wide exclusive scan of
//                   the per-view tile counts is fused in.
//  scan_block_sums: prefix over the CTA totals (one CTA), total instances.
//  duplicate      : writes (global tile << 32 | depth bits, Gaussian id) for
//                   every kept tile (Sec. 3.2 "Sorting").
//  preprocess_bwd : chain rule from dL/d(mu2D, conic, o, rgb) to the raw
//                   parameters, summed over the views; writes every
//                   Gaussian's gradient (zero where invisible).
#include <algorithm>

#include "adam_math.cuh"

namespace fgs {

// Asks L2 for the 128-byte line holding p (no register is written).
__device__ __forceinline__ void prefetch_l2(const void* p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Exclusive scan of one value per thread over a kPreBlock-thread CTA.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot,
                                                         uint32_t& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kPreBlock / 32 ? warp_tot[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kPreBlock / 32) warp_tot[lane] = w;  // inclusive
    }
    __syncthreads();
    const uint32_t base = warp > 0 ? warp_tot[warp - 1] : 0u;
    total = warp_tot[kPreBlock / 32 - 1];
    __syncthreads();
    return base + x - v;
}

constexpr int kBigRect = 32;  // rectangles with more tiles are culled by the whole warp

// Per-view screen geometry of one Gaussian (Eq. 1-2, Suppl. B.1 tests,
// Suppl. C dilation, Sec. 3.2 opacity-aware rectangle).
struct Geo {
    float mx, my, k, depth;
    EigenConic e;
    int tx0, ty0, tw, ntiles;  // tile rectangle (ntiles = 0: not rendered)
};

// Every rounding is explicit (see quat_to_rot_rn).
__device__ __forceinline__ void project(const Cam& cam, const float mu[3], const float M[9], float o,
                                        Geo& g)
{
    g.ntiles = 0;
    float t[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
        t[r] = __fadd_rn(__fmaf_rn(cam.R[3 * r + 2], mu[2],
                                   __fmaf_rn(cam.R[3 * r + 1], mu[1], __fmul_rn(cam.R[3 * r], mu[0]))),
                         cam.t[r]);
    if (!(t[2] > cam.near_plane)) return;
    const float iz = __fdiv_rn(1.0f, t[2]);
    // Eq. 2: J (2x3) and T2 = J Rcam; M2 = T2 M, Sigma2D = M2 M2^T
    const float j00 = __fmul_rn(cam.fx, iz), j02 = -__fmul_rn(__fmul_rn(__fmul_rn(cam.fx, t[0]), iz), iz);
    const float j11 = __fmul_rn(cam.fy, iz), j12 = -__fmul_rn(__fmul_rn(__fmul_rn(cam.fy, t[1]), iz), iz);
    float T2[6];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T2[c] = __fmaf_rn(j02, cam.R[6 + c], __fmul_rn(j00, cam.R[c]));
        T2[3 + c] = __fmaf_rn(j12, cam.R[6 + c], __fmul_rn(j11, cam.R[3 + c]));
    }
    float M2[6];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            M2[3 * r + c] = __fmaf_rn(T2[3 * r + 2], M[6 + c],
                                      __fmaf_rn(T2[3 * r + 1], M[3 + c], __fmul_rn(T2[3 * r], M[c])));
    const float ca = __fmaf_rn(M2[2], M2[2], __fmaf_rn(M2[1], M2[1], __fmul_rn(M2[0], M2[0])));
    const float cb = __fmaf_rn(M2[2], M2[5], __fmaf_rn(M2[1], M2[4], __fmul_rn(M2[0], M2[3])));
    const float cc = __fmaf_rn(M2[5], M2[5], __fmaf_rn(M2[4], M2[4], __fmul_rn(M2[3], M2[3])));
    // Cauchy-Binet: det(M2 M2^T) = sum of squared 2x2 minors (no cancellation)
    const float m01 = __fmaf_rn(M2[0], M2[4], -__fmul_rn(M2[1], M2[3]));
    const float m02 = __fmaf_rn(M2[0], M2[5], -__fmul_rn(M2[2], M2[3]));
    const float m12 = __fmaf_rn(M2[1], M2[5], -__fmul_rn(M2[2], M2[4]));
    const float det2 = __fmaf_rn(m12, m12, __fmaf_rn(m02, m02, __fmul_rn(m01, m01)));
    if (!(det2 >= kDetMin)) return;
    const float da = __fadd_rn(ca, kDilation), dc = __fadd_rn(cc, kDilation);
    const float detd = __fadd_rn(__fmaf_rn(kDilation, __fadd_rn(ca, cc), det2), kDilation * kDilation);
    // conic = (Sigma2D + 0.3 I)^-1 in eigen form: the dilated covariance has
    // eigenvalues lmax = (da + dc)/2 + r, r = sqrt(((ca - cc)/2)^2 + cb^2) (no
    // cancellation) and lmin = detd / lmax.  Its major axis makes the angle th
    // with cos 2th = h / r, sin 2th = cb / r (h = (ca - cc)/2); the half-angle
    // identities give (cos th, sin th) with the larger one from a sum of
    // non-negative terms and the other from sin 2th = 2 sin th cos th.
    const float h = __fmul_rn(0.5f, __fsub_rn(ca, cc));
    const float r = __fsqrt_rn(__fmaf_rn(h, h, __fmul_rn(cb, cb)));
    const float lmax = __fadd_rn(__fmul_rn(0.5f, __fadd_rn(da, dc)), r);
    g.e.ls = __fdiv_rn(1.0f, lmax);
    g.e.lb = __fdiv_rn(lmax, detd);
    if (!(r > 0.0f)) {
        g.e.c = 1.0f;
        g.e.s = 0.0f;
    } else if (h >= 0.0f) {
        g.e.c = __fsqrt_rn(__fdiv_rn(__fadd_rn(r, h), __fmul_rn(2.0f, r)));
        g.e.s = __fdiv_rn(cb, __fmul_rn(__fmul_rn(2.0f, r), g.e.c));
    } else {
        g.e.s = copysignf(__fsqrt_rn(__fdiv_rn(__fsub_rn(r, h), __fmul_rn(2.0f, r))), cb);
        g.e.c = __fdiv_rn(cb, __fmul_rn(__fmul_rn(2.0f, r), g.e.s));
    }
    g.mx = __fmaf_rn(__fmul_rn(cam.fx, t[0]), iz, cam.cx);
    g.my = __fmaf_rn(__fmul_rn(cam.fy, t[1]), iz, cam.cy);
    g.depth = t[2];
    g.k = opacity_k(o);
    const float ex = __fsqrt_rn(__fmul_rn(g.k, da)), ey = __fsqrt_rn(__fmul_rn(g.k, dc));
    const float u0 = fmaxf(ceilf(__fsub_rn(__fsub_rn(g.mx, ex), 0.5f)), 0.0f);
    const float u1 = fminf(floorf(__fsub_rn(__fadd_rn(g.mx, ex), 0.5f)), (float)(cam.width - 1));
    const float v0 = fmaxf(ceilf(__fsub_rn(__fsub_rn(g.my, ey), 0.5f)), 0.0f);
    const float v1 = fminf(floorf(__fsub_rn(__fadd_rn(g.my, ey), 0.5f)), (float)(cam.height - 1));
    if (!(u0 <= u1 && v0 <= v1)) return;
    g.tx0 = (int)u0 / kTile;
    g.ty0 = (int)v0 / kTile;
    g.tw = (int)u1 / kTile - g.tx0 + 1;
    g.ntiles = g.tw * ((int)v1 / kTile - g.ty0 + 1);
}

// Kept tiles of one Gaussian: the thread alone for small rectangles; for
// large ones every lane of the warp takes a stride of the rectangle and the
// counts are reduced (the warp must be converged; `g` is per lane).
// For small rectangles `keep` receives the kept tiles (bit t = tile t).
__device__ __forceinline__ uint32_t count_tiles(const Geo& g, bool has, int width, int height,
                                                uint32_t& keep)
{
    const int lane = threadIdx.x & 31;
    uint32_t count = 0;
    keep = 0;
    const bool big = has && g.ntiles > kBigRect;
    TileCull cull;
    if (has) cull = make_cull(g.mx, g.my, g.e, g.k);
    if (has && !big) {
        int t = 0;
        for (int ty = g.ty0; t < g.ntiles; ++ty)
            for (int tx = g.tx0; tx < g.tx0 + g.tw; ++tx, ++t)
                if (tile_keep(cull, tx, ty, width, height)) keep |= 1u << t;
        count = __popc(keep);
    }
    unsigned bigmask = __ballot_sync(0xffffffffu, big);
    while (bigmask) {
        const int src = __ffs(bigmask) - 1;
        bigmask &= bigmask - 1;
        TileCull c;
        c.mx = __shfl_sync(0xffffffffu, cull.mx, src);
        c.my = __shfl_sync(0xffffffffu, cull.my, src);
        c.k = __shfl_sync(0xffffffffu, cull.k, src);
        c.rx = __shfl_sync(0xffffffffu, cull.rx, src);
        c.ry = __shfl_sync(0xffffffffu, cull.ry, src);
        c.e.lb = __shfl_sync(0xffffffffu, cull.e.lb, src);
        c.e.ls = __shfl_sync(0xffffffffu, cull.e.ls, src);
        c.e.c = __shfl_sync(0xffffffffu, cull.e.c, src);
        c.e.s = __shfl_sync(0xffffffffu, cull.e.s, src);
        const int tx0 = __shfl_sync(0xffffffffu, g.tx0, src), ty0 = __shfl_sync(0xffffffffu, g.ty0, src);
        const int tw = __shfl_sync(0xffffffffu, g.tw, src), nt = __shfl_sync(0xffffffffu, g.ntiles, src);
        // lane's tile t = lane + 32 j at (col, row) of the rectangle, stepped without divisions
        const int step_r = 32 / tw, step_c = 32 - step_r * tw;
        int row = lane / tw, col = lane - row * tw;
        uint32_t part = 0;
        for (int t = lane; t < nt; t += 32) {
            part += tile_keep(c, tx0 + col, ty0 + row, width, height);
            col += step_c;
            row += step_r;
            if (col >= tw) {
                col -= tw;
                ++row;
            }
        }
        part = __reduce_add_sync(0xffffffffu, part);
        if (lane == src) count = part;
    }
    return count;
}

// Compiled for 8 CTAs of 128 threads per SM (64 registers, a few spilled):
// warps of a CTA finish at different times (culling and colour run for a
// third of the Gaussians) and wait at the per-view scan, so more, smaller CTAs
// keep the SM busier -- 0.32 ms per 3M-Gaussian view against 0.39 ms with 3
// CTAs of 256 threads.
template <typename SHT, bool MOTION>
__global__ void __launch_bounds__(kPreBlock, 8)
preprocess_fwd_kernel(int64_t n, int sh_degree, const float* __restrict__ means,
                      const float* __restrict__ log_scales, const float* __restrict__ quats,
                      const float* __restrict__ opac, const SHT* __restrict__ sh_dc,
                      const SHT* __restrict__ sh_rest, const fgs_camera* __restrict__ cams,
                      ViewTable vt, Screen* __restrict__ screen, TileRect* __restrict__ rects,
                      uint32_t* __restrict__ local_off, uint32_t* __restrict__ block_sum,
                      int nblk, Motion mo, int ahead)
{
    // two buffers, alternating by view: a warp still reading view v's totals
    // cannot be overtaken by a write of view v + 2 (view v + 1's barriers lie
    // between them)
    __shared__ uint32_t warp_tot[2][kPreBlock / 32];
    const int64_t i = (int64_t)blockIdx.x * kPreBlock + threadIdx.x;
    const bool valid = i < n;
    {
        // the parameter lines of the block `ahead` blocks on (half a wave of
        // resident CTAs), asked of L2 so that its loads find them there
        // (0.171 -> 0.167 ms at 3M Gaussians); 44 lines of 128 bytes
        const int64_t j0 = ((int64_t)blockIdx.x + ahead) * kPreBlock;
        const int t = threadIdx.x;
        if (j0 + kPreBlock <= n) {
            if (t < 12) prefetch_l2(means + 3 * j0 + 32 * t);
            else if (t < 28) prefetch_l2(quats + 4 * j0 + 32 * (t - 12));
            else if (t < 40) prefetch_l2(log_scales + 3 * j0 + 32 * (t - 28));
            else if (t < 44) prefetch_l2(opac + j0 + 32 * (t - 40));
        }
    }
    float mu[3] = {0.f, 0.f, 0.f}, M[9], o = 0.f, vel[3] = {0.f, 0.f, 0.f}, t0 = 0.f;
    bool ok = false;
    if (valid) {
        mu[0] = means[3 * i];
        mu[1] = means[3 * i + 1];
        mu[2] = means[3 * i + 2];
        const float4 q4 = *reinterpret_cast<const float4*>(quats + 4 * i);  // rows are 16-byte aligned
        const float qw = q4.x, qx = q4.y, qy = q4.z, qz = q4.w;
        const float qn = __fsqrt_rn(__fmaf_rn(qz, qz, __fmaf_rn(qy, qy, __fmaf_rn(qx, qx, __fmul_rn(qw, qw)))));
        const float inv = qn > 0.f ? __fdiv_rn(1.0f, qn) : 0.f;
        float Rq[9];
        quat_to_rot_rn(__fmul_rn(qw, inv), __fmul_rn(qx, inv), __fmul_rn(qy, inv), __fmul_rn(qz, inv), Rq);
        const float s0 = __expf(log_scales[3 * i]), s1 = __expf(log_scales[3 * i + 1]),
                    s2 = __expf(log_scales[3 * i + 2]);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            M[3 * r] = Rq[3 * r] * s0;
            M[3 * r + 1] = Rq[3 * r + 1] * s1;
            M[3 * r + 2] = Rq[3 * r + 2] * s2;
        }
        o = __fdiv_rn(1.0f, __fadd_rn(1.0f, __expf(-opac[i])));
        ok = qn >= kQNormMin;
        if (MOTION) {
            vel[0] = mo.vel[3 * i]; vel[1] = mo.vel[3 * i + 1]; vel[2] = mo.vel[3 * i + 2];
            t0 = mo.t0[i];
        }
    }
    const int ncoef = (sh_degree + 1) * (sh_degree + 1);
    for (int v = 0; v < vt.n_views; ++v) {
        const Cam cam = load_cam(cams, v);
        // the Gaussian at this view's time (static ones: as stored)
        float mv[3] = {mu[0], mu[1], mu[2]}, ov = o;
        if (MOTION) {
            const float dt = cam.time - t0;
#pragma unroll
            for (int a = 0; a < 3; ++a) mv[a] = __fmaf_rn(vel[a], dt, mu[a]);
            ov = __fmul_rn(o, temporal_weight(dt, mo.inv_var));
        }
        Geo g;
        g.ntiles = 0;
        if (ok && ov >= kAlphaMin) project(cam, mv, M, ov, g);
        const bool has = g.ntiles > 0;
        if (has) {
            // the colour's SH lines, asked of L2 while the tiles are culled
            // (0.1745 -> 0.1714 ms at 3M Gaussians)
            const char* row = reinterpret_cast<const char*>(sh_rest + 45 * i);
            prefetch_l2(row);
            prefetch_l2(row + 64 * sizeof(SHT) / 2);
            prefetch_l2(row + 45 * sizeof(SHT) - 1);
            prefetch_l2(sh_dc + 3 * i);
        }
        uint32_t keep;
        const uint32_t count = count_tiles(g, has, cam.width, cam.height, keep);
        Screen rec;
        rec.q0 = make_float4(0.f, 0.f, 0.f, 0.f);
        rec.q1 = make_float4(0.f, 0.f, 0.f, 0.f);
        rec.q2 = make_float4(0.f, 0.f, 0.f, 0.f);
        TileRect rect;
        rect.r = make_ushort4(1, 1, 0, 0);
        rect.keep = keep;
        rect.count = count;
        if (count > 0) {
            rect.r = make_ushort4((unsigned short)g.tx0, (unsigned short)g.ty0,
                                  (unsigned short)(g.tx0 + g.tw - 1),
                                  (unsigned short)(g.ty0 + g.ntiles / g.tw - 1));
            // SH colour from the view direction, streamed from memory
            float d0 = __fsub_rn(mv[0], cam.pos[0]), d1 = __fsub_rn(mv[1], cam.pos[1]),
                  d2 = __fsub_rn(mv[2], cam.pos[2]);
            const float il = rsqrtf(__fmaf_rn(d2, d2, __fmaf_rn(d1, d1, __fmul_rn(d0, d0))));
            d0 = __fmul_rn(d0, il);
            d1 = __fmul_rn(d1, il);
            d2 = __fmul_rn(d2, il);
            float Y[16];
            sh_basis_rn(d0, d1, d2, sh_degree, Y);
            float r0 = __fmaf_rn(Y[0], to_f32(sh_dc[3 * i]), 0.5f);
            float r1 = __fmaf_rn(Y[0], to_f32(sh_dc[3 * i + 1]), 0.5f);
            float r2 = __fmaf_rn(Y[0], to_f32(sh_dc[3 * i + 2]), 0.5f);
            const SHT* rest = sh_rest + 45 * i;
#pragma unroll
            for (int kk = 1; kk < 16; ++kk) {
                if (kk < ncoef) {
                    r0 = __fmaf_rn(Y[kk], to_f32(rest[3 * (kk - 1)]), r0);
                    r1 = __fmaf_rn(Y[kk], to_f32(rest[3 * (kk - 1) + 1]), r1);
                    r2 = __fmaf_rn(Y[kk], to_f32(rest[3 * (kk - 1) + 2]), r2);
                }
            }
            uint32_t bits = 8u;  // visible
            if (r0 < 0.f) { bits |= 1u; r0 = 0.f; }
            if (r1 < 0.f) { bits |= 2u; r1 = 0.f; }
            if (r2 < 0.f) { bits |= 4u; r2 = 0.f; }
            rec.q0 = make_float4(g.mx, g.my, g.e.lb, g.e.ls);
            rec.q1 = make_float4(g.e.c, g.e.s, ov, g.depth);
            rec.q2 = make_float4(r0, r1, r2, __uint_as_float(bits));
        }
        const int64_t vi = (int64_t)v * n + i;
        if (valid) {
            // the screen record only where the pair is rendered: every reader
            // takes the rendered flag from the tile record's count
            if (count > 0) screen[vi] = rec;
            rects[vi] = rect;
        }
        // compaction offsets of the rendered (view, Gaussian) pairs
        uint32_t total;
        const uint32_t excl = block_exclusive_scan(count > 0 ? 1u : 0u, warp_tot[v & 1], total);
        if (valid) local_off[vi] = excl;
        if (threadIdx.x == 0) block_sum[(int64_t)v * nblk + blockIdx.x] = total;
    }
}

// Exclusive prefix of the CTA totals (one CTA).  instances: the totals are
// instance counts -- writes the total (may exceed k_max), the clamped count
// the tile sort uses (counters[0]) and the capacity flag; otherwise they
// count rendered (view, Gaussian) pairs -- writes that count (counters[1]).
__global__ void __launch_bounds__(1024)
scan_block_sums_kernel(uint32_t* __restrict__ block_sum, int64_t count, WsHeader* __restrict__ hdr,
                       int64_t k_max, bool instances)
{
    __shared__ unsigned long long wsum[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // each thread a run of a multiple of 4 values (16-byte vectors; the
    // array starts 256-byte aligned)
    const int64_t chunk = (((count + 1023) / 1024) + 3) & ~(int64_t)3;
    const int64_t b = t * chunk, e = min(count, b + chunk);
    unsigned long long s = 0;
#pragma unroll 4
    for (int64_t j = b; j < e; j += 4) {
        if (j + 4 <= e) {
            const uint4 q = *reinterpret_cast<const uint4*>(block_sum + j);
            s += (unsigned long long)q.x + q.y + q.z + q.w;
        } else {
            for (int64_t jj = j; jj < e; ++jj) s += block_sum[jj];
        }
    }
    // exclusive scan of the run totals: shuffles within warps, then the warp totals
    unsigned long long x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    unsigned long long run = x - s + (warp > 0 ? wsum[warp - 1] : 0ull);
    for (int64_t j = b; j < e; j += 4) {
        if (j + 4 <= e) {
            const uint4 q = *reinterpret_cast<const uint4*>(block_sum + j);
            uint4 o;
            o.x = (uint32_t)min(run, 0xffffffffull); run += q.x;
            o.y = (uint32_t)min(run, 0xffffffffull); run += q.y;
            o.z = (uint32_t)min(run, 0xffffffffull); run += q.z;
            o.w = (uint32_t)min(run, 0xffffffffull); run += q.w;
            *reinterpret_cast<uint4*>(block_sum + j) = o;
        } else {
            for (int64_t jj = j; jj < e; ++jj) {
                const uint32_t q = block_sum[jj];
                block_sum[jj] = (uint32_t)min(run, 0xffffffffull);
                run += q;
            }
        }
    }
    if (t == 1023) {
        const unsigned long long tot = wsum[31];
        if (instances) {
            hdr->counters[2] = 0;  // the split duplication's large-rectangle list
            hdr->instances = tot;
            hdr->counters[0] = (uint32_t)min(tot, (unsigned long long)k_max);
            if (tot > (unsigned long long)k_max) set_flag(hdr, FGS_FLAG_CAPACITY);
        } else {
            hdr->counters[1] = (uint32_t)tot;
        }
    }
}

// Rendered (view, Gaussian) pairs in (view, id) order, as (depth bits,
// view * n + id) for the depth sort (depths are > 0, so their float bits
// order like the values).
__global__ void __launch_bounds__(256)
compact_visible_kernel(int64_t n, ViewTable vt, const Screen* __restrict__ screen,
                       const TileRect* __restrict__ rects, const uint32_t* __restrict__ local_off,
                       const uint32_t* __restrict__ block_sum, int nblk, uint32_t* __restrict__ dkeys,
                       uint32_t* __restrict__ dvals)
{
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= (int64_t)vt.n_views * n) return;
    const ushort4 r = rects[gi].r;
    if (r.x > r.z) return;
    const int v = (int)(gi / n);
    const int64_t i = gi - (int64_t)v * n;
    const uint32_t pos = local_off[gi] + block_sum[(int64_t)v * nblk + i / kPreBlock];
    dkeys[pos] = __float_as_uint(screen[gi].q1.w);
    dvals[pos] = (uint32_t)gi;
}

// Instance offsets in depth order: exclusive prefix, within each CTA of
// kCountTile sorted entries, of their instance counts, and the CTA totals.
constexpr int kCountItems = 4;
constexpr int kCountTile = kPreBlock * kCountItems;

__global__ void __launch_bounds__(kPreBlock)
sorted_count_scan_kernel(const uint32_t* __restrict__ n_dev, const uint32_t* __restrict__ svals,
                         const TileRect* __restrict__ rects, uint32_t* __restrict__ sorted_off,
                         uint32_t* __restrict__ sorted_block)
{
    __shared__ uint32_t warp_tot[kPreBlock / 32];
    const uint32_t F = *n_dev;
    const int64_t base = (int64_t)blockIdx.x * kCountTile + (int64_t)threadIdx.x * kCountItems;
    uint32_t c[kCountItems], sum = 0;
#pragma unroll
    for (int q = 0; q < kCountItems; ++q) {
        const int64_t j = base + q;
        c[q] = j < (int64_t)F ? rects[svals[j]].count : 0u;
        sum += c[q];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(sum, warp_tot, total);
#pragma unroll
    for (int q = 0; q < kCountItems; ++q) {
        const int64_t j = base + q;
        if (j < (int64_t)F) sorted_off[j] = run;
        run += c[q];
    }
    if (threadIdx.x == 0) sorted_block[blockIdx.x] = total;
}

// Emits (global tile, Gaussian id) for every kept tile of every rendered
// (view, Gaussian) pair into the range its depth-order offset gives it, so
// that a stable sort by tile keeps depth order, ties by id, inside each
// tile.  Small rectangles walk the kept-tile mask the preprocess recorded;
// large ones are culled again by the whole warp, 32 tiles per step, with a
// ballot prefix.  Lane l of warp w takes entry l * W + w (W warps in use):
// near splats, which have the large rectangles, come first in depth order,
// and this spreads them over all warps instead of a few.
__global__ void __launch_bounds__(256)
duplicate_kernel(int64_t n, ViewTable vt, const Screen* __restrict__ screen,
                 const TileRect* __restrict__ rects, const uint32_t* __restrict__ n_vis,
                 const uint32_t* __restrict__ svals, const uint32_t* __restrict__ sorted_off,
                 const uint32_t* __restrict__ sorted_block, int64_t k_max, uint32_t* __restrict__ keys,
                 uint32_t* __restrict__ vals)
{
    const int lane = threadIdx.x & 31;
    const int64_t F = *n_vis;
    const int64_t W = (F + 31) / 32;
    const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t j = (int64_t)lane * W + wg;
    const bool has = wg < W && j < F;
    int v = 0;
    int64_t i = 0, gi = 0;
    TileRect tr;
    tr.r = make_ushort4(1, 1, 0, 0);
    tr.keep = 0;
    uint64_t off = 0;
    if (has) {
        gi = svals[j];
        v = (int)(gi / n);
        i = gi - (int64_t)v * n;
        tr = rects[gi];
        off = (uint64_t)sorted_off[j] + sorted_block[j / kCountTile];
    }
    const ushort4 r = tr.r;
    const int tw = (int)r.z - (int)r.x + 1;
    const int nt = has ? tw * ((int)r.w - (int)r.y + 1) : 0;
    const bool big = has && nt > kBigRect;
    float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0;
    if (big) {
        q0 = screen[gi].q0;
        q1 = screen[gi].q1;
    }
    if (has && !big) {
        const uint32_t toff = (uint32_t)vt.tile_off[v];
        const int tx_n = vt.tiles_x[v];
        for (uint32_t m = tr.keep; m; m &= m - 1) {
            const int t = __ffs(m) - 1;
            const int tx = r.x + t % tw, ty = r.y + t / tw;
            if (off < (uint64_t)k_max) {
                keys[off] = toff + (uint32_t)(ty * tx_n + tx);
                vals[off] = (uint32_t)i;
            }
            ++off;
        }
    }
    unsigned bigmask = __ballot_sync(0xffffffffu, big);
    while (bigmask) {
        const int src = __ffs(bigmask) - 1;
        bigmask &= bigmask - 1;
        const TileCull c = make_cull(__shfl_sync(0xffffffffu, q0.x, src), __shfl_sync(0xffffffffu, q0.y, src),
                                     eigen_from_stored(__shfl_sync(0xffffffffu, q0.z, src),
                                                       __shfl_sync(0xffffffffu, q0.w, src),
                                                       __shfl_sync(0xffffffffu, q1.x, src),
                                                       __shfl_sync(0xffffffffu, q1.y, src)),
                                     opacity_k(__shfl_sync(0xffffffffu, q1.z, src)));
        const int sv = __shfl_sync(0xffffffffu, v, src);
        const uint32_t sid = (uint32_t)__shfl_sync(0xffffffffu, (unsigned long long)i, src);
        const int tx0 = __shfl_sync(0xffffffffu, (int)r.x, src), ty0 = __shfl_sync(0xffffffffu, (int)r.y, src);
        const int stw = __shfl_sync(0xffffffffu, tw, src), snt = __shfl_sync(0xffffffffu, nt, src);
        uint64_t soff = __shfl_sync(0xffffffffu, (unsigned long long)off, src);
        const int width = vt.width[sv], height = vt.height[sv], tx_n = vt.tiles_x[sv];
        const uint32_t toff = (uint32_t)vt.tile_off[sv];
        // lane's tile base + lane at (col, row) of the rectangle, stepped without divisions
        const int step_r = 32 / stw, step_c = 32 - step_r * stw;
        int row = lane / stw, col = lane - row * stw;
        for (int base = 0; base < snt; base += 32) {
            const int t = base + lane;
            const int tx = tx0 + col, ty = ty0 + row;
            const bool keep = t < snt && tile_keep(c, tx, ty, width, height);
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            const uint64_t pos = soff + __popc(m & ((1u << lane) - 1u));
            if (keep && pos < (uint64_t)k_max) {
                keys[pos] = toff + (uint32_t)(ty * tx_n + tx);
                vals[pos] = sid;
            }
            soff += __popc(m);
            col += step_c;
            row += step_r;
            if (col >= stw) {
                col -= stw;
                ++row;
            }
        }
    }
}

// The same emission in the split order (FGS_DUPLICATE_SPLIT): consecutive
// threads take consecutive entries, so a warp's stores fill one contiguous
// run of the instance arrays (the strided order scatters them over 32 runs;
// with the instance arrays of a batch of eight views, 184 MB, well beyond
// L2, this order measured 0.34 against 0.61 ms).  Small rectangles walk the
// kept-tile mask the preprocess recorded; large ones are appended to `big`
// (count in *n_big, zeroed by the instance scan) for duplicate_big_kernel:
// the near splats, which have them, come first in depth order, and culling
// them here would load a few warps with most of the work.
__global__ void __launch_bounds__(256)
duplicate_split_kernel(int64_t n, ViewTable vt, const TileRect* __restrict__ rects,
                       const uint32_t* __restrict__ n_vis, const uint32_t* __restrict__ svals,
                       const uint32_t* __restrict__ sorted_off, const uint32_t* __restrict__ sorted_block,
                       int64_t k_max, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                       uint32_t* __restrict__ big, uint32_t* __restrict__ n_big)
{
    const int lane = threadIdx.x & 31;
    const int64_t F = *n_vis;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool has = j < F;
    bool is_big = false;
    if (has) {
        const int64_t gi = svals[j];
        const int v = (int)(gi / n);
        const int64_t i = gi - (int64_t)v * n;
        const TileRect tr = rects[gi];
        const ushort4 r = tr.r;
        const int tw = (int)r.z - (int)r.x + 1;
        const int nt = tw * ((int)r.w - (int)r.y + 1);
        is_big = nt > kBigRect;
        if (!is_big) {
            uint64_t off = (uint64_t)sorted_off[j] + sorted_block[j / kCountTile];
            const uint32_t toff = (uint32_t)vt.tile_off[v];
            const int tx_n = vt.tiles_x[v];
            for (uint32_t m = tr.keep; m; m &= m - 1) {
                const int t = __ffs(m) - 1;
                const int tx = r.x + t % tw, ty = r.y + t / tw;
                if (off < (uint64_t)k_max) {
                    keys[off] = toff + (uint32_t)(ty * tx_n + tx);
                    vals[off] = (uint32_t)i;
                }
                ++off;
            }
        }
    }
    // one list append per warp (entries fit 32 bits: n_views * n < 2^32)
    const unsigned bm = __ballot_sync(0xffffffffu, is_big);
    if (bm) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(n_big, (uint32_t)__popc(bm));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (is_big) big[base + __popc(bm & ((1u << lane) - 1u))] = (uint32_t)j;
    }
}

// The large rectangles listed by duplicate_kernel, one warp per entry (a
// grid-stride loop over the list): the warp culls 32 tiles per step and
// writes the kept ones with a ballot prefix, in row-major order.
__global__ void __launch_bounds__(256)
duplicate_big_kernel(int64_t n, ViewTable vt, const Screen* __restrict__ screen,
                     const TileRect* __restrict__ rects, const uint32_t* __restrict__ svals,
                     const uint32_t* __restrict__ sorted_off, const uint32_t* __restrict__ sorted_block,
                     const uint32_t* __restrict__ big, const uint32_t* __restrict__ n_big, int64_t k_max,
                     uint32_t* __restrict__ keys, uint32_t* __restrict__ vals)
{
    const int lane = threadIdx.x & 31;
    const int64_t nb = *n_big;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nb; b += warps) {
        // warp-uniform: every lane loads the same entry
        const int64_t j = big[b];
        const int64_t gi = svals[j];
        const int v = (int)(gi / n);
        const uint32_t id = (uint32_t)(gi - (int64_t)v * n);
        const ushort4 r = rects[gi].r;
        const int tx0 = r.x, ty0 = r.y;
        const int stw = (int)r.z - (int)r.x + 1;
        const int snt = stw * ((int)r.w - (int)r.y + 1);
        uint64_t soff = (uint64_t)sorted_off[j] + sorted_block[j / kCountTile];
        const float4 q0 = screen[gi].q0, q1 = screen[gi].q1;
        const TileCull c = make_cull(q0.x, q0.y, eigen_from_stored(q0.z, q0.w, q1.x, q1.y), opacity_k(q1.z));
        const int width = vt.width[v], height = vt.height[v], tx_n = vt.tiles_x[v];
        const uint32_t toff = (uint32_t)vt.tile_off[v];
        // lane's tile base + lane at (col, row) of the rectangle, stepped without divisions
        const int step_r = 32 / stw, step_c = 32 - step_r * stw;
        int row = lane / stw, col = lane - row * stw;
        for (int base = 0; base < snt; base += 32) {
            const int t = base + lane;
            const int tx = tx0 + col, ty = ty0 + row;
            const bool keep = t < snt && tile_keep(c, tx, ty, width, height);
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            const uint64_t pos = soff + __popc(m & ((1u << lane) - 1u));
            if (keep && pos < (uint64_t)k_max) {
                keys[pos] = toff + (uint32_t)(ty * tx_n + tx);
                vals[pos] = id;
            }
            soff += __popc(m);
            col += step_c;
            row += step_r;
            if (col >= stw) {
                col -= stw;
                ++row;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Backward of the preprocessing (chain rule, summed over views)
// ---------------------------------------------------------------------------
constexpr int kBwdBlock = 128;

// dir, colour gradient (clamped channels masked) of one visible view.
__device__ __forceinline__ void view_colour_grad(const Cam& cam, const float mu[3], uint32_t bits,
                                                 const ScreenGrad& g, float d[3], float& il,
                                                 float grgb[3])
{
    d[0] = mu[0] - cam.pos[0];
    d[1] = mu[1] - cam.pos[1];
    d[2] = mu[2] - cam.pos[2];
    il = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    d[0] *= il; d[1] *= il; d[2] *= il;
    grgb[0] = (bits & 1u) ? 0.f : g.g1.z;
    grgb[1] = (bits & 2u) ? 0.f : g.g1.w;
    grgb[2] = (bits & 4u) ? 0.f : g.g2.x;
}

// Parameters, moments and device state of the fused Adam step (Sec. 3.3
// "Fusing Backward and Optimizer"); the parameters alias the ones the
// gradient pass reads, so neither is declared __restrict__.
struct AdamArgs {
    void* p[8];
    void* m[8];
    void* v[8];
    const fgs_adam_state* st;
    WsHeader* hdr;  // receives FGS_FLAG_NONFINITE
};

// True unless all three are finite (v >= 0; a NaN fails the comparison, and
// a sum beyond the float range counts as non-finite too).
__device__ __forceinline__ bool adam_nonfinite(float p, float m, float v)
{
    return !(fabsf(p) + fabsf(m) + v <= 3.402823466e38f);
}

// Four consecutive elements of a storage type as one 16-byte (float32) or
// 8-byte (bf16, fp16) access.
template <typename T> struct Pack4;
template <> struct Pack4<float> {
    static __device__ __forceinline__ void load(const float* p, float o[4])
    {
        const float4 x = *reinterpret_cast<const float4*>(p);
        o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
    }
    static __device__ __forceinline__ void store(float* p, const float o[4])
    {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
};
template <typename H> struct Pack4Half {
    static __device__ __forceinline__ void load(const H* p, float o[4])
    {
        const uint2 x = *reinterpret_cast<const uint2*>(p);
        const H* h = reinterpret_cast<const H*>(&x);
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = to_f32(h[j]);
    }
    static __device__ __forceinline__ void store(H* p, const float o[4])
    {
        uint2 x;
        H* h = reinterpret_cast<H*>(&x);
#pragma unroll
        for (int j = 0; j < 4; ++j) h[j] = from_f32<H>(o[j]);
        *reinterpret_cast<uint2*>(p) = x;
    }
};
template <> struct Pack4<__nv_bfloat16> : Pack4Half<__nv_bfloat16> {};
template <> struct Pack4<__half> : Pack4Half<__half> {};

template <typename T> __device__ __forceinline__ bool aligned_for_pack(const void* p)
{
    return ((uintptr_t)p % (4 * sizeof(T))) == 0;
}

// Adam over one contiguous slice of a group (cnt elements from `base`),
// gradients from shared memory; optionally stores the gradients too.  Four
// elements per access and kAdamPacks packs per thread in flight; a scalar
// loop takes what is left (the partial last CTA, or unaligned buffers).
// PREFETCH: every iteration also asks L2 for the packs two iterations ahead
// (the next iteration's were asked for before the loop or by the previous
// iteration), so a thread keeps three iterations of parameter and moment
// lines in flight with registers for one.
constexpr int kAdamPacks = 2;
template <typename PT, typename MT, int PACKS = kAdamPacks, bool PREFETCH = false>
__device__ __forceinline__ void adam_slice(void* p, void* m, void* v, const float* sg, float* g_out,
                                           int64_t base, int64_t cnt, const AdamScalars& a, bool& bad)
{
    PT* __restrict__ pp = static_cast<PT*>(p) + base;
    MT* __restrict__ mm = static_cast<MT*>(m) + base;
    MT* __restrict__ vv = static_cast<MT*>(v) + base;
    float* __restrict__ go = g_out ? g_out + base : nullptr;
    const bool vec = aligned_for_pack<PT>(pp) && aligned_for_pack<MT>(mm) && aligned_for_pack<MT>(vv) &&
                     (!go || aligned_for_pack<float>(go));
    const int64_t n4 = vec ? cnt / 4 : 0;
    if (PREFETCH) {
#pragma unroll
        for (int u = 0; u < PACKS; ++u) {
            const int64_t q = threadIdx.x + (int64_t)(PACKS + u) * kBwdBlock;
            if (q < n4) {
                prefetch_l2(pp + 4 * q);
                prefetch_l2(mm + 4 * q);
                prefetch_l2(vv + 4 * q);
            }
        }
    }
    for (int64_t q0 = threadIdx.x; q0 < n4; q0 += PACKS * kBwdBlock) {
        float pv[PACKS][4], mv[PACKS][4], vvv[PACKS][4];
        int64_t qs[PACKS];
#pragma unroll
        for (int u = 0; u < PACKS; ++u) qs[u] = q0 + u * kBwdBlock;
        if (PREFETCH) {
#pragma unroll
            for (int u = 0; u < PACKS; ++u) {
                const int64_t q = qs[u] + (int64_t)(2 * PACKS) * kBwdBlock;
                if (q < n4) {
                    prefetch_l2(pp + 4 * q);
                    prefetch_l2(mm + 4 * q);
                    prefetch_l2(vv + 4 * q);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < PACKS; ++u) {
            if (qs[u] < n4) {
                Pack4<PT>::load(pp + 4 * qs[u], pv[u]);
                Pack4<MT>::load(mm + 4 * qs[u], mv[u]);
                Pack4<MT>::load(vv + 4 * qs[u], vvv[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < PACKS; ++u) {
            if (qs[u] >= n4) continue;
            const float4 g4 = *reinterpret_cast<const float4*>(sg + 4 * qs[u]);
            const float gg[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float vf = v_decode<MT>(vvv[u][j]);
                pv[u][j] = adam_update(pv[u][j], gg[j], mv[u][j], vf, a);
                bad |= adam_nonfinite(pv[u][j], mv[u][j], vf);
                if (v_vanishes<MT>(vf)) mv[u][j] = 0.f;
                vvv[u][j] = v_encode<MT>(vf);
            }
            Pack4<PT>::store(pp + 4 * qs[u], pv[u]);
            Pack4<MT>::store(mm + 4 * qs[u], mv[u]);
            Pack4<MT>::store(vv + 4 * qs[u], vvv[u]);
            if (go) Pack4<float>::store(go + 4 * qs[u], gg);
        }
    }
    for (int64_t e = 4 * n4 + threadIdx.x; e < cnt; e += kBwdBlock) {
        const float g = sg[e];
        float mf = to_f32(mm[e]);
        float vf = VStore<MT>::load(vv[e]);
        const float pf = adam_update(to_f32(pp[e]), g, mf, vf, a);
        bad |= adam_nonfinite(pf, mf, vf);
        if (v_vanishes<MT>(vf)) mf = 0.f;
        pp[e] = from_f32<PT>(pf);
        mm[e] = from_f32<MT>(mf);
        vv[e] = VStore<MT>::store(vf);
        if (go) go[e] = g;
    }
}

// One 4-element pack of one group's Adam slice, split into its loads and its
// update + stores, so that the packs of several small groups are in flight
// together (one memory round trip for all of them instead of one per group).
template <typename PT, typename MT> struct AdamPack {
    float p[4], m[4], v[4];
    bool on;
    __device__ __forceinline__ void load(const void* pp, const void* mm, const void* vv, int64_t e, bool use)
    {
        on = use;
        if (!use) return;
        Pack4<PT>::load(static_cast<const PT*>(pp) + e, p);
        Pack4<MT>::load(static_cast<const MT*>(mm) + e, m);
        Pack4<MT>::load(static_cast<const MT*>(vv) + e, v);
    }
    __device__ __forceinline__ void finish(void* pp, void* mm, void* vv, int64_t e, const float* sg, float* g_out,
                                           const AdamScalars& a, bool& bad)
    {
        if (!on) return;
        const float4 g4 = *reinterpret_cast<const float4*>(sg);
        const float gg[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float vf = v_decode<MT>(v[j]);
            p[j] = adam_update(p[j], gg[j], m[j], vf, a);
            bad |= adam_nonfinite(p[j], m[j], vf);
            if (v_vanishes<MT>(vf)) m[j] = 0.f;
            v[j] = v_encode<MT>(vf);
        }
        Pack4<PT>::store(static_cast<PT*>(pp) + e, p);
        Pack4<MT>::store(static_cast<MT*>(mm) + e, m);
        Pack4<MT>::store(static_cast<MT*>(vv) + e, v);
        if (g_out) Pack4<float>::store(g_out + e, gg);
    }
};

template <typename PT, typename MT>
__device__ __forceinline__ bool group_vectorisable(const AdamArgs& aa, int g, const float* g_out)
{
    return aligned_for_pack<PT>(aa.p[g]) && aligned_for_pack<MT>(aa.m[g]) && aligned_for_pack<MT>(aa.v[g]) &&
           (!g_out || aligned_for_pack<float>(g_out));
}

// L2 prefetches of one full CTA's Adam data, thread t its own packs: the
// merged small-group rounds (means, log-scales, quaternions, opacity,
// sh_dc) and the first two iterations of the sh_rest slice.
template <typename SHT, typename MT>
__device__ __forceinline__ void prefetch_cta(const AdamArgs& aa, int64_t i0, int t, bool small, bool rest)
{
    auto three = [&](const void* p, const void* m, const void* v, int64_t e, size_t pb) {
        prefetch_l2(static_cast<const char*>(p) + e * pb);
        prefetch_l2(static_cast<const char*>(m) + e * sizeof(MT));
        prefetch_l2(static_cast<const char*>(v) + e * sizeof(MT));
    };
    if (small) {
        if (t < 96) {
            three(aa.p[0], aa.m[0], aa.v[0], 3 * i0 + 4 * t, sizeof(float));
            three(aa.p[1], aa.m[1], aa.v[1], 3 * i0 + 4 * t, sizeof(float));
            three(aa.p[4], aa.m[4], aa.v[4], 3 * i0 + 4 * t, sizeof(SHT));
        }
        three(aa.p[2], aa.m[2], aa.v[2], 4 * i0 + 4 * t, sizeof(float));
        if (t < 32) three(aa.p[3], aa.m[3], aa.v[3], i0 + 4 * t, sizeof(float));
    }
    if (rest) {
#pragma unroll
        for (int u = 0; u < 2 * kAdamPacks; ++u)
            three(aa.p[5], aa.m[5], aa.v[5], 45 * i0 + 4 * (t + (int64_t)u * kBwdBlock), sizeof(SHT));
    }
}

// Gradients of all parameters of 128 Gaussians per CTA, summed over the
// views.  FUSED: instead of (only) storing them, the CTA applies the Adam
// step to its Gaussians right away -- every Gaussian, visible or not
// (Sec. 3.3) -- reading the step sizes from the device state; the gradient
// stores are then optional (null pointers skip them).
// The fused kernel is bound by how many bytes the Adam tail keeps in flight,
// i.e. by resident CTAs: compiled for 6 per SM (80 registers, a few spilled)
// it ran 1.11 ms per step on the 3M-Gaussian scene against 1.34 ms at 4 per
// SM (104 registers) and 1.19-1.24 ms at 7; at 5 (96 registers, no spill)
// 0.91 against 0.87 ms in z-order.  The motion variant spills twice as much
// at 6 and runs best at 5: 0.364 against 0.428 ms on the dynamic workload.
// A full CTA takes the small groups' Adam in two memory round trips (means,
// log-scales and quaternions; then opacity and sh_dc) instead of one per
// group: 0.831 against 0.900 ms.
constexpr int kFusedMinBlocks = 6;
constexpr int kFusedMinBlocksMotion = 5;

template <typename SHT, typename MT, bool FUSED, bool MOTION>
__global__ void __launch_bounds__(kBwdBlock, FUSED ? (MOTION ? kFusedMinBlocksMotion : kFusedMinBlocks) : 1)
preprocess_bwd_kernel(int64_t n, int sh_degree, const float* means, const float* log_scales,
                      const float* quats, const float* opac, const SHT* sh_dc, const SHT* sh_rest,
                      const fgs_camera* __restrict__ cams, ViewTable vt,
                      const Screen* __restrict__ screen, const TileRect* __restrict__ rects,
                      const ScreenGrad* __restrict__ sgrad,
                      float* __restrict__ g_means, float* __restrict__ g_scales,
                      float* __restrict__ g_quats, float* __restrict__ g_opac,
                      float* __restrict__ g_dc, float* __restrict__ g_rest, float* __restrict__ g_vel,
                      float* __restrict__ g_t0, Motion mo, AdamArgs aa)
{
    __shared__ __align__(16) float s_rest[kBwdBlock * 45];
    // FUSED: gradients of the small groups, one contiguous slice per group
    constexpr int kSmall = FUSED ? kBwdBlock * 18 : 1;
    __shared__ __align__(16) float s_small[kSmall];
    const int64_t i0 = (int64_t)blockIdx.x * kBwdBlock;
    const int64_t i = i0 + threadIdx.x;
    const bool valid = i < n;
    // FUSED, a full CTA: the small groups' Adam lines are asked of L2 before
    // the gradient pass, the first sh_rest lines before the small groups' rounds
    if (FUSED && i0 + kBwdBlock <= n) prefetch_cta<SHT, MT>(aa, i0, threadIdx.x, true, false);
    float gmu[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};
    float gw = 0.f;
    float gdc[3] = {0.f, 0.f, 0.f};
    float gvel[3] = {0.f, 0.f, 0.f}, gt0 = 0.f;  // dynamic Gaussians
    uint32_t vis_mask = 0;
    if (valid)
        for (int v = 0; v < vt.n_views; ++v)
            if (rects[(int64_t)v * n + i].count > 0) vis_mask |= 1u << v;
    float mu[3] = {0.f, 0.f, 0.f};
    const int ncoef = (sh_degree + 1) * (sh_degree + 1);
    // this Gaussian's sh_rest gradient row in shared memory (stride 45 floats:
    // consecutive threads fall in different banks), summed over the views
    float* my = s_rest + 45 * threadIdx.x;
#pragma unroll
    for (int q = 0; q < 45; ++q) my[q] = 0.f;
    if (vis_mask) {
        // the SH row the view-direction gradient reads, asked of L2 ahead of
        // the geometry (0.770 -> 0.756 ms at 3M Gaussians)
        const char* row = reinterpret_cast<const char*>(sh_rest + 45 * i);
        prefetch_l2(row);
        prefetch_l2(row + 64 * sizeof(SHT) / 2);
        prefetch_l2(row + 45 * sizeof(SHT) - 1);
        mu[0] = means[3 * i]; mu[1] = means[3 * i + 1]; mu[2] = means[3 * i + 2];
        const float4 q4 = *reinterpret_cast<const float4*>(quats + 4 * i);  // rows are 16-byte aligned
        const float qw = q4.x, qx = q4.y, qy = q4.z, qz = q4.w;
        const float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        const float inv = 1.0f / qn;
        const float qh[4] = {qw * inv, qx * inv, qy * inv, qz * inv};
        float Rq[9], s[3], M[9];
        quat_to_rot(qh[0], qh[1], qh[2], qh[3], Rq);
#pragma unroll
        for (int a = 0; a < 3; ++a) s[a] = __expf(log_scales[3 * i + a]);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) M[3 * r + c] = Rq[3 * r + c] * s[c];
        float dM_acc[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) dM_acc[a] = 0.f;
        // dynamic Gaussians: velocity, temporal centre and the opacity before
        // the temporal factor
        float vel[3] = {0.f, 0.f, 0.f}, t0 = 0.f, obase = 0.f;
        if (MOTION) {
            vel[0] = mo.vel[3 * i]; vel[1] = mo.vel[3 * i + 1]; vel[2] = mo.vel[3 * i + 2];
            t0 = mo.t0[i];
            obase = 1.0f / (1.0f + __expf(-opac[i]));
        }
        for (int v = 0; v < vt.n_views; ++v) {
            if (!(vis_mask >> v & 1u)) continue;
            const int64_t vi = (int64_t)v * n + i;
            const Screen rec = screen[vi];
            const uint32_t bits = __float_as_uint(rec.q2.w);
            const ScreenGrad g = sgrad[vi];
            const Cam cam = load_cam(cams, v);
            const float o = rec.q1.z;  // the opacity this view saw
            // the mean at this view's time
            const float dtime = MOTION ? cam.time - t0 : 0.f;
            float mv[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) mv[a] = MOTION ? mu[a] + vel[a] * dtime : mu[a];
            float t[3];
#pragma unroll
            for (int r = 0; r < 3; ++r)
                t[r] = cam.R[3 * r] * mv[0] + cam.R[3 * r + 1] * mv[1] + cam.R[3 * r + 2] * mv[2] + cam.t[r];
            const float iz = 1.0f / t[2], iz2 = iz * iz;
            float dmu[3] = {0.f, 0.f, 0.f}, dt[3] = {0.f, 0.f, 0.f};

            // opacity: o = sigmoid(w) (times the temporal factor p for dynamic
            // Gaussians: do/dw = p sigmoid' = o (1 - sigmoid), do/dt0 = o (t - t0) / sigma^2)
            gw += g.g1.y * o * (1.0f - (MOTION ? obase : o));
            if (MOTION) gt0 += g.g1.y * o * dtime * mo.inv_var;

            // colour -> view direction -> mean
            {
                float d[3], il, grgb[3];
                view_colour_grad(cam, mv, bits, g, d, il, grgb);
                float coef[16];
#pragma unroll
                for (int kk = 0; kk < 16; ++kk) coef[kk] = 0.f;
#pragma unroll
                for (int kk = 1; kk < 16; ++kk) {
                    if (kk < ncoef) {
                        const SHT* r3 = sh_rest + 45 * i + 3 * (kk - 1);
                        coef[kk] = to_f32(r3[0]) * grgb[0] + to_f32(r3[1]) * grgb[1] + to_f32(r3[2]) * grgb[2];
                    }
                }
                float gd[3];
                sh_dir_grad(d[0], d[1], d[2], sh_degree, coef, gd);
                const float dd = gd[0] * d[0] + gd[1] * d[1] + gd[2] * d[2];
#pragma unroll
                for (int a = 0; a < 3; ++a) dmu[a] += (gd[a] - d[a] * dd) * il;
                // band 0 (Y_0 is constant)
#pragma unroll
                for (int c = 0; c < 3; ++c) gdc[c] += SHC::c0 * grgb[c];
                // bands 1..3: d/dsh_kc += Y_k(dir) grgb_c
                float Y[16];
                sh_basis(d[0], d[1], d[2], sh_degree, Y);
#pragma unroll
                for (int kk = 1; kk < 16; ++kk)
                    if (kk < ncoef)
#pragma unroll
                        for (int c = 0; c < 3; ++c) my[3 * (kk - 1) + c] += Y[kk] * grgb[c];
            }

            // Eq. 1: mu2D = (fx tx/tz + cx, fy ty/tz + cy)
            const float gx = g.g0.x, gy = g.g0.y;
            dt[0] += gx * cam.fx * iz;
            dt[1] += gy * cam.fy * iz;
            dt[2] += -(gx * cam.fx * t[0] + gy * cam.fy * t[1]) * iz2;

            // the blend backward accumulates dL/dSigma2D (full symmetric, the
            // dilation has unit Jacobian): H = [[S00, S01], [S01, S11]]
            const float S00 = g.g0.z, S01 = g.g0.w, S11 = g.g1.x;

            // Sigma2D = T2 Sigma T2^T = (T2 M)(T2 M)^T with T2 = J Rcam
            const float j00 = cam.fx * iz, j02 = -cam.fx * t[0] * iz2;
            const float j11 = cam.fy * iz, j12 = -cam.fy * t[1] * iz2;
            float T2[6];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                T2[c] = j00 * cam.R[c] + j02 * cam.R[6 + c];
                T2[3 + c] = j11 * cam.R[3 + c] + j12 * cam.R[6 + c];
            }
            float M2[6];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    M2[3 * r + c] = T2[3 * r] * M[c] + T2[3 * r + 1] * M[3 + c] + T2[3 * r + 2] * M[6 + c];
            // dL/dM2 = 2 GS M2; dL/dT2 = dM2 M^T; dL/dM = T2^T dM2
            float dM2[6];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dM2[c] = 2.0f * (S00 * M2[c] + S01 * M2[3 + c]);
                dM2[3 + c] = 2.0f * (S01 * M2[c] + S11 * M2[3 + c]);
            }
            float dT2[6];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    dT2[3 * r + c] = dM2[3 * r] * M[3 * c] + dM2[3 * r + 1] * M[3 * c + 1] +
                                     dM2[3 * r + 2] * M[3 * c + 2];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) dM_acc[3 * r + c] += T2[r] * dM2[c] + T2[3 + r] * dM2[3 + c];
            // dJ = dT2 Rcam^T ; J entries used: j00, j02, j11, j12
            const float dj00 = dT2[0] * cam.R[0] + dT2[1] * cam.R[1] + dT2[2] * cam.R[2];
            const float dj02 = dT2[0] * cam.R[6] + dT2[1] * cam.R[7] + dT2[2] * cam.R[8];
            const float dj11 = dT2[3] * cam.R[3] + dT2[4] * cam.R[4] + dT2[5] * cam.R[5];
            const float dj12 = dT2[3] * cam.R[6] + dT2[4] * cam.R[7] + dT2[5] * cam.R[8];
            dt[0] += -dj02 * cam.fx * iz2;
            dt[1] += -dj12 * cam.fy * iz2;
            dt[2] += -dj00 * cam.fx * iz2 + 2.0f * dj02 * cam.fx * t[0] * iz2 * iz -
                     dj11 * cam.fy * iz2 + 2.0f * dj12 * cam.fy * t[1] * iz2 * iz;
            // t = Rcam mu(t) + tcam; mu(t) = mu + v (t - t0)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float dmv = dmu[a] + cam.R[a] * dt[0] + cam.R[3 + a] * dt[1] + cam.R[6 + a] * dt[2];
                gmu[a] += dmv;
                if (MOTION) {
                    gvel[a] += dmv * dtime;
                    gt0 -= dmv * vel[a];
                }
            }
        }
        // M = Rq S: dS, dRq -> log-scales and the quaternion
#pragma unroll
        for (int c = 0; c < 3; ++c)
            gls[c] = (dM_acc[c] * Rq[c] + dM_acc[3 + c] * Rq[3 + c] + dM_acc[6 + c] * Rq[6 + c]) * s[c];
        float G[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) G[3 * r + c] = dM_acc[3 * r + c] * s[c];
        const float w = qh[0], x = qh[1], y = qh[2], z = qh[3];
        float dq[4];
        dq[0] = 2.0f * (-z * G[1] + y * G[2] + z * G[3] - x * G[5] - y * G[6] + x * G[7]);
        dq[1] = 2.0f * (y * G[1] + z * G[2] + y * G[3] - 2.0f * x * G[4] - w * G[5] + z * G[6] +
                        w * G[7] - 2.0f * x * G[8]);
        dq[2] = 2.0f * (-2.0f * y * G[0] + x * G[1] + w * G[2] + x * G[3] + z * G[5] - w * G[6] +
                        z * G[7] - 2.0f * y * G[8]);
        dq[3] = 2.0f * (-2.0f * z * G[0] - w * G[1] + x * G[2] + w * G[3] - 2.0f * z * G[4] +
                        y * G[5] + x * G[6] + y * G[7]);
        const float qd = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
#pragma unroll
        for (int a = 0; a < 4; ++a) gq[a] = (dq[a] - qh[a] * qd) / qn;
    }
    if (FUSED) {
        // slices: means [0, 384), log-scales [384, 768), quats [768, 1280),
        // opacity [1280, 1408), sh_dc [1408, 1792), velocity [1792, 2176),
        // t0 [2176, 2304)
        const int t = threadIdx.x;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            s_small[3 * t + a] = gmu[a];
            s_small[3 * kBwdBlock + 3 * t + a] = gls[a];
            s_small[11 * kBwdBlock + 3 * t + a] = gdc[a];
            s_small[14 * kBwdBlock + 3 * t + a] = gvel[a];
        }
        s_small[17 * kBwdBlock + t] = gt0;
#pragma unroll
        for (int a = 0; a < 4; ++a) s_small[6 * kBwdBlock + 4 * t + a] = gq[a];
        s_small[10 * kBwdBlock + t] = gw;
        __syncthreads();
        bool bad = false;
        const int64_t nb = min((int64_t)kBwdBlock, n - i0);
        const bool merged = nb == kBwdBlock && group_vectorisable<float, MT>(aa, 0, g_means) &&
                      group_vectorisable<float, MT>(aa, 1, g_scales) &&
                      group_vectorisable<float, MT>(aa, 2, g_quats) &&
                      group_vectorisable<float, MT>(aa, 3, g_opac) && group_vectorisable<SHT, MT>(aa, 4, g_dc);
        if (merged) prefetch_cta<SHT, MT>(aa, i0, t, false, true);
        if (merged) {
            // a full CTA: the small groups' packs in two memory round trips,
            // thread t taking pack t of each (means, log-scales and sh_dc have
            // 96 packs, quaternions 128, opacity 32)
            {
                AdamPack<float, MT> a0, a1, a2;
                a0.load(aa.p[0], aa.m[0], aa.v[0], 3 * i0 + 4 * t, t < 96);
                a1.load(aa.p[1], aa.m[1], aa.v[1], 3 * i0 + 4 * t, t < 96);
                a2.load(aa.p[2], aa.m[2], aa.v[2], 4 * i0 + 4 * t, true);
                a0.finish(aa.p[0], aa.m[0], aa.v[0], 3 * i0 + 4 * t, s_small + 4 * t, g_means,
                          resolve(AdamScalars{}, aa.st, 0), bad);
                a1.finish(aa.p[1], aa.m[1], aa.v[1], 3 * i0 + 4 * t, s_small + 3 * kBwdBlock + 4 * t, g_scales,
                          resolve(AdamScalars{}, aa.st, 1), bad);
                a2.finish(aa.p[2], aa.m[2], aa.v[2], 4 * i0 + 4 * t, s_small + 6 * kBwdBlock + 4 * t, g_quats,
                          resolve(AdamScalars{}, aa.st, 2), bad);
            }
            {
                AdamPack<float, MT> b0;
                AdamPack<SHT, MT> b1;
                b0.load(aa.p[3], aa.m[3], aa.v[3], i0 + 4 * t, t < 32);
                b1.load(aa.p[4], aa.m[4], aa.v[4], 3 * i0 + 4 * t, t < 96);
                b0.finish(aa.p[3], aa.m[3], aa.v[3], i0 + 4 * t, s_small + 10 * kBwdBlock + 4 * t, g_opac,
                          resolve(AdamScalars{}, aa.st, 3), bad);
                b1.finish(aa.p[4], aa.m[4], aa.v[4], 3 * i0 + 4 * t, s_small + 11 * kBwdBlock + 4 * t, g_dc,
                          resolve(AdamScalars{}, aa.st, 4), bad);
            }
        } else {
            adam_slice<float, MT>(aa.p[0], aa.m[0], aa.v[0], s_small, g_means, 3 * i0, 3 * nb,
                                  resolve(AdamScalars{}, aa.st, 0), bad);
            adam_slice<float, MT>(aa.p[1], aa.m[1], aa.v[1], s_small + 3 * kBwdBlock, g_scales, 3 * i0,
                                  3 * nb, resolve(AdamScalars{}, aa.st, 1), bad);
            adam_slice<float, MT>(aa.p[2], aa.m[2], aa.v[2], s_small + 6 * kBwdBlock, g_quats, 4 * i0,
                                  4 * nb, resolve(AdamScalars{}, aa.st, 2), bad);
            adam_slice<float, MT>(aa.p[3], aa.m[3], aa.v[3], s_small + 10 * kBwdBlock, g_opac, i0, nb,
                                  resolve(AdamScalars{}, aa.st, 3), bad);
            adam_slice<SHT, MT>(aa.p[4], aa.m[4], aa.v[4], s_small + 11 * kBwdBlock, g_dc, 3 * i0, 3 * nb,
                                resolve(AdamScalars{}, aa.st, 4), bad);
        }
        // sh_rest, 76 % of the Adam bytes, with L2 prefetches two iterations
        // ahead: 0.832 -> 0.791 ms at 3M Gaussians (three ahead: 0.799); with
        // the CTA's first lines asked for earlier (prefetch_cta): 0.771
        adam_slice<SHT, MT, kAdamPacks, true>(aa.p[5], aa.m[5], aa.v[5], s_rest, g_rest, 45 * i0, 45 * nb,
                            resolve(AdamScalars{}, aa.st, 5), bad);
        if (MOTION) {
            adam_slice<float, MT>(aa.p[6], aa.m[6], aa.v[6], s_small + 14 * kBwdBlock, g_vel, 3 * i0, 3 * nb,
                                  resolve(AdamScalars{}, aa.st, 6), bad);
            adam_slice<float, MT>(aa.p[7], aa.m[7], aa.v[7], s_small + 17 * kBwdBlock, g_t0, i0, nb,
                                  resolve(AdamScalars{}, aa.st, 7), bad);
        }
        if (__syncthreads_or(bad) && threadIdx.x == 0) set_flag(aa.hdr, FGS_FLAG_NONFINITE);
        return;
    }
    if (valid) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            g_means[3 * i + a] = gmu[a];
            g_scales[3 * i + a] = gls[a];
            g_dc[3 * i + a] = gdc[a];
        }
        if (((uintptr_t)g_quats & 15) == 0) {
            *reinterpret_cast<float4*>(g_quats + 4 * i) = make_float4(gq[0], gq[1], gq[2], gq[3]);
        } else {
#pragma unroll
            for (int a = 0; a < 4; ++a) g_quats[4 * i + a] = gq[a];
        }
        g_opac[i] = gw;
        if (MOTION) {
#pragma unroll
            for (int a = 0; a < 3; ++a) g_vel[3 * i + a] = gvel[a];
            g_t0[i] = gt0;
        }
    }
    __syncthreads();
    // coalesced copy of the block's sh_rest gradients (128 * 45 floats)
    const int64_t cnt = min((int64_t)kBwdBlock, n - i0) * 45;
    float* dst = g_rest + i0 * 45;
    if (((uintptr_t)dst & 15) == 0) {
        const int64_t c4 = cnt / 4;
        for (int64_t e = threadIdx.x; e < c4; e += kBwdBlock)
            reinterpret_cast<float4*>(dst)[e] = reinterpret_cast<const float4*>(s_rest)[e];
        for (int64_t e = 4 * c4 + threadIdx.x; e < cnt; e += kBwdBlock) dst[e] = s_rest[e];
    } else {
        for (int64_t e = threadIdx.x; e < cnt; e += kBwdBlock) dst[e] = s_rest[e];
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static Motion motion_of(const fgs_params* p)
{
    Motion m{nullptr, nullptr, 0.f};
    if (p->data[6] && p->data[7]) {
        m.vel = (const float*)p->data[6];
        m.t0 = (const float*)p->data[7];
        m.inv_var = 1.0f / (p->sigma_t * p->sigma_t);
    }
    return m;
}

template <typename SHT>
static cudaError_t launch_pre_fwd_t(int64_t n, int deg, const fgs_params* p, const fgs_camera* cams,
                                    const ViewTable& vt, Screen* screen, TileRect* rects,
                                    uint32_t* local_off, uint32_t* block_sum, cudaStream_t st)
{
    const int nblk = (int)((n + kPreBlock - 1) / kPreBlock);
    const Motion mo = motion_of(p);
    auto kernel = mo.vel ? preprocess_fwd_kernel<SHT, true> : preprocess_fwd_kernel<SHT, false>;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ahead = (sms > 0 ? sms : 1) * 4;  // half of the 8 resident CTAs per SM
    kernel<<<nblk, kPreBlock, 0, st>>>(
        n, deg, (const float*)p->data[0], (const float*)p->data[1], (const float*)p->data[2],
        (const float*)p->data[3], (const SHT*)p->data[4], (const SHT*)p->data[5], cams, vt, screen,
        rects, local_off, block_sum, nblk, mo, ahead);
    profile_mark(st, "preprocess_fwd");
    return cudaGetLastError();
}

cudaError_t launch_preprocess_fwd(int64_t n, int deg, const fgs_params* p, const fgs_camera* cams,
                                  const ViewTable& vt, Screen* screen, TileRect* rects,
                                  uint32_t* local_off, uint32_t* block_sum, cudaStream_t st)
{
    switch (p->dtype[4]) {
    case FGS_BF16:
        return launch_pre_fwd_t<__nv_bfloat16>(n, deg, p, cams, vt, screen, rects, local_off, block_sum, st);
    case FGS_F16:
        return launch_pre_fwd_t<__half>(n, deg, p, cams, vt, screen, rects, local_off, block_sum, st);
    default:
        return launch_pre_fwd_t<float>(n, deg, p, cams, vt, screen, rects, local_off, block_sum, st);
    }
}

// After the preprocess: prefix of the CTA totals of rendered (view,
// Gaussian) pairs and their compaction into (depth bits, view * n + id) for
// the depth sort.
cudaError_t launch_compact_visible(int64_t n, const ViewTable& vt, const Screen* screen,
                                   const TileRect* rects, const uint32_t* local_off, uint32_t* block_sum,
                                   WsHeader* hdr, uint32_t* dkeys, uint32_t* dvals, cudaStream_t st)
{
    const int nblk = (int)((n + kPreBlock - 1) / kPreBlock);
    scan_block_sums_kernel<<<1, 1024, 0, st>>>(block_sum, (int64_t)vt.n_views * nblk, hdr, 0, false);
    profile_mark(st, "scan_block_sums");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)vt.n_views * n;
    compact_visible_kernel<<<(int)((total + 255) / 256), 256, 0, st>>>(n, vt, screen, rects, local_off,
                                                                       block_sum, nblk, dkeys, dvals);
    profile_mark(st, "compact_visible");
    return cudaGetLastError();
}

int64_t count_scan_blocks(int64_t pairs) { return (pairs + kCountTile - 1) / kCountTile; }

// After the depth sort (svals: view * n + id in depth order): the instance
// offsets in that order and the emission of the (tile, id) pairs.
// Grid of duplicate_big_kernel: 8 CTAs of 8 warps per SM, fewer for small
// inputs (at most one warp per rendered pair).
static int big_grid(int64_t pairs)
{
    static int sms[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (!sms[dev] && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms[dev] = 1;
    const int64_t want = (pairs + 7) / 8;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms[dev] * 8));
}

// `big`: scratch for the split order's large-rectangle list, one uint32 per
// rendered pair; `order`: FGS_DUPLICATE_STRIDED or FGS_DUPLICATE_SPLIT.
cudaError_t launch_sorted_duplicate(int64_t n, const ViewTable& vt, const Screen* screen,
                                    const TileRect* rects, const uint32_t* svals, uint32_t* sorted_off,
                                    uint32_t* sorted_block, WsHeader* hdr, int64_t k_max, uint32_t* keys,
                                    uint32_t* vals, uint32_t* big, int order, cudaStream_t st)
{
    const int64_t total = (int64_t)vt.n_views * n;
    const int64_t nb = count_scan_blocks(total);
    const uint32_t* n_vis = &hdr->counters[1];
    sorted_count_scan_kernel<<<(int)nb, kPreBlock, 0, st>>>(n_vis, svals, rects, sorted_off, sorted_block);
    profile_mark(st, "count_scan");
    scan_block_sums_kernel<<<1, 1024, 0, st>>>(sorted_block, nb, hdr, k_max, true);
    profile_mark(st, "scan_instance_sums");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int grid = (int)((total + 255) / 256);
    if (order == FGS_DUPLICATE_SPLIT) {
        duplicate_split_kernel<<<grid, 256, 0, st>>>(n, vt, rects, n_vis, svals, sorted_off, sorted_block, k_max,
                                                     keys, vals, big, &hdr->counters[2]);
        profile_mark(st, "duplicate");
        duplicate_big_kernel<<<big_grid(total), 256, 0, st>>>(n, vt, screen, rects, svals, sorted_off,
                                                              sorted_block, big, &hdr->counters[2], k_max, keys,
                                                              vals);
        profile_mark(st, "duplicate_big");
    } else {
        duplicate_kernel<<<grid, 256, 0, st>>>(n, vt, screen, rects, n_vis, svals, sorted_off, sorted_block,
                                               k_max, keys, vals);
        profile_mark(st, "duplicate");
    }
    return cudaGetLastError();
}

template <typename SHT>
static cudaError_t launch_pre_bwd_t(int64_t n, int deg, const fgs_params* p, const fgs_camera* cams,
                                    const ViewTable& vt, const Screen* screen, const TileRect* rects,
                                    const ScreenGrad* sgrad, const fgs_params* g, cudaStream_t st)
{
    const int grid = (int)((n + kBwdBlock - 1) / kBwdBlock);
    const Motion mo = motion_of(p);
    auto kernel = mo.vel ? preprocess_bwd_kernel<SHT, float, false, true>
                         : preprocess_bwd_kernel<SHT, float, false, false>;
    kernel<<<grid, kBwdBlock, 0, st>>>(
        n, deg, (const float*)p->data[0], (const float*)p->data[1], (const float*)p->data[2],
        (const float*)p->data[3], (const SHT*)p->data[4], (const SHT*)p->data[5], cams, vt, screen,
        rects, sgrad, (float*)g->data[0], (float*)g->data[1], (float*)g->data[2], (float*)g->data[3],
        (float*)g->data[4], (float*)g->data[5], (float*)g->data[6], (float*)g->data[7], mo,
        AdamArgs{});
    profile_mark(st, "preprocess_bwd");
    return cudaGetLastError();
}

cudaError_t launch_preprocess_bwd(int64_t n, int deg, const fgs_params* p, const fgs_camera* cams,
                                  const ViewTable& vt, const Screen* screen, const TileRect* rects,
                                  const ScreenGrad* sgrad, const fgs_params* g, cudaStream_t st)
{
    switch (p->dtype[4]) {
    case FGS_BF16:
        return launch_pre_bwd_t<__nv_bfloat16>(n, deg, p, cams, vt, screen, rects, sgrad, g, st);
    case FGS_F16:
        return launch_pre_bwd_t<__half>(n, deg, p, cams, vt, screen, rects, sgrad, g, st);
    default:
        return launch_pre_bwd_t<float>(n, deg, p, cams, vt, screen, rects, sgrad, g, st);
    }
}

template <typename SHT, typename MT>
static cudaError_t launch_pre_bwd_adam_t(int64_t n, int deg, const fgs_params* p, const fgs_camera* cams,
                                         const ViewTable& vt, const Screen* screen, const TileRect* rects,
                                         const ScreenGrad* sgrad,
                                         const fgs_params* g, const fgs_params* m, const fgs_params* v,
                                         const fgs_adam_state* ds, WsHeader* hdr, cudaStream_t st)
{
    const int grid = (int)((n + kBwdBlock - 1) / kBwdBlock);
    AdamArgs aa;
    aa.hdr = hdr;
    for (int k = 0; k < FGS_NUM_GROUPS; ++k) {
        aa.p[k] = p->data[k];
        aa.m[k] = m->data[k];
        aa.v[k] = v->data[k];
    }
    aa.st = ds;
    float* gp[FGS_NUM_GROUPS] = {};
    if (g)
        for (int k = 0; k < FGS_NUM_GROUPS; ++k) gp[k] = (float*)g->data[k];
    const Motion mo = motion_of(p);
    auto kernel = mo.vel ? preprocess_bwd_kernel<SHT, MT, true, true> : preprocess_bwd_kernel<SHT, MT, true, false>;
    kernel<<<grid, kBwdBlock, 0, st>>>(
        n, deg, (const float*)p->data[0], (const float*)p->data[1], (const float*)p->data[2],
        (const float*)p->data[3], (const SHT*)p->data[4], (const SHT*)p->data[5], cams, vt, screen,
        rects, sgrad, gp[0], gp[1], gp[2], gp[3], gp[4], gp[5], gp[6], gp[7], mo, aa);
    profile_mark(st, "preprocess_bwd_adam");
    return cudaGetLastError();
}

// Fused backward + Adam for the supported storage pairs: SH in float32 with
// float32 moments, SH in bf16 / fp16 with float32 moments or moments of the
// SH type.  Returns cudaErrorInvalidValue for any other pair (the caller
// checks first).
cudaError_t launch_preprocess_bwd_adam(int64_t n, int deg, const fgs_params* p, const fgs_camera* cams,
                                       const ViewTable& vt, const Screen* screen, const TileRect* rects,
                                       const ScreenGrad* sgrad,
                                       const fgs_params* g, const fgs_params* m, const fgs_params* v,
                                       const fgs_adam_state* ds, WsHeader* hdr, cudaStream_t st)
{
    const int sht = p->dtype[4], mt = m->dtype[0];
#define FGS_PB(S, M) launch_pre_bwd_adam_t<S, M>(n, deg, p, cams, vt, screen, rects, sgrad, g, m, v, ds, hdr, st)
    if (sht == FGS_F32 && mt == FGS_F32) return FGS_PB(float, float);
    if (sht == FGS_BF16 && mt == FGS_F32) return FGS_PB(__nv_bfloat16, float);
    if (sht == FGS_BF16 && mt == FGS_BF16) return FGS_PB(__nv_bfloat16, __nv_bfloat16);
    if (sht == FGS_F16 && mt == FGS_F32) return FGS_PB(__half, float);
    if (sht == FGS_F16 && mt == FGS_F16) return FGS_PB(__half, __half);
#undef FGS_PB
    return cudaErrorInvalidValue;
}

bool fused_adam_supported(int sh_dtype, int moment_dtype)
{
    return (sh_dtype == FGS_F32 && moment_dtype == FGS_F32) ||
           ((sh_dtype == FGS_BF16 || sh_dtype == FGS_F16) &&
            (moment_dtype == FGS_F32 || moment_dtype == sh_dtype));
}

}  // namespace fgs
