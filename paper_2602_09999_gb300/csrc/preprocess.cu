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
#include "fgs_common.cuh"

namespace fgs {

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

template <typename SHT>
__device__ __forceinline__ void load_sh(const SHT* __restrict__ sh_dc, const SHT* __restrict__ sh_rest,
                                        int64_t i, int degree, float sh[16][3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) sh[0][c] = to_f32(sh_dc[3 * i + c]);
    const int ncoef = (degree + 1) * (degree + 1);
#pragma unroll
    for (int k = 1; k < 16; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            sh[k][c] = k < ncoef ? to_f32(sh_rest[45 * i + 3 * (k - 1) + c]) : 0.0f;
}

template <typename SHT>
__global__ void __launch_bounds__(kPreBlock)
preprocess_fwd_kernel(int64_t n, int sh_degree, const float* __restrict__ means,
                      const float* __restrict__ log_scales, const float* __restrict__ quats,
                      const float* __restrict__ opac, const SHT* __restrict__ sh_dc,
                      const SHT* __restrict__ sh_rest, const fgs_camera* __restrict__ cams,
                      ViewTable vt, Screen* __restrict__ screen, ushort4* __restrict__ rects,
                      uint32_t* __restrict__ local_off, uint32_t* __restrict__ block_sum,
                      int nblk)
{
    __shared__ uint32_t warp_tot[kPreBlock / 32];
    const int64_t i = (int64_t)blockIdx.x * kPreBlock + threadIdx.x;
    const bool valid = i < n;
    float mu[3] = {0.f, 0.f, 0.f}, M[9], o = 0.f;
    bool ok = false;
    if (valid) {
        mu[0] = means[3 * i];
        mu[1] = means[3 * i + 1];
        mu[2] = means[3 * i + 2];
        const float qw = quats[4 * i], qx = quats[4 * i + 1], qy = quats[4 * i + 2], qz = quats[4 * i + 3];
        const float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        const float inv = qn > 0.f ? 1.0f / qn : 0.f;
        float Rq[9];
        quat_to_rot(qw * inv, qx * inv, qy * inv, qz * inv, Rq);
        const float s0 = __expf(log_scales[3 * i]), s1 = __expf(log_scales[3 * i + 1]),
                    s2 = __expf(log_scales[3 * i + 2]);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            M[3 * r] = Rq[3 * r] * s0;
            M[3 * r + 1] = Rq[3 * r + 1] * s1;
            M[3 * r + 2] = Rq[3 * r + 2] * s2;
        }
        o = 1.0f / (1.0f + __expf(-opac[i]));
        ok = qn >= kQNormMin && o >= kAlphaMin;
    }
    float sh[16][3];
    bool sh_loaded = false;
    for (int v = 0; v < vt.n_views; ++v) {
        uint32_t count = 0;
        Screen rec;
        rec.q0 = make_float4(0.f, 0.f, 0.f, 0.f);
        rec.q1 = make_float4(0.f, 0.f, 0.f, 0.f);
        rec.q2 = make_float4(0.f, 0.f, 0.f, 0.f);
        ushort4 rect = make_ushort4(1, 1, 0, 0);
        if (ok) {
            const Cam cam = load_cam(cams, v);
            float t[3];
#pragma unroll
            for (int r = 0; r < 3; ++r)
                t[r] = cam.R[3 * r] * mu[0] + cam.R[3 * r + 1] * mu[1] + cam.R[3 * r + 2] * mu[2] + cam.t[r];
            if (t[2] > cam.near_plane) {
                const float iz = 1.0f / t[2];
                // Eq. 2: J (2x3) and T2 = J Rcam; M2 = T2 M, Sigma2D = M2 M2^T
                const float j00 = cam.fx * iz, j02 = -cam.fx * t[0] * iz * iz;
                const float j11 = cam.fy * iz, j12 = -cam.fy * t[1] * iz * iz;
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
                const float ca = M2[0] * M2[0] + M2[1] * M2[1] + M2[2] * M2[2];
                const float cb = M2[0] * M2[3] + M2[1] * M2[4] + M2[2] * M2[5];
                const float cc = M2[3] * M2[3] + M2[4] * M2[4] + M2[5] * M2[5];
                // Cauchy-Binet: det(M2 M2^T) = sum of squared 2x2 minors
                const float m01 = M2[0] * M2[4] - M2[1] * M2[3];
                const float m02 = M2[0] * M2[5] - M2[2] * M2[3];
                const float m12 = M2[1] * M2[5] - M2[2] * M2[4];
                const float det2 = m01 * m01 + m02 * m02 + m12 * m12;
                if (det2 >= kDetMin) {
                    const float da = ca + kDilation, dc = cc + kDilation;
                    const float detd = det2 + kDilation * (ca + cc) + kDilation * kDilation;
                    const float idet = 1.0f / detd;
                    const float conic_a = dc * idet, conic_b = -cb * idet, conic_c = da * idet;
                    const float mx = cam.fx * t[0] * iz + cam.cx;
                    const float my = cam.fy * t[1] * iz + cam.cy;
                    const float k = fmaxf(2.0f * __logf(255.0f * o), 0.0f);
                    const float ex = sqrtf(k * da), ey = sqrtf(k * dc);
                    const float u0 = fmaxf(ceilf(mx - ex - 0.5f), 0.0f);
                    const float u1 = fminf(floorf(mx + ex - 0.5f), (float)(cam.width - 1));
                    const float v0 = fmaxf(ceilf(my - ey - 0.5f), 0.0f);
                    const float v1 = fminf(floorf(my + ey - 0.5f), (float)(cam.height - 1));
                    if (u0 <= u1 && v0 <= v1) {
                        const int tx0 = (int)u0 / kTile, tx1 = (int)u1 / kTile;
                        const int ty0 = (int)v0 / kTile, ty1 = (int)v1 / kTile;
                        for (int ty = ty0; ty <= ty1; ++ty)
                            for (int tx = tx0; tx <= tx1; ++tx)
                                count += tile_keep(mx, my, conic_a, conic_b, conic_c, k, tx, ty,
                                                   cam.width, cam.height);
                        if (count > 0) {
                            rect = make_ushort4((unsigned short)tx0, (unsigned short)ty0,
                                                (unsigned short)tx1, (unsigned short)ty1);
                            if (!sh_loaded) {
                                load_sh(sh_dc, sh_rest, i, sh_degree, sh);
                                sh_loaded = true;
                            }
                            float d0 = mu[0] - cam.pos[0], d1 = mu[1] - cam.pos[1], d2 = mu[2] - cam.pos[2];
                            const float il = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
                            d0 *= il; d1 *= il; d2 *= il;
                            float Y[16];
                            sh_basis(d0, d1, d2, sh_degree, Y);
                            float rgb[3];
                            uint32_t bits = 8u;  // visible
#pragma unroll
                            for (int ch = 0; ch < 3; ++ch) {
                                float acc = 0.5f;
#pragma unroll
                                for (int kk = 0; kk < 16; ++kk) acc += Y[kk] * sh[kk][ch];
                                if (acc < 0.0f) {
                                    bits |= 1u << ch;
                                    acc = 0.0f;
                                }
                                rgb[ch] = acc;
                            }
                            rec.q0 = make_float4(mx, my, conic_a, conic_b);
                            rec.q1 = make_float4(conic_c, o, k, t[2]);
                            rec.q2 = make_float4(rgb[0], rgb[1], rgb[2], __uint_as_float(bits));
                        }
                    }
                }
            }
        }
        const int64_t vi = (int64_t)v * n + i;
        if (valid) {
            screen[vi] = rec;
            rects[vi] = rect;
        }
        uint32_t total;
        const uint32_t excl = block_exclusive_scan(count, warp_tot, total);
        if (valid) local_off[vi] = excl;
        if (threadIdx.x == 0) block_sum[(int64_t)v * nblk + blockIdx.x] = total;
    }
}

// Exclusive prefix of the CTA totals (one CTA); writes the total instance
// count (may exceed k_max) and the clamped count used by the sort.
__global__ void __launch_bounds__(1024)
scan_block_sums_kernel(uint32_t* __restrict__ block_sum, int64_t count, WsHeader* __restrict__ hdr,
                       int64_t k_max)
{
    __shared__ unsigned long long part[1024];
    const int t = threadIdx.x;
    const int64_t chunk = (count + 1023) / 1024;
    const int64_t b = t * chunk, e = min(count, b + chunk);
    unsigned long long s = 0;
    for (int64_t j = b; j < e; ++j) s += block_sum[j];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const unsigned long long y = t >= o ? part[t - o] : 0ull;
        __syncthreads();
        part[t] += y;
        __syncthreads();
    }
    unsigned long long run = part[t] - s;
    for (int64_t j = b; j < e; ++j) {
        const uint32_t x = block_sum[j];
        block_sum[j] = (uint32_t)min(run, 0xffffffffull);
        run += x;
    }
    if (t == 1023) {
        const unsigned long long tot = part[1023];
        hdr->instances = tot;
        hdr->counters[0] = (uint32_t)min(tot, (unsigned long long)k_max);
        if (tot > (unsigned long long)k_max) set_flag(hdr, FGS_FLAG_CAPACITY);
    }
}

__global__ void __launch_bounds__(256)
duplicate_kernel(int64_t n, ViewTable vt, const Screen* __restrict__ screen,
                 const ushort4* __restrict__ rects, const uint32_t* __restrict__ local_off,
                 const uint32_t* __restrict__ block_sum, int nblk, int64_t k_max,
                 unsigned long long* __restrict__ keys, uint32_t* __restrict__ vals)
{
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= (int64_t)vt.n_views * n) return;
    const int v = (int)(gi / n);
    const int64_t i = gi - (int64_t)v * n;
    const float4 q2 = screen[gi].q2;
    if (!(__float_as_uint(q2.w) & 8u)) return;
    const float4 q0 = screen[gi].q0;
    const float4 q1 = screen[gi].q1;
    const ushort4 r = rects[gi];
    uint64_t off = (uint64_t)local_off[gi] + block_sum[(int64_t)v * nblk + i / kPreBlock];
    const unsigned long long depth_bits = __float_as_uint(q1.w);
    const int width = vt.width[v], height = vt.height[v], tx_n = vt.tiles_x[v], toff = vt.tile_off[v];
    for (int ty = r.y; ty <= r.w; ++ty)
        for (int tx = r.x; tx <= r.z; ++tx) {
            if (!tile_keep(q0.x, q0.y, q0.z, q0.w, q1.x, q1.z, tx, ty, width, height)) continue;
            if (off < (uint64_t)k_max) {
                const unsigned long long tile = (unsigned long long)(toff + ty * tx_n + tx);
                keys[off] = (tile << 32) | depth_bits;
                vals[off] = (uint32_t)i;
            }
            ++off;
        }
}

// ---------------------------------------------------------------------------
// Backward of the preprocessing (chain rule, summed over views)
// ---------------------------------------------------------------------------
template <typename SHT>
__global__ void __launch_bounds__(128)
preprocess_bwd_kernel(int64_t n, int sh_degree, const float* __restrict__ means,
                      const float* __restrict__ log_scales, const float* __restrict__ quats,
                      const float* __restrict__ opac, const SHT* __restrict__ sh_dc,
                      const SHT* __restrict__ sh_rest, const fgs_camera* __restrict__ cams,
                      ViewTable vt, const Screen* __restrict__ screen,
                      const ScreenGrad* __restrict__ sgrad, float* __restrict__ g_means,
                      float* __restrict__ g_scales, float* __restrict__ g_quats,
                      float* __restrict__ g_opac, float* __restrict__ g_dc,
                      float* __restrict__ g_rest)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gmu[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};
    float gw = 0.f;
    float gsh[16][3];
#pragma unroll
    for (int k = 0; k < 16; ++k) gsh[k][0] = gsh[k][1] = gsh[k][2] = 0.f;
    bool any = false;
    float mu[3], qh[4], qn = 0.f, s[3], Rq[9], M[9], o = 0.f;
    float sh[16][3];
    for (int v = 0; v < vt.n_views; ++v) {
        const int64_t vi = (int64_t)v * n + i;
        const Screen rec = screen[vi];
        const uint32_t bits = __float_as_uint(rec.q2.w);
        if (!(bits & 8u)) continue;
        const ScreenGrad g = sgrad[vi];
        if (!any) {
            any = true;
            mu[0] = means[3 * i]; mu[1] = means[3 * i + 1]; mu[2] = means[3 * i + 2];
            const float qw = quats[4 * i], qx = quats[4 * i + 1], qy = quats[4 * i + 2], qz = quats[4 * i + 3];
            qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
            const float inv = 1.0f / qn;
            qh[0] = qw * inv; qh[1] = qx * inv; qh[2] = qy * inv; qh[3] = qz * inv;
            quat_to_rot(qh[0], qh[1], qh[2], qh[3], Rq);
#pragma unroll
            for (int a = 0; a < 3; ++a) s[a] = __expf(log_scales[3 * i + a]);
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) M[3 * r + c] = Rq[3 * r + c] * s[c];
            o = rec.q1.y;
            load_sh(sh_dc, sh_rest, i, sh_degree, sh);
        }
        const Cam cam = load_cam(cams, v);
        float t[3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
            t[r] = cam.R[3 * r] * mu[0] + cam.R[3 * r + 1] * mu[1] + cam.R[3 * r + 2] * mu[2] + cam.t[r];
        const float iz = 1.0f / t[2], iz2 = iz * iz;
        float dmu[3] = {0.f, 0.f, 0.f}, dt[3] = {0.f, 0.f, 0.f};

        // opacity: o = sigmoid(w)
        gw += g.g1.y * o * (1.0f - o);

        // colour: rgb_c = max(0, sum_k Y_k sh_kc + 0.5)
        {
            float d0 = mu[0] - cam.pos[0], d1 = mu[1] - cam.pos[1], d2 = mu[2] - cam.pos[2];
            const float len = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
            const float il = 1.0f / len;
            d0 *= il; d1 *= il; d2 *= il;
            float Y[16];
            sh_basis(d0, d1, d2, sh_degree, Y);
            const float grgb[3] = {(bits & 1u) ? 0.f : g.g1.z, (bits & 2u) ? 0.f : g.g1.w,
                                   (bits & 4u) ? 0.f : g.g2.x};
            float coef[16];
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                coef[kk] = 0.f;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    gsh[kk][ch] += Y[kk] * grgb[ch];
                    coef[kk] += sh[kk][ch] * grgb[ch];
                }
            }
            float gd[3];
            sh_dir_grad(d0, d1, d2, sh_degree, coef, gd);
            const float dd = gd[0] * d0 + gd[1] * d1 + gd[2] * d2;
            dmu[0] += (gd[0] - d0 * dd) * il;
            dmu[1] += (gd[1] - d1 * dd) * il;
            dmu[2] += (gd[2] - d2 * dd) * il;
        }

        // Eq. 1: mu2D = (fx tx/tz + cx, fy ty/tz + cy)
        const float gx = g.g0.x, gy = g.g0.y;
        dt[0] += gx * cam.fx * iz;
        dt[1] += gy * cam.fy * iz;
        dt[2] += -(gx * cam.fx * t[0] + gy * cam.fy * t[1]) * iz2;

        // conic = (Sigma2D + 0.3 I)^-1 : dSigma = -conic G conic, with G the
        // full symmetric gradient [[ga, gb/2], [gb/2, gc]]
        const float ca = rec.q0.z, cb = rec.q0.w, cc = rec.q1.x;
        const float ga = g.g0.z, gb = 0.5f * g.g0.w, gc = g.g1.x;
        const float P00 = ca * ga + cb * gb, P01 = ca * gb + cb * gc;
        const float P10 = cb * ga + cc * gb, P11 = cb * gb + cc * gc;
        const float S00 = -(P00 * ca + P01 * cb);
        const float S01 = -(P00 * cb + P01 * cc);
        const float S11 = -(P10 * cb + P11 * cc);

        // Sigma2D = T2 Sigma T2^T with T2 = J Rcam, Sigma = M M^T
        const float j00 = cam.fx * iz, j02 = -cam.fx * t[0] * iz2;
        const float j11 = cam.fy * iz, j12 = -cam.fy * t[1] * iz2;
        float T2[6];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T2[c] = j00 * cam.R[c] + j02 * cam.R[6 + c];
            T2[3 + c] = j11 * cam.R[3 + c] + j12 * cam.R[6 + c];
        }
        float Sig[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                Sig[3 * r + c] = M[3 * r] * M[3 * c] + M[3 * r + 1] * M[3 * c + 1] + M[3 * r + 2] * M[3 * c + 2];
        // U = T2 Sigma (2x3); dT2 = 2 GS U
        float U[6];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                U[3 * r + c] = T2[3 * r] * Sig[c] + T2[3 * r + 1] * Sig[3 + c] + T2[3 * r + 2] * Sig[6 + c];
        float dT2[6];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dT2[c] = 2.0f * (S00 * U[c] + S01 * U[3 + c]);
            dT2[3 + c] = 2.0f * (S01 * U[c] + S11 * U[3 + c]);
        }
        // dSigma = T2^T GS T2
        float dSig[9];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float a0 = S00 * T2[r] + S01 * T2[3 + r];
            const float a1 = S01 * T2[r] + S11 * T2[3 + r];
#pragma unroll
            for (int c = 0; c < 3; ++c) dSig[3 * r + c] = a0 * T2[c] + a1 * T2[3 + c];
        }
        // dJ = dT2 Rcam^T ; J entries used: j00, j02, j11, j12
        const float dj00 = dT2[0] * cam.R[0] + dT2[1] * cam.R[1] + dT2[2] * cam.R[2];
        const float dj02 = dT2[0] * cam.R[6] + dT2[1] * cam.R[7] + dT2[2] * cam.R[8];
        const float dj11 = dT2[3] * cam.R[3] + dT2[4] * cam.R[4] + dT2[5] * cam.R[5];
        const float dj12 = dT2[3] * cam.R[6] + dT2[4] * cam.R[7] + dT2[5] * cam.R[8];
        dt[0] += -dj02 * cam.fx * iz2;
        dt[1] += -dj12 * cam.fy * iz2;
        dt[2] += -dj00 * cam.fx * iz2 + 2.0f * dj02 * cam.fx * t[0] * iz2 * iz -
                 dj11 * cam.fy * iz2 + 2.0f * dj12 * cam.fy * t[1] * iz2 * iz;
        // t = Rcam mu + tcam
#pragma unroll
        for (int a = 0; a < 3; ++a)
            dmu[a] += cam.R[a] * dt[0] + cam.R[3 + a] * dt[1] + cam.R[6 + a] * dt[2];
#pragma unroll
        for (int a = 0; a < 3; ++a) gmu[a] += dmu[a];
        // Sigma = M M^T: dM = 2 dSigma M (dSigma symmetric); M = Rq S
        float dM[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                dM[3 * r + c] = 2.0f * (dSig[3 * r] * M[c] + dSig[3 * r + 1] * M[3 + c] + dSig[3 * r + 2] * M[6 + c]);
#pragma unroll
        for (int c = 0; c < 3; ++c)
            gls[c] += (dM[c] * Rq[c] + dM[3 + c] * Rq[3 + c] + dM[6 + c] * Rq[6 + c]) * s[c];
        float G[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) G[3 * r + c] = dM[3 * r + c] * s[c];
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
        for (int a = 0; a < 4; ++a) gq[a] += (dq[a] - qh[a] * qd) / qn;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        g_means[3 * i + a] = gmu[a];
        g_scales[3 * i + a] = gls[a];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) g_quats[4 * i + a] = gq[a];
    g_opac[i] = gw;
#pragma unroll
    for (int c = 0; c < 3; ++c) g_dc[3 * i + c] = gsh[0][c];
#pragma unroll
    for (int k = 1; k < 16; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) g_rest[45 * i + 3 * (k - 1) + c] = gsh[k][c];
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
template <typename SHT>
static cudaError_t launch_pre_fwd_t(int64_t n, int deg, const fgs_params* p, const fgs_camera* cams,
                                    const ViewTable& vt, Screen* screen, ushort4* rects,
                                    uint32_t* local_off, uint32_t* block_sum, cudaStream_t st)
{
    const int nblk = (int)((n + kPreBlock - 1) / kPreBlock);
    preprocess_fwd_kernel<SHT><<<nblk, kPreBlock, 0, st>>>(
        n, deg, (const float*)p->data[0], (const float*)p->data[1], (const float*)p->data[2],
        (const float*)p->data[3], (const SHT*)p->data[4], (const SHT*)p->data[5], cams, vt, screen,
        rects, local_off, block_sum, nblk);
    profile_mark(st, "preprocess_fwd");
    return cudaGetLastError();
}

cudaError_t launch_preprocess_fwd(int64_t n, int deg, const fgs_params* p, const fgs_camera* cams,
                                  const ViewTable& vt, Screen* screen, ushort4* rects,
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

cudaError_t launch_scan_and_duplicate(int64_t n, const ViewTable& vt, const Screen* screen,
                                      const ushort4* rects, const uint32_t* local_off,
                                      uint32_t* block_sum, WsHeader* hdr, int64_t k_max,
                                      unsigned long long* keys, uint32_t* vals, cudaStream_t st)
{
    const int nblk = (int)((n + kPreBlock - 1) / kPreBlock);
    scan_block_sums_kernel<<<1, 1024, 0, st>>>(block_sum, (int64_t)vt.n_views * nblk, hdr, k_max);
    profile_mark(st, "scan_block_sums");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)vt.n_views * n;
    const int grid = (int)((total + 255) / 256);
    duplicate_kernel<<<grid, 256, 0, st>>>(n, vt, screen, rects, local_off, block_sum, nblk, k_max,
                                           keys, vals);
    profile_mark(st, "duplicate");
    return cudaGetLastError();
}

template <typename SHT>
static cudaError_t launch_pre_bwd_t(int64_t n, int deg, const fgs_params* p, const fgs_camera* cams,
                                    const ViewTable& vt, const Screen* screen,
                                    const ScreenGrad* sgrad, const fgs_params* g, cudaStream_t st)
{
    const int grid = (int)((n + 127) / 128);
    preprocess_bwd_kernel<SHT><<<grid, 128, 0, st>>>(
        n, deg, (const float*)p->data[0], (const float*)p->data[1], (const float*)p->data[2],
        (const float*)p->data[3], (const SHT*)p->data[4], (const SHT*)p->data[5], cams, vt, screen,
        sgrad, (float*)g->data[0], (float*)g->data[1], (float*)g->data[2], (float*)g->data[3],
        (float*)g->data[4], (float*)g->data[5]);
    profile_mark(st, "preprocess_bwd");
    return cudaGetLastError();
}

cudaError_t launch_preprocess_bwd(int64_t n, int deg, const fgs_params* p, const fgs_camera* cams,
                                  const ViewTable& vt, const Screen* screen,
                                  const ScreenGrad* sgrad, const fgs_params* g, cudaStream_t st)
{
    switch (p->dtype[4]) {
    case FGS_BF16:
        return launch_pre_bwd_t<__nv_bfloat16>(n, deg, p, cams, vt, screen, sgrad, g, st);
    case FGS_F16:
        return launch_pre_bwd_t<__half>(n, deg, p, cams, vt, screen, sgrad, g, st);
    default:
        return launch_pre_bwd_t<float>(n, deg, p, cams, vt, screen, sgrad, g, st);
    }
}

}  // namespace fgs
