// loss.cu -- fused L1 + D-SSIM loss and its gradient (Suppl. A: weights 0.8
// and 0.2; Sec. 4.1: the fused SSIM used by every compared method).
//
// SSIM of each channel uses local statistics under an 11x11 Gaussian window
// (sigma 1.5, normalised, zero padding): mu_x, mu_y, E[x^2], E[y^2], E[xy].
// For the gradient, with S the SSIM map,
//   dS/dx(p) = (w * D0)(p) + 2 x(p) (w * D1)(p) + y(p) (w * D2)(p)
// where D0 = dS/dmu_x (raw moments held fixed), D1 = dS/dE[x^2] and
// D2 = dS/dE[xy] are per-pixel maps and * is the same zero-padded blur.
//
//   ssim_fwd : per 32x16 block of pixels and channel: the block with its
//              5-pixel halo for x and y in shared memory (the next channel's
//              halo copied in asynchronously, into a second buffer, while
//              this channel computes), horizontal then
//              vertical blur of the five moments, SSIM, D0..D2 written to the
//              workspace maps, per-CTA sums of |x - y| and S.
//   ssim_bwd : per 32x16 block and channel: halo block of D0..D2, blur, and
//              dL/dx = s ((1 - lambda) sign(x - y) - lambda dS/dx) with
//              s = 1 / (3 H W n_views).
//              Its first CTA, before its own block, also sums the per-CTA
//              partials of ssim_fwd per view in a fixed order (double
//              precision) and writes the scalar loss.  A non-finite loss or
//              dL/dx sets the workspace's sticky FGS_FLAG_NONFINITE.
// The window weights are computed once on the host (double precision,
// rounded to float) and passed by value with the CTA grid of the views.
#include <cmath>

#include "fgs_common.cuh"

namespace fgs {

constexpr int kHalo = 5;
constexpr int kLTW = 32, kLTH = 16;         // output block of one CTA
constexpr int kSpanX = kLTW + 2 * kHalo;    // 42
constexpr int kSpanY = kLTH + 2 * kHalo;    // 26
constexpr int kLX = 32, kLY = 8;            // CTA shape (threadIdx.x, threadIdx.y)
constexpr int kSpanXP = 44;                 // even row stride: 8-byte loads of pixel pairs

// The CTA grid over all views and the window, passed by value.
struct LossGrid {
    int32_t cta_off[FGS_MAX_VIEWS + 1];  // first CTA of each view
    int32_t ctas_x[FGS_MAX_VIEWS];       // CTAs per block row of each view
    float w[11];                         // normalised Gaussian window, sigma 1.5
};

__device__ __forceinline__ int view_of_cta(const LossGrid& g, int nv, int b)
{
    int v = 0;
    while (v + 1 < nv && b >= g.cta_off[v + 1]) ++v;
    return v;
}

// Sums a and b over the CTA (256 threads) into red; valid in thread 0.
__device__ __forceinline__ void cta_sum2(float& a, float& b, float (*red)[kLY], int tid)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = a;
        red[1][tid >> 5] = b;
    }
    __syncthreads();
}

// 4-byte asynchronous copy global -> shared (cp.async), zero-filled when
// `in` is false (no byte of src is then read).
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool in)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(in ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Waits until at most N committed copy groups of this thread are in flight.
template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__global__ void __launch_bounds__(kLX * kLY)
ssim_fwd_kernel(ViewTable vt, LossGrid lg, const float* __restrict__ images,
                const float* __restrict__ targets, float* __restrict__ maps,
                double* __restrict__ partials)
{
    __shared__ __align__(8) float sxb[2][kSpanY][kSpanXP];
    __shared__ __align__(8) float syb[2][kSpanY][kSpanXP];
    __shared__ float hs[5][kSpanY][kLTW + 1];
    __shared__ float red[2][kLY];
    const int b = blockIdx.x;
    const int v = view_of_cta(lg, vt.n_views, b);
    const int lb = b - lg.cta_off[v];
    const int W = vt.width[v], H = vt.height[v];
    const int x0 = (lb % lg.ctas_x[v]) * kLTW, y0 = (lb / lg.ctas_x[v]) * kLTH;
    const int64_t P = (int64_t)W * H;
    const int64_t ptot = vt.total_pixels;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kLX + tx;
    const int px = x0 + tx;
    float l1 = 0.f, ssum = 0.f;
    // channel c's halo into buffer c & 1, in flight while channel c - 1 computes
    auto prefetch = [&](int c) {
        const float* X = images + 3 * vt.pix_off[v] + c * P;
        const float* Yt = targets + 3 * vt.pix_off[v] + c * P;
        for (int r = ty; r < kSpanY; r += kLY) {
            const int gy = y0 - kHalo + r;
            for (int cc = tx; cc < kSpanX; cc += kLX) {
                const int gx = x0 - kHalo + cc;
                const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
                const int64_t o = in ? (int64_t)gy * W + gx : 0;
                cp_async4(&sxb[c & 1][r][cc], X + o, in);
                cp_async4(&syb[c & 1][r][cc], Yt + o, in);
            }
        }
        cp_async_commit();
    };
    prefetch(0);
    for (int ch = 0; ch < 3; ++ch) {
        __syncthreads();  // iteration ch - 1 is done with buffer (ch + 1) & 1
        if (ch + 1 < 3) {
            prefetch(ch + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        float (*sx)[kSpanXP] = sxb[ch & 1];
        float (*sy)[kSpanXP] = syb[ch & 1];
        // horizontal blur: each thread two adjacent columns of one row, from
        // the 12 pixels both windows cover (six 8-byte loads per image)
        for (int r = tid >> 4; r < kSpanY; r += kLX * kLY / 16) {
            const int c2 = 2 * (tid & 15);
            float xv[12], yv[12];
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                const float2 x2 = *reinterpret_cast<const float2*>(&sx[r][c2 + 2 * j]);
                const float2 y2 = *reinterpret_cast<const float2*>(&sy[r][c2 + 2 * j]);
                xv[2 * j] = x2.x; xv[2 * j + 1] = x2.y;
                yv[2 * j] = y2.x; yv[2 * j + 1] = y2.y;
            }
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                float a = 0.f, bb_ = 0.f, aa = 0.f, yy = 0.f, ab = 0.f;
#pragma unroll
                for (int k = 0; k < 11; ++k) {
                    const float w = lg.w[k];
                    const float x = xv[o + k], y = yv[o + k];
                    a += w * x;
                    bb_ += w * y;
                    aa += w * x * x;
                    yy += w * y * y;
                    ab += w * x * y;
                }
                hs[0][r][c2 + o] = a; hs[1][r][c2 + o] = bb_; hs[2][r][c2 + o] = aa;
                hs[3][r][c2 + o] = yy; hs[4][r][c2 + o] = ab;
            }
        }
        __syncthreads();
        // vertical blur: each thread two adjacent rows of one column, one
        // moment at a time from the 12 rows both windows cover
        float mom[2][5];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            float hv[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) hv[k] = hs[m][2 * ty + k][tx];
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < 11; ++k) acc += lg.w[k] * hv[o + k];
                mom[o][m] = acc;
            }
        }
        for (int o = 0; o < 2; ++o) {
            const int oy = 2 * ty + o;
            const int py = y0 + oy;
            if (!(px < W && py < H)) continue;
            const float mx = mom[o][0], my = mom[o][1], exx = mom[o][2], eyy = mom[o][3], exy = mom[o][4];
            const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
            const float vx = exx - mx * mx, vy = eyy - my * my, cxy = exy - mx * my;
            const float n1 = 2.f * mx * my + C1, n2 = 2.f * cxy + C2;
            const float d1 = mx * mx + my * my + C1, d2 = vx + vy + C2;
            // S = n1 n2 / (d1 d2) and its partials, none of them divided by n1
            // or n2: n2 = 2 cov + C2 vanishes where the covariance is -C2 / 2,
            // and 2 S / n2 would then be 0 / 0
            const float den = d1 * d2;
            const float S = (n1 * n2) / den;
            const float dS_dmx = 2.f * my * n2 / den - 2.f * mx * S / d1;
            const float dS_dvx = -S / d2;
            const float dS_dcxy = 2.f * n1 / den;
            const int64_t gp = vt.pix_off[v] + (int64_t)py * W + px;
            maps[(int64_t)(3 * ch + 0) * ptot + gp] = dS_dmx - 2.f * mx * dS_dvx - my * dS_dcxy;
            maps[(int64_t)(3 * ch + 1) * ptot + gp] = dS_dvx;
            maps[(int64_t)(3 * ch + 2) * ptot + gp] = dS_dcxy;
            ssum += S;
            l1 += fabsf(sx[oy + kHalo][tx + kHalo] - sy[oy + kHalo][tx + kHalo]);
        }
    }
    cta_sum2(l1, ssum, red, tid);
    if (tid == 0) {
        double a = 0.0, c = 0.0;
        for (int w = 0; w < kLY; ++w) {
            a += red[0][w];
            c += red[1][w];
        }
        partials[2 * b] = a;
        partials[2 * b + 1] = c;
    }
}

// The scalar loss from the per-CTA partials (256 threads; red: scratch).
__device__ void reduce_loss(const ViewTable& vt, const LossGrid& lg, const double* __restrict__ partials,
                            float lambda, float* __restrict__ loss_out, double (*red)[256], int tid,
                            WsHeader* __restrict__ hdr)
{
    double total = 0.0;
    for (int v = 0; v < vt.n_views; ++v) {
        double a = 0.0, b = 0.0;
        for (int t = lg.cta_off[v] + tid; t < lg.cta_off[v + 1]; t += 256) {
            a += partials[2 * t];
            b += partials[2 * t + 1];
        }
        red[0][tid] = a;
        red[1][tid] = b;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (tid < o) {
                red[0][tid] += red[0][tid + o];
                red[1][tid] += red[1][tid + o];
            }
            __syncthreads();
        }
        const double inv = 1.0 / (3.0 * (double)vt.width[v] * (double)vt.height[v]);
        total += (1.0 - lambda) * red[0][0] * inv + lambda * (1.0 - red[1][0] * inv);
        __syncthreads();
    }
    if (tid == 0) {
        const float loss = (float)(total / vt.n_views);
        loss_out[0] = loss;
        if (!isfinite(loss)) set_flag(hdr, FGS_FLAG_NONFINITE);
    }
}

__global__ void __launch_bounds__(kLX * kLY)
ssim_bwd_kernel(ViewTable vt, LossGrid lg, const float* __restrict__ images,
                const float* __restrict__ targets, const float* __restrict__ maps, float lambda,
                float* __restrict__ dL, const double* __restrict__ partials, float* __restrict__ loss_out,
                WsHeader* __restrict__ hdr)
{
    __shared__ __align__(16) float sm[3][kSpanY][kSpanX + 1];
    __shared__ float hs[3][kSpanY][kLTW + 1];
    static_assert(sizeof(sm) >= 2 * 256 * sizeof(double), "room for the loss reduction");
    const int b = blockIdx.x;
    // the first CTA (scheduled first) sums ssim_fwd's partials, complete
    // before this kernel started, then takes its own block
    if (b == 0)
        reduce_loss(vt, lg, partials, lambda, loss_out, reinterpret_cast<double(*)[256]>(&sm[0][0][0]),
                    threadIdx.y * kLX + threadIdx.x, hdr);
    const int v = view_of_cta(lg, vt.n_views, b);
    const int lb = b - lg.cta_off[v];
    const int W = vt.width[v], H = vt.height[v];
    const int x0 = (lb % lg.ctas_x[v]) * kLTW, y0 = (lb / lg.ctas_x[v]) * kLTH;
    const int64_t P = (int64_t)W * H;
    const int64_t ptot = vt.total_pixels;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int px = x0 + tx;
    const float scale = 1.0f / (3.0f * (float)P * (float)vt.n_views);
    bool nonfinite = false;
    for (int ch = 0; ch < 3; ++ch) {
        __syncthreads();
        for (int r = ty; r < kSpanY; r += kLY) {
            const int gy = y0 - kHalo + r;
            for (int c = tx; c < kSpanX; c += kLX) {
                const int gx = x0 - kHalo + c;
                const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
                const int64_t gp = vt.pix_off[v] + (int64_t)gy * W + gx;
#pragma unroll
                for (int m = 0; m < 3; ++m) sm[m][r][c] = in ? maps[(int64_t)(3 * ch + m) * ptot + gp] : 0.f;
            }
        }
        __syncthreads();
        for (int r = ty; r < kSpanY; r += kLY) {
            float a = 0.f, bb_ = 0.f, d = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) {
                const float w = lg.w[k];
                a += w * sm[0][r][tx + k];
                bb_ += w * sm[1][r][tx + k];
                d += w * sm[2][r][tx + k];
            }
            hs[0][r][tx] = a; hs[1][r][tx] = bb_; hs[2][r][tx] = d;
        }
        __syncthreads();
        for (int oy = ty; oy < kLTH; oy += kLY) {
            const int py = y0 + oy;
            if (!(px < W && py < H)) continue;
            float b0 = 0.f, b1 = 0.f, b2 = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) {
                const float w = lg.w[k];
                b0 += w * hs[0][oy + k][tx];
                b1 += w * hs[1][oy + k][tx];
                b2 += w * hs[2][oy + k][tx];
            }
            const int64_t off = 3 * vt.pix_off[v] + ch * P + (int64_t)py * W + px;
            const float x = images[off], y = targets[off];
            const float dssim = b0 + 2.f * x * b1 + y * b2;
            const float diff = x - y;
            const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
            const float grad = scale * ((1.0f - lambda) * sgn - lambda * dssim);
            dL[off] = grad;
            nonfinite |= !isfinite(grad);
        }
    }
    if (__syncthreads_or(nonfinite) && threadIdx.x == 0 && threadIdx.y == 0) set_flag(hdr, FGS_FLAG_NONFINITE);
}

static LossGrid loss_grid(const ViewTable& vt)
{
    LossGrid g;
    int32_t off = 0;
    for (int v = 0; v < vt.n_views; ++v) {
        g.cta_off[v] = off;
        g.ctas_x[v] = (vt.width[v] + kLTW - 1) / kLTW;
        off += g.ctas_x[v] * ((vt.height[v] + kLTH - 1) / kLTH);
    }
    for (int v = vt.n_views; v <= FGS_MAX_VIEWS; ++v) g.cta_off[v] = off;
    for (int v = vt.n_views; v < FGS_MAX_VIEWS; ++v) g.ctas_x[v] = 1;
    double s = 0.0;
    for (int i = 0; i < 11; ++i) s += std::exp(-(double)((i - 5) * (i - 5)) / 4.5);
    for (int i = 0; i < 11; ++i) g.w[i] = (float)(std::exp(-(double)((i - 5) * (i - 5)) / 4.5) / s);
    return g;
}

cudaError_t launch_loss(const ViewTable& vt, const float* images, const float* targets, float lambda,
                        float* maps, double* partials, float* loss_out, float* dL, WsHeader* hdr,
                        cudaStream_t st)
{
    if (vt.total_tiles <= 0) return cudaSuccess;
    const LossGrid lg = loss_grid(vt);
    const int ctas = lg.cta_off[vt.n_views];
    const dim3 block(kLX, kLY);
    ssim_fwd_kernel<<<ctas, block, 0, st>>>(vt, lg, images, targets, maps, partials);
    profile_mark(st, "loss_ssim_fwd");
    ssim_bwd_kernel<<<ctas, block, 0, st>>>(vt, lg, images, targets, maps, lambda, dL, partials, loss_out,
                                                hdr);
    profile_mark(st, "loss_ssim_bwd");
    return cudaGetLastError();
}

}  // namespace fgs
