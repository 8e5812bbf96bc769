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
//   ssim_fwd : per 16x16 tile and channel: halo tile of x and y in shared
//              memory, horizontal then vertical blur of the five moments,
//              SSIM, D0..D2 written to the workspace maps, per-CTA sums of
//              |x - y| and S.
//   ssim_bwd : per 16x16 tile and channel: halo tile of D0..D2, blur, and
//              dL/dx = s ((1 - lambda) sign(x - y) - lambda dS/dx) with
//              s = 1 / (3 H W n_views).
//   loss_reduce : one CTA sums the per-CTA partials per view in a fixed
//              order (double precision) and writes the scalar loss.
#include "fgs_common.cuh"

namespace fgs {

constexpr int kHalo = 5;
constexpr int kSpan = kTile + 2 * kHalo;  // 26

// Normalised 11-tap Gaussian window (sigma 1.5) into shared memory; every
// CTA computes it, so no upload or synchronisation is needed.
__device__ __forceinline__ void load_window(float* w)
{
    if (threadIdx.x < 11) {
        float s = 0.f;
        for (int i = 0; i < 11; ++i) s += expf(-(float)((i - 5) * (i - 5)) / 4.5f);
        const int d = (int)threadIdx.x - 5;
        w[threadIdx.x] = expf(-(float)(d * d) / 4.5f) / s;
    }
}

__global__ void __launch_bounds__(256)
ssim_fwd_kernel(ViewTable vt, const float* __restrict__ images, const float* __restrict__ targets,
                float* __restrict__ maps, double* __restrict__ partials)
{
    __shared__ float sx[kSpan][kSpan + 1], sy[kSpan][kSpan + 1];
    __shared__ float hs[5][kSpan][kTile + 1];
    __shared__ float red[2][8];
    __shared__ float c_win[11];
    load_window(c_win);
    const int tile = blockIdx.x;
    const int v = view_of_tile(vt, tile);
    const int lt = tile - vt.tile_off[v];
    const int W = vt.width[v], H = vt.height[v];
    const int x0 = (lt % vt.tiles_x[v]) * kTile, y0 = (lt / vt.tiles_x[v]) * kTile;
    const int64_t P = (int64_t)W * H;
    const int64_t ptot = vt.total_pixels;
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
    const int px = x0 + tx, py = y0 + ty;
    const bool inside = px < W && py < H;
    const int64_t pix = (int64_t)py * W + px;
    float l1 = 0.f, ssum = 0.f;
    for (int ch = 0; ch < 3; ++ch) {
        const float* X = images + 3 * vt.pix_off[v] + ch * P;
        const float* Yt = targets + 3 * vt.pix_off[v] + ch * P;
        __syncthreads();
        for (int e = threadIdx.x; e < kSpan * kSpan; e += 256) {
            const int r = e / kSpan, c = e % kSpan;
            const int gx = x0 - kHalo + c, gy = y0 - kHalo + r;
            const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
            sx[r][c] = in ? X[(int64_t)gy * W + gx] : 0.f;
            sy[r][c] = in ? Yt[(int64_t)gy * W + gx] : 0.f;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < kSpan * kTile; e += 256) {
            const int r = e / kTile, c = e % kTile;
            float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) {
                const float w = c_win[k];
                const float xv = sx[r][c + k], yv = sy[r][c + k];
                a += w * xv;
                b += w * yv;
                aa += w * xv * xv;
                bb += w * yv * yv;
                ab += w * xv * yv;
            }
            hs[0][r][c] = a; hs[1][r][c] = b; hs[2][r][c] = aa; hs[3][r][c] = bb; hs[4][r][c] = ab;
        }
        __syncthreads();
        float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) {
            const float w = c_win[k];
            mx += w * hs[0][ty + k][tx];
            my += w * hs[1][ty + k][tx];
            exx += w * hs[2][ty + k][tx];
            eyy += w * hs[3][ty + k][tx];
            exy += w * hs[4][ty + k][tx];
        }
        if (inside) {
            const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
            const float vx = exx - mx * mx, vy = eyy - my * my, cxy = exy - mx * my;
            const float n1 = 2.f * mx * my + C1, n2 = 2.f * cxy + C2;
            const float d1 = mx * mx + my * my + C1, d2 = vx + vy + C2;
            const float S = (n1 * n2) / (d1 * d2);
            const float dS_dmx = S * (2.f * my / n1 - 2.f * mx / d1);
            const float dS_dvx = -S / d2;
            const float dS_dcxy = 2.f * S / n2;
            const int64_t gp = vt.pix_off[v] + pix;
            maps[(int64_t)(3 * ch + 0) * ptot + gp] = dS_dmx - 2.f * mx * dS_dvx - my * dS_dcxy;
            maps[(int64_t)(3 * ch + 1) * ptot + gp] = dS_dvx;
            maps[(int64_t)(3 * ch + 2) * ptot + gp] = dS_dcxy;
            ssum += S;
            l1 += fabsf(sx[ty + kHalo][tx + kHalo] - sy[ty + kHalo][tx + kHalo]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l1 += __shfl_xor_sync(0xffffffffu, l1, o);
        ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = l1;
        red[1][threadIdx.x >> 5] = ssum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 8; ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        partials[2 * tile] = a;
        partials[2 * tile + 1] = b;
    }
}

__global__ void __launch_bounds__(256)
ssim_bwd_kernel(ViewTable vt, const float* __restrict__ images, const float* __restrict__ targets,
                const float* __restrict__ maps, float lambda, float* __restrict__ dL)
{
    __shared__ float sm[3][kSpan][kSpan + 1];
    __shared__ float hs[3][kSpan][kTile + 1];
    __shared__ float c_win[11];
    load_window(c_win);
    const int tile = blockIdx.x;
    const int v = view_of_tile(vt, tile);
    const int lt = tile - vt.tile_off[v];
    const int W = vt.width[v], H = vt.height[v];
    const int x0 = (lt % vt.tiles_x[v]) * kTile, y0 = (lt / vt.tiles_x[v]) * kTile;
    const int64_t P = (int64_t)W * H;
    const int64_t ptot = vt.total_pixels;
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
    const int px = x0 + tx, py = y0 + ty;
    const bool inside = px < W && py < H;
    const int64_t pix = (int64_t)py * W + px;
    const float scale = 1.0f / (3.0f * (float)P * (float)vt.n_views);
    for (int ch = 0; ch < 3; ++ch) {
        __syncthreads();
        for (int e = threadIdx.x; e < kSpan * kSpan; e += 256) {
            const int r = e / kSpan, c = e % kSpan;
            const int gx = x0 - kHalo + c, gy = y0 - kHalo + r;
            const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
            const int64_t gp = vt.pix_off[v] + (int64_t)gy * W + gx;
#pragma unroll
            for (int m = 0; m < 3; ++m) sm[m][r][c] = in ? maps[(int64_t)(3 * ch + m) * ptot + gp] : 0.f;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < kSpan * kTile; e += 256) {
            const int r = e / kTile, c = e % kTile;
            float a = 0.f, b = 0.f, d = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) {
                const float w = c_win[k];
                a += w * sm[0][r][c + k];
                b += w * sm[1][r][c + k];
                d += w * sm[2][r][c + k];
            }
            hs[0][r][c] = a; hs[1][r][c] = b; hs[2][r][c] = d;
        }
        __syncthreads();
        if (inside) {
            float b0 = 0.f, b1 = 0.f, b2 = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) {
                const float w = c_win[k];
                b0 += w * hs[0][ty + k][tx];
                b1 += w * hs[1][ty + k][tx];
                b2 += w * hs[2][ty + k][tx];
            }
            const int64_t off = 3 * vt.pix_off[v] + ch * P + pix;
            const float x = images[off], y = targets[off];
            const float dssim = b0 + 2.f * x * b1 + y * b2;
            const float diff = x - y;
            const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
            dL[off] = scale * ((1.0f - lambda) * sgn - lambda * dssim);
        }
    }
}

__global__ void __launch_bounds__(256)
loss_reduce_kernel(ViewTable vt, const double* __restrict__ partials, float lambda,
                   float* __restrict__ loss_out)
{
    __shared__ double red[2][256];
    double total = 0.0;
    for (int v = 0; v < vt.n_views; ++v) {
        double a = 0.0, b = 0.0;
        for (int t = vt.tile_off[v] + threadIdx.x; t < vt.tile_off[v + 1]; t += 256) {
            a += partials[2 * t];
            b += partials[2 * t + 1];
        }
        red[0][threadIdx.x] = a;
        red[1][threadIdx.x] = b;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                red[0][threadIdx.x] += red[0][threadIdx.x + o];
                red[1][threadIdx.x] += red[1][threadIdx.x + o];
            }
            __syncthreads();
        }
        const double inv = 1.0 / (3.0 * (double)vt.width[v] * (double)vt.height[v]);
        total += (1.0 - lambda) * red[0][0] * inv + lambda * (1.0 - red[1][0] * inv);
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_out[0] = (float)(total / vt.n_views);
}

cudaError_t launch_loss(const ViewTable& vt, const float* images, const float* targets, float lambda,
                        float* maps, double* partials, float* loss_out, float* dL, cudaStream_t st)
{
    if (vt.total_tiles <= 0) return cudaSuccess;
    ssim_fwd_kernel<<<vt.total_tiles, 256, 0, st>>>(vt, images, targets, maps, partials);
    profile_mark(st, "loss_ssim_fwd");
    ssim_bwd_kernel<<<vt.total_tiles, 256, 0, st>>>(vt, images, targets, maps, lambda, dL);
    profile_mark(st, "loss_ssim_bwd");
    loss_reduce_kernel<<<1, 256, 0, st>>>(vt, partials, lambda, loss_out);
    profile_mark(st, "loss_reduce");
    return cudaGetLastError();
}

}  // namespace fgs
