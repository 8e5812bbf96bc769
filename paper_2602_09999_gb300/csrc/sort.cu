// sort.cu -- stable LSD radix sort of (uint32 or uint64 key, uint32 value)
// pairs and the per-tile range extraction (Sec. 3.2 "Sorting", Suppl. B.2:
// O(k n) for k key bits).  The render path sorts in two stages: the visible
// (view, Gaussian) pairs by their 32-bit depth, then the instances emitted
// in that order by their tile id alone (a stable sort keeps the depth order
// inside each tile); the standalone entry points sort 64-bit keys.
//
// Each pass orders RB key bits (the last pass only the remaining ones; RB =
// 8 or 11, a launch choice that changes speed, never results) with three
// kernels:
//   upsweep   : per-CTA digit histogram of 4096 keys -> hist[digit][cta]
//   scan      : one CTA per digit, exclusive prefix over the CTAs
//   downsweep : stable rank of each key inside its CTA (warp ballots give
//               the peers with the same digit; per-warp digit counters keep
//               the input order), scatter to shared memory in digit order,
//               then coalesced writes of each digit run to its global slot.
// The number of valid keys is read from device memory, so the grid is sized
// for the capacity and the sort can be captured in a CUDA graph.
#include "fgs_common.cuh"

namespace fgs {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys per CTA
constexpr int kSortWarps = kSortThreads / 32;

// Digit histogram of 4096 keys per CTA.  With 8-bit digits each warp keeps
// its own copy (fewer shared-atomic collisions); with 11-bit digits two
// copies are shared by the warps (16 KB of shared memory).
template <typename KT, int RB>
__global__ void __launch_bounds__(kSortThreads)
radix_upsweep_kernel(const KT* __restrict__ keys, const uint32_t* __restrict__ n_dev,
                     int shift, uint32_t dmask, int nb_max, uint32_t* __restrict__ hist)
{
    constexpr int kRadix = 1 << RB;
    constexpr int kCopies = RB <= 8 ? kSortWarps : 2;
    __shared__ uint32_t h[kCopies][kRadix];
    const uint32_t n = *n_dev;
    const int nb = (int)((n + kSortTile - 1) / kSortTile);
    const int copy = (threadIdx.x >> 5) % kCopies;
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        const int64_t base = (int64_t)b * kSortTile;
        for (int d = threadIdx.x; d < kCopies * kRadix; d += kSortThreads) (&h[0][0])[d] = 0;
        __syncthreads();
        // all loads in flight before the first counter update
        KT k[kSortItems];
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const int64_t idx = base + (int64_t)r * kSortThreads + threadIdx.x;
            k[r] = idx < n ? __ldg(keys + idx) : (KT)0;
        }
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const int64_t idx = base + (int64_t)r * kSortThreads + threadIdx.x;
            if (idx < n) atomicAdd(&h[copy][(uint32_t)(k[r] >> shift) & dmask], 1u);
        }
        __syncthreads();
        for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
            uint32_t s = 0;
#pragma unroll
            for (int w = 0; w < kCopies; ++w) s += h[w][d];
            hist[(int64_t)d * nb_max + b] = s;
        }
        __syncthreads();
    }
}

// One CTA per digit: exclusive prefix of hist[d][0..nb) in place; the digit
// total goes to dtot[d].
__global__ void __launch_bounds__(256)
radix_scan_kernel(uint32_t* __restrict__ hist, const uint32_t* __restrict__ n_dev, int nb_max,
                  uint32_t* __restrict__ dtot)
{
    __shared__ uint32_t wsum[8];
    const uint32_t n = *n_dev;
    const int nb = (int)((n + kSortTile - 1) / kSortTile);
    uint32_t* row = hist + (int64_t)blockIdx.x * nb_max;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int chunk = (nb + 255) / 256;
    const int b0 = t * chunk, b1 = min(nb, b0 + chunk);
    uint32_t s = 0;
    for (int j = b0; j < b1; ++j) s += row[j];
    // exclusive scan of the 256 run totals: shuffles, then the 8 warp totals
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        before += w < warp ? wsum[w] : 0u;
        total += wsum[w];
    }
    uint32_t run = before + x - s;
    for (int j = b0; j < b1; ++j) {
        const uint32_t v = row[j];
        row[j] = run;
        run += v;
    }
    if (t == 255) dtot[blockIdx.x] = total;
}

template <typename KT, int RB> struct DownSmem {
    KT keys[kSortTile];
    uint32_t vals[kSortTile];
    uint32_t cnt[kSortWarps][1 << RB];  // per-warp digit counts, then their start in the tile
    uint32_t glob_off[1 << RB];
    uint32_t wsum[2][kSortWarps];
};

// Exclusive prefix over the CTA's 256 threads of (a, b); returns the
// prefixes, and the totals through ta, tb.  s_w: 2 x 8 words of scratch.
__device__ __forceinline__ void block_scan2(uint32_t a, uint32_t b, uint32_t& pa, uint32_t& pb, uint32_t& ta,
                                            uint32_t& tb, uint32_t (*s_w)[kSortWarps])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t xa = a, xb = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t ya = __shfl_up_sync(0xffffffffu, xa, o);
        const uint32_t yb = __shfl_up_sync(0xffffffffu, xb, o);
        if (lane >= o) {
            xa += ya;
            xb += yb;
        }
    }
    if (lane == 31) {
        s_w[0][warp] = xa;
        s_w[1][warp] = xb;
    }
    __syncthreads();
    uint32_t ba = 0, bb = 0;
    ta = tb = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
        ba += w < warp ? s_w[0][w] : 0u;
        bb += w < warp ? s_w[1][w] : 0u;
        ta += s_w[0][w];
        tb += s_w[1][w];
    }
    pa = ba + xa - a;
    pb = bb + xb - b;
}

template <typename KT, int RB>
__device__ __forceinline__ void radix_downsweep_tile(DownSmem<KT, RB>& S, const KT* __restrict__ keys_in,
                                                     const uint32_t* __restrict__ vals_in,
                                                     KT* __restrict__ keys_out,
                                                     uint32_t* __restrict__ vals_out,
                                                     const uint32_t* __restrict__ hist,
                                                     const uint32_t* __restrict__ dtot, uint32_t n,
                                                     int shift, uint32_t dmask, int nb_max, int b)
{
    constexpr int kRadix = 1 << RB;
    constexpr int kDpt = kRadix / kSortThreads;  // digits per thread in the digit scans
    const int64_t base = (int64_t)b * kSortTile;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int d = tid; d < kSortWarps * kRadix; d += kSortThreads) (&S.cnt[0][0])[d] = 0;
    __syncthreads();

    KT k[kSortItems];
    uint32_t val[kSortItems];
    uint32_t dr[kSortItems];  // digit (bits 20..31) | rank within the warp (bits 0..19)
    // all loads in flight before the ranking (its warp barriers would order them)
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t idx = base + (int64_t)warp * (kSortItems * 32) + r * 32 + lane;
        const bool valid = idx < n;
        k[r] = valid ? __ldg(keys_in + idx) : (KT)0;
        val[r] = valid ? __ldg(vals_in + idx) : 0u;
    }
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t idx = base + (int64_t)warp * (kSortItems * 32) + r * 32 + lane;
        const bool valid = idx < n;
        const uint32_t d = (uint32_t)(k[r] >> shift) & dmask;
        uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int bit = 0; bit < RB; ++bit) {
            const uint32_t bb = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
            peers &= ((d >> bit) & 1u) ? bb : ~bb;
        }
        const uint32_t before = __popc(peers & lt_mask);
        const uint32_t prior = valid ? S.cnt[warp][d] : 0u;
        __syncwarp();
        if (valid && before == (uint32_t)__popc(peers) - 1u) S.cnt[warp][d] = prior + __popc(peers);
        __syncwarp();
        dr[r] = valid ? ((d << 20) | (prior + before)) : 0xffffffffu;
    }
    __syncthreads();
    // per digit: prefix over the warps (in place) and the CTA total; thread t
    // owns digits t kDpt .. t kDpt + kDpt - 1
    uint32_t run[kDpt], gt[kDpt], sa = 0, sb = 0;
#pragma unroll
    for (int q = 0; q < kDpt; ++q) {
        const int d = tid * kDpt + q;
        uint32_t r = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = S.cnt[w][d];
            S.cnt[w][d] = r;
            r += c;
        }
        run[q] = r;
        gt[q] = dtot[d];
        sa += r;
        sb += gt[q];
    }
    // exclusive scans over the digits: CTA-local starts and global digit bases
    uint32_t pa, pb, ta, tb;
    block_scan2(sa, sb, pa, pb, ta, tb, S.wsum);
#pragma unroll
    for (int q = 0; q < kDpt; ++q) {
        const int d = tid * kDpt + q;
        // the digit's start in the tile goes into every warp's count
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) S.cnt[w][d] += pa;
        S.glob_off[d] = pb + hist[(int64_t)d * nb_max + b] - pa;
        pa += run[q];
        pb += gt[q];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        if (dr[r] == 0xffffffffu) continue;
        const uint32_t dd = dr[r] >> 20;
        const uint32_t pos = S.cnt[warp][dd] + (dr[r] & 0xfffffu);
        S.keys[pos] = k[r];
        S.vals[pos] = val[r];
    }
    __syncthreads();
    const int count = (int)min((int64_t)kSortTile, (int64_t)n - base);
    for (int j = tid; j < count; j += kSortThreads) {
        const KT key = S.keys[j];
        const uint32_t dd = (uint32_t)(key >> shift) & dmask;
        const uint32_t g = S.glob_off[dd] + j;
        keys_out[g] = key;
        vals_out[g] = S.vals[j];
    }
}

template <typename KT, int RB>
__global__ void __launch_bounds__(kSortThreads)
radix_downsweep_kernel(const KT* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                       KT* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                       const uint32_t* __restrict__ hist, const uint32_t* __restrict__ dtot,
                       const uint32_t* __restrict__ n_dev, int shift, uint32_t dmask, int nb_max)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DownSmem<KT, RB>& S = *reinterpret_cast<DownSmem<KT, RB>*>(smem_raw);
    const uint32_t n = *n_dev;
    const int nb = (int)((n + kSortTile - 1) / kSortTile);
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        radix_downsweep_tile(S, keys_in, vals_in, keys_out, vals_out, hist, dtot, n, shift, dmask, nb_max, b);
        __syncthreads();
    }
}

// [start, end) of each tile's run in the sorted tile keys; ranges must be
// zeroed.
__global__ void __launch_bounds__(256)
tile_ranges_kernel(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ n_dev,
                   uint2* __restrict__ ranges)
{
    const uint32_t n = *n_dev;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t tile = keys[j];
        if (j == 0) {
            ranges[tile].x = 0;
        } else {
            const uint32_t prev = keys[j - 1];
            if (prev != tile) {
                ranges[prev].y = (uint32_t)j;
                ranges[tile].x = (uint32_t)j;
            }
        }
        if (j == (int64_t)n - 1) ranges[tile].y = (uint32_t)n;
    }
}

// CTAs per SM times the SM count of the current device.
static int resident_grid(int per_sm)
{
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms * per_sm;
}

__global__ void set_count_kernel(uint32_t* dst, uint32_t value) { *dst = value; }

cudaError_t launch_set_count(uint32_t* dst, uint32_t value, cudaStream_t st)
{
    set_count_kernel<<<1, 1, 0, st>>>(dst, value);
    return cudaGetLastError();
}

// Histogram bytes of a sort of up to n_max keys with rb-bit digits: one row
// of CTA counts per digit, then the digit totals.
size_t sort_hist_bytes(int64_t n_max, int rb)
{
    const int64_t nb = (n_max + kSortTile - 1) / kSortTile;
    const int64_t radix = (int64_t)1 << rb;
    return (size_t)(radix * (nb > 0 ? nb : 1) + radix + 64) * sizeof(uint32_t);
}

// Passes of a sort of `bits` key bits with digits of rb bits.
int radix_passes(int bits, int rb) { return (bits + rb - 1) / rb; }

// Sorts n_dev[0] pairs on bits [0, bits) with RB-bit digits.  Returns 1 when
// the result is in the *_alt buffers.  hist: sort_hist_bytes(n_max) bytes.
// `labels` name the per-kernel profiling marks.
template <typename KT, int RB>
static int radix_sort_t(KT* keys, uint32_t* vals, KT* keys_alt, uint32_t* vals_alt, int64_t n_max,
                        const uint32_t* n_dev, int bits, uint32_t* hist, cudaStream_t st, cudaError_t* err,
                        const char* const labels[3])
{
    constexpr int kRadix = 1 << RB;
    const int smem = (int)sizeof(DownSmem<KT, RB>);
    cudaFuncSetAttribute(radix_downsweep_kernel<KT, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    const int nb_max = (int)((n_max + kSortTile - 1) / kSortTile);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, radix_downsweep_kernel<KT, RB>, kSortThreads,
                                                      smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int grid = nb_max < resident_grid(per_sm) ? nb_max : resident_grid(per_sm);
    uint32_t* dtot = hist + (int64_t)kRadix * (nb_max > 0 ? nb_max : 1);
    const int passes = radix_passes(bits, RB);
    KT *ki = keys, *ko = keys_alt;
    uint32_t *vi = vals, *vo = vals_alt;
    *err = cudaSuccess;
    if (nb_max == 0) return 0;
    for (int p = 0; p < passes; ++p) {
        const int shift = RB * p;
        const int dbits = bits - shift < RB ? bits - shift : RB;  // the last pass may be narrower
        const uint32_t dmask = (1u << dbits) - 1u;
        radix_upsweep_kernel<KT, RB><<<grid, kSortThreads, 0, st>>>(ki, n_dev, shift, dmask, nb_max, hist);
        profile_mark(st, labels[0]);
        radix_scan_kernel<<<kRadix, 256, 0, st>>>(hist, n_dev, nb_max, dtot);
        profile_mark(st, labels[1]);
        radix_downsweep_kernel<KT, RB><<<grid, kSortThreads, smem, st>>>(ki, vi, ko, vo, hist, dtot, n_dev,
                                                                         shift, dmask, nb_max);
        profile_mark(st, labels[2]);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            *err = e;
            return 0;
        }
        KT* tk = ki; ki = ko; ko = tk;
        uint32_t* tv = vi; vi = vo; vo = tv;
    }
    return passes & 1;
}

static const char* const kSortLabels[3] = {"sort_upsweep", "sort_scan", "sort_downsweep"};
static const char* const kDepthSortLabels[3] = {"depth_sort_upsweep", "depth_sort_scan",
                                                "depth_sort_downsweep"};

int radix_sort(unsigned long long* keys, uint32_t* vals, unsigned long long* keys_alt,
               uint32_t* vals_alt, int64_t n_max, const uint32_t* n_dev, int bits,
               uint32_t* hist, cudaStream_t st, cudaError_t* err)
{
    return radix_sort_t<unsigned long long, 8>(keys, vals, keys_alt, vals_alt, n_max, n_dev, bits, hist, st,
                                               err, kSortLabels);
}

// 32-bit keys: the depth sort (depth = true) and the tile sort of the render
// path, with digits of rb bits (8 or 11).
int radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, int64_t n_max,
                   const uint32_t* n_dev, int bits, uint32_t* hist, bool depth, int rb, cudaStream_t st,
                   cudaError_t* err)
{
    const char* const* labels = depth ? kDepthSortLabels : kSortLabels;
    if (rb == 11)
        return radix_sort_t<uint32_t, 11>(keys, vals, keys_alt, vals_alt, n_max, n_dev, bits, hist, st, err,
                                          labels);
    return radix_sort_t<uint32_t, 8>(keys, vals, keys_alt, vals_alt, n_max, n_dev, bits, hist, st, err, labels);
}

// 32-bit keys with the caller's profiling labels (the z-order sort).
int radix_sort_u32_labeled(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                           int64_t n_max, const uint32_t* n_dev, int bits, uint32_t* hist,
                           const char* const labels[3], cudaStream_t st, cudaError_t* err)
{
    return radix_sort_t<uint32_t, 8>(keys, vals, keys_alt, vals_alt, n_max, n_dev, bits, hist, st, err,
                                     labels);
}

cudaError_t launch_tile_ranges(const uint32_t* keys, const uint32_t* n_dev, int64_t n_max,
                               uint2* ranges, int total_tiles, cudaStream_t st)
{
    cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)total_tiles, st);
    profile_mark(st, "zero_ranges");
    const int grid = (int)min((n_max + 255) / 256, (int64_t)resident_grid(8));
    if (grid > 0) tile_ranges_kernel<<<grid, 256, 0, st>>>(keys, n_dev, ranges);
    profile_mark(st, "tile_ranges");
    return cudaGetLastError();
}

}  // namespace fgs
