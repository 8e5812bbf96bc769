// morton.cu -- locality-preserving order of the Gaussians (Sec. 3.3,
// "Locality-preserving densification"): z-order (Morton) codes of the means
// over their bounding box, a stable radix sort of (code, index), and a
// gather of every per-Gaussian buffer by the resulting permutation.
//
// After densification appends Gaussians at the end of the buffers, threads
// that are neighbours in a warp hold Gaussians far apart in space: their
// visibility differs (divergence in the preprocess and its backward) and
// the screen records a tile reads are scattered (cache misses).  Sorting by
// a z-order code puts Gaussians that are close in 3D close in memory.
//
// Bounding box: one pass over the means with float min/max taken as
// unsigned atomics on an order-preserving integer image of the float (sign
// bit flipped for non-negative values, all bits flipped for negative ones).
// Codes: 10 bits per axis in float32 with explicit round-to-nearest
// intrinsics (no contraction), so that any other float32 evaluation of the
// same expression gives the same integers.  Sort: the library's 32-bit
// radix sort on the low 30 bits (4 passes; stable, so equal codes keep
// index order).
#include "fgs_common.cuh"

namespace fgs {
int radix_sort_u32_labeled(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                           int64_t n_max, const uint32_t* n_dev, int bits, uint32_t* hist,
                           const char* const labels[3], cudaStream_t st, cudaError_t* err);
cudaError_t launch_set_count(uint32_t* dst, uint32_t value, cudaStream_t st);
size_t sort_hist_bytes(int64_t n_max, int rb);

namespace {

constexpr int kMortonBits = 10;                    // per axis
constexpr int kCodeBits = 3 * kMortonBits;         // 30
constexpr int kBoundsThreads = 192;                // a multiple of 3: fixed axis per thread
constexpr int kCodeThreads = 256;
constexpr int kPermuteThreads = 256;

const char* const kMortonLabels[3] = {"morton_sort_upsweep", "morton_sort_scan",
                                      "morton_sort_downsweep"};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Order-preserving map of a float to an unsigned integer and back.
__device__ __forceinline__ uint32_t float_key(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_float(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// box[0..2]: min keys, box[3..5]: max keys.
__global__ void bounds_init_kernel(uint32_t* box, uint32_t* n_dev, uint32_t n)
{
    const int t = threadIdx.x;
    if (t < 3) box[t] = 0xffffffffu;
    else if (t < 6) box[t] = 0u;
    else if (t == 6) *n_dev = n;
}

// Grid-stride over the 3n floats; the stride is a multiple of 3, so every
// thread sees one axis only.
__global__ void __launch_bounds__(kBoundsThreads)
bounds_kernel(const float* __restrict__ means, int64_t total, uint32_t* __restrict__ box)
{
    __shared__ uint32_t s_box[6];
    if (threadIdx.x < 6) s_box[threadIdx.x] = threadIdx.x < 3 ? 0xffffffffu : 0u;
    __syncthreads();
    const int64_t start = (int64_t)blockIdx.x * kBoundsThreads + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * kBoundsThreads;
    const int axis = (int)(start % 3);
    uint32_t lo = 0xffffffffu, hi = 0u;
    for (int64_t j = start; j < total; j += stride) {
        const uint32_t k = float_key(__ldg(means + j));
        lo = min(lo, k);
        hi = max(hi, k);
    }
    if (start < total) {
        atomicMin(&s_box[axis], lo);
        atomicMax(&s_box[3 + axis], hi);
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        if (s_box[threadIdx.x] != 0xffffffffu) atomicMin(&box[threadIdx.x], s_box[threadIdx.x]);
    } else if (threadIdx.x < 6) {
        if (s_box[threadIdx.x] != 0u) atomicMax(&box[threadIdx.x], s_box[threadIdx.x]);
    }
}

// Spreads the low 10 bits of v so that bit b moves to bit 3b.
__device__ __forceinline__ uint32_t spread3(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t quantise(float x, float lo, float s)
{
    // (x - lo) * s, each rounded to nearest; NaN (non-finite input) maps to 0
    const float v = __fmul_rn(__fsub_rn(x, lo), s);
    return (uint32_t)fminf(fmaxf(floorf(v), 0.0f), (float)((1 << kMortonBits) - 1));
}

__global__ void __launch_bounds__(kCodeThreads)
codes_kernel(const float* __restrict__ means, int64_t n, const uint32_t* __restrict__ box,
             uint32_t* __restrict__ codes, uint32_t* __restrict__ ids)
{
    __shared__ float s_lo[3], s_s[3];
    if (threadIdx.x < 3) {
        const float lo = key_float(box[threadIdx.x]);
        const float hi = key_float(box[3 + threadIdx.x]);
        const float ext = __fsub_rn(hi, lo);
        s_lo[threadIdx.x] = lo;
        s_s[threadIdx.x] = ext > 0.0f ? __fdiv_rn((float)(1 << kMortonBits), ext) : 0.0f;
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * kCodeThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kCodeThreads) {
        const float* m = means + 3 * i;
        const uint32_t qx = quantise(__ldg(m), s_lo[0], s_s[0]);
        const uint32_t qy = quantise(__ldg(m + 1), s_lo[1], s_s[1]);
        const uint32_t qz = quantise(__ldg(m + 2), s_lo[2], s_s[2]);
        codes[i] = spread3(qx) | (spread3(qy) << 1) | (spread3(qz) << 2);
        ids[i] = (uint32_t)i;
    }
}

// dst row i = src row order[i] (or row i when order is NULL), T the element.
template <typename T>
__global__ void __launch_bounds__(kPermuteThreads)
permute_kernel(const T* __restrict__ src, T* __restrict__ dst, const uint32_t* __restrict__ order,
               int64_t n, int width)
{
    const int64_t total = n * width;
    for (int64_t e = (int64_t)blockIdx.x * kPermuteThreads + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * kPermuteThreads) {
        const int64_t i = e / width;
        const int k = (int)(e - i * width);
        const int64_t from = order ? (int64_t)__ldg(order + i) : i;
        if (from < n) dst[e] = src[from * width + k];
    }
}

int grid_for(int64_t work, int threads, int per_sm)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    const int64_t need = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)sms * per_sm;
    return (int)(need < 1 ? 1 : (need < cap ? need : cap));
}

const int64_t kGroupWidth[FGS_NUM_GROUPS] = {3, 3, 4, 1, 3, 45, 3, 1};

size_t elem_size(int32_t dtype)
{
    return dtype == FGS_F32 ? 4 : (dtype == FGS_BF16 || dtype == FGS_F16) ? 2 : 0;
}

// Scratch: [count | box | codes (when the caller passes none) | codes alt | ids alt | histograms]
struct MortonScratch {
    size_t count, box, codes, codes_alt, ids_alt, hist, total;
};

MortonScratch morton_scratch(int64_t n)
{
    MortonScratch s;
    const size_t v = align256(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    s.count = 0;
    s.box = align256(sizeof(uint32_t) * 4);
    s.codes = s.box + align256(sizeof(uint32_t) * 6);
    s.codes_alt = s.codes + v;
    s.ids_alt = s.codes_alt + v;
    s.hist = s.ids_alt + v;
    s.total = s.hist + align256(sort_hist_bytes(n > 0 ? n : 0, 8));
    return s;
}

}  // namespace
}  // namespace fgs

using namespace fgs;

extern "C" {

size_t fgs_morton_scratch_bytes(int64_t n)
{
    return morton_scratch(n).total;
}

int fgs_morton_order(const float* means, int64_t n, uint32_t* order, uint32_t* codes, void* scratch,
                     size_t scratch_bytes, void* stream)
{
    if (n < 0 || n > 0x7fffffffll) return FGS_ERR_SHAPE;
    if (n == 0) return FGS_OK;
    if (!means || !order || !scratch) return FGS_ERR_NULL;
    const MortonScratch L = morton_scratch(n);
    if (scratch_bytes < L.total) return FGS_ERR_WORKSPACE;
    if ((uintptr_t)scratch % 256 != 0) return FGS_ERR_ALIGN;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = (unsigned char*)scratch;
    uint32_t* n_dev = (uint32_t*)(base + L.count);
    uint32_t* box = (uint32_t*)(base + L.box);
    uint32_t* keys = codes ? codes : (uint32_t*)(base + L.codes);
    uint32_t* keys_alt = (uint32_t*)(base + L.codes_alt);
    uint32_t* ids_alt = (uint32_t*)(base + L.ids_alt);
    uint32_t* hist = (uint32_t*)(base + L.hist);

    bounds_init_kernel<<<1, 32, 0, st>>>(box, n_dev, (uint32_t)n);
    profile_mark(st, "morton_bounds_init");
    bounds_kernel<<<grid_for(3 * n, kBoundsThreads, 4), kBoundsThreads, 0, st>>>(means, 3 * n, box);
    profile_mark(st, "morton_bounds");
    codes_kernel<<<grid_for(n, kCodeThreads, 8), kCodeThreads, 0, st>>>(means, n, box, keys, order);
    profile_mark(st, "morton_codes");
    if (cudaGetLastError() != cudaSuccess) return FGS_ERR_CUDA;
    cudaError_t e;
    const int in_alt = radix_sort_u32_labeled(keys, order, keys_alt, ids_alt, n, n_dev, kCodeBits, hist,
                                              kMortonLabels, st, &e);
    if (e != cudaSuccess) return FGS_ERR_CUDA;
    if (in_alt) {
        if (cudaMemcpyAsync(order, ids_alt, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess)
            return FGS_ERR_CUDA;
        if (codes && cudaMemcpyAsync(codes, keys_alt, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice,
                                     st) != cudaSuccess)
            return FGS_ERR_CUDA;
    }
    return FGS_OK;
}

int fgs_permute_params(const fgs_params* src, const fgs_params* dst, const uint32_t* order, void* stream)
{
    if (!src || !dst) return FGS_ERR_NULL;
    const int64_t n = src->n;
    if (n < 0 || n > 0x7fffffffll || dst->n != n) return FGS_ERR_SHAPE;
    if ((src->data[6] == nullptr) != (src->data[7] == nullptr)) return FGS_ERR_NULL;
    const int ng = src->data[6] ? FGS_NUM_GROUPS : 6;
    for (int g = 0; g < FGS_NUM_GROUPS; ++g) {
        const bool want = g < ng;
        if (want && (!src->data[g] || !dst->data[g])) return FGS_ERR_NULL;
        if (!want && dst->data[g]) return FGS_ERR_ARG;
        if (!want) continue;
        if (src->dtype[g] != dst->dtype[g] || elem_size(src->dtype[g]) == 0) return FGS_ERR_DTYPE;
        const size_t bytes = elem_size(src->dtype[g]) * (size_t)(kGroupWidth[g] * n);
        const uintptr_t a = (uintptr_t)src->data[g], b = (uintptr_t)dst->data[g];
        if (a < b + bytes && b < a + bytes) return FGS_ERR_ARG;   // overlapping src and dst
    }
    if (n == 0) return FGS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    for (int g = 0; g < ng; ++g) {
        const int w = (int)kGroupWidth[g];
        const int grid = grid_for(n * w, kPermuteThreads, 8);
        if (elem_size(src->dtype[g]) == 4)
            permute_kernel<uint32_t><<<grid, kPermuteThreads, 0, st>>>(
                (const uint32_t*)src->data[g], (uint32_t*)dst->data[g], order, n, w);
        else
            permute_kernel<uint16_t><<<grid, kPermuteThreads, 0, st>>>(
                (const uint16_t*)src->data[g], (uint16_t*)dst->data[g], order, n, w);
        profile_mark(st, "permute");
        if (cudaGetLastError() != cudaSuccess) return FGS_ERR_CUDA;
    }
    return FGS_OK;
}

}  // extern "C"
