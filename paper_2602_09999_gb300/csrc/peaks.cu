// peaks.cu -- microbenchmarks of the rates that bound the blend kernels,
// which a plain copy and a dense GEMM do not measure: FP32 fused
// multiply-adds, the special-function unit's 2^x (ex2.approx, the one
// transcendental per evaluated fragment), and reads served by the L2 (the
// blends gather their screen records from L2).  The caller times each
// launch with CUDA events; the kernels only do the work and write a value
// that depends on all of it, so nothing can be optimised away.
#include "fgs_common.cuh"

namespace fgs {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;  // independent dependency chains per thread

__global__ void __launch_bounds__(kPeakThreads) fma_kernel(int iters, float a, float* __restrict__ out)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = __fmaf_rn(x[c], a, 0.5f);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) out[blockIdx.x] = s;  // never true for the arguments used; keeps the work
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void __launch_bounds__(kPeakThreads) ex2_kernel(int iters, float* __restrict__ out)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = -0.001f * (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = -ex2_approx(x[c]);  // stays in [-1, -0.5]
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads)
l2_read_kernel(const float4* __restrict__ buf, int64_t n4, int reps, float* __restrict__ out)
{
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t stride = (int64_t)gridDim.x * kPeakThreads;
    for (int r = 0; r < reps; ++r)
        for (int64_t i = (int64_t)blockIdx.x * kPeakThreads + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(buf + i);  // cached in L2 only
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
    const float s = acc.x + acc.y + acc.z + acc.w;
    if (s == 12345.678f) out[blockIdx.x] = s;
}

int peak_grid(int per_sm)
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms * per_sm;
}

}  // namespace
}  // namespace fgs

using namespace fgs;

extern "C" {

// FP32 FMA: grid_out receives the grid used; work = grid * 256 threads *
// iters * 8 fused multiply-adds (2 FLOP each).  out: device float[grid]
// (never written in practice).
int fgs_peak_fma(int32_t iters, float* out, int32_t* grid_out, void* stream)
{
    if (!out || !grid_out) return FGS_ERR_NULL;
    if (iters < 1) return FGS_ERR_ARG;
    const int grid = peak_grid(8);
    *grid_out = grid;
    fma_kernel<<<grid, kPeakThreads, 0, (cudaStream_t)stream>>>(iters, 0.999f, out);
    return cudaGetLastError() == cudaSuccess ? FGS_OK : FGS_ERR_CUDA;
}

// ex2.approx: work = grid * 256 * iters * 8 evaluations.
int fgs_peak_ex2(int32_t iters, float* out, int32_t* grid_out, void* stream)
{
    if (!out || !grid_out) return FGS_ERR_NULL;
    if (iters < 1) return FGS_ERR_ARG;
    const int grid = peak_grid(8);
    *grid_out = grid;
    ex2_kernel<<<grid, kPeakThreads, 0, (cudaStream_t)stream>>>(iters, out);
    return cudaGetLastError() == cudaSuccess ? FGS_OK : FGS_ERR_CUDA;
}

// L2 reads: `reps` passes over buf (n4 16-byte words, device, 16-byte
// aligned; small enough to stay in L2 after the first pass); work = reps *
// n4 * 16 bytes.
int fgs_peak_l2_read(const void* buf, int64_t n4, int32_t reps, float* out, int32_t* grid_out,
                     void* stream)
{
    if (!buf || !out || !grid_out) return FGS_ERR_NULL;
    if (n4 < 1 || reps < 1) return FGS_ERR_ARG;
    if ((uintptr_t)buf % 16 != 0) return FGS_ERR_ALIGN;
    const int grid = peak_grid(8);
    *grid_out = grid;
    l2_read_kernel<<<grid, kPeakThreads, 0, (cudaStream_t)stream>>>((const float4*)buf, n4, reps, out);
    return cudaGetLastError() == cudaSuccess ? FGS_OK : FGS_ERR_CUDA;
}

}  // extern "C"
