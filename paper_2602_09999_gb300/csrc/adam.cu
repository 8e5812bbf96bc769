// adam.cu -- fused Adam update (Suppl. A: beta = (0.9, 0.999), eps = 1e-15;
// Sec. 3.3 "Parameter Updates": one fused kernel with PyTorch's Adam
// formula, its roundings spelled out in adam_math.cuh).  Per element, in
// float32:
//   m = m + (1 - b1) (g - m)                     (PyTorch forms m with lerp)
//   v = b2 v + (1 - b2) g^2
//   p = p - step_size * m / (sqrt(v) / sqrt(1 - b2^t) + eps)
// with step_size = lr / (1 - b1^t), 1 - b1 and 1 - b2 formed in double and
// rounded once (0.999 is not a float32), as PyTorch does.
// Every element is updated, zero gradients included (Sec. 3.3).
// Storage: parameters float32 / bf16 / fp16; moments float32 / bf16 / fp16.
// An fp16 second moment is stored as sqrt(v): g^2 underflows fp16 for
// |g| < 2.4e-4 while |g| itself stays representable.  A second moment that
// still rounds to zero in its storage type stores the first moment as zero
// too (v_vanishes).
#include "adam_math.cuh"

namespace fgs {

// Advance the step and derive the step sizes (double precision) with the
// exponential decay of the means learning rate of Suppl. A (one thread).
__device__ void adam_prepare(fgs_adam_state* st)
{
    const int t = st->step + 1;
    st->step = t;
    const double bc1 = 1.0 - pow(st->beta1, (double)t);
    const double bc2 = 1.0 - pow(st->beta2, (double)t);
    for (int g = 0; g < FGS_NUM_GROUPS; ++g) {
        double lr = st->lr[g];
        if (g == 0 && st->lr_means_final > 0.0f && st->decay_steps > 0) {
            const double f = fmin((double)(t - 1) / (double)st->decay_steps, 1.0);
            lr = exp((1.0 - f) * log((double)st->lr[0]) + f * log((double)st->lr_means_final));
        }
        st->step_size[g] = (float)(lr / bc1);
    }
    st->inv_bc2_sqrt = (float)(1.0 / sqrt(bc2));
    st->beta1_f = (float)st->beta1;
    st->beta2_f = (float)st->beta2;
    st->one_minus_beta1_f = (float)(1.0 - st->beta1);
    st->one_minus_beta2_f = (float)(1.0 - st->beta2);
    st->eps_f = (float)st->eps;
}

__global__ void adam_prepare_kernel(fgs_adam_state* st) { adam_prepare(st); }

// Zeroes the screen-gradient records of every (view, 128-Gaussian block)
// with a rendered pair, one warp per (view, block); thread 0 of CTA 0 also
// prepares the Adam step (st non-null): the double-precision scalars take
// one thread about as long as the clear takes the grid, so the two share one
// launch.  Those records are the only ones the blend backward adds to and
// the preprocess backward reads (a pair is visible exactly when it is
// rendered).  block_sum: the forward's exclusive prefixes of rendered pairs
// per (view, block), view-major; total: their sum.
__global__ void __launch_bounds__(256)
zero_prepare_kernel(float4* __restrict__ dst, const uint32_t* __restrict__ block_sum,
                    const uint32_t* __restrict__ total, int64_t n, int nv, fgs_adam_state* st)
{
    if (st && blockIdx.x == 0 && threadIdx.x == 0) adam_prepare(st);
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t nblk = (n + kPreBlock - 1) / kPreBlock, pairs = nv * nblk;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < pairs; k += nwarps) {
        const uint32_t end = k + 1 < pairs ? block_sum[k + 1] : *total;
        if (end == block_sum[k]) continue;
        const int64_t v = k / nblk, i0 = (k - v * nblk) * kPreBlock;
        const int64_t words = 3 * min((int64_t)kPreBlock, n - i0);  // three 16-byte words a record
        float4* base = dst + 3 * (v * n + i0);
        for (int64_t w = lane; w < words; w += 32) base[w] = z;
    }
}

template <typename PT, typename MT>
__global__ void __launch_bounds__(256)
adam_kernel(int64_t count, PT* __restrict__ p, const float* __restrict__ g, MT* __restrict__ m,
            MT* __restrict__ v, AdamScalars a0, const fgs_adam_state* __restrict__ st, int grp)
{
    const AdamScalars a = resolve(a0, st, grp);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        float mm = to_f32(m[i]);
        float vv = VStore<MT>::load(v[i]);
        const float pn = adam_update(to_f32(p[i]), g[i], mm, vv, a);
        if (v_vanishes<MT>(vv)) mm = 0.f;
        p[i] = from_f32<PT>(pn);
        m[i] = from_f32<MT>(mm);
        v[i] = VStore<MT>::store(vv);
    }
}

// float32 everything, 16-byte aligned: four elements per thread and step.
__global__ void __launch_bounds__(256)
adam_f32x4_kernel(int64_t count4, float4* __restrict__ p, const float4* __restrict__ g,
                  float4* __restrict__ m, float4* __restrict__ v, AdamScalars a0,
                  const fgs_adam_state* __restrict__ st, int grp)
{
    const AdamScalars a = resolve(a0, st, grp);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count4; i += stride) {
        float4 pp = p[i], gg = __ldcs(&g[i]), mm = m[i], vv = v[i];
        pp.x = adam_update(pp.x, gg.x, mm.x, vv.x, a);
        pp.y = adam_update(pp.y, gg.y, mm.y, vv.y, a);
        pp.z = adam_update(pp.z, gg.z, mm.z, vv.z, a);
        pp.w = adam_update(pp.w, gg.w, mm.w, vv.w, a);
        if (vv.x == 0.f) mm.x = 0.f;
        if (vv.y == 0.f) mm.y = 0.f;
        if (vv.z == 0.f) mm.z = 0.f;
        if (vv.w == 0.f) mm.w = 0.f;
        p[i] = pp;
        m[i] = mm;
        v[i] = vv;
    }
}

static int grid_for(int64_t work)
{
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (work + 255) / 256;
    const int64_t cap = (int64_t)sms * 8;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

template <typename PT, typename MT>
static cudaError_t launch_typed(int64_t count, void* p, const float* g, void* m, void* v,
                                const AdamScalars& a, const fgs_adam_state* ds, int grp,
                                cudaStream_t st)
{
    adam_kernel<PT, MT><<<grid_for(count), 256, 0, st>>>(count, (PT*)p, g, (MT*)m, (MT*)v, a, ds, grp);
    profile_mark(st, "adam");
    return cudaGetLastError();
}

template <typename PT>
static cudaError_t launch_m(int mdt, int64_t count, void* p, const float* g, void* m, void* v,
                            const AdamScalars& a, const fgs_adam_state* ds, int grp, cudaStream_t st)
{
    switch (mdt) {
    case FGS_BF16: return launch_typed<PT, __nv_bfloat16>(count, p, g, m, v, a, ds, grp, st);
    case FGS_F16: return launch_typed<PT, __half>(count, p, g, m, v, a, ds, grp, st);
    default: return launch_typed<PT, float>(count, p, g, m, v, a, ds, grp, st);
    }
}

// sgrad: the [n_views * n] screen-gradient records; ds nullable.
cudaError_t launch_zero_and_adam_prepare(ScreenGrad* sgrad, const uint32_t* block_sum, const uint32_t* total,
                                         int64_t n, int nv, fgs_adam_state* ds, cudaStream_t st)
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t pairs = (int64_t)nv * ((n + kPreBlock - 1) / kPreBlock);
    const int64_t need = (pairs + 7) / 8, cap = (int64_t)sms * 8;  // 8 warps a CTA
    const int grid = (int)(need < 1 ? 1 : (need < cap ? need : cap));
    zero_prepare_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<float4*>(sgrad), block_sum, total, n, nv, ds);
    profile_mark(st, "zero_screen_grads");
    return cudaGetLastError();
}

cudaError_t launch_adam_prepare(fgs_adam_state* ds, cudaStream_t st)
{
    adam_prepare_kernel<<<1, 1, 0, st>>>(ds);
    profile_mark(st, "adam_prepare");
    return cudaGetLastError();
}

// One parameter group.  pdt / mdt: storage of the parameter and of both
// moments (the two moments share a type).  ds (nullable): device state whose
// scalars replace the host ones.
cudaError_t launch_adam_group(int64_t count, int pdt, int mdt, void* p, const float* g, void* m,
                              void* v, float step_size, float inv_bc2_sqrt, double b1, double b2,
                              double eps, const fgs_adam_state* ds, int grp, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const AdamScalars a{step_size, inv_bc2_sqrt, (float)b1, (float)b2, (float)(1.0 - b1),
                        (float)(1.0 - b2), (float)eps};
    const bool aligned = ((uintptr_t)p | (uintptr_t)g | (uintptr_t)m | (uintptr_t)v) % 16 == 0;
    if (pdt == FGS_F32 && mdt == FGS_F32 && aligned) {
        const int64_t c4 = count / 4;
        if (c4 > 0) {
            adam_f32x4_kernel<<<grid_for(c4), 256, 0, st>>>(c4, (float4*)p, (const float4*)g, (float4*)m,
                                                            (float4*)v, a, ds, grp);
            profile_mark(st, "adam");
        }
        const int64_t rest = count - 4 * c4;
        if (rest > 0) {
            adam_kernel<float, float><<<1, 32, 0, st>>>(rest, (float*)p + 4 * c4, g + 4 * c4,
                                                        (float*)m + 4 * c4, (float*)v + 4 * c4, a, ds, grp);
            profile_mark(st, "adam_tail");
        }
        return cudaGetLastError();
    }
    switch (pdt) {
    case FGS_BF16: return launch_m<__nv_bfloat16>(mdt, count, p, g, m, v, a, ds, grp, st);
    case FGS_F16: return launch_m<__half>(mdt, count, p, g, m, v, a, ds, grp, st);
    default: return launch_m<float>(mdt, count, p, g, m, v, a, ds, grp, st);
    }
}

}  // namespace fgs
