// adam_math.cuh -- the per-element Adam update shared by the standalone
// Adam kernels and the fused preprocess-backward + Adam kernel, so both take
// exactly the same steps (Suppl. A hyper-parameters; Sec. 3.3 "Parameter
// Updates").  It is PyTorch's formula, not its instruction sequence: the
// second-moment and parameter updates are fused multiply-adds, and the
// denominator is sqrt(v) * (1 / sqrt(1 - b2^t)) + eps in one fused step where
// PyTorch divides by sqrt(1 - b2^t) and then adds eps, so a result can differ
// from torch.optim.Adam in float32 by a few ulps.
#pragma once
#include "fgs_common.cuh"

namespace fgs {

template <typename MT> struct VStore {
    static __device__ __forceinline__ float load(MT x) { return to_f32(x); }
    static __device__ __forceinline__ MT store(float v) { return from_f32<MT>(v); }
};
template <> struct VStore<__half> {
    static __device__ __forceinline__ float load(__half x) { const float s = __half2float(x); return s * s; }
    static __device__ __forceinline__ __half store(float v) { return __float2half_rn(sqrtf(v)); }
};

// The same second-moment encoding on float values (fp16 holds sqrt(v)):
// VStore<MT>::load(x) == v_decode<MT>(to_f32(x)) and
// VStore<MT>::store(v) == from_f32<MT>(v_encode<MT>(v)).
template <typename MT> __device__ __forceinline__ float v_decode(float stored) { return stored; }
template <> __device__ __forceinline__ float v_decode<__half>(float s) { return s * s; }
template <typename MT> __device__ __forceinline__ float v_encode(float v) { return v; }
template <> __device__ __forceinline__ float v_encode<__half>(float v) { return sqrtf(v); }

// True when the second moment v (decoded value) rounds to zero in its
// storage type.  The first moment is then stored as zero too: an FP16 sqrt(v)
// underflows below |g| of about 2e-6 while m = (1 - b1) g still fits, and a
// later step would divide that m by eps = 1e-15 alone (a parameter thrown by
// 1e5 learning rates).  With float32 or bf16 storage v rounds to zero only
// when it is zero.
template <typename MT> __device__ __forceinline__ bool v_vanishes(float v) { return v == 0.f; }
template <> __device__ __forceinline__ bool v_vanishes<__nv_bfloat16>(float v)
{
    return __bfloat162float(__float2bfloat16_rn(v)) == 0.f;
}
template <> __device__ __forceinline__ bool v_vanishes<__half>(float v)
{
    return __half2float(__float2half_rn(sqrtf(v))) == 0.f;
}

struct AdamScalars {
    float step_size, inv_bc2_sqrt, b1, b2, omb1, omb2, eps;
};

// Scalars of group g: from the kernel argument, or from the device state.
__device__ __forceinline__ AdamScalars resolve(AdamScalars a, const fgs_adam_state* st, int g)
{
    if (st) {
        a.step_size = st->step_size[g];
        a.inv_bc2_sqrt = st->inv_bc2_sqrt;
        a.b1 = st->beta1_f;
        a.b2 = st->beta2_f;
        a.omb1 = st->one_minus_beta1_f;
        a.omb2 = st->one_minus_beta2_f;
        a.eps = st->eps_f;
    }
    return a;
}

// Every rounding is spelled out (no contraction left to the compiler), so
// the kernels that inline this take bit-identical steps.
__device__ __forceinline__ float adam_update(float p, float g, float& m, float& v, const AdamScalars& a)
{
    m = __fmaf_rn(a.omb1, __fsub_rn(g, m), m);
    v = __fmaf_rn(v, a.b2, __fmul_rn(__fmul_rn(a.omb2, g), g));
    const float denom = __fmaf_rn(__fsqrt_rn(v), a.inv_bc2_sqrt, a.eps);
    return __fmaf_rn(-a.step_size, __fdiv_rn(m, denom), p);
}

}  // namespace fgs
