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
// atomics this design reduces).  The per-Gaussian screen gradient it
// accumulates is dL/dSigma2D directly, dpow (C d)(C d)^T / 2 per fragment,
// instead of dL/dconic followed by -C G C: for needle-like splats the conic
// gradient is large and C G C cancels by orders of magnitude in float32,
// while C d is well conditioned.  It sums these in the conic's eigen basis
// (frag_moments) and rotates the sums once per entry.  The CTA walks the same list back to front
// from the largest last-contributor position of its pixels; each pixel
// recovers T_i = T_{i+1} / (1 - alpha_i) and the colour behind it,
// A_i = alpha_{i+1} c_{i+1} + (1 - alpha_{i+1}) A_{i+1} (A = bg behind the
// last), so dC/dalpha_i = T_i (c_i - A_i) and dC/dc_i = alpha_i T_i; only
// the scalar g . A_i is kept, g = dL/dC of the pixel.  The 9
// per-fragment sums are summed over the warp with shuffles, over the
// CTA with shared-memory atomics, and leave the CTA as one set of global
// vector atomics per (instance, CTA).
//
// Per-Gaussian backward (Sec. 3.2 "Per-Gaussian Backward" and its details in
// the supplement, after Mallick et al.), selected by fgs_tuning: each tile's
// list is cut into buckets of 32 entries.  The forward also stores, for every
// pixel still blending there, (T, C) in front of each bucket's first entry.
// The backward runs one warp per bucket, lane j holding entry j: the lanes
// replay the blend front to back as a pipeline over the tile's pixels that
// are still active at the bucket (at step s lane j works on pixel s - j and
// hands (T, C) to lane j + 1 with shuffles); the colour behind entry j is
// R_j = (C_pixel - C_{<=j}) / T_{j+1}, and each lane sums its entry's
// gradients over the pixels in registers, then adds them with one set of
// atomics per bucket.  Per-pixel inputs are staged in shared memory 32
// pixels at a time by the whole warp (the paper's refinement).
#include "fgs_common.cuh"

namespace fgs {

constexpr float kLog2e = 1.4426950408889634f;

// 2 ln 2: converts the exp2-scaled axis coordinates back to C d (below).
constexpr float kTwoLn2 = 1.3862943611198906f;

// One list entry staged in shared memory for one tile: the conic's eigen
// form as its two axes pre-scaled for exp2, the scaled axis coordinates at
// the tile's first pixel centre, colour and opacity.  With a = ls log2(e) /
// 2, b = lb log2(e) / 2 and the major axis (c, s), coef = (c sqrt(a),
// s sqrt(a), c sqrt(b), s sqrt(b)), so that with u' = coef.x dx + coef.y dy
// and w' = coef.z dy - coef.w dx the exponent of Eq. 3 in base 2 is
// -(u'^2 + w'^2) = -(log2 e / 2) d^T conic d, never positive.  Both
// coordinates are affine in the pixel position, so a pixel at (lx, ly)
// within the tile has u' = uw0.x + coef.x lx + coef.y ly (and likewise
// w'), which pixels of one row share in part (eval_frag).
// The first 16 bytes also carry the entry's block mask (block_mask), so a
// warp reads the mask and the coordinates in one load and skips the rest of
// the entry when the mask misses its blocks.
struct Entry {
    float2 uw0;
    uint32_t mask, pad;
    float4 coef;
    float4 rgbo;  // r, g, b, o
};

// uw0 and the mask of a staged entry in one 16-byte shared-memory load.
__device__ __forceinline__ uint32_t load_head(const Entry& s, float2& uw0)
{
    const float4 h = *reinterpret_cast<const float4*>(&s);
    uw0 = make_float2(h.x, h.y);
    return __float_as_uint(h.z);
}

// Thread -> pixel map with PPT pixels per thread: the CTA covers one 16x16
// tile, split into 8 blocks of 8 columns x 4 rows (block b: columns
// 8 (b & 1) .. +7, rows 4 (b >> 1) .. +3).  Pixel k of warp w lies in block
// w PPT + k, lane l at the block's column l & 7 and row l >> 3, so a warp
// can skip, per pixel slot, the blocks a splat's footprint misses.
template <int PPT> struct TileMap {
    static constexpr int NT = kTilePixels / PPT;
    static constexpr int NW = NT / 32;
    static_assert(NW * PPT == 8, "eight blocks per tile");
    int v, W, H, x0, y0;
    int px[PPT], py[PPT];
    float lx[PPT], ly[PPT];  // pixel position within the tile, as floats
    bool inside[PPT];
    __device__ __forceinline__ TileMap(const ViewTable& vt, int tile)
    {
        v = view_of_tile(vt, tile);
        const int lt = tile - vt.tile_off[v];
        x0 = (lt % vt.tiles_x[v]) * kTile;
        y0 = (lt / vt.tiles_x[v]) * kTile;
        W = vt.width[v];
        H = vt.height[v];
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            // block w PPT + k; slots k and k ^ 1 share the block row when PPT >= 2
            const int bcol = PPT >= 2 ? (k & 1) : (w & 1);
            const int brow = PPT >= 2 ? w * (PPT / 2) + (k >> 1) : (w >> 1);
            const int cx = 8 * bcol + (lane & 7), cy = 4 * brow + (lane >> 3);
            px[k] = x0 + cx;
            py[k] = y0 + cy;
            lx[k] = (float)cx;
            ly[k] = (float)cy;
            inside[k] = px[k] < W && py[k] < H;
        }
    }
};

// Bit b set when the bounding box of the ellipse d^T conic d <= k (where
// alpha can reach 1/255), widened by 1% and 0.01 px against float32
// rounding of the alpha test, meets the pixel centres of block b of the
// tile at (x0, y0).  The half-extents are sqrt(k Sigma_xx), sqrt(k Sigma_yy)
// with Sigma_xx = c^2 / ls + s^2 / lb and Sigma_yy = s^2 / ls + c^2 / lb.
__device__ __forceinline__ uint32_t block_mask(const Screen& rec, int x0, int y0)
{
    const float c = rec.q1.x, sn = rec.q1.y;
    const float kk = opacity_k(rec.q1.z);
    const float sxx = c * c / rec.q0.w + sn * sn / rec.q0.z;
    const float syy = sn * sn / rec.q0.w + c * c / rec.q0.z;
    const float ex = sqrtf(kk * sxx) * 1.01f + 0.01f;
    const float ey = sqrtf(kk * syy) * 1.01f + 0.01f;
    const float mx = rec.q0.x, my = rec.q0.y;
    if (!(ex == ex && ey == ey)) return 0xffu;
    uint32_t m = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const float bx0 = (float)(x0 + 8 * (b & 1)) + 0.5f, by0 = (float)(y0 + 4 * (b >> 1)) + 0.5f;
        if (mx + ex >= bx0 && mx - ex <= bx0 + 7.0f && my + ey >= by0 && my - ey <= by0 + 3.0f) m |= 1u << b;
    }
    return m;
}

__device__ __forceinline__ void stage_entry(const Screen& rec, int x0, int y0, Entry& e)
{
    const float sa = sqrtf(0.5f * kLog2e * rec.q0.w), sb = sqrtf(0.5f * kLog2e * rec.q0.z);
    const float c = rec.q1.x, sn = rec.q1.y;
    e.coef = make_float4(c * sa, sn * sa, c * sb, sn * sb);
    const float dx0 = __fsub_rn((float)x0 + 0.5f, rec.q0.x);
    const float dy0 = __fsub_rn((float)y0 + 0.5f, rec.q0.y);
    e.uw0 = make_float2(__fmaf_rn(e.coef.x, dx0, __fmul_rn(e.coef.y, dy0)),
                        __fmaf_rn(e.coef.z, dy0, -__fmul_rn(e.coef.w, dx0)));
    e.rgbo = make_float4(rec.q2.x, rec.q2.y, rec.q2.z, rec.q1.z);
    e.mask = block_mask(rec, x0, y0);
    e.pad = 0;
}

// 2^x for x <= 0 on the special-function unit; results below 2^-126 flush to
// zero, far below any alpha that is blended.
__device__ __forceinline__ float exp2_ftz(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Alpha of one fragment (Eq. 3 with the 3DGS rules) at the pixel (lx, ly)
// of the entry's tile, shared by the forward and both backwards so all take
// the same decisions: skip alpha < 1/255; alpha = min(0.99, o G).  The
// coordinates are evaluated in one fixed order of roundings, the row term
// first, so every launch configuration computes them bit for bit alike.  The
// exponent is a negated sum of squares, so the positive-exponent case cannot
// arise.  Also returns the scaled offsets u' (along the major axis) and w'
// (across it) for the backward.
__device__ __forceinline__ bool eval_frag(float lx, float ly, const Entry& e, Frag& f, float& u, float& w)
{
    u = __fmaf_rn(e.coef.x, lx, __fmaf_rn(e.coef.y, ly, e.uw0.x));
    w = __fmaf_rn(-e.coef.w, lx, __fmaf_rn(e.coef.z, ly, e.uw0.y));
    const float l2 = -__fmaf_rn(u, u, __fmul_rn(w, w));
    f.G = exp2_ftz(l2);
    const float oG = __fmul_rn(e.rgbo.w, f.G);
    f.clamped = oG >= kAlphaMax;
    f.alpha = fminf(oG, kAlphaMax);
    return oG >= kAlphaMin;  // false for a NaN oG, like the test on alpha
}

// Adds one blended fragment to the nine sums m[9] from which the entry's
// screen-space gradients follow (entry_grads below), given dL/dalpha, wT =
// alpha T and the pixel's dL/dC = g.  With q = dL/dalpha G (zero where alpha
// is clamped, since it then does not depend on the Gaussian's geometry or
// opacity) the sums are q u, q w, q u^2, q u w, q w^2, q and wT g: the
// gradients of the mean and of Sigma2D are linear in the first five, with
// coefficients that depend on the entry alone, so the per-fragment work is
// these eight products instead of forming C d and (C d)(C d)^T per fragment.
// u and w are the exp2-scaled axis coordinates of eval_frag; the sums stay
// in the conic's eigen basis, where C d is a positive diagonal scaling, and
// are rotated back once per entry.
__device__ __forceinline__ void frag_moments(const Frag& f, float u, float w, float dalpha, float wT,
                                             float g0, float g1, float g2, float m[9])
{
    m[6] = __fmaf_rn(wT, g0, m[6]);
    m[7] = __fmaf_rn(wT, g1, m[7]);
    m[8] = __fmaf_rn(wT, g2, m[8]);
    const float q = f.clamped ? 0.0f : dalpha * f.G;
    m[5] += q;
    m[0] = __fmaf_rn(q, u, m[0]);
    m[1] = __fmaf_rn(q, w, m[1]);
    const float qu = q * u;
    m[2] = __fmaf_rn(qu, u, m[2]);
    m[3] = __fmaf_rn(qu, w, m[3]);
    m[4] = __fmaf_rn(q, __fmul_rn(w, w), m[4]);
}

// The entry's screen-space gradients from its sums m[9] over the pixels
// (frag_moments): dL/dmu2D, dL/dSigma2D (H00, H01, H11 of the full symmetric
// gradient), dL/do and dL/drgb.  Per fragment the exponent's derivative is
// dpow = dL/dalpha alpha = o q (power = -d^T C d / 2), and with the eigen
// form C d = 2 ln 2 (vx, vy), vx = cx u - cw w, vy = cy u + cz w (coef =
// (cx, cy, cz, cw)):
//   dL/dmu    = sum dpow C d                  = 2 ln 2 o (cx S_u - cw S_w, cy S_u + cz S_w)
//   dL/dSigma = sum dpow (C d)(C d)^T / 2     = 2 (ln 2)^2 o sum q (vx, vy)(vx, vy)^T
// expanded in S_uu, S_uw, S_ww.  The dense C G C product of the conic
// gradient, which cancels for needle-like splats in float32, never forms.
__device__ __forceinline__ void entry_grads(const Entry& e, const float m[9], float4& ga, float4& gb,
                                            float& gblue)
{
    const float o = e.rgbo.w;
    const float cx = e.coef.x, cy = e.coef.y, cz = e.coef.z, cw = e.coef.w;
    const float k1 = kTwoLn2 * o;
    const float k2 = (0.5f * kTwoLn2 * kTwoLn2) * o;
    ga.x = k1 * (cx * m[0] - cw * m[1]);
    ga.y = k1 * (cy * m[0] + cz * m[1]);
    ga.z = k2 * (cx * cx * m[2] - 2.0f * cx * cw * m[3] + cw * cw * m[4]);
    ga.w = k2 * (cx * cy * m[2] + (cx * cz - cw * cy) * m[3] - cw * cz * m[4]);
    gb.x = k2 * (cy * cy * m[2] + 2.0f * cy * cz * m[3] + cz * cz * m[4]);
    gb.y = m[5];
    gb.z = m[6];
    gb.w = m[7];
    gblue = m[8];
}

// Buffers of the per-Gaussian backward (state == nullptr: not in use).
struct PgBuffers {
    const uint32_t* bucket_off;  // [total_tiles + 1]
    uint32_t* bucket_tile;       // [max_buckets]
    float4* state;               // [max_buckets * 256]
    float4* pixel_final;         // [total_pixels]: the pixel's output colour (C + T bg)
    int64_t max_buckets;
};

// Tile scheduling.  With a queue (head != nullptr) the CTAs of a resident
// grid take the next entry of `order` (tiles by descending list length) until
// it is exhausted, and the last CTA out zeroes the counters for the next
// launch; nothing waits on another CTA.  Without one, CTA b takes tile b.
struct TileSched {
    uint32_t* head;   // next queue position
    uint32_t* exits;  // CTAs that found the queue empty
    const uint32_t* order;
};

__device__ __forceinline__ int sched_next(const TileSched& s, int total, int& iter, uint32_t& s_slot)
{
    if (!s.head) return iter++ == 0 ? (int)blockIdx.x : -1;
    __syncthreads();  // every thread is done with the previous tile's shared state
    if (threadIdx.x == 0) {
        const uint32_t i = atomicAdd(s.head, 1u);
        if (i < (uint32_t)total) {
            s_slot = s.order[i];
        } else {
            s_slot = 0xffffffffu;
            // each CTA exits once, after its last use of the head
            if (atomicAdd(s.exits, 1u) == gridDim.x - 1) {
                *s.head = 0;
                *s.exits = 0;
            }
        }
    }
    __syncthreads();
    return s_slot == 0xffffffffu ? -1 : (int)s_slot;
}

// Bucket of a tile's list length for the queue order: a quarter octave per
// bucket, longest first (a longest-processing-time order needs only rough
// sorting); empty tiles last.
constexpr int kOrderBuckets = 130;

__device__ __forceinline__ int length_bucket(uint2 r)
{
    const uint32_t c = r.y - r.x;
    if (c == 0) return kOrderBuckets - 1;
    const int e = 31 - __clz(c);
    const uint32_t m = e >= 2 ? (c >> (e - 2)) & 3u : (c << (2 - e)) & 3u;
    return 128 - (4 * e + (int)m);
}

// One CTA: counting sort of all tiles by length_bucket into q[4..], and
// zeroes the four queue counters q[0..3].
__global__ void __launch_bounds__(1024) tile_order_kernel(const uint2* __restrict__ ranges, int total,
                                                          uint32_t* __restrict__ q)
{
    __shared__ uint32_t s_cnt[kOrderBuckets];
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) s_cnt[b] = 0;
    if (threadIdx.x < 4) q[threadIdx.x] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < total; t += blockDim.x) atomicAdd(&s_cnt[length_bucket(ranges[t])], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int b = 0; b < kOrderBuckets; ++b) {
            const uint32_t c = s_cnt[b];
            s_cnt[b] = acc;
            acc += c;
        }
    }
    __syncthreads();
    uint32_t* order = q + 4;
    for (int t = threadIdx.x; t < total; t += blockDim.x)
        order[atomicAdd(&s_cnt[length_bucket(ranges[t])], 1u)] = (uint32_t)t;
}

// Forward of one tile (the whole CTA): front-to-back blending of its list.
template <int PPT, int BATCH, bool CKPT>
__device__ __forceinline__ void blend_fwd_tile(const ViewTable& vt, int64_t n, const uint2* __restrict__ ranges,
                                               const uint32_t* __restrict__ gids,
                                               const Screen* __restrict__ screen, float bg0, float bg1,
                                               float bg2, float* __restrict__ images,
                                               float* __restrict__ T_final, uint32_t* __restrict__ n_contrib,
                                               uint32_t* __restrict__ n_blended, const PgBuffers& pg, int tile)
{
    using Map = TileMap<PPT>;
    __shared__ Entry s_e[BATCH];
    const Map tm(vt, tile);
    const int warp = threadIdx.x >> 5;
    const uint2 range = ranges[tile];
    const Screen* scr = screen + (int64_t)tm.v * n;
    float T[PPT], C0[PPT], C1[PPT], C2[PPT];
    uint32_t last[PPT], blended[PPT];
    bool done[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        T[k] = 1.0f;
        C0[k] = C1[k] = C2[k] = 0.f;
        last[k] = 0;
        blended[k] = 0;
        done[k] = !tm.inside[k];
    }
    const int64_t bucket0 = CKPT ? (int64_t)pg.bucket_off[tile] : 0;
    float4* ckpt = CKPT ? pg.state + bucket0 * kTilePixels : nullptr;
    for (uint32_t start = range.x; start < range.y; start += BATCH) {
        bool all_done = true;
#pragma unroll
        for (int k = 0; k < PPT; ++k) all_done &= done[k];
        if (__syncthreads_count(all_done) == Map::NT) break;
        for (int e = threadIdx.x; e < BATCH; e += Map::NT) {
            const uint32_t j = start + e;
            if (j < range.y) {
                const Screen rec = scr[gids[j]];
                stage_entry(rec, tm.x0, tm.y0, s_e[e]);
            }
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)BATCH, range.y - start);
        for (int jj = 0; jj < cnt && !all_done; ++jj) {
            if (CKPT && (jj & 31) == 0 && bucket0 + ((start - range.x + jj) >> 5) < pg.max_buckets) {
                // (T, C) in front of a bucket's first entry (BATCH is a multiple of 32)
                float4* st = ckpt + (int64_t)((start - range.x + jj) >> 5) * kTilePixels;
#pragma unroll
                for (int k = 0; k < PPT; ++k)
                    if (!done[k])
                        st[(tm.py[k] - tm.y0) * kTile + (tm.px[k] - tm.x0)] = make_float4(T[k], C0[k], C1[k], C2[k]);
            }
            Entry e;
            const uint32_t wm = (load_head(s_e[jj], e.uw0) >> (warp * PPT)) & ((1u << PPT) - 1u);
            if (!wm) continue;  // uniform over the warp
            e.coef = s_e[jj].coef;
            e.rgbo = s_e[jj].rgbo;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                // a stopped pixel evaluates along with the warp's others but
                // takes no decision (no branch of its own)
                Frag f;
                float u, w;
                if (((wm >> k) & 1u) && eval_frag(tm.lx[k], tm.ly[k], e, f, u, w) && !done[k]) {
                    // T (1 - alpha) in one rounding
                    const float test = __fmaf_rn(-f.alpha, T[k], T[k]);
                    if (test < kTMin) {
                        done[k] = true;
                        continue;
                    }
                    // explicit roundings: the per-Gaussian backward replays these exactly
                    const float wt = __fmul_rn(f.alpha, T[k]);
                    C0[k] = __fmaf_rn(wt, e.rgbo.x, C0[k]);
                    C1[k] = __fmaf_rn(wt, e.rgbo.y, C1[k]);
                    C2[k] = __fmaf_rn(wt, e.rgbo.z, C2[k]);
                    T[k] = test;
                    last[k] = start + jj - range.x + 1;
                    ++blended[k];
                }
            }
            all_done = true;
#pragma unroll
            for (int k = 0; k < PPT; ++k) all_done &= done[k];
        }
    }
    const int64_t P = (int64_t)tm.W * tm.H;
    float* img = images + 3 * vt.pix_off[tm.v];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (!tm.inside[k]) continue;
        const int64_t pix = (int64_t)tm.py[k] * tm.W + tm.px[k];
        const float o0 = __fmaf_rn(T[k], bg0, C0[k]), o1 = __fmaf_rn(T[k], bg1, C1[k]),
                    o2 = __fmaf_rn(T[k], bg2, C2[k]);
        img[pix] = o0;
        img[P + pix] = o1;
        img[2 * P + pix] = o2;
        if (CKPT) pg.pixel_final[vt.pix_off[tm.v] + pix] = make_float4(o0, o1, o2, 0.0f);
        T_final[vt.pix_off[tm.v] + pix] = T[k];
        n_contrib[vt.pix_off[tm.v] + pix] = last[k];
        n_blended[vt.pix_off[tm.v] + pix] = blended[k];
    }
}

template <int PPT, int BATCH, bool CKPT>
__global__ void __launch_bounds__(kTilePixels / PPT)
blend_fwd_kernel(ViewTable vt, int64_t n, const uint2* __restrict__ ranges,
                 const uint32_t* __restrict__ gids, const Screen* __restrict__ screen, float bg0,
                 float bg1, float bg2, float* __restrict__ images, float* __restrict__ T_final,
                 uint32_t* __restrict__ n_contrib, uint32_t* __restrict__ n_blended, TileSched sched,
                 PgBuffers pg)
{
    __shared__ uint32_t s_slot;
    int iter = 0;
    for (int tile; (tile = sched_next(sched, vt.total_tiles, iter, s_slot)) >= 0;)
        blend_fwd_tile<PPT, BATCH, CKPT>(vt, n, ranges, gids, screen, bg0, bg1, bg2, images, T_final,
                                         n_contrib, n_blended, pg, tile);
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

// Backward of one tile (the whole CTA): back-to-front over its list.
template <int PPT, int BATCH>
__device__ __forceinline__ void blend_bwd_tile(const ViewTable& vt, int64_t n, const uint2* __restrict__ ranges,
                                               const uint32_t* __restrict__ gids,
                                               const Screen* __restrict__ screen, float bg0, float bg1,
                                               float bg2, const float* __restrict__ dL_dimg,
                                               const float* __restrict__ T_final,
                                               const uint32_t* __restrict__ n_contrib,
                                               ScreenGrad* __restrict__ sgrad, int tile)
{
    using Map = TileMap<PPT>;
    __shared__ Entry s_e[BATCH];
    __shared__ uint32_t s_gid[BATCH];
    // one row per value; the row padding puts the 9 values of one entry in
    // 9 different banks for the scattered shared atomics below
    __shared__ float s_acc[9][BATCH + 1];
    __shared__ uint32_t s_max;
    const Map tm(vt, tile);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint2 range = ranges[tile];
    const Screen* scr = screen + (int64_t)tm.v * n;
    ScreenGrad* sg = sgrad + (int64_t)tm.v * n;
    const int64_t P = (int64_t)tm.W * tm.H;
    const float* dl = dL_dimg + 3 * vt.pix_off[tm.v];

    // S = g . A: the colour behind the entry (A, normalised by T after the
    // entry; bg behind the last) enters the gradients only through its dot
    // product with the pixel's dL/dC = g, so one scalar replaces A
    float T[PPT], g0[PPT], g1[PPT], g2[PPT], S[PPT];
    uint32_t last[PPT];
    uint32_t my_max = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        T[k] = 1.0f;
        g0[k] = g1[k] = g2[k] = 0.f;
        S[k] = 0.f;
        last[k] = 0;
        if (tm.inside[k]) {
            const int64_t pix = (int64_t)tm.py[k] * tm.W + tm.px[k];
            g0[k] = dl[pix];
            g1[k] = dl[P + pix];
            g2[k] = dl[2 * P + pix];
            S[k] = g0[k] * bg0 + g1[k] * bg1 + g2[k] * bg2;
            T[k] = T_final[vt.pix_off[tm.v] + pix];
            last[k] = n_contrib[vt.pix_off[tm.v] + pix];
            my_max = max(my_max, last[k]);
        }
    }
    const uint32_t warp_max = __reduce_max_sync(0xffffffffu, my_max);
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    if (lane == 0 && warp_max) atomicMax(&s_max, warp_max);
    __syncthreads();
    const uint32_t end = range.x + s_max;

    for (uint32_t bend = end; bend > range.x;) {
        const uint32_t bstart = bend > range.x + BATCH ? bend - BATCH : range.x;
        const int cnt = (int)(bend - bstart);
        __syncthreads();
        for (int e = threadIdx.x; e < BATCH; e += Map::NT) {
            if (e < cnt) {
                const uint32_t j = bend - 1 - e;  // slot 0 is the back-most entry
                const uint32_t g = gids[j];
                const Screen rec = scr[g];
                s_gid[e] = g;
                stage_entry(rec, tm.x0, tm.y0, s_e[e]);
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) s_acc[k][e] = 0.f;
        }
        __syncthreads();
        for (int jj = 0; jj < cnt; ++jj) {
            const uint32_t pos = bend - jj - range.x;  // 1-based list position
            Entry e;
            const uint32_t wm = (load_head(s_e[jj], e.uw0) >> (warp * PPT)) & ((1u << PPT) - 1u);
            if (pos > warp_max || !wm) continue;  // uniform over the warp
            e.coef = s_e[jj].coef;
            e.rgbo = s_e[jj].rgbo;
            float d[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) d[k] = 0.f;
            bool any = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                Frag f;
                float u, w;
                if (!(((wm >> k) & 1u) && pos <= last[k] &&
                      eval_frag(tm.lx[k], tm.ly[k], e, f, u, w)))
                    continue;
                any = true;
                // transmittance in front of the entry; 1 - alpha >= 0.01, so the
                // approximate divide (2 ulp) is in range
                const float Ti = __fdividef(T[k], 1.0f - f.alpha);
                // g . (c - A) = g . c - S as three FMAs from -S, shared by
                // dL/dalpha and the update of the colour behind, A <- A + alpha (c - A)
                const float gc = fmaf(g0[k], e.rgbo.x, fmaf(g1[k], e.rgbo.y, fmaf(g2[k], e.rgbo.z, -S[k])));
                const float dalpha = Ti * gc;
                frag_moments(f, u, w, dalpha, f.alpha * Ti, g0[k], g1[k], g2[k], d);
                S[k] += f.alpha * gc;
                T[k] = Ti;
            }
            if (!__any_sync(0xffffffffu, any)) continue;
            // value index of lane l after the scatter: (l >> 2) & 7
            const float part = warp_sum8_scatter(d, lane);
            const float last_v = warp_sum(d[8]);
            if ((lane & 3) == 0) atomicAdd(&s_acc[(lane >> 2) & 7][jj], part);
            if (lane == 1) atomicAdd(&s_acc[8][jj], last_v);
        }
        __syncthreads();
        for (int s = threadIdx.x; s < cnt; s += Map::NT) {
            float m[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) m[k] = s_acc[k][s];
            if (m[0] != 0.f || m[1] != 0.f || m[2] != 0.f || m[3] != 0.f || m[4] != 0.f || m[5] != 0.f ||
                m[6] != 0.f || m[7] != 0.f || m[8] != 0.f) {
                float4 ga, gb;
                float gblue;
                entry_grads(s_e[s], m, ga, gb, gblue);
                ScreenGrad* dst = sg + s_gid[s];
                atomicAdd(&dst->g0, ga);
                atomicAdd(&dst->g1, gb);
                atomicAdd(&dst->g2.x, gblue);
            }
        }
        bend = bstart;
    }
}

template <int PPT, int BATCH>
__global__ void __launch_bounds__(kTilePixels / PPT)
blend_bwd_kernel(ViewTable vt, int64_t n, const uint2* __restrict__ ranges,
                 const uint32_t* __restrict__ gids, const Screen* __restrict__ screen, float bg0,
                 float bg1, float bg2, const float* __restrict__ dL_dimg,
                 const float* __restrict__ T_final, const uint32_t* __restrict__ n_contrib,
                 ScreenGrad* __restrict__ sgrad, TileSched sched)
{
    __shared__ uint32_t s_slot;
    int iter = 0;
    for (int tile; (tile = sched_next(sched, vt.total_tiles, iter, s_slot)) >= 0;)
        blend_bwd_tile<PPT, BATCH>(vt, n, ranges, gids, screen, bg0, bg1, bg2, dL_dimg, T_final, n_contrib,
                                   sgrad, tile);
}

// ---------------------------------------------------------------------------
// Per-Gaussian backward
// ---------------------------------------------------------------------------
constexpr int kBucket = 32;             // entries per bucket (one per lane)
constexpr int kPgWarps = 8;             // buckets in flight per CTA
constexpr int kScanThreads = 1024;

// One CTA: bucket_off[t] = sum over tiles u < t of ceil(len_u / 32),
// bucket_off[total] = the number of buckets, and bucket_tile[b] = the tile
// of bucket b.  Buckets beyond max_buckets (more instances than the
// workspace was sized for, which the capacity flag already reports) are
// dropped by clamping the offsets.
__global__ void __launch_bounds__(kScanThreads)
bucket_scan_kernel(const uint2* __restrict__ ranges, int total, uint32_t* __restrict__ bucket_off,
                   uint32_t* __restrict__ bucket_tile, uint32_t max_buckets)
{
    __shared__ uint32_t s_sum[kScanThreads];
    const int per = (total + kScanThreads - 1) / kScanThreads;
    const int t0 = threadIdx.x * per, t1 = min(total, t0 + per);
    uint32_t mine = 0;
    for (int t = t0; t < t1; ++t) {
        const uint2 r = ranges[t];
        mine += (r.y - r.x + kBucket - 1) / kBucket;
    }
    s_sum[threadIdx.x] = mine;
    __syncthreads();
    // inclusive Hillis-Steele scan of the per-thread totals
    for (int o = 1; o < kScanThreads; o <<= 1) {
        const uint32_t add = threadIdx.x >= o ? s_sum[threadIdx.x - o] : 0u;
        __syncthreads();
        s_sum[threadIdx.x] += add;
        __syncthreads();
    }
    uint32_t acc = s_sum[threadIdx.x] - mine;
    for (int t = t0; t < t1; ++t) {
        const uint2 r = ranges[t];
        const uint32_t nb = (r.y - r.x + kBucket - 1) / kBucket;
        bucket_off[t] = min(acc, max_buckets);
        for (uint32_t b = acc; b < acc + nb && b < max_buckets; ++b) bucket_tile[b] = (uint32_t)t;
        acc += nb;
    }
    if (threadIdx.x == kScanThreads - 1) bucket_off[total] = min(s_sum[kScanThreads - 1], max_buckets);
}

// Per-warp staging of 32 active pixels: state in front of the bucket, dL/dC,
// the output colour, last-contributor position and tile-local index.
struct PgStage {
    float T[kBucket], C0[kBucket], C1[kBucket], C2[kBucket];
    float g0[kBucket], g1[kBucket], g2[kBucket];
    float o0[kBucket], o1[kBucket], o2[kBucket];
    uint32_t last[kBucket];
    uint32_t p[kBucket];
};

__global__ void __launch_bounds__(kPgWarps * 32, 4)
blend_bwd_pg_kernel(ViewTable vt, int64_t n, const uint2* __restrict__ ranges,
                    const uint32_t* __restrict__ gids, const Screen* __restrict__ screen,
                    const float* __restrict__ dL_dimg, const uint32_t* __restrict__ n_contrib,
                    PgBuffers pg, ScreenGrad* __restrict__ sgrad)
{
    __shared__ PgStage s_stage[kPgWarps][2];
    __shared__ uint8_t s_list[kPgWarps][kTilePixels];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t full = 0xffffffffu;
    const uint32_t nb = pg.bucket_off[vt.total_tiles];
    for (uint32_t b = blockIdx.x * kPgWarps + warp; b < nb; b += gridDim.x * kPgWarps) {
        const int tile = (int)pg.bucket_tile[b];
        const uint32_t first = (b - pg.bucket_off[tile]) * kBucket;  // list position of lane 0
        const int v = view_of_tile(vt, tile);
        const int lt = tile - vt.tile_off[v];
        const int x0 = (lt % vt.tiles_x[v]) * kTile, y0 = (lt / vt.tiles_x[v]) * kTile;
        const int W = vt.width[v], H = vt.height[v];
        const int64_t P = (int64_t)W * H, poff = vt.pix_off[v];
        const uint2 range = ranges[tile];
        const uint32_t j = range.x + first + lane;
        const bool has = j < range.y;
        const uint32_t pos = first + lane + 1;  // 1-based list position of this lane's entry
        Entry e;
        uint32_t gid = 0, bmask = 0;
        if (has) {
            gid = gids[j];
            const Screen rec = screen[(int64_t)v * n + gid];
            stage_entry(rec, x0, y0, e);
            bmask = e.mask;
        } else {
            e.uw0 = make_float2(0.f, 0.f);
            e.coef = make_float4(0.f, 0.f, 0.f, 0.f);
            e.rgbo = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        // the tile's pixels still blending in front of this bucket
        int na = 0;
        for (int c = 0; c < kTilePixels / 32; ++c) {
            const int p = 32 * c + lane;
            const int px = x0 + (p & (kTile - 1)), py = y0 + (p >> 4);
            const bool act = px < W && py < H && n_contrib[poff + (int64_t)py * W + px] > first;
            const uint32_t bal = __ballot_sync(full, act);
            if (act) s_list[warp][na + __popc(bal & ((1u << lane) - 1u))] = (uint8_t)p;
            na += __popc(bal);
        }
        __syncwarp();
        const float4* st = pg.state + (int64_t)b * kTilePixels;
        float d[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) d[k] = 0.f;
        float To = 0.f, Co0 = 0.f, Co1 = 0.f, Co2 = 0.f;  // state this lane hands on
        for (int s = 0; s < na + kBucket - 1; ++s) {
            if ((s & (kBucket - 1)) == 0 && s < na) {
                // stage pixels s .. s + 31 (the buffer last read at step s - 2)
                PgStage& sg = s_stage[warp][(s >> 5) & 1];
                const int i = s + lane;
                if (i < na) {
                    const int p = s_list[warp][i];
                    const int64_t pix = (int64_t)(y0 + (p >> 4)) * W + x0 + (p & (kTile - 1));
                    const float4 t4 = st[p];
                    const float4 o4 = pg.pixel_final[poff + pix];
                    sg.T[lane] = t4.x;
                    sg.C0[lane] = t4.y;
                    sg.C1[lane] = t4.z;
                    sg.C2[lane] = t4.w;
                    sg.g0[lane] = dL_dimg[3 * poff + pix];
                    sg.g1[lane] = dL_dimg[3 * poff + P + pix];
                    sg.g2[lane] = dL_dimg[3 * poff + 2 * P + pix];
                    sg.o0[lane] = o4.x;
                    sg.o1[lane] = o4.y;
                    sg.o2[lane] = o4.z;
                    sg.last[lane] = n_contrib[poff + pix];
                    sg.p[lane] = (uint32_t)p;
                }
                __syncwarp();
            }
            // the state lane - 1 produced for the pixel this lane takes now
            float T = __shfl_up_sync(full, To, 1);
            float C0 = __shfl_up_sync(full, Co0, 1);
            float C1 = __shfl_up_sync(full, Co1, 1);
            float C2 = __shfl_up_sync(full, Co2, 1);
            const int i = s - lane;
            if (i < 0 || i >= na) continue;
            const PgStage& sg = s_stage[warp][(i >> 5) & 1];
            const int k = i & (kBucket - 1);
            if (lane == 0) {
                T = sg.T[k];
                C0 = sg.C0[k];
                C1 = sg.C1[k];
                C2 = sg.C2[k];
            }
            const int p = (int)sg.p[k];
            const int lx = p & (kTile - 1), ly = p >> 4;
            Frag f;
            float u, w;
            if (has && pos <= sg.last[k] && ((bmask >> ((lx >> 3) | ((ly >> 2) << 1))) & 1u) &&
                eval_frag((float)lx, (float)ly, e, f, u, w)) {
                // the forward's update, rounding for rounding
                const float Tn = __fmaf_rn(-f.alpha, T, T);
                const float wT = __fmul_rn(f.alpha, T);
                C0 = __fmaf_rn(wT, e.rgbo.x, C0);
                C1 = __fmaf_rn(wT, e.rgbo.y, C1);
                C2 = __fmaf_rn(wT, e.rgbo.z, C2);
                // colour behind the entry, normalised by T after it (Tn >= 1e-4)
                const float iT = __fdividef(1.0f, Tn);
                const float g0 = sg.g0[k], g1 = sg.g1[k], g2 = sg.g2[k];
                const float c0 = e.rgbo.x - (sg.o0[k] - C0) * iT;
                const float c1 = e.rgbo.y - (sg.o1[k] - C1) * iT;
                const float c2 = e.rgbo.z - (sg.o2[k] - C2) * iT;
                const float dalpha = T * (g0 * c0 + g1 * c1 + g2 * c2);
                frag_moments(f, u, w, dalpha, wT, g0, g1, g2, d);
                T = Tn;
            }
            To = T;
            Co0 = C0;
            Co1 = C1;
            Co2 = C2;
        }
        if (has && (d[0] != 0.f || d[1] != 0.f || d[2] != 0.f || d[3] != 0.f || d[4] != 0.f || d[5] != 0.f ||
                    d[6] != 0.f || d[7] != 0.f || d[8] != 0.f)) {
            float4 ga, gb;
            float gblue;
            entry_grads(e, d, ga, gb, gblue);
            ScreenGrad* dst = sgrad + (int64_t)v * n + gid;
            atomicAdd(&dst->g0, ga);
            atomicAdd(&dst->g1, gb);
            atomicAdd(&dst->g2.x, gblue);
        }
        __syncwarp();  // s_list and the stages are reused by the next bucket
    }
}

// Launch configurations the tuner may pick: pixels per thread x batch, and
// the schedule.  A queue launch is one resident grid: SMs x CTAs per SM.
static int sm_count()
{
    static int cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cache[dev]) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = sms > 0 ? sms : 1;
    }
    return cache[dev];
}

template <typename K>
static int grid_for(K kernel, int threads, int total_tiles, const TileSched& sched)
{
    if (!sched.head) return total_tiles;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const long long g = (long long)per_sm * sm_count();
    return (int)(g < total_tiles ? g : total_tiles);
}

template <int PPT, int BATCH, bool CKPT>
static void launch_pair_fwd(const ViewTable& vt, int64_t n, const uint2* ranges, const uint32_t* gids,
                            const Screen* screen, const float bg[3], float* images, float* T_final,
                            uint32_t* n_contrib, uint32_t* n_blended, const TileSched& sched,
                            const PgBuffers& pg, cudaStream_t st)
{
    const int threads = kTilePixels / PPT;
    const int grid = grid_for(blend_fwd_kernel<PPT, BATCH, CKPT>, threads, vt.total_tiles, sched);
    blend_fwd_kernel<PPT, BATCH, CKPT><<<grid, threads, 0, st>>>(vt, n, ranges, gids, screen, bg[0], bg[1],
                                                                 bg[2], images, T_final, n_contrib,
                                                                 n_blended, sched, pg);
}

template <int PPT, int BATCH>
static void launch_pair_bwd(const ViewTable& vt, int64_t n, const uint2* ranges, const uint32_t* gids,
                            const Screen* screen, const float bg[3], const float* dL_dimg,
                            const float* T_final, const uint32_t* n_contrib, ScreenGrad* sgrad,
                            const TileSched& sched, cudaStream_t st)
{
    const int threads = kTilePixels / PPT;
    const int grid = grid_for(blend_bwd_kernel<PPT, BATCH>, threads, vt.total_tiles, sched);
    blend_bwd_kernel<PPT, BATCH><<<grid, threads, 0, st>>>(vt, n, ranges, gids, screen, bg[0], bg[1], bg[2],
                                                           dL_dimg, T_final, n_contrib, sgrad, sched);
}

#define FGS_BLEND_CONFIGS(X) X(1, 256) X(2, 128) X(2, 256) X(4, 64) X(4, 128) X(4, 256)

bool blend_config_supported(int ppt, int batch)
{
#define FGS_CHECK(P, Bt) if (ppt == P && batch == Bt) return true;
    FGS_BLEND_CONFIGS(FGS_CHECK)
#undef FGS_CHECK
    return false;
}

cudaError_t launch_tile_order(const uint2* ranges, int total_tiles, uint32_t* queue, cudaStream_t st)
{
    if (total_tiles <= 0) return cudaSuccess;
    tile_order_kernel<<<1, 1024, 0, st>>>(ranges, total_tiles, queue);
    profile_mark(st, "tile_order");
    return cudaGetLastError();
}

static TileSched make_sched(uint32_t* queue, int schedule, bool backward)
{
    TileSched s{nullptr, nullptr, nullptr};
    if (schedule == FGS_SCHEDULE_QUEUE && queue) {
        s.head = queue + (backward ? 2 : 0);
        s.exits = queue + (backward ? 3 : 1);
        s.order = queue + 4;
    }
    return s;
}

// pg_* non-null: also store the per-Gaussian backward's bucket states (after
// computing the bucket offsets).
cudaError_t launch_blend_fwd(const ViewTable& vt, int64_t n, const uint2* ranges, const uint32_t* gids,
                             const Screen* screen, const float bg[3], float* images, float* T_final,
                             uint32_t* n_contrib, uint32_t* n_blended, uint32_t* queue, int ppt, int batch,
                             int schedule, uint32_t* pg_bucket_off, uint32_t* pg_bucket_tile,
                             float4* pg_state, float4* pg_pixel_final, int64_t pg_max_buckets,
                             cudaStream_t st)
{
    if (vt.total_tiles <= 0) return cudaSuccess;
    const TileSched sched = make_sched(queue, schedule, false);
    const PgBuffers pg{pg_bucket_off, pg_bucket_tile, pg_state, pg_pixel_final, pg_max_buckets};
    if (pg_state) {
        bucket_scan_kernel<<<1, kScanThreads, 0, st>>>(ranges, vt.total_tiles, pg_bucket_off, pg_bucket_tile,
                                                       (uint32_t)pg_max_buckets);
        profile_mark(st, "bucket_scan");
#define FGS_GO(P, Bt) \
        if (ppt == P && batch == Bt) launch_pair_fwd<P, Bt, true>(vt, n, ranges, gids, screen, bg, images, T_final, n_contrib, n_blended, sched, pg, st);
        FGS_BLEND_CONFIGS(FGS_GO)
#undef FGS_GO
    } else {
#define FGS_GO(P, Bt) \
        if (ppt == P && batch == Bt) launch_pair_fwd<P, Bt, false>(vt, n, ranges, gids, screen, bg, images, T_final, n_contrib, n_blended, sched, pg, st);
        FGS_BLEND_CONFIGS(FGS_GO)
#undef FGS_GO
    }
    profile_mark(st, "blend_fwd");
    return cudaGetLastError();
}

cudaError_t launch_blend_bwd_pg(const ViewTable& vt, int64_t n, const uint2* ranges, const uint32_t* gids,
                                const Screen* screen, const float* dL_dimg, const uint32_t* n_contrib,
                                uint32_t* pg_bucket_off, uint32_t* pg_bucket_tile, float4* pg_state,
                                float4* pg_pixel_final, int64_t pg_max_buckets, ScreenGrad* sgrad,
                                cudaStream_t st)
{
    if (vt.total_tiles <= 0) return cudaSuccess;
    const PgBuffers pg{pg_bucket_off, pg_bucket_tile, pg_state, pg_pixel_final, pg_max_buckets};
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, blend_bwd_pg_kernel, kPgWarps * 32, 0) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int64_t need = (pg_max_buckets + kPgWarps - 1) / kPgWarps;
    const int64_t cap = (int64_t)per_sm * sm_count();
    const int grid = (int)(need < cap ? (need > 0 ? need : 1) : cap);
    blend_bwd_pg_kernel<<<grid, kPgWarps * 32, 0, st>>>(vt, n, ranges, gids, screen, dL_dimg, n_contrib, pg,
                                                        sgrad);
    profile_mark(st, "blend_bwd_pg");
    return cudaGetLastError();
}

cudaError_t launch_blend_bwd(const ViewTable& vt, int64_t n, const uint2* ranges, const uint32_t* gids,
                             const Screen* screen, const float bg[3], const float* dL_dimg,
                             const float* T_final, const uint32_t* n_contrib, ScreenGrad* sgrad,
                             uint32_t* queue, int ppt, int batch, int schedule, cudaStream_t st)
{
    if (vt.total_tiles <= 0) return cudaSuccess;
    const TileSched sched = make_sched(queue, schedule, true);
#define FGS_GO(P, Bt) \
    if (ppt == P && batch == Bt) launch_pair_bwd<P, Bt>(vt, n, ranges, gids, screen, bg, dL_dimg, T_final, n_contrib, sgrad, sched, st);
    FGS_BLEND_CONFIGS(FGS_GO)
#undef FGS_GO
    profile_mark(st, "blend_bwd");
    return cudaGetLastError();
}

}  // namespace fgs
