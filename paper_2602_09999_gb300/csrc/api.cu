// api.cu -- the C ABI of libfastergs.so (declared in include/fastergs.h):
// argument checks, workspace layout and the launch sequence of each call.
// Nothing here allocates device memory or synchronises, except
// fgs_get_error.
#include <math.h>
#include <string.h>

#include "fgs_common.cuh"

namespace fgs {
cudaError_t launch_preprocess_fwd(int64_t n, int deg, const fgs_params* p, const fgs_camera* cams,
                                  const ViewTable& vt, Screen* screen, TileRect* rects,
                                  uint32_t* local_off, uint32_t* block_sum, cudaStream_t st);
cudaError_t launch_compact_visible(int64_t n, const ViewTable& vt, const Screen* screen,
                                   const TileRect* rects, const uint32_t* local_off, uint32_t* block_sum,
                                   WsHeader* hdr, uint32_t* dkeys, uint32_t* dvals, cudaStream_t st);
cudaError_t launch_sorted_duplicate(int64_t n, const ViewTable& vt, const Screen* screen,
                                    const TileRect* rects, const uint32_t* svals, uint32_t* sorted_off,
                                    uint32_t* sorted_block, WsHeader* hdr, int64_t k_max, uint32_t* keys,
                                    uint32_t* vals, uint32_t* big, int order, cudaStream_t st);
int64_t count_scan_blocks(int64_t pairs);
cudaError_t launch_preprocess_bwd(int64_t n, int deg, const fgs_params* p, const fgs_camera* cams,
                                  const ViewTable& vt, const Screen* screen, const TileRect* rects,
                                  const ScreenGrad* sgrad, const fgs_params* g, cudaStream_t st);
size_t sort_hist_bytes(int64_t n_max, int rb);
int radix_passes(int bits, int rb);
int radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, int64_t n_max,
                   const uint32_t* n_dev, int bits, uint32_t* hist, bool depth, int rb, cudaStream_t st,
                   cudaError_t* err);
int radix_sort(unsigned long long* keys, uint32_t* vals, unsigned long long* keys_alt,
               uint32_t* vals_alt, int64_t n_max, const uint32_t* n_dev, int bits, uint32_t* hist,
               cudaStream_t st, cudaError_t* err);
cudaError_t launch_set_count(uint32_t* dst, uint32_t value, cudaStream_t st);
cudaError_t launch_tile_ranges(const uint32_t* keys, const uint32_t* n_dev, int64_t n_max,
                               uint2* ranges, int total_tiles, cudaStream_t st);
cudaError_t launch_tile_order(const uint2* ranges, int total_tiles, uint32_t* queue, cudaStream_t st);
cudaError_t launch_blend_fwd(const ViewTable& vt, int64_t n, const uint2* ranges, const uint32_t* gids,
                             const Screen* screen, const float bg[3], float* images, float* T_final,
                             uint32_t* n_contrib, uint32_t* n_blended, uint32_t* queue, int ppt, int batch,
                             int schedule, uint32_t* pg_bucket_off, uint32_t* pg_bucket_tile,
                             float4* pg_state, float4* pg_pixel_final, int64_t pg_max_buckets,
                             cudaStream_t st);
cudaError_t launch_blend_bwd_pg(const ViewTable& vt, int64_t n, const uint2* ranges, const uint32_t* gids,
                                const Screen* screen, const float* dL_dimg, const uint32_t* n_contrib,
                                uint32_t* pg_bucket_off, uint32_t* pg_bucket_tile, float4* pg_state,
                                float4* pg_pixel_final, int64_t pg_max_buckets, ScreenGrad* sgrad,
                                cudaStream_t st);
cudaError_t launch_blend_bwd(const ViewTable& vt, int64_t n, const uint2* ranges, const uint32_t* gids,
                             const Screen* screen, const float bg[3], const float* dL_dimg,
                             const float* T_final, const uint32_t* n_contrib, ScreenGrad* sgrad,
                             uint32_t* queue, int ppt, int batch, int schedule, cudaStream_t st);
bool blend_config_supported(int ppt, int batch);

static const int kDefaultPPT = 2, kDefaultBatch = 128;
cudaError_t launch_loss(const ViewTable& vt, const float* images, const float* targets, float lambda,
                        float* maps, double* partials, float* loss_out, float* dL, WsHeader* hdr,
                        cudaStream_t st);
cudaError_t launch_adam_group(int64_t count, int pdt, int mdt, void* p, const float* g, void* m,
                              void* v, float step_size, float inv_bc2_sqrt, double b1, double b2,
                              double eps, const fgs_adam_state* ds, int grp, cudaStream_t st);
cudaError_t launch_adam_prepare(fgs_adam_state* ds, cudaStream_t st);
cudaError_t launch_zero_and_adam_prepare(ScreenGrad* sgrad, const uint32_t* block_sum, const uint32_t* total,
                                         int64_t n, int nv, fgs_adam_state* ds, cudaStream_t st);
cudaError_t launch_preprocess_bwd_adam(int64_t n, int deg, const fgs_params* p, const fgs_camera* cams,
                                       const ViewTable& vt, const Screen* screen, const TileRect* rects,
                                       const ScreenGrad* sgrad,
                                       const fgs_params* g, const fgs_params* m, const fgs_params* v,
                                       const fgs_adam_state* ds, WsHeader* hdr, cudaStream_t st);
bool fused_adam_supported(int sh_dtype, int moment_dtype);

static const int64_t kGroupWidth[FGS_NUM_GROUPS] = {3, 3, 4, 1, 3, 45, 3, 1};
static const int kStaticGroups = 6;  // groups 6 and 7 (velocity, t0) are optional

// Groups present: all 8 for dynamic Gaussians (velocity and t0 set), else 6.
static int groups_of(const fgs_params* p)
{
    return p->data[6] ? FGS_NUM_GROUPS : kStaticGroups;
}

static int check_adam_args(const fgs_params* params, const fgs_params* grads, const fgs_params* m,
                           const fgs_params* v)
{
    if (!params || !grads || !m || !v) return FGS_ERR_NULL;
    const int64_t n = params->n;
    if (n < 1 || grads->n != n || m->n != n || v->n != n) return FGS_ERR_SHAPE;
    if ((params->data[6] == nullptr) != (params->data[7] == nullptr)) return FGS_ERR_NULL;
    const int ng = groups_of(params);
    for (int g = 0; g < ng; ++g) {
        if (!params->data[g] || !grads->data[g] || !m->data[g] || !v->data[g]) return FGS_ERR_NULL;
        if (grads->dtype[g] != FGS_F32) return FGS_ERR_DTYPE;
        if (m->dtype[g] != v->dtype[g]) return FGS_ERR_DTYPE;
        for (const fgs_params* q : {params, m})
            if (q->dtype[g] != FGS_F32 && q->dtype[g] != FGS_BF16 && q->dtype[g] != FGS_F16)
                return FGS_ERR_DTYPE;
        if (g >= kStaticGroups && params->dtype[g] != FGS_F32) return FGS_ERR_DTYPE;
    }
    return FGS_OK;
}

// ---- optional per-kernel profiling events (host state, one per process)
static cudaEvent_t* g_prof_events = nullptr;
static const char** g_prof_labels = nullptr;
static int32_t g_prof_cap = 0;
static int32_t g_prof_count = 0;

void profile_mark(cudaStream_t st, const char* label)
{
    if (!g_prof_events || g_prof_count >= g_prof_cap) return;
    cudaEventRecord(g_prof_events[g_prof_count], st);
    g_prof_labels[g_prof_count] = label;
    ++g_prof_count;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int build_views(const fgs_camera* cams, int32_t nv, ViewTable* vt)
{
    if (!cams) return FGS_ERR_NULL;
    if (nv < 1 || nv > FGS_MAX_VIEWS) return FGS_ERR_VIEWS;
    memset(vt, 0, sizeof(*vt));
    vt->n_views = nv;
    int64_t tiles = 0, pix = 0;
    for (int v = 0; v < nv; ++v) {
        const int W = cams[v].width, H = cams[v].height;
        if (W < 1 || H < 1 || W > 65535 || H > 65535) return FGS_ERR_SHAPE;
        vt->width[v] = W;
        vt->height[v] = H;
        vt->tiles_x[v] = (W + kTile - 1) / kTile;
        vt->tile_off[v] = (int32_t)tiles;
        vt->pix_off[v] = pix;
        tiles += (int64_t)vt->tiles_x[v] * ((H + kTile - 1) / kTile);
        pix += (int64_t)W * H;
    }
    if (tiles >= (1ll << 31)) return FGS_ERR_SHAPE;
    vt->tile_off[nv] = (int32_t)tiles;
    vt->pix_off[nv] = pix;
    vt->total_tiles = (int32_t)tiles;
    vt->total_pixels = pix;
    return FGS_OK;
}

// Key bits of the tile sort: enough for every global tile id.
static int sort_bits_for(int64_t total_tiles)
{
    int b = 1;
    while ((1ll << b) < total_tiles) ++b;
    return b;
}

// The depth sort orders all 32 bits of the (positive) float depths.
static const int kDepthBits = 32;

// Radix digit widths of the render path's sorts (a launch choice): 8 or 11
// bits, 0 meaning 8.
static const int kMaxDigitBits = 11;
static int digit_bits(int32_t choice) { return choice ? choice : 8; }
static bool digit_bits_ok(int32_t choice) { return choice == 0 || choice == 8 || choice == 11; }

// Buckets of 32 list entries the per-Gaussian backward can meet: every
// instance in one, plus a partial bucket per tile.
static int64_t max_buckets_for(int64_t k_max, int64_t total_tiles)
{
    return (k_max + 31) / 32 + total_tiles;
}

static int layout_impl(int64_t n, const fgs_camera* cams, int32_t nv, int64_t k_max, int32_t flags,
                       fgs_workspace_layout* L, ViewTable* vt)
{
    if (!L) return FGS_ERR_NULL;
    if (n < 1 || n > 0x7fffffffll) return FGS_ERR_SHAPE;
    if (k_max < 0 || k_max > 0x7fffffffll) return FGS_ERR_ARG;
    if (flags & ~FGS_WS_PER_GAUSSIAN) return FGS_ERR_ARG;
    const int rc = build_views(cams, nv, vt);
    if (rc != FGS_OK) return rc;
    memset(L, 0, sizeof(*L));
    const int64_t vn = (int64_t)nv * n;
    // a rendered (view, Gaussian) pair travels through the depth sort as
    // the 32-bit value view * n + index
    if (vn > 0xffffffffll) return FGS_ERR_SHAPE;
    const int64_t nblk = (n + kPreBlock - 1) / kPreBlock;
    size_t sz[FGS_WS_NUM_SLOTS];
    sz[FGS_WS_HEADER] = sizeof(WsHeader);
    sz[FGS_WS_SCREEN] = sizeof(Screen) * (size_t)vn;
    sz[FGS_WS_RECT] = sizeof(TileRect) * (size_t)vn;
    sz[FGS_WS_LOCAL_OFF] = sizeof(uint32_t) * (size_t)vn;
    sz[FGS_WS_BLOCK_SUM] = sizeof(uint32_t) * (size_t)(nv * nblk + 1);
    sz[FGS_WS_KEYS] = sizeof(uint32_t) * (size_t)k_max;
    sz[FGS_WS_VALS] = sizeof(uint32_t) * (size_t)k_max;
    sz[FGS_WS_KEYS_ALT] = sz[FGS_WS_KEYS];
    sz[FGS_WS_VALS_ALT] = sz[FGS_WS_VALS];
    sz[FGS_WS_SORT_HIST] = sort_hist_bytes(k_max > vn ? k_max : vn, kMaxDigitBits);
    sz[FGS_WS_RANGES] = sizeof(uint2) * (size_t)vt->total_tiles;
    sz[FGS_WS_T_FINAL] = sizeof(float) * (size_t)vt->total_pixels;
    sz[FGS_WS_N_CONTRIB] = sizeof(uint32_t) * (size_t)vt->total_pixels;
    sz[FGS_WS_SCREEN_GRAD] = sizeof(ScreenGrad) * (size_t)vn;
    sz[FGS_WS_LOSS_MAPS] = sizeof(float) * 9 * (size_t)vt->total_pixels;
    sz[FGS_WS_LOSS_PART] = sizeof(double) * 2 * (size_t)vt->total_tiles;
    sz[FGS_WS_N_BLENDED] = sizeof(uint32_t) * (size_t)vt->total_pixels;
    sz[FGS_WS_TILE_QUEUE] = sizeof(uint32_t) * (4 + (size_t)vt->total_tiles);
    sz[FGS_WS_DEPTH_KEYS] = sizeof(uint32_t) * (size_t)vn;
    sz[FGS_WS_DEPTH_VALS] = sizeof(uint32_t) * (size_t)vn;
    sz[FGS_WS_DEPTH_KEYS_ALT] = sizeof(uint32_t) * (size_t)vn;
    sz[FGS_WS_DEPTH_VALS_ALT] = sizeof(uint32_t) * (size_t)vn;
    sz[FGS_WS_SORTED_OFF] = sizeof(uint32_t) * (size_t)vn;
    sz[FGS_WS_SORTED_BLOCK] = sizeof(uint32_t) * (size_t)(count_scan_blocks(vn) + 1);
    const bool pg = flags & FGS_WS_PER_GAUSSIAN;
    const int64_t mb = max_buckets_for(k_max, vt->total_tiles);
    sz[FGS_WS_BUCKET_OFF] = pg ? sizeof(uint32_t) * ((size_t)vt->total_tiles + 1) : 0;
    sz[FGS_WS_BUCKET_TILE] = pg ? sizeof(uint32_t) * (size_t)mb : 0;
    sz[FGS_WS_BUCKET_STATE] = pg ? sizeof(float4) * (size_t)kTilePixels * (size_t)mb : 0;
    sz[FGS_WS_PIXEL_FINAL] = pg ? sizeof(float4) * (size_t)vt->total_pixels : 0;
    size_t off = 0;
    for (int s = 0; s < FGS_WS_NUM_SLOTS; ++s) {
        L->offset[s] = off;
        L->bytes[s] = sz[s];
        off = align256(off + sz[s]);
    }
    L->total_bytes = off;
    L->n = n;
    L->k_max = k_max;
    L->n_views = nv;
    L->total_tiles = vt->total_tiles;
    L->total_pixels = vt->total_pixels;
    L->sort_bits = sort_bits_for(vt->total_tiles);
    L->sorted_in_alt = radix_passes(L->sort_bits, 8) & 1;
    L->flags = flags;
    L->tuning.blend_pixels_per_thread = kDefaultPPT;
    L->tuning.blend_batch = kDefaultBatch;
    L->tuning.blend_schedule = FGS_SCHEDULE_QUEUE;
    return FGS_OK;
}

// Recomputes the layout from the call's cameras and checks it matches.
static int check_layout(void* ws, const fgs_workspace_layout* L, const fgs_camera* cams, ViewTable* vt)
{
    if (!ws || !L || !cams) return FGS_ERR_NULL;
    if ((uintptr_t)ws % 256 != 0) return FGS_ERR_ALIGN;
    fgs_workspace_layout mine;
    const int rc = layout_impl(L->n, cams, L->n_views, L->k_max, L->flags, &mine, vt);
    if (rc != FGS_OK) return rc;
    if (memcmp(mine.offset, L->offset, sizeof(mine.offset)) != 0 || mine.total_bytes != L->total_bytes)
        return FGS_ERR_WORKSPACE;
    if (!blend_config_supported(L->tuning.blend_pixels_per_thread, L->tuning.blend_batch))
        return FGS_ERR_ARG;
    if ((L->tuning.backward_pixels_per_thread || L->tuning.backward_batch) &&
        !blend_config_supported(L->tuning.backward_pixels_per_thread, L->tuning.backward_batch))
        return FGS_ERR_ARG;
    if (L->tuning.blend_schedule != FGS_SCHEDULE_QUEUE && L->tuning.blend_schedule != FGS_SCHEDULE_GRID)
        return FGS_ERR_ARG;
    if (!digit_bits_ok(L->tuning.depth_sort_digit_bits) || !digit_bits_ok(L->tuning.tile_sort_digit_bits))
        return FGS_ERR_ARG;
    // where the tile sort leaves its result follows from its digit width
    if (L->sorted_in_alt != (radix_passes(L->sort_bits, digit_bits(L->tuning.tile_sort_digit_bits)) & 1))
        return FGS_ERR_WORKSPACE;
    if (L->tuning.duplicate_order != FGS_DUPLICATE_STRIDED && L->tuning.duplicate_order != FGS_DUPLICATE_SPLIT)
        return FGS_ERR_ARG;
    if (L->tuning.blend_backward != FGS_BACKWARD_PER_PIXEL &&
        L->tuning.blend_backward != FGS_BACKWARD_PER_GAUSSIAN)
        return FGS_ERR_ARG;
    if (L->tuning.blend_backward == FGS_BACKWARD_PER_GAUSSIAN && !(L->flags & FGS_WS_PER_GAUSSIAN))
        return FGS_ERR_WORKSPACE;
    return FGS_OK;
}

template <typename T> static T* slot(void* ws, const fgs_workspace_layout* L, int s)
{
    return reinterpret_cast<T*>(static_cast<unsigned char*>(ws) + L->offset[s]);
}

// Parameters (or their gradients: like = the parameters, float32 only):
// groups 0..5 always, 6 and 7 (velocity, t0; float32) both or neither, and a
// gradient struct has exactly the parameters' groups.
static int check_params(const fgs_params* p, int64_t n, bool grads, const fgs_params* like = nullptr)
{
    if (!p) return FGS_ERR_NULL;
    if (p->n != n) return FGS_ERR_SHAPE;
    if ((p->data[6] == nullptr) != (p->data[7] == nullptr)) return FGS_ERR_NULL;
    if (like && (p->data[6] == nullptr) != (like->data[6] == nullptr)) return FGS_ERR_NULL;
    const int ng = groups_of(p);
    for (int g = 0; g < ng; ++g) {
        if (!p->data[g]) return FGS_ERR_NULL;
        const int dt = p->dtype[g];
        if (dt != FGS_F32 && dt != FGS_BF16 && dt != FGS_F16) return FGS_ERR_DTYPE;
        if ((grads || g < 4 || g >= kStaticGroups) && dt != FGS_F32) return FGS_ERR_DTYPE;
    }
    if (p->dtype[4] != p->dtype[5]) return FGS_ERR_DTYPE;
    if (!grads && ng == FGS_NUM_GROUPS && !(p->sigma_t > 0.0f)) return FGS_ERR_ARG;
    if (!grads && (uintptr_t)p->data[2] % 16 != 0) return FGS_ERR_ALIGN;  // quaternions: one 16-byte load
    return FGS_OK;
}

static int cuda_rc(cudaError_t e) { return e == cudaSuccess ? FGS_OK : FGS_ERR_CUDA; }

}  // namespace fgs

using namespace fgs;

extern "C" {

int fgs_workspace_size(int64_t n, const fgs_camera* cams_host, int32_t n_views, int64_t k_max,
                       fgs_workspace_layout* out_host)
{
    ViewTable vt;
    return layout_impl(n, cams_host, n_views, k_max, 0, out_host, &vt);
}

int fgs_workspace_size_ex(int64_t n, const fgs_camera* cams_host, int32_t n_views, int64_t k_max,
                          int32_t flags, fgs_workspace_layout* out_host)
{
    ViewTable vt;
    return layout_impl(n, cams_host, n_views, k_max, flags, out_host, &vt);
}

int fgs_render_forward(void* ws, const fgs_workspace_layout* L, const fgs_params* params,
                       int32_t sh_degree, const fgs_camera* cams_host, const fgs_camera* cams_device,
                       const float bg[3], float* images, void* stream)
{
    ViewTable vt;
    int rc = check_layout(ws, L, cams_host, &vt);
    if (rc != FGS_OK) return rc;
    if (!cams_device || !bg || !images) return FGS_ERR_NULL;
    if (sh_degree < 0 || sh_degree > 3) return FGS_ERR_SH_DEGREE;
    if ((rc = check_params(params, L->n, false)) != FGS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    profile_mark(st, "begin");
    const int64_t n = L->n;
    WsHeader* hdr = slot<WsHeader>(ws, L, FGS_WS_HEADER);
    Screen* screen = slot<Screen>(ws, L, FGS_WS_SCREEN);
    TileRect* rects = slot<TileRect>(ws, L, FGS_WS_RECT);
    uint32_t* local_off = slot<uint32_t>(ws, L, FGS_WS_LOCAL_OFF);
    uint32_t* block_sum = slot<uint32_t>(ws, L, FGS_WS_BLOCK_SUM);
    uint32_t* keys = slot<uint32_t>(ws, L, FGS_WS_KEYS);
    uint32_t* vals = slot<uint32_t>(ws, L, FGS_WS_VALS);
    uint32_t* keys_alt = slot<uint32_t>(ws, L, FGS_WS_KEYS_ALT);
    uint32_t* vals_alt = slot<uint32_t>(ws, L, FGS_WS_VALS_ALT);
    uint32_t* dkeys = slot<uint32_t>(ws, L, FGS_WS_DEPTH_KEYS);
    uint32_t* dvals = slot<uint32_t>(ws, L, FGS_WS_DEPTH_VALS);
    uint32_t* dkeys_alt = slot<uint32_t>(ws, L, FGS_WS_DEPTH_KEYS_ALT);
    uint32_t* dvals_alt = slot<uint32_t>(ws, L, FGS_WS_DEPTH_VALS_ALT);
    uint32_t* hist = slot<uint32_t>(ws, L, FGS_WS_SORT_HIST);
    const int64_t vn = (int64_t)vt.n_views * n;
    if ((rc = cuda_rc(launch_preprocess_fwd(n, sh_degree, params, cams_device, vt, screen, rects,
                                            local_off, block_sum, st))) != FGS_OK)
        return rc;
    // stage 1: the rendered (view, Gaussian) pairs by depth (stable: ties keep (view, id) order)
    if ((rc = cuda_rc(launch_compact_visible(n, vt, screen, rects, local_off, block_sum, hdr, dkeys, dvals,
                                             st))) != FGS_OK)
        return rc;
    cudaError_t e;
    const int dalt = radix_sort_u32(dkeys, dvals, dkeys_alt, dvals_alt, vn, &hdr->counters[1], kDepthBits,
                                    hist, true, digit_bits(L->tuning.depth_sort_digit_bits), st, &e);
    if (e != cudaSuccess) return FGS_ERR_CUDA;
    // stage 2: their instances, emitted in depth order, stably by tile id
    // (the depth keys are spent: their slot holds the split duplication's
    // list of large rectangles)
    if ((rc = cuda_rc(launch_sorted_duplicate(n, vt, screen, rects, dalt ? dvals_alt : dvals,
                                              slot<uint32_t>(ws, L, FGS_WS_SORTED_OFF),
                                              slot<uint32_t>(ws, L, FGS_WS_SORTED_BLOCK), hdr, L->k_max,
                                              keys, vals, dkeys, L->tuning.duplicate_order, st))) != FGS_OK)
        return rc;
    const uint32_t* k_dev = &hdr->counters[0];
    const int alt = radix_sort_u32(keys, vals, keys_alt, vals_alt, L->k_max, k_dev, L->sort_bits, hist,
                                   false, digit_bits(L->tuning.tile_sort_digit_bits), st, &e);
    if (e != cudaSuccess) return FGS_ERR_CUDA;
    const uint32_t* skeys = alt ? keys_alt : keys;
    const uint32_t* svals = alt ? vals_alt : vals;
    uint2* ranges = slot<uint2>(ws, L, FGS_WS_RANGES);
    if ((rc = cuda_rc(launch_tile_ranges(skeys, k_dev, L->k_max, ranges, vt.total_tiles, st))) != FGS_OK)
        return rc;
    uint32_t* queue = slot<uint32_t>(ws, L, FGS_WS_TILE_QUEUE);
    if (L->tuning.blend_schedule == FGS_SCHEDULE_QUEUE &&
        (rc = cuda_rc(launch_tile_order(ranges, vt.total_tiles, queue, st))) != FGS_OK)
        return rc;
    const bool pg = L->tuning.blend_backward == FGS_BACKWARD_PER_GAUSSIAN;
    return cuda_rc(launch_blend_fwd(vt, n, ranges, svals, screen, bg, images,
                                    slot<float>(ws, L, FGS_WS_T_FINAL),
                                    slot<uint32_t>(ws, L, FGS_WS_N_CONTRIB),
                                    slot<uint32_t>(ws, L, FGS_WS_N_BLENDED), queue,
                                    L->tuning.blend_pixels_per_thread, L->tuning.blend_batch,
                                    L->tuning.blend_schedule,
                                    pg ? slot<uint32_t>(ws, L, FGS_WS_BUCKET_OFF) : nullptr,
                                    pg ? slot<uint32_t>(ws, L, FGS_WS_BUCKET_TILE) : nullptr,
                                    pg ? slot<float4>(ws, L, FGS_WS_BUCKET_STATE) : nullptr,
                                    pg ? slot<float4>(ws, L, FGS_WS_PIXEL_FINAL) : nullptr,
                                    max_buckets_for(L->k_max, vt.total_tiles), st));
}

int fgs_loss_l1_dssim(void* ws, const fgs_workspace_layout* L, const fgs_camera* cams_host,
                      const float* images, const float* targets, float lambda, float* loss_out,
                      float* dl_dimages, void* stream)
{
    ViewTable vt;
    int rc = check_layout(ws, L, cams_host, &vt);
    if (rc != FGS_OK) return rc;
    if (!images || !targets || !loss_out || !dl_dimages) return FGS_ERR_NULL;
    if (!(lambda >= 0.0f && lambda <= 1.0f)) return FGS_ERR_ARG;
    profile_mark((cudaStream_t)stream, "begin");
    return cuda_rc(launch_loss(vt, images, targets, lambda, slot<float>(ws, L, FGS_WS_LOSS_MAPS),
                               slot<double>(ws, L, FGS_WS_LOSS_PART), loss_out, dl_dimages,
                               slot<WsHeader>(ws, L, FGS_WS_HEADER), (cudaStream_t)stream));
}

// The per-pixel blend backward's launch pair: its own when set, else the
// forward's.
static int backward_ppt(const fgs_tuning& t)
{
    return t.backward_pixels_per_thread ? t.backward_pixels_per_thread : t.blend_pixels_per_thread;
}
static int backward_batch(const fgs_tuning& t)
{
    return t.backward_pixels_per_thread ? t.backward_batch : t.blend_batch;
}

// Blend backward into the screen-gradient records (shared by both backward
// entry points).  adam (nullable): also prepare that Adam step, in the launch
// that zeroes the records.
static int backward_blend(void* ws, const fgs_workspace_layout* L, const ViewTable& vt, const float bg[3],
                          const float* dl_dimages, fgs_adam_state* adam, cudaStream_t st)
{
    const int64_t n = L->n;
    const uint32_t* svals = slot<uint32_t>(ws, L, L->sorted_in_alt ? FGS_WS_VALS_ALT : FGS_WS_VALS);
    Screen* screen = slot<Screen>(ws, L, FGS_WS_SCREEN);
    ScreenGrad* sgrad = slot<ScreenGrad>(ws, L, FGS_WS_SCREEN_GRAD);
    // clears the records of the (view, block)s with a rendered pair (and
    // prepares the Adam step of the fused call)
    if (launch_zero_and_adam_prepare(sgrad, slot<uint32_t>(ws, L, FGS_WS_BLOCK_SUM),
                                     &slot<WsHeader>(ws, L, FGS_WS_HEADER)->counters[1], n, vt.n_views, adam,
                                     st) != cudaSuccess)
        return FGS_ERR_CUDA;
    if (L->tuning.blend_backward == FGS_BACKWARD_PER_GAUSSIAN)
        return cuda_rc(launch_blend_bwd_pg(vt, n, slot<uint2>(ws, L, FGS_WS_RANGES), svals, screen, dl_dimages,
                                           slot<uint32_t>(ws, L, FGS_WS_N_CONTRIB),
                                           slot<uint32_t>(ws, L, FGS_WS_BUCKET_OFF),
                                           slot<uint32_t>(ws, L, FGS_WS_BUCKET_TILE),
                                           slot<float4>(ws, L, FGS_WS_BUCKET_STATE),
                                           slot<float4>(ws, L, FGS_WS_PIXEL_FINAL),
                                           max_buckets_for(L->k_max, vt.total_tiles), sgrad, st));
    return cuda_rc(launch_blend_bwd(vt, n, slot<uint2>(ws, L, FGS_WS_RANGES), svals, screen, bg, dl_dimages,
                                    slot<float>(ws, L, FGS_WS_T_FINAL),
                                    slot<uint32_t>(ws, L, FGS_WS_N_CONTRIB), sgrad,
                                    slot<uint32_t>(ws, L, FGS_WS_TILE_QUEUE),
                                    backward_ppt(L->tuning), backward_batch(L->tuning),
                                    L->tuning.blend_schedule, st));
}

int fgs_render_backward(void* ws, const fgs_workspace_layout* L, const fgs_params* params,
                        int32_t sh_degree, const fgs_camera* cams_host,
                        const fgs_camera* cams_device, const float bg[3], const float* dl_dimages,
                        const fgs_params* grads, void* stream)
{
    ViewTable vt;
    int rc = check_layout(ws, L, cams_host, &vt);
    if (rc != FGS_OK) return rc;
    if (!cams_device || !bg || !dl_dimages) return FGS_ERR_NULL;
    if (sh_degree < 0 || sh_degree > 3) return FGS_ERR_SH_DEGREE;
    if ((rc = check_params(params, L->n, false)) != FGS_OK) return rc;
    if ((rc = check_params(grads, L->n, true, params)) != FGS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    profile_mark(st, "begin");
    if ((rc = backward_blend(ws, L, vt, bg, dl_dimages, nullptr, st)) != FGS_OK) return rc;
    return cuda_rc(launch_preprocess_bwd(L->n, sh_degree, params, cams_device, vt,
                                         slot<Screen>(ws, L, FGS_WS_SCREEN), slot<TileRect>(ws, L, FGS_WS_RECT),
                                         slot<ScreenGrad>(ws, L, FGS_WS_SCREEN_GRAD), grads, st));
}

int fgs_render_backward_adam(void* ws, const fgs_workspace_layout* L, const fgs_params* params,
                             int32_t sh_degree, const fgs_camera* cams_host,
                             const fgs_camera* cams_device, const float bg[3], const float* dl_dimages,
                             const fgs_params* exp_avg, const fgs_params* exp_avg_sq,
                             fgs_adam_state* state_device, const fgs_params* grads, void* stream)
{
    ViewTable vt;
    int rc = check_layout(ws, L, cams_host, &vt);
    if (rc != FGS_OK) return rc;
    if (!cams_device || !bg || !dl_dimages || !exp_avg || !exp_avg_sq || !state_device) return FGS_ERR_NULL;
    if (sh_degree < 0 || sh_degree > 3) return FGS_ERR_SH_DEGREE;
    if ((rc = check_params(params, L->n, false)) != FGS_OK) return rc;
    if (grads && (rc = check_params(grads, L->n, true, params)) != FGS_OK) return rc;
    if (exp_avg->n != L->n || exp_avg_sq->n != L->n) return FGS_ERR_SHAPE;
    for (int g = 0; g < groups_of(params); ++g) {
        if (!exp_avg->data[g] || !exp_avg_sq->data[g]) return FGS_ERR_NULL;
        if (exp_avg->dtype[g] != exp_avg->dtype[0] || exp_avg_sq->dtype[g] != exp_avg->dtype[0])
            return FGS_ERR_DTYPE;
    }
    if (!fused_adam_supported(params->dtype[4], exp_avg->dtype[0])) return FGS_ERR_DTYPE;
    cudaStream_t st = (cudaStream_t)stream;
    profile_mark(st, "begin");
    if ((rc = backward_blend(ws, L, vt, bg, dl_dimages, state_device, st)) != FGS_OK) return rc;
    return cuda_rc(launch_preprocess_bwd_adam(L->n, sh_degree, params, cams_device, vt,
                                              slot<Screen>(ws, L, FGS_WS_SCREEN), slot<TileRect>(ws, L, FGS_WS_RECT),
                                              slot<ScreenGrad>(ws, L, FGS_WS_SCREEN_GRAD), grads, exp_avg,
                                              exp_avg_sq, state_device, slot<WsHeader>(ws, L, FGS_WS_HEADER),
                                              st));
}

int fgs_adam_step(const fgs_params* params, const fgs_params* grads, const fgs_params* exp_avg,
                  const fgs_params* exp_avg_sq, const float lr[8], double beta1, double beta2,
                  double eps, int32_t step, void* stream)
{
    int rc = check_adam_args(params, grads, exp_avg, exp_avg_sq);
    if (rc != FGS_OK) return rc;
    if (!lr) return FGS_ERR_NULL;
    if (step < 1) return FGS_ERR_ARG;
    const double bc1 = 1.0 - pow(beta1, (double)step);
    const double bc2 = 1.0 - pow(beta2, (double)step);
    profile_mark((cudaStream_t)stream, "begin");
    for (int g = 0; g < groups_of(params); ++g) {
        const float step_size = (float)((double)lr[g] / bc1);
        const float inv_bc2_sqrt = (float)(1.0 / sqrt(bc2));
        const cudaError_t e = launch_adam_group(params->n * kGroupWidth[g], params->dtype[g],
                                                exp_avg->dtype[g], params->data[g],
                                                (const float*)grads->data[g], exp_avg->data[g],
                                                exp_avg_sq->data[g], step_size, inv_bc2_sqrt, beta1,
                                                beta2, eps, nullptr, g, (cudaStream_t)stream);
        if (e != cudaSuccess) return FGS_ERR_CUDA;
    }
    return FGS_OK;
}

int fgs_adam_step_device(const fgs_params* params, const fgs_params* grads, const fgs_params* exp_avg,
                         const fgs_params* exp_avg_sq, fgs_adam_state* state_device, void* stream)
{
    int rc = check_adam_args(params, grads, exp_avg, exp_avg_sq);
    if (rc != FGS_OK) return rc;
    if (!state_device) return FGS_ERR_NULL;
    cudaStream_t st = (cudaStream_t)stream;
    profile_mark(st, "begin");
    if (launch_adam_prepare(state_device, st) != cudaSuccess) return FGS_ERR_CUDA;
    for (int g = 0; g < groups_of(params); ++g) {
        const cudaError_t e = launch_adam_group(params->n * kGroupWidth[g], params->dtype[g],
                                                exp_avg->dtype[g], params->data[g],
                                                (const float*)grads->data[g], exp_avg->data[g],
                                                exp_avg_sq->data[g], 0.f, 0.f, 0.0, 0.0, 0.0,
                                                state_device, g, st);
        if (e != cudaSuccess) return FGS_ERR_CUDA;
    }
    return FGS_OK;
}

size_t fgs_sort_scratch_bytes(int64_t n)
{
    return align256(sizeof(uint32_t) * 4) + sort_hist_bytes(n > 0 ? n : 0, 8);
}

int fgs_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
                   int32_t bits, void* scratch, size_t scratch_bytes, int32_t* result_in_alt,
                   void* stream)
{
    if (!keys || !vals || !keys_alt || !vals_alt || !scratch || !result_in_alt) return FGS_ERR_NULL;
    if (n < 0 || n > 0x7fffffffll) return FGS_ERR_SHAPE;
    if (bits < 1 || bits > 64) return FGS_ERR_ARG;
    if (scratch_bytes < fgs_sort_scratch_bytes(n)) return FGS_ERR_WORKSPACE;
    if ((uintptr_t)scratch % 256 != 0) return FGS_ERR_ALIGN;
    if ((uintptr_t)keys % 8 != 0 || (uintptr_t)keys_alt % 8 != 0 || (uintptr_t)vals % 4 != 0 ||
        (uintptr_t)vals_alt % 4 != 0)
        return FGS_ERR_ALIGN;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t* n_dev = (uint32_t*)scratch;
    if (launch_set_count(n_dev, (uint32_t)n, st) != cudaSuccess) return FGS_ERR_CUDA;
    uint32_t* hist = (uint32_t*)((unsigned char*)scratch + align256(sizeof(uint32_t) * 4));
    cudaError_t e;
    *result_in_alt = radix_sort((unsigned long long*)keys, vals, (unsigned long long*)keys_alt,
                                vals_alt, n, n_dev, bits, hist, st, &e);
    return cuda_rc(e);
}

int fgs_get_error(void* ws, uint32_t* flags_host, uint64_t* instances_host, int32_t clear, void* stream)
{
    if (!ws) return FGS_ERR_NULL;
    cudaStream_t st = (cudaStream_t)stream;
    WsHeader h;
    if (cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return FGS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FGS_ERR_CUDA;
    if (flags_host) *flags_host = h.flags;
    if (instances_host) *instances_host = h.instances;
    if (clear) {
        if (cudaMemsetAsync(ws, 0, sizeof(uint32_t), st) != cudaSuccess) return FGS_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return FGS_ERR_CUDA;
    }
    return FGS_OK;
}

int fgs_profile_attach(void** events, const char** labels, int32_t capacity)
{
    if (!events || !labels || capacity <= 0) {
        g_prof_events = nullptr;
        g_prof_labels = nullptr;
        g_prof_cap = 0;
        g_prof_count = 0;
        return FGS_OK;
    }
    g_prof_events = reinterpret_cast<cudaEvent_t*>(events);
    g_prof_labels = labels;
    g_prof_cap = capacity;
    g_prof_count = 0;
    return FGS_OK;
}

int32_t fgs_profile_count(void) { return g_prof_count; }

const char* fgs_strerror(int code)
{
    switch (code) {
    case FGS_OK: return "ok";
    case FGS_ERR_NULL: return "a required pointer is NULL";
    case FGS_ERR_SHAPE: return "bad size (Gaussian count, image size or tile count)";
    case FGS_ERR_SH_DEGREE: return "SH degree outside 0..3";
    case FGS_ERR_WORKSPACE: return "workspace layout does not match the call or is too small";
    case FGS_ERR_DTYPE: return "unsupported storage type";
    case FGS_ERR_CUDA: return "CUDA launch failed";
    case FGS_ERR_VIEWS: return "view count outside 1..16";
    case FGS_ERR_ALIGN: return "pointer not aligned";
    case FGS_ERR_ARG: return "argument out of range";
    case FGS_ERR_TOO_LARGE: return "more pairs than the static sort scratch holds";
    default: return "unknown status";
    }
}

const char* fgs_flag_string(uint32_t flag)
{
    switch (flag) {
    case FGS_FLAG_CAPACITY: return "instances exceeded the workspace capacity k_max (extra ones dropped)";
    case FGS_FLAG_NONFINITE: return "a NaN or infinity reached the loss or an Adam update";
    default: return "unknown flag";
    }
}

}  // extern "C"
