// (d) Tile-binned, depth-sorted, front-to-back Gaussian splatting - the 3DGS
// rasteriser the paper renders with (Sec. 3.1), black background (Sec. 4.2).
//
// Pipeline (all on the device, no host synchronisation; the pair count is
// data dependent and only ever read on the device):
//   project   one thread per Gaussian: EWA projection, conic, tile-independent
//             pixel rect, pair count, depth key, packed blend records.
//   depth sort  stable LSD radix sort of (depth bits, index) over G keys.
//   scan      exclusive scan of pair counts in depth order -> pair offsets.
//   emit      each Gaussian writes (tile id, index) for its tiles at its
//             offset; emission follows depth order.
//   tile sort stable LSD radix sort of the pairs on the tile id only; with
//             the depth-ordered emission this yields (tile, depth, index).
//   ranges    begin/end of every tile's run.
//   blend     one warp per (tile, pixel box), independent of the others:
//             32-entry record batches prefetched into the warp's own
//             shared-memory buffers; the warp leaves as soon as its pixels
//             are saturated.
// Backward: reverse traversal from the per-pixel checkpoint (T_final,
// n_last) with warp-reduced atomics, then a per-Gaussian projection adjoint.
#include "splat_dev.cuh"

namespace {

struct SplatWs {
    uint32_t *dkey_a, *dkey_b;   // [G] depth keys
    int32_t *dval_a, *dval_b;    // [G] Gaussian indices
    int32_t *npairs;             // [G]
    int32_t *offsets;            // [G]
    uint32_t *pkey_a, *pkey_b;   // [cap] tile keys
    int32_t *pval_b;             // [cap] ping-pong partner of pair_gauss
    float4 *rec0;                // [G] (mx, my, qa, qb): log2-domain conic, see bin_keys_kernel
    float4 *rec1;                // [G] (qc, log2 o, x0 | y0 << 16, x1 | y1 << 16) rect bits
    float4 *rec2;                // [G] (r, g, b, o)
    int32_t *sort_hist;          // [OS_MAX_PASSES][RADIX] digit histograms + [OS_MAX_PASSES] tile tickets
    unsigned *sort_desc;         // [OS_MAX_PASSES][tiles][RADIX] look-back descriptors
    int32_t *block_sums;         // [NB]
    int32_t *count_g;            // [1] = G on the device
    float *d_mean2d;             // [2][G]
    float *d_conic;              // [3][G]
    int32_t *tile_order;         // [ntiles] tiles by descending list length (bucketed)
    int NB;
    bool masks;                  // region masks in the pair keys (AVATAR_TUNE_REGION_MASKS)
};

// Fixed radix grid: two blocks per SM of a 152-SM GB300.
constexpr int RADIX_BLOCKS = 304;
int radix_blocks(const avatar_ctx *) { return RADIX_BLOCKS; }

size_t splat_ws_layout(const avatar_splat_args *a, int NB, void *base, size_t cap, SplatWs *out)
{
    WsCarver c(base, cap);
    SplatWs w;
    size_t G = (size_t)(a->G > 0 ? a->G : 1);
    size_t P = (size_t)(a->pair_capacity > 0 ? a->pair_capacity : 1);
    w.dkey_a = c.take<uint32_t>(G);
    w.dkey_b = c.take<uint32_t>(G);
    w.dval_a = c.take<int32_t>(G);
    w.dval_b = c.take<int32_t>(G);
    w.npairs = c.take<int32_t>(G);
    w.offsets = c.take<int32_t>(G);
    w.pkey_a = c.take<uint32_t>(P);
    w.pkey_b = c.take<uint32_t>(P);
    w.pval_b = c.take<int32_t>(P);
    w.rec0 = c.take<float4>(G);
    w.rec1 = c.take<float4>(G);
    w.rec2 = c.take<float4>(G);
    w.sort_hist = c.take<int32_t>((size_t)(4 * RADIX + 4));
    {
        size_t t = (size_t)((P > G ? P : G) + 2047) / 2048;
        w.sort_desc = c.take<unsigned>(4 * t * RADIX);
    }
    w.block_sums = c.take<int32_t>((size_t)NB);
    w.count_g = c.take<int32_t>(1);
    w.d_mean2d = c.take<float>(2 * G);
    w.d_conic = c.take<float>(3 * G);
    {
        const int ts = a->tile == 0 ? 16 : a->tile;
        const size_t nt = (size_t)((a->cam.width + ts - 1) / ts) * ((a->cam.height + ts - 1) / ts);
        w.tile_order = c.take<int32_t>(nt > 0 ? nt : 1);
    }
    w.NB = NB;
    if (out) *out = w;
    return c.off;
}

// ---------------------------------------------------------------- project
__global__ void __launch_bounds__(256)
project_kernel(avatar_splat_args a, CamDev cam)
{
    const int G = a.G;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const float o = ld_attr(a.opacity, g, a.attr_dtype);
        const Splat2D s = project_gaussian(a.xd, a.cov, G, g, o, a.cull && a.cull[g], cam);
        store_splat(s, G, g, a.mean2d, a.conic, a.depth, a.rect);
    }
}

// Per-Gaussian pair count, depth key and the geometric blend records (rec0,
// rec1), from the caller-visible projection buffers (rect, depth, mean2d,
// conic) and the opacity; the colour record is completed by the blend call,
// so binning does not wait for shading.
__global__ void __launch_bounds__(256)
bin_keys_kernel(avatar_splat_args a, int TS, SplatWs w)
{
    const int G = a.G;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        int x0 = a.rect[g], y0 = a.rect[G + g], x1 = a.rect[2 * G + g], y1 = a.rect[3 * G + g];
        int n = rect_tiles(x0, y0, x1, y1, a.cam.width, a.cam.height, TS);
        w.npairs[g] = n;
        w.dkey_a[g] = n > 0 ? __float_as_uint(a.depth[g]) : 0xffffffffu;
        w.dval_a[g] = g;
        float o = ld_attr(a.opacity, g, a.attr_dtype);
        float4 r2;
        make_records(a.mean2d[g], a.mean2d[G + g], a.conic[g], a.conic[G + g], a.conic[2 * G + g], x0, y0, x1, y1,
                     0.f, 0.f, 0.f, o, w.rec0[g], w.rec1[g], r2);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *w.count_g = G;
}

// The colour blend record (r, g, b, opacity) of every Gaussian.
__global__ void __launch_bounds__(256)
color_records_kernel(avatar_splat_args a, SplatWs w)
{
    const int G = a.G;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x)
        w.rec2[g] = make_float4(__ldg(a.color + g), __ldg(a.color + G + g), __ldg(a.color + 2 * (size_t)G + g),
                                ld_attr(a.opacity, g, a.attr_dtype));
}

__global__ void __launch_bounds__(256)
emit_pairs_kernel(const int32_t *__restrict__ sorted_idx, const int32_t *__restrict__ offsets,
                  const int32_t *__restrict__ npairs, const int32_t *__restrict__ rect,
                  const float4 *__restrict__ rec0, const float4 *__restrict__ rec1, int G, int TS, int ntx,
                  int rmode, long cap, uint32_t *__restrict__ keys, int32_t *__restrict__ vals)
{
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < G; base += warps * 32) {
        const int i = base + (threadIdx.x & 31);
        int g = 0, n = 0, tx0 = 0, ty0 = 0, w = 1;
        long off = 0;
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
        if (i < G) {
            g = sorted_idx[i];
            n = npairs[g];
            off = offsets[i];
            if (n > 0) {
                tx0 = rect[g] / TS;
                ty0 = rect[G + g] / TS;
                w = rect[2 * G + g] / TS - tx0 + 1;
                r0 = rec0[g];
                r1 = rec1[g];
            }
        }
        emit_pairs_warp(n, off, g, tx0, ty0, w, 0, ntx, tile_reach_of(r0, r1), TS, rmode, cap, keys, vals);
    }
}

// The blend kernels' tile order: tiles by the bit length of their list
// length, longest first (one block; the order within a length class is
// arbitrary).  Blocks start in index order, so the costly tiles start first
// and the last wave holds the cheap ones.
__global__ void __launch_bounds__(1024)
tile_order_kernel(const int2 *__restrict__ ranges, int ntiles, int32_t *__restrict__ order)
{
    __shared__ int cnt[33];
    if (threadIdx.x < 33) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        const int2 r = __ldg(ranges + t);
        const int len = max(r.y - r.x, 0);
        atomicAdd(&cnt[len > 0 ? __clz(len) : 32], 1);  // class 0 = the longest lists
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int k = 0; k < 33; ++k) {
            const int n = cnt[k];
            cnt[k] = run;
            run += n;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        const int2 r = __ldg(ranges + t);
        const int len = max(r.y - r.x, 0);
        order[atomicAdd(&cnt[len > 0 ? __clz(len) : 32], 1)] = t;
    }
}

template <int TS, int PPT>
__global__ void __launch_bounds__(BWD_WARPS * 32)
blend_kernel(const int2 *__restrict__ ranges, const int32_t *__restrict__ pair_gauss, const float4 *__restrict__ rec0,
             const float4 *__restrict__ rec1, const float4 *__restrict__ rec2, int W, int H, int ntx, int ntiles,
             const uint32_t *__restrict__ pkeys, int rmode, float *__restrict__ image,
             float *__restrict__ T_final, int32_t *__restrict__ n_last, const int32_t *__restrict__ torder)
{
    constexpr int NB = TS * TS / (32 * PPT);  // pixel boxes per tile
    __shared__ float4 s0[BWD_WARPS][2][32];
    __shared__ float4 s1[BWD_WARPS][2][32];
    __shared__ float4 s2[BWD_WARPS][2][32];
    const int warp = threadIdx.x >> 5;
    const int item = blockIdx.x * BWD_WARPS + warp;
    constexpr int NBD = NB > 0 ? NB : 1;  // NB = 0: a split the tile cannot hold (never launched)
    if (item >= ntiles * NB) return;      // warp-uniform; the kernel has no CTA barrier
    const int tile = __ldg(torder + item / NBD);
    blend_box<TS, PPT>(ranges[tile], pair_gauss, rec0, rec1, rec2, W, H, tile % ntx, tile / ntx, item % NBD, pkeys,
                       rmode, image, T_final, n_last, s0[warp], s1[warp], s2[warp]);
}

// BWD_WARPS independent warps per CTA, each one (tile, pixel box) item.
template <int TS, int PPT>
__global__ void __launch_bounds__(BWD_WARPS * 32)
blend_backward_kernel(const int2 *__restrict__ ranges, const int32_t *__restrict__ pair_gauss,
                      const float4 *__restrict__ rec0, const float4 *__restrict__ rec1, const float4 *__restrict__ rec2,
                      int W, int H, int ntx, int ntiles, const uint32_t *__restrict__ pkeys, int rmode,
                      const float *__restrict__ T_final, const int32_t *__restrict__ n_last,
                      const float *__restrict__ d_image, int G,
                      float *__restrict__ d_mean2d, float *__restrict__ d_conic, float *__restrict__ d_opacity,
                      float *__restrict__ d_color, const int32_t *__restrict__ torder)
{
    constexpr int NB = TS * TS / (32 * PPT);  // pixel boxes per tile
    __shared__ float4 s0[BWD_WARPS][2][32];
    __shared__ float4 s1[BWD_WARPS][2][32];
    __shared__ float4 s2[BWD_WARPS][2][32];
    __shared__ int sg[BWD_WARPS][2][32];
    const int warp = threadIdx.x >> 5;
    const int item = blockIdx.x * BWD_WARPS + warp;
    constexpr int NBD = NB > 0 ? NB : 1;  // NB = 0: a split the tile cannot hold (never launched)
    if (item >= ntiles * NB) return;      // warp-uniform; the kernel has no CTA barrier
    const int tile = __ldg(torder + item / NBD);
    blend_backward_box<TS, PPT>(ranges[tile], pair_gauss, rec0, rec1, rec2, W, H, tile % ntx, tile / ntx, item % NBD,
                                pkeys, rmode, T_final, n_last, d_image, (size_t)G, d_mean2d, d_conic, d_opacity,
                                d_color, s0[warp], s1[warp], s2[warp], sg[warp]);
}

__global__ void __launch_bounds__(256)
project_backward_kernel(avatar_splat_args a, CamDev cam, const float *__restrict__ d_mean2d,
                        const float *__restrict__ d_conic, float *__restrict__ d_xd, float *__restrict__ d_cov)
{
    const int G = a.G;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        float dmx = d_mean2d[g], dmy = d_mean2d[G + g];
        float da = d_conic[g], db = d_conic[G + g], dc = d_conic[2 * G + g];
        bool has = a.rect[2 * G + g] >= a.rect[g];
        float gx[3] = {0.f, 0.f, 0.f}, gc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (has && !(dmx == 0.f && dmy == 0.f && da == 0.f && db == 0.f && dc == 0.f))
            project_adjoint(a.xd, a.cov, G, g, cam, dmx, dmy, da, db, dc, gx, gc);
#pragma unroll
        for (int i = 0; i < 3; ++i) d_xd[i * G + g] = gx[i];
#pragma unroll
        for (int i = 0; i < 6; ++i) d_cov[i * G + g] = gc[i];
    }
}


// Sizes only (what the workspace and tile-count queries need).
int check_splat_dims(const avatar_splat_args *a)
{
    if (!a || a->G < 0) return AVATAR_ERR_INVALID_ARG;
    if (a->cam.width < 1 || a->cam.height < 1 || a->cam.width > 16384 || a->cam.height > 16384)
        return AVATAR_ERR_INVALID_ARG;
    int ts = a->tile == 0 ? 16 : a->tile;
    if (ts != 8 && ts != 16 && ts != 32) return AVATAR_ERR_INVALID_ARG;
    if (a->pair_capacity < 1 || a->pair_capacity > 0x7fffffffL) return AVATAR_ERR_INVALID_ARG;
    return AVATAR_OK;
}

int check_splat(const avatar_splat_args *a)
{
    AV_TRY(check_splat_dims(a));
    if (a->G > 0 && (!a->xd || !a->cov || !a->opacity || !a->color || !a->mean2d || !a->conic || !a->depth ||
                     !a->rect))
        return AVATAR_ERR_INVALID_ARG;
    if (!a->tile_range || !a->pair_gauss || !a->num_pairs || !a->image || !a->T_final || !a->n_last)
        return AVATAR_ERR_INVALID_ARG;
    if (a->attr_dtype != AVATAR_DTYPE_F32 && a->attr_dtype != AVATAR_DTYPE_BF16) return AVATAR_ERR_INVALID_ARG;
    return AVATAR_OK;
}

int tile_of(const avatar_splat_args *a) { return a->tile == 0 ? 16 : a->tile; }

int ntiles_of(const avatar_splat_args *a)
{
    int ts = tile_of(a);
    return ((a->cam.width + ts - 1) / ts) * ((a->cam.height + ts - 1) / ts);
}

int prep(avatar_ctx *ctx, const avatar_splat_args *a, void *ws, size_t ws_bytes, SplatWs *w)
{
    if (!ctx) return AVATAR_ERR_INVALID_ARG;
    AV_TRY(check_splat(a));
    if (!ws || (((uintptr_t)ws) & 255)) return AVATAR_ERR_WORKSPACE;
    if (splat_ws_layout(a, radix_blocks(ctx), ws, ws_bytes, w) > ws_bytes) return AVATAR_ERR_WORKSPACE;
    w->masks = ctx->tune[AVATAR_TUNE_REGION_MASKS] != 0;
    return AVATAR_OK;
}

int grid_cap(const avatar_ctx *ctx, long n, int threads, int per_sm)
{
    long b = (n + threads - 1) / threads;
    long cap = (long)ctx->sm_count * per_sm;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}


}  // namespace

extern "C" int avatar_splat_num_tiles(const avatar_splat_args *a)
{
    if (check_splat_dims(a) != AVATAR_OK) return 0;
    return ntiles_of(a);
}

extern "C" size_t avatar_splat_workspace_size(const avatar_splat_args *a)
{
    if (check_splat_dims(a) != AVATAR_OK) return 0;
    return splat_ws_layout(a, RADIX_BLOCKS, nullptr, 0, nullptr);
}

extern "C" int avatar_splat_project(avatar_ctx *ctx, const avatar_splat_args *a, void *ws, size_t ws_bytes,
                                    avatar_stream_t stream)
{
    SplatWs w;
    AV_TRY(prep(ctx, a, ws, ws_bytes, &w));
    cudaStream_t st = (cudaStream_t)stream;
    if (a->G == 0) return AVATAR_OK;
    project_kernel<<<grid_cap(ctx, a->G, 256, 8), 256, 0, st>>>(*a, to_dev(a->cam));
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}

extern "C" int avatar_splat_bin(avatar_ctx *ctx, const avatar_splat_args *a, void *ws, size_t ws_bytes,
                                avatar_stream_t stream)
{
    SplatWs w;
    AV_TRY(prep(ctx, a, ws, ws_bytes, &w));
    cudaStream_t st = (cudaStream_t)stream;
    const int ntiles = ntiles_of(a);
    if (cudaMemsetAsync(a->tile_range, 0, (size_t)ntiles * 2 * sizeof(int32_t), st) != cudaSuccess)
        return AVATAR_ERR_CUDA;
    if (a->G == 0) {
        if (cudaMemsetAsync(a->num_pairs, 0, sizeof(int32_t), st) != cudaSuccess) return AVATAR_ERR_CUDA;
        tile_order_kernel<<<1, 1024, 0, st>>>((const int2 *)a->tile_range, ntiles, w.tile_order);
        AV_CHECK_LAUNCH();
        return AVATAR_OK;
    }
    const int G = a->G;
    const long cap = a->pair_capacity;
    // 0. pair counts, depth keys and blend records from the projection buffers
    bin_keys_kernel<<<grid_cap(ctx, G, 256, 8), 256, 0, st>>>(*a, tile_of(a), w);
    AV_CHECK_LAUNCH();
    // 1. stable depth sort of all Gaussians (4 passes -> result back in dkey_a/dval_a)
    AV_TRY(radix_sort(w.dkey_a, w.dval_a, w.dkey_b, w.dval_b, 32, w.count_g, G, SortWs{w.sort_hist, w.sort_desc},
                       a->status, st, sort_spin_limit(ctx)));
    // 2. pair offsets in depth order
    pair_scan_reduce_kernel<<<w.NB, 1024, 0, st>>>(w.dval_a, w.npairs, G, w.NB, w.block_sums);
    pair_scan_down_kernel<<<w.NB, 1024, 0, st>>>(w.dval_a, w.npairs, G, w.NB, w.block_sums, w.offsets, a->num_pairs,
                                                 cap, a->status);
    AV_CHECK_LAUNCH();
    // 3. emit in depth order into the buffer that makes the tile sort end in pair_gauss
    const int ts = tile_of(a);
    const int ntx = (a->cam.width + ts - 1) / ts;
    int tbits = bits_for(ntiles);
    int passes = tbits <= 8 ? 1 : (tbits + 7) / 8;
    const int rmode = region_mode(ntiles, ts, w.masks);
    uint32_t *k_emit = (passes % 2 == 0) ? w.pkey_a : w.pkey_b;
    int32_t *v_emit = (passes % 2 == 0) ? a->pair_gauss : w.pval_b;
    uint32_t *k_other = (passes % 2 == 0) ? w.pkey_b : w.pkey_a;
    int32_t *v_other = (passes % 2 == 0) ? w.pval_b : a->pair_gauss;
    emit_pairs_kernel<<<grid_cap(ctx, G, 256, 8), 256, 0, st>>>(w.dval_a, w.offsets, w.npairs, a->rect, w.rec0,
                                                                 w.rec1, G, ts, ntx, rmode, cap, k_emit, v_emit);
    AV_CHECK_LAUNCH();
    // 4. stable sort of the pairs on the tile id
    AV_TRY(radix_sort(k_emit, v_emit, k_other, v_other, passes * 8, a->num_pairs, (int)cap,
                       SortWs{w.sort_hist, w.sort_desc}, a->status, st, sort_spin_limit(ctx)));
    // 5. tile ranges (sorted keys are in pkey_a)
    tile_ranges_kernel<<<ctx->sm_count * 8, 256, 0, st>>>(w.pkey_a, a->num_pairs, cap, ntiles,
                                                          tile_key_mask(ntiles, ts, w.masks), (int2 *)a->tile_range);
    // 6. the blend's tile order, longest lists first
    tile_order_kernel<<<1, 1024, 0, st>>>((const int2 *)a->tile_range, ntiles, w.tile_order);
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}

template <int TS, int PPT>
void launch_blend(const avatar_splat_args *a, const SplatWs &w, int ntiles, int ntx, cudaStream_t st)
{
    constexpr int NB = TS * TS / (32 * PPT);
    const int blocks = (int)(((long long)ntiles * NB + BWD_WARPS - 1) / BWD_WARPS);
    blend_kernel<TS, PPT><<<blocks, BWD_WARPS * 32, 0, st>>>((const int2 *)a->tile_range, a->pair_gauss, w.rec0,
                                                             w.rec1, w.rec2, a->cam.width, a->cam.height, ntx, ntiles,
                                                             w.pkey_a, region_mode(ntiles, TS, w.masks), a->image,
                                                             a->T_final, a->n_last, w.tile_order);
}

template <int TS>
void launch_blend_ppt(int ppt, const avatar_splat_args *a, const SplatWs &w, int ntiles, int ntx, cudaStream_t st)
{
    if (ppt == 4) launch_blend<TS, 4>(a, w, ntiles, ntx, st);
    else if (ppt == 2) launch_blend<TS, 2>(a, w, ntiles, ntx, st);
    else launch_blend<TS, 1>(a, w, ntiles, ntx, st);
}

extern "C" int avatar_splat_blend(avatar_ctx *ctx, const avatar_splat_args *a, void *ws, size_t ws_bytes,
                                  avatar_stream_t stream)
{
    SplatWs w;
    AV_TRY(prep(ctx, a, ws, ws_bytes, &w));
    cudaStream_t st = (cudaStream_t)stream;
    const int ts = tile_of(a);
    const int ntx = (a->cam.width + ts - 1) / ts;
    const int ntiles = ntiles_of(a);
    const int ppt = ctx->tune[AVATAR_TUNE_BLEND_PPT];
    if (a->G > 0) {
        color_records_kernel<<<grid_cap(ctx, a->G, 256, 8), 256, 0, st>>>(*a, w);
        AV_CHECK_LAUNCH();
    }
    switch (ts) {
        case 8: launch_blend_ppt<8>(ppt > 2 ? 2 : ppt, a, w, ntiles, ntx, st); break;
        case 32: launch_blend_ppt<32>(ppt, a, w, ntiles, ntx, st); break;
        default: launch_blend_ppt<16>(ppt, a, w, ntiles, ntx, st); break;
    }
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}

extern "C" int avatar_splat(avatar_ctx *ctx, const avatar_splat_args *a, void *ws, size_t ws_bytes,
                            avatar_stream_t stream)
{
    AV_TRY(avatar_splat_project(ctx, a, ws, ws_bytes, stream));
    AV_TRY(avatar_splat_bin(ctx, a, ws, ws_bytes, stream));
    return avatar_splat_blend(ctx, a, ws, ws_bytes, stream);
}

template <int TS, int PPT>
void launch_blend_bwd(const avatar_splat_args *a, const avatar_splat_grads *g, const SplatWs &w, int ntiles, int ntx,
                      int G, cudaStream_t st)
{
    constexpr int NB = TS * TS / (32 * PPT);
    const int blocks = (int)(((long long)ntiles * NB + BWD_WARPS - 1) / BWD_WARPS);
    blend_backward_kernel<TS, PPT><<<blocks, BWD_WARPS * 32, 0, st>>>(
        (const int2 *)a->tile_range, a->pair_gauss, w.rec0, w.rec1, w.rec2, a->cam.width, a->cam.height, ntx, ntiles,
        w.pkey_a, region_mode(ntiles, TS, w.masks), a->T_final, a->n_last, g->d_image, G, w.d_mean2d, w.d_conic,
        g->d_opacity, g->d_color, w.tile_order);
}

template <int TS>
void launch_blend_bwd_ppt(int ppt, const avatar_splat_args *a, const avatar_splat_grads *g, const SplatWs &w,
                          int ntiles, int ntx, int G, cudaStream_t st)
{
    if (ppt == 4) launch_blend_bwd<TS, 4>(a, g, w, ntiles, ntx, G, st);
    else if (ppt == 2) launch_blend_bwd<TS, 2>(a, g, w, ntiles, ntx, G, st);
    else launch_blend_bwd<TS, 1>(a, g, w, ntiles, ntx, G, st);
}

extern "C" int avatar_splat_backward(avatar_ctx *ctx, const avatar_splat_args *a, const avatar_splat_grads *g,
                                     void *ws, size_t ws_bytes, avatar_stream_t stream)
{
    SplatWs w;
    AV_TRY(prep(ctx, a, ws, ws_bytes, &w));
    if (!g || !g->d_image || !g->d_xd || !g->d_cov || !g->d_opacity || !g->d_color) return AVATAR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int G = a->G;
    if (G == 0) return AVATAR_OK;
    if (cudaMemsetAsync(w.d_mean2d, 0, (size_t)2 * G * sizeof(float), st) != cudaSuccess ||
        cudaMemsetAsync(w.d_conic, 0, (size_t)3 * G * sizeof(float), st) != cudaSuccess ||
        cudaMemsetAsync(g->d_opacity, 0, (size_t)G * sizeof(float), st) != cudaSuccess ||
        cudaMemsetAsync(g->d_color, 0, (size_t)3 * G * sizeof(float), st) != cudaSuccess)
        return AVATAR_ERR_CUDA;
    const int ts = tile_of(a);
    const int ntx = (a->cam.width + ts - 1) / ts;
    const int ntiles = ntiles_of(a);
    const int bppt = ctx->tune[AVATAR_TUNE_BLEND_BWD_PPT];
    switch (ts) {
        case 8: launch_blend_bwd_ppt<8>(bppt > 2 ? 2 : bppt, a, g, w, ntiles, ntx, G, st); break;
        case 32: launch_blend_bwd_ppt<32>(bppt, a, g, w, ntiles, ntx, G, st); break;
        default: launch_blend_bwd_ppt<16>(bppt, a, g, w, ntiles, ntx, G, st); break;
    }
    AV_CHECK_LAUNCH();
    project_backward_kernel<<<grid_cap(ctx, G, 256, 8), 256, 0, st>>>(*a, to_dev(a->cam), w.d_mean2d, w.d_conic,
                                                                       g->d_xd, g->d_cov);
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}
