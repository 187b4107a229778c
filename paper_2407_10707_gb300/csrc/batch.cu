// Batched rendering: B poses with their own environment lights, seen by V
// cameras of mixed resolution, with one launch per step for the whole batch
// (the relighting-under-novel-poses use of Sec. 3.5 at scale).
//
//   skin        grid.y = pose       (a) Eq. 1 + LBS of every pose
//   visibility  grid.z = pose       (b) depth maps and vertex tests
//   shade       grid.y = view       (c) Eq. 2 with the view's pose and light
//   project     grid.y = view       (d) EWA projection into the view's camera
//   bin         one depth sort over all V G Gaussians, one pair scan, pairs
//               keyed by a global tile id (view tiles back to back), one
//               stable tile sort, one range pass
//   blend       persistent warps take (global tile, pixel box) items from a
//               device counter, so views of different size and tiles of
//               different load balance without host involvement
// The backward mirrors it: one persistent blend adjoint, the shading adjoint
// over the views, a per-Gaussian pass that applies the projection adjoint
// and sums every view's gradients into its pose (and the pose-independent
// attributes into one set), and the skinning adjoint over the poses.
//
// Per-view Gaussian arrays are concatenated (element v G + g, channel stride
// V G); per-pose arrays likewise (element p G + g, stride B G).
#include <algorithm>
#include <cmath>
#include <vector>

#include "batch_internal.h"
#include "splat_dev.cuh"

namespace {

constexpr int SETUP_CHUNK = 32;
constexpr int MAX_K = 8;

struct BatchView {
    CamDev cam;
    float cc[3];    // camera centre (world)
    int pose;
    int ntx;        // tiles per image row
    int tile_base;  // first global tile of the view
    int pix_off;    // first pixel of the view in the concatenated images
};

struct SetupChunk {
    int first, n;
    BatchView v[SETUP_CHUNK];
};

__global__ void batch_setup_kernel(SetupChunk c, BatchView *views, int32_t *view_pose, float *view_cc)
{
    const int i = threadIdx.x;
    if (i >= c.n) return;
    const int v = c.first + i;
    views[v] = c.v[i];
    view_pose[v] = c.v[i].pose;
    view_cc[3 * v] = c.v[i].cc[0];
    view_cc[3 * v + 1] = c.v[i].cc[1];
    view_cc[3 * v + 2] = c.v[i].cc[2];
}

// ---------------------------------------------------------------- workspace
struct BatchWs {
    // device view table
    BatchView *views;
    int32_t *view_pose;
    float *view_cc;
    // (a) per pose
    float *bone, *xp, *xd, *cov, *nd;
    float *ag, *rg, *pg, *ubar;  // pose independent
    void *skin_ws;
    size_t skin_ws_bytes;
    // (b)
    uint32_t *bits;
    void *vis_ws;
    size_t vis_ws_bytes;
    // (c), (d) per view
    float *color, *radiance;
    uint8_t *cull;
    float *mean2d, *conic, *depth;
    int32_t *rect;
    float4 *rec0, *rec1, *rec2;
    uint32_t *dkey_a, *dkey_b;
    int32_t *dval_a, *dval_b, *npairs, *offsets;
    uint32_t *pkey_a, *pkey_b;
    int32_t *pval_a, *pval_b;
    int2 *ranges;
    float *T_final;
    int32_t *n_last;
    int32_t *sort_hist;
    unsigned *sort_desc;
    int32_t *block_sums;
    int32_t *count_vg;
    int32_t *counter;
    int32_t *tune_status;
    // backward
    float *d_color, *d_opacity_v, *d_mean2d, *d_conic;
    float *ds_xd, *ds_nd, *ds_ag, *ds_rg, *ds_pg, *ds_ubar;  // shading adjoint per view
    float *dp_xd, *dp_cov, *dp_nd;                         // summed per pose
    float *dg_ag, *dg_rg, *dg_pg, *dg_ubar;                 // summed over views
    void *skin_bwd_ws;
    size_t skin_bwd_ws_bytes;
};

struct BatchDims {
    int G, Nv, K, J, NL, OW, B, V;
    long long VG, BG;
    long long pixels;      // over all views
    long long tiles_max;   // over all views at the smallest tile edge (8)
    long long cap;
};

int batch_dims(const avatar_batch_desc *d, BatchDims *o)
{
    if (!d) return AVATAR_ERR_INVALID_ARG;
    const avatar_skin_args &a = d->avatar;
    if (a.G < 1 || a.Nv < 1 || a.K < 1 || a.K > MAX_K || a.J < 1 || a.J > 64) return AVATAR_ERR_INVALID_ARG;
    if (d->B < 1 || d->B > 65535 || d->V < 1 || d->V > AVATAR_BATCH_MAX_VIEWS || !d->views) return AVATAR_ERR_INVALID_ARG;
    if (d->NL < 1 || d->NL > 4096 || d->tile < 0) return AVATAR_ERR_INVALID_ARG;
    if (d->tile != 0 && d->tile != 8 && d->tile != 16 && d->tile != 32) return AVATAR_ERR_INVALID_ARG;
    if (d->pair_capacity < 1 || d->pair_capacity > 0x7fffffffLL) return AVATAR_ERR_INVALID_ARG;
    BatchDims m;
    m.G = a.G;
    m.Nv = a.Nv;
    m.K = a.K;
    m.J = a.J;
    m.NL = d->NL;
    m.OW = (d->NL + 31) / 32;
    m.B = d->B;
    m.V = d->V;
    m.VG = (long long)d->V * a.G;
    m.BG = (long long)d->B * a.G;
    m.pixels = 0;
    m.tiles_max = 0;
    for (int v = 0; v < d->V; ++v) {
        const avatar_camera &c = d->views[v].cam;
        if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384) return AVATAR_ERR_INVALID_ARG;
        if (d->views[v].pose < 0 || d->views[v].pose >= d->B) return AVATAR_ERR_INVALID_ARG;
        m.pixels += (long long)c.width * c.height;
        m.tiles_max += (long long)((c.width + 7) / 8) * ((c.height + 7) / 8);
    }
    if (m.VG > 0x7fffffffLL || m.BG * 6 > (1LL << 40) || m.pixels * 3 > 0x7fffffffLL) return AVATAR_ERR_INVALID_ARG;
    m.cap = d->pair_capacity;
    *o = m;
    return AVATAR_OK;
}

avatar_skin_args skin_struct(const avatar_batch_desc *d, const BatchWs &w)
{
    avatar_skin_args s = d->avatar;
    s.pose = d->poses;
    s.bone = w.bone;
    s.xp = w.xp;
    s.xd = w.xd;
    s.cov = w.cov;
    s.nd = w.nd;
    s.ag = w.ag;
    s.rg = w.rg;
    s.pg = w.pg;
    s.ubar = w.ubar;
    s.status = d->status;
    return s;
}

avatar_vis_args vis_struct(const avatar_batch_desc *d, const BatchWs &w)
{
    avatar_vis_args v = {};
    v.Nv = d->avatar.Nv;
    v.F = d->F;
    v.D = d->D;
    v.R = d->R;
    v.xp = w.xp;
    v.faces = d->faces;
    v.frames = d->frames;
    for (int i = 0; i < 3; ++i) v.center[i] = d->center[i];
    v.half_extent = d->half_extent;
    v.bias = d->bias;
    v.NL = d->NL;
    v.dmap = d->dmap;
    v.bits = w.bits;
    v.status = d->status;
    v.cull_back = d->cull_back;
    return v;
}

avatar_shade_args shade_struct(const avatar_batch_desc *d, const BatchWs &w)
{
    avatar_shade_args s = {};
    s.G = d->avatar.G;
    s.K = d->avatar.K;
    s.NL = d->NL;
    s.Nv = d->avatar.Nv;
    s.xd = w.xd;
    s.nd = w.nd;
    s.ag = w.ag;
    s.rg = w.rg;
    s.pg = w.pg;
    s.ubar = w.ubar;
    s.knn = d->avatar.knn;
    s.bits = w.bits;
    s.light_L = d->light_L;
    s.light_A = d->light_A;
    s.light_w = d->light_w;
    s.color = w.color;
    s.radiance = w.radiance;
    s.cull = w.cull;
    s.status = d->status;
    return s;
}

size_t batch_layout(const avatar_batch_desc *d, const BatchDims &m, void *base, size_t cap, BatchWs *out)
{
    WsCarver c(base, cap);
    BatchWs w;
    const size_t G = m.G, Nv = m.Nv, B = m.B, V = m.V, VG = m.VG, BG = m.BG, K = m.K;
    const size_t P = (size_t)m.cap;
    w.views = c.take<BatchView>(V);
    w.view_pose = c.take<int32_t>(V);
    w.view_cc = c.take<float>(3 * V);
    w.bone = c.take<float>(B * m.J * 12);
    w.xp = c.take<float>(3 * B * Nv);
    w.xd = c.take<float>(3 * BG);
    w.cov = c.take<float>(6 * BG);
    w.nd = c.take<float>(3 * BG);
    w.ag = c.take<float>(3 * G);
    w.rg = c.take<float>(G);
    w.pg = c.take<float>(G);
    w.ubar = c.take<float>(K * G);
    avatar_skin_args sa = d->avatar;
    w.skin_ws_bytes = av_skin_batch_workspace_size(&sa, m.B);
    w.skin_ws = c.take<unsigned char>(w.skin_ws_bytes);
    w.bits = c.take<uint32_t>(B * Nv * m.OW);
    {
        // the size depends on the counts only: stand-in pointers for a size query
        static uint32_t stand_in[4];
        avatar_vis_args va = vis_struct(d, w);
        if (!va.xp) va.xp = reinterpret_cast<const float *>(stand_in);
        if (!va.bits) va.bits = stand_in;
        if (!va.frames) va.frames = reinterpret_cast<const float *>(stand_in);
        if (!va.faces) va.faces = reinterpret_cast<const int32_t *>(stand_in);
        w.vis_ws_bytes = av_visibility_batch_workspace_size(&va, m.B);
    }
    w.vis_ws = c.take<unsigned char>(w.vis_ws_bytes);
    w.color = c.take<float>(3 * VG);
    w.radiance = c.take<float>(3 * VG);
    w.cull = c.take<uint8_t>(VG);
    w.mean2d = c.take<float>(2 * VG);
    w.conic = c.take<float>(3 * VG);
    w.depth = c.take<float>(VG);
    w.rect = c.take<int32_t>(4 * VG);
    w.rec0 = c.take<float4>(VG);
    w.rec1 = c.take<float4>(VG);
    w.rec2 = c.take<float4>(VG);
    w.dkey_a = c.take<uint32_t>(VG);
    w.dkey_b = c.take<uint32_t>(VG);
    w.dval_a = c.take<int32_t>(VG);
    w.dval_b = c.take<int32_t>(VG);
    w.npairs = c.take<int32_t>(VG);
    w.offsets = c.take<int32_t>(VG);
    w.pkey_a = c.take<uint32_t>(P);
    w.pkey_b = c.take<uint32_t>(P);
    w.pval_a = c.take<int32_t>(P);
    w.pval_b = c.take<int32_t>(P);
    w.ranges = c.take<int2>((size_t)m.tiles_max);
    w.T_final = c.take<float>((size_t)m.pixels);
    w.n_last = c.take<int32_t>((size_t)m.pixels);
    w.sort_hist = c.take<int32_t>((size_t)OS_MAX_PASSES * RADIX + OS_MAX_PASSES);
    w.sort_desc = c.take<unsigned>(sort_desc_words(std::max(P, VG)));
    w.block_sums = c.take<int32_t>(1024);
    w.count_vg = c.take<int32_t>(1);
    w.counter = c.take<int32_t>(1);
    w.tune_status = c.take<int32_t>(1);
    w.d_color = c.take<float>(3 * VG);
    w.d_opacity_v = c.take<float>(VG);
    w.d_mean2d = c.take<float>(2 * VG);
    w.d_conic = c.take<float>(3 * VG);
    w.ds_xd = c.take<float>(3 * VG);
    w.ds_nd = c.take<float>(3 * VG);
    w.ds_ag = c.take<float>(3 * VG);
    w.ds_rg = c.take<float>(VG);
    w.ds_pg = c.take<float>(VG);
    w.ds_ubar = c.take<float>(K * VG);
    w.dp_xd = c.take<float>(3 * BG);
    w.dp_cov = c.take<float>(6 * BG);
    w.dp_nd = c.take<float>(3 * BG);
    w.dg_ag = c.take<float>(3 * G);
    w.dg_rg = c.take<float>(G);
    w.dg_pg = c.take<float>(G);
    w.dg_ubar = c.take<float>(K * G);
    w.skin_bwd_ws_bytes = av_skin_batch_backward_workspace_size(&sa, m.B);
    w.skin_bwd_ws = c.take<unsigned char>(w.skin_bwd_ws_bytes);
    if (out) *out = w;
    return c.off;
}

// ---------------------------------------------------------------- (d) kernels
__global__ void __launch_bounds__(256)
project_batch_kernel(const BatchView *__restrict__ views, int G, long long BG, long long VG,
                     const float *__restrict__ xd, const float *__restrict__ cov, const void *opacity, int dtype,
                     const uint8_t *__restrict__ cull, float *mean2d, float *conic, float *depth, int32_t *rect)
{
    const int v = blockIdx.y;
    const CamDev cam = views[v].cam;
    const size_t op = (size_t)views[v].pose * G, ov = (size_t)v * G;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const float o = ld_attr(opacity, g, dtype);
        const Splat2D s = project_gaussian(xd, cov, (size_t)BG, op + g, o, cull[ov + g] != 0, cam);
        store_splat(s, (size_t)VG, ov + g, mean2d, conic, depth, rect);
    }
}

__global__ void __launch_bounds__(256)
bin_keys_batch_kernel(const BatchView *__restrict__ views, int G, long long VG, int TS, const void *opacity,
                      int dtype, const float *__restrict__ mean2d, const float *__restrict__ conic,
                      const float *__restrict__ depth, const int32_t *__restrict__ rect,
                      const float *__restrict__ color, int32_t *npairs, uint32_t *dkey, int32_t *dval, float4 *rec0,
                      float4 *rec1, float4 *rec2, int32_t *count_vg)
{
    const int v = blockIdx.y;
    const int W = views[v].cam.W, H = views[v].cam.H;
    const size_t cs = (size_t)VG;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const size_t i = (size_t)v * G + g;
        int x0 = rect[i], y0 = rect[cs + i], x1 = rect[2 * cs + i], y1 = rect[3 * cs + i];
        int n = rect_tiles(x0, y0, x1, y1, W, H, TS);
        npairs[i] = n;
        dkey[i] = n > 0 ? __float_as_uint(depth[i]) : 0xffffffffu;
        dval[i] = (int32_t)i;
        float o = ld_attr(opacity, g, dtype);
        make_records(mean2d[i], mean2d[cs + i], conic[i], conic[cs + i], conic[2 * cs + i], x0, y0, x1, y1, color[i],
                     color[cs + i], color[2 * cs + i], o, rec0[i], rec1[i], rec2[i]);
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *count_vg = (int32_t)VG;
}

// Pairs (global tile, Gaussian) in depth order; the global tile of view v's
// tile (tx, ty) is tile_base(v) + ty ntx(v) + tx.
__global__ void __launch_bounds__(256)
emit_batch_kernel(const BatchView *__restrict__ views, int G, long long VG, int TS,
                  const int32_t *__restrict__ sorted_idx, const int32_t *__restrict__ offsets,
                  const int32_t *__restrict__ npairs, const int32_t *__restrict__ rect,
                  const float4 *__restrict__ rec0, const float4 *__restrict__ rec1, int rmode, long cap,
                  uint32_t *__restrict__ keys, int32_t *__restrict__ vals)
{
    const size_t cs = (size_t)VG;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long base = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < VG;
         base += warps * 32) {
        const long long k = base + (threadIdx.x & 31);
        int gi = 0, n = 0, tx0 = 0, ty0 = 0, w = 1, kbase = 0, ntx = 1;
        long off = 0;
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
        if (k < VG) {
            gi = sorted_idx[k];
            n = npairs[gi];
            off = offsets[k];
            if (n > 0) {
                const int v = gi / G;
                ntx = views[v].ntx;
                kbase = views[v].tile_base;
                tx0 = rect[gi] / TS;
                ty0 = rect[cs + gi] / TS;
                w = rect[2 * cs + gi] / TS - tx0 + 1;
                r0 = rec0[gi];
                r1 = rec1[gi];
            }
        }
        emit_pairs_warp(n, off, gi, tx0, ty0, w, kbase, ntx, tile_reach_of(r0, r1), TS, rmode, cap, keys, vals);
    }
}

// View of global tile t: the last view whose first tile is <= t.
__device__ __forceinline__ int view_of_tile(const BatchView *__restrict__ views, int V, int t)
{
    int lo = 0, hi = V - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&views[mid].tile_base) <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Persistent blend over every tile of every view.
template <int TS, int PPT>
__global__ void __launch_bounds__(BWD_WARPS * 32)
blend_batch_kernel(const BatchView *__restrict__ views, int V, int T, const int2 *__restrict__ ranges,
                   const int32_t *__restrict__ pairs, const float4 *__restrict__ rec0, const float4 *__restrict__ rec1,
                   const float4 *__restrict__ rec2, const uint32_t *__restrict__ pkeys, int rmode, float *images,
                   float *T_final, int32_t *n_last, int32_t *counter)
{
    // persistent warps take (tile, pixel box) items from the device counter
    constexpr int NB = TS * TS / (32 * PPT);
    __shared__ float4 s0[BWD_WARPS][2][32];
    __shared__ float4 s1[BWD_WARPS][2][32];
    __shared__ float4 s2[BWD_WARPS][2][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int items = T * NB;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(counter, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= items) break;
        const int t = it / NB;
        const int v = view_of_tile(views, V, t);
        const int W = views[v].cam.W, H = views[v].cam.H, ntx = views[v].ntx;
        const int local = t - views[v].tile_base;
        const size_t po = (size_t)views[v].pix_off;
        blend_box<TS, PPT>(ranges[t], pairs, rec0, rec1, rec2, W, H, local % ntx, local / ntx, it % NB, pkeys,
                           rmode, images + 3 * po, T_final + po, n_last + po, s0[warp], s1[warp], s2[warp]);
    }
}

template <int TS, int PPT>
__global__ void __launch_bounds__(BWD_WARPS * 32)
blend_backward_batch_kernel(const BatchView *__restrict__ views, int V, int T, const int2 *__restrict__ ranges,
                            const int32_t *__restrict__ pairs, const float4 *__restrict__ rec0,
                            const float4 *__restrict__ rec1, const float4 *__restrict__ rec2,
                            const uint32_t *__restrict__ pkeys, int rmode,
                            const float *__restrict__ T_final, const int32_t *__restrict__ n_last,
                            const float *__restrict__ d_images, long long VG, float *d_mean2d, float *d_conic,
                            float *d_opacity, float *d_color, int32_t *counter)
{
    // persistent warps take (tile, pixel box) items from the device counter
    constexpr int NB = TS * TS / (32 * PPT);
    __shared__ float4 s0[BWD_WARPS][2][32];
    __shared__ float4 s1[BWD_WARPS][2][32];
    __shared__ float4 s2[BWD_WARPS][2][32];
    __shared__ int sg[BWD_WARPS][2][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int items = T * NB;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(counter, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= items) break;
        const int t = it / NB;
        const int v = view_of_tile(views, V, t);
        const int W = views[v].cam.W, H = views[v].cam.H, ntx = views[v].ntx;
        const int local = t - views[v].tile_base;
        const size_t po = (size_t)views[v].pix_off;
        blend_backward_box<TS, PPT>(ranges[t], pairs, rec0, rec1, rec2, W, H, local % ntx, local / ntx, it % NB,
                                    pkeys, rmode, T_final + po, n_last + po, d_images + 3 * po, (size_t)VG,
                                    d_mean2d, d_conic, d_opacity, d_color, s0[warp], s1[warp], s2[warp], sg[warp]);
    }
}

// Per Gaussian, over every view: projection adjoint of the view's splat
// gradients plus the view's shading gradients, summed into the view's pose
// (position, covariance, normal) and over all views (albedo, roughness,
// tint, Eq. 1 weights, opacity).
struct ReduceArgs {
    const BatchView *views;
    int G, K, V;
    long long VG, BG;
    const float *xd, *cov;               // per pose
    const int32_t *rect;                 // per view
    const float *d_mean2d, *d_conic;     // per view
    const float *ds_xd, *ds_nd, *ds_ag, *ds_rg, *ds_pg, *ds_ubar, *d_opacity_v;
    float *dp_xd, *dp_cov, *dp_nd;       // per pose (accumulated with +=; zeroed before)
    float *dg_ag, *dg_rg, *dg_pg, *dg_ubar, *d_opacity;
};

__global__ void __launch_bounds__(256)
batch_grad_reduce_kernel(ReduceArgs r)
{
    const size_t vs = (size_t)r.VG, bs = (size_t)r.BG;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < r.G; g += gridDim.x * blockDim.x) {
        float sag[3] = {0.f, 0.f, 0.f}, srg = 0.f, spg = 0.f, sop = 0.f, sub[MAX_K];
#pragma unroll
        for (int j = 0; j < MAX_K; ++j) sub[j] = 0.f;
        float px[3] = {0.f, 0.f, 0.f}, pc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, pn[3] = {0.f, 0.f, 0.f};
        int cur = -1;
        auto flush = [&](int p) {
            const size_t i = (size_t)p * r.G + g;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                r.dp_xd[c * bs + i] += px[c];
                r.dp_nd[c * bs + i] += pn[c];
                px[c] = pn[c] = 0.f;
            }
#pragma unroll
            for (int e = 0; e < 6; ++e) {
                r.dp_cov[e * bs + i] += pc[e];
                pc[e] = 0.f;
            }
        };
        for (int v = 0; v < r.V; ++v) {
            const int p = __ldg(&r.views[v].pose);
            if (p != cur) {
                if (cur >= 0) flush(cur);
                cur = p;
            }
            const size_t i = (size_t)v * r.G + g;
            // splatting: projection adjoint in view v's camera
            const float dmx = r.d_mean2d[i], dmy = r.d_mean2d[vs + i];
            const float da = r.d_conic[i], db = r.d_conic[vs + i], dc = r.d_conic[2 * vs + i];
            if (r.rect[2 * vs + i] >= r.rect[i] && !(dmx == 0.f && dmy == 0.f && da == 0.f && db == 0.f && dc == 0.f)) {
                const CamDev cam = r.views[v].cam;
                float gx[3], gc[6];
                project_adjoint(r.xd, r.cov, bs, (size_t)p * r.G + g, cam, dmx, dmy, da, db, dc, gx, gc);
#pragma unroll
                for (int c = 0; c < 3; ++c) px[c] += gx[c];
#pragma unroll
                for (int e = 0; e < 6; ++e) pc[e] += gc[e];
            }
            // shading
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                px[c] += r.ds_xd[c * vs + i];
                pn[c] += r.ds_nd[c * vs + i];
                sag[c] += r.ds_ag[c * vs + i];
            }
            srg += r.ds_rg[i];
            spg += r.ds_pg[i];
            sop += r.d_opacity_v[i];
            for (int j = 0; j < r.K; ++j) sub[j] += r.ds_ubar[j * vs + i];
        }
        if (cur >= 0) flush(cur);
#pragma unroll
        for (int c = 0; c < 3; ++c) r.dg_ag[(size_t)c * r.G + g] = sag[c];
        r.dg_rg[g] = srg;
        r.dg_pg[g] = spg;
        r.d_opacity[g] = sop;
        for (int j = 0; j < r.K; ++j) r.dg_ubar[(size_t)j * r.G + g] = sub[j];
    }
}

// ---------------------------------------------------------------- host
int grid_cap(const avatar_ctx *ctx, long long n, int threads, int per_sm)
{
    long long b = (n + threads - 1) / threads;
    long long cap = (long long)ctx->sm_count * per_sm;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

int tile_of(const avatar_ctx *ctx, const avatar_batch_desc *d)
{
    int t = d->tile ? d->tile : ctx->tune[AVATAR_TUNE_BATCH_TILE];
    return (t == 8 || t == 32) ? t : 16;
}

// Host view table for tile edge TS; returns the total tile count.
long long view_table(const avatar_batch_desc *d, int TS, std::vector<BatchView> &tab)
{
    tab.resize(d->V);
    long long tiles = 0, pix = 0;
    for (int v = 0; v < d->V; ++v) {
        const avatar_camera &c = d->views[v].cam;
        BatchView &b = tab[v];
        b.cam = to_dev(c);
        for (int i = 0; i < 3; ++i) b.cc[i] = d->views[v].center[i];
        b.pose = d->views[v].pose;
        b.ntx = (c.width + TS - 1) / TS;
        b.tile_base = (int)tiles;
        b.pix_off = (int)pix;
        tiles += (long long)b.ntx * ((c.height + TS - 1) / TS);
        pix += (long long)c.width * c.height;
    }
    return tiles;
}

int prep(avatar_ctx *ctx, const avatar_batch_desc *d, void *ws, size_t ws_bytes, BatchDims *m, BatchWs *w)
{
    if (!ctx) return AVATAR_ERR_INVALID_ARG;
    AV_TRY(batch_dims(d, m));
    if (!d->poses || !d->light_L || !d->light_A || !d->light_w || !d->dmap || !d->opacity || !d->images ||
        !d->num_pairs || !d->frames || (d->F > 0 && !d->faces))
        return AVATAR_ERR_INVALID_ARG;
    if (d->avatar.attr_dtype != AVATAR_DTYPE_F32 && d->avatar.attr_dtype != AVATAR_DTYPE_BF16)
        return AVATAR_ERR_INVALID_ARG;
    if (!ws || (((uintptr_t)ws) & 255)) return AVATAR_ERR_WORKSPACE;
    if (batch_layout(d, *m, ws, ws_bytes, w) > ws_bytes) return AVATAR_ERR_WORKSPACE;
    if (w->skin_ws_bytes == 0 || w->vis_ws_bytes == 0) return AVATAR_ERR_INVALID_ARG;
    return AVATAR_OK;
}

bool masks_on(const avatar_ctx *ctx) { return ctx->tune[AVATAR_TUNE_REGION_MASKS] != 0; }
int masks_mode(const avatar_ctx *ctx, long T, int TS) { return region_mode(T, TS, masks_on(ctx)); }

template <int TS, int PPT>
int launch_blend_batch(const avatar_ctx *ctx, const avatar_batch_desc *d, const BatchWs &w, int T, cudaStream_t st)
{
    auto kern = blend_batch_kernel<TS, PPT>;
    constexpr int NB = TS * TS / (32 * PPT);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BWD_WARPS * 32, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long wblocks = ((long long)std::max(T, 1) * NB + BWD_WARPS - 1) / BWD_WARPS;
    const int grid = (int)std::min<long long>((long long)ctx->sm_count * per_sm, wblocks);
    kern<<<grid, BWD_WARPS * 32, 0, st>>>(w.views, d->V, T, w.ranges, w.pval_a, w.rec0, w.rec1, w.rec2, w.pkey_a,
                                         masks_mode(ctx, T, TS), d->images, w.T_final, w.n_last, w.counter);
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}

template <int TS, int PPT>
int launch_blend_bwd_batch(const avatar_ctx *ctx, const avatar_batch_desc *d, const avatar_batch_grads *g,
                           const BatchWs &w, const BatchDims &m, int T, cudaStream_t st)
{
    auto kern = blend_backward_batch_kernel<TS, PPT>;
    constexpr int NB = TS * TS / (32 * PPT);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BWD_WARPS * 32, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long wblocks = ((long long)std::max(T, 1) * NB + BWD_WARPS - 1) / BWD_WARPS;
    const int grid = (int)std::min<long long>((long long)ctx->sm_count * per_sm, wblocks);
    kern<<<grid, BWD_WARPS * 32, 0, st>>>(w.views, d->V, T, w.ranges, w.pval_a, w.rec0, w.rec1, w.rec2, w.pkey_a,
                                         masks_mode(ctx, T, TS), w.T_final, w.n_last, g->d_images, m.VG, w.d_mean2d,
                                         w.d_conic, w.d_opacity_v, w.d_color, w.counter);
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}

int blend_dispatch(const avatar_ctx *ctx, const avatar_batch_desc *d, const BatchWs &w, int TS, int ppt, int T,
                   cudaStream_t st)
{
    switch (TS) {
        case 8: return ppt >= 2 ? launch_blend_batch<8, 2>(ctx, d, w, T, st) : launch_blend_batch<8, 1>(ctx, d, w, T, st);
        case 32:
            return ppt == 4 ? launch_blend_batch<32, 4>(ctx, d, w, T, st)
                   : ppt == 2 ? launch_blend_batch<32, 2>(ctx, d, w, T, st)
                              : launch_blend_batch<32, 1>(ctx, d, w, T, st);
        default:
            return ppt == 4 ? launch_blend_batch<16, 4>(ctx, d, w, T, st)
                   : ppt == 2 ? launch_blend_batch<16, 2>(ctx, d, w, T, st)
                              : launch_blend_batch<16, 1>(ctx, d, w, T, st);
    }
}

int blend_bwd_dispatch(const avatar_ctx *ctx, const avatar_batch_desc *d, const avatar_batch_grads *g,
                       const BatchWs &w, const BatchDims &m, int TS, int ppt, int T, cudaStream_t st)
{
    switch (TS) {
        case 8:
            return ppt >= 2 ? launch_blend_bwd_batch<8, 2>(ctx, d, g, w, m, T, st)
                            : launch_blend_bwd_batch<8, 1>(ctx, d, g, w, m, T, st);
        case 32:
            return ppt == 4 ? launch_blend_bwd_batch<32, 4>(ctx, d, g, w, m, T, st)
                   : ppt == 2 ? launch_blend_bwd_batch<32, 2>(ctx, d, g, w, m, T, st)
                              : launch_blend_bwd_batch<32, 1>(ctx, d, g, w, m, T, st);
        default:
            return ppt == 4 ? launch_blend_bwd_batch<16, 4>(ctx, d, g, w, m, T, st)
                   : ppt == 2 ? launch_blend_bwd_batch<16, 2>(ctx, d, g, w, m, T, st)
                              : launch_blend_bwd_batch<16, 1>(ctx, d, g, w, m, T, st);
    }
}

// Forward with an explicit tile edge and blend split.
int render_batch(avatar_ctx *ctx, const avatar_batch_desc *d, void *ws, size_t ws_bytes, int TS, int ppt,
                 cudaStream_t st)
{
    BatchDims m;
    BatchWs w;
    AV_TRY(prep(ctx, d, ws, ws_bytes, &m, &w));
    std::vector<BatchView> tab;
    const long long T = view_table(d, TS, tab);
    if (T > 0x7fffffffLL) return AVATAR_ERR_INVALID_ARG;
    for (int first = 0; first < d->V; first += SETUP_CHUNK) {
        SetupChunk c;
        c.first = first;
        c.n = std::min(SETUP_CHUNK, d->V - first);
        for (int i = 0; i < c.n; ++i) c.v[i] = tab[first + i];
        batch_setup_kernel<<<1, SETUP_CHUNK, 0, st>>>(c, w.views, w.view_pose, w.view_cc);
    }
    AV_CHECK_LAUNCH();
    // (a) skinning of every pose
    avatar_skin_args sa = skin_struct(d, w);
    AV_TRY(av_skin_batch(ctx, &sa, m.B, w.skin_ws, w.skin_ws_bytes, st));
    // (b) visibility of every pose
    avatar_vis_args va = vis_struct(d, w);
    AV_TRY(av_visibility_batch(ctx, &va, m.B, w.vis_ws, w.vis_ws_bytes, st));
    // (c) shading of every view
    avatar_shade_args ha = shade_struct(d, w);
    AV_TRY(av_shade_batch(ctx, &ha, m.B, m.V, w.view_pose, w.view_cc, st));
    // (d) projection of every view
    project_batch_kernel<<<dim3(grid_cap(ctx, m.G, 256, 8), m.V), 256, 0, st>>>(
        w.views, m.G, m.BG, m.VG, w.xd, w.cov, d->opacity, d->avatar.attr_dtype, w.cull, w.mean2d, w.conic, w.depth,
        w.rect);
    AV_CHECK_LAUNCH();
    // binning over all views
    if (cudaMemsetAsync(w.ranges, 0, (size_t)T * sizeof(int2), st) != cudaSuccess) return AVATAR_ERR_CUDA;
    bin_keys_batch_kernel<<<dim3(grid_cap(ctx, m.G, 256, 8), m.V), 256, 0, st>>>(
        w.views, m.G, m.VG, TS, d->opacity, d->avatar.attr_dtype, w.mean2d, w.conic, w.depth, w.rect, w.color,
        w.npairs, w.dkey_a, w.dval_a, w.rec0, w.rec1, w.rec2, w.count_vg);
    AV_CHECK_LAUNCH();
    const SortWs sw{w.sort_hist, w.sort_desc};
    const int VGi = (int)m.VG;
    AV_TRY(radix_sort(w.dkey_a, w.dval_a, w.dkey_b, w.dval_b, 32, w.count_vg, VGi, sw, d->status, st, sort_spin_limit(ctx)));
    const int NB = std::min(1024, std::max(1, (VGi + 8191) / 8192));
    pair_scan_reduce_kernel<<<NB, 1024, 0, st>>>(w.dval_a, w.npairs, VGi, NB, w.block_sums);
    pair_scan_down_kernel<<<NB, 1024, 0, st>>>(w.dval_a, w.npairs, VGi, NB, w.block_sums, w.offsets, d->num_pairs,
                                               (long)m.cap, d->status);
    AV_CHECK_LAUNCH();
    const int tbits = bits_for(T);
    const int passes = tbits <= 8 ? 1 : (tbits + 7) / 8;
    if (passes > OS_MAX_PASSES) return AVATAR_ERR_INVALID_ARG;
    uint32_t *k_emit = (passes % 2 == 0) ? w.pkey_a : w.pkey_b;
    int32_t *v_emit = (passes % 2 == 0) ? w.pval_a : w.pval_b;
    uint32_t *k_other = (passes % 2 == 0) ? w.pkey_b : w.pkey_a;
    int32_t *v_other = (passes % 2 == 0) ? w.pval_b : w.pval_a;
    emit_batch_kernel<<<grid_cap(ctx, m.VG, 256, 8), 256, 0, st>>>(w.views, m.G, m.VG, TS, w.dval_a, w.offsets,
                                                                    w.npairs, w.rect, w.rec0, w.rec1,
                                                                    masks_mode(ctx, T, TS), (long)m.cap, k_emit,
                                                                    v_emit);
    AV_CHECK_LAUNCH();
    AV_TRY(radix_sort(k_emit, v_emit, k_other, v_other, passes * 8, d->num_pairs, (int)m.cap, sw, d->status, st, sort_spin_limit(ctx)));
    tile_ranges_kernel<<<ctx->sm_count * 8, 256, 0, st>>>(w.pkey_a, d->num_pairs, (long)m.cap, (int)T,
                                                          tile_key_mask(T, TS, masks_on(ctx)), w.ranges);
    AV_CHECK_LAUNCH();
    // persistent blend over every view's tiles
    if (cudaMemsetAsync(w.counter, 0, sizeof(int32_t), st) != cudaSuccess) return AVATAR_ERR_CUDA;
    return blend_dispatch(ctx, d, w, TS, ppt, (int)T, st);
}

int render_batch_backward(avatar_ctx *ctx, const avatar_batch_desc *d, const avatar_batch_grads *g, void *ws,
                          size_t ws_bytes, int TS, int bppt, cudaStream_t st)
{
    BatchDims m;
    BatchWs w;
    AV_TRY(prep(ctx, d, ws, ws_bytes, &m, &w));
    if (!g || !g->d_images || !g->d_xg || !g->d_logscale || !g->d_quat || !g->d_opacity || !g->d_wv || !g->d_av ||
        !g->d_rv || !g->d_pv || !g->d_light_L)
        return AVATAR_ERR_INVALID_ARG;
    std::vector<BatchView> tab;
    const long long T = view_table(d, TS, tab);
    const size_t VG = m.VG, BG = m.BG;
    // splatting adjoint over every view's tiles
    if (cudaMemsetAsync(w.d_color, 0, 3 * VG * sizeof(float), st) != cudaSuccess ||
        cudaMemsetAsync(w.d_opacity_v, 0, VG * sizeof(float), st) != cudaSuccess ||
        cudaMemsetAsync(w.d_mean2d, 0, 2 * VG * sizeof(float), st) != cudaSuccess ||
        cudaMemsetAsync(w.d_conic, 0, 3 * VG * sizeof(float), st) != cudaSuccess ||
        cudaMemsetAsync(w.counter, 0, sizeof(int32_t), st) != cudaSuccess)
        return AVATAR_ERR_CUDA;
    AV_TRY(blend_bwd_dispatch(ctx, d, g, w, m, TS, bppt, (int)T, st));
    // shading adjoint of every view
    avatar_shade_args ha = shade_struct(d, w);
    avatar_shade_grads hg = {};
    hg.d_color = w.d_color;
    hg.d_xd = w.ds_xd;
    hg.d_nd = w.ds_nd;
    hg.d_ag = w.ds_ag;
    hg.d_rg = w.ds_rg;
    hg.d_pg = w.ds_pg;
    hg.d_ubar = w.ds_ubar;
    hg.d_light_L = g->d_light_L;
    AV_TRY(av_shade_batch_backward(ctx, &ha, &hg, m.B, m.V, w.view_pose, w.view_cc, st));
    // projection adjoint and the sums over views
    if (cudaMemsetAsync(w.dp_xd, 0, 3 * BG * sizeof(float), st) != cudaSuccess ||
        cudaMemsetAsync(w.dp_cov, 0, 6 * BG * sizeof(float), st) != cudaSuccess ||
        cudaMemsetAsync(w.dp_nd, 0, 3 * BG * sizeof(float), st) != cudaSuccess)
        return AVATAR_ERR_CUDA;
    ReduceArgs r;
    r.views = w.views;
    r.G = m.G;
    r.K = m.K;
    r.V = m.V;
    r.VG = m.VG;
    r.BG = m.BG;
    r.xd = w.xd;
    r.cov = w.cov;
    r.rect = w.rect;
    r.d_mean2d = w.d_mean2d;
    r.d_conic = w.d_conic;
    r.ds_xd = w.ds_xd;
    r.ds_nd = w.ds_nd;
    r.ds_ag = w.ds_ag;
    r.ds_rg = w.ds_rg;
    r.ds_pg = w.ds_pg;
    r.ds_ubar = w.ds_ubar;
    r.d_opacity_v = w.d_opacity_v;
    r.dp_xd = w.dp_xd;
    r.dp_cov = w.dp_cov;
    r.dp_nd = w.dp_nd;
    r.dg_ag = w.dg_ag;
    r.dg_rg = w.dg_rg;
    r.dg_pg = w.dg_pg;
    r.dg_ubar = w.dg_ubar;
    r.d_opacity = g->d_opacity;
    batch_grad_reduce_kernel<<<grid_cap(ctx, m.G, 256, 8), 256, 0, st>>>(r);
    AV_CHECK_LAUNCH();
    // skinning adjoint over the poses
    avatar_skin_args sa = skin_struct(d, w);
    avatar_skin_grads kg = {};
    kg.d_xd = w.dp_xd;
    kg.d_cov = w.dp_cov;
    kg.d_nd = w.dp_nd;
    kg.d_ag = w.dg_ag;
    kg.d_rg = w.dg_rg;
    kg.d_pg = w.dg_pg;
    kg.d_ubar = w.dg_ubar;
    kg.d_xg = g->d_xg;
    kg.d_logscale = g->d_logscale;
    kg.d_quat = g->d_quat;
    kg.d_wv = g->d_wv;
    kg.d_av = g->d_av;
    kg.d_rv = g->d_rv;
    kg.d_pv = g->d_pv;
    return av_skin_batch_backward(ctx, &sa, &kg, m.B, w.skin_ws, w.skin_bwd_ws, w.skin_bwd_ws_bytes, st);
}

int clamp_ppt(int TS, int ppt) { return TS == 8 ? std::min(ppt, 2) : ppt; }

}  // namespace

extern "C" size_t avatar_render_batch_workspace_size(const avatar_batch_desc *d)
{
    BatchDims m;
    if (batch_dims(d, &m) != AVATAR_OK) return 0;
    return batch_layout(d, m, nullptr, 0, nullptr);
}

extern "C" int avatar_render_batch(avatar_ctx *ctx, const avatar_batch_desc *d, void *ws, size_t ws_bytes,
                                   avatar_stream_t stream)
{
    if (!ctx || !d) return AVATAR_ERR_INVALID_ARG;
    const int TS = tile_of(ctx, d);
    return render_batch(ctx, d, ws, ws_bytes, TS, clamp_ppt(TS, ctx->tune[AVATAR_TUNE_BLEND_PPT]),
                        (cudaStream_t)stream);
}

extern "C" int avatar_render_batch_backward(avatar_ctx *ctx, const avatar_batch_desc *d, const avatar_batch_grads *g,
                                            void *ws, size_t ws_bytes, avatar_stream_t stream)
{
    if (!ctx || !d) return AVATAR_ERR_INVALID_ARG;
    const int TS = tile_of(ctx, d);
    return render_batch_backward(ctx, d, g, ws, ws_bytes, TS, clamp_ppt(TS, ctx->tune[AVATAR_TUNE_BLEND_BWD_PPT]),
                                 (cudaStream_t)stream);
}

namespace {

// Median time (ms) of `reps` runs of fn on the stream, after one warm-up
// run; a negative value when a run fails or reports a device error.
template <class F>
float time_runs(F fn, cudaStream_t st, int32_t *dev_status, int reps)
{
    if (cudaMemsetAsync(dev_status, 0, sizeof(int32_t), st) != cudaSuccess) return -1.f;
    if (fn() != AVATAR_OK) return -1.f;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1.f;
    }
    std::vector<float> t;
    bool ok = true;
    for (int r = 0; r < reps && ok; ++r) {
        cudaEventRecord(e0, st);
        ok = fn() == AVATAR_OK;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        t.push_back(ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int32_t host_status = 0;
    if (cudaMemcpyAsync(&host_status, dev_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return -1.f;
    if (!ok || host_status != 0 || t.empty()) return -1.f;
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

}  // namespace

extern "C" int avatar_render_batch_autotune(avatar_ctx *ctx, const avatar_batch_desc *d, const avatar_batch_grads *g,
                                            void *ws, size_t ws_bytes, avatar_stream_t stream, int *tuned)
{
    if (!ctx || !d) return AVATAR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return AVATAR_ERR_INVALID_ARG;
    BatchDims m;
    BatchWs w;
    AV_TRY(prep(ctx, d, ws, ws_bytes, &m, &w));
    // candidates run with a private status word, so an overflow in one of
    // them does not reach the caller's
    avatar_batch_desc dd = *d;
    dd.status = w.tune_status;
    const int reps = 3;
    int best_ts = 0, best_ppt = 1, best_bppt = 2;
    float best = -1.f;
    const int tiles[3] = {16, 8, 32};
    for (int ts : tiles) {
        const int ppt = clamp_ppt(ts, ctx->tune[AVATAR_TUNE_BLEND_PPT]);
        const int bppt = clamp_ppt(ts, ctx->tune[AVATAR_TUNE_BLEND_BWD_PPT]);
        float ms = time_runs(
            [&]() {
                int rc = render_batch(ctx, &dd, ws, ws_bytes, ts, ppt, st);
                if (rc == AVATAR_OK && g) rc = render_batch_backward(ctx, &dd, g, ws, ws_bytes, ts, bppt, st);
                return rc;
            },
            st, w.tune_status, reps);
        if (ms > 0.f && (best < 0.f || ms < best)) {
            best = ms;
            best_ts = ts;
        }
    }
    if (best_ts == 0) return AVATAR_ERR_OVERFLOW;  // no tile edge fits pair_capacity
    // work split of the blend (and its adjoint) at the chosen tile edge
    best = -1.f;
    const int ppts[3] = {1, 2, 4};
    for (int ppt : ppts) {
        if (ppt != clamp_ppt(best_ts, ppt)) continue;
        float ms = time_runs([&]() { return render_batch(ctx, &dd, ws, ws_bytes, best_ts, ppt, st); }, st,
                             w.tune_status, reps);
        if (ms > 0.f && (best < 0.f || ms < best)) {
            best = ms;
            best_ppt = ppt;
        }
    }
    if (g) {
        AV_TRY(render_batch(ctx, &dd, ws, ws_bytes, best_ts, best_ppt, st));
        best = -1.f;
        for (int ppt : ppts) {
            if (ppt != clamp_ppt(best_ts, ppt)) continue;
            float ms = time_runs([&]() { return render_batch_backward(ctx, &dd, g, ws, ws_bytes, best_ts, ppt, st); },
                                 st, w.tune_status, reps);
            if (ms > 0.f && (best < 0.f || ms < best)) {
                best = ms;
                best_bppt = ppt;
            }
        }
    } else {
        best_bppt = ctx->tune[AVATAR_TUNE_BLEND_BWD_PPT];
    }
    ctx->tune[AVATAR_TUNE_BATCH_TILE] = best_ts;
    ctx->tune[AVATAR_TUNE_BLEND_PPT] = best_ppt;
    ctx->tune[AVATAR_TUNE_BLEND_BWD_PPT] = best_bppt;
    if (tuned) {
        tuned[0] = best_ts;
        tuned[1] = best_ppt;
        tuned[2] = best_bppt;
    }
    return AVATAR_OK;
}
