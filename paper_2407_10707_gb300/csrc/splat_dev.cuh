// Device code of the splatting stage (d) shared by the single-view entry
// points (splat.cu) and the batched launch over many views (batch.cu):
// EWA projection and its adjoint, blend records, the stable onesweep radix
// sort, the pair scan, tile ranges, and the per-tile blend and its adjoint.
//
// Arrays of per-Gaussian values are structure-of-arrays with an explicit
// channel stride ("cs"): a single view uses cs = G, a batch concatenates the
// views' Gaussians (index v * G + g) and uses cs = V * G.
#pragma once

#include "common.cuh"

namespace {

constexpr int RADIX = 256;
constexpr float NEAR_Z = 0.2f;
constexpr float ALPHA_MIN = 1.0f / 255.0f;
constexpr float T_MIN = 1e-4f;
constexpr float LOG2_ALPHA_MIN = -7.99435343685886f;  // log2(1/255)
constexpr float L2E = 1.4426950408889634f;            // log2(e)

struct CamDev {
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    int W, H;
};

inline CamDev to_dev(const avatar_camera &c)
{
    CamDev d;
    d.fx = c.fx;
    d.fy = c.fy;
    d.cx = c.cx;
    d.cy = c.cy;
    for (int i = 0; i < 9; ++i) d.R[i] = c.R[i];
    for (int i = 0; i < 3; ++i) d.t[i] = c.t[i];
    d.W = c.width;
    d.H = c.height;
    return d;
}

// ---------------------------------------------------------------- projection
struct Splat2D {
    float u, v, ca, cb, cc, z;
    int x0, y0, x1, y1;  // inclusive pixel rect; x0 > x1 when empty
};

// EWA projection of Gaussian i of (xd [3][cs], cov [6][cs]) with opacity o:
// mean, conic of Sigma' = T Sigma T^T + 0.3 I (T = J R), view depth, and the
// pixel rect of the ellipse q <= 2 ln(255 o) padded by one pixel.
__device__ __forceinline__ Splat2D project_gaussian(const float *__restrict__ xd, const float *__restrict__ cov,
                                                    size_t cs, size_t i, float o, bool culled, const CamDev &cam)
{
    Splat2D s;
    float x = xd[i], y = xd[cs + i], z = xd[2 * cs + i];
    float px = cam.R[0] * x + cam.R[1] * y + cam.R[2] * z + cam.t[0];
    float py = cam.R[3] * x + cam.R[4] * y + cam.R[5] * z + cam.t[1];
    float pz = cam.R[6] * x + cam.R[7] * y + cam.R[8] * z + cam.t[2];
    bool ok = !culled && pz > NEAR_Z && o > ALPHA_MIN;
    float u = 0.f, v = 0.f, ca = 0.f, cb = 0.f, cc = 0.f;
    int x0 = 0, y0 = 0, x1 = -1, y1 = -1;
    if (ok) {
        float iz = 1.0f / pz;
        u = cam.fx * px * iz + cam.cx;
        v = cam.fy * py * iz + cam.cy;
        float j00 = cam.fx * iz, j02 = -cam.fx * px * iz * iz;
        float j11 = cam.fy * iz, j12 = -cam.fy * py * iz * iz;
        float T0[3], T1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T0[k] = j00 * cam.R[k] + j02 * cam.R[6 + k];
            T1[k] = j11 * cam.R[3 + k] + j12 * cam.R[6 + k];
        }
        float c0 = cov[i], c1 = cov[cs + i], c2 = cov[2 * cs + i];
        float c3 = cov[3 * cs + i], c4 = cov[4 * cs + i], c5 = cov[5 * cs + i];
        float S0[3] = {c0 * T0[0] + c1 * T0[1] + c2 * T0[2], c1 * T0[0] + c3 * T0[1] + c4 * T0[2],
                       c2 * T0[0] + c4 * T0[1] + c5 * T0[2]};
        float S1[3] = {c0 * T1[0] + c1 * T1[1] + c2 * T1[2], c1 * T1[0] + c3 * T1[1] + c4 * T1[2],
                       c2 * T1[0] + c4 * T1[1] + c5 * T1[2]};
        float s00 = T0[0] * S0[0] + T0[1] * S0[1] + T0[2] * S0[2] + 0.3f;
        float s01 = T1[0] * S0[0] + T1[1] * S0[1] + T1[2] * S0[2];
        float s11 = T1[0] * S1[0] + T1[1] * S1[1] + T1[2] * S1[2] + 0.3f;
        float det = s00 * s11 - s01 * s01;
        if (det > 0.f) {
            float id = 1.0f / det;
            ca = s11 * id;
            cb = -s01 * id;
            cc = s00 * id;
            float r2 = 2.0f * logf(255.0f * o);
            float ex = sqrtf(r2 * s00) + 1.0f, ey = sqrtf(r2 * s11) + 1.0f;
            float fx0 = ceilf(u - ex - 0.5f), fx1 = floorf(u + ex - 0.5f);
            float fy0 = ceilf(v - ey - 0.5f), fy1 = floorf(v + ey - 0.5f);
            fx0 = fmaxf(fx0, 0.f);
            fy0 = fmaxf(fy0, 0.f);
            fx1 = fminf(fx1, (float)(cam.W - 1));
            fy1 = fminf(fy1, (float)(cam.H - 1));
            if (fx0 <= fx1 && fy0 <= fy1) {
                x0 = (int)fx0;
                x1 = (int)fx1;
                y0 = (int)fy0;
                y1 = (int)fy1;
            }
        } else {
            ok = false;
        }
    }
    if (!ok) {
        u = v = ca = cb = cc = 0.f;
        x0 = y0 = 0;
        x1 = y1 = -1;
    }
    s.u = u;
    s.v = v;
    s.ca = ca;
    s.cb = cb;
    s.cc = cc;
    s.z = pz;
    s.x0 = x0;
    s.y0 = y0;
    s.x1 = x1;
    s.y1 = y1;
    return s;
}

// Writes a projection into the caller-visible buffers (mean2d [2][cs],
// conic [3][cs], depth [cs], rect [4][cs]) at index i.
__device__ __forceinline__ void store_splat(const Splat2D &s, size_t cs, size_t i, float *mean2d, float *conic,
                                            float *depth, int32_t *rect)
{
    mean2d[i] = s.u;
    mean2d[cs + i] = s.v;
    conic[i] = s.ca;
    conic[cs + i] = s.cb;
    conic[2 * cs + i] = s.cc;
    depth[i] = s.z;
    rect[i] = s.x0;
    rect[cs + i] = s.y0;
    rect[2 * cs + i] = s.x1;
    rect[3 * cs + i] = s.y1;
}

// Tiles of edge TS that the rect touches (0 for an empty or out-of-image rect).
__device__ __forceinline__ int rect_tiles(int x0, int y0, int x1, int y1, int W, int H, int TS)
{
    if (x0 <= x1 && y0 <= y1 && x0 >= 0 && y0 >= 0 && x1 < W && y1 < H)
        return (x1 / TS - x0 / TS + 1) * (y1 / TS - y0 / TS + 1);
    return 0;
}

// Blend records of one Gaussian.  The conic is held in log2 units,
//   log2(alpha_raw) = qa dx^2 + qb dx dy + qc dy^2 + log2 o
// with qa = -a/2 log2(e), qb = -b log2(e), qc = -c/2 log2(e), so that a pixel
// rejects a Gaussian (alpha < 1/255) with a few FMAs and no exponential.
__device__ __forceinline__ void make_records(float mx, float my, float ca, float cb, float cc, int x0, int y0,
                                             int x1, int y1, float r, float g, float b, float o, float4 &rec0,
                                             float4 &rec1, float4 &rec2)
{
    rec0 = make_float4(mx, my, -0.5f * L2E * ca, -L2E * cb);
    rec1 = make_float4(-0.5f * L2E * cc, o > 0.f ? log2f(o) : -1e30f, __int_as_float((x0 & 0xffff) | (y0 << 16)),
                       __int_as_float((x1 & 0xffff) | (y1 << 16)));
    rec2 = make_float4(r, g, b, o);
}

// The set a Gaussian can reach in the blend, from its blend records: the
// pixel centres d = p - mean with qa dx^2 + qb dx dy + qc dy^2 + log2 o >=
// log2(1/255), i.e. the ellipse A dx^2 + 2 Bh dx dy + C dy^2 <= R with
// A = -qa, Bh = -qb / 2, C = -qc, R = log2 o - log2(1/255).  Held as what
// the tile test needs: the centre, 1/A, Bh, det = A C - Bh^2, A R, the
// ellipse's half height ey and dyR, the height of its rightmost point.  A
// Gaussian whose ellipse is degenerate (or not finite) keeps every tile of
// its rect: AR = 3e38 makes the test pass.
struct TileReach {
    float u, v, iA, Bh, det, AR, ey, dyR;
};

__device__ __forceinline__ TileReach tile_reach_of(float4 r0, float4 r1)
{
    TileReach t;
    t.u = r0.x;
    t.v = r0.y;
    const float A = -r0.z, Bh = -0.5f * r0.w, C = -r1.x, R = r1.y - LOG2_ALPHA_MIN;
    const float det = A * C - Bh * Bh;
    if (A > 0.f && C > 0.f && R > 0.f && det > 1e-6f * A * C && det < 3e38f && R < 3e38f) {
        const float ex = sqrtf(R * C / det);
        t.ey = sqrtf(R * A / det);
        t.dyR = -Bh * ex / C;
        t.iA = 1.f / A;
        t.Bh = Bh;
        t.det = det;
        t.AR = A * R;
    } else {
        t.ey = 3e38f;
        t.dyR = 0.f;
        t.iA = 1.f;
        t.Bh = 0.f;
        t.det = 0.f;
        t.AR = 3e38f;
    }
    return t;
}

// The regions of a tile that a Gaussian's ellipse comes within one pixel
// of: the tile split into C columns x 4 rows of (TS / C) x (TS / 4) pixels,
// bit C ry + rx.  Per row band (padded by one pixel, clipped to the
// ellipse's height) the ellipse's x range [xl, xr]: the right boundary
// dx = (-Bh dy + sqrt(AR - det dy^2)) / A is concave in dy, so its maximum
// over the band is at dyR clamped into it (the left boundary's minimum at
// -dyR likewise); a column is reached where that range meets it, padded by
// one pixel.  The padding keeps the test conservative by 1.5 pixels beyond
// every pixel centre of a region, far above the FP32 rounding of either
// side.  Pair keys carry the mask above the tile id: region mode 2 (tile
// ids below 2^16) a 16-bit mask of 4 x 4 regions at bit 16, mode 1 (below
// 2^24) an 8-bit mask of 2 x 4 regions at bit 24, mode 0 none.  A blend
// pixel box of one pixel per thread (8 x 4) is exactly two regions at
// 16-pixel tiles and half of one at 32.
__host__ __device__ __forceinline__ int region_shift(int rmode) { return rmode == 2 ? 16 : 24; }
__host__ __device__ __forceinline__ int region_cols(int rmode) { return rmode == 2 ? 4 : 2; }

__device__ __forceinline__ unsigned tile_regions(const TileReach &t, int tx, int ty, int TS, int cols)
{
    unsigned m = 0u;
    const float x0 = (float)(TS * tx) - t.u, cw = (float)TS / (float)cols;
#pragma unroll
    for (int ry = 0; ry < 4; ++ry) {
        const float y0 = (float)(TS * ty) + 0.25f * TS * ry;
        const float lo = fmaxf(y0 - 1.f - t.v, -t.ey);
        const float hi = fminf(y0 + 0.25f * TS + 1.f - t.v, t.ey);
        if (lo > hi) continue;
        const float dr = fminf(fmaxf(t.dyR, lo), hi), dl = fminf(fmaxf(-t.dyR, lo), hi);
        const float xr = (-t.Bh * dr + sqrtf(fmaxf(0.f, t.AR - t.det * dr * dr))) * t.iA;
        const float xl = (-t.Bh * dl - sqrtf(fmaxf(0.f, t.AR - t.det * dl * dl))) * t.iA;
        // column c spans [x0 + c cw - 1, x0 + (c + 1) cw + 1] (padded by one pixel)
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (c < cols && xr >= x0 + c * cw - 1.f && xl <= x0 + (c + 1) * cw + 1.f) m |= 1u << (cols * ry + c);
    }
    return m;
}

// The regions (bits as in tile_regions) that blend pixel box wbox of a TS
// tile overlaps: the box is 8 x 4 PPT pixels, BoxMap's layout.
template <int TS, int PPT>
__device__ __forceinline__ unsigned box_regions(int wbox, int cols)
{
    constexpr int BW = 8, BH = 4 * PPT, BPR = TS / BW, RH = TS / 4;
    const int RW = TS / cols;
    const int x0 = (wbox % BPR) * BW, y0 = (wbox / BPR) * BH;
    unsigned m = 0u;
#pragma unroll
    for (int ry = 0; ry < 4; ++ry)
#pragma unroll
        for (int rx = 0; rx < 4; ++rx)
            if (rx < cols && rx * RW < x0 + BW && x0 < (rx + 1) * RW && ry * RH < y0 + BH && y0 < (ry + 1) * RH)
                m |= 1u << (cols * ry + rx);
    return m;
}

// ---------------------------------------------------------------- scans
__device__ __forceinline__ int chunk_range(int n, int NB, int b, int &begin)
{
    int chunk = (n + NB - 1) / NB;
    begin = b * chunk;
    int end = begin + chunk;
    if (end > n) end = n;
    if (begin > n) begin = n;
    return end;
}

// Exclusive block-wide scan of one value per thread (blockDim <= 1024).
__device__ __forceinline__ int block_exclusive_scan(int v, int &total)
{
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (warp == 0) {
        int s = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        wsum[lane] = s;  // inclusive warp prefix
    }
    __syncthreads();
    int warp_base = warp > 0 ? wsum[warp - 1] : 0;
    total = wsum[nw - 1];
    __syncthreads();
    return warp_base + x - v;
}

// ---------------------------------------------------------------- radix sort
// Stable LSD radix sort, 8-bit digits, one kernel per digit pass:
//   sort_hist_kernel   global digit histograms of every pass in one read
//   onesweep_kernel    each block takes the next 2048-key tile (ticket order),
//                      ranks its keys stably in shared memory, publishes its
//                      digit counts and finds its global offsets by
//                      decoupled look-back over earlier tiles, then scatters.
// Look-back spins are bounded (spin_limit polls of one predecessor's word):
// a block whose wait expires reports AVATAR_ERR_TIMEOUT and takes its
// offsets the slow, exact way - it counts the digits of every earlier tile's
// keys itself - so it never hangs, never writes out of bounds, and the
// result stays the sorted order.
constexpr int OS_THREADS = 256;
constexpr int OS_WARPS = OS_THREADS / 32;
constexpr int OS_ITEMS = 8;
constexpr int OS_TILE = OS_THREADS * OS_ITEMS;  // 2048 keys per tile
constexpr int OS_MAX_PASSES = 4;
constexpr unsigned FLAG_AGG = 1u << 30, FLAG_INC = 2u << 30, FLAG_MASK = 3u << 30;
constexpr int SPIN_LIMIT = 1 << 22;   // default polls of one look-back word
constexpr int OS_LOOKBACK = 16;

__device__ __forceinline__ unsigned ld_volatile(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void st_volatile(unsigned *p, unsigned v)
{
    asm volatile("st.volatile.global.u32 [%0], %1;" ::"l"(p), "r"(v));
}

__global__ void __launch_bounds__(OS_THREADS)
sort_hist_kernel(const uint32_t *__restrict__ keys, const int32_t *__restrict__ n_ptr, int cap, int passes,
                 int32_t *__restrict__ hist)
{
    __shared__ int cnt[OS_MAX_PASSES][RADIX];
    for (int i = threadIdx.x; i < OS_MAX_PASSES * RADIX; i += blockDim.x) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const int n = min(*n_ptr, cap);
    // warp-aggregated counts: the lanes that share a digit add once (keys of
    // one frame often share their high digits, which would serialise the
    // shared-memory atomics)
    // eight independent key loads in flight per thread per round; a warp's
    // lanes stay together (whole 32-key groups), so the matches are uniform
    constexpr int U = 8;
    const int stride = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int w0 = blockIdx.x * blockDim.x + threadIdx.x - lane; w0 < n; w0 += U * stride) {  // warp-uniform
        uint32_t k[U];
        bool in[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = w0 + lane + u * stride;
            in[u] = i < n;
            k[u] = in[u] ? keys[i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!__any_sync(0xffffffffu, in[u])) break;
            for (int p = 0; p < passes; ++p) {
                const unsigned d = in[u] ? (k[u] >> (8 * p)) & 255u : 256u;
                const unsigned peers = __match_any_sync(0xffffffffu, d);
                if (in[u] && (peers & lanemask_lt()) == 0) atomicAdd(&cnt[p][d], __popc(peers));
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x) {
        int v = (&cnt[0][0])[i];
        if (v) atomicAdd(hist + i, v);
    }
}

// Four blocks per SM (64 registers, no spills): the pass is latency-bound on
// its loads and look-back, and at the 119 registers it takes unbounded only
// two blocks fit (paper-scale frame 1,058 -> 1,036 us, 128-view batch 56.8 ->
// 55.3 ms, measured alternately in one session).
__global__ void __launch_bounds__(OS_THREADS, 4)
onesweep_kernel(const uint32_t *__restrict__ kin, const int32_t *__restrict__ vin, uint32_t *__restrict__ kout,
                int32_t *__restrict__ vout, const int32_t *__restrict__ n_ptr, int cap, int shift,
                const int32_t *__restrict__ hist, unsigned *__restrict__ desc, int32_t *__restrict__ ticket,
                int32_t *status, int spin_limit)
{
    __shared__ int s_tile;
    __shared__ int s_wcnt[OS_WARPS][RADIX];  // running, then exclusive-over-warps digit counts
    __shared__ int s_gbase[RADIX];           // global offset of digit d, less its offset within the tile
    __shared__ uint32_t s_key[OS_TILE];      // the tile's keys and values in tile-sorted order
    __shared__ int32_t s_val[OS_TILE];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(ticket, 1);
    for (int i = tid; i < OS_WARPS * RADIX; i += OS_THREADS) (&s_wcnt[0][0])[i] = 0;
    __syncthreads();
    const int tile = s_tile;
    const int n = min(*n_ptr, cap);
    const int base = tile * OS_TILE;
    if (base >= n) return;  // tickets are taken in order: no later tile waits on this one
    // warp w owns the contiguous segment [base + 256 w, base + 256 (w + 1))
    uint32_t key[OS_ITEMS];
    int32_t val[OS_ITEMS];
    int rank[OS_ITEMS];
    int dig[OS_ITEMS];
#pragma unroll
    for (int i = 0; i < OS_ITEMS; ++i) {
        int idx = base + warp * (32 * OS_ITEMS) + i * 32 + lane;
        bool ok = idx < n;
        key[i] = ok ? kin[idx] : 0u;
        val[i] = ok ? vin[idx] : 0;
        dig[i] = ok ? (int)((key[i] >> shift) & 255u) : RADIX;
    }
#pragma unroll
    for (int i = 0; i < OS_ITEMS; ++i) {
        unsigned peers = __match_any_sync(0xffffffffu, dig[i]);
        int before = dig[i] < RADIX ? s_wcnt[warp][dig[i]] : 0;
        rank[i] = before + __popc(peers & lanemask_lt());
        __syncwarp();
        if (dig[i] < RADIX && (peers & lanemask_lt()) == 0) s_wcnt[warp][dig[i]] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // thread d: exclusive scan of digit d over warps, publish, look back
    {
        const int d = tid;
        int sum = 0;
#pragma unroll
        for (int w = 0; w < OS_WARPS; ++w) {
            int c = s_wcnt[w][d];
            s_wcnt[w][d] = sum;
            sum += c;
        }
        unsigned *my = desc + (size_t)tile * RADIX + d;
        st_volatile(my, (tile == 0 ? FLAG_INC : FLAG_AGG) | (unsigned)sum);
        // decoupled look-back, OS_LOOKBACK predecessors per round trip
        int prefix = 0;
        bool found = tile == 0, expired = false;
        for (int p = tile - 1; p >= 0 && !found && !expired; p -= OS_LOOKBACK) {
            unsigned v[OS_LOOKBACK];
#pragma unroll
            for (int i = 0; i < OS_LOOKBACK; ++i)
                v[i] = (p - i >= 0) ? ld_volatile(desc + (size_t)(p - i) * RADIX + d) : FLAG_INC;
#pragma unroll
            for (int i = 0; i < OS_LOOKBACK; ++i) {
                if (found) break;
                unsigned x = v[i];
                if (p - i >= 0) {
                    int spins = 0;
                    while ((x & FLAG_MASK) == 0) {
                        if (++spins > spin_limit) {
                            expired = true;
                            break;
                        }
                        __nanosleep(32);
                        x = ld_volatile(desc + (size_t)(p - i) * RADIX + d);
                    }
                    if (expired) break;
                }
                prefix += (int)(x & ~FLAG_MASK);
                if ((x & FLAG_MASK) == FLAG_INC) found = true;
            }
        }
        // a wait expired somewhere in the block: every digit's prefix is
        // recounted from the keys of the earlier tiles (base of them), all of
        // which this pass reads and none of which it writes
        if (__syncthreads_or(expired)) {
            s_gbase[d] = 0;
            __syncthreads();
            for (int i = tid; i < base; i += OS_THREADS) atomicAdd(&s_gbase[(kin[i] >> shift) & 255u], 1);
            __syncthreads();
            prefix = s_gbase[d];
            if (tid == 0) av_report(status, AVATAR_ERR_TIMEOUT);
            __syncthreads();
        }
        if (tile > 0) st_volatile(my, FLAG_INC | (unsigned)(prefix + sum));
        // global base of digit d (exclusive scan of this pass's histogram plus
        // the earlier tiles' count) less its base within the tile (exclusive
        // scan of the tile's counts), so a key at tile position j goes to
        // s_gbase[d] + j
        int tot;
        const int gex = block_exclusive_scan(hist[d], tot);
        const int tex = block_exclusive_scan(sum, tot);
        s_gbase[d] = gex + prefix - tex;
        s_wcnt[0][d] = tex;  // every warp's exclusive offsets are read below before this row is
    }
    __syncthreads();
    // stage the tile in tile-sorted order, then write each digit's run with
    // consecutive threads on consecutive addresses
    const int tile_n = min(OS_TILE, n - base);
    {
        int pos[OS_ITEMS];
#pragma unroll
        for (int i = 0; i < OS_ITEMS; ++i)
            pos[i] = dig[i] < RADIX ? s_wcnt[0][dig[i]] + (warp == 0 ? 0 : s_wcnt[warp][dig[i]]) + rank[i] : -1;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < OS_ITEMS; ++i)
            if (pos[i] >= 0) {
                s_key[pos[i]] = key[i];
                s_val[pos[i]] = val[i];
            }
    }
    __syncthreads();
    for (int j = tid; j < tile_n; j += OS_THREADS) {
        const uint32_t k = s_key[j];
        const int dst = s_gbase[(k >> shift) & 255u] + j;
        kout[dst] = k;
        vout[dst] = s_val[j];
    }
}

// Look-back polls the context allows (AVATAR_TUNE_WAIT_LIMIT; 0 = default).
inline int sort_spin_limit(const avatar_ctx *ctx)
{
    const int v = ctx ? ctx->tune[AVATAR_TUNE_WAIT_LIMIT] : 0;
    return v > 0 ? v : SPIN_LIMIT;
}

// Scratch of the radix sort: [OS_MAX_PASSES][RADIX] histograms followed by
// [OS_MAX_PASSES] tile tickets, and [passes][tiles][RADIX] look-back words.
struct SortWs {
    int32_t *hist;
    unsigned *desc;
};

inline size_t sort_desc_words(size_t max_items)
{
    return (size_t)OS_MAX_PASSES * ((max_items + OS_TILE - 1) / OS_TILE) * RADIX;
}

// Sorts (k0, v0) of *n_ptr (<= cap) items stably on bits [0, bits) in 8-bit
// passes, ping-ponging with (k1, v1): an even number of passes ends in
// (k0, v0), an odd number in (k1, v1).
inline int radix_sort(uint32_t *k0, int32_t *v0, uint32_t *k1, int32_t *v1, int bits, const int32_t *n_ptr, int cap,
                      const SortWs &w, int32_t *status, cudaStream_t st, int spin_limit = SPIN_LIMIT)
{
    int passes = (bits + 7) / 8;
    if (passes < 1) passes = 1;
    if (passes > OS_MAX_PASSES) return AVATAR_ERR_INVALID_ARG;
    const int ntiles = (cap + OS_TILE - 1) / OS_TILE;
    if (cudaMemsetAsync(w.hist, 0, sizeof(int32_t) * (OS_MAX_PASSES * RADIX + OS_MAX_PASSES), st) != cudaSuccess ||
        cudaMemsetAsync(w.desc, 0, sizeof(unsigned) * (size_t)passes * ntiles * RADIX, st) != cudaSuccess)
        return AVATAR_ERR_CUDA;
    int hgrid = (cap + OS_THREADS * 8 - 1) / (OS_THREADS * 8);
    if (hgrid > 304) hgrid = 304;
    if (hgrid < 1) hgrid = 1;
    sort_hist_kernel<<<hgrid, OS_THREADS, 0, st>>>(k0, n_ptr, cap, passes, w.hist);
    uint32_t *kin = k0, *kout = k1;
    int32_t *vin = v0, *vout = v1;
    int32_t *tickets = w.hist + OS_MAX_PASSES * RADIX;
    for (int p = 0; p < passes; ++p) {
        onesweep_kernel<<<ntiles, OS_THREADS, 0, st>>>(kin, vin, kout, vout, n_ptr, cap, 8 * p, w.hist + p * RADIX,
                                                       w.desc + (size_t)p * ntiles * RADIX, tickets + p, status,
                                                       spin_limit);
        uint32_t *tk = kin;
        kin = kout;
        kout = tk;
        int32_t *tv = vin;
        vin = vout;
        vout = tv;
    }
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}

// Bits of a tile sort over ntiles tiles: 2^bits >= ntiles + 1, so that
// KEY_NO_TILE's sorted bits (all ones) order after every tile.
inline int bits_for(long ntiles)
{
    ++ntiles;
    int b = 0;
    while ((1L << b) < ntiles) ++b;
    return b;
}

// The region mode of a tile sort over ntiles tiles of edge TS: the mask
// sits above the bits the sort's passes cover.  32-pixel tiles take the
// 4 x 4 grid (mode 2) where the sort covers at most 16 bits, so that a blend
// box is half a region; other tiles take the 2 x 4 grid (mode 1, exact boxes
// at 16 pixels, and cheaper to emit) where it covers at most 24; else none.
inline int region_mode(long ntiles, int TS, bool allowed = true)
{
    if (!allowed) return 0;
    const int tb = bits_for(ntiles);
    const int sorted = tb <= 8 ? 8 : (tb + 7) / 8 * 8;
    return TS == 32 && sorted <= 16 ? 2 : sorted <= 24 ? 1 : 0;
}
inline uint32_t tile_key_mask(long ntiles, int TS, bool allowed = true)
{
    const int rm = region_mode(ntiles, TS, allowed);
    return rm ? (1u << region_shift(rm)) - 1u : 0xffffffffu;
}

// ---------------------------------------------------------------- pair scan
__global__ void __launch_bounds__(1024)
pair_scan_reduce_kernel(const int32_t *__restrict__ sorted_idx, const int32_t *__restrict__ npairs, int G, int NB,
                        int32_t *__restrict__ block_sums)
{
    int begin;
    int end = chunk_range(G, NB, blockIdx.x, begin);
    long s = 0;
    for (int i = begin + threadIdx.x; i < end; i += blockDim.x) s += npairs[sorted_idx[i]];
    int v = (int)min(s, (long)0x3fffffff);
    int tot;
    block_exclusive_scan(v, tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024)
pair_scan_down_kernel(const int32_t *__restrict__ sorted_idx, const int32_t *__restrict__ npairs, int G, int NB,
                      const int32_t *__restrict__ block_sums, int32_t *__restrict__ offsets,
                      int32_t *__restrict__ num_pairs, long cap, int32_t *status)
{
    __shared__ long s_base;
    if (threadIdx.x == 0) {
        long b = 0, tot = 0;
        for (int i = 0; i < NB; ++i) {
            if (i < (int)blockIdx.x) b += block_sums[i];
            tot += block_sums[i];
        }
        s_base = b;
        if (blockIdx.x == 0) {
            long t = tot > 0x7fffffffL ? 0x7fffffffL : tot;
            *num_pairs = (int32_t)t;
            if (tot > cap) av_report(status, AVATAR_ERR_OVERFLOW);
        }
    }
    __syncthreads();
    long running = s_base;
    int begin;
    int end = chunk_range(G, NB, blockIdx.x, begin);
    for (int tb = begin; tb < end; tb += blockDim.x) {
        int i = tb + threadIdx.x;
        int v = i < end ? npairs[sorted_idx[i]] : 0;
        int tot;
        int ex = block_exclusive_scan(v, tot);
        if (i < end) offsets[i] = (int32_t)min(running + ex, (long)0x7fffffff);
        running += tot;
    }
}

__global__ void __launch_bounds__(256)
tile_ranges_kernel(const uint32_t *__restrict__ keys, const int32_t *__restrict__ num_pairs, long cap, int ntiles,
                   uint32_t tile_mask, int2 *__restrict__ ranges)
{
    // after an overflow the pair list is incomplete: leave every tile empty
    if ((long)*num_pairs > cap) return;
    int n = *num_pairs;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t t = keys[i] & tile_mask;  // the tile id below the region mask
        if (t >= (uint32_t)ntiles) continue;
        if (i == 0 || (keys[i - 1] & tile_mask) != t) ranges[t].x = i;
        if (i == n - 1 || (keys[i + 1] & tile_mask) != t) ranges[t].y = i + 1;
    }
}

// ---------------------------------------------------------------- blend
// One CTA per TS x TS tile.  Warp w owns an 8 x (4 PPT) pixel box of the
// tile (lane l, pixel k at (l % 8, l / 8 + 4 k) inside it); Gaussians are
// staged NTH at a time in shared memory, and a warp skips every Gaussian
// whose pixel rect misses its box, or whose ellipse (alpha >= 1/255) reaches
// none of the tile regions the box overlaps (the region mask in the pair's
// key): no pixel there can reach alpha = 1/255.
template <int TS, int PPT>
struct BoxMap {
    static constexpr int BW = 8, BH = 4 * PPT, BPR = TS / BW;
    int x0, y0;  // box origin (pixels)
    __device__ BoxMap(int tx, int ty, int warp)
    {
        x0 = tx * TS + (warp % BPR) * BW;
        y0 = ty * TS + (warp / BPR) * BH;
    }
    __device__ int px(int lane) const { return x0 + (lane & 7); }
    __device__ int py(int lane, int k) const { return y0 + (lane >> 3) + 4 * k; }
};

// Warps per CTA of the kernels built on blend_box and blend_backward_box.
constexpr int BWD_WARPS = 4;

// Front-to-back blend of pixel box wbox of tile (tx, ty) of a W x H image
// over the tile's sorted pairs [rg.x, rg.y), by one warp on its own; writes
// the box's pixels of image [3][H][W], T_final and n_last.  The list is
// walked 32 entries at a time: each batch's records go to the warp's two
// buffers (s0/s1/s2 [2][32]) by asynchronous copies while the previous batch
// is walked, the lanes test the batch's rects and region masks against the
// box for a hit mask (a Gaussian whose rect misses the box, or whose ellipse
// reaches none of the regions the box overlaps, cannot reach alpha = 1/255
// in it; a fifth of the rect hits are such), hits are evaluated two at a time (their exponents are independent of
// T), and the warp leaves as soon as its own pixels are saturated.
template <int TS, int PPT>
__device__ __forceinline__ void blend_box(int2 rg, const int32_t *__restrict__ pair_gauss,
                                          const float4 *__restrict__ rec0, const float4 *__restrict__ rec1,
                                          const float4 *__restrict__ rec2, int W, int H, int tx, int ty, int wbox,
                                          const uint32_t *__restrict__ pkeys, int rmode,
                                          float *__restrict__ image, float *__restrict__ T_final,
                                          int32_t *__restrict__ n_last, float4 (*s0)[32], float4 (*s1)[32],
                                          float4 (*s2)[32])
{
    using Box = BoxMap<TS, PPT>;
    const int lane = threadIdx.x & 31;
    const Box box(tx, ty, wbox);
    const int bx0 = box.x0, by0 = box.y0, bx1 = bx0 + Box::BW - 1, by1 = by0 + Box::BH - 1;
    float fx[PPT], fy[PPT], T[PPT], C0[PPT], C1[PPT], C2[PPT];
    int last[PPT];
    bool live[PPT];
    bool any_live = false;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int px = box.px(lane), py = box.py(lane, k);
        fx[k] = px + 0.5f;
        fy[k] = py + 0.5f;
        T[k] = 1.f;
        C0[k] = C1[k] = C2[k] = 0.f;
        last[k] = 0;
        live[k] = px < W && py < H;
        any_live = any_live || live[k];
    }
    const int n = rg.y - rg.x;
    // the records of list entries [base, base + 32) into buffer b, Gaussian
    // g for this lane's entry
    auto issue = [&](int base, int b, int g) {
        if (base + lane < n) {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(&s0[b][lane])),
                         "l"(rec0 + g)
                         : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(&s1[b][lane])),
                         "l"(rec1 + g)
                         : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(&s2[b][lane])),
                         "l"(rec2 + g)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto gauss = [&](int idx) { return idx < n ? pair_gauss[rg.x + idx] : 0; };
    // the entry's key: its region mask above the tile id (all ones without
    // masks), tested against the regions this box overlaps
    auto keyat = [&](int idx) { return rmode && idx < n ? pkeys[rg.x + idx] : 0xffffffffu; };
    const unsigned bmask = box_regions<TS, PPT>(wbox, region_cols(rmode));
    const int rshift = region_shift(rmode);
    if (n > 0 && __any_sync(0xffffffffu, any_live)) {
        // indices and keys run two batches ahead of the walk and records one,
        // so no load's latency is waited for in the loop
        int g_next = gauss(32 + lane);
        uint32_t k_next = keyat(32 + lane);
        issue(0, 0, gauss(lane));
        uint32_t k_cur = keyat(lane);
        int b = 0;
        for (int base = 0; base < n; base += 32, b ^= 1) {
            const bool more = base + 32 < n;
            if (more) issue(base + 32, b ^ 1, g_next);
            const uint32_t k_issued = k_next;
            g_next = gauss(base + 64 + lane);
            k_next = keyat(base + 64 + lane);
            if (more)
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            else
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncwarp();  // every lane's copies of batch b are visible to the warp
            // the batch's hit mask from the rects now in shared memory
            bool hit = false;
            if (base + lane < n) {
                const float4 r1 = s1[b][lane];
                const int ra = __float_as_int(r1.z), rc = __float_as_int(r1.w);
                hit = (rc & 0xffff) >= bx0 && (ra & 0xffff) <= bx1 && (int)((unsigned)rc >> 16) >= by0 &&
                      (int)((unsigned)ra >> 16) <= by1 && ((k_cur >> rshift) & bmask) != 0u;
            }
            unsigned hits = __ballot_sync(0xffffffffu, hit);
            // one Gaussian's contribution to pixel k (the front-to-back step),
            // without branches: a lane that does not take the Gaussian adds
            // zero weight and keeps its T and last index (the same values the
            // branching form leaves)
            auto step = [&](int sj, int k, float l2a) {
                const bool reach = live[k] && l2a >= LOG2_ALPHA_MIN;
                const float alpha = fminf(0.99f, exp2f(l2a));
                const float test_T = T[k] * (1.f - alpha);
                const bool stop = test_T < T_MIN;
                const bool take = reach && !stop;
                live[k] = live[k] && !(reach && stop);
                const float4 c = s2[b][sj];
                const float wgt = take ? alpha * T[k] : 0.f;
                C0[k] = fmaf(c.x, wgt, C0[k]);
                C1[k] = fmaf(c.y, wgt, C1[k]);
                C2[k] = fmaf(c.z, wgt, C2[k]);
                T[k] = take ? test_T : T[k];
                last[k] = take ? base + sj + 1 : last[k];
            };
            auto l2alpha = [&](int sj, int k) {
                const float4 r0 = s0[b][sj];
                const float4 r1 = s1[b][sj];
                float dx = fx[k] - r0.x, dy = fy[k] - r0.y;
                return fmaf(fmaf(r0.z, dx, r0.w * dy), dx, fmaf(r1.x * dy, dy, r1.y));
            };
            // two Gaussians per iteration: both exponents are independent of T
            while (hits) {
                const int j0 = __ffs(hits) - 1;
                hits &= hits - 1;
                const bool two = hits != 0;
                const int j1 = two ? __ffs(hits) - 1 : j0;
                if (two) hits &= hits - 1;
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    const float a0 = l2alpha(j0, k);
                    const float a1 = two ? l2alpha(j1, k) : -1e30f;
                    // the warp skips the pair where no live pixel reaches alpha 1/255
                    if (!__any_sync(0xffffffffu, live[k] && fmaxf(a0, a1) >= LOG2_ALPHA_MIN)) continue;
                    step(j0, k, a0);
                    step(j1, k, a1);
                }
                any_live = false;
#pragma unroll
                for (int k = 0; k < PPT; ++k) any_live = any_live || live[k];
                if (!__any_sync(0xffffffffu, any_live)) break;
            }
            __syncwarp();  // every lane is done with buffer b before it is refilled
            if (!__any_sync(0xffffffffu, any_live)) break;
            k_cur = k_issued;
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");  // no copy outlives the walk
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int px = box.px(lane), py = box.py(lane, k);
        if (px < W && py < H) {
            const int pix = py * W + px;
            image[pix] = C0[k];
            image[W * H + pix] = C1[k];
            image[2 * W * H + pix] = C2[k];
            T_final[pix] = T[k];
            n_last[pix] = last[k];
        }
    }
}

// Key of a pair whose Gaussian cannot reach its tile: it sorts after every
// tile (the tile sort covers bits_for(ntiles) bits, 2^bits > ntiles) and the
// tile ranges skip it, so no list holds it.
constexpr uint32_t KEY_NO_TILE = 0xffffffffu;

// Pair emission by one warp for 32 consecutive Gaussians of the depth order
// (lane j: n pairs starting at output offset off; an offset scan in that
// order makes the warp's pairs one contiguous range).  The warp writes the
// range slot by slot: lane j takes slot c + j, finds the Gaussian owning it
// by a binary search over the lanes' inclusive counts, and its tile from the
// slot's place in that Gaussian's tile rectangle (w tiles wide, row-major
// from (tx0, ty0)); key = kbase + ty kstride + tx, value gval, or
// KEY_NO_TILE where the Gaussian's ellipse cannot reach the tile (the rect
// is the ellipse's bounding box: about a fifth of its tiles lie in the
// corners the ellipse misses).  In region modes 1 and 2 the key carries
// above the tile id the mask of the tile's regions the ellipse reaches
// (tile_regions), which the blend tests instead of evaluating the ellipse
// per box; the tile sort covers only the tile bits and moves the mask with
// the key.
// Every store is coalesced; slots at or beyond cap are not written.
__device__ __forceinline__ void emit_pairs_warp(int n, long off, int gval, int tx0, int ty0, int w, int kbase,
                                                int kstride, const TileReach &tr, int TS, int rmode, long cap,
                                                uint32_t *__restrict__ keys, int32_t *__restrict__ vals)
{
    const int lane = threadIdx.x & 31;
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const long start = __shfl_sync(0xffffffffu, off, 0);
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int c = 0; c < total; c += 32) {
        const int sl = c + lane;
        int own = 0;  // lanes whose inclusive count is <= sl
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int v = __shfl_sync(0xffffffffu, incl, own + step - 1);
            if (v <= sl) own += step;
        }
        own = min(own, 31);
        const int o_g = __shfl_sync(0xffffffffu, gval, own);
        const int o_excl = __shfl_sync(0xffffffffu, incl - n, own);
        const int o_tx0 = __shfl_sync(0xffffffffu, tx0, own);
        const int o_ty0 = __shfl_sync(0xffffffffu, ty0, own);
        const int o_w = __shfl_sync(0xffffffffu, w, own);
        const int o_base = __shfl_sync(0xffffffffu, kbase, own);
        const int o_stride = __shfl_sync(0xffffffffu, kstride, own);
        TileReach o_tr;
        o_tr.u = __shfl_sync(0xffffffffu, tr.u, own);
        o_tr.v = __shfl_sync(0xffffffffu, tr.v, own);
        o_tr.iA = __shfl_sync(0xffffffffu, tr.iA, own);
        o_tr.Bh = __shfl_sync(0xffffffffu, tr.Bh, own);
        o_tr.det = __shfl_sync(0xffffffffu, tr.det, own);
        o_tr.AR = __shfl_sync(0xffffffffu, tr.AR, own);
        o_tr.ey = __shfl_sync(0xffffffffu, tr.ey, own);
        o_tr.dyR = __shfl_sync(0xffffffffu, tr.dyR, own);
        const long dst = start + sl;
        if (sl < total && dst < cap) {
            const int local = sl - o_excl;
            const int q = (int)__fdividef((float)local + 0.5f, (float)o_w);  // exact for local < 2^22
            const int tx = o_tx0 + (local - q * o_w), ty = o_ty0 + q;
            const unsigned m = tile_regions(o_tr, tx, ty, TS, region_cols(rmode));
            keys[dst] = m ? (uint32_t)(o_base + ty * o_stride + tx) | (rmode ? m << region_shift(rmode) : 0u)
                          : KEY_NO_TILE;
            vals[dst] = o_g;
        }
    }
}

// Adjoint of blend_box for pixel box wbox of tile (tx, ty), by one warp on
// its own: reverse traversal of the tile's list from the per-pixel
// checkpoint (T_final, n_last), starting at the box's largest n_last, 32
// entries at a time.  Each batch's records go to the warp's two buffers
// (s0/s1/s2/sg [2][32]) by asynchronous copies while the previous batch is
// walked, and the lanes test the batch's rects and region masks against the
// box for a hit mask, so no warp waits for another.  Per hit Gaussian the warp's nine sums
// (d_color [3][cs], d_opacity [cs], d_mean2d [2][cs], d_conic [3][cs] at the
// Gaussian's pair value) are reduced together (eight by recursive halving,
// the ninth by a butterfly) and added by nine lanes with one atomic each.
template <int TS, int PPT>
__device__ __forceinline__ void blend_backward_box(int2 rg, const int32_t *__restrict__ pair_gauss,
                                                   const float4 *__restrict__ rec0, const float4 *__restrict__ rec1,
                                                   const float4 *__restrict__ rec2, int W, int H, int tx, int ty,
                                                   int wbox, const uint32_t *__restrict__ pkeys, int rmode,
                                                   const float *__restrict__ T_final,
                                                   const int32_t *__restrict__ n_last,
                                                   const float *__restrict__ d_image, size_t cs,
                                                   float *__restrict__ d_mean2d, float *__restrict__ d_conic,
                                                   float *__restrict__ d_opacity, float *__restrict__ d_color,
                                                   float4 (*s0)[32], float4 (*s1)[32], float4 (*s2)[32],
                                                   int (*sg)[32])
{
    using Box = BoxMap<TS, PPT>;
    constexpr float LN2 = 0.6931471805599453f;
    const int lane = threadIdx.x & 31;
    const Box box(tx, ty, wbox);
    const int bx0 = box.x0, by0 = box.y0, bx1 = bx0 + Box::BW - 1, by1 = by0 + Box::BH - 1;
    float fx[PPT], fy[PPT], T[PPT], dC0[PPT], dC1[PPT], dC2[PPT], acc0[PPT], acc1[PPT], acc2[PPT];
    int my_last[PPT];
    int mx_last = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int px = box.px(lane), py = box.py(lane, k);
        const bool inside = px < W && py < H;
        const int pix = py * W + px;
        fx[k] = px + 0.5f;
        fy[k] = py + 0.5f;
        my_last[k] = inside ? n_last[pix] : 0;
        T[k] = inside ? T_final[pix] : 1.f;
        dC0[k] = inside ? d_image[pix] : 0.f;
        dC1[k] = inside ? d_image[W * H + pix] : 0.f;
        dC2[k] = inside ? d_image[2 * W * H + pix] : 0.f;
        acc0[k] = acc1[k] = acc2[k] = 0.f;
        mx_last = max(mx_last, my_last[k]);
    }
    const int n = (int)__reduce_max_sync(0xffffffffu, (unsigned)mx_last);
    // the records of list entries [end - 32, end) into buffer b, Gaussian g
    // for this lane's entry
    auto issue = [&](int end, int b, int g) {
        if (end - 32 + lane >= 0) {
            sg[b][lane] = g;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(&s0[b][lane])),
                         "l"(rec0 + g)
                         : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(&s1[b][lane])),
                         "l"(rec1 + g)
                         : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(&s2[b][lane])),
                         "l"(rec2 + g)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto gauss = [&](int idx) { return idx >= 0 ? pair_gauss[rg.x + idx] : 0; };
    auto keyat = [&](int idx) { return rmode && idx >= 0 ? pkeys[rg.x + idx] : 0xffffffffu; };
    const unsigned bmask = box_regions<TS, PPT>(wbox, region_cols(rmode));
    const int rshift = region_shift(rmode);
    if (n == 0) return;
    // indices and keys run two batches ahead of the walk and records one
    int g_next = gauss(n - 64 + lane);
    uint32_t k_next = keyat(n - 64 + lane);
    issue(n, 0, gauss(n - 32 + lane));
    uint32_t k_cur = keyat(n - 32 + lane);
    int b = 0;
    for (int end = n; end > 0; end -= 32, b ^= 1) {
        const bool more = end > 32;
        if (more) issue(end - 32, b ^ 1, g_next);
        const uint32_t k_issued = k_next;
        g_next = gauss(end - 96 + lane);
        k_next = keyat(end - 96 + lane);
        if (more)
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        else
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();  // every lane's copies of batch b are visible to the warp
        // the batch's hit mask from the rects now in shared memory
        bool hit = false;
        if (end - 32 + lane >= 0) {
            const float4 q1 = s1[b][lane];
            const int ra = __float_as_int(q1.z), rc = __float_as_int(q1.w);
            hit = (rc & 0xffff) >= bx0 && (ra & 0xffff) <= bx1 && (int)((unsigned)rc >> 16) >= by0 &&
                  (int)((unsigned)ra >> 16) <= by1 && ((k_cur >> rshift) & bmask) != 0u;
        }
        unsigned hits = __ballot_sync(0xffffffffu, hit);
        while (hits) {
            const int sj = 31 - __clz(hits);
            hits &= ~(1u << sj);
            const int j = end - 32 + sj;
            const float4 r1 = s1[b][sj];
            const float4 r0 = s0[b][sj];
            const float4 c = s2[b][sj];
            float g_col0 = 0.f, g_col1 = 0.f, g_col2 = 0.f, g_op = 0.f, g_mx = 0.f, g_my = 0.f, g_ca = 0.f,
                  g_cb = 0.f, g_cc = 0.f;
            bool contrib = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (j >= my_last[k]) continue;
                float dx = fx[k] - r0.x, dy = fy[k] - r0.y;
                float l2a = fmaf(fmaf(r0.z, dx, r0.w * dy), dx, fmaf(r1.x * dy, dy, r1.y));
                if (l2a < LOG2_ALPHA_MIN) continue;
                float raw = exp2f(l2a);
                float alpha = fminf(0.99f, raw);
                contrib = true;
                T[k] = __fdividef(T[k], 1.f - alpha);  // 1 - alpha >= 0.01: the fast form is within 2 ulp
                float wgt = alpha * T[k];
                g_col0 = fmaf(wgt, dC0[k], g_col0);
                g_col1 = fmaf(wgt, dC1[k], g_col1);
                g_col2 = fmaf(wgt, dC2[k], g_col2);
                float dalpha = T[k] * ((c.x - acc0[k]) * dC0[k] + (c.y - acc1[k]) * dC1[k] + (c.z - acc2[k]) * dC2[k]);
                acc0[k] = alpha * c.x + (1.f - alpha) * acc0[k];
                acc1[k] = alpha * c.y + (1.f - alpha) * acc1[k];
                acc2[k] = alpha * c.z + (1.f - alpha) * acc2[k];
                if (raw < 0.99f) {
                    float dpow = dalpha * raw;
                    g_op += dpow;
                    float ca = -2.f * LN2 * r0.z, cb = -LN2 * r0.w, cc = -2.f * LN2 * r1.x;
                    g_mx = fmaf(dpow, ca * dx + cb * dy, g_mx);
                    g_my = fmaf(dpow, cb * dx + cc * dy, g_my);
                    g_ca = fmaf(-0.5f * dpow, dx * dx, g_ca);
                    g_cb = fmaf(-dpow, dx * dy, g_cb);
                    g_cc = fmaf(-0.5f * dpow, dy * dy, g_cc);
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
                const float v[9] = {g_col0, g_col1, g_col2, g_op, g_mx, g_my, g_ca, g_cb, g_cc};
                float tot_cc;
                const float tot = warp_reduce_scatter9(v, tot_cc);
                const size_t g = (size_t)sg[b][sj];
                if ((lane & 3) == 0) {
                    const int vi = lane >> 2;
                    float *dst = vi < 3   ? d_color + (size_t)vi * cs
                                 : vi == 3 ? d_opacity
                                 : vi < 6  ? d_mean2d + (size_t)(vi - 4) * cs
                                           : d_conic + (size_t)(vi - 6) * cs;
                    atomicAdd(dst + g, vi == 3 ? tot / c.w : tot);
                } else if (lane == 1) {
                    atomicAdd(d_conic + 2 * cs + g, tot_cc);
                }
            }
        }
        __syncwarp();  // every lane is done with buffer b before it is refilled
        k_cur = k_issued;
    }
}

// ---------------------------------------------------------------- projection adjoint
// Gradients of the EWA projection of Gaussian i (xd [3][cs], cov [6][cs])
// from d_mean2d (dmx, dmy) and d_conic (da, db, dc): d_xd[3], d_cov[6].
__device__ __forceinline__ void project_adjoint(const float *__restrict__ xd, const float *__restrict__ cov, size_t cs,
                                                size_t i, const CamDev &cam, float dmx, float dmy, float da, float db,
                                                float dc, float (&d_xd)[3], float (&d_cov)[6])
{
    float x = xd[i], y = xd[cs + i], z = xd[2 * cs + i];
    float px = cam.R[0] * x + cam.R[1] * y + cam.R[2] * z + cam.t[0];
    float py = cam.R[3] * x + cam.R[4] * y + cam.R[5] * z + cam.t[1];
    float pz = cam.R[6] * x + cam.R[7] * y + cam.R[8] * z + cam.t[2];
    float iz = 1.0f / pz;
    float j00 = cam.fx * iz, j02 = -cam.fx * px * iz * iz;
    float j11 = cam.fy * iz, j12 = -cam.fy * py * iz * iz;
    float T0[3], T1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        T0[k] = j00 * cam.R[k] + j02 * cam.R[6 + k];
        T1[k] = j11 * cam.R[3 + k] + j12 * cam.R[6 + k];
    }
    float c[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) c[e] = cov[e * cs + i];
    float S[9] = {c[0], c[1], c[2], c[1], c[3], c[4], c[2], c[4], c[5]};
    float S0[3], S1[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        S0[r] = S[3 * r] * T0[0] + S[3 * r + 1] * T0[1] + S[3 * r + 2] * T0[2];
        S1[r] = S[3 * r] * T1[0] + S[3 * r + 1] * T1[1] + S[3 * r + 2] * T1[2];
    }
    float s00 = T0[0] * S0[0] + T0[1] * S0[1] + T0[2] * S0[2] + 0.3f;
    float s01 = T1[0] * S0[0] + T1[1] * S0[1] + T1[2] * S0[2];
    float s11 = T1[0] * S1[0] + T1[1] * S1[1] + T1[2] * S1[2] + 0.3f;
    float det = s00 * s11 - s01 * s01;
    float id = 1.0f / det;
    float ca = s11 * id, cb = -s01 * id, cc = s00 * id;
    // conic (a,b,c) -> Sigma' entries (s00, s01 (scalar, both positions), s11)
    float ds00 = -ca * ca * da - ca * cb * db - cb * cb * dc;
    float ds11 = -cb * cb * da - cb * cc * db - cc * cc * dc;
    float ds01 = -2.f * ca * cb * da - (ca * cc + cb * cb) * db - 2.f * cb * cc * dc;
    // symmetric 2x2 gradient
    float g00 = ds00, g01 = 0.5f * ds01, g11 = ds11;
    // dSigma = T^T Gm T (3x3 symmetric)
    float dS[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            dS[3 * r + j] = T0[r] * (g00 * T0[j] + g01 * T1[j]) + T1[r] * (g01 * T0[j] + g11 * T1[j]);
    d_cov[0] = dS[0];
    d_cov[1] = dS[1] + dS[3];
    d_cov[2] = dS[2] + dS[6];
    d_cov[3] = dS[4];
    d_cov[4] = dS[5] + dS[7];
    d_cov[5] = dS[8];
    // dT = 2 Gm T Sigma  (rows 0 and 1)
    float dT0[3], dT1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dT0[k] = 2.f * (g00 * S0[k] + g01 * S1[k]);
        dT1[k] = 2.f * (g01 * S0[k] + g11 * S1[k]);
    }
    // T = J R -> dJ = dT R^T (only the non-zero entries of J)
    float dj00 = dT0[0] * cam.R[0] + dT0[1] * cam.R[1] + dT0[2] * cam.R[2];
    float dj02 = dT0[0] * cam.R[6] + dT0[1] * cam.R[7] + dT0[2] * cam.R[8];
    float dj11 = dT1[0] * cam.R[3] + dT1[1] * cam.R[4] + dT1[2] * cam.R[5];
    float dj12 = dT1[0] * cam.R[6] + dT1[1] * cam.R[7] + dT1[2] * cam.R[8];
    float iz2 = iz * iz, iz3 = iz2 * iz;
    float dpx = dmx * cam.fx * iz - dj02 * cam.fx * iz2;
    float dpy = dmy * cam.fy * iz - dj12 * cam.fy * iz2;
    float dpz = -dmx * cam.fx * px * iz2 - dmy * cam.fy * py * iz2 - dj00 * cam.fx * iz2 +
                dj02 * 2.f * cam.fx * px * iz3 - dj11 * cam.fy * iz2 + dj12 * 2.f * cam.fy * py * iz3;
    d_xd[0] = cam.R[0] * dpx + cam.R[3] * dpy + cam.R[6] * dpz;
    d_xd[1] = cam.R[1] * dpx + cam.R[4] * dpy + cam.R[7] * dpz;
    d_xd[2] = cam.R[2] * dpx + cam.R[5] * dpy + cam.R[8] * dpz;
}

}  // namespace
