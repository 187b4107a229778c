// K nearest neighbours: the vertex sets S_g of Eq. 1 (the K_g nearest mesh
// vertices of each Gaussian, Sec. 3.1) and S_v of the visibility filters (the
// K_v nearest vertices of each vertex, Sec. 3.2), recomputed on the device
// whenever the canonical positions change (rebinding).
//
//   bbox      min / max of the reference points (ordered-integer atomics)
//   grid      a uniform grid over the box with about two points per cell
//   bin       counting sort of the reference points into their cells, as
//             packed (x, y, z, index) records in cell order
//   query     one thread per query point visits Chebyshev shells of cells
//             around its own until the K-th best distance is below the
//             distance to every unvisited cell; an FP32 distance (within
//             4e-7 relative of the exact one) rejects every candidate that
//             cannot enter the K best, the survivors are kept sorted by
//             (FP64 squared distance, index)
// The squared distance is the FP64 value of (d0 d0 + d1 d1) + d2 d2 of the
// FP32 coordinates, every operation rounded to nearest (no contraction), so
// the order - and the result - is exactly that definition's.
#include <algorithm>

#include "common.cuh"

namespace {

constexpr int KNN_THREADS = 256;
constexpr int KNN_MAX_K = 32;
constexpr int SCAN_BLOCK = 1024;

struct GridDev {
    float ox, oy, oz;  // grid origin (box minimum)
    float h, inv_h;    // cell edge
    int nx, ny, nz;
};

__device__ __forceinline__ int ordered(float f)
{
    const int b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float unordered(int o) { return __int_as_float(o >= 0 ? o : o ^ 0x7fffffff); }

__global__ void __launch_bounds__(KNN_THREADS)
knn_bbox_kernel(const float *__restrict__ ref, int M, int *__restrict__ box)
{
    int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, hi[3] = {(int)0x80000000, (int)0x80000000, (int)0x80000000};
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int o = ordered(__ldg(ref + (size_t)c * M + j));
            lo[c] = min(lo[c], o);
            hi[c] = max(hi[c], o);
        }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            lo[c] = min(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], s));
            hi[c] = max(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], s));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(box + c, lo[c]);
            atomicMax(box + 3 + c, hi[c]);
        }
    }
}

// Grid of edge h over the box with at most cap cells (about one point per cell).
__global__ void knn_grid_kernel(const int *__restrict__ box, int M, int cap, GridDev *g)
{
    float lo[3], ext[3];
    for (int c = 0; c < 3; ++c) {
        lo[c] = unordered(box[c]);
        ext[c] = fmaxf(unordered(box[3 + c]) - lo[c], 1e-6f);
    }
    const float target = fmaxf((float)M, 1.0f);
    float h = cbrtf(ext[0] * ext[1] * ext[2] / target);
    h = fmaxf(h, fmaxf(ext[0], fmaxf(ext[1], ext[2])) / 1024.0f);
    int n[3];
    for (int it = 0; it < 64; ++it) {
        long long cells = 1;
        for (int c = 0; c < 3; ++c) {
            n[c] = max(1, (int)ceilf(ext[c] / h));
            cells *= n[c];
        }
        if (cells <= cap) break;
        h *= 1.25f;
    }
    g->ox = lo[0];
    g->oy = lo[1];
    g->oz = lo[2];
    g->h = h;
    g->inv_h = 1.0f / h;
    g->nx = n[0];
    g->ny = n[1];
    g->nz = n[2];
}

__device__ __forceinline__ int cell_coord(float x, float o, float inv_h, int n)
{
    const int c = (int)floorf((x - o) * inv_h);
    return min(max(c, 0), n - 1);
}

__global__ void __launch_bounds__(KNN_THREADS)
knn_count_kernel(const float *__restrict__ ref, int M, const GridDev *__restrict__ gp, int *__restrict__ count,
                 int *__restrict__ cell_of)
{
    const GridDev g = *gp;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
        const int cx = cell_coord(__ldg(ref + j), g.ox, g.inv_h, g.nx);
        const int cy = cell_coord(__ldg(ref + (size_t)M + j), g.oy, g.inv_h, g.ny);
        const int cz = cell_coord(__ldg(ref + (size_t)2 * M + j), g.oz, g.inv_h, g.nz);
        const int cell = (cz * g.ny + cy) * g.nx + cx;
        cell_of[j] = cell;
        atomicAdd(count + cell, 1);
    }
}

// Exclusive scan of n ints, three phases: per-block totals, one block scans
// the totals, then each block scans its part with its offset.
__device__ __forceinline__ int block_scan_excl(int v, int &total)
{
    __shared__ int ws[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    total = ws[(blockDim.x >> 5) - 1];
    const int r = (warp > 0 ? ws[warp - 1] : 0) + x - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_BLOCK)
scan_totals_kernel(const int *__restrict__ in, int n, int *__restrict__ totals)
{
    const int i = blockIdx.x * SCAN_BLOCK + threadIdx.x;
    int total;
    block_scan_excl(i < n ? in[i] : 0, total);
    if (threadIdx.x == 0) totals[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_BLOCK)
scan_offsets_kernel(int *__restrict__ totals, int nb)
{
    int carry = 0;
    for (int base = 0; base < nb; base += SCAN_BLOCK) {
        const int i = base + threadIdx.x;
        int total;
        const int ex = block_scan_excl(i < nb ? totals[i] : 0, total);
        if (i < nb) totals[i] = carry + ex;
        carry += total;
    }
}

__global__ void __launch_bounds__(SCAN_BLOCK)
scan_apply_kernel(const int *__restrict__ in, int n, const int *__restrict__ offsets, int *__restrict__ out,
                  int *__restrict__ cursor)
{
    const int i = blockIdx.x * SCAN_BLOCK + threadIdx.x;
    int total;
    const int ex = block_scan_excl(i < n ? in[i] : 0, total) + offsets[blockIdx.x];
    if (i < n) {
        out[i] = ex;
        cursor[i] = ex;
    }
}

__global__ void __launch_bounds__(KNN_THREADS)
knn_scatter_kernel(const float *__restrict__ ref, const int *__restrict__ cell_of, int M, int *__restrict__ cursor,
                   float4 *__restrict__ pts)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x)
        pts[atomicAdd(cursor + cell_of[j], 1)] =
            make_float4(__ldg(ref + j), __ldg(ref + (size_t)M + j), __ldg(ref + (size_t)2 * M + j), __int_as_float(j));
}

// (d0 d0 + d1 d1) + d2 d2 in FP64, each operation rounded to nearest
__device__ __forceinline__ double dist2_rn(float x0, float x1, float x2, float r0, float r1, float r2)
{
    const double d0 = __dsub_rn((double)x0, (double)r0);
    const double d1 = __dsub_rn((double)x1, (double)r1);
    const double d2 = __dsub_rn((double)x2, (double)r2);
    return __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
}

// Queries in grid-cell order: query i goes to position order[...] of its cell,
// so the 32 queries of a warp search the same few cells (coherent loops and
// loads); their results do not depend on the order.
__global__ void __launch_bounds__(KNN_THREADS)
knn_order_kernel(const int *__restrict__ cell_of, int N, int *__restrict__ cursor, int *__restrict__ order)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        order[atomicAdd(cursor + cell_of[i], 1)] = i;
}

template <int KMAX>
__global__ void __launch_bounds__(KNN_THREADS)
knn_query_kernel(const float *__restrict__ x, int N, const float *__restrict__ ref, int M, int K,
                 const GridDev *__restrict__ gp, const int *__restrict__ start, const int *__restrict__ count,
                 const float4 *__restrict__ pts, const int *__restrict__ order, int32_t *__restrict__ knn,
                 float *__restrict__ dist2)
{
    const GridDev g = *gp;
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < N; o += gridDim.x * blockDim.x) {
        const int i = __ldg(order + o);
        const float x0 = __ldg(x + i), x1 = __ldg(x + (size_t)N + i), x2 = __ldg(x + (size_t)2 * N + i);
        const int cx = cell_coord(x0, g.ox, g.inv_h, g.nx);
        const int cy = cell_coord(x1, g.oy, g.inv_h, g.ny);
        const int cz = cell_coord(x2, g.oz, g.inv_h, g.nz);
        // The list keeps FP32 distances; the FP64 value of the fixed operation
        // order (which defines the order, with the index for ties) is formed
        // only when two FP32 values lie within 1e-6 relative of each other: the
        // FP32 value of (d0 d0 + d1 d1) + d2 d2 is within 3e-7 relative of it,
        // so outside that margin the FP32 comparison already decides.
        float bf[KMAX];  // FP32 distance
        int bi[KMAX];    // reference index
        int bt[KMAX];    // position of the reference point in pts (its coordinates for an exact comparison)
        int n = 0;
        float thr = INFINITY;  // FP32 rejection threshold: above it a candidate cannot enter
        const int smax = max(g.nx, max(g.ny, g.nz));
        for (int s = 0; s <= smax; ++s) {
            const int z0 = max(cz - s, 0), z1 = min(cz + s, g.nz - 1);
            const int y0 = max(cy - s, 0), y1 = min(cy + s, g.ny - 1);
            const int xa = max(cx - s, 0), xb = min(cx + s, g.nx - 1);
            for (int zz = z0; zz <= z1; ++zz)
                for (int yy = y0; yy <= y1; ++yy) {
                    const bool face = abs(zz - cz) == s || abs(yy - cy) == s;
                    // on the shell: whole rows on a z / y face, else the two x ends only
                    const int step = face ? 1 : max(1, 2 * s);
                    for (int xx = face ? xa : cx - s; xx <= (face ? xb : cx + s); xx += step) {
                        if (xx < 0 || xx >= g.nx) continue;
                        const int cell = (zz * g.ny + yy) * g.nx + xx;
                        const int b = __ldg(start + cell), e = b + __ldg(count + cell);
                        for (int t = b; t < e; ++t) {
                            const float4 q = __ldg(pts + t);
                            const float e0 = x0 - q.x, e1 = x1 - q.y, e2 = x2 - q.z;
                            const float df = fmaf(e2, e2, fmaf(e1, e1, e0 * e0));
                            if (df > thr && df >= 1e-30f) continue;
                            const int j = __float_as_int(q.w);
                            double D = -1.0;  // the candidate's FP64 value, formed on first need
                            // does the candidate precede list entry m?
                            auto precedes = [&](int m) -> bool {
                                // (values near FP32 underflow lose the relative bound: exact)
                                if (df >= 1e-30f && bf[m] >= 1e-30f) {
                                    if (df < bf[m] * (1.0f - 1e-6f)) return true;
                                    if (df > bf[m] * (1.0f + 1e-6f)) return false;
                                }
                                if (D < 0.0) D = dist2_rn(x0, x1, x2, q.x, q.y, q.z);
                                const float4 r = __ldg(pts + bt[m]);
                                const double Dm = dist2_rn(x0, x1, x2, r.x, r.y, r.z);
                                return D < Dm || (D == Dm && j < bi[m]);
                            };
                            if (n == K && !precedes(K - 1)) continue;
                            int pos = n < K ? n++ : K - 1;
                            while (pos > 0 && precedes(pos - 1)) {
                                bf[pos] = bf[pos - 1];
                                bi[pos] = bi[pos - 1];
                                bt[pos] = bt[pos - 1];
                                --pos;
                            }
                            bf[pos] = df;
                            bi[pos] = j;
                            bt[pos] = t;
                            if (n == K) thr = bf[K - 1] * (1.0f + 1e-6f);
                        }
                    }
                }
            // every unvisited cell lies at least s h from the point (less a rounding
            // margin); strictly closer K-th best: no unvisited point can precede it
            if (n == K) {
                const double bound = fmax(0.0, ((double)s - 1e-3) * (double)g.h);
                // an upper bound of the K-th distance's FP64 value
                const double kth = (double)bf[K - 1] * (1.0 + 1e-6);
                if (kth < bound * bound) break;
            }
        }
        for (int k = 0; k < K; ++k) {
            knn[(size_t)k * N + i] = k < n ? bi[k] : -1;
            if (dist2) {
                float dk = INFINITY;
                if (k < n) {
                    const float4 r = __ldg(pts + bt[k]);
                    dk = (float)dist2_rn(x0, x1, x2, r.x, r.y, r.z);
                }
                dist2[(size_t)k * N + i] = dk;
            }
        }
    }
}

struct KnnWs {
    int *box;       // [6]
    GridDev *grid;  // [1]
    int *count, *start, *cursor;  // [cap]
    int *totals;    // [ceil(cap / SCAN_BLOCK)]
    int *cell_of;   // [M]
    float4 *pts;    // [M] reference points in cell order (x, y, z, index)
    int *qcount, *qstart, *qcursor;  // [cap] queries per cell
    int *qtotals;   // [ceil(cap / SCAN_BLOCK)]
    int *qcell;     // [N]
    int *order;     // [N] queries in cell order
};

int cells_cap(int M) { return std::max(64, 2 * M); }

size_t knn_layout(const avatar_knn_args *a, void *base, size_t cap, KnnWs *out)
{
    WsCarver c(base, cap);
    const int C = cells_cap(a->M);
    KnnWs w;
    w.box = c.take<int>(6);
    w.grid = c.take<GridDev>(1);
    w.count = c.take<int>(C);
    w.start = c.take<int>(C);
    w.cursor = c.take<int>(C);
    w.totals = c.take<int>((C + SCAN_BLOCK - 1) / SCAN_BLOCK);
    w.cell_of = c.take<int>(a->M);
    w.pts = c.take<float4>(a->M);
    w.qcount = c.take<int>(C);
    w.qstart = c.take<int>(C);
    w.qcursor = c.take<int>(C);
    w.qtotals = c.take<int>((C + SCAN_BLOCK - 1) / SCAN_BLOCK);
    w.qcell = c.take<int>((size_t)std::max(a->N, 1));
    w.order = c.take<int>((size_t)std::max(a->N, 1));
    if (out) *out = w;
    return c.off;
}

int check_knn(const avatar_knn_args *a)
{
    if (!a || a->N < 0 || a->M < 1 || a->K < 1 || a->K > KNN_MAX_K || a->K > a->M) return AVATAR_ERR_INVALID_ARG;
    return AVATAR_OK;
}

template <int KMAX>
void launch_query(const avatar_knn_args *a, const KnnWs &w, int grid, cudaStream_t st)
{
    knn_query_kernel<KMAX><<<grid, KNN_THREADS, 0, st>>>(a->x, a->N, a->ref, a->M, a->K, w.grid, w.start, w.count,
                                                         w.pts, w.order, a->knn, a->dist2);
}

}  // namespace

extern "C" size_t avatar_knn_workspace_size(const avatar_knn_args *a)
{
    if (check_knn(a) != AVATAR_OK) return 0;
    return knn_layout(a, nullptr, 0, nullptr);
}

extern "C" int avatar_knn(avatar_ctx *ctx, const avatar_knn_args *a, void *ws, size_t ws_bytes,
                          avatar_stream_t stream)
{
    if (!ctx) return AVATAR_ERR_INVALID_ARG;
    AV_TRY(check_knn(a));
    if (!a->ref || (a->N > 0 && (!a->x || !a->knn))) return AVATAR_ERR_INVALID_ARG;
    if (!ws || (((uintptr_t)ws) & 255)) return AVATAR_ERR_WORKSPACE;
    KnnWs w;
    if (knn_layout(a, ws, ws_bytes, &w) > ws_bytes) return AVATAR_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    const int M = a->M, C = cells_cap(M);
    // box minima start at 0x7f7f7f7f and maxima at 0x80808080: above / below
    // the ordered integer of any finite float
    if (cudaMemsetAsync(w.box, 0x7f, 3 * sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(w.box + 3, 0x80, 3 * sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(w.count, 0, (size_t)C * sizeof(int), st) != cudaSuccess)
        return AVATAR_ERR_CUDA;
    const int gM = std::min((M + KNN_THREADS - 1) / KNN_THREADS, ctx->sm_count * 8);
    knn_bbox_kernel<<<gM, KNN_THREADS, 0, st>>>(a->ref, M, w.box);
    knn_grid_kernel<<<1, 1, 0, st>>>(w.box, M, C, w.grid);
    knn_count_kernel<<<gM, KNN_THREADS, 0, st>>>(a->ref, M, w.grid, w.count, w.cell_of);
    const int nb = (C + SCAN_BLOCK - 1) / SCAN_BLOCK;
    scan_totals_kernel<<<nb, SCAN_BLOCK, 0, st>>>(w.count, C, w.totals);
    scan_offsets_kernel<<<1, SCAN_BLOCK, 0, st>>>(w.totals, nb);
    scan_apply_kernel<<<nb, SCAN_BLOCK, 0, st>>>(w.count, C, w.totals, w.start, w.cursor);
    knn_scatter_kernel<<<gM, KNN_THREADS, 0, st>>>(a->ref, w.cell_of, M, w.cursor, w.pts);
    AV_CHECK_LAUNCH();
    if (a->N == 0) return AVATAR_OK;
    const int gN = std::min((a->N + KNN_THREADS - 1) / KNN_THREADS, ctx->sm_count * 16);
    // the queries in cell order (counting sort on the same grid)
    if (cudaMemsetAsync(w.qcount, 0, (size_t)C * sizeof(int), st) != cudaSuccess) return AVATAR_ERR_CUDA;
    knn_count_kernel<<<gN, KNN_THREADS, 0, st>>>(a->x, a->N, w.grid, w.qcount, w.qcell);
    scan_totals_kernel<<<nb, SCAN_BLOCK, 0, st>>>(w.qcount, C, w.qtotals);
    scan_offsets_kernel<<<1, SCAN_BLOCK, 0, st>>>(w.qtotals, nb);
    scan_apply_kernel<<<nb, SCAN_BLOCK, 0, st>>>(w.qcount, C, w.qtotals, w.qstart, w.qcursor);
    knn_order_kernel<<<gN, KNN_THREADS, 0, st>>>(w.qcell, a->N, w.qcursor, w.order);
    if (a->K <= 4) launch_query<4>(a, w, gN, st);
    else if (a->K <= 8) launch_query<8>(a, w, gN, st);
    else if (a->K <= 20) launch_query<20>(a, w, gN, st);
    else launch_query<KNN_MAX_K>(a, w, gN, st);
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}
