// (b) Visibility of the posed mesh toward D directions - Sec. 3.2, in its
// depth-map form: every direction gets an orthographic integer depth map of
// the posed mesh, and each vertex is depth-tested against it.
//
// GB300 layout: one thread-block cluster per direction holds that
// direction's R x R int32 depth map in the shared memory of its CL CTAs
// (row band r lives in CTA r / (R/CL)); triangles are spread over the whole
// cluster and write with atomicMin into the owning CTA's shared memory
// through distributed shared memory.  After a cluster barrier, every warp
// tests 32 vertices and forms one 32-bit word per direction with a ballot.
// The depth map never leaves shared memory.  A final ballot transpose turns
// direction-major words into vertex-major words (optionally re-ordered per
// light through d(k)).
//
// All arithmetic is exact integer arithmetic (bounds in the header), so the
// bits are reproducible bit for bit by any correct implementation.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int VIS_THREADS = 512;
constexpr int EMPTY_DEPTH = 0x7fffffff;

struct VisParams {
    int Nv, F, D, R, NW;
    int H, M, biasq;
    int rows_per_cta;
};

__global__ void vis_quantize_kernel(const float *__restrict__ xp, int Nv, int qc0, int qc1, int qc2,
                                    int4 *__restrict__ qv, int32_t *status)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < Nv; v += gridDim.x * blockDim.x) {
        int q0 = (int)rintf(xp[v] * 8192.0f) - qc0;
        int q1 = (int)rintf(xp[Nv + v] * 8192.0f) - qc1;
        int q2 = (int)rintf(xp[2 * Nv + v] * 8192.0f) - qc2;
        int bad = (q0 <= -65536 || q0 >= 65536 || q1 <= -65536 || q1 >= 65536 || q2 <= -65536 || q2 >= 65536);
        if (bad) {
            av_report(status, AVATAR_ERR_INVALID_ARG);
            q0 = q1 = q2 = 0;
        }
        qv[v] = make_int4(q0, q1, q2, bad);
    }
}

struct Proj {
    int X, Y, Z;
    bool in;
};

__device__ __forceinline__ Proj project_vertex(int4 q, const int *B, const VisParams &p)
{
    int s = B[0] * q.x + B[1] * q.y + B[2] * q.z;
    int t = B[3] * q.x + B[4] * q.y + B[5] * q.z;
    int z = B[6] * q.x + B[7] * q.y + B[8] * q.z;
    Proj r;
    r.X = (int)((((long long)s + p.H) * (long long)p.M) >> 32);
    r.Y = (int)((((long long)t + p.H) * (long long)p.M) >> 32);
    r.Z = (-z) >> 10;
    const int lim = 16 * p.R;
    r.in = (q.w == 0) && ((unsigned)r.X < (unsigned)lim) && ((unsigned)r.Y < (unsigned)lim);
    return r;
}

// floor(num / den) for den > 0 and a quotient known to be below 2^21 in
// magnitude: a float estimate (relative error < 2^-21.8) corrected by exact
// integer remainders.
__device__ __forceinline__ int floor_div_small(long long num, int den)
{
    long long q = (long long)floorf(__fdiv_rn((float)num, (float)den));
    long long r = num - q * (long long)den;
#pragma unroll
    for (int it = 0; it < 2; ++it)
        if (r < 0) {
            --q;
            r += den;
        }
#pragma unroll
    for (int it = 0; it < 2; ++it)
        if (r >= den) {
            ++q;
            r -= den;
        }
    return (int)q;
}

template <int CL>
__global__ void __launch_bounds__(VIS_THREADS)
vis_raster_test_kernel(VisParams p, const int4 *__restrict__ qv, const int32_t *__restrict__ faces,
                       const float *__restrict__ frames, uint32_t *__restrict__ dirbits, int32_t *status)
{
    extern __shared__ int slab[];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int d = blockIdx.y;
    const int R = p.R;
    const int slab_elems = p.rows_per_cta * R;

    for (int i = threadIdx.x; i < slab_elems; i += blockDim.x) slab[i] = EMPTY_DEPTH;

    int B[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) B[i] = (int)rintf(__ldg(frames + 9 * d + i) * 8192.0f);
    bool frame_ok = true;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        long long n2 = (long long)B[3 * r] * B[3 * r] + (long long)B[3 * r + 1] * B[3 * r + 1] +
                       (long long)B[3 * r + 2] * B[3 * r + 2];
        if (n2 > 8194LL * 8194LL) frame_ok = false;
    }
    if (!frame_ok) {
        if (threadIdx.x == 0) av_report(status, AVATAR_ERR_INVALID_ARG);
#pragma unroll
        for (int i = 0; i < 9; ++i) B[i] = 0;
    }

    int *slabs[CL];
#pragma unroll
    for (int c = 0; c < CL; ++c) slabs[c] = cluster.map_shared_rank(slab, c);
    cluster.sync();

    // ---- rasterise this CTA's share of the triangles
    const int stride = CL * blockDim.x;
    for (int f = rank * blockDim.x + threadIdx.x; f < p.F; f += stride) {
        int ia = __ldg(faces + 3 * f), ib = __ldg(faces + 3 * f + 1), ic = __ldg(faces + 3 * f + 2);
        if ((unsigned)ia >= (unsigned)p.Nv || (unsigned)ib >= (unsigned)p.Nv || (unsigned)ic >= (unsigned)p.Nv) {
            av_report(status, AVATAR_ERR_INDEX);
            continue;
        }
        Proj a = project_vertex(__ldg(qv + ia), B, p);
        Proj b = project_vertex(__ldg(qv + ib), B, p);
        Proj c = project_vertex(__ldg(qv + ic), B, p);
        if (!(a.in && b.in && c.in)) continue;
        int area = (b.X - a.X) * (c.Y - a.Y) - (b.Y - a.Y) * (c.X - a.X);
        if (area == 0) continue;
        if (area < 0) {
            Proj t = b;
            b = c;
            c = t;
            area = -area;
        }
        int xmin = min(a.X, min(b.X, c.X)), xmax = max(a.X, max(b.X, c.X));
        int ymin = min(a.Y, min(b.Y, c.Y)), ymax = max(a.Y, max(b.Y, c.Y));
        int i0 = max(0, (xmin + 7) >> 4), i1 = min(R - 1, (xmax - 8) >> 4);
        int j0 = max(0, (ymin + 7) >> 4), j1 = min(R - 1, (ymax - 8) >> 4);
        for (int j = j0; j <= j1; ++j) {
            const int py = 16 * j + 8;
            int *dst = slabs[j / p.rows_per_cta] + (j % p.rows_per_cta) * R;
            for (int i = i0; i <= i1; ++i) {
                const int px = 16 * i + 8;
                int wa = (c.X - b.X) * (py - b.Y) - (c.Y - b.Y) * (px - b.X);
                int wb = (a.X - c.X) * (py - c.Y) - (a.Y - c.Y) * (px - c.X);
                int wc = (b.X - a.X) * (py - a.Y) - (b.Y - a.Y) * (px - a.X);
                if ((wa | wb | wc) < 0) continue;
                long long num = (long long)wa * a.Z + (long long)wb * b.Z + (long long)wc * c.Z;
                atomicMin(dst + i, floor_div_small(num, area));
            }
        }
    }
    cluster.sync();

    // ---- depth-test vertices: one warp -> one 32-bit word of this direction
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    for (int w = rank * nwarps + warp; w < p.NW; w += CL * nwarps) {
        int v = w * 32 + lane;
        bool vis = false;
        if (v < p.Nv) {
            Proj q = project_vertex(__ldg(qv + v), B, p);
            if (!q.in) {
                vis = true;
            } else {
                int row = q.Y >> 4, col = q.X >> 4;
                int dep = slabs[row / p.rows_per_cta][(row % p.rows_per_cta) * R + col];
                vis = (dep == EMPTY_DEPTH) || (q.Z <= dep + p.biasq);
            }
        }
        unsigned word = __ballot_sync(0xffffffffu, vis);
        if (lane == 0) dirbits[(size_t)d * p.NW + w] = word;
    }
    cluster.sync();  // keep every slab alive until all remote reads are done
}

// bits[v][ow] bit l = dirbits[src(32 ow + l)][v/32] bit (v%32), src = dmap or identity.
__global__ void vis_transpose_kernel(const uint32_t *__restrict__ dirbits, int NW, int Nv, int D, int nout,
                                     int OW, const int32_t *__restrict__ dmap, uint32_t *__restrict__ bits,
                                     int32_t *status)
{
    const int lane = threadIdx.x & 31;
    const long total = (long)NW * OW;
    for (long t = (long)(blockIdx.x * blockDim.x + threadIdx.x) / 32; t < total;
         t += (long)gridDim.x * blockDim.x / 32) {
        int vw = (int)(t / OW), ow = (int)(t % OW);
        int k = ow * 32 + lane;
        unsigned src = 0;
        if (k < nout) {
            int dsrc = dmap ? __ldg(dmap + k) : k;
            if ((unsigned)dsrc >= (unsigned)D) {
                av_report(status, AVATAR_ERR_INDEX);
            } else {
                src = __ldg(dirbits + (size_t)dsrc * NW + vw);
            }
        }
        unsigned mine = 0;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            unsigned word = __ballot_sync(0xffffffffu, (src >> i) & 1u);
            if (lane == i) mine = word;
        }
        int v = vw * 32 + lane;
        if (v < Nv) bits[(size_t)v * OW + ow] = mine;
    }
}

template <int CL>
int launch_raster(const VisParams &p, const int4 *qv, const int32_t *faces, const float *frames,
                  uint32_t *dirbits, int32_t *status, size_t smem, cudaStream_t st)
{
    auto kern = vis_raster_test_kernel<CL>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return AVATAR_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, p.D, 1);
    cfg.blockDim = dim3(VIS_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kern, p, qv, faces, frames, dirbits, status) != cudaSuccess) {
        (void)cudaGetLastError();
        return AVATAR_ERR_CUDA;
    }
    return AVATAR_OK;
}

int cluster_size_for(int R)
{
    long bytes = (long)R * R * 4;
    int cl = (int)((bytes + 65535) / 65536);
    if (cl < 1) cl = 1;
    int p2 = 1;
    while (p2 < cl) p2 <<= 1;
    return p2 > 8 ? 8 : p2;
}

int check_vis(const avatar_vis_args *a)
{
    if (!a || a->Nv < 1 || a->F < 0 || a->D < 32 || a->D % 32 != 0 || a->D > 4096) return AVATAR_ERR_INVALID_ARG;
    if (a->R < 8 || a->R > 512 || a->R % 8 != 0) return AVATAR_ERR_INVALID_ARG;
    if (!a->xp || (a->F > 0 && !a->faces) || !a->frames || !a->bits) return AVATAR_ERR_INVALID_ARG;
    if (a->dmap && a->NL < 1) return AVATAR_ERR_INVALID_ARG;
    return AVATAR_OK;
}

struct VisWs {
    int4 *qv;
    uint32_t *dirbits;
};

size_t vis_ws_layout(const avatar_vis_args *a, void *base, size_t cap, VisWs *out)
{
    WsCarver c(base, cap);
    int NW = (a->Nv + 31) / 32;
    VisWs w;
    w.qv = c.take<int4>((size_t)a->Nv);
    w.dirbits = c.take<uint32_t>((size_t)a->D * NW);
    if (out) *out = w;
    return c.off;
}

}  // namespace

extern "C" size_t avatar_visibility_workspace_size(const avatar_vis_args *a)
{
    if (check_vis(a) != AVATAR_OK) return 0;
    return vis_ws_layout(a, nullptr, 0, nullptr);
}

extern "C" int avatar_visibility(avatar_ctx *ctx, const avatar_vis_args *a, void *ws, size_t ws_bytes,
                                 avatar_stream_t stream)
{
    if (!ctx) return AVATAR_ERR_INVALID_ARG;
    AV_TRY(check_vis(a));
    if (!ws || (((uintptr_t)ws) & 255)) return AVATAR_ERR_WORKSPACE;
    VisWs w;
    if (vis_ws_layout(a, ws, ws_bytes, &w) > ws_bytes) return AVATAR_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;

    long long H = llrint((double)a->half_extent * 67108864.0);
    if (!(H > 16LL * a->R && H <= (1LL << 30))) return AVATAR_ERR_INVALID_ARG;
    long long M = ((long long)a->R << 35) / H;
    if (M <= 0 || M >= (1LL << 31)) return AVATAR_ERR_INVALID_ARG;
    long long biasq = llrint((double)a->bias * 65536.0);
    if (biasq < 0 || biasq > (1LL << 30)) return AVATAR_ERR_INVALID_ARG;
    int qc[3];
    for (int i = 0; i < 3; ++i) {
        long long q = llrint((double)a->center[i] * 8192.0);
        if (q < -(1LL << 30) || q > (1LL << 30)) return AVATAR_ERR_INVALID_ARG;
        qc[i] = (int)q;
    }

    VisParams p;
    p.Nv = a->Nv;
    p.F = a->F;
    p.D = a->D;
    p.R = a->R;
    p.NW = (a->Nv + 31) / 32;
    p.H = (int)H;
    p.M = (int)M;
    p.biasq = (int)biasq;
    int CL = cluster_size_for(a->R);
    p.rows_per_cta = a->R / CL;
    size_t smem = (size_t)p.rows_per_cta * a->R * sizeof(int);

    int qgrid = (int)((a->Nv + 255) / 256);
    if (qgrid > ctx->sm_count * 8) qgrid = ctx->sm_count * 8;
    vis_quantize_kernel<<<qgrid, 256, 0, st>>>(a->xp, a->Nv, qc[0], qc[1], qc[2], w.qv, a->status);
    AV_CHECK_LAUNCH();

    int rc;
    switch (CL) {
        case 1: rc = launch_raster<1>(p, w.qv, a->faces, a->frames, w.dirbits, a->status, smem, st); break;
        case 2: rc = launch_raster<2>(p, w.qv, a->faces, a->frames, w.dirbits, a->status, smem, st); break;
        case 4: rc = launch_raster<4>(p, w.qv, a->faces, a->frames, w.dirbits, a->status, smem, st); break;
        default: rc = launch_raster<8>(p, w.qv, a->faces, a->frames, w.dirbits, a->status, smem, st); break;
    }
    if (rc != AVATAR_OK) return rc;

    int nout = a->dmap ? a->NL : a->D;
    int OW = (nout + 31) / 32;
    long warps = (long)p.NW * OW;
    long tgrid = (warps * 32 + 255) / 256;
    if (tgrid > (long)ctx->sm_count * 16) tgrid = (long)ctx->sm_count * 16;
    vis_transpose_kernel<<<(int)tgrid, 256, 0, st>>>(w.dirbits, p.NW, a->Nv, a->D, nout, OW, a->dmap, a->bits,
                                                      a->status);
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}
