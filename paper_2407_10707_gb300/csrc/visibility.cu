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
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "batch_internal.h"
#include "common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int VIS_THREADS = 256;
constexpr int EMPTY_DEPTH = 0x7fffffff;

struct VisParams {
    int B;  // poses in the launch (blockIdx.z)
    int Nv, F, D, R, NW;
    int H, M, biasq;
    int rows_per_cta;
    int inv_rows;  // ceil(2^20 / rows_per_cta): row / rows_per_cta == (row * inv_rows) >> 20 for row < 2^11
    int route;     // vertex words routed to the CTA owning their first vertex's depth row (inbox of NW ints)
};

// blockIdx.y = pose: xp holds gridDim.y poses ([3][B Nv]), qv [B Nv].
__global__ void vis_quantize_kernel(const float *__restrict__ xp, int Nv, int qc0, int qc1, int qc2,
                                    int4 *__restrict__ qv, int32_t *status)
{
    const size_t SN = (size_t)gridDim.y * Nv, op = (size_t)blockIdx.y * Nv;
    xp += op;
    qv += op;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < Nv; v += gridDim.x * blockDim.x) {
        int q0 = (int)rintf(xp[v] * 8192.0f) - qc0;
        int q1 = (int)rintf(xp[SN + v] * 8192.0f) - qc1;
        int q2 = (int)rintf(xp[2 * SN + v] * 8192.0f) - qc2;
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
    // X = floor((s + H) M / 2^32): one high-half multiply when s + H >= 0
    // (s + H < 2^31 by the bounds); s + H < 0 lies left of the window
    const int sh = s + p.H, th = t + p.H;
    r.X = sh >= 0 ? (int)__umulhi((unsigned)sh, (unsigned)p.M) : -1;
    r.Y = th >= 0 ? (int)__umulhi((unsigned)th, (unsigned)p.M) : -1;
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
    // estimate (|error| < 1.5), then the exact remainder decides the last step
    int q = (int)floorf(__fdividef((float)num, (float)den));
    int r = (int)(num - (long long)q * den);  // |r| < 3 den < 2^30
    if (r < 0) {
        --q;
        r += den;
        if (r < 0) {
            --q;
            r += den;
        }
    } else if (r >= den) {
        ++q;
        r -= den;
        if (r >= den) ++q;
    }
    return q;
}

// Packed projected vertex for the shared-memory cache: X | Y << 16 (0xffffffff
// = outside the window) and Z.
constexpr unsigned OUTSIDE = 0xffffffffu;
constexpr int VIS_CHUNK = AVATAR_VIS_FACE_CHUNK;  // triangles per CTA per chunk
constexpr int VIS_TPT = VIS_CHUNK / VIS_THREADS; // triangles per thread per chunk
constexpr int VIS_VCAP = 1024;                   // cached projected vertices per chunk (10-bit offsets)
static_assert(VIS_VCAP == 1024, "packed face offsets are 10 bits");
constexpr int VIS_SLAB_BYTES = 32 * 1024;        // depth-map share of one CTA (R <= 256)
constexpr size_t VIS_INBOX_MAX = 8 * 1024;       // routed vertex test: at most 2,048 words (65,536 vertices)

__device__ __forceinline__ uint2 pack_proj(const Proj &q)
{
    return make_uint2(q.in ? ((unsigned)q.X | ((unsigned)q.Y << 16)) : OUTSIDE, (unsigned)q.Z);
}

// floor(num / den) for 0 < den < 2^20 and a quotient below 2^10 in magnitude
// (|num| < 2^31): float estimate plus exact 32-bit remainder corrections.
__device__ __forceinline__ int floor_div_i32(int num, int den)
{
    int q = (int)floorf(__fdividef((float)num, (float)den));
    int r = num - q * den;
    if (r < 0) {
        --q;
        r += den;
        if (r < 0) --q;
    } else if (r >= den) {
        ++q;
        r -= den;
        if (r >= den) ++q;
    }
    return q;
}

template <int CL, bool CULL_BACK>
__device__ __forceinline__ void raster_triangle(uint2 pa, uint2 pb, uint2 pc, int *slab, const VisParams &p,
                                                cg::cluster_group &cluster)
{
    if (pa.x == OUTSIDE || pb.x == OUTSIDE || pc.x == OUTSIDE) return;
    int ax = pa.x & 0xffff, ay = pa.x >> 16, az = (int)pa.y;
    int bx = pb.x & 0xffff, by = pb.x >> 16, bz = (int)pb.y;
    int cx = pc.x & 0xffff, cy = pc.x >> 16, cz = (int)pc.y;
    const int R = p.R;
    // orientation first (two products: it drops the half of the triangles
    // that face away before the costlier box), then the pixel centres 16i+8
    // inside the bounding box (most triangles have none)
    int area = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
    if (CULL_BACK) {
        if (area <= 0) return;  // faces away from the light (outward winding)
    } else {
        if (area == 0) return;
        if (area < 0) {
            int t;
            t = bx; bx = cx; cx = t;
            t = by; by = cy; cy = t;
            t = bz; bz = cz; cz = t;
            area = -area;
        }
    }
    // pixel centres 16i+8 inside the box; every vertex lies in [0, 16R), so
    // i0 >= 0 and i1 <= R - 1 hold without clamps (i1 = -1 when all lie
    // left of the first centre)
    int i0 = (min(ax, min(bx, cx)) + 7) >> 4, i1 = (max(ax, max(bx, cx)) - 8) >> 4;
    int j0 = (min(ay, min(by, cy)) + 7) >> 4, j1 = (max(ay, max(by, cy)) - 8) >> 4;
    if (i0 > i1 || j0 > j1) return;
    // depth = az + floor((wb (bz - az) + wc (cz - az)) / area) since wa + wb + wc = area;
    // 32-bit arithmetic when the products provably fit, else 64-bit
    const int dzb = bz - az, dzc = cz - az;
    const bool small = area < (1 << 20) && abs(dzb) < (1 << 10) && abs(dzc) < (1 << 10);
    for (int j = j0; j <= j1; ++j) {
        const int py = 16 * j + 8;
        int *dst;
        if (CL == 1) {
            dst = slab + j * R;
        } else {
            int owner = (j * p.inv_rows) >> 20;  // exact j / rows_per_cta for j < 2^11
            dst = cluster.map_shared_rank(slab, owner) + (j - owner * p.rows_per_cta) * R;
        }
        for (int i = i0; i <= i1; ++i) {
            const int px = 16 * i + 8;
            int wa = (cx - bx) * (py - by) - (cy - by) * (px - bx);
            int wb = (ax - cx) * (py - cy) - (ay - cy) * (px - cx);
            int wc = (bx - ax) * (py - ay) - (by - ay) * (px - ax);
            if ((wa | wb | wc) < 0) continue;
            int dep;
            if (small) {
                dep = az + floor_div_i32(wb * dzb + wc * dzc, area);
            } else {
                long long num = (long long)wa * az + (long long)wb * bz + (long long)wc * cz;
                dep = floor_div_small(num, area);
            }
            atomicMin(dst + i, dep);
        }
    }
}

// Second pass of the paper's visibility: true iff at some pixel the triangle
// covers its depth (the same coverage and depth as raster_triangle) equals
// the finished depth map's - the triangle appears in the image.  Stops at
// the first such pixel.
template <int CL, bool CULL_BACK>
__device__ __forceinline__ bool triangle_appears(uint2 pa, uint2 pb, uint2 pc, const int *depth_slab,
                                                 const VisParams &p, cg::cluster_group &cluster)
{
    if (pa.x == OUTSIDE || pb.x == OUTSIDE || pc.x == OUTSIDE) return false;
    int ax = pa.x & 0xffff, ay = pa.x >> 16, az = (int)pa.y;
    int bx = pb.x & 0xffff, by = pb.x >> 16, bz = (int)pb.y;
    int cx = pc.x & 0xffff, cy = pc.x >> 16, cz = (int)pc.y;
    const int R = p.R;
    // pixel centres 16i+8 inside the box; every vertex lies in [0, 16R), so
    // i0 >= 0 and i1 <= R - 1 hold without clamps (i1 = -1 when all lie
    // left of the first centre)
    int i0 = (min(ax, min(bx, cx)) + 7) >> 4, i1 = (max(ax, max(bx, cx)) - 8) >> 4;
    int j0 = (min(ay, min(by, cy)) + 7) >> 4, j1 = (max(ay, max(by, cy)) - 8) >> 4;
    if (i0 > i1 || j0 > j1) return false;
    int area = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
    if (CULL_BACK) {
        if (area <= 0) return false;
    } else {
        if (area == 0) return false;
        if (area < 0) {
            int t;
            t = bx; bx = cx; cx = t;
            t = by; by = cy; cy = t;
            t = bz; bz = cz; cz = t;
            area = -area;
        }
    }
    const int dzb = bz - az, dzc = cz - az;
    const bool small = area < (1 << 20) && abs(dzb) < (1 << 10) && abs(dzc) < (1 << 10);
    for (int j = j0; j <= j1; ++j) {
        const int py = 16 * j + 8;
        const int *drow;
        if (CL == 1) {
            drow = depth_slab + j * R;
        } else {
            int owner = (j * p.inv_rows) >> 20;
            drow = cluster.map_shared_rank(depth_slab, owner) + (j - owner * p.rows_per_cta) * R;
        }
        for (int i = i0; i <= i1; ++i) {
            const int px = 16 * i + 8;
            int wa = (cx - bx) * (py - by) - (cy - by) * (px - bx);
            int wb = (ax - cx) * (py - cy) - (ay - cy) * (px - cx);
            int wc = (bx - ax) * (py - ay) - (by - ay) * (px - ax);
            if ((wa | wb | wc) < 0) continue;
            int dep;
            if (small) {
                dep = az + floor_div_i32(wb * dzb + wc * dzc, area);
            } else {
                long long num = (long long)wa * az + (long long)wb * bz + (long long)wc * cz;
                dep = floor_div_small(num, area);
            }
            if (dep == drow[i]) return true;
        }
    }
    return false;
}

// Direction-independent per-chunk vertex range [min, max] of the indices a
// chunk of VIS_CHUNK triangles references (x > y: a bad index, or no faces).
// With pf, the chunk's faces as offsets from the range's first vertex, 10
// bits each (a | b << 10 | c << 20), where the range fits the vertex cache.
__global__ void vis_chunk_ranges_kernel(const int32_t *__restrict__ faces, int F, int Nv, int2 *__restrict__ vr,
                                        int32_t *__restrict__ pf, int32_t *status)
{
    const int c = blockIdx.x;
    int vmin = 0x7fffffff, vmax = -1;
    bool bad = false;
    for (int f = c * VIS_CHUNK + threadIdx.x; f < min(F, (c + 1) * VIS_CHUNK); f += blockDim.x)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            int v = __ldg(faces + 3 * f + k);
            if ((unsigned)v >= (unsigned)Nv) bad = true;
            vmin = min(vmin, v);
            vmax = max(vmax, v);
        }
    __shared__ int smin, smax, sbad;
    if (threadIdx.x == 0) {
        smin = 0x7fffffff;
        smax = -1;
        sbad = 0;
    }
    __syncthreads();
    atomicMin(&smin, vmin);
    atomicMax(&smax, vmax);
    if (bad) atomicOr(&sbad, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (sbad) {
            av_report(status, AVATAR_ERR_INDEX);
            vr[c] = make_int2(1, 0);
        } else {
            vr[c] = make_int2(smin, smax);
        }
    }
    if (pf && !sbad && smax >= smin && smax - smin < VIS_VCAP)
        for (int f = c * VIS_CHUNK + threadIdx.x; f < min(F, (c + 1) * VIS_CHUNK); f += blockDim.x)
            pf[f] = (__ldg(faces + 3 * f) - smin) | ((__ldg(faces + 3 * f + 1) - smin) << 10) |
                    ((__ldg(faces + 3 * f + 2) - smin) << 20);
}

// NT threads per CTA: 256, or 512 with 4-CTA clusters (their 64 KB slabs hold
// two CTAs per SM, so 512 threads keep the resident warps of 8-CTA clusters
// of 256); at most 64 registers either way.
template <int CL, bool CULL_BACK, bool BATCH, int NT>
__global__ void __launch_bounds__(NT, NT == 512 ? 2 : 4)
vis_raster_test_kernel(VisParams p, const int4 *__restrict__ qv, const int32_t *__restrict__ faces,
                       const int32_t *__restrict__ pfaces, const int2 *__restrict__ vranges,
                       const float *__restrict__ frames, uint32_t *__restrict__ dirbits, int32_t *status)
{
    constexpr int TPT = VIS_CHUNK / NT;  // triangles per thread per chunk
    extern __shared__ int slab[];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = CL == 1 ? 0 : (int)cluster.block_rank();
    const int d = blockIdx.y;
    // pose blockIdx.z of a batch (its words: row z D + d below); a single pose
    // keeps qv in the parameter bank instead of a register pair
    if (BATCH) qv += (size_t)blockIdx.z * p.Nv;
    const int R = p.R;
    const int slab_elems = p.rows_per_cta * R;
    uint2 *vcache = reinterpret_cast<uint2 *>(slab + slab_elems);

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

    // packed faces of this CTA's first chunk (the next chunk's are prefetched
    // while the current one is rasterised); -1 past the last face
    int cur[TPT];
    auto load_faces = [&](int chunk, int (&dst)[TPT]) {
#pragma unroll
        for (int t = 0; t < TPT; ++t) {
            const int f = chunk * VIS_CHUNK + t * NT + threadIdx.x;
            dst[t] = f < p.F ? __ldg(pfaces + f) : -1;
        }
    };
    const int nchunks = (p.F + VIS_CHUNK - 1) / VIS_CHUNK;
    // Chunks after the first CL are handed out by a counter in rank 0's
    // shared memory (one remote atomic per chunk), so a CTA that draws cheap
    // chunks (mostly back-facing) takes more and the cluster reaches its
    // barrier together; the depth map is a minimum, so the order is free.
    __shared__ int s_chunk_ctr, s_next;
    __shared__ int s_in_count, s_in_next;  // this CTA's inbox of vertex words (routed test)
    int *inbox = reinterpret_cast<int *>(vcache + VIS_VCAP);
    int chunk = rank;
    if (CL > 1 && rank == 0 && threadIdx.x == 0) s_chunk_ctr = CL;
    if (threadIdx.x == 0) {
        s_in_count = 0;
        s_in_next = 0;
    }
    if (chunk < nchunks) load_faces(chunk, cur);
    cluster.sync();

    while (chunk < nchunks) {
        int taken = 0;
        if (threadIdx.x == 0) {
            if constexpr (CL == 1)
                taken = chunk + 1;
            else
                taken = atomicAdd(cluster.map_shared_rank(&s_chunk_ctr, 0), 1);
        }
        const int2 vr = __ldg(vranges + chunk);
        const int v0 = vr.x, nv = vr.y - vr.x + 1;
        // nv <= 0: a bad index (reported) or no faces; the packed offsets
        // exist only where the range fits the cache
        const bool cached = nv > 0 && nv <= VIS_VCAP;
        if (cached) {
#pragma unroll 4
            for (int i = threadIdx.x; i < nv; i += NT)
                vcache[i] = pack_proj(project_vertex(__ldg(qv + v0 + i), B, p));
        }
        if (threadIdx.x == 0) s_next = taken;
        __syncthreads();
        const int next = s_next;
        int nxt[TPT];
        if (next < nchunks) load_faces(next, nxt);
        if (nv > 0) {
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                const int f = chunk * VIS_CHUNK + t * NT + threadIdx.x;
                if (f >= p.F) continue;
                uint2 pa, pb, pc;
                if (cached) {
                    pa = vcache[cur[t] & 1023];
                    pb = vcache[(cur[t] >> 10) & 1023];
                    pc = vcache[(cur[t] >> 20) & 1023];
                } else {
                    pa = pack_proj(project_vertex(__ldg(qv + __ldg(faces + 3 * f)), B, p));
                    pb = pack_proj(project_vertex(__ldg(qv + __ldg(faces + 3 * f + 1)), B, p));
                    pc = pack_proj(project_vertex(__ldg(qv + __ldg(faces + 3 * f + 2)), B, p));
                }
                raster_triangle<CL, CULL_BACK>(pa, pb, pc, slab, p, cluster);
            }
        }
        __syncthreads();  // the next chunk overwrites the cache (and s_next)
#pragma unroll
        for (int t = 0; t < TPT; ++t) cur[t] = nxt[t];
        chunk = next;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = NT / 32;
    const int wstride = CL * nwarps;
    if (CL > 1 && p.route) {
        // route every vertex word to the CTA owning the depth row of its
        // first vertex: a word's 32 vertices lie close on the surface, so
        // that CTA reads most of their depths from its own slab
        for (int wb = (rank * nwarps + warp) * 32; wb < p.NW; wb += wstride * 32) {
            const int w = wb + lane;
            if (w < p.NW) {
                int owner = rank;
                const Proj pr = project_vertex(__ldg(qv + (size_t)w * 32), B, p);
                if (pr.in) owner = ((pr.Y >> 4) * p.inv_rows) >> 20;
                const int slot = atomicAdd(cluster.map_shared_rank(&s_in_count, owner), 1);
                cluster.map_shared_rank(inbox, owner)[slot] = w;
            }
        }
    }
    cluster.sync();

    // ---- depth-test vertices: one warp -> 32-bit words of this direction,
    // four words in flight per iteration (a word index of -1: none)
    auto test_words = [&](const int (&ws)[4]) {
        int4 qq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int v = ws[u] * 32 + lane;
            qq[u] = (ws[u] >= 0 && v < p.Nv) ? __ldg(qv + v) : make_int4(0, 0, 0, 2);
        }
        int dep[4];
        Proj pr[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            pr[u] = project_vertex(qq[u], B, p);
            dep[u] = EMPTY_DEPTH;
            if (pr[u].in) {
                int row = pr[u].Y >> 4, col = pr[u].X >> 4;
                int owner = CL == 1 ? 0 : (row * p.inv_rows) >> 20;
                const int *src = CL == 1 ? slab : cluster.map_shared_rank(slab, owner);
                dep[u] = src[(row - owner * p.rows_per_cta) * R + col];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            bool vis = !pr[u].in || dep[u] == EMPTY_DEPTH || pr[u].Z <= dep[u] + p.biasq;
            unsigned word = __ballot_sync(0xffffffffu, vis && qq[u].w != 2);
            if (lane == 0 && ws[u] >= 0) dirbits[((size_t)blockIdx.z * p.D + d) * p.NW + ws[u]] = word;
        }
    };
    if (CL > 1 && p.route) {
        // this CTA's inbox first, then the others' (a CTA whose slab holds
        // much of the body has more words than the rest): four words per grab
        for (int k = 0; k < CL; ++k) {
            const int owner = rank + k < CL ? rank + k : rank + k - CL;
            int *nextp = cluster.map_shared_rank(&s_in_next, owner);
            const int count = *cluster.map_shared_rank(&s_in_count, owner);
            const int *box = cluster.map_shared_rank(inbox, owner);
            for (;;) {
                int base = 0;
                if (lane == 0) base = atomicAdd(nextp, 4);
                base = __shfl_sync(0xffffffffu, base, 0);
                if (base >= count) break;
                int ws[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) ws[u] = base + u < count ? box[base + u] : -1;
                test_words(ws);
            }
        }
    } else {
        for (int w0 = rank * nwarps + warp; w0 < p.NW; w0 += 4 * wstride) {
            int ws[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) ws[u] = w0 + u * wstride < p.NW ? w0 + u * wstride : -1;
            test_words(ws);
        }
    }
    cluster.sync();  // keep every slab alive until all remote reads are done
}

// bits[v][ow] bit l = dirbits[src(32 ow + l)][v/32] bit (v%32), src = dmap or identity.
// A block takes TR_VW consecutive vertex words and TR_ROWS outputs (lights):
// blockIdx.x the vertex words, blockIdx.y the outputs, blockIdx.z the pose of
// a batch.  It stages, per output, the source direction's TR_VW words (one
// 32-byte sector) in shared memory with all its loads in flight at once; warp
// w then transposes the 32 x 32 bit blocks of vertex word w by five
// shuffle-xor exchange rounds (a lane starts with one output's 32 vertex bits
// and ends with its vertex's 32 output bits), and every lane writes its
// vertex's TR_ROWS / 32 words, in one 16-byte store when OW is a multiple of
// four.
constexpr int TR_VW = 8, TR_ROWS = 128, TR_THREADS = 256;
constexpr int TR_PER = TR_ROWS * TR_VW / TR_THREADS;  // staged words per thread

__device__ __forceinline__ uint32_t transpose32_lane(uint32_t x, int lane)
{
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        const uint32_t m = j == 16 ? 0x0000ffffu : j == 8 ? 0x00ff00ffu : j == 4 ? 0x0f0f0f0fu
                         : j == 2 ? 0x33333333u : 0x55555555u;
        const uint32_t t = __shfl_xor_sync(0xffffffffu, x, j);
        x = (lane & j) ? ((x & ~m) | ((t & ~m) >> j)) : ((x & m) | ((t & m) << j));
    }
    return x;
}

__global__ void __launch_bounds__(TR_THREADS)
vis_transpose_kernel(const uint32_t *__restrict__ dirbits, int NW, int Nv, int D, int nout, int OW,
                     const int32_t *__restrict__ dmap, uint32_t *__restrict__ bits, int32_t *status)
{
    __shared__ uint32_t tile[TR_ROWS][TR_VW + 1];  // padded: a column read is conflict-free
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    dirbits += (size_t)blockIdx.z * D * NW;  // pose blockIdx.z of a batch
    bits += (size_t)blockIdx.z * Nv * OW;
    const int vw0 = blockIdx.x * TR_VW, k0 = blockIdx.y * TR_ROWS;
    int dsrc[TR_PER];
#pragma unroll
    for (int u = 0; u < TR_PER; ++u) {
        const int k = k0 + (threadIdx.x + u * TR_THREADS) / TR_VW;
        dsrc[u] = k < nout ? (dmap ? __ldg(dmap + k) : k) : D;   // D: no output there (a zero word)
    }
    uint32_t word[TR_PER];
#pragma unroll
    for (int u = 0; u < TR_PER; ++u) {
        const int i = threadIdx.x + u * TR_THREADS, c = i % TR_VW, k = k0 + i / TR_VW;
        word[u] = 0u;
        if ((unsigned)dsrc[u] < (unsigned)D) {
            if (vw0 + c < NW) word[u] = __ldg(dirbits + (size_t)dsrc[u] * NW + vw0 + c);
        } else if (k < nout && c == 0) {
            av_report(status, AVATAR_ERR_INDEX);
        }
    }
#pragma unroll
    for (int u = 0; u < TR_PER; ++u) {
        const int i = threadIdx.x + u * TR_THREADS;
        tile[i / TR_VW][i % TR_VW] = word[u];
    }
    __syncthreads();
    const int vw = vw0 + warp, v = vw * 32 + lane;
    if (vw >= NW) return;
    const int ow0 = k0 / 32, nspan = min(TR_ROWS / 32, OW - ow0);
    uint32_t out[TR_ROWS / 32];
#pragma unroll
    for (int q = 0; q < TR_ROWS / 32; ++q)
        out[q] = q < nspan ? transpose32_lane(tile[q * 32 + lane][warp], lane) : 0u;  // nspan is warp-uniform
    if (v >= Nv) return;
    uint32_t *dst = bits + (size_t)v * OW + ow0;
    if (nspan == 4 && (OW & 3) == 0 && (reinterpret_cast<uintptr_t>(bits) & 15) == 0) {
        *reinterpret_cast<uint4 *>(dst) = make_uint4(out[0], out[1], out[2], out[3]);
    } else {
#pragma unroll
        for (int q = 0; q < TR_ROWS / 32; ++q)
            if (q < nspan) dst[q] = out[q];
    }
}

// ---------------------------------------------------------------------------
// The paper's own visibility (Sec. 3.2, Eqs. 3-4): triangle-ID images and the
// median / median / mean vertex filters.
//
// vis_tri_kernel: one cluster per direction holds the direction's R x R
// depth map in its CTAs' shared memory.  Pass A is the depth-map raster;
// pass B visits the triangles again and marks, in the CTA's shared-memory
// bitmap, the vertices of every triangle that attains the least depth at a
// pixel it covers (it appears in the triangle-ID image).  The cluster then
// ORs the bitmaps (plus the vertices outside the window) into
// direction-major words.
template <int CL, bool CULL_BACK>
__global__ void __launch_bounds__(VIS_THREADS)
vis_tri_kernel(VisParams p, const int4 *__restrict__ qv, const int32_t *__restrict__ faces,
               const int2 *__restrict__ vranges, const float *__restrict__ frames, uint32_t *__restrict__ dirbits,
               int32_t *status)
{
    extern __shared__ int depth[];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = CL == 1 ? 0 : (int)cluster.block_rank();
    const int d = blockIdx.y;
    const int R = p.R;
    const int slab_elems = p.rows_per_cta * R;
    uint2 *vcache = reinterpret_cast<uint2 *>(depth + slab_elems);
    unsigned *bitmap = reinterpret_cast<unsigned *>(vcache + VIS_VCAP);  // [NW] vertices marked by this CTA

    for (int i = threadIdx.x; i < slab_elems; i += blockDim.x) depth[i] = EMPTY_DEPTH;
    for (int i = threadIdx.x; i < p.NW; i += blockDim.x) bitmap[i] = 0u;

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
    const int nchunks = (p.F + VIS_CHUNK - 1) / VIS_CHUNK;
    cluster.sync();
    for (int pass = 0; pass < 2; ++pass) {
        for (int chunk = rank; chunk < nchunks; chunk += CL) {
            const int2 vr = __ldg(vranges + chunk);
            const int v0 = vr.x, nv = vr.y - vr.x + 1;
            const bool cached = nv > 0 && nv <= VIS_VCAP;
            if (cached)
                for (int i = threadIdx.x; i < nv; i += VIS_THREADS)
                    vcache[i] = pack_proj(project_vertex(__ldg(qv + v0 + i), B, p));
            __syncthreads();
            if (nv > 0) {
#pragma unroll
                for (int t = 0; t < VIS_TPT; ++t) {
                    const int f = chunk * VIS_CHUNK + t * VIS_THREADS + threadIdx.x;
                    if (f >= p.F) continue;
                    const int a = __ldg(faces + 3 * f), b = __ldg(faces + 3 * f + 1), c = __ldg(faces + 3 * f + 2);
                    uint2 pa, pb, pc;
                    if (cached) {
                        pa = vcache[a - v0];
                        pb = vcache[b - v0];
                        pc = vcache[c - v0];
                    } else {
                        pa = pack_proj(project_vertex(__ldg(qv + a), B, p));
                        pb = pack_proj(project_vertex(__ldg(qv + b), B, p));
                        pc = pack_proj(project_vertex(__ldg(qv + c), B, p));
                    }
                    if (pass == 0) {
                        raster_triangle<CL, CULL_BACK>(pa, pb, pc, depth, p, cluster);
                    } else if (triangle_appears<CL, CULL_BACK>(pa, pb, pc, depth, p, cluster)) {
                        atomicOr(bitmap + (a >> 5), 1u << (a & 31));
                        atomicOr(bitmap + (b >> 5), 1u << (b & 31));
                        atomicOr(bitmap + (c >> 5), 1u << (c & 31));
                    }
                }
            }
            __syncthreads();  // the next chunk overwrites the cache
        }
        cluster.sync();  // the depth map is complete before pass B; every bitmap before the OR
    }
    // one warp per 32-vertex word: OR of the cluster's bitmaps and the
    // vertices outside the window (visible, as in the depth-map form)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = VIS_THREADS / 32;
    for (int w = rank * nwarps + warp; w < p.NW; w += CL * nwarps) {
        const int v = w * 32 + lane;
        const bool outside = v < p.Nv && !project_vertex(__ldg(qv + v), B, p).in;
        unsigned word = __ballot_sync(0xffffffffu, outside);
        if (lane < CL) {
            const unsigned *src = CL == 1 ? bitmap : cluster.map_shared_rank(bitmap, lane);
            word |= src[w];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) word |= __shfl_xor_sync(0xffffffffu, word, o);
        if (lane == 0) dirbits[(size_t)d * p.NW + w] = word;
    }
    cluster.sync();  // keep every bitmap alive until all remote reads are done
}

// Bit-sliced count of Kv neighbour words: planes c[0..5] hold, per bit
// position, the count of ones in binary (Kv <= 63).
__device__ __forceinline__ void count_neighbours(const uint32_t *__restrict__ in, const int32_t *__restrict__ knn_v,
                                                 int Nv, int OW, int Kv, int v, int w, unsigned (&c)[6],
                                                 int32_t *status)
{
#pragma unroll
    for (int b = 0; b < 6; ++b) c[b] = 0u;
    for (int j = 0; j < Kv; ++j) {
        const int u = __ldg(knn_v + (size_t)j * Nv + v);
        if ((unsigned)u >= (unsigned)Nv) {
            av_report(status, AVATAR_ERR_INDEX);
            continue;
        }
        unsigned carry = __ldg(in + (size_t)u * OW + w);
#pragma unroll
        for (int b = 0; b < 6; ++b) {
            const unsigned t = c[b] & carry;
            c[b] ^= carry;
            carry = t;
        }
    }
}

// median filter: bit = (count >= (Kv + 1) / 2), per vertex and 32 directions
__global__ void __launch_bounds__(256)
vis_median_kernel(const uint32_t *__restrict__ in, const int32_t *__restrict__ knn_v, int Nv, int OW, int Kv,
                  uint32_t *__restrict__ out, int32_t *status)
{
    const int m = (Kv + 1) / 2;
    const long total = (long)Nv * OW;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int v = (int)(t / OW), w = (int)(t % OW);
        unsigned c[6];
        count_neighbours(in, knn_v, Nv, OW, Kv, v, w, c, status);
        // count >= m, bit-sliced from the most significant plane down
        unsigned gt = 0u, eq = ~0u;
#pragma unroll
        for (int b = 5; b >= 0; --b) {
            if ((m >> b) & 1) {
                eq &= c[b];
            } else {
                gt |= eq & c[b];
                eq &= ~c[b];
            }
        }
        out[(size_t)v * OW + w] = gt | eq;
    }
}

// mean filter: count in 0..Kv per vertex and direction, written in light
// order (light k takes direction dmap[k]) or direction order (dmap NULL)
__global__ void __launch_bounds__(256)
vis_mean_kernel(const uint32_t *__restrict__ in, const int32_t *__restrict__ knn_v, int Nv, int OW, int Kv,
                uint8_t *__restrict__ dir_count, int32_t *status)
{
    const long total = (long)Nv * OW;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int v = (int)(t / OW), w = (int)(t % OW);
        unsigned c[6];
        count_neighbours(in, knn_v, Nv, OW, Kv, v, w, c, status);
        uint32_t packed[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            uint32_t word = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int bit = 4 * q + k;
                unsigned n = 0;
#pragma unroll
                for (int b = 0; b < 6; ++b) n |= ((c[b] >> bit) & 1u) << b;
                word |= n << (8 * k);
            }
            packed[q] = word;
        }
        uint4 *dst = reinterpret_cast<uint4 *>(dir_count + (size_t)v * OW * 32 + (size_t)w * 32);
        dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
    }
}

__global__ void __launch_bounds__(256)
vis_light_order_kernel(const uint8_t *__restrict__ dir_count, int Nv, int D, int NL, const int32_t *__restrict__ dmap,
                       uint8_t *__restrict__ out, int32_t *status)
{
    const long total = (long)Nv * NL;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int v = (int)(t / NL), k = (int)(t % NL);
        const int d = __ldg(dmap + k);
        uint8_t c = 0;
        if ((unsigned)d >= (unsigned)D) av_report(status, AVATAR_ERR_INDEX);
        else c = dir_count[(size_t)v * D + d];
        out[t] = c;
    }
}

template <int CL, bool CULL_BACK>
int launch_tri(const VisParams &p, const int4 *qv, const int32_t *faces, const int2 *vranges, const float *frames,
               uint32_t *dirbits, int32_t *status, size_t smem, cudaStream_t st)
{
    auto kern = vis_tri_kernel<CL, CULL_BACK>;
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
    if (cudaLaunchKernelEx(&cfg, kern, p, qv, faces, vranges, frames, dirbits, status) != cudaSuccess) {
        (void)cudaGetLastError();
        return AVATAR_ERR_CUDA;
    }
    return AVATAR_OK;
}

template <int CL, bool CULL_BACK>
int launch_raster(const VisParams &p, const int4 *qv, const int32_t *faces, const int32_t *pfaces,
                  const int2 *vranges, const float *frames, uint32_t *dirbits, int32_t *status, size_t smem,
                  cudaStream_t st)
{
    constexpr int NT = CL == 4 ? 512 : 256;
    auto kern = p.B > 1 ? vis_raster_test_kernel<CL, CULL_BACK, true, NT> : vis_raster_test_kernel<CL, CULL_BACK, false, NT>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return AVATAR_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, p.D, p.B);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kern, p, qv, faces, pfaces, vranges, frames, dirbits, status) != cudaSuccess) {
        (void)cudaGetLastError();
        return AVATAR_ERR_CUDA;
    }
    return AVATAR_OK;
}

int cluster_size_for(int R)
{
    long bytes = (long)R * R * 4;
    int cl = (int)((bytes + VIS_SLAB_BYTES - 1) / VIS_SLAB_BYTES);
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
    int2 *vranges;
    int32_t *pfaces;  // [F] packed chunk-relative faces
};

size_t vis_ws_layout(const avatar_vis_args *a, int B, void *base, size_t cap, VisWs *out)
{
    WsCarver c(base, cap);
    int NW = (a->Nv + 31) / 32;
    VisWs w;
    w.qv = c.take<int4>((size_t)B * a->Nv);
    w.dirbits = c.take<uint32_t>((size_t)B * a->D * NW);
    w.vranges = c.take<int2>((size_t)(a->F + VIS_CHUNK - 1) / VIS_CHUNK + 1);
    w.pfaces = c.take<int32_t>((size_t)a->F + 1);
    if (out) *out = w;
    return c.off;
}

}  // namespace

extern "C" size_t avatar_visibility_workspace_size(const avatar_vis_args *a)
{
    if (check_vis(a) != AVATAR_OK) return 0;
    return vis_ws_layout(a, 1, nullptr, 0, nullptr);
}

namespace {

// Visibility of B poses at once: xp [3][B Nv], bits [B Nv][OW] (pose p's
// vertices at rows p Nv ...); one launch per step for the whole batch.
int vis_run(avatar_ctx *ctx, const avatar_vis_args *a, int B, void *ws, size_t ws_bytes, cudaStream_t st)
{
    if (!ctx || B < 1) return AVATAR_ERR_INVALID_ARG;
    AV_TRY(check_vis(a));
    if (!ws || (((uintptr_t)ws) & 255)) return AVATAR_ERR_WORKSPACE;
    VisWs w;
    if (vis_ws_layout(a, B, ws, ws_bytes, &w) > ws_bytes) return AVATAR_ERR_WORKSPACE;

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
    p.B = B;
    p.Nv = a->Nv;
    p.F = a->F;
    p.D = a->D;
    p.R = a->R;
    p.NW = (a->Nv + 31) / 32;
    p.H = (int)H;
    p.M = (int)M;
    p.biasq = (int)biasq;
    int CL = ctx->tune[AVATAR_TUNE_VIS_CLUSTER] ? ctx->tune[AVATAR_TUNE_VIS_CLUSTER] : cluster_size_for(a->R);
    while (CL < 8 && (size_t)(a->R / CL) * a->R * sizeof(int) + (size_t)VIS_VCAP * sizeof(uint2) >
                         (size_t)ctx->max_smem_optin)
        CL <<= 1;
    p.rows_per_cta = a->R / CL;
    p.inv_rows = ((1 << 20) + p.rows_per_cta - 1) / p.rows_per_cta;
    size_t smem = (size_t)p.rows_per_cta * a->R * sizeof(int) + (size_t)VIS_VCAP * sizeof(uint2);
    // the routed vertex test keeps an inbox of word indices per CTA (a CTA
    // may receive every word), where it fits beside four slabs per SM
    const size_t inbox = ((size_t)p.NW * sizeof(int) + 15) & ~(size_t)15;
    p.route = CL > 1 && inbox <= VIS_INBOX_MAX && smem + inbox <= (size_t)ctx->max_smem_optin;
    if (p.route) smem += inbox;

    int qgrid = (int)((a->Nv + 255) / 256);
    if (qgrid > ctx->sm_count * 8) qgrid = ctx->sm_count * 8;
    vis_quantize_kernel<<<dim3(qgrid, B), 256, 0, st>>>(a->xp, a->Nv, qc[0], qc[1], qc[2], w.qv, a->status);
    AV_CHECK_LAUNCH();

    int nchunks = (a->F + VIS_CHUNK - 1) / VIS_CHUNK;
    if (nchunks > 0) {
        vis_chunk_ranges_kernel<<<nchunks, 256, 0, st>>>(a->faces, a->F, a->Nv, w.vranges, w.pfaces, a->status);
        AV_CHECK_LAUNCH();
    }
    int rc;
    const bool cb = a->cull_back != 0;
#define AV_RASTER(CLV)                                                                                          \
    (cb ? launch_raster<CLV, true>(p, w.qv, a->faces, w.pfaces, w.vranges, a->frames, w.dirbits, a->status, smem,   \
                                   st)                                                                              \
        : launch_raster<CLV, false>(p, w.qv, a->faces, w.pfaces, w.vranges, a->frames, w.dirbits, a->status, smem, \
                                    st))
    switch (CL) {
        case 1: rc = AV_RASTER(1); break;
        case 2: rc = AV_RASTER(2); break;
        case 4: rc = AV_RASTER(4); break;
        default: rc = AV_RASTER(8); break;
    }
#undef AV_RASTER
    if (rc != AVATAR_OK) return rc;

    int nout = a->dmap ? a->NL : a->D;
    int OW = (nout + 31) / 32;
    const int tgrid = (p.NW + TR_VW - 1) / TR_VW, tspans = (nout + TR_ROWS - 1) / TR_ROWS;
    vis_transpose_kernel<<<dim3(tgrid, tspans, B), TR_THREADS, 0, st>>>(w.dirbits, p.NW, a->Nv, a->D, nout, OW, a->dmap,
                                                               a->bits, a->status);
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}

}  // namespace

size_t av_visibility_batch_workspace_size(const avatar_vis_args *a, int B)
{
    if (check_vis(a) != AVATAR_OK || B < 1) return 0;
    return vis_ws_layout(a, B, nullptr, 0, nullptr);
}

int av_visibility_batch(avatar_ctx *ctx, const avatar_vis_args *a, int B, void *ws, size_t ws_bytes, cudaStream_t st)
{
    return vis_run(ctx, a, B, ws, ws_bytes, st);
}

extern "C" int avatar_visibility(avatar_ctx *ctx, const avatar_vis_args *a, void *ws, size_t ws_bytes,
                                 avatar_stream_t stream)
{
    return vis_run(ctx, a, 1, ws, ws_bytes, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// The paper's visibility with its filters (header: avatar_visibility_soft).
namespace {

struct VisSoftWs {
    int4 *qv;
    uint32_t *dirbits;
    int2 *vranges;
    uint32_t *vm, *m1, *m2;  // [Nv][D/32] vertex-major, direction order
    uint8_t *dir_count;      // [Nv][D]
};

int check_vis_soft(const avatar_vis_soft_args *a)
{
    if (!a) return AVATAR_ERR_INVALID_ARG;
    const avatar_vis_args &b = a->base;
    if (b.Nv < 1 || b.F < 0 || b.D < 32 || b.D % 32 != 0 || b.D > 4096) return AVATAR_ERR_INVALID_ARG;
    if (b.R < 8 || b.R > 512 || b.R % 8 != 0) return AVATAR_ERR_INVALID_ARG;
    if (a->Kv < 1 || a->Kv > 63 || a->Kv % 2 == 0) return AVATAR_ERR_INVALID_ARG;
    if (b.dmap && b.NL < 1) return AVATAR_ERR_INVALID_ARG;
    return AVATAR_OK;
}

size_t vis_soft_layout(const avatar_vis_soft_args *a, void *base, size_t cap, VisSoftWs *out)
{
    WsCarver c(base, cap);
    const avatar_vis_args &b = a->base;
    const int NW = (b.Nv + 31) / 32, OW = b.D / 32;
    VisSoftWs w;
    w.qv = c.take<int4>((size_t)b.Nv);
    w.dirbits = c.take<uint32_t>((size_t)b.D * NW);
    w.vranges = c.take<int2>((size_t)(b.F + VIS_CHUNK - 1) / VIS_CHUNK + 1);
    w.vm = c.take<uint32_t>((size_t)b.Nv * OW);
    w.m1 = c.take<uint32_t>((size_t)b.Nv * OW);
    w.m2 = c.take<uint32_t>((size_t)b.Nv * OW);
    w.dir_count = c.take<uint8_t>((size_t)b.Nv * b.D);
    if (out) *out = w;
    return c.off;
}

// Shared memory of one CTA of the triangle-ID kernel with CL CTAs per direction.
size_t tri_smem(int R, int CL, int Nv)
{
    return (size_t)(R / CL) * R * sizeof(int) + (size_t)VIS_VCAP * sizeof(uint2) +
           (size_t)((Nv + 31) / 32) * sizeof(unsigned);
}

// CTAs per direction: as many as the depth-map form uses (32 KB of map per
// CTA), more only if the map share and the bitmap would not fit one SM
int tri_cluster_size(int R, int Nv, int smem_cap)
{
    for (int cl = cluster_size_for(R); cl <= 8; cl <<= 1)
        if (R % cl == 0 && tri_smem(R, cl, Nv) <= (size_t)smem_cap) return cl;
    return 0;
}

}  // namespace

extern "C" size_t avatar_visibility_soft_workspace_size(const avatar_vis_soft_args *a)
{
    if (check_vis_soft(a) != AVATAR_OK) return 0;
    return vis_soft_layout(a, nullptr, 0, nullptr);
}

extern "C" int avatar_visibility_soft(avatar_ctx *ctx, const avatar_vis_soft_args *a, void *ws, size_t ws_bytes,
                                      avatar_stream_t stream)
{
    if (!ctx) return AVATAR_ERR_INVALID_ARG;
    AV_TRY(check_vis_soft(a));
    const avatar_vis_args &b = a->base;
    if (!b.xp || (b.F > 0 && !b.faces) || !b.frames || !a->knn_v || !a->vis_count) return AVATAR_ERR_INVALID_ARG;
    // direction-ordered counts are written 16 bytes at a time
    if (!b.dmap && (((uintptr_t)a->vis_count) & 15)) return AVATAR_ERR_INVALID_ARG;
    if (!ws || (((uintptr_t)ws) & 255)) return AVATAR_ERR_WORKSPACE;
    VisSoftWs w;
    if (vis_soft_layout(a, ws, ws_bytes, &w) > ws_bytes) return AVATAR_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    long long H = llrint((double)b.half_extent * 67108864.0);
    if (!(H > 16LL * b.R && H <= (1LL << 30))) return AVATAR_ERR_INVALID_ARG;
    long long M = ((long long)b.R << 35) / H;
    if (M <= 0 || M >= (1LL << 31)) return AVATAR_ERR_INVALID_ARG;
    int qc[3];
    for (int i = 0; i < 3; ++i) {
        long long q = llrint((double)b.center[i] * 8192.0);
        if (q < -(1LL << 30) || q > (1LL << 30)) return AVATAR_ERR_INVALID_ARG;
        qc[i] = (int)q;
    }
    VisParams p;
    p.route = 0;
    p.B = 1;
    p.Nv = b.Nv;
    p.F = b.F;
    p.D = b.D;
    p.R = b.R;
    p.NW = (b.Nv + 31) / 32;
    p.H = (int)H;
    p.M = (int)M;
    p.biasq = 0;
    const int CL = tri_cluster_size(b.R, b.Nv, ctx->max_smem_optin);
    if (CL == 0) return AVATAR_ERR_UNSUPPORTED;
    p.rows_per_cta = b.R / CL;
    p.inv_rows = ((1 << 20) + p.rows_per_cta - 1) / p.rows_per_cta;
    const size_t smem = tri_smem(b.R, CL, b.Nv);

    int qgrid = (int)((b.Nv + 255) / 256);
    if (qgrid > ctx->sm_count * 8) qgrid = ctx->sm_count * 8;
    vis_quantize_kernel<<<dim3(qgrid, 1), 256, 0, st>>>(b.xp, b.Nv, qc[0], qc[1], qc[2], w.qv, b.status);
    AV_CHECK_LAUNCH();
    const int nchunks = (b.F + VIS_CHUNK - 1) / VIS_CHUNK;
    if (nchunks > 0) {
        vis_chunk_ranges_kernel<<<nchunks, 256, 0, st>>>(b.faces, b.F, b.Nv, w.vranges, nullptr, b.status);
        AV_CHECK_LAUNCH();
    }
    int rc;
    const bool cb = b.cull_back != 0;
#define AV_TRI(CLV)                                                                                     \
    (cb ? launch_tri<CLV, true>(p, w.qv, b.faces, w.vranges, b.frames, w.dirbits, b.status, smem, st)  \
        : launch_tri<CLV, false>(p, w.qv, b.faces, w.vranges, b.frames, w.dirbits, b.status, smem, st))
    switch (CL) {
        case 1: rc = AV_TRI(1); break;
        case 2: rc = AV_TRI(2); break;
        case 4: rc = AV_TRI(4); break;
        default: rc = AV_TRI(8); break;
    }
#undef AV_TRI
    if (rc != AVATAR_OK) return rc;
    // V vertex-major in direction order, then median, median, mean
    const int OW = b.D / 32;
    uint32_t *vm = b.bits ? b.bits : w.vm;
    const int tgrid = (p.NW + TR_VW - 1) / TR_VW, tspans = (b.D + TR_ROWS - 1) / TR_ROWS;
    vis_transpose_kernel<<<dim3(tgrid, tspans, 1), TR_THREADS, 0, st>>>(w.dirbits, p.NW, b.Nv, b.D, b.D, OW, nullptr, vm,
                                                               b.status);
    long items = (long)b.Nv * OW;
    int fgrid = (int)std::min<long>((items + 255) / 256, (long)ctx->sm_count * 16);
    vis_median_kernel<<<fgrid, 256, 0, st>>>(vm, a->knn_v, b.Nv, OW, a->Kv, w.m1, b.status);
    vis_median_kernel<<<fgrid, 256, 0, st>>>(w.m1, a->knn_v, b.Nv, OW, a->Kv, w.m2, b.status);
    uint8_t *dc = b.dmap ? w.dir_count : a->vis_count;
    vis_mean_kernel<<<fgrid, 256, 0, st>>>(w.m2, a->knn_v, b.Nv, OW, a->Kv, dc, b.status);
    AV_CHECK_LAUNCH();
    if (b.dmap) {
        long n = (long)b.Nv * b.NL;
        int lgrid = (int)std::min<long>((n + 255) / 256, (long)ctx->sm_count * 16);
        vis_light_order_kernel<<<lgrid, 256, 0, st>>>(w.dir_count, b.Nv, b.D, b.NL, b.dmap, a->vis_count, b.status);
        AV_CHECK_LAUNCH();
    }
    return AVATAR_OK;
}

// ---------------------------------------------------------------------------
// Entry point without a workspace, for callers that cannot allocate device
// memory (see the header).  Its scratch is a fixed-size array in the device
// image of this library, shared by every call on a device.
namespace {

constexpr size_t VIS_STATIC_SCRATCH_BYTES = (size_t)8 << 20;  // 8 MiB per device, held until exit
__device__ __align__(256) unsigned char g_vis_static_scratch[VIS_STATIC_SCRATCH_BYTES];

constexpr int VIS_MAX_DEVICES = 64;
std::mutex g_vis_static_mu;
void *g_vis_static_ptr[VIS_MAX_DEVICES];  // device address of the array, per device
CUcontext g_vis_static_cuctx[VIS_MAX_DEVICES];  // the CUDA context that address belongs to

// cuCtxGetCurrent through the runtime's driver entry point (no link to the
// driver library); NULL if the driver does not provide it.
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
CtxGetCurrentFn ctx_get_current()
{
    static CtxGetCurrentFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrentFn)p;
        else
            (void)cudaGetLastError();
    }
    return fn;
}

// Looks up the array's device address on the context's device, with that
// device current: on the first call for the device, and again whenever the
// device's CUDA context is not the one the cached address came from (after
// cudaDeviceReset, say).  The host-side symbol g_vis_static_scratch is only a
// stand-in and must never be handed to a kernel.
int vis_static_scratch(const avatar_ctx *ctx, void **out)
{
    if (ctx->device < 0 || ctx->device >= VIS_MAX_DEVICES) return AVATAR_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_vis_static_mu);
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return AVATAR_ERR_CUDA;
    if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return AVATAR_ERR_CUDA;
    CUcontext cur = nullptr;
    CtxGetCurrentFn get = ctx_get_current();
    if (get && get(&cur) != CUDA_SUCCESS) cur = nullptr;
    int rc = AVATAR_OK;
    if (!g_vis_static_ptr[ctx->device] || cur != g_vis_static_cuctx[ctx->device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_vis_static_scratch) != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            rc = AVATAR_ERR_CUDA;
        } else {
            g_vis_static_ptr[ctx->device] = p;
            g_vis_static_cuctx[ctx->device] = cur;
        }
    }
    if (prev != ctx->device) cudaSetDevice(prev);
    if (rc != AVATAR_OK) return rc;
    *out = g_vis_static_ptr[ctx->device];
    return AVATAR_OK;
}

}  // namespace

extern "C" size_t avatar_visibility_static_scratch_bytes(void) { return VIS_STATIC_SCRATCH_BYTES; }

extern "C" int avatar_visibility_static_scratch(avatar_ctx *ctx, const avatar_vis_args *a, avatar_stream_t stream)
{
    if (!ctx) return AVATAR_ERR_INVALID_ARG;
    AV_TRY(check_vis(a));
    if (vis_ws_layout(a, 1, nullptr, 0, nullptr) > VIS_STATIC_SCRATCH_BYTES) return AVATAR_ERR_WORKSPACE;
    void *scratch = nullptr;
    AV_TRY(vis_static_scratch(ctx, &scratch));
    // Everything the visibility kernels read from scratch is written earlier in
    // the same call, so nothing needs clearing between calls.
    return avatar_visibility(ctx, a, scratch, VIS_STATIC_SCRATCH_BYTES, stream);
}
