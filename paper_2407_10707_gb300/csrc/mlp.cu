// The pose-dependent displacement MLP of Sec. 3.1 (design in Sec. 4: four
// layers of width 256, ReLU, random Fourier features of the coordinates),
// dx = d(x, theta), on the tcgen05 tensor cores:
//   gamma(x) = [sin(2 pi B x), cos(2 pi B x)]  (64 frequencies -> 128 features)
//   h1 = relu(W1f gamma(x) + (W1p theta + b1))   the pose part of layer 1 is a
//                                               per-frame bias, folded in once
//   h2 = relu(W2 h1 + b2),  h3 = relu(W3 h2 + b3),  dx = W4 h3 + b4
//
// One persistent CTA per SM keeps two tiles of 128 points in flight (slots
// 0 and 1), each with its own 64 KB BF16 activation buffer in shared memory
// (features, then each layer's output written in place over its input) and
// its own 256-column FP32 accumulator in TMEM.  A layer needs all of the
// previous one, so a single tile would leave the tensor core idle at every
// layer boundary (drain, epilogue, refill); with two slots the MMAs of one
// slot run while the other slot's epilogue works.  Warp roles:
//   warp 0 (one lane)  streams the pre-packed BF16 weight chunks (N x 32 K,
//                      canonical no-swizzle K-major, mlp_pack_kernel) into a
//                      five-stage ring with bulk asynchronous copies, in the
//                      order the MMAs consume them (per layer: slot 0, slot 1);
//   warp 1 (one lane)  issues tcgen05.mma.kind::f16 (BF16 x BF16 -> FP32,
//                      M = 128, N = 256, or 16 for the output layer);
//   warps 2..          the epilogues (tcgen05.ld, bias, ReLU, BF16 into the
//                      slot's buffer) and the Fourier features of a slot's
//                      next tile, written as soon as its last layer's MMAs
//                      have finished reading the buffer.
// Every mbarrier wait is bounded; the first wait that runs out sets
// AVATAR_ERR_TIMEOUT and makes all later waits of the CTA return at once,
// and the CTA still drains its copies and MMAs before it frees TMEM.
#include "umma.cuh"

namespace {

constexpr int MLP_M = 128;          // points per tile
constexpr int MLP_W = 256;          // hidden width
constexpr int MLP_NF = 64;          // Fourier frequencies (128 features)
constexpr int MLP_KC = 32;          // K chunk of the weight stream
constexpr int MLP_MAX_P = 128;      // pose dimensions
constexpr int L1_CHUNKS = 2 * MLP_NF / MLP_KC;       // layer 1 (K = 128)
constexpr int LW_CHUNKS = MLP_W / MLP_KC;            // layers 2..4 (K = 256)
constexpr int BIG_CHUNKS = L1_CHUNKS + 2 * LW_CHUNKS;  // N = 256 (layers 1..3); layer 4 has N = 16
constexpr int MLP_STAGES = 5;       // weight ring depth
constexpr int MATH_WARPS = 8;       // epilogue / feature warps (a multiple of 4)
constexpr int MLP_THREADS = 64 + 32 * MATH_WARPS;
constexpr int MATH_THREADS = 32 * MATH_WARPS;
constexpr int COL_PARTS = MATH_WARPS / 4;            // warps sharing one TMEM lane quarter
constexpr int PART_COLS = MLP_W / COL_PARTS;         // accumulator columns per epilogue warp
constexpr int F_PARTS = MATH_THREADS / MLP_M;        // threads sharing one row's features
constexpr int F_PER = MLP_NF / F_PARTS;              // frequencies per thread
constexpr int STAGE_BYTES = MLP_W * MLP_KC * 2;      // 16 KB
constexpr int SMALL_BYTES = 16 * MLP_KC * 2;         // a layer-4 chunk
constexpr int ACT_BYTES = MLP_M * MLP_W * 2;         // 64 KB activations per slot
constexpr int A_KC8 = MLP_W / 8;                     // core matrices along K (activations)
constexpr int B_KC8 = MLP_KC / 8;                    // (weight chunks)
// ring, two activation buffers, biases (layer 1 per slot, layers 2, 3 and 4), frequencies
constexpr size_t MLP_SMEM = (size_t)MLP_STAGES * STAGE_BYTES + 2 * ACT_BYTES + 4 * MLP_W * 4 + 16 * 4 + MLP_NF * 16;
static_assert(PART_COLS % 32 == 0 && F_PER % 8 == 0, "epilogue and feature work split");
static_assert(MATH_THREADS >= MLP_W, "bias setup");

struct ChunkInfo {
    int layer, kchunk, n, bytes, off;  // weight rows n (256 or 16), byte offset in the packed stream
};

__host__ __device__ inline ChunkInfo chunk_info(int q)
{
    ChunkInfo c;
    c.layer = q < L1_CHUNKS ? 0 : 1 + (q - L1_CHUNKS) / LW_CHUNKS;
    c.kchunk = q < L1_CHUNKS ? q : (q - L1_CHUNKS) % LW_CHUNKS;
    c.n = c.layer == 3 ? 16 : MLP_W;
    c.bytes = c.n * MLP_KC * 2;
    c.off = q < BIG_CHUNKS ? q * STAGE_BYTES : BIG_CHUNKS * STAGE_BYTES + (q - BIG_CHUNKS) * SMALL_BYTES;
    return c;
}

constexpr size_t MLP_PACKED_BYTES = (size_t)BIG_CHUNKS * STAGE_BYTES + (size_t)LW_CHUNKS * SMALL_BYTES;

// Packs W1's feature part, W2, W3 and W4 (FP32, [out][in]) into the BF16
// chunk stream in the canonical layout (rows of W4 beyond 3 are zero).
__global__ void __launch_bounds__(256)
mlp_pack_kernel(const float *__restrict__ W1, int in1, const float *__restrict__ W2, const float *__restrict__ W3,
                const float *__restrict__ W4, unsigned char *__restrict__ packed)
{
    const long big = (long)BIG_CHUNKS * MLP_W * MLP_KC;
    const long total = big + (long)LW_CHUNKS * 16 * MLP_KC;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        int q;
        long r;
        if (e < big) {
            q = (int)(e / (MLP_W * MLP_KC));
            r = e % (MLP_W * MLP_KC);
        } else {
            q = BIG_CHUNKS + (int)((e - big) / (16 * MLP_KC));
            r = (e - big) % (16 * MLP_KC);
        }
        const ChunkInfo c = chunk_info(q);
        const int n = (int)(r / MLP_KC), k = (int)(r % MLP_KC);
        const int kin = c.kchunk * MLP_KC + k;  // input index of the layer
        float v = 0.f;
        if (c.layer == 0) v = __ldg(W1 + (size_t)n * in1 + kin);
        else if (c.layer == 1) v = __ldg(W2 + (size_t)n * MLP_W + kin);
        else if (c.layer == 2) v = __ldg(W3 + (size_t)n * MLP_W + kin);
        else if (n < 3) v = __ldg(W4 + (size_t)n * MLP_W + kin);
        *reinterpret_cast<__nv_bfloat16 *>(packed + c.off + canon_off(n, k, B_KC8)) = __float2bfloat16_rn(v);
    }
}

struct MlpParams {
    int N, T;                // points, poses
    float inv_T;
    const float *x, *Bf, *b2, *b3, *b4;
    const float *c1;         // [T][256] layer-1 bias with each pose folded in
    const unsigned char *packed;
    float *dx;
    int32_t *status;
};

// Layer-1 bias of every pose: c1[t][n] = b1[n] + sum_p W1[n][128 + p] theta[t][p].
// One block per pose (grid-stride over poses); a warp takes a row n, its lanes
// the pose dimensions (coalesced), four rows in flight, and reduces by shuffles.
__global__ void __launch_bounds__(MLP_W)
mlp_pose_bias_kernel(const float *__restrict__ W1, const float *__restrict__ b1, const float *__restrict__ theta,
                     int P, int T, float *__restrict__ c1)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int in1 = 2 * MLP_NF + P;
    for (int t = blockIdx.x; t < T; t += gridDim.x) {
        const float *th = theta + (size_t)t * P;
        for (int n0 = warp * 4; n0 < MLP_W; n0 += nw * 4) {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            for (int p = lane; p < P; p += 32) {
                const float tp = __ldg(th + p);
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[r] = fmaf(__ldg(W1 + (size_t)(n0 + r) * in1 + 2 * MLP_NF + p), tp, acc[r]);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float v = warp_sum(acc[r]);
                if (lane == 0) c1[(size_t)t * MLP_W + n0 + r] = __ldg(b1 + n0 + r) + v;
            }
        }
    }
}

struct MlpBars {
    uint64_t full[MLP_STAGES], empty[MLP_STAGES];  // weight ring: copy landed / MMAs done with the stage
    uint64_t acc[2];                               // slot s: a layer's MMAs have completed
    uint64_t epi[2];                               // slot s: a hidden layer's output is in the buffer
    uint64_t feat[2];                              // slot s: the next tile's features are in the buffer
    uint64_t fin;                                  // every MMA of the CTA has completed
};

// Bounded wait; once any wait of the CTA has run out, every later one
// returns false at once.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, int32_t *status, volatile int *abort)
{
    for (int it = 0; it < UMMA_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done)
                     : "r"(smem_u32(bar)), "r"(parity)
                     : "memory");
        if (done) return true;
        if ((it & 63) == 63 && *abort) return false;
    }
    *abort = 1;
    av_report(status, AVATAR_ERR_TIMEOUT);
    return false;
}

__device__ __forceinline__ void bar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ int layer_chunks(int L) { return L == 0 ? L1_CHUNKS : LW_CHUNKS; }
__device__ __forceinline__ int chunk_index(int L, int k) { return L == 0 ? k : L1_CHUNKS + (L - 1) * LW_CHUNKS + k; }

// Features of tile `tile` into columns 0..127 of a slot's buffer: math
// thread mt takes row mt % 128 and F_PER frequencies.  The phase t = B x
// (cycles) is reduced exactly to r = t - rint(t) in [-1/2, 1/2] before the
// hardware sine and cosine of 2 pi r (absolute error about 4e-7 on
// [-pi, pi], below the FP32 error of t itself).
__device__ __forceinline__ void write_features(const MlpParams &P, int tile, int mt, const float4 *sfreq,
                                               unsigned char *act)
{
    const int row = mt & (MLP_M - 1), part = mt / MLP_M;
    const int g = tile * MLP_M + row;
    const bool in = g < P.N;
    const float x0 = in ? __ldg(P.x + g) : 0.f;
    const float x1 = in ? __ldg(P.x + (size_t)P.N + g) : 0.f;
    const float x2 = in ? __ldg(P.x + (size_t)2 * P.N + g) : 0.f;
#pragma unroll
    for (int j8 = 0; j8 < F_PER; j8 += 8) {
        uint32_t sv[4], cv[4];
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
            float s2[2], c2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float4 b = sfreq[part * F_PER + j8 + i + h];
                const float t = fmaf(b.z, x2, fmaf(b.y, x1, b.x * x0));
                const float z = 6.28318530717959f * (t - rintf(t));
                s2[h] = __sinf(z);
                c2[h] = __cosf(z);
            }
            const __nv_bfloat162 sp = __floats2bfloat162_rn(s2[0], s2[1]);
            const __nv_bfloat162 cp = __floats2bfloat162_rn(c2[0], c2[1]);
            sv[i / 2] = *reinterpret_cast<const uint32_t *>(&sp);
            cv[i / 2] = *reinterpret_cast<const uint32_t *>(&cp);
        }
        const int k0 = part * F_PER + j8;
        *reinterpret_cast<uint4 *>(act + canon_off(row, k0, A_KC8)) = make_uint4(sv[0], sv[1], sv[2], sv[3]);
        *reinterpret_cast<uint4 *>(act + canon_off(row, MLP_NF + k0, A_KC8)) = make_uint4(cv[0], cv[1], cv[2], cv[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__global__ void __launch_bounds__(MLP_THREADS, 1)
mlp_forward_kernel(MlpParams P)
{
    extern __shared__ __align__(1024) unsigned char mlp_smem[];
    unsigned char *ring = mlp_smem;                                   // [5][16 KB] weight chunks
    unsigned char *act = ring + MLP_STAGES * STAGE_BYTES;             // [2][128][256] BF16 activations
    float *sbias = reinterpret_cast<float *>(act + 2 * ACT_BYTES);    // [2][256] slot's layer-1 bias; b2; b3
    float *sb4 = sbias + 4 * MLP_W;                                   // [16]
    float4 *sfreq = reinterpret_cast<float4 *>(sb4 + 16);             // [64] frequencies (x, y, z, 0)
    __shared__ MlpBars bars;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (P.N + MLP_M - 1) / MLP_M;
    const int grid = gridDim.x;
    volatile int *abort = &abort_flag;
    // Work items (point tile, pose): this CTA's point tiles blockIdx.x + k grid,
    // each with all T poses in order (so a point tile's mean stays on one CTA).
    const int my_tiles = ntiles > (int)blockIdx.x ? (ntiles - (int)blockIdx.x + grid - 1) / grid : 0;
    const int n_items = my_tiles * P.T;
    auto item_tile = [&](int i) { return (int)blockIdx.x + (i / P.T) * grid; };
    auto item_pose = [&](int i) { return i % P.T; };

    if (warp >= 2 && tid - 64 < MLP_W) {  // the pose-independent biases, the frequencies
        const int n = tid - 64;
        sbias[2 * MLP_W + n] = __ldg(P.b2 + n);
        sbias[3 * MLP_W + n] = __ldg(P.b3 + n);
        if (n < 16) sb4[n] = n < 3 ? __ldg(P.b4 + n) : 0.f;
        if (n < MLP_NF) sfreq[n] = make_float4(__ldg(P.Bf + 3 * n), __ldg(P.Bf + 3 * n + 1), __ldg(P.Bf + 3 * n + 2), 0.f);
    }
    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < MLP_STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars.full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars.empty[s])));
        }
        for (int s = 0; s < 2; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars.acc[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars.epi[s])), "r"(MATH_THREADS));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars.feat[s])), "r"(MATH_THREADS));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars.fin)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = tmem_base;

    // Items go in pairs: pair m holds items 2 m (slot 0) and 2 m + 1 (slot 1,
    // if it exists).  Per pair and layer, slot 0 then slot 1, in all three roles.
    if (warp == 0) {
        // ---------------------------------------------------------------- weight producer
        if (lane == 0) {
            int c = 0;
            for (int i0 = 0; i0 < n_items; i0 += 2) {
                const int ns = i0 + 1 < n_items ? 2 : 1;
                for (int L = 0; L < 4; ++L)
                    for (int s = 0; s < ns; ++s)
                        for (int k = 0; k < layer_chunks(L); ++k, ++c) {
                            const int st = c % MLP_STAGES;
                            if (c >= MLP_STAGES)
                                wait_or_abort(&bars.empty[st], ((c / MLP_STAGES) - 1) & 1, P.status, abort);
                            const ChunkInfo ci = chunk_info(chunk_index(L, k));
                            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                             smem_u32(&bars.full[st])),
                                         "r"(ci.bytes)
                                         : "memory");
                            asm volatile(
                                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                                "[%3];" ::"r"(smem_u32(ring + st * STAGE_BYTES)),
                                "l"(P.packed + ci.off), "r"(ci.bytes), "r"(smem_u32(&bars.full[st]))
                                : "memory");
                        }
            }
            // drain: each stage's last copy has landed (bounded even after an abort)
            for (int cc = c - MLP_STAGES < 0 ? 0 : c - MLP_STAGES; cc < c; ++cc)
                bar_wait(&bars.full[cc % MLP_STAGES], (cc / MLP_STAGES) & 1, nullptr);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            int c = 0, m = 0;
            for (int i0 = 0; i0 < n_items; i0 += 2, ++m) {
                const int ns = i0 + 1 < n_items ? 2 : 1;
                for (int L = 0; L < 4; ++L) {
                    const uint32_t idesc = umma_idesc(MLP_M, L == 3 ? 16 : MLP_W);
                    for (int s = 0; s < ns; ++s) {
                        // the slot's input is complete and its accumulator has been read
                        if (L == 0) wait_or_abort(&bars.feat[s], m & 1, P.status, abort);
                        else wait_or_abort(&bars.epi[s], (3 * m + L - 1) & 1, P.status, abort);
                        const uint32_t acc = tbase + (uint32_t)(s * MLP_W);
                        const uint32_t a0 = smem_u32(act + s * ACT_BYTES);
                        for (int k = 0; k < layer_chunks(L); ++k, ++c) {
                            const int st = c % MLP_STAGES;
                            wait_or_abort(&bars.full[st], (c / MLP_STAGES) & 1, P.status, abort);
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            const uint32_t b0 = smem_u32(ring + st * STAGE_BYTES);
#pragma unroll
                            for (int kk = 0; kk < MLP_KC / 16; ++kk) {
                                const uint64_t ad = umma_desc(a0 + (k * B_KC8 + kk * 2) * 128, 128, A_KC8 * 128);
                                const uint64_t bd = umma_desc(b0 + kk * 2 * 128, 128, B_KC8 * 128);
                                mma_bf16(acc, ad, bd, idesc, (k > 0 || kk > 0) ? 1u : 0u);
                            }
                            mma_commit(&bars.empty[st]);
                        }
                        mma_commit(&bars.acc[s]);
                    }
                }
            }
            mma_commit(&bars.fin);
            bar_wait(&bars.fin, 0, nullptr);  // every MMA has completed (bounded even after an abort)
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- epilogues and features
        const int mt = tid - 64;
        const int quarter = warp & 3, part = (warp - 2) >> 2;
        const int row = quarter * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        // a slot's input: the point tile's features and the pose's layer-1 bias
        // (a named barrier of the math warps makes the bias row visible to all)
        auto prepare = [&](int i, int s) {
            write_features(P, item_tile(i), mt, sfreq, act + s * ACT_BYTES);
            if (mt < MLP_W) sbias[s * MLP_W + mt] = __ldg(P.c1 + (size_t)item_pose(i) * MLP_W + mt);
            asm volatile("bar.sync 1, %0;" ::"r"(MATH_THREADS) : "memory");
            bar_arrive(&bars.feat[s]);
        };
        for (int s = 0; s < 2 && s < n_items; ++s) prepare(s, s);
        float mean[3] = {0.f, 0.f, 0.f};  // running sum over the poses of the current point tile
        int cur_tile = n_items > 0 ? item_tile(0) : -1;
        auto flush = [&]() {
            const int gr = cur_tile * MLP_M + row;
            if (part == 0 && gr < P.N)
#pragma unroll
                for (int j = 0; j < 3; ++j) P.dx[(size_t)j * P.N + gr] = mean[j] * P.inv_T;
            mean[0] = mean[1] = mean[2] = 0.f;
        };
        for (int i0 = 0; i0 < n_items; i0 += 2) {
            const int ns = i0 + 1 < n_items ? 2 : 1;
            for (int L = 0; L < 4; ++L)
                for (int s = 0; s < ns; ++s) {
                    const int item = i0 + s;
                    unsigned char *buf = act + s * ACT_BYTES;
                    wait_or_abort(&bars.acc[s], L & 1, P.status, abort);
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t acc = tbase + lane_off + (uint32_t)(s * MLP_W);
                    if (L < 3) {
                        const float *bias = sbias + (L == 0 ? s : L + 1) * MLP_W;
#pragma unroll 1
                        for (int c0 = part * PART_COLS; c0 < (part + 1) * PART_COLS; c0 += 32) {
                            float v[32];
                            tmem_ld32(acc + c0, v);
#pragma unroll
                            for (int j8 = 0; j8 < 32; j8 += 8) {
                                const float4 ba = *reinterpret_cast<const float4 *>(bias + c0 + j8);
                                const float4 bb = *reinterpret_cast<const float4 *>(bias + c0 + j8 + 4);
                                const float bv[8] = {ba.x, ba.y, ba.z, ba.w, bb.x, bb.y, bb.z, bb.w};
                                uint32_t hv[4];
#pragma unroll
                                for (int j = 0; j < 8; j += 2) {
                                    const __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(v[j8 + j] + bv[j], 0.f),
                                                                                   fmaxf(v[j8 + j + 1] + bv[j + 1], 0.f));
                                    hv[j / 2] = *reinterpret_cast<const uint32_t *>(&h);
                                }
                                *reinterpret_cast<uint4 *>(buf + canon_off(row, c0 + j8, A_KC8)) =
                                    make_uint4(hv[0], hv[1], hv[2], hv[3]);
                            }
                        }
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                        bar_arrive(&bars.epi[s]);
                    } else {
                        float v[16];
                        tmem_ld16(acc, v);  // read before the next tile's MMAs may overwrite the accumulator
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                        if (item + 2 < n_items) prepare(item + 2, s);  // the output layer's MMAs no longer read the buffer
                        if (item_tile(item) != cur_tile) {
                            flush();
                            cur_tile = item_tile(item);
                        }
#pragma unroll
                        for (int j = 0; j < 3; ++j) mean[j] += v[j] + sb4[j];
                    }
                }
        }
        if (n_items > 0) flush();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512));
}

int check_mlp(const avatar_mlp_args *a)
{
    if (!a || a->N < 0 || a->P < 0 || a->P > MLP_MAX_P || a->T < 1 || a->T > (1 << 20)) return AVATAR_ERR_INVALID_ARG;
    return AVATAR_OK;
}

size_t mlp_ws(const avatar_mlp_args *a, size_t *c1_off)
{
    const size_t packed = av_align256(MLP_PACKED_BYTES);
    if (c1_off) *c1_off = packed;
    return packed + av_align256((size_t)a->T * MLP_W * sizeof(float));
}

}  // namespace

extern "C" size_t avatar_mlp_workspace_size(const avatar_mlp_args *a)
{
    if (check_mlp(a) != AVATAR_OK) return 0;
    return mlp_ws(a, nullptr);
}

extern "C" int avatar_mlp(avatar_ctx *ctx, const avatar_mlp_args *a, void *ws, size_t ws_bytes,
                          avatar_stream_t stream)
{
    if (!ctx) return AVATAR_ERR_INVALID_ARG;
    AV_TRY(check_mlp(a));
    if (a->N == 0) return AVATAR_OK;
    if (!a->x || !a->Bf || !a->W1 || !a->b1 || !a->W2 || !a->b2 || !a->W3 || !a->b3 || !a->W4 || !a->b4 || !a->dx ||
        (a->P > 0 && !a->theta))
        return AVATAR_ERR_INVALID_ARG;
    size_t c1_off;
    if (!ws || (((uintptr_t)ws) & 255) || ws_bytes < mlp_ws(a, &c1_off)) return AVATAR_ERR_WORKSPACE;
    if (MLP_SMEM + 1024 > (size_t)ctx->max_smem_optin) return AVATAR_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *packed = (unsigned char *)ws;
    float *c1 = (float *)((unsigned char *)ws + c1_off);
    mlp_pack_kernel<<<ctx->sm_count * 2, 256, 0, st>>>(a->W1, 2 * MLP_NF + a->P, a->W2, a->W3, a->W4, packed);
    AV_CHECK_LAUNCH();
    const int pgrid = a->T < ctx->sm_count * 4 ? a->T : ctx->sm_count * 4;
    mlp_pose_bias_kernel<<<pgrid, MLP_W, 0, st>>>(a->W1, a->b1, a->theta, a->P, a->T, c1);
    AV_CHECK_LAUNCH();
    if (cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_SMEM) !=
        cudaSuccess)
        return AVATAR_ERR_CUDA;
    MlpParams p;
    p.N = a->N;
    p.T = a->T;
    p.inv_T = 1.0f / (float)a->T;
    p.x = a->x;
    p.Bf = a->Bf;
    p.b2 = a->b2;
    p.b3 = a->b3;
    p.b4 = a->b4;
    p.c1 = c1;
    p.packed = packed;
    p.dx = a->dx;
    p.status = a->status;
    const int tiles = (a->N + MLP_M - 1) / MLP_M;
    const int grid = tiles < ctx->sm_count ? tiles : ctx->sm_count;
    mlp_forward_kernel<<<grid, MLP_THREADS, MLP_SMEM, st>>>(p);
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}
