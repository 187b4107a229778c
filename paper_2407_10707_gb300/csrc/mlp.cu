// The pose-dependent displacement MLP of Sec. 3.1 (design in Sec. 4: four
// layers of width 256, ReLU, random Fourier features of the coordinates),
// dx = d(x, theta), on the tcgen05 tensor cores:
//   gamma(x) = [sin(2 pi B x), cos(2 pi B x)]  (64 frequencies -> 128 features)
//   h1 = relu(W1f gamma(x) + (W1p theta + b1))   the pose part of layer 1 is a
//                                               per-frame bias, folded in once
//   h2 = relu(W2 h1 + b2),  h3 = relu(W3 h2 + b3),  dx = W4 h3 + b4
// Persistent CTAs take 128 points at a time.  The features and every hidden
// activation are BF16 operands in shared memory (canonical no-swizzle K-major
// layout, one 64 KB buffer reused layer after layer); the weights stream
// through two 32 KB shared-memory buffers in 64-wide K chunks, pre-packed in
// the same layout (mlp_pack_kernel); one thread issues
// tcgen05.mma.kind::f16 (BF16 x BF16 -> FP32) into a 128 x 256 TMEM
// accumulator; each layer's epilogue reads it with tcgen05.ld, adds the bias,
// applies the ReLU and writes the next layer's operand in place.
#include "umma.cuh"

namespace {

constexpr int MLP_M = 128;        // points per tile
constexpr int MLP_THREADS = 256;
constexpr int MLP_W = 256;        // hidden width
constexpr int MLP_NF = 64;        // Fourier frequencies (128 features)
constexpr int MLP_KC = 64;        // K chunk of a weight stream
constexpr int MLP_MAX_P = 128;    // pose dimensions
constexpr int MLP_CHUNKS = 14;    // 2 (layer 1, K = 128) + 4 + 4 + 4 (layer 4, N = 16)
constexpr int A_KC8 = MLP_W / 8;  // core matrices along K in the activation buffer

struct ChunkInfo {
    int layer, kchunk, n, bytes, off;  // weight rows n (256 or 16), byte offset in the packed stream
};

__host__ __device__ inline ChunkInfo chunk_info(int q)
{
    ChunkInfo c;
    if (q < 2) {
        c.layer = 0;
        c.kchunk = q;
    } else if (q < 6) {
        c.layer = 1;
        c.kchunk = q - 2;
    } else if (q < 10) {
        c.layer = 2;
        c.kchunk = q - 6;
    } else {
        c.layer = 3;
        c.kchunk = q - 10;
    }
    c.n = c.layer == 3 ? 16 : MLP_W;
    c.bytes = c.n * MLP_KC * 2;
    const int big = MLP_W * MLP_KC * 2;
    c.off = q < 10 ? q * big : 10 * big + (q - 10) * 16 * MLP_KC * 2;
    return c;
}

constexpr size_t MLP_PACKED_BYTES = (size_t)10 * MLP_W * MLP_KC * 2 + (size_t)4 * 16 * MLP_KC * 2;

// Packs W1's feature part, W2, W3 and W4 (FP32, [out][in]) into the BF16
// chunk stream in the canonical layout (rows of W4 beyond 3 are zero).
__global__ void __launch_bounds__(256)
mlp_pack_kernel(const float *__restrict__ W1, int in1, const float *__restrict__ W2, const float *__restrict__ W3,
                const float *__restrict__ W4, unsigned char *__restrict__ packed)
{
    const long total = (long)10 * MLP_W * MLP_KC + 4L * 16 * MLP_KC;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        int q;
        long r;
        if (e < 10L * MLP_W * MLP_KC) {
            q = (int)(e / (MLP_W * MLP_KC));
            r = e % (MLP_W * MLP_KC);
        } else {
            const long e2 = e - 10L * MLP_W * MLP_KC;
            q = 10 + (int)(e2 / (16 * MLP_KC));
            r = e2 % (16 * MLP_KC);
        }
        const ChunkInfo c = chunk_info(q);
        const int n = (int)(r / MLP_KC), k = (int)(r % MLP_KC);
        const int kin = c.kchunk * MLP_KC + k;  // input index of the layer
        float v = 0.f;
        if (c.layer == 0) v = __ldg(W1 + (size_t)n * in1 + kin);
        else if (c.layer == 1) v = __ldg(W2 + (size_t)n * MLP_W + kin);
        else if (c.layer == 2) v = __ldg(W3 + (size_t)n * MLP_W + kin);
        else if (n < 3) v = __ldg(W4 + (size_t)n * MLP_W + kin);
        *reinterpret_cast<__nv_bfloat16 *>(packed + c.off + canon_off(n, k, MLP_KC / 8)) = __float2bfloat16_rn(v);
    }
}

struct MlpParams {
    int N, P;
    const float *x, *theta, *Bf, *W1, *b1, *b2, *b3, *b4;
    const unsigned char *packed;
    float *dx;
    int32_t *status;
};

__global__ void __launch_bounds__(MLP_THREADS, 1)
mlp_forward_kernel(MlpParams P)
{
    extern __shared__ __align__(1024) unsigned char mlp_smem[];
    unsigned char *sA = mlp_smem;                       // [128][256] BF16 activations
    unsigned char *sB = sA + MLP_M * MLP_W * 2;         // [2][32 KB] weight chunks
    float *sbias = reinterpret_cast<float *>(sB + 2 * MLP_W * MLP_KC * 2);  // [3][256] + [16]
    float *sfreq = sbias + 3 * MLP_W + 16;             // [64][3]
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t mbar[2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = tid & (MLP_M - 1), half = tid >> 7;
    const int in1 = 2 * MLP_NF + P.P;

    // layer-1 bias with the pose folded in, the other biases, the frequencies
    {
        float acc = __ldg(P.b1 + tid);
        for (int p = 0; p < P.P; ++p) acc = fmaf(__ldg(P.W1 + (size_t)tid * in1 + 2 * MLP_NF + p), __ldg(P.theta + p), acc);
        sbias[tid] = acc;
        sbias[MLP_W + tid] = __ldg(P.b2 + tid);
        sbias[2 * MLP_W + tid] = __ldg(P.b3 + tid);
        if (tid < 16) sbias[3 * MLP_W + tid] = tid < 3 ? __ldg(P.b4 + tid) : 0.f;
        if (tid < 3 * MLP_NF) sfreq[tid] = __ldg(P.Bf + tid);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = tmem_base;
    uint32_t uses[2] = {0, 0};
    int gq = 0;  // chunks issued by this CTA (buffer = gq & 1)

    for (int tile = blockIdx.x; tile * MLP_M < P.N; tile += gridDim.x) {
        const int g = tile * MLP_M + row;
        const bool in = g < P.N;
        // Fourier features of this row: half h takes frequencies 32h .. 32h + 31
        {
            const float x0 = in ? __ldg(P.x + g) : 0.f;
            const float x1 = in ? __ldg(P.x + (size_t)P.N + g) : 0.f;
            const float x2 = in ? __ldg(P.x + (size_t)2 * P.N + g) : 0.f;
#pragma unroll
            for (int j8 = 0; j8 < 4; ++j8) {
                __align__(16) __nv_bfloat16 sv[8], cv[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int j = half * 32 + j8 * 8 + i;
                    const float t = 2.f * (sfreq[3 * j] * x0 + sfreq[3 * j + 1] * x1 + sfreq[3 * j + 2] * x2);
                    float s, c;
                    sincospif(t, &s, &c);  // sin(pi t), cos(pi t) = sin, cos of 2 pi B x
                    sv[i] = __float2bfloat16_rn(s);
                    cv[i] = __float2bfloat16_rn(c);
                }
                const int k0 = half * 32 + j8 * 8;
                *reinterpret_cast<uint4 *>(sA + canon_off(row, k0, A_KC8)) = *reinterpret_cast<uint4 *>(sv);
                *reinterpret_cast<uint4 *>(sA + canon_off(row, MLP_NF + k0, A_KC8)) = *reinterpret_cast<uint4 *>(cv);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int q = 0; q < MLP_CHUNKS; ++q, ++gq) {
            const ChunkInfo c = chunk_info(q);
            const int buf = gq & 1;
            unsigned char *bb = sB + buf * (MLP_W * MLP_KC * 2);
            // the MMAs that last read this buffer must be done before it is refilled
            if (uses[buf] > 0) bar_wait(&mbar[buf], (uses[buf] - 1) & 1, P.status);
            const uint4 *src = reinterpret_cast<const uint4 *>(P.packed + c.off);
            for (int i = tid; i < c.bytes / 16; i += MLP_THREADS) reinterpret_cast<uint4 *>(bb)[i] = __ldg(src + i);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (tid == 0) {
                const uint32_t idesc = umma_idesc(MLP_M, c.n);
#pragma unroll
                for (int kk = 0; kk < MLP_KC / 16; ++kk) {
                    const int kcore = (c.kchunk * MLP_KC + kk * 16) / 8;  // core-matrix column in the activations
                    const uint64_t ad = umma_desc(smem_u32(sA) + kcore * 128, 128, A_KC8 * 128);
                    const uint64_t bd = umma_desc(smem_u32(bb) + kk * 2 * 128, 128, (MLP_KC / 8) * 128);
                    mma_bf16(tbase, ad, bd, idesc, (c.kchunk > 0 || kk > 0) ? 1u : 0u);
                }
                mma_commit(&mbar[buf]);
            }
            uses[buf] += 1;
            const bool last = (q == 1 || q == 5 || q == 9 || q == 13);
            if (!last) continue;
            // layer done: every MMA issued so far has completed when this commit lands
            bar_wait(&mbar[buf], (uses[buf] - 1) & 1, P.status);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int wl = warp & 3;
            const uint32_t lane_off = (uint32_t)(wl * 32) << 16;
            const int r = wl * 32 + lane;
            if (c.layer < 3) {
                const float *bias = sbias + c.layer * MLP_W;
                const int col0 = (warp >> 2) * (MLP_W / 2);
                for (int c0 = col0; c0 < col0 + MLP_W / 2; c0 += 16) {
                    float v[16];
                    tmem_ld16(tbase + lane_off + c0, v);
                    __align__(16) __nv_bfloat16 hv[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) hv[i] = __float2bfloat16_rn(fmaxf(v[i] + bias[c0 + i], 0.f));
                    *reinterpret_cast<uint4 *>(sA + canon_off(r, c0, A_KC8)) = *reinterpret_cast<uint4 *>(hv);
                    *reinterpret_cast<uint4 *>(sA + canon_off(r, c0 + 8, A_KC8)) = *reinterpret_cast<uint4 *>(hv + 8);
                }
            } else if (warp < 4) {
                float v[16];
                tmem_ld16(tbase + lane_off, v);
                const int gr = tile * MLP_M + r;
                if (gr < P.N)
#pragma unroll
                    for (int i = 0; i < 3; ++i) P.dx[(size_t)i * P.N + gr] = v[i] + sbias[3 * MLP_W + i];
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();  // the next layer's operand is complete; the accumulator is free
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(256));
}

size_t mlp_smem_bytes()
{
    return (size_t)MLP_M * MLP_W * 2 + (size_t)2 * MLP_W * MLP_KC * 2 + (size_t)(3 * MLP_W + 16 + 3 * MLP_NF) * 4;
}

int check_mlp(const avatar_mlp_args *a)
{
    if (!a || a->N < 0 || a->P < 0 || a->P > MLP_MAX_P) return AVATAR_ERR_INVALID_ARG;
    return AVATAR_OK;
}

}  // namespace

extern "C" size_t avatar_mlp_workspace_size(const avatar_mlp_args *a)
{
    if (check_mlp(a) != AVATAR_OK) return 0;
    return av_align256(MLP_PACKED_BYTES);
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
    if (!ws || (((uintptr_t)ws) & 255) || ws_bytes < av_align256(MLP_PACKED_BYTES)) return AVATAR_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *packed = (unsigned char *)ws;
    mlp_pack_kernel<<<ctx->sm_count * 2, 256, 0, st>>>(a->W1, 2 * MLP_NF + a->P, a->W2, a->W3, a->W4, packed);
    AV_CHECK_LAUNCH();
    const size_t smem = mlp_smem_bytes();
    if (smem > (size_t)ctx->max_smem_optin) return AVATAR_ERR_UNSUPPORTED;
    if (cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return AVATAR_ERR_CUDA;
    MlpParams p;
    p.N = a->N;
    p.P = a->P;
    p.x = a->x;
    p.theta = a->theta;
    p.Bf = a->Bf;
    p.W1 = a->W1;
    p.b1 = a->b1;
    p.b2 = a->b2;
    p.b3 = a->b3;
    p.b4 = a->b4;
    p.packed = packed;
    p.dx = a->dx;
    p.status = a->status;
    const int tiles = (a->N + MLP_M - 1) / MLP_M;
    const int grid = tiles < ctx->sm_count ? tiles : ctx->sm_count;
    mlp_forward_kernel<<<grid, MLP_THREADS, smem, st>>>(p);
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}
