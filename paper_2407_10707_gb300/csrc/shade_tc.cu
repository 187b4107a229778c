// (c') Relighting one posed, viewed avatar under many environment lights at
// once - the relighting use of Sec. 3.5 (swap L for new maps) applied to Eq. 2.
//
// For n_env lights that share the texel geometry (directions w_k, solid angles
// A_k) the shading sums of Eq. 2 factor into two matrix products:
//   L_o[g, (l, c)] = a_gc / pi * (D B)[g, (l, c)] + p_g * (S B)[g, (l, c)]
//   D[g, k] = vis_gk max(0, n_g . w_k)          (diffuse weight)
//   S[g, k] = D[g, k] f_s(g, k)                 (specular weight, App. A)
//   B[k, (l, c)] = L^(l)_kc A_k                 (all lights stacked)
// D and S are computed per 64-light chunk by the CUDA cores (BF16, in the
// tensor-core canonical layout in shared memory, double-buffered); one thread
// issues tcgen05.mma (kind::f16, BF16 in, FP32 accumulate in TMEM) against the
// stacked light matrix, which stays resident in shared memory; the epilogue
// reads the accumulators with tcgen05.ld and writes gamma-corrected colours.
// Persistent CTAs, one per SM, each with 256 TMEM columns.
#include "umma.cuh"

namespace {

constexpr int TC_M = 128;        // Gaussians per tile (tensor-core M)
constexpr int TC_THREADS = 512;  // four threads per Gaussian row (16 lights each per chunk)
constexpr int TC_KC = 64;        // lights per chunk
constexpr int TC_MAX_ENV = 32;   // N = 3 * n_env <= 96
constexpr int TC_MAX_K = 2048;   // resident stacked-light matrix (shared-memory size permitting)
constexpr int TC_TMEM_COLS = 256;
constexpr float FRES_C1 = -5.55473f;
constexpr float FRES_C0 = -6.98316f;
constexpr float INV_GAMMA = 1.0f / 2.2f;

// Exact FP32 back-face decision, identical to the single-light kernel.
__device__ __forceinline__ bool culled_fp32(const float *x, const float *n, const float *C)
{
    float d0 = __fsub_rn(C[0], x[0]), d1 = __fsub_rn(C[1], x[1]), d2 = __fsub_rn(C[2], x[2]);
    float s = __fmaf_rn(n[2], d2, __fmaf_rn(n[1], d1, __fmul_rn(n[0], d0)));
    return !(s > 0.0f);
}

struct TcParams {
    avatar_shade_args s;
    int n_env;
    int N;  // 3 * n_env padded to a multiple of 16
    const float *env_L;
    float *env_color;
    const int32_t *live_list;  // [G] indices of live Gaussians (first *live_count)
    const int32_t *live_count;
};

constexpr int TC_COMPACT_THREADS = 256;

// First pass: back-face / index test of every Gaussian (exact FP32, as in the
// single-light kernel), cull flag, colour 0 for the dead, and a list of the
// live ones (block-ordered, so the tiles read nearly contiguous Gaussians).
__global__ void __launch_bounds__(TC_COMPACT_THREADS)
tc_compact_kernel(avatar_shade_args s, int n_env, float *env_color, int32_t *live_list, int32_t *live_count)
{
    __shared__ int s_warp[TC_COMPACT_THREADS / 32];
    __shared__ int s_base;
    const int g = blockIdx.x * TC_COMPACT_THREADS + threadIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    bool live = false;
    if (g < s.G) {
        float x[3], n[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            x[i] = __ldg(s.xd + (size_t)i * s.G + g);
            n[i] = __ldg(s.nd + (size_t)i * s.G + g);
        }
        bool ok = true;
        for (int j = 0; j < s.K; ++j)
            if ((unsigned)__ldg(s.knn + (size_t)j * s.G + g) >= (unsigned)s.Nv) ok = false;
        if (!ok) av_report(s.status, AVATAR_ERR_INDEX);
        live = ok && !culled_fp32(x, n, s.cam_center);
        if (s.cull) s.cull[g] = (uint8_t)(live ? 0 : 1);
        if (!live) {
            for (int c = 0; c < 3 * n_env; ++c) env_color[(size_t)c * s.G + g] = 0.f;
            if (s.radiance && n_env == 1)
                for (int c = 0; c < 3; ++c) s.radiance[(size_t)c * s.G + g] = 0.f;
        }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, live);
    if (lane == 0) s_warp[warp] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < TC_COMPACT_THREADS / 32; ++w) {
            const int c = s_warp[w];
            s_warp[w] = tot;
            tot += c;
        }
        s_base = tot ? atomicAdd(live_count, tot) : 0;
    }
    __syncthreads();
    if (live) live_list[s_base + s_warp[warp] + __popc(bal & lanemask_lt())] = g;
}

template <int K>
__global__ void __launch_bounds__(TC_THREADS, 1)
shade_multi_tc_kernel(TcParams P)
{
    const avatar_shade_args &s = P.s;
    const int NL = s.NL, G = s.G, N = P.N;
    const int kc8_B = NL / 8;  // core matrices along K in the resident B
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char *sB = tc_smem;                                   // [N][NL] BF16, canonical
    unsigned char *sA = sB + (size_t)N * NL * 2;                   // [2 buffers][D|S][128][64] BF16
    float4 *sW = reinterpret_cast<float4 *>(sA + 2 * 2 * TC_M * TC_KC * 2);  // [NL] light directions
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ int s_g[TC_M];  // Gaussian of each tile row, -1 past the live count
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = tid & (TC_M - 1), quarter = tid >> 7;

    // stacked light matrix B[n = 3l + c][k] = L^(l)_kc A_k (rows >= 3 n_env are 0)
    for (int i = tid; i < N * NL; i += TC_THREADS) {
        int n = i / NL, k = i % NL;
        float v = 0.f;
        if (n < 3 * P.n_env) {
            int l = n / 3, c = n % 3;
            v = __ldg(P.env_L + ((size_t)l * NL + k) * 3 + c) * __ldg(s.light_A + k);
        }
        *reinterpret_cast<__nv_bfloat16 *>(sB + canon_off(n, k, kc8_B)) = __float2bfloat16_rn(v);
    }
    for (int k = tid; k < NL; k += TC_THREADS)
        sW[k] = make_float4(__ldg(s.light_w + 3 * k), __ldg(s.light_w + 3 * k + 1), __ldg(s.light_w + 3 * k + 2), 0.f);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = tmem_base;
    const uint32_t t_diff = tbase, t_spec = tbase + 128;  // accumulator column offsets
    const uint32_t idesc = umma_idesc(TC_M, N);
    const float C[3] = {s.cam_center[0], s.cam_center[1], s.cam_center[2]};
    const int OW = (NL + 31) / 32;
    const int nchunks = NL / TC_KC;
    uint32_t uses[2] = {0, 0};  // completed-or-issued uses of each A buffer
    int q = 0;                  // global chunk counter (buffer = q & 1)

    const int nlive = *P.live_count;
    for (int tile = blockIdx.x; tile * TC_M < nlive; tile += gridDim.x) {
        const int li_row = tile * TC_M + row;
        const bool in = li_row < nlive;
        const int g = in ? __ldg(P.live_list + li_row) : 0;
        if (quarter == 0) s_g[row] = in ? g : -1;
        // per-Gaussian state (all four threads of a row compute it)
        float x[3] = {0, 0, 0}, n[3] = {0, 0, 1}, r = 0.5f;
        float ub[K];
        int nb[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            ub[j] = 0.f;
            nb[j] = 0;
        }
        const bool live = in;
        if (in) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                x[i] = __ldg(s.xd + (size_t)i * G + g);
                n[i] = __ldg(s.nd + (size_t)i * G + g);
            }
            r = __ldg(s.rg + g);
#pragma unroll
            for (int j = 0; j < K; ++j) {
                ub[j] = __ldg(s.ubar + (size_t)j * G + g);
                nb[j] = __ldg(s.knn + (size_t)j * G + g);
            }
        }
        float wo[3], co_raw, a2, kk, Go;
        {
            float v0 = C[0] - x[0], v1 = C[1] - x[1], v2 = C[2] - x[2];
            float il = rsqrtf(v0 * v0 + v1 * v1 + v2 * v2 + 1e-30f);
            wo[0] = v0 * il;
            wo[1] = v1 * il;
            wo[2] = v2 * il;
            co_raw = n[0] * wo[0] + n[1] * wo[1] + n[2] * wo[2];
            float alpha = r * r;
            a2 = alpha * alpha;
            kk = (r + 1.f) * (r + 1.f) * 0.125f;
            Go = fmaxf(co_raw, 0.f) * (1.f - kk) + kk;
        }
        const float spec_scale = a2 / (4.f * AV_PI * Go);

        for (int ch = 0; ch < nchunks; ++ch, ++q) {
            const int buf = q & 1;
            // wait until the MMAs that last read this buffer are done
            if (uses[buf] > 0) bar_wait(&mbar[buf], (uses[buf] - 1) & 1, s.status);
            unsigned char *aD = sA + (size_t)buf * 2 * TC_M * TC_KC * 2;
            unsigned char *aS = aD + TC_M * TC_KC * 2;
            // this thread's 16 lights of the chunk: k = ch*64 + quarter*16 + i, computed
            // without branches (every lane of a warp does the same work)
            const int k0 = ch * TC_KC + quarter * 16;
            const int sh = k0 & 31;
            unsigned words[K];
            unsigned all = 0xffffffffu;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                words[j] = live ? (__ldg(s.bits + (size_t)nb[j] * OW + (k0 >> 5)) >> sh) : 0u;
                all &= words[j];
            }
#pragma unroll
            for (int i8 = 0; i8 < 2; ++i8) {  // 2 groups of 8 lights -> one 16-byte row segment each
                __align__(16) __nv_bfloat16 dv[8], sv[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int li = i8 * 8 + i;
                    const float4 w = sW[k0 + li];
                    const float ci = n[0] * w.x + n[1] * w.y + n[2] * w.z;
                    float vis = 0.f;
#pragma unroll
                    for (int j = 0; j < K; ++j) vis += ((words[j] >> li) & 1u) ? ub[j] : 0.f;
                    vis = ((all >> li) & 1u) ? 1.f : vis;
                    const float Dw = (live && ci > 0.f) ? vis * ci : 0.f;
                    const float dwo = w.x * wo[0] + w.y * wo[1] + w.z * wo[2];
                    const float rinv = rsqrtf(fmaxf(2.f + 2.f * dwo, 1e-20f));
                    const float nh = (ci + co_raw) * rinv;
                    const float voh = (1.f + dwo) * rinv;
                    const float den = fmaf(nh * nh, a2 - 1.f, 1.f);
                    const float Fr = fmaf(0.96f, exp2f(fmaf(FRES_C1, voh, FRES_C0) * voh), 0.04f);
                    const float Gi = fmaf(fmaxf(ci, 0.f), 1.f - kk, kk);
                    const float Sw = Dw * spec_scale * __fdividef(Fr, den * den * Gi);
                    dv[i] = __float2bfloat16_rn(Dw);
                    sv[i] = __float2bfloat16_rn(Sw);
                }
                const int kl = quarter * 16 + i8 * 8;  // k within the chunk
                *reinterpret_cast<uint4 *>(aD + canon_off(row, kl, TC_KC / 8)) = *reinterpret_cast<uint4 *>(dv);
                *reinterpret_cast<uint4 *>(aS + canon_off(row, kl, TC_KC / 8)) = *reinterpret_cast<uint4 *>(sv);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (tid == 0) {
#pragma unroll
                for (int kk16 = 0; kk16 < TC_KC / 16; ++kk16) {
                    const uint32_t koff = kk16 * 2 * 128;  // two core matrices along K per MMA
                    const uint64_t bdesc =
                        umma_desc(smem_u32(sB) + ((ch * TC_KC / 8 + kk16 * 2) << 7), 128, kc8_B * 128);
                    const uint32_t acc = (ch > 0 || kk16 > 0) ? 1u : 0u;
                    mma_bf16(t_diff, umma_desc(smem_u32(aD) + koff, 128, (TC_KC / 8) * 128), bdesc, idesc, acc);
                    mma_bf16(t_spec, umma_desc(smem_u32(aS) + koff, 128, (TC_KC / 8) * 128), bdesc, idesc, acc);
                }
                mma_commit(&mbar[buf]);
            }
            uses[buf] += 1;
        }
        // epilogue: all MMAs of this tile are done when the last commit lands
        {
            const int lastbuf = (q - 1) & 1;
            bar_wait(&mbar[lastbuf], (uses[lastbuf] - 1) & 1, s.status);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // warp w reads TMEM lanes 32 (w % 4) ..; warps 0-3 take columns
            // [0, N/2), warps 4-7 take [N/2, N) of both accumulators
            const int wl = warp & 3;
            const int col0 = ((warp >> 2) & 1) * (N / 2);
            const bool epi = warp < 8;  // warps 0-7 read the accumulators
            const int gr = s_g[wl * 32 + lane];
            const bool want_rad = s.radiance != nullptr && P.n_env == 1;
            const bool ok = gr >= 0;
            float ar[3] = {0, 0, 0}, pr = 0.f;
            if (ok) {
                ar[0] = __ldg(s.ag + gr) * (1.f / AV_PI);
                ar[1] = __ldg(s.ag + (size_t)G + gr) * (1.f / AV_PI);
                ar[2] = __ldg(s.ag + (size_t)2 * G + gr) * (1.f / AV_PI);
                pr = __ldg(s.pg + gr);
            }
            for (int c0 = col0; epi && c0 < col0 + N / 2; c0 += 16) {
                float dv[16], sv[16];
                const uint32_t lane_off = (uint32_t)(wl * 32) << 16;
                tmem_ld16(t_diff + lane_off + c0, dv);
                tmem_ld16(t_spec + lane_off + c0, sv);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int nn = c0 + i;
                    if (!ok || nn >= 3 * P.n_env) continue;
                    const float Lo = ar[nn % 3] * dv[i] + pr * sv[i];
                    P.env_color[(size_t)nn * G + gr] = exp2f(log2f(fmaxf(Lo, 1e-6f)) * INV_GAMMA);
                    if (want_rad) s.radiance[(size_t)nn * G + gr] = Lo;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();  // accumulators read before the next tile overwrites them
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TC_TMEM_COLS));
}

template <int K>
int launch_tc(const TcParams &P, int grid, size_t smem, cudaStream_t st)
{
    if (cudaFuncSetAttribute(shade_multi_tc_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return AVATAR_ERR_CUDA;
    shade_multi_tc_kernel<K><<<grid, TC_THREADS, smem, st>>>(P);
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}

struct TcWs {
    int32_t *count;
    int32_t *list;
};

size_t tc_carve(const avatar_shade_multi_args *m, TcWs *w)
{
    WsCarver c(m ? m->workspace : nullptr, m ? m->workspace_bytes : 0);
    const int G = m ? m->base.G : 0;
    TcWs t;
    t.count = c.take<int32_t>(1);
    t.list = c.take<int32_t>((size_t)(G > 0 ? G : 1));
    if (w) *w = t;
    return c.off;
}

}  // namespace

extern "C" size_t avatar_shade_multi_workspace_size(const avatar_shade_multi_args *m)
{
    if (!m || m->base.G < 0) return 0;
    avatar_shade_multi_args q = *m;
    q.workspace = nullptr;
    return tc_carve(&q, nullptr);
}

extern "C" int avatar_shade_multi(avatar_ctx *ctx, const avatar_shade_multi_args *m, avatar_stream_t stream)
{
    if (!ctx || !m) return AVATAR_ERR_INVALID_ARG;
    const avatar_shade_args &s = m->base;
    if (s.G < 0 || s.K < 1 || s.K > 8 || s.Nv < 1 || m->n_env < 1 || m->n_env > TC_MAX_ENV) return AVATAR_ERR_INVALID_ARG;
    if (s.NL < TC_KC || s.NL > TC_MAX_K || s.NL % TC_KC != 0) return AVATAR_ERR_UNSUPPORTED;
    if (!m->env_L || !m->env_color || !s.light_A || !s.light_w) return AVATAR_ERR_INVALID_ARG;
    if (s.vis_count) return AVATAR_ERR_UNSUPPORTED;  // hard visibility bits only
    if (s.G > 0 && (!s.xd || !s.nd || !s.ag || !s.rg || !s.pg || !s.ubar || !s.knn || !s.bits))
        return AVATAR_ERR_INVALID_ARG;
    if (s.G == 0) return AVATAR_OK;
    TcWs w;
    const size_t need = tc_carve(m, &w);
    if (!m->workspace || m->workspace_bytes < need) return AVATAR_ERR_WORKSPACE;
    TcParams P;
    P.s = s;
    P.n_env = m->n_env;
    P.N = ((3 * m->n_env + 15) / 16) * 16;
    P.env_L = m->env_L;
    P.env_color = m->env_color;
    P.live_list = w.list;
    P.live_count = w.count;
    size_t smem = (size_t)P.N * s.NL * 2 + (size_t)2 * 2 * TC_M * TC_KC * 2 + (size_t)s.NL * sizeof(float4);
    if (smem > (size_t)ctx->max_smem_optin) return AVATAR_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(w.count, 0, sizeof(int32_t), st) != cudaSuccess) return AVATAR_ERR_CUDA;
    tc_compact_kernel<<<(s.G + TC_COMPACT_THREADS - 1) / TC_COMPACT_THREADS, TC_COMPACT_THREADS, 0, st>>>(
        s, m->n_env, m->env_color, w.list, w.count);
    AV_CHECK_LAUNCH();
    // grid: one persistent CTA per SM, or fewer if even an all-live G has fewer tiles
    const int tiles = (s.G + TC_M - 1) / TC_M;
    const int grid = tiles < ctx->sm_count ? tiles : ctx->sm_count;
    switch (s.K) {
        case 1: return launch_tc<1>(P, grid, smem, st);
        case 2: return launch_tc<2>(P, grid, smem, st);
        case 3: return launch_tc<3>(P, grid, smem, st);
        case 4: return launch_tc<4>(P, grid, smem, st);
        case 5: return launch_tc<5>(P, grid, smem, st);
        case 6: return launch_tc<6>(P, grid, smem, st);
        case 7: return launch_tc<7>(P, grid, smem, st);
        default: return launch_tc<8>(P, grid, smem, st);
    }
}
