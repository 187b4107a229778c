// The training regularisers of Sec. 3.3 (the terms of Eq. 6 beside the
// image loss), with their gradients:
//   L_smooth = sum_i sum_{k in S_v^i} |a_i - a_k|_1 + |gamma_i - gamma_k| + |p_i - p_k|
//   L_mdist  = sum_i sum_{k in S_g^i} || x_g^i - x_v^k ||_2
//   L_disp   = sum_i || dx^i ||_2
//   L_scale  = sum_i sum_c max(0, exp(logscale_ic) - s0)
// Two launches (one thread per Gaussian, one per vertex) accumulate their
// gradients into the caller's buffers and write per-block FP64 partial sums;
// a one-block reduction forms the four sums and adds the weighted total to
// the loss (deterministic).  The scatter of the smoothness gradient to the
// neighbours uses atomics.
#include "common.cuh"

namespace {

constexpr int REG_THREADS = 256;
constexpr int REG_MAX_K = 64;
constexpr int REG_MAX_BLOCKS = 1024;

__device__ __forceinline__ float sgn(float v) { return v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f); }

__device__ __forceinline__ void block_sum2(double a, double b, double *out)
{
    __shared__ double s[2][REG_THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s[0][threadIdx.x >> 5] = a;
        s[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int w = 0; w < REG_THREADS / 32; ++w) {
            x += s[0][w];
            y += s[1][w];
        }
        out[2 * blockIdx.x] = x;
        out[2 * blockIdx.x + 1] = y;
    }
}

// per Gaussian: mesh distance (terms[1]) and scale hinge (terms[3])
__global__ void __launch_bounds__(REG_THREADS)
reg_gauss_kernel(avatar_reg_args a, double *__restrict__ part)
{
    double s_md = 0.0, s_sc = 0.0;
    const int G = a.G, Nv = a.Nv;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const float x0 = a.xg[g], x1 = a.xg[G + g], x2 = a.xg[2 * G + g];
        float dx[3] = {0.f, 0.f, 0.f};
        for (int j = 0; j < a.Kg; ++j) {
            const int v = __ldg(a.knn + (size_t)j * G + g);
            if ((unsigned)v >= (unsigned)Nv) {
                av_report(a.status, AVATAR_ERR_INDEX);
                continue;
            }
            const float e0 = x0 - __ldg(a.xv + v), e1 = x1 - __ldg(a.xv + Nv + v), e2 = x2 - __ldg(a.xv + 2 * Nv + v);
            const float n = sqrtf(e0 * e0 + e1 * e1 + e2 * e2);
            s_md += n;
            if (n > 0.f) {
                const float inv = 1.f / n;
                dx[0] += e0 * inv;
                dx[1] += e1 * inv;
                dx[2] += e2 * inv;
            }
        }
        if (a.d_xg)
#pragma unroll
            for (int c = 0; c < 3; ++c) a.d_xg[(size_t)c * G + g] += a.w_mdist * dx[c];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float s = expf(ld_attr(a.logscale, (size_t)c * G + g, a.attr_dtype));
            if (s > a.s0) {
                s_sc += s - a.s0;
                if (a.d_logscale) a.d_logscale[(size_t)c * G + g] += a.w_scale * s;
            }
        }
    }
    block_sum2(s_md, s_sc, part);
}

// per vertex: smoothness (terms[0]) and displacement (terms[2])
__global__ void __launch_bounds__(REG_THREADS)
reg_vertex_kernel(avatar_reg_args a, double *__restrict__ part)
{
    double s_sm = 0.0, s_dp = 0.0;
    const int Nv = a.Nv;
    const int dt = a.attr_dtype;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < Nv; v += gridDim.x * blockDim.x) {
        float m[5];
#pragma unroll
        for (int c = 0; c < 3; ++c) m[c] = ld_attr(a.av, (size_t)c * Nv + v, dt);
        m[3] = ld_attr(a.rv, v, dt);
        m[4] = ld_attr(a.pv, v, dt);
        float gm[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        for (int j = 0; j < a.Kv; ++j) {
            const int k = __ldg(a.knn_v + (size_t)j * Nv + v);
            if ((unsigned)k >= (unsigned)Nv) {
                av_report(a.status, AVATAR_ERR_INDEX);
                continue;
            }
            float o[5];
#pragma unroll
            for (int c = 0; c < 3; ++c) o[c] = ld_attr(a.av, (size_t)c * Nv + k, dt);
            o[3] = ld_attr(a.rv, k, dt);
            o[4] = ld_attr(a.pv, k, dt);
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                const float d = m[c] - o[c];
                s_sm += fabsf(d);
                const float s = sgn(d);
                gm[c] += s;
                if (s != 0.f) {
                    float *dst = c < 3 ? (a.d_av ? a.d_av + (size_t)c * Nv + k : nullptr)
                                       : (c == 3 ? (a.d_rv ? a.d_rv + k : nullptr) : (a.d_pv ? a.d_pv + k : nullptr));
                    if (dst) atomicAdd(dst, -a.w_smooth * s);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (a.d_av) atomicAdd(a.d_av + (size_t)c * Nv + v, a.w_smooth * gm[c]);
        if (a.d_rv) atomicAdd(a.d_rv + v, a.w_smooth * gm[3]);
        if (a.d_pv) atomicAdd(a.d_pv + v, a.w_smooth * gm[4]);
        if (a.dxv) {
            const float d0 = a.dxv[v], d1 = a.dxv[Nv + v], d2 = a.dxv[2 * Nv + v];
            const float n = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
            s_dp += n;
            if (a.d_dxv && n > 0.f) {
                const float k = a.w_disp / n;
                a.d_dxv[v] += k * d0;
                a.d_dxv[Nv + v] += k * d1;
                a.d_dxv[2 * Nv + v] += k * d2;
            }
        }
    }
    block_sum2(s_sm, s_dp, part);
}

__global__ void __launch_bounds__(256)
reg_reduce_kernel(const double *__restrict__ pg, int ng, const double *__restrict__ pv, int nv, avatar_reg_args a)
{
    if (threadIdx.x == 0) {
        double md = 0.0, sc = 0.0, sm = 0.0, dp = 0.0;
        for (int i = 0; i < ng; ++i) {
            md += pg[2 * i];
            sc += pg[2 * i + 1];
        }
        for (int i = 0; i < nv; ++i) {
            sm += pv[2 * i];
            dp += pv[2 * i + 1];
        }
        if (a.terms) {
            a.terms[0] = (float)sm;
            a.terms[1] = (float)md;
            a.terms[2] = (float)dp;
            a.terms[3] = (float)sc;
        }
        const double total = a.w_smooth * sm + a.w_mdist * md + a.w_disp * dp + a.w_scale * sc;
        if (a.loss) *a.loss = a.accumulate ? *a.loss + (float)total : (float)total;
    }
}

int check_reg(const avatar_reg_args *a)
{
    if (!a || a->G < 0 || a->Nv < 1 || a->Kg < 0 || a->Kg > REG_MAX_K || a->Kv < 0 || a->Kv > REG_MAX_K)
        return AVATAR_ERR_INVALID_ARG;
    if (a->attr_dtype != AVATAR_DTYPE_F32 && a->attr_dtype != AVATAR_DTYPE_BF16) return AVATAR_ERR_INVALID_ARG;
    if (a->G > 0 && (!a->xg || !a->logscale || (a->Kg > 0 && !a->knn))) return AVATAR_ERR_INVALID_ARG;
    if (!a->xv || !a->av || !a->rv || !a->pv || (a->Kv > 0 && !a->knn_v)) return AVATAR_ERR_INVALID_ARG;
    return AVATAR_OK;
}

int grid_of(const avatar_ctx *ctx, int n)
{
    int b = (n + REG_THREADS - 1) / REG_THREADS;
    if (b > ctx->sm_count * 8) b = ctx->sm_count * 8;
    if (b > REG_MAX_BLOCKS) b = REG_MAX_BLOCKS;
    return b < 1 ? 1 : b;
}

const size_t REG_HALF = av_align256((size_t)2 * REG_MAX_BLOCKS * sizeof(double));

}  // namespace

extern "C" size_t avatar_regularizers_workspace_size(const avatar_reg_args *a)
{
    if (check_reg(a) != AVATAR_OK) return 0;
    return 2 * REG_HALF;  // per-block partial sums of the two kernels
}

extern "C" int avatar_regularizers(avatar_ctx *ctx, const avatar_reg_args *a, void *ws, size_t ws_bytes,
                                   avatar_stream_t stream)
{
    if (!ctx) return AVATAR_ERR_INVALID_ARG;
    AV_TRY(check_reg(a));
    if (!ws || (((uintptr_t)ws) & 255)) return AVATAR_ERR_WORKSPACE;
    const int gg = grid_of(ctx, a->G), gv = grid_of(ctx, a->Nv);
    if (ws_bytes < 2 * REG_HALF) return AVATAR_ERR_WORKSPACE;
    double *pg = (double *)ws, *pv = (double *)((char *)ws + REG_HALF);
    cudaStream_t st = (cudaStream_t)stream;
    reg_gauss_kernel<<<gg, REG_THREADS, 0, st>>>(*a, pg);
    reg_vertex_kernel<<<gv, REG_THREADS, 0, st>>>(*a, pv);
    reg_reduce_kernel<<<1, 256, 0, st>>>(pg, gg, pv, gv, *a);
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}
