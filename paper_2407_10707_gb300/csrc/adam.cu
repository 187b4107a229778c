// The Adam update of the training step (Kingma and Ba's algorithm, the
// optimiser of 3DGS training), all parameter groups in one launch:
//   m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2
//   p <- p - (lr / (1 - b1^t)) m / (sqrt(v) / sqrt(1 - b2^t) + eps)
// in FP32 (bias corrections formed on the host in FP64); BF16 parameters are
// read, updated in FP32 and rounded back (nearest even).  The groups form one
// index space of 4-element units, so a launch is balanced whatever the group
// sizes; a unit of a group whose four arrays are 16-byte aligned (8 bytes for
// a BF16 parameter) moves as vectors.  Bound by HBM: 28 B per FP32 element.
#include "common.cuh"

namespace {

constexpr int ADAM_THREADS = 256;

struct AdamParams {
    avatar_adam_group g[AVATAR_ADAM_MAX_GROUPS];
    long long off[AVATAR_ADAM_MAX_GROUPS + 1];  // first unit of each group; off[n_groups] = total
    float step_size[AVATAR_ADAM_MAX_GROUPS];    // lr / (1 - b1^t)
    int vec[AVATAR_ADAM_MAX_GROUPS];
    int n_groups;
    float b1, b2, eps, inv_sqrt_bc2;            // 1 / sqrt(1 - b2^t)
};

__device__ __forceinline__ float adam_one(float p, float g, float &m, float &v, float step, const AdamParams &P)
{
    m = fmaf(P.b1, m, (1.f - P.b1) * g);
    v = fmaf(P.b2, v, (1.f - P.b2) * g * g);
    return p - step * m / fmaf(sqrtf(v), P.inv_sqrt_bc2, P.eps);
}

__global__ void __launch_bounds__(ADAM_THREADS)
adam_kernel(AdamParams P)
{
    const long long total = P.off[P.n_groups];
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < total;
         u += (long long)gridDim.x * blockDim.x) {
        int k = 0;
        while (k + 1 < P.n_groups && u >= P.off[k + 1]) ++k;
        const avatar_adam_group &G = P.g[k];
        const long long i0 = (u - P.off[k]) * 4;
        const float step = P.step_size[k];
        const bool bf = G.dtype == AVATAR_DTYPE_BF16;
        if (P.vec[k] && i0 + 4 <= G.n) {
            float4 g4 = *reinterpret_cast<const float4 *>(G.grad + i0);
            float4 m4 = *reinterpret_cast<const float4 *>(G.m + i0);
            float4 v4 = *reinterpret_cast<const float4 *>(G.v + i0);
            float pv[4];
            if (bf) {
                const uint2 raw = *reinterpret_cast<const uint2 *>(reinterpret_cast<const __nv_bfloat16 *>(G.param) + i0);
                const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162 *>(&raw.x);
                const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162 *>(&raw.y);
                pv[0] = __low2float(lo);
                pv[1] = __high2float(lo);
                pv[2] = __low2float(hi);
                pv[3] = __high2float(hi);
            } else {
                const float4 p4 = *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(G.param) + i0);
                pv[0] = p4.x;
                pv[1] = p4.y;
                pv[2] = p4.z;
                pv[3] = p4.w;
            }
            pv[0] = adam_one(pv[0], g4.x, m4.x, v4.x, step, P);
            pv[1] = adam_one(pv[1], g4.y, m4.y, v4.y, step, P);
            pv[2] = adam_one(pv[2], g4.z, m4.z, v4.z, step, P);
            pv[3] = adam_one(pv[3], g4.w, m4.w, v4.w, step, P);
            *reinterpret_cast<float4 *>(G.m + i0) = m4;
            *reinterpret_cast<float4 *>(G.v + i0) = v4;
            if (bf) {
                const __nv_bfloat162 lo = __floats2bfloat162_rn(pv[0], pv[1]);
                const __nv_bfloat162 hi = __floats2bfloat162_rn(pv[2], pv[3]);
                uint2 raw;
                raw.x = *reinterpret_cast<const uint32_t *>(&lo);
                raw.y = *reinterpret_cast<const uint32_t *>(&hi);
                *reinterpret_cast<uint2 *>(reinterpret_cast<__nv_bfloat16 *>(G.param) + i0) = raw;
            } else {
                *reinterpret_cast<float4 *>(reinterpret_cast<float *>(G.param) + i0) =
                    make_float4(pv[0], pv[1], pv[2], pv[3]);
            }
        } else {
            for (long long i = i0; i < i0 + 4 && i < G.n; ++i) {
                float m = G.m[i], v = G.v[i];
                if (bf) {
                    __nv_bfloat16 *p = reinterpret_cast<__nv_bfloat16 *>(G.param) + i;
                    *p = __float2bfloat16_rn(adam_one(__bfloat162float(*p), G.grad[i], m, v, step, P));
                } else {
                    float *p = reinterpret_cast<float *>(G.param) + i;
                    *p = adam_one(*p, G.grad[i], m, v, step, P);
                }
                G.m[i] = m;
                G.v[i] = v;
            }
        }
    }
}

bool aligned(const void *p, uintptr_t a) { return (((uintptr_t)p) & (a - 1)) == 0; }

}  // namespace

extern "C" int avatar_adam(avatar_ctx *ctx, const avatar_adam_args *a, avatar_stream_t stream)
{
    if (!ctx || !a || a->n_groups < 0 || a->n_groups > AVATAR_ADAM_MAX_GROUPS || a->step < 1)
        return AVATAR_ERR_INVALID_ARG;
    if (!(a->beta1 >= 0.f && a->beta1 < 1.f) || !(a->beta2 >= 0.f && a->beta2 < 1.f) || !(a->eps > 0.f))
        return AVATAR_ERR_INVALID_ARG;
    AdamParams P;
    P.n_groups = a->n_groups;
    P.b1 = a->beta1;
    P.b2 = a->beta2;
    P.eps = a->eps;
    const double bc1 = 1.0 - pow((double)a->beta1, (double)a->step);
    const double bc2 = 1.0 - pow((double)a->beta2, (double)a->step);
    P.inv_sqrt_bc2 = (float)(1.0 / sqrt(bc2));
    long long total = 0;
    for (int k = 0; k < a->n_groups; ++k) {
        const avatar_adam_group &G = a->group[k];
        if (G.n < 0 || (G.dtype != AVATAR_DTYPE_F32 && G.dtype != AVATAR_DTYPE_BF16)) return AVATAR_ERR_INVALID_ARG;
        if (G.n > 0 && (!G.param || !G.grad || !G.m || !G.v)) return AVATAR_ERR_INVALID_ARG;
        P.g[k] = G;
        P.off[k] = total;
        total += (G.n + 3) / 4;
        P.step_size[k] = (float)((double)G.lr / bc1);
        P.vec[k] = aligned(G.grad, 16) && aligned(G.m, 16) && aligned(G.v, 16) &&
                   aligned(G.param, G.dtype == AVATAR_DTYPE_BF16 ? 8 : 16);
    }
    P.off[a->n_groups] = total;
    if (total == 0) return AVATAR_OK;
    long long blocks = (total + ADAM_THREADS - 1) / ADAM_THREADS;
    if (blocks > (long long)ctx->sm_count * 8) blocks = (long long)ctx->sm_count * 8;
    adam_kernel<<<(int)blocks, ADAM_THREADS, 0, (cudaStream_t)stream>>>(P);
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}
