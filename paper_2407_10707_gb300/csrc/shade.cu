// (c) Shading of every Gaussian with the discrete rendering equation -
// Eq. 2, BRDF of App. A, back-face cull and gamma of Sec. 3.1.
//
// Work split: one warp per Gaussian, lanes over the lights (light k is
// handled by lane k % 32 in chunk k / 32).  The light table (w_k, L_k A_k)
// is staged once per block in shared memory; the visibility words of the K
// neighbours for a 32-light chunk are warp-uniform loads, and each lane
// extracts its own bit.  Per-Gaussian sums are reduced with shuffles.  The
// backward pass finds the lit lights the same way, queues them per warp and
// evaluates their adjoint terms 32 at a time; per-light gradients accumulate
// in shared memory and are flushed once per block.
#include <algorithm>

#include "batch_internal.h"
#include "common.cuh"

namespace {

constexpr int SHADE_THREADS = 256;
constexpr int SHADE_Q = 64;  // backward: per-warp queue of lit lights (float4 entries)
constexpr size_t SHADE_Q_BYTES = (size_t)(SHADE_THREADS / 32) * SHADE_Q * sizeof(float4);
constexpr float FRES_C1 = -5.55473f;
constexpr float FRES_C0 = -6.98316f;
constexpr float INV_GAMMA = 1.0f / 2.2f;

template <int K>
struct GaussIn {
    float x[3], n[3], a[3], r, p;
    float ub[K];
    int nb[K];
};

// Batched launches (blockIdx.y = view): the views' poses, camera centres and
// the two strides.  Per-pose arrays (xd, nd, bits, light_L) hold B poses
// with channel stride B G; per-view arrays (color, radiance, cull and the
// gradients) hold V views with channel stride V G.  A single frame is
// B = V = 1 with null tables.
struct ShadeBatch {
    int B, V;
    const int32_t *view_pose;  // [V] or NULL
    const float *view_cc;      // [V][3] or NULL (then args.cam_center)
    int dB_copies;             // backward: light-gradient accumulator copies (1, or one per warp)
};

struct ShadeSlot {
    int p, y;       // pose, view
    size_t SG, VG;  // channel strides of per-pose and per-view arrays
    size_t op, oy;  // element offsets p G and y G
    float C[3];     // camera centre
};

__device__ __forceinline__ ShadeSlot shade_slot(const avatar_shade_args &s, const ShadeBatch &sb)
{
    ShadeSlot t;
    t.y = blockIdx.y;
    t.p = sb.view_pose ? __ldg(sb.view_pose + t.y) : 0;
    t.SG = (size_t)sb.B * s.G;
    t.VG = (size_t)sb.V * s.G;
    t.op = (size_t)t.p * s.G;
    t.oy = (size_t)t.y * s.G;
#pragma unroll
    for (int i = 0; i < 3; ++i) t.C[i] = sb.view_cc ? __ldg(sb.view_cc + 3 * t.y + i) : s.cam_center[i];
    return t;
}

template <int K>
__device__ __forceinline__ bool load_gauss(const avatar_shade_args &s, int g, GaussIn<K> &q, size_t SG = 0,
                                           size_t op = 0)
{
    const int G = s.G;
    if (SG == 0) SG = (size_t)G;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        q.x[i] = __ldg(s.xd + (size_t)i * SG + op + g);
        q.n[i] = __ldg(s.nd + (size_t)i * SG + op + g);
        q.a[i] = __ldg(s.ag + (size_t)i * G + g);
    }
    q.r = __ldg(s.rg + g);
    q.p = __ldg(s.pg + g);
    bool ok = true;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        q.ub[j] = __ldg(s.ubar + (size_t)j * G + g);
        q.nb[j] = __ldg(s.knn + (size_t)j * G + g);
        if ((unsigned)q.nb[j] >= (unsigned)s.Nv) ok = false;
    }
    return ok;
}

// Exact FP32 back-face decision (identical operation order to the header).
__device__ __forceinline__ bool is_culled(const float *x, const float *n, const float *C)
{
    float d0 = __fsub_rn(C[0], x[0]), d1 = __fsub_rn(C[1], x[1]), d2 = __fsub_rn(C[2], x[2]);
    float s = __fmaf_rn(n[2], d2, __fmaf_rn(n[1], d1, __fmul_rn(n[0], d0)));
    return !(s > 0.0f);
}

struct Frame {
    float wo[3];
    float co_raw, co;
    float a2, kk, Go;
    float inv_len;
};

template <int K>
__device__ __forceinline__ Frame view_frame(const GaussIn<K> &q, const float *C)
{
    Frame f;
    float v0 = C[0] - q.x[0], v1 = C[1] - q.x[1], v2 = C[2] - q.x[2];
    float il = rsqrtf(v0 * v0 + v1 * v1 + v2 * v2);
    f.inv_len = il;
    f.wo[0] = v0 * il;
    f.wo[1] = v1 * il;
    f.wo[2] = v2 * il;
    f.co_raw = q.n[0] * f.wo[0] + q.n[1] * f.wo[1] + q.n[2] * f.wo[2];
    f.co = fmaxf(f.co_raw, 0.f);
    float alpha = q.r * q.r;
    f.a2 = alpha * alpha;
    f.kk = (q.r + 1.f) * (q.r + 1.f) * 0.125f;
    f.Go = f.co * (1.f - f.kk) + f.kk;
    return f;
}

// Neighbour visibility words of one 32-light chunk (warp-uniform loads) and
// their AND / OR, which settle vis = 1 / vis = 0 without per-bit work.
template <int K>
struct ChunkBits {
    unsigned w[K];
    unsigned all, any;
};

template <int K>
__device__ __forceinline__ void load_chunk(const uint32_t *__restrict__ bits, const GaussIn<K> &q, int OW, int ch,
                                           ChunkBits<K> &cb)
{
    cb.all = 0xffffffffu;
    cb.any = 0u;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        cb.w[j] = __ldg(bits + (size_t)q.nb[j] * OW + ch);
        cb.all &= cb.w[j];
        cb.any |= cb.w[j];
    }
}

// vis = sum_j ubar_j bit_j for this lane's light (Eq. 1 applied to v).
template <int K>
__device__ __forceinline__ float lane_vis(const ChunkBits<K> &cb, const GaussIn<K> &q, unsigned bit)
{
    if (cb.all & bit) return 1.0f;  // sum of the normalised Eq. 1 weights
    if (!(cb.any & bit)) return 0.0f;
    float vis = 0.f;
#pragma unroll
    for (int j = 0; j < K; ++j)
        if (cb.w[j] & bit) vis += q.ub[j];
    return vis;
}

// Soft visibility of light k (lane) from the filtered vertex counts.
template <int K>
__device__ __forceinline__ float soft_vis(const uint8_t *__restrict__ vc, int NL, const GaussIn<K> &q, int k,
                                          float inv_den, float (&c)[K])
{
    float vis = 0.f;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        c[j] = (float)__ldg(vc + (size_t)q.nb[j] * NL + k) * inv_den;
        vis = fmaf(q.ub[j], c[j], vis);
    }
    return vis;
}

template <int K, bool SOFT>
__global__ void __launch_bounds__(SHADE_THREADS)
shade_kernel(avatar_shade_args s, ShadeBatch sb)
{
    extern __shared__ float4 lsm[];  // [NL] (w, 0) then [NL] (L*A, 0)
    const int NL = s.NL, G = s.G;
    const ShadeSlot t = shade_slot(s, sb);
    const int OW = (NL + 31) / 32;
    const float *light_L = s.light_L + (size_t)t.p * NL * 3;
    const uint32_t *bits = s.bits + (size_t)t.p * s.Nv * OW;
    float *color = s.color + t.oy;
    float *radiance = s.radiance ? s.radiance + t.oy : nullptr;
    uint8_t *cull = s.cull ? s.cull + t.oy : nullptr;
    float4 *lw = lsm, *lb = lsm + NL;
    for (int k = threadIdx.x; k < NL; k += blockDim.x) {
        float A = __ldg(s.light_A + k);
        lw[k] = make_float4(__ldg(s.light_w + 3 * k), __ldg(s.light_w + 3 * k + 1), __ldg(s.light_w + 3 * k + 2), 0.f);
        lb[k] = make_float4(__ldg(light_L + 3 * k) * A, __ldg(light_L + 3 * k + 1) * A, __ldg(light_L + 3 * k + 2) * A,
                            0.f);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned bit = 1u << lane;
    const int warps_total = gridDim.x * (blockDim.x >> 5);
    const float *C = t.C;
    for (int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < G; g += warps_total) {
        GaussIn<K> q;
        bool ok = load_gauss<K>(s, g, q, t.SG, t.op);
        if (!ok && lane == 0) av_report(s.status, AVATAR_ERR_INDEX);
        if (is_culled(q.x, q.n, C) || !ok) {
            if (lane < 3) {
                color[(size_t)lane * t.VG + g] = 0.f;
                if (radiance) radiance[(size_t)lane * t.VG + g] = 0.f;
            }
            if (lane == 0 && cull) cull[g] = 1;
            continue;
        }
        Frame f = view_frame<K>(q, C);
        const float spec_scale = f.a2 / (4.f * AV_PI * f.Go);
        const float a2m1 = f.a2 - 1.f, omk = 1.f - f.kk;
        const float ia0 = q.a[0] * (1.f / AV_PI), ia1 = q.a[1] * (1.f / AV_PI), ia2 = q.a[2] * (1.f / AV_PI);
        float L0 = 0.f, L1 = 0.f, L2 = 0.f;  // this lane's share of L_o
        for (int ch = 0; ch < OW; ++ch) {
            const int k = ch * 32 + lane;
            float vis;
            if constexpr (SOFT) {
                if (k >= NL) continue;
                float cj[K];
                vis = soft_vis<K>(s.vis_count, NL, q, k, 1.0f / (float)s.vis_den, cj);
                if (vis == 0.f) continue;
            } else {
                ChunkBits<K> cb;
                load_chunk<K>(bits, q, OW, ch, cb);
                if (k >= NL || !(cb.any & bit)) continue;
                vis = lane_vis<K>(cb, q, bit);
            }
            float4 w = lw[k];
            float ci = q.n[0] * w.x + q.n[1] * w.y + q.n[2] * w.z;
            if (!(ci > 0.f)) continue;
            float fw = vis * ci;
            float4 B = lb[k];
            float dwo = w.x * f.wo[0] + w.y * f.wo[1] + w.z * f.wo[2];
            float fs = 0.f;
            float len2 = 2.f + 2.f * dwo;
            if (len2 > 0.f) {
                float rinv = rsqrtf(len2);
                float nh = (ci + f.co_raw) * rinv;
                float voh = (1.f + dwo) * rinv;
                float den = fmaf(nh * nh, a2m1, 1.f);
                float Fr = fmaf(0.96f, exp2f(fmaf(FRES_C1, voh, FRES_C0) * voh), 0.04f);
                float Gi = fmaf(ci, omk, f.kk);
                fs = spec_scale * __fdividef(Fr, den * den * Gi);
            }
            float ps = q.p * fs;
            L0 = fmaf(B.x * fw, ia0 + ps, L0);
            L1 = fmaf(B.y * fw, ia1 + ps, L1);
            L2 = fmaf(B.z * fw, ia2 + ps, L2);
        }
        L0 = warp_sum(L0);
        L1 = warp_sum(L1);
        L2 = warp_sum(L2);
        if (lane < 3) {
            float Lo = lane == 0 ? L0 : (lane == 1 ? L1 : L2);
            float col = exp2f(log2f(fmaxf(Lo, 1e-6f)) * INV_GAMMA);
            color[(size_t)lane * t.VG + g] = col;
            if (radiance) radiance[(size_t)lane * t.VG + g] = Lo;
        }
        if (lane == 0 && cull) cull[g] = 0;
    }
}

// ---------------------------------------------------------------- backward
template <int K, bool SOFT>
__global__ void __launch_bounds__(SHADE_THREADS)
shade_backward_kernel(avatar_shade_args s, avatar_shade_grads gr, ShadeBatch sb)
{
    extern __shared__ float4 lsm[];  // [NL] (w, A) ; [NL] (L*A) ; per warp [NL] dL/dB accumulators (x, y, z, -)
    const int NL = s.NL, G = s.G;
    const ShadeSlot t = shade_slot(s, sb);
    const int OW = (NL + 31) / 32;
    const size_t VG = t.VG;
    const float *light_L = s.light_L + (size_t)t.p * NL * 3;
    const uint32_t *bits = s.bits + (size_t)t.p * s.Nv * OW;
    const float *radiance = s.radiance + t.oy;
    // per-view gradient slices; dL/dL^k of the view's pose
    gr.d_color += t.oy;
    gr.d_xd += t.oy;
    gr.d_nd += t.oy;
    gr.d_ag += t.oy;
    gr.d_rg += t.oy;
    gr.d_pg += t.oy;
    gr.d_ubar += t.oy;
    gr.d_light_L += (size_t)t.p * NL * 3;
    float4 *lw = lsm, *lb = lsm + NL;
    // With one accumulator copy per warp, each warp adds dL/dB of the lights its
    // lanes own (light k belongs to lane k % 32 in every warp) to its own slots
    // without atomics, and the copies are summed once at the end; with a single
    // copy (many lights) the warps add with shared-memory atomics.
    const int copies = sb.dB_copies;
    const bool private_dB = copies == (int)(blockDim.x >> 5);
    float4 *dBall = lsm + 2 * NL;
    float4 *dB = dBall + (size_t)(private_dB ? (threadIdx.x >> 5) : 0) * NL;
    for (int k = threadIdx.x; k < NL; k += blockDim.x) {
        float A = __ldg(s.light_A + k);
        lw[k] = make_float4(__ldg(s.light_w + 3 * k), __ldg(s.light_w + 3 * k + 1), __ldg(s.light_w + 3 * k + 2), A);
        lb[k] = make_float4(__ldg(light_L + 3 * k) * A, __ldg(light_L + 3 * k + 1) * A, __ldg(light_L + 3 * k + 2) * A,
                            0.f);
    }
    for (int i = threadIdx.x; i < copies * NL; i += blockDim.x) dBall[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned bit = 1u << lane;
    const int warps_total = gridDim.x * (blockDim.x >> 5);
    const float *C = t.C;
    for (int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < G; g += warps_total) {
        GaussIn<K> q;
        bool ok = load_gauss<K>(s, g, q, t.SG, t.op);
        float dLo[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float Lo = __ldg(radiance + (size_t)c * VG + g);
            float dc = __ldg(gr.d_color + (size_t)c * VG + g);
            dLo[c] = (Lo > 1e-6f) ? dc * INV_GAMMA * exp2f(log2f(Lo) * (INV_GAMMA - 1.f)) : 0.f;
        }
        if (!ok || is_culled(q.x, q.n, C) || (dLo[0] == 0.f && dLo[1] == 0.f && dLo[2] == 0.f)) {
            if (lane < 3) {
                gr.d_xd[(size_t)lane * VG + g] = 0.f;
                gr.d_nd[(size_t)lane * VG + g] = 0.f;
                gr.d_ag[(size_t)lane * VG + g] = 0.f;
            }
            if (lane == 0) {
                gr.d_rg[g] = 0.f;
                gr.d_pg[g] = 0.f;
            }
            if (lane < K) gr.d_ubar[(size_t)lane * VG + g] = 0.f;
            continue;
        }
        Frame f = view_frame<K>(q, C);
        const float spec_scale = f.a2 / (4.f * AV_PI * f.Go);
        const float a2m1 = f.a2 - 1.f, omk = 1.f - f.kk;
        const float ia0 = q.a[0] * (1.f / AV_PI), ia1 = q.a[1] * (1.f / AV_PI), ia2 = q.a[2] * (1.f / AV_PI);
        float E0 = 0.f, E1 = 0.f, E2 = 0.f;
        float dnv0 = 0.f, dnv1 = 0.f, dnv2 = 0.f, dwv0 = 0.f, dwv1 = 0.f, dwv2 = 0.f;
        float dco = 0.f, da2 = 0.f, dkk = 0.f, dp = 0.f;
        float dub[K];
#pragma unroll
        for (int j = 0; j < K; ++j) dub[j] = 0.f;
        // light k, lit (ci > 0) with visibility vis and per-neighbour
        // visibilities cj: its terms of the adjoint
        auto lit = [&](int k, float vis, float ci, const float (&cj)[K]) {
            const float4 w = lw[k];
            float4 B = lb[k];
            float Q = dLo[0] * B.x + dLo[1] * B.y + dLo[2] * B.z;
            float Qa = ia0 * dLo[0] * B.x + ia1 * dLo[1] * B.y + ia2 * dLo[2] * B.z;
            float fw = vis * ci;
            E0 = fmaf(B.x, fw, E0);
            E1 = fmaf(B.y, fw, E1);
            E2 = fmaf(B.z, fw, E2);
            float fs = 0.f, dci = 0.f;
            float dwo = w.x * f.wo[0] + w.y * f.wo[1] + w.z * f.wo[2];
            float len2 = 2.f + 2.f * dwo;
            if (len2 > 0.f) {
                float rinv = rsqrtf(len2);
                float nh = (ci + f.co_raw) * rinv;
                float voh = (1.f + dwo) * rinv;
                float den = fmaf(nh * nh, a2m1, 1.f);
                float ex = exp2f(fmaf(FRES_C1, voh, FRES_C0) * voh);
                float Fr = fmaf(0.96f, ex, 0.04f);
                float Gi = fmaf(ci, omk, f.kk);
                float base = spec_scale * __fdividef(1.f, den * den * Gi);  // fs / Fr
                fs = base * Fr;
                float dfs = fw * q.p * Q;
                dp = fmaf(fw * fs, Q, dp);
                // fs = a2 Fr / (4 pi den^2 Gi Go)
                float dFr = dfs * base;
                float dden = -2.f * dfs * fs * __fdividef(1.f, den);
                float dGi = -dfs * fs * __fdividef(1.f, Gi);
                float dGo = -dfs * fs * __fdividef(1.f, f.Go);
                da2 += dfs * fs * __fdividef(1.f, f.a2) + dden * nh * nh;
                float dnh = dden * 2.f * nh * a2m1;
                float dvoh = dFr * 0.96f * ex * 0.69314718056f * (2.f * FRES_C1 * voh + FRES_C0);
                dci += dGi * omk;
                dkk += dGi * (1.f - ci) + dGo * (1.f - f.co);
                if (f.co_raw > 0.f) dco += dGo * omk;
                dci += dnh * rinv;
                dco += dnh * rinv;
                float drinv = dnh * (ci + f.co_raw) + dvoh * (1.f + dwo);
                float ddwo = dvoh * rinv - drinv * rinv * rinv * rinv;
                dwv0 = fmaf(ddwo, w.x, dwv0);
                dwv1 = fmaf(ddwo, w.y, dwv1);
                dwv2 = fmaf(ddwo, w.z, dwv2);
            }
            float term = Qa + q.p * fs * Q;  // sum_c dLo_c B_c (a_c/pi + p fs)
            dci += vis * term;
            float dvis = ci * term;
#pragma unroll
            for (int j = 0; j < K; ++j) dub[j] = fmaf(dvis, cj[j], dub[j]);
            dnv0 = fmaf(dci, w.x, dnv0);
            dnv1 = fmaf(dci, w.y, dnv1);
            dnv2 = fmaf(dci, w.z, dnv2);
            // dL/dB_kc = dLo_c vis ci (a_c/pi + p fs)
            float ps = q.p * fs;
            if (private_dB) {
                float4 acc = dB[k];
                acc.x = fmaf(dLo[0] * fw, ia0 + ps, acc.x);
                acc.y = fmaf(dLo[1] * fw, ia1 + ps, acc.y);
                acc.z = fmaf(dLo[2] * fw, ia2 + ps, acc.z);
                dB[k] = acc;
            } else {
                atomicAdd(&dB[k].x, dLo[0] * fw * (ia0 + ps));
                atomicAdd(&dB[k].y, dLo[1] * fw * (ia1 + ps));
                atomicAdd(&dB[k].z, dLo[2] * fw * (ia2 + ps));
            }
        };
        if constexpr (SOFT) {
            for (int ch = 0; ch < OW; ++ch) {
                const int k = ch * 32 + lane;
                if (k >= NL) continue;
                float cj[K];
                const float vis = soft_vis<K>(s.vis_count, NL, q, k, 1.0f / (float)s.vis_den, cj);
                if (vis == 0.f) continue;
                const float4 w = lw[k];
                const float ci = q.n[0] * w.x + q.n[1] * w.y + q.n[2] * w.z;
                if (ci > 0.f) lit(k, vis, ci, cj);
            }
        } else {
            // Lanes find the lit lights of each 32-light chunk that some
            // neighbour sees; they go to the warp's queue (light, vis, ci,
            // neighbour bits), whose terms are evaluated 32 at a time, so no
            // lane idles through the adjoint of a dark light.  Within a
            // Gaussian every light appears once, so the lanes of a round own
            // distinct dL/dB slots.  (The forward's term is too cheap to pay
            // for the queue: 211 us with the per-lane loop, 227 us queued.)
            float4 *qe = lsm + (size_t)(2 + copies) * NL + (threadIdx.x >> 5) * SHADE_Q;
            auto run = [&](const float4 &e) {
                const int cb = __float_as_int(e.w);
                float cj[K];
#pragma unroll
                for (int j = 0; j < K; ++j) cj[j] = (cb >> j) & 1 ? 1.f : 0.f;
                lit(__float_as_int(e.x), e.y, e.z, cj);
            };
            int qn = 0;  // warp-uniform
            for (int ch = 0; ch < OW; ++ch) {
                const int k = ch * 32 + lane;
                ChunkBits<K> cb;
                load_chunk<K>(bits, q, OW, ch, cb);
                bool on = false;
                float vis = 0.f, ci = 0.f;
                int nbits = 0;
                if (k < NL && (cb.any & bit)) {
                    vis = lane_vis<K>(cb, q, bit);
                    const float4 w = lw[k];
                    ci = q.n[0] * w.x + q.n[1] * w.y + q.n[2] * w.z;
                    on = ci > 0.f;
#pragma unroll
                    for (int j = 0; j < K; ++j) nbits |= (cb.w[j] & bit) ? 1 << j : 0;
                }
                const unsigned m = __ballot_sync(0xffffffffu, on);
                if (on) qe[qn + __popc(m & (bit - 1u))] = make_float4(__int_as_float(k), vis, ci, __int_as_float(nbits));
                qn += __popc(m);
                if (qn >= 32) {
                    __syncwarp();
                    const float4 e = qe[qn - 32 + lane];
                    __syncwarp();
                    run(e);
                    qn -= 32;
                }
            }
            __syncwarp();
            if (lane < qn) run(qe[lane]);
            __syncwarp();
        }
        {
            // the 13 + K sums: sixteen at once by recursive halving, gathered to lane 0
            constexpr int NV = 13 + K;
            float vals[NV] = {E0, E1, E2, dnv0, dnv1, dnv2, dwv0, dwv1, dwv2, dco, da2, dkk, dp};
#pragma unroll
            for (int j = 0; j < K; ++j) vals[13 + j] = dub[j];
            float v16[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) v16[i] = i < NV ? vals[i] : 0.f;
            const float tot = warp_reduce_scatter16(v16);
#pragma unroll
            for (int i = 0; i < NV; ++i)
                vals[i] = i < 16 ? __shfl_sync(0xffffffffu, tot, 2 * i) : warp_sum(vals[i]);
            E0 = vals[0], E1 = vals[1], E2 = vals[2];
            dnv0 = vals[3], dnv1 = vals[4], dnv2 = vals[5];
            dwv0 = vals[6], dwv1 = vals[7], dwv2 = vals[8];
            dco = vals[9], da2 = vals[10], dkk = vals[11], dp = vals[12];
#pragma unroll
            for (int j = 0; j < K; ++j) dub[j] = vals[13 + j];
        }
        if (lane == 0) {
            float dn[3] = {dnv0 + dco * f.wo[0], dnv1 + dco * f.wo[1], dnv2 + dco * f.wo[2]};
            float dw[3] = {dwv0 + dco * q.n[0], dwv1 + dco * q.n[1], dwv2 + dco * q.n[2]};
            float dd = dw[0] * f.wo[0] + dw[1] * f.wo[1] + dw[2] * f.wo[2];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                gr.d_nd[(size_t)c * VG + g] = dn[c];
                gr.d_xd[(size_t)c * VG + g] = -(dw[c] - dd * f.wo[c]) * f.inv_len;
            }
            gr.d_ag[g] = dLo[0] * E0 * (1.f / AV_PI);
            gr.d_ag[VG + g] = dLo[1] * E1 * (1.f / AV_PI);
            gr.d_ag[2 * VG + g] = dLo[2] * E2 * (1.f / AV_PI);
            float alpha = q.r * q.r;
            gr.d_rg[g] = da2 * 4.f * alpha * q.r + dkk * (q.r + 1.f) * 0.25f;
            gr.d_pg[g] = dp;
#pragma unroll
            for (int j = 0; j < K; ++j) gr.d_ubar[(size_t)j * VG + g] = dub[j];
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NL; k += blockDim.x) {
        const float A = lw[k].w;
        float4 v = dBall[k];
        for (int w = 1; w < copies; ++w) {
            const float4 u = dBall[(size_t)w * NL + k];
            v.x += u.x;
            v.y += u.y;
            v.z += u.z;
        }
        if (v.x != 0.f) atomicAdd(gr.d_light_L + 3 * k, v.x * A);
        if (v.y != 0.f) atomicAdd(gr.d_light_L + 3 * k + 1, v.y * A);
        if (v.z != 0.f) atomicAdd(gr.d_light_L + 3 * k + 2, v.z * A);
    }
}

// Light-gradient accumulator copies of the backward: one per warp when they
// fit in shared memory beside the light tables, else one shared copy.
int bwd_copies(const avatar_ctx *ctx, int NL)
{
    const size_t per_warp = (size_t)(2 + SHADE_THREADS / 32) * NL * sizeof(float4) + SHADE_Q_BYTES;
    return per_warp <= (size_t)ctx->max_smem_optin ? SHADE_THREADS / 32 : 1;
}

template <int K>
int launch_shade(const avatar_shade_args &a, const ShadeBatch &sb, int grid, size_t smem, cudaStream_t st)
{
    auto kern = a.vis_count ? shade_kernel<K, true> : shade_kernel<K, false>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return AVATAR_ERR_CUDA;
    kern<<<dim3(grid, sb.V), SHADE_THREADS, smem, st>>>(a, sb);
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}

template <int K>
int launch_shade_bwd(const avatar_shade_args &a, const avatar_shade_grads &g, const ShadeBatch &sb, int grid,
                     size_t smem, int sm_count, cudaStream_t st)
{
    auto kern = a.vis_count ? shade_backward_kernel<K, true> : shade_backward_kernel<K, false>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return AVATAR_ERR_CUDA;
    // One wave of resident blocks: every block ends with a barrier before its
    // light-gradient flush, so many Gaussians per warp (whose cost ranges from
    // a culled one's few instructions to a lit one's thousands) keep the
    // block's warps finishing together, and fewer blocks flush.
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SHADE_THREADS, smem) == cudaSuccess && per_sm > 0)
        grid = std::min(grid, per_sm * sm_count);
    kern<<<dim3(grid, sb.V), SHADE_THREADS, smem, st>>>(a, g, sb);
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}

int check_shade(const avatar_shade_args *a)
{
    if (!a || a->G < 0 || a->K < 1 || a->K > 8 || a->NL < 1 || a->NL > 4096 || a->Nv < 1)
        return AVATAR_ERR_INVALID_ARG;
    if (a->G > 0 && (!a->xd || !a->nd || !a->ag || !a->rg || !a->pg || !a->ubar || !a->knn ||
                     (!a->bits && !a->vis_count) || !a->color))
        return AVATAR_ERR_INVALID_ARG;
    if (a->vis_count && a->vis_den < 1) return AVATAR_ERR_INVALID_ARG;
    if (!a->light_L || !a->light_A || !a->light_w) return AVATAR_ERR_INVALID_ARG;
    return AVATAR_OK;
}

int shade_grid(const avatar_ctx *ctx, int G)
{
    long warps = G;
    long blocks = (warps + SHADE_THREADS / 32 - 1) / (SHADE_THREADS / 32);
    long cap = (long)ctx->sm_count * 8;
    if (blocks > cap) blocks = cap;
    return blocks < 1 ? 1 : (int)blocks;
}

__global__ void __launch_bounds__(256)
cull_kernel(const float *__restrict__ xd, const float *__restrict__ nd, int G, float c0, float c1, float c2,
            uint8_t *__restrict__ cull)
{
    const float C[3] = {c0, c1, c2};
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const float x[3] = {__ldg(xd + g), __ldg(xd + (size_t)G + g), __ldg(xd + 2 * (size_t)G + g)};
        const float n[3] = {__ldg(nd + g), __ldg(nd + (size_t)G + g), __ldg(nd + 2 * (size_t)G + g)};
        cull[g] = is_culled(x, n, C) ? 1 : 0;
    }
}

}  // namespace

extern "C" int avatar_cull(avatar_ctx *ctx, const avatar_shade_args *a, avatar_stream_t stream)
{
    if (!ctx || !a || a->G < 0) return AVATAR_ERR_INVALID_ARG;
    if (a->G == 0) return AVATAR_OK;
    if (!a->xd || !a->nd || !a->cull) return AVATAR_ERR_INVALID_ARG;
    long blocks = ((long)a->G + 255) / 256;
    if (blocks > (long)ctx->sm_count * 8) blocks = (long)ctx->sm_count * 8;
    cull_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(a->xd, a->nd, a->G, a->cam_center[0], a->cam_center[1],
                                                               a->cam_center[2], a->cull);
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}

extern "C" int avatar_shade(avatar_ctx *ctx, const avatar_shade_args *a, avatar_stream_t stream)
{
    if (!ctx) return AVATAR_ERR_INVALID_ARG;
    AV_TRY(check_shade(a));
    if (a->G == 0) return AVATAR_OK;
    size_t smem = (size_t)2 * a->NL * sizeof(float4);
    int grid = shade_grid(ctx, a->G);
    cudaStream_t st = (cudaStream_t)stream;
    const ShadeBatch sb{1, 1, nullptr, nullptr, 1};
    switch (a->K) {
        case 1: return launch_shade<1>(*a, sb, grid, smem, st);
        case 2: return launch_shade<2>(*a, sb, grid, smem, st);
        case 3: return launch_shade<3>(*a, sb, grid, smem, st);
        case 4: return launch_shade<4>(*a, sb, grid, smem, st);
        case 5: return launch_shade<5>(*a, sb, grid, smem, st);
        case 6: return launch_shade<6>(*a, sb, grid, smem, st);
        case 7: return launch_shade<7>(*a, sb, grid, smem, st);
        default: return launch_shade<8>(*a, sb, grid, smem, st);
    }
}

extern "C" int avatar_shade_backward(avatar_ctx *ctx, const avatar_shade_args *a, const avatar_shade_grads *g,
                                     avatar_stream_t stream)
{
    if (!ctx || !g) return AVATAR_ERR_INVALID_ARG;
    AV_TRY(check_shade(a));
    if (!a->radiance || !g->d_color || !g->d_xd || !g->d_nd || !g->d_ag || !g->d_rg || !g->d_pg || !g->d_ubar ||
        !g->d_light_L)
        return AVATAR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(g->d_light_L, 0, (size_t)a->NL * 3 * sizeof(float), st) != cudaSuccess)
        return AVATAR_ERR_CUDA;
    if (a->G == 0) return AVATAR_OK;
    const int copies = bwd_copies(ctx, a->NL);
    size_t smem = (size_t)(2 + copies) * a->NL * sizeof(float4) + SHADE_Q_BYTES;
    int grid = shade_grid(ctx, a->G);
    const ShadeBatch sb{1, 1, nullptr, nullptr, copies};
    switch (a->K) {
        case 1: return launch_shade_bwd<1>(*a, *g, sb, grid, smem, ctx->sm_count, st);
        case 2: return launch_shade_bwd<2>(*a, *g, sb, grid, smem, ctx->sm_count, st);
        case 3: return launch_shade_bwd<3>(*a, *g, sb, grid, smem, ctx->sm_count, st);
        case 4: return launch_shade_bwd<4>(*a, *g, sb, grid, smem, ctx->sm_count, st);
        case 5: return launch_shade_bwd<5>(*a, *g, sb, grid, smem, ctx->sm_count, st);
        case 6: return launch_shade_bwd<6>(*a, *g, sb, grid, smem, ctx->sm_count, st);
        case 7: return launch_shade_bwd<7>(*a, *g, sb, grid, smem, ctx->sm_count, st);
        default: return launch_shade_bwd<8>(*a, *g, sb, grid, smem, ctx->sm_count, st);
    }
}

int av_shade_batch(avatar_ctx *ctx, const avatar_shade_args *a, int B, int V, const int32_t *view_pose,
                   const float *view_cc, cudaStream_t st)
{
    if (!ctx || B < 1 || V < 1 || V > 65535 || !view_pose || !view_cc) return AVATAR_ERR_INVALID_ARG;
    AV_TRY(check_shade(a));
    if (a->G == 0) return AVATAR_OK;
    size_t smem = (size_t)2 * a->NL * sizeof(float4);
    int grid = shade_grid(ctx, a->G);
    const ShadeBatch sb{B, V, view_pose, view_cc, 1};
    switch (a->K) {
        case 1: return launch_shade<1>(*a, sb, grid, smem, st);
        case 2: return launch_shade<2>(*a, sb, grid, smem, st);
        case 3: return launch_shade<3>(*a, sb, grid, smem, st);
        case 4: return launch_shade<4>(*a, sb, grid, smem, st);
        case 5: return launch_shade<5>(*a, sb, grid, smem, st);
        case 6: return launch_shade<6>(*a, sb, grid, smem, st);
        case 7: return launch_shade<7>(*a, sb, grid, smem, st);
        default: return launch_shade<8>(*a, sb, grid, smem, st);
    }
}

int av_shade_batch_backward(avatar_ctx *ctx, const avatar_shade_args *a, const avatar_shade_grads *g, int B, int V,
                            const int32_t *view_pose, const float *view_cc, cudaStream_t st)
{
    if (!ctx || !g || B < 1 || V < 1 || V > 65535 || !view_pose || !view_cc) return AVATAR_ERR_INVALID_ARG;
    AV_TRY(check_shade(a));
    if (!a->radiance || !g->d_color || !g->d_xd || !g->d_nd || !g->d_ag || !g->d_rg || !g->d_pg || !g->d_ubar ||
        !g->d_light_L)
        return AVATAR_ERR_INVALID_ARG;
    if (cudaMemsetAsync(g->d_light_L, 0, (size_t)B * a->NL * 3 * sizeof(float), st) != cudaSuccess)
        return AVATAR_ERR_CUDA;
    if (a->G == 0) return AVATAR_OK;
    const int copies = bwd_copies(ctx, a->NL);
    size_t smem = (size_t)(2 + copies) * a->NL * sizeof(float4) + SHADE_Q_BYTES;
    int grid = shade_grid(ctx, a->G);
    const ShadeBatch sb{B, V, view_pose, view_cc, copies};
    switch (a->K) {
        case 1: return launch_shade_bwd<1>(*a, *g, sb, grid, smem, ctx->sm_count, st);
        case 2: return launch_shade_bwd<2>(*a, *g, sb, grid, smem, ctx->sm_count, st);
        case 3: return launch_shade_bwd<3>(*a, *g, sb, grid, smem, ctx->sm_count, st);
        case 4: return launch_shade_bwd<4>(*a, *g, sb, grid, smem, ctx->sm_count, st);
        case 5: return launch_shade_bwd<5>(*a, *g, sb, grid, smem, ctx->sm_count, st);
        case 6: return launch_shade_bwd<6>(*a, *g, sb, grid, smem, ctx->sm_count, st);
        case 7: return launch_shade_bwd<7>(*a, *g, sb, grid, smem, ctx->sm_count, st);
        default: return launch_shade_bwd<8>(*a, *g, sb, grid, smem, ctx->sm_count, st);
    }
}
