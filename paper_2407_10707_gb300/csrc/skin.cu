// (a) Skinning of the canonical avatar into posed space - Sec. 3.1, Eq. 1.
//
// Two launches per frame:
//   skin_vertices  : forward kinematics (recomputed per block into shared
//                    memory), per-vertex blended transform A_v, posed vertex
//                    xp_v, and a packed 112-byte record per vertex
//                    {A_v rows, x+roughness, albedo+tint, normal+dx} that the
//                    Gaussian kernel gathers with seven 16-byte loads.
//   skin_gaussians : Eq. 1 weights over the K nearest vertices, interpolated
//                    attributes, A_g = sum_j ubar_j A_j (equal to
//                    sum_k w_gk bone_k by linearity), posed mean, covariance
//                    and normal.
// Backward: per-Gaussian adjoint with atomic scatter into per-vertex
// accumulators, then a per-vertex pass turning dA_v into dw_v.
#include "batch_internal.h"
#include "common.cuh"

namespace {

constexpr int SKIN_THREADS = 256;
// The vertex kernel recomputes forward kinematics in every block, then each
// thread blends one vertex's transform; small blocks spread the 50k
// vertices of the paper-scale mesh over every SM (196 blocks of 256 would
// leave most SMs with one).
constexpr int SKIN_VTX_THREADS = 64;
constexpr int MAX_J = 64;

struct VertexRec {  // 7 x float4 = 112 bytes
    float4 a0, a1, a2;  // rows of A_v = [M | t]
    float4 xr;          // canonical position, roughness
    float4 ap;          // albedo, specular tint
    float4 nd0;         // normal, dx.x
    float4 d12;         // dx.y, dx.z, 0, 0
};

__device__ void rodrigues(float rx, float ry, float rz, float *R)
{
    float th2 = rx * rx + ry * ry + rz * rz;
    float th = sqrtf(th2);
    float a, b;
    if (th < 1e-4f) {
        a = 1.0f - th2 / 6.0f;
        b = 0.5f - th2 / 24.0f;
    } else {
        a = sinf(th) / th;
        b = (1.0f - cosf(th)) / th2;
    }
    // R = I + a K + b K^2, K = [r]x
    float K[9] = {0.f, -rz, ry, rz, 0.f, -rx, -ry, rx, 0.f};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float k2 = K[3 * i] * K[j] + K[3 * i + 1] * K[3 + j] + K[3 * i + 2] * K[6 + j];
            R[3 * i + j] = (i == j ? 1.f : 0.f) + a * K[3 * i + j] + b * k2;
        }
}

// Forward kinematics into shared memory: lane j walks its ancestor chain,
// left-multiplying the local transforms, then removes the rest position.
__device__ void fk_shared(int J, const int32_t *parents, const float *joints, const float *pose,
                          float *bone_s, int32_t *status)
{
    __shared__ float loc_s[MAX_J][12];
    __shared__ int par_s[MAX_J];
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        int p = parents[j];
        if (p >= j || p < -1) {
            av_report(status, AVATAR_ERR_INDEX);
            p = -1;
        }
        par_s[j] = p;
        float R[9];
        rodrigues(pose[3 * j], pose[3 * j + 1], pose[3 * j + 2], R);
        float ox = joints[3 * j], oy = joints[3 * j + 1], oz = joints[3 * j + 2];
        if (p >= 0) {
            ox -= joints[3 * p];
            oy -= joints[3 * p + 1];
            oz -= joints[3 * p + 2];
        }
        for (int i = 0; i < 3; ++i) {
            loc_s[j][4 * i + 0] = R[3 * i + 0];
            loc_s[j][4 * i + 1] = R[3 * i + 1];
            loc_s[j][4 * i + 2] = R[3 * i + 2];
        }
        loc_s[j][3] = ox;
        loc_s[j][7] = oy;
        loc_s[j][11] = oz;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        float T[12];
        for (int i = 0; i < 12; ++i) T[i] = loc_s[j][i];
        int p = par_s[j];
        int guard = 0;
        while (p >= 0 && guard++ < MAX_J) {
            const float *L = loc_s[p];
            float N[12];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    N[4 * i + k] = L[4 * i] * T[k] + L[4 * i + 1] * T[4 + k] + L[4 * i + 2] * T[8 + k];
                N[4 * i + 3] = L[4 * i] * T[3] + L[4 * i + 1] * T[7] + L[4 * i + 2] * T[11] + L[4 * i + 3];
            }
#pragma unroll
            for (int i = 0; i < 12; ++i) T[i] = N[i];
            p = par_s[p];
        }
        float jx = joints[3 * j], jy = joints[3 * j + 1], jz = joints[3 * j + 2];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            bone_s[12 * j + 4 * i + 0] = T[4 * i + 0];
            bone_s[12 * j + 4 * i + 1] = T[4 * i + 1];
            bone_s[12 * j + 4 * i + 2] = T[4 * i + 2];
            bone_s[12 * j + 4 * i + 3] =
                T[4 * i + 3] - (T[4 * i] * jx + T[4 * i + 1] * jy + T[4 * i + 2] * jz);
        }
    }
    __syncthreads();
}

// blockIdx.y = pose of a batch of gridDim.y poses (pose [B][J][3], bone
// [B][J][12], xp [3][B Nv], records [B Nv]).
__global__ void __launch_bounds__(SKIN_VTX_THREADS)
skin_vertices_kernel(avatar_skin_args a, VertexRec *__restrict__ rec)
{
    __shared__ float bone_s[MAX_J * 12];
    const int pb = blockIdx.y;
    const size_t SN = (size_t)gridDim.y * a.Nv;  // channel stride of xp
    a.pose += (size_t)pb * 3 * a.J;
    a.bone += (size_t)pb * 12 * a.J;
    a.xp += (size_t)pb * a.Nv;
    rec += (size_t)pb * a.Nv;
    fk_shared(a.J, a.parents, a.joints, a.pose, bone_s, a.status);
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < 12 * a.J; i += blockDim.x) a.bone[i] = bone_s[i];
    const int Nv = a.Nv, J = a.J;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < Nv; v += gridDim.x * blockDim.x) {
        float A[12];
#pragma unroll
        for (int i = 0; i < 12; ++i) A[i] = 0.f;
        const float *w = a.wv + (size_t)v * J;
        if ((J & 3) == 0) {
            for (int k = 0; k < J; k += 4) {
                float4 w4 = __ldg(reinterpret_cast<const float4 *>(w + k));
                float ws[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                for (int m = 0; m < 4; ++m)
#pragma unroll
                    for (int i = 0; i < 12; ++i) A[i] = fmaf(ws[m], bone_s[12 * (k + m) + i], A[i]);
            }
        } else {
            for (int k = 0; k < J; ++k) {
                float wk = __ldg(w + k);
#pragma unroll
                for (int i = 0; i < 12; ++i) A[i] = fmaf(wk, bone_s[12 * k + i], A[i]);
            }
        }
        float x = a.xv[v], y = a.xv[Nv + v], z = a.xv[2 * Nv + v];
        float dx = 0.f, dy = 0.f, dz = 0.f;
        if (a.dxv) {
            dx = a.dxv[v];
            dy = a.dxv[Nv + v];
            dz = a.dxv[2 * Nv + v];
        }
        float px = x + dx, py = y + dy, pz = z + dz;
#pragma unroll
        for (int i = 0; i < 3; ++i)
            a.xp[i * SN + v] = fmaf(A[4 * i], px, fmaf(A[4 * i + 1], py, fmaf(A[4 * i + 2], pz, A[4 * i + 3])));
        VertexRec r;
        r.a0 = make_float4(A[0], A[1], A[2], A[3]);
        r.a1 = make_float4(A[4], A[5], A[6], A[7]);
        r.a2 = make_float4(A[8], A[9], A[10], A[11]);
        r.xr = make_float4(x, y, z, ld_attr(a.rv, v, a.attr_dtype));
        r.ap = make_float4(ld_attr(a.av, v, a.attr_dtype), ld_attr(a.av, (size_t)Nv + v, a.attr_dtype),
                           ld_attr(a.av, (size_t)2 * Nv + v, a.attr_dtype), ld_attr(a.pv, v, a.attr_dtype));
        r.nd0 = make_float4(a.nv[v], a.nv[Nv + v], a.nv[2 * Nv + v], dx);
        r.d12 = make_float4(dy, dz, 0.f, 0.f);
        rec[v] = r;
    }
}

__device__ __forceinline__ void quat_to_rot(float qw, float qx, float qy, float qz, float *R)
{
    R[0] = 1.f - 2.f * (qy * qy + qz * qz);
    R[1] = 2.f * (qx * qy - qw * qz);
    R[2] = 2.f * (qx * qz + qw * qy);
    R[3] = 2.f * (qx * qy + qw * qz);
    R[4] = 1.f - 2.f * (qx * qx + qz * qz);
    R[5] = 2.f * (qy * qz - qw * qx);
    R[6] = 2.f * (qx * qz - qw * qy);
    R[7] = 2.f * (qy * qz + qw * qx);
    R[8] = 1.f - 2.f * (qx * qx + qy * qy);
}

// Per-Gaussian state shared by the forward and backward kernels.
template <int K>
struct GaussState {
    float x[3];
    int idx[K];
    float dist[K];
    float ub[K];
    float usum;
    float A[12];
    float a[3], r, p, n[3], dx[3];
};

template <int K>
__device__ __forceinline__ bool gauss_gather(const avatar_skin_args &a, const VertexRec *__restrict__ rec,
                                             int g, GaussState<K> &s)
{
    const int G = a.G;
    s.x[0] = a.xg[g];
    s.x[1] = a.xg[G + g];
    s.x[2] = a.xg[2 * G + g];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        int v = a.knn[j * G + g];
        if (v < 0 || v >= a.Nv) {
            ok = false;
            v = 0;
        }
        s.idx[j] = v;
    }
    // one pass: each neighbour's record is read once, the sums taken with the
    // unnormalised weights 1/d_j and scaled by 1/sum_j(1/d_j) at the end, so
    // no neighbour's loads wait for another's distance
    s.usum = 0.f;
#pragma unroll
    for (int i = 0; i < 12; ++i) s.A[i] = 0.f;
    s.a[0] = s.a[1] = s.a[2] = s.r = s.p = 0.f;
    s.n[0] = s.n[1] = s.n[2] = s.dx[0] = s.dx[1] = s.dx[2] = 0.f;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const VertexRec *vr = rec + s.idx[j];
        float4 a0 = __ldg(&vr->a0), a1 = __ldg(&vr->a1), a2 = __ldg(&vr->a2);
        float4 xr = __ldg(&vr->xr), ap = __ldg(&vr->ap), n0 = __ldg(&vr->nd0), d12 = __ldg(&vr->d12);
        float ex = s.x[0] - xr.x, ey = s.x[1] - xr.y, ez = s.x[2] - xr.z;
        float d = sqrtf(ex * ex + ey * ey + ez * ez);
        s.dist[j] = d;
        float u = 1.0f / fmaxf(d, 1e-8f);
        s.ub[j] = u;
        s.usum += u;
        s.A[0] = fmaf(u, a0.x, s.A[0]);
        s.A[1] = fmaf(u, a0.y, s.A[1]);
        s.A[2] = fmaf(u, a0.z, s.A[2]);
        s.A[3] = fmaf(u, a0.w, s.A[3]);
        s.A[4] = fmaf(u, a1.x, s.A[4]);
        s.A[5] = fmaf(u, a1.y, s.A[5]);
        s.A[6] = fmaf(u, a1.z, s.A[6]);
        s.A[7] = fmaf(u, a1.w, s.A[7]);
        s.A[8] = fmaf(u, a2.x, s.A[8]);
        s.A[9] = fmaf(u, a2.y, s.A[9]);
        s.A[10] = fmaf(u, a2.z, s.A[10]);
        s.A[11] = fmaf(u, a2.w, s.A[11]);
        s.r = fmaf(u, xr.w, s.r);
        s.a[0] = fmaf(u, ap.x, s.a[0]);
        s.a[1] = fmaf(u, ap.y, s.a[1]);
        s.a[2] = fmaf(u, ap.z, s.a[2]);
        s.p = fmaf(u, ap.w, s.p);
        s.n[0] = fmaf(u, n0.x, s.n[0]);
        s.n[1] = fmaf(u, n0.y, s.n[1]);
        s.n[2] = fmaf(u, n0.z, s.n[2]);
        s.dx[0] = fmaf(u, n0.w, s.dx[0]);
        s.dx[1] = fmaf(u, d12.x, s.dx[1]);
        s.dx[2] = fmaf(u, d12.y, s.dx[2]);
    }
    const float inv = 1.0f / s.usum;
#pragma unroll
    for (int j = 0; j < K; ++j) s.ub[j] *= inv;
#pragma unroll
    for (int i = 0; i < 12; ++i) s.A[i] *= inv;
    s.a[0] *= inv;
    s.a[1] *= inv;
    s.a[2] *= inv;
    s.r *= inv;
    s.p *= inv;
    s.n[0] *= inv;
    s.n[1] *= inv;
    s.n[2] *= inv;
    s.dx[0] *= inv;
    s.dx[1] *= inv;
    s.dx[2] *= inv;
    return ok;
}

// Three blocks per SM (80 registers): the one-pass gather keeps the four
// neighbours' 28 record loads in flight; unbounded it takes 87 registers and
// two blocks.
template <int K>
__global__ void __launch_bounds__(SKIN_THREADS, 3)
skin_gaussians_kernel(avatar_skin_args a, const VertexRec *__restrict__ rec)
{
    // blockIdx.y = pose of a batch: xd, nd [3][B G], cov [6][B G], records
    // [B Nv]; the pose-independent ag, rg, pg, ubar are written by pose 0.
    const int G = a.G;
    const int pb = blockIdx.y;
    const size_t SG = (size_t)gridDim.y * G;
    a.xd += (size_t)pb * G;
    a.cov += (size_t)pb * G;
    a.nd += (size_t)pb * G;
    rec += (size_t)pb * a.Nv;
    const bool shared_out = pb == 0;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        GaussState<K> s;
        if (!gauss_gather<K>(a, rec, g, s)) av_report(a.status, AVATAR_ERR_INDEX);
        const float *A = s.A;
        float xb0 = s.x[0] + s.dx[0], xb1 = s.x[1] + s.dx[1], xb2 = s.x[2] + s.dx[2];
#pragma unroll
        for (int i = 0; i < 3; ++i)
            a.xd[i * SG + g] = fmaf(A[4 * i], xb0, fmaf(A[4 * i + 1], xb1, fmaf(A[4 * i + 2], xb2, A[4 * i + 3])));
        // covariance
        const int dt = a.attr_dtype;
        float qw = ld_attr(a.quat, g, dt), qx = ld_attr(a.quat, (size_t)G + g, dt),
              qy = ld_attr(a.quat, (size_t)2 * G + g, dt), qz = ld_attr(a.quat, (size_t)3 * G + g, dt);
        float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        float R[9];
        quat_to_rot(qw * qn, qx * qn, qy * qn, qz * qn, R);
        float s2[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) s2[i] = expf(2.f * ld_attr(a.logscale, (size_t)i * G + g, dt));
        // MR = M * R * diag(s):  cov = (MR)(MR)^T
        float MR[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                MR[3 * i + k] = A[4 * i] * R[k] + A[4 * i + 1] * R[3 + k] + A[4 * i + 2] * R[6 + k];
        float c[6];
        const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
        for (int e = 0; e < 6; ++e) {
            int i = ii[e], j = jj[e];
            c[e] = MR[3 * i] * MR[3 * j] * s2[0] + MR[3 * i + 1] * MR[3 * j + 1] * s2[1] +
                   MR[3 * i + 2] * MR[3 * j + 2] * s2[2];
        }
#pragma unroll
        for (int e = 0; e < 6; ++e) a.cov[e * SG + g] = c[e];
        // normal
        float nl = rsqrtf(s.n[0] * s.n[0] + s.n[1] * s.n[1] + s.n[2] * s.n[2]);
        float n0 = s.n[0] * nl, n1 = s.n[1] * nl, n2 = s.n[2] * nl;
        float m0 = A[0] * n0 + A[1] * n1 + A[2] * n2;
        float m1 = A[4] * n0 + A[5] * n1 + A[6] * n2;
        float m2 = A[8] * n0 + A[9] * n1 + A[10] * n2;
        float ml = rsqrtf(m0 * m0 + m1 * m1 + m2 * m2);
        a.nd[g] = m0 * ml;
        a.nd[SG + g] = m1 * ml;
        a.nd[2 * SG + g] = m2 * ml;
        if (!shared_out) continue;
        a.ag[g] = s.a[0];
        a.ag[G + g] = s.a[1];
        a.ag[2 * G + g] = s.a[2];
        a.rg[g] = s.r;
        a.pg[g] = s.p;
#pragma unroll
        for (int j = 0; j < K; ++j) a.ubar[j * G + g] = s.ub[j];
    }
}

// ---------------------------------------------------------------- backward
struct SkinBwdWs {
    float *dA;  // [Nv][12] accumulated dL/dA_v
};

__device__ __forceinline__ float ld_or0(const float *p, size_t i) { return p ? __ldg(p + i) : 0.f; }

// Two blocks per SM: unbounded the adjoint takes 180 registers and one
// block; at 128 (8 bytes spilled) twice the warps hide its gathers and atomics.
template <int K>
__global__ void __launch_bounds__(SKIN_THREADS, 2)
skin_gaussians_backward_kernel(avatar_skin_args a, avatar_skin_grads gr, const VertexRec *__restrict__ rec,
                               float *__restrict__ dAv, int B)
{
    // B poses: upstream d_xd, d_xd2, d_nd [3][B G] and d_cov [6][B G] per pose,
    // d_ag, d_rg, d_pg, d_ubar once; records and dA_v accumulators per pose
    // ([B Nv]); the canonical gradients are summed over the poses here.
    const int G = a.G, Nv = a.Nv;
    const size_t SG = (size_t)B * G;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        float dxg_s[3] = {0.f, 0.f, 0.f}, dls_s[3] = {0.f, 0.f, 0.f}, dq_s[4] = {0.f, 0.f, 0.f, 0.f};
        for (int pb = 0; pb < B; ++pb) {
        const VertexRec *recp = rec + (size_t)pb * Nv;
        float *dAvp = dAv + (size_t)pb * Nv * 12;
        const size_t gi = (size_t)pb * G + g;  // element of the per-pose arrays (stride SG)
        const bool shared_in = pb == 0;        // pose-independent upstream enters once
        GaussState<K> s;
        gauss_gather<K>(a, recp, g, s);
        const float *A = s.A;
        float dM[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        float dt[3];
        float xb[3] = {s.x[0] + s.dx[0], s.x[1] + s.dx[1], s.x[2] + s.dx[2]};
        // ---- position: xd = M xb + t
        float dxd[3] = {ld_or0(gr.d_xd, gi) + ld_or0(gr.d_xd2, gi), ld_or0(gr.d_xd, SG + gi) + ld_or0(gr.d_xd2, SG + gi),
                        ld_or0(gr.d_xd, 2 * SG + gi) + ld_or0(gr.d_xd2, 2 * SG + gi)};
        float dxb[3] = {0, 0, 0};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            dt[i] = dxd[i];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                dM[3 * i + k] += dxd[i] * xb[k];
                dxb[k] += A[4 * i + k] * dxd[i];
            }
        }
        // ---- covariance: cov = M Sigma M^T, Sigma = R diag(s2) R^T
        const int adt = a.attr_dtype;
        float qw0 = ld_attr(a.quat, g, adt), qx0 = ld_attr(a.quat, (size_t)G + g, adt),
              qy0 = ld_attr(a.quat, (size_t)2 * G + g, adt), qz0 = ld_attr(a.quat, (size_t)3 * G + g, adt);
        float qinv = rsqrtf(qw0 * qw0 + qx0 * qx0 + qy0 * qy0 + qz0 * qz0);
        float qw = qw0 * qinv, qx = qx0 * qinv, qy = qy0 * qinv, qz = qz0 * qinv;
        float R[9];
        quat_to_rot(qw, qx, qy, qz, R);
        float s2[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) s2[i] = expf(2.f * ld_attr(a.logscale, (size_t)i * G + g, adt));
        float dls[3] = {0, 0, 0}, dq[4] = {0, 0, 0, 0};
        if (gr.d_cov) {
            float dc[6];
#pragma unroll
            for (int e = 0; e < 6; ++e) dc[e] = __ldg(gr.d_cov + (size_t)e * SG + gi);
            float Gc[9] = {dc[0], 0.5f * dc[1], 0.5f * dc[2], 0.5f * dc[1], dc[3], 0.5f * dc[4],
                           0.5f * dc[2], 0.5f * dc[4], dc[5]};
            float Sg[9];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    Sg[3 * i + j] = R[3 * i] * R[3 * j] * s2[0] + R[3 * i + 1] * R[3 * j + 1] * s2[1] +
                                    R[3 * i + 2] * R[3 * j + 2] * s2[2];
            float M[9] = {A[0], A[1], A[2], A[4], A[5], A[6], A[8], A[9], A[10]};
            // dM += 2 Gc M Sigma
            float GM[9], MS[9];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    GM[3 * i + j] = Gc[3 * i] * M[j] + Gc[3 * i + 1] * M[3 + j] + Gc[3 * i + 2] * M[6 + j];
                    MS[3 * i + j] = M[3 * i] * Sg[j] + M[3 * i + 1] * Sg[3 + j] + M[3 * i + 2] * Sg[6 + j];
                }
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    dM[3 * i + j] += 2.f * (Gc[3 * i] * MS[j] + Gc[3 * i + 1] * MS[3 + j] + Gc[3 * i + 2] * MS[6 + j]);
            // dSigma = M^T Gc M
            float dS[9];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    dS[3 * i + j] = M[i] * GM[j] + M[3 + i] * GM[3 + j] + M[6 + i] * GM[6 + j];
            // dR = 2 dS R diag(s2); ds2_i = (R^T dS R)_ii
            float dR[9];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    dR[3 * i + k] = 2.f * s2[k] * (dS[3 * i] * R[k] + dS[3 * i + 1] * R[3 + k] + dS[3 * i + 2] * R[6 + k]);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float acc = 0.f;
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) acc += R[3 * i + k] * dS[3 * i + j] * R[3 * j + k];
                dls[k] = acc * 2.f * s2[k];
            }
            float gw = 2.f * (-qz * dR[1] + qy * dR[2] + qz * dR[3] - qx * dR[5] - qy * dR[6] + qx * dR[7]);
            float gx = 2.f * (qy * dR[1] + qz * dR[2] + qy * dR[3] - 2.f * qx * dR[4] - qw * dR[5] + qz * dR[6] +
                              qw * dR[7] - 2.f * qx * dR[8]);
            float gy = 2.f * (-2.f * qy * dR[0] + qx * dR[1] + qw * dR[2] + qx * dR[3] + qz * dR[5] - qw * dR[6] +
                              qz * dR[7] - 2.f * qy * dR[8]);
            float gz = 2.f * (-2.f * qz * dR[0] - qw * dR[1] + qx * dR[2] + qw * dR[3] - 2.f * qz * dR[4] +
                              qy * dR[5] + qx * dR[6] + qy * dR[7]);
            float dot = gw * qw + gx * qx + gy * qy + gz * qz;
            dq[0] = (gw - dot * qw) * qinv;
            dq[1] = (gx - dot * qx) * qinv;
            dq[2] = (gy - dot * qy) * qinv;
            dq[3] = (gz - dot * qz) * qinv;
        }
        // ---- normal: nd = normalize(M nhat), nhat = normalize(n_g)
        float dn_g[3] = {0, 0, 0};
        if (gr.d_nd) {
            float dnd[3] = {__ldg(gr.d_nd + gi), __ldg(gr.d_nd + SG + gi), __ldg(gr.d_nd + 2 * SG + gi)};
            // one reciprocal per length, then products (the divisions were IEEE)
            float inl = 1.f / sqrtf(s.n[0] * s.n[0] + s.n[1] * s.n[1] + s.n[2] * s.n[2]);
            float nh[3] = {s.n[0] * inl, s.n[1] * inl, s.n[2] * inl};
            float m[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) m[i] = A[4 * i] * nh[0] + A[4 * i + 1] * nh[1] + A[4 * i + 2] * nh[2];
            float iml = 1.f / sqrtf(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
            float nd[3] = {m[0] * iml, m[1] * iml, m[2] * iml};
            float dd = dnd[0] * nd[0] + dnd[1] * nd[1] + dnd[2] * nd[2];
            float dm[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) dm[i] = (dnd[i] - dd * nd[i]) * iml;
            float dnh[3] = {0, 0, 0};
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    dM[3 * i + k] += dm[i] * nh[k];
                    dnh[k] += A[4 * i + k] * dm[i];
                }
            float d2 = dnh[0] * nh[0] + dnh[1] * nh[1] + dnh[2] * nh[2];
#pragma unroll
            for (int i = 0; i < 3; ++i) dn_g[i] = (dnh[i] - d2 * nh[i]) * inl;
        }
        float dag[3] = {0.f, 0.f, 0.f}, drg = 0.f, dpg = 0.f;
        if (shared_in) {
            dag[0] = ld_or0(gr.d_ag, g);
            dag[1] = ld_or0(gr.d_ag, G + g);
            dag[2] = ld_or0(gr.d_ag, 2 * G + g);
            drg = ld_or0(gr.d_rg, g);
            dpg = ld_or0(gr.d_pg, g);
        }
        // ---- scatter through Eq. 1 and accumulate dubar
        float dA[12] = {dM[0], dM[1], dM[2], dt[0], dM[3], dM[4], dM[5], dt[1], dM[6], dM[7], dM[8], dt[2]};
        float dub[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const VertexRec *vr = recp + s.idx[j];
            const int v = s.idx[j];
            const float u = s.ub[j];
            float4 a0 = __ldg(&vr->a0), a1 = __ldg(&vr->a1), a2 = __ldg(&vr->a2);
            float4 xr = __ldg(&vr->xr), ap = __ldg(&vr->ap), n0 = __ldg(&vr->nd0), d12 = __ldg(&vr->d12);
            float acc = shared_in ? ld_or0(gr.d_ubar, (size_t)j * G + g) : 0.f;
            acc += dA[0] * a0.x + dA[1] * a0.y + dA[2] * a0.z + dA[3] * a0.w;
            acc += dA[4] * a1.x + dA[5] * a1.y + dA[6] * a1.z + dA[7] * a1.w;
            acc += dA[8] * a2.x + dA[9] * a2.y + dA[10] * a2.z + dA[11] * a2.w;
            acc += dag[0] * ap.x + dag[1] * ap.y + dag[2] * ap.z + dpg * ap.w + drg * xr.w;
            acc += dn_g[0] * n0.x + dn_g[1] * n0.y + dn_g[2] * n0.z;
            acc += dxb[0] * n0.w + dxb[1] * d12.x + dxb[2] * d12.y;
            dub[j] = acc;
            float *dst = dAvp + (size_t)v * 12;
#pragma unroll
            for (int i = 0; i < 12; ++i)
                if (dA[i] != 0.f) atomicAdd(dst + i, u * dA[i]);
            if (gr.d_av && shared_in) {
                atomicAdd(gr.d_av + v, u * dag[0]);
                atomicAdd(gr.d_av + Nv + v, u * dag[1]);
                atomicAdd(gr.d_av + 2 * Nv + v, u * dag[2]);
            }
            if (gr.d_rv && shared_in) atomicAdd(gr.d_rv + v, u * drg);
            if (gr.d_pv && shared_in) atomicAdd(gr.d_pv + v, u * dpg);
            if (gr.d_dxv) {
                atomicAdd(gr.d_dxv + v, u * dxb[0]);
                atomicAdd(gr.d_dxv + Nv + v, u * dxb[1]);
                atomicAdd(gr.d_dxv + 2 * Nv + v, u * dxb[2]);
            }
        }
        // ---- ubar = u / sum u, u = 1/max(d, eps)
        float sdot = 0.f;
#pragma unroll
        for (int j = 0; j < K; ++j) sdot += dub[j] * s.ub[j];
        float dxg[3] = {dxb[0], dxb[1], dxb[2]};
        const float ius = 1.f / s.usum;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            float du = (dub[j] - sdot) * ius;
            float d = s.dist[j];
            if (d > 1e-8f) {
                float4 xr = __ldg(&recp[s.idx[j]].xr);
                const float id = 1.f / d;
                float f = -du * id * id * id;  // d(1/d)/dd = -1/d^2, and d|x - y| / dx = (x - y) / d
                dxg[0] += f * (s.x[0] - xr.x);
                dxg[1] += f * (s.x[1] - xr.y);
                dxg[2] += f * (s.x[2] - xr.z);
            }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            dxg_s[i] += dxg[i];
            dls_s[i] += dls[i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) dq_s[i] += dq[i];
        }  // poses
        if (gr.d_xg) {
            gr.d_xg[g] = dxg_s[0];
            gr.d_xg[G + g] = dxg_s[1];
            gr.d_xg[2 * G + g] = dxg_s[2];
        }
        if (gr.d_logscale)
#pragma unroll
            for (int i = 0; i < 3; ++i) gr.d_logscale[i * G + g] = dls_s[i];
        if (gr.d_quat)
#pragma unroll
            for (int i = 0; i < 4; ++i) gr.d_quat[i * G + g] = dq_s[i];
    }
}

__global__ void __launch_bounds__(SKIN_THREADS)
skin_vertices_backward_kernel(avatar_skin_args a, avatar_skin_grads gr, const float *__restrict__ dAv, int B)
{
    // dw_vk = sum over poses of dA_v . bone_k (bones [B][J][12], dA_v [B Nv][12])
    __shared__ float bone_s[MAX_J * 12];
    const int Nv = a.Nv, J = a.J;
    for (int pb = 0; pb < B; ++pb) {
        __syncthreads();
        for (int i = threadIdx.x; i < 12 * J; i += blockDim.x) bone_s[i] = a.bone[(size_t)pb * 12 * J + i];
        __syncthreads();
        const float *dAvp = dAv + (size_t)pb * Nv * 12;
        for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < Nv; v += gridDim.x * blockDim.x) {
            float d[12];
#pragma unroll
            for (int i = 0; i < 12; ++i) d[i] = dAvp[(size_t)v * 12 + i];
            float *out = gr.d_wv + (size_t)v * J;
            for (int k = 0; k < J; ++k) {
                float acc = pb == 0 ? 0.f : out[k];
#pragma unroll
                for (int i = 0; i < 12; ++i) acc = fmaf(d[i], bone_s[12 * k + i], acc);
                out[k] = acc;
            }
        }
    }
}

template <int K>
void launch_gauss_fwd(const avatar_skin_args &a, const VertexRec *rec, int B, int grid, cudaStream_t st)
{
    skin_gaussians_kernel<K><<<dim3(grid, B), SKIN_THREADS, 0, st>>>(a, rec);
}

template <int K>
void launch_gauss_bwd(const avatar_skin_args &a, const avatar_skin_grads &g, const VertexRec *rec,
                      float *dAv, int B, int grid, cudaStream_t st)
{
    skin_gaussians_backward_kernel<K><<<grid, SKIN_THREADS, 0, st>>>(a, g, rec, dAv, B);
}

int check_skin_args(const avatar_skin_args *a)
{
    if (!a) return AVATAR_ERR_INVALID_ARG;
    if (a->G < 0 || a->Nv < 1 || a->K < 1 || a->K > 8 || a->J < 1 || a->J > MAX_J)
        return AVATAR_ERR_INVALID_ARG;
    if (!a->xv || !a->wv || !a->av || !a->rv || !a->pv || !a->nv || !a->parents || !a->joints ||
        !a->pose || !a->bone || !a->xp)
        return AVATAR_ERR_INVALID_ARG;
    if (a->G > 0 && (!a->xg || !a->logscale || !a->quat || !a->knn || !a->xd || !a->cov || !a->nd ||
                     !a->ag || !a->rg || !a->pg || !a->ubar))
        return AVATAR_ERR_INVALID_ARG;
    if ((a->J & 3) == 0 && (((uintptr_t)a->wv) & 15)) return AVATAR_ERR_INVALID_ARG;
    if (a->attr_dtype != AVATAR_DTYPE_F32 && a->attr_dtype != AVATAR_DTYPE_BF16) return AVATAR_ERR_INVALID_ARG;
    return AVATAR_OK;
}

int grid_for(const avatar_ctx *ctx, long n, int threads)
{
    long blocks = (n + threads - 1) / threads;
    long cap = (long)ctx->sm_count * 8;
    if (blocks > cap) blocks = cap;
    return blocks < 1 ? 1 : (int)blocks;
}

}  // namespace

namespace {

// Forward of B poses (see the batched launcher's declaration for layouts).
int skin_run(avatar_ctx *ctx, const avatar_skin_args *a, int B, void *ws, size_t ws_bytes, cudaStream_t st)
{
    if (!ctx || B < 1 || B > 65535) return AVATAR_ERR_INVALID_ARG;
    AV_TRY(check_skin_args(a));
    if (!ws || (((uintptr_t)ws) & 255) || ws_bytes < av_align256((size_t)B * a->Nv * sizeof(VertexRec)))
        return AVATAR_ERR_WORKSPACE;
    VertexRec *rec = (VertexRec *)ws;
    skin_vertices_kernel<<<dim3(grid_for(ctx, a->Nv, SKIN_VTX_THREADS), B), SKIN_VTX_THREADS, 0, st>>>(*a, rec);
    AV_CHECK_LAUNCH();
    if (a->G > 0) {
        int grid = grid_for(ctx, a->G, SKIN_THREADS);
        switch (a->K) {
            case 1: launch_gauss_fwd<1>(*a, rec, B, grid, st); break;
            case 2: launch_gauss_fwd<2>(*a, rec, B, grid, st); break;
            case 3: launch_gauss_fwd<3>(*a, rec, B, grid, st); break;
            case 4: launch_gauss_fwd<4>(*a, rec, B, grid, st); break;
            case 5: launch_gauss_fwd<5>(*a, rec, B, grid, st); break;
            case 6: launch_gauss_fwd<6>(*a, rec, B, grid, st); break;
            case 7: launch_gauss_fwd<7>(*a, rec, B, grid, st); break;
            default: launch_gauss_fwd<8>(*a, rec, B, grid, st); break;
        }
        AV_CHECK_LAUNCH();
    }
    return AVATAR_OK;
}

int skin_bwd_run(avatar_ctx *ctx, const avatar_skin_args *a, const avatar_skin_grads *g, int B, const void *fwd_ws,
                 void *ws, size_t ws_bytes, cudaStream_t st)
{
    if (!ctx || !g || B < 1) return AVATAR_ERR_INVALID_ARG;
    AV_TRY(check_skin_args(a));
    if (B > 1 && g->d_xd2) return AVATAR_ERR_INVALID_ARG;
    if (!fwd_ws || (((uintptr_t)fwd_ws) & 255)) return AVATAR_ERR_WORKSPACE;
    const int Nv = a->Nv, G = a->G;
    if (!ws || (((uintptr_t)ws) & 255) || ws_bytes < av_align256((size_t)B * Nv * 12 * sizeof(float)))
        return AVATAR_ERR_WORKSPACE;
    float *dAv = (float *)ws;
    if (cudaMemsetAsync(dAv, 0, (size_t)B * Nv * 12 * sizeof(float), st) != cudaSuccess) return AVATAR_ERR_CUDA;
    if (g->d_av && cudaMemsetAsync(g->d_av, 0, (size_t)3 * Nv * sizeof(float), st) != cudaSuccess)
        return AVATAR_ERR_CUDA;
    if (g->d_rv && cudaMemsetAsync(g->d_rv, 0, (size_t)Nv * sizeof(float), st) != cudaSuccess)
        return AVATAR_ERR_CUDA;
    if (g->d_pv && cudaMemsetAsync(g->d_pv, 0, (size_t)Nv * sizeof(float), st) != cudaSuccess)
        return AVATAR_ERR_CUDA;
    if (g->d_dxv && cudaMemsetAsync(g->d_dxv, 0, (size_t)3 * Nv * sizeof(float), st) != cudaSuccess)
        return AVATAR_ERR_CUDA;
    const VertexRec *rec = (const VertexRec *)fwd_ws;
    if (G > 0) {
        int grid = grid_for(ctx, G, SKIN_THREADS);
        switch (a->K) {
            case 1: launch_gauss_bwd<1>(*a, *g, rec, dAv, B, grid, st); break;
            case 2: launch_gauss_bwd<2>(*a, *g, rec, dAv, B, grid, st); break;
            case 3: launch_gauss_bwd<3>(*a, *g, rec, dAv, B, grid, st); break;
            case 4: launch_gauss_bwd<4>(*a, *g, rec, dAv, B, grid, st); break;
            case 5: launch_gauss_bwd<5>(*a, *g, rec, dAv, B, grid, st); break;
            case 6: launch_gauss_bwd<6>(*a, *g, rec, dAv, B, grid, st); break;
            case 7: launch_gauss_bwd<7>(*a, *g, rec, dAv, B, grid, st); break;
            default: launch_gauss_bwd<8>(*a, *g, rec, dAv, B, grid, st); break;
        }
        AV_CHECK_LAUNCH();
    }
    if (g->d_wv) {
        skin_vertices_backward_kernel<<<grid_for(ctx, Nv, SKIN_THREADS), SKIN_THREADS, 0, st>>>(*a, *g, dAv, B);
        AV_CHECK_LAUNCH();
    }
    return AVATAR_OK;
}

}  // namespace

size_t av_skin_batch_workspace_size(const avatar_skin_args *a, int B)
{
    if (!a || a->Nv < 1 || B < 1) return 0;
    return av_align256((size_t)B * a->Nv * sizeof(VertexRec));
}

int av_skin_batch(avatar_ctx *ctx, const avatar_skin_args *a, int B, void *ws, size_t ws_bytes, cudaStream_t st)
{
    return skin_run(ctx, a, B, ws, ws_bytes, st);
}

size_t av_skin_batch_backward_workspace_size(const avatar_skin_args *a, int B)
{
    if (!a || a->Nv < 1 || B < 1) return 0;
    return av_align256((size_t)B * a->Nv * 12 * sizeof(float));
}

int av_skin_batch_backward(avatar_ctx *ctx, const avatar_skin_args *a, const avatar_skin_grads *g, int B,
                           const void *fwd_ws, void *ws, size_t ws_bytes, cudaStream_t st)
{
    return skin_bwd_run(ctx, a, g, B, fwd_ws, ws, ws_bytes, st);
}

extern "C" size_t avatar_skin_workspace_size(const avatar_skin_args *a)
{
    return av_skin_batch_workspace_size(a, 1);
}

extern "C" int avatar_skin(avatar_ctx *ctx, const avatar_skin_args *a, void *ws, size_t ws_bytes,
                           avatar_stream_t stream)
{
    return skin_run(ctx, a, 1, ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" size_t avatar_skin_backward_workspace_size(const avatar_skin_args *a)
{
    return av_skin_batch_backward_workspace_size(a, 1);
}

extern "C" int avatar_skin_backward(avatar_ctx *ctx, const avatar_skin_args *a, const avatar_skin_grads *g,
                                    const void *fwd_ws, void *ws, size_t ws_bytes, avatar_stream_t stream)
{
    return skin_bwd_run(ctx, a, g, 1, fwd_ws, ws, ws_bytes, (cudaStream_t)stream);
}
