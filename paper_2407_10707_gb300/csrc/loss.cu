// Image loss of Eq. 5 (Sec. 3.3), the 3DGS form:
//   L_img = (1 - lambda) mean |x - y| + lambda (1 - mean SSIM(x, y))
// with SSIM under an 11 x 11 Gaussian window (sigma 1.5, zero padding),
// C1 = 0.01^2, C2 = 0.03^2, per channel and pixel.
//
// Two fused tile kernels (32 x 32 pixels, separable blurs in shared memory;
// each thread slides an 11-tap register window along 8 outputs of a row or
// 4 of a column, so a tap costs an FMA and no shared-memory load):
//   forward   blurs x, y, x^2, y^2, x y; per pixel the SSIM, |x - y| and the
//             coefficients of dSSIM with respect to the blurred x, x^2, x y
//             (A, B, C below); per-block partial sums
//   backward  blurs A, B, C and combines them with x and y:
//             dSSIM_total / dx_p = (A * w)_p + 2 x_p (B * w)_p + y_p (C * w)_p
// A final one-block reduction in FP64 gives the loss (deterministic).
#include "common.cuh"

namespace {

constexpr int TS = 32;            // output tile edge
constexpr int R = 5;              // window radius
constexpr int WT = TS + 2 * R;    // tile with halo
constexpr int LOSS_THREADS = 256;
constexpr int RBH = 8;            // outputs per thread of a horizontal blur (register window)
constexpr int RBV = 4;            // outputs per thread of a vertical blur
constexpr float C1 = 0.01f * 0.01f;
constexpr float C2 = 0.03f * 0.03f;

// Normalised Gaussian taps, sigma 1.5: exp(-k^2 / 4.5) / sum, computed by
// the first 11 threads of a block into shared memory.
__device__ __forceinline__ void make_taps(float *w)
{
    if (threadIdx.x <= 2 * R) {
        float s = 0.f;
        for (int k = -R; k <= R; ++k) s += expf(-(float)(k * k) / 4.5f);
        const int k = (int)threadIdx.x - R;
        w[threadIdx.x] = expf(-(float)(k * k) / 4.5f) / s;
    }
}

struct LossDims {
    int C, H, W;
    int tx, ty;  // tiles per row / column
};

__device__ __forceinline__ float load_or0(const float *p, int H, int W, int y, int x)
{
    return (x >= 0 && x < W && y >= 0 && y < H) ? __ldg(p + (size_t)y * W + x) : 0.f;
}

__global__ void __launch_bounds__(LOSS_THREADS)
ssim_forward_kernel(const float *__restrict__ img, const float *__restrict__ tgt, LossDims d,
                    float *__restrict__ coefA, float *__restrict__ coefB, float *__restrict__ coefC,
                    double *__restrict__ part)
{
    __shared__ float sx[WT][WT], sy[WT][WT];
    __shared__ float h[5][WT][TS];
    __shared__ double red[2][LOSS_THREADS / 32];
    __shared__ float c_w[2 * R + 1];
    make_taps(c_w);
    const int c = blockIdx.z, x0 = blockIdx.x * TS, y0 = blockIdx.y * TS;
    const size_t plane = (size_t)d.H * d.W;
    const float *X = img + c * plane, *Y = tgt + c * plane;
    for (int i = threadIdx.x; i < WT * WT; i += LOSS_THREADS) {
        const int r = i / WT, q = i % WT;
        sx[r][q] = load_or0(X, d.H, d.W, y0 - R + r, x0 - R + q);
        sy[r][q] = load_or0(Y, d.H, d.W, y0 - R + r, x0 - R + q);
    }
    __syncthreads();
    float wt[2 * R + 1];
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) wt[k] = c_w[k];
    // horizontal blurs: a thread slides the window along RBH outputs of a row
    for (int i = threadIdx.x; i < WT * (TS / RBH); i += LOSS_THREADS) {
        const int r = i / (TS / RBH), q0 = (i % (TS / RBH)) * RBH;
        float u[RBH + 2 * R], v[RBH + 2 * R];
#pragma unroll
        for (int k = 0; k < RBH + 2 * R; ++k) {
            u[k] = sx[r][q0 + k];
            v[k] = sy[r][q0 + k];
        }
#pragma unroll
        for (int o = 0; o < RBH; ++o) {
            float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
            for (int k = 0; k <= 2 * R; ++k) {
                const float uu = u[o + k], vv = v[o + k];
                a = fmaf(wt[k], uu, a);
                b = fmaf(wt[k], vv, b);
                aa = fmaf(wt[k], uu * uu, aa);
                bb = fmaf(wt[k], vv * vv, bb);
                ab = fmaf(wt[k], uu * vv, ab);
            }
            h[0][r][q0 + o] = a;
            h[1][r][q0 + o] = b;
            h[2][r][q0 + o] = aa;
            h[3][r][q0 + o] = bb;
            h[4][r][q0 + o] = ab;
        }
    }
    __syncthreads();
    float f_ssim = 0.f, f_l1 = 0.f;  // a thread's few pixels in FP32, the block's sums in FP64
    // vertical blurs: a thread slides the window down RBV outputs of a column
    // (one map at a time, so the window stays in registers)
    for (int i = threadIdx.x; i < (TS / RBV) * TS; i += LOSS_THREADS) {
        const int r0 = (i / TS) * RBV, q = i % TS;
        float m[5][RBV];
#pragma unroll
        for (int e = 0; e < 5; ++e) {
            float col[RBV + 2 * R];
#pragma unroll
            for (int k = 0; k < RBV + 2 * R; ++k) col[k] = h[e][r0 + k][q];
#pragma unroll
            for (int o = 0; o < RBV; ++o) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k <= 2 * R; ++k) acc = fmaf(wt[k], col[o + k], acc);
                m[e][o] = acc;
            }
        }
#pragma unroll
        for (int t = 0; t < RBV; ++t) {
            const int r = r0 + t;
            const int y = y0 + r, x = x0 + q;
            if (y >= d.H || x >= d.W) continue;
            const float mx = m[0][t], my = m[1][t];
            const float sxx = m[2][t] - mx * mx, syy = m[3][t] - my * my, sxy = m[4][t] - mx * my;
            const float A1 = 2.f * mx * my + C1, A2 = 2.f * sxy + C2;
            const float B1 = mx * mx + my * my + C1, B2 = sxx + syy + C2;
            // B1 >= C1 and B2 >= C2: the fast reciprocals are within 2 ulp
            const float inv = __fdividef(1.f, B1 * B2);
            const float S = A1 * A2 * inv;
            // derivatives with respect to mu_x, E[x^2], E[x y] (through s_xx, s_xy)
            const float dS_dsxx = -S * __fdividef(1.f, B2);
            const float dS_dsxy = 2.f * A1 * inv;
            const float dS_dmx = 2.f * my * A2 * inv - S * 2.f * mx * __fdividef(1.f, B1);
            const size_t o = c * plane + (size_t)y * d.W + x;
            coefA[o] = dS_dmx - 2.f * mx * dS_dsxx - my * dS_dsxy;
            coefB[o] = dS_dsxx;
            coefC[o] = dS_dsxy;
            f_ssim += S;
            f_l1 += fabsf(sx[r + R][q + R] - sy[r + R][q + R]);
        }
    }
    double s_ssim = f_ssim, s_l1 = f_l1;
    // block sums in FP64
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s_ssim += __shfl_xor_sync(0xffffffffu, s_ssim, o);
        s_l1 += __shfl_xor_sync(0xffffffffu, s_l1, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[0][warp] = s_ssim;
        red[1][warp] = s_l1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < LOSS_THREADS / 32; ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        part[2 * blk] = a;
        part[2 * blk + 1] = b;
    }
}

__global__ void __launch_bounds__(LOSS_THREADS)
ssim_backward_kernel(const float *__restrict__ img, const float *__restrict__ tgt, LossDims d,
                     const float *__restrict__ coefA, const float *__restrict__ coefB, const float *__restrict__ coefC,
                     float lambda, float weight, float *__restrict__ d_img)
{
    __shared__ float sa[3][WT][WT];
    __shared__ float h[3][WT][TS];
    __shared__ float c_w[2 * R + 1];
    make_taps(c_w);
    const int c = blockIdx.z, x0 = blockIdx.x * TS, y0 = blockIdx.y * TS;
    const size_t plane = (size_t)d.H * d.W;
    const float *P[3] = {coefA + c * plane, coefB + c * plane, coefC + c * plane};
    for (int i = threadIdx.x; i < WT * WT; i += LOSS_THREADS) {
        const int r = i / WT, q = i % WT;
#pragma unroll
        for (int e = 0; e < 3; ++e) sa[e][r][q] = load_or0(P[e], d.H, d.W, y0 - R + r, x0 - R + q);
    }
    __syncthreads();
    float wt[2 * R + 1];
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) wt[k] = c_w[k];
    // horizontal blurs of A, B, C: a register window along RBH outputs of a row
    for (int i = threadIdx.x; i < WT * (TS / RBH); i += LOSS_THREADS) {
        const int r = i / (TS / RBH), q0 = (i % (TS / RBH)) * RBH;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            float u[RBH + 2 * R];
#pragma unroll
            for (int k = 0; k < RBH + 2 * R; ++k) u[k] = sa[e][r][q0 + k];
#pragma unroll
            for (int o = 0; o < RBH; ++o) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k <= 2 * R; ++k) acc = fmaf(wt[k], u[o + k], acc);
                h[e][r][q0 + o] = acc;
            }
        }
    }
    __syncthreads();
    const float n = (float)((double)d.C * d.H * d.W);
    const float k_l1 = weight * (1.f - lambda) / n, k_ss = -weight * lambda / n;
    // vertical blurs and the per-pixel combination: a register window down
    // RBV outputs of a column
    for (int i = threadIdx.x; i < (TS / RBV) * TS; i += LOSS_THREADS) {
        const int r0 = (i / TS) * RBV, q = i % TS;
        float acc[3][RBV];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            float col[RBV + 2 * R];
#pragma unroll
            for (int k = 0; k < RBV + 2 * R; ++k) col[k] = h[e][r0 + k][q];
#pragma unroll
            for (int t = 0; t < RBV; ++t) {
                float a = 0.f;
#pragma unroll
                for (int k = 0; k <= 2 * R; ++k) a = fmaf(wt[k], col[t + k], a);
                acc[e][t] = a;
            }
        }
#pragma unroll
        for (int t = 0; t < RBV; ++t) {
            const int y = y0 + r0 + t, x = x0 + q;
            if (y >= d.H || x >= d.W) continue;
            const size_t o = c * plane + (size_t)y * d.W + x;
            const float xv = __ldg(img + o), yv = __ldg(tgt + o);
            const float diff = xv - yv;
            const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
            const float dssim = acc[0][t] + 2.f * xv * acc[1][t] + yv * acc[2][t];
            d_img[o] = k_l1 * sgn + k_ss * dssim;
        }
    }
}

__global__ void __launch_bounds__(1024)
loss_reduce_kernel(const double *__restrict__ part, int nblk, double n, float lambda, float weight, int accumulate,
                   float *__restrict__ loss)
{
    __shared__ double s[2][32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
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
        double ss = 0.0, l1 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            ss += s[0][w];
            l1 += s[1][w];
        }
        const double L = (1.0 - lambda) * (l1 / n) + lambda * (1.0 - ss / n);
        const float v = (float)(weight * L);
        *loss = accumulate ? *loss + v : v;
    }
}

int check_loss(const avatar_image_loss_args *a)
{
    if (!a || a->C < 1 || a->H < 1 || a->W < 1 || a->H > 65536 || a->W > 65536) return AVATAR_ERR_INVALID_ARG;
    if (!(a->lambda >= 0.f && a->lambda <= 1.f) || !(a->weight >= 0.f)) return AVATAR_ERR_INVALID_ARG;
    return AVATAR_OK;
}

LossDims dims_of(const avatar_image_loss_args *a)
{
    LossDims d;
    d.C = a->C;
    d.H = a->H;
    d.W = a->W;
    d.tx = (a->W + TS - 1) / TS;
    d.ty = (a->H + TS - 1) / TS;
    return d;
}

size_t loss_layout(const avatar_image_loss_args *a, void *base, size_t cap, float **A, float **B, float **Cc,
                   double **part)
{
    WsCarver c(base, cap);
    const LossDims d = dims_of(a);
    const size_t n = (size_t)a->C * a->H * a->W;
    float *pa = c.take<float>(n), *pb = c.take<float>(n), *pc = c.take<float>(n);
    double *pp = c.take<double>((size_t)2 * d.tx * d.ty * a->C);
    if (A) {
        *A = pa;
        *B = pb;
        *Cc = pc;
        *part = pp;
    }
    return c.off;
}

}  // namespace

extern "C" size_t avatar_image_loss_workspace_size(const avatar_image_loss_args *a)
{
    if (check_loss(a) != AVATAR_OK) return 0;
    return loss_layout(a, nullptr, 0, nullptr, nullptr, nullptr, nullptr);
}

extern "C" int avatar_image_loss(avatar_ctx *ctx, const avatar_image_loss_args *a, void *ws, size_t ws_bytes,
                                 avatar_stream_t stream)
{
    if (!ctx) return AVATAR_ERR_INVALID_ARG;
    AV_TRY(check_loss(a));
    if (!a->img || !a->target || !a->loss) return AVATAR_ERR_INVALID_ARG;
    if (!ws || (((uintptr_t)ws) & 255)) return AVATAR_ERR_WORKSPACE;
    float *A, *B, *Cc;
    double *part;
    if (loss_layout(a, ws, ws_bytes, &A, &B, &Cc, &part) > ws_bytes) return AVATAR_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    const LossDims d = dims_of(a);
    const dim3 grid(d.tx, d.ty, d.C);
    ssim_forward_kernel<<<grid, LOSS_THREADS, 0, st>>>(a->img, a->target, d, A, B, Cc, part);
    AV_CHECK_LAUNCH();
    const double n = (double)a->C * a->H * a->W;
    loss_reduce_kernel<<<1, 1024, 0, st>>>(part, d.tx * d.ty * d.C, n, a->lambda, a->weight, a->accumulate,
                                           a->loss);
    AV_CHECK_LAUNCH();
    if (a->d_img) {
        ssim_backward_kernel<<<grid, LOSS_THREADS, 0, st>>>(a->img, a->target, d, A, B, Cc, a->lambda, a->weight,
                                                            a->d_img);
        AV_CHECK_LAUNCH();
    }
    return AVATAR_OK;
}
