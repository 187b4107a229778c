// Density-based Gaussian densification (App. B, Alg. 1): Gaussians are
// added on the mesh triangles whose Gaussian density, estimated from the
// nearest-vertex sets S_g of Eq. 1, is below d0.
//   D_v[k] = #{i : k in S_g^i}                         (integer atomics)
//   S_f    = D_v[a] + D_v[b] + D_v[c],  d_f = S_f / (6 K_g)
//   w_f    = max(0, d0 6 K_g - S_f)   (P_f = w_f / (6 K_g), exact integers)
//   W = sum w_f (inclusive scan),  N' = floor((p0 W) / (6 K_g)) in FP64
//   draw j: s_j = floor(r0_j W / 2^32), triangle t_j = min{f : cum_f > s_j},
//           u, v = (r1_j >> 8) 2^-24, (r2_j >> 8) 2^-24, reflected if u + v > 1,
//           x_j = a + u (b - a) + v (c - a)
// Every decision is integer (or exact FP32), so the counts, the number of
// draws and each draw's triangle are bit-identical to the oracle; only the
// FP32 positions round.  Five launches, no host synchronisation.
#include "common.cuh"

namespace {

constexpr int DN_THREADS = 256;
constexpr int DN_PER = 4;                         // faces per thread in the scan
constexpr int DN_BLOCK = DN_THREADS * DN_PER;     // faces per scan block
constexpr int DN_MAX_BLOCKS = 1 << 16;            // F < 2^26

__global__ void __launch_bounds__(DN_THREADS)
dens_count_kernel(const int32_t *__restrict__ knn, long n, int Nv, int32_t *__restrict__ Dv, int32_t *status)
{
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const int k = __ldg(knn + e);
        if ((unsigned)k >= (unsigned)Nv) {
            av_report(status, AVATAR_ERR_INDEX);
            continue;
        }
        atomicAdd(Dv + k, 1);
    }
}

// Per face: S_f, d_f, the weight w_f; per block the sum of its weights.
__global__ void __launch_bounds__(DN_THREADS)
dens_face_kernel(const int32_t *__restrict__ faces, int F, int Nv, int Kg, long long thr,
                 const int32_t *__restrict__ Dv, float *__restrict__ df, long long *__restrict__ w,
                 long long *__restrict__ block_sum, int32_t *status)
{
    __shared__ long long s_part[DN_THREADS / 32];
    long long acc = 0;
#pragma unroll
    for (int i = 0; i < DN_PER; ++i) {
        const int f = blockIdx.x * DN_BLOCK + i * DN_THREADS + threadIdx.x;
        if (f >= F) break;
        long long S = 0;
        bool ok = true;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int v = __ldg(faces + 3 * (size_t)f + c);
            if ((unsigned)v >= (unsigned)Nv) {
                ok = false;
            } else {
                S += __ldg(Dv + v);
            }
        }
        if (!ok) av_report(status, AVATAR_ERR_INDEX);
        const long long wf = ok && S < thr ? thr - S : 0;
        w[f] = wf;
        if (df) df[f] = (float)((double)S / (double)(6 * Kg));
        acc += wf;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int i = 0; i < DN_THREADS / 32; ++i) t += s_part[i];
        block_sum[blockIdx.x] = t;
    }
}

// One block: exclusive offsets of the block sums, W, and N'.
__global__ void __launch_bounds__(1024)
dens_total_kernel(long long *__restrict__ block_sum, int nblocks, int Kg, double p0, int capacity,
                  long long *__restrict__ W_out, int32_t *__restrict__ n_out, int32_t *__restrict__ count,
                  int32_t *status)
{
    __shared__ long long s_carry;
    __shared__ long long s_warp[32];
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < nblocks; base += 1024) {
        const int i = base + threadIdx.x;
        const long long v = i < nblocks ? block_sum[i] : 0;
        long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            long long t = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            s_warp[lane] = t;
        }
        __syncthreads();
        const long long incl = x + (warp > 0 ? s_warp[warp - 1] : 0) + s_carry;
        if (i < nblocks) block_sum[i] = incl - v;  // exclusive offset
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long W = s_carry;
        *W_out = W;
        long long n = 0;
        if (W > 0) {
            const double q = floor(__dmul_rn(p0, (double)W) / (double)(6 * Kg));
            n = q > 2147483647.0 ? 2147483647LL : (long long)q;
        }
        *count = (int32_t)n;
        if (n > capacity) {
            av_report(status, AVATAR_ERR_OVERFLOW);
            n = capacity;
        }
        *n_out = (int32_t)n;
    }
}

// Inclusive cumulative weights: the block's offset plus its local scan.
__global__ void __launch_bounds__(DN_THREADS)
dens_cum_kernel(const long long *__restrict__ w, int F, const long long *__restrict__ block_off,
                long long *__restrict__ cum)
{
    __shared__ long long s_warp[DN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int f0 = blockIdx.x * DN_BLOCK + threadIdx.x * DN_PER;  // DN_PER consecutive faces per thread
    long long loc[DN_PER];
    long long run = 0;
#pragma unroll
    for (int i = 0; i < DN_PER; ++i) {
        run += f0 + i < F ? w[f0 + i] : 0;
        loc[i] = run;
    }
    long long x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long t = lane < DN_THREADS / 32 ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < DN_THREADS / 32) s_warp[lane] = t;
    }
    __syncthreads();
    const long long before = block_off[blockIdx.x] + (x - run) + (warp > 0 ? s_warp[warp - 1] : 0);
#pragma unroll
    for (int i = 0; i < DN_PER; ++i)
        if (f0 + i < F) cum[f0 + i] = before + loc[i];
}

__global__ void __launch_bounds__(DN_THREADS)
dens_sample_kernel(const long long *__restrict__ cum, int F, const long long *__restrict__ W_in,
                   const int32_t *__restrict__ n_in, int capacity, const uint32_t *__restrict__ rand,
                   const int32_t *__restrict__ faces, const float *__restrict__ xv, int Nv,
                   int32_t *__restrict__ tri, float *__restrict__ x, int32_t *__restrict__ ng)
{
    const int n = *n_in;
    const unsigned long long W = (unsigned long long)*W_in;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const uint32_t r0 = __ldg(rand + j), r1 = __ldg(rand + (size_t)capacity + j),
                       r2 = __ldg(rand + 2 * (size_t)capacity + j);
        const long long s = (long long)__umul64hi((unsigned long long)r0 << 32, W);  // floor(r0 W / 2^32)
        int lo = 0, hi = F - 1;                                                      // min f with cum[f] > s
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(cum + mid) > s) hi = mid;
            else lo = mid + 1;
        }
        tri[j] = lo;
        if (ng) atomicAdd(ng + lo, 1);
        // u + v > 1 decided on the integers (the FP32 sum can round at 1 + 2^-24)
        uint32_t ku = r1 >> 8, kv = r2 >> 8;
        if (ku + kv > (1u << 24)) {
            ku = (1u << 24) - ku;
            kv = (1u << 24) - kv;
        }
        const float u = (float)ku * 0x1p-24f, v = (float)kv * 0x1p-24f;
        const int a = __ldg(faces + 3 * (size_t)lo), b = __ldg(faces + 3 * (size_t)lo + 1),
                  c = __ldg(faces + 3 * (size_t)lo + 2);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float pa = __ldg(xv + (size_t)k * Nv + a), pb = __ldg(xv + (size_t)k * Nv + b),
                        pc = __ldg(xv + (size_t)k * Nv + c);
            x[(size_t)k * capacity + j] = pa + u * (pb - pa) + v * (pc - pa);
        }
    }
}

struct DensWs {
    int32_t *Dv;
    long long *w, *cum, *block_sum, *W;
    int32_t *n;
};

size_t dens_ws_layout(const avatar_densify_args *a, void *base, size_t cap, DensWs *out)
{
    WsCarver c(base, cap);
    DensWs d;
    const int nb = (a->F + DN_BLOCK - 1) / DN_BLOCK;
    d.Dv = c.take<int32_t>((size_t)a->Nv);
    d.w = c.take<long long>((size_t)a->F);
    d.cum = c.take<long long>((size_t)a->F);
    d.block_sum = c.take<long long>((size_t)(nb > 0 ? nb : 1));
    d.W = c.take<long long>(1);
    d.n = c.take<int32_t>(1);
    if (out) *out = d;
    return c.off;
}

int check_densify(const avatar_densify_args *a)
{
    if (!a || a->G < 0 || a->Nv < 1 || a->F < 1 || a->Kg < 1 || a->Kg > 64 || a->capacity < 0)
        return AVATAR_ERR_INVALID_ARG;
    if ((a->F + DN_BLOCK - 1) / DN_BLOCK > DN_MAX_BLOCKS) return AVATAR_ERR_UNSUPPORTED;
    const double thr = (double)a->d0 * 6.0 * a->Kg;
    if (!(thr >= 0.0) || thr > 1e15 || thr != floor(thr)) return AVATAR_ERR_INVALID_ARG;
    if (!(a->p0 >= 0.0) || !(a->p0 < 1e9)) return AVATAR_ERR_INVALID_ARG;
    if ((a->G > 0 && !a->knn) || !a->faces || !a->xv || !a->count) return AVATAR_ERR_INVALID_ARG;
    if (a->capacity > 0 && (!a->rand || !a->tri || !a->x)) return AVATAR_ERR_INVALID_ARG;
    return AVATAR_OK;
}

}  // namespace

extern "C" size_t avatar_densify_workspace_size(const avatar_densify_args *a)
{
    if (check_densify(a) != AVATAR_OK) return 0;
    return dens_ws_layout(a, nullptr, 0, nullptr);
}

extern "C" int avatar_densify(avatar_ctx *ctx, const avatar_densify_args *a, void *ws, size_t ws_bytes,
                              avatar_stream_t stream)
{
    if (!ctx) return AVATAR_ERR_INVALID_ARG;
    AV_TRY(check_densify(a));
    if (!ws || (((uintptr_t)ws) & 255) || ws_bytes < dens_ws_layout(a, nullptr, 0, nullptr))
        return AVATAR_ERR_WORKSPACE;
    DensWs d;
    dens_ws_layout(a, ws, ws_bytes, &d);
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *Dv = a->Dv ? a->Dv : d.Dv;
    if (cudaMemsetAsync(Dv, 0, sizeof(int32_t) * (size_t)a->Nv, st) != cudaSuccess) return AVATAR_ERR_CUDA;
    if (a->ng && cudaMemsetAsync(a->ng, 0, sizeof(int32_t) * (size_t)a->F, st) != cudaSuccess)
        return AVATAR_ERR_CUDA;
    const long n = (long)a->Kg * a->G;
    if (n > 0) {
        long blocks = (n + DN_THREADS - 1) / DN_THREADS;
        if (blocks > (long)ctx->sm_count * 16) blocks = (long)ctx->sm_count * 16;
        dens_count_kernel<<<(int)blocks, DN_THREADS, 0, st>>>(a->knn, n, a->Nv, Dv, a->status);
    }
    const int nb = (a->F + DN_BLOCK - 1) / DN_BLOCK;
    const long long thr = (long long)((double)a->d0 * 6.0 * a->Kg);
    dens_face_kernel<<<nb, DN_THREADS, 0, st>>>(a->faces, a->F, a->Nv, a->Kg, thr, Dv, a->df, d.w, d.block_sum,
                                                a->status);
    dens_total_kernel<<<1, 1024, 0, st>>>(d.block_sum, nb, a->Kg, a->p0, a->capacity, d.W, d.n, a->count,
                                          a->status);
    dens_cum_kernel<<<nb, DN_THREADS, 0, st>>>(d.w, a->F, d.block_sum, d.cum);
    if (a->capacity > 0) {
        int blocks = (a->capacity + DN_THREADS - 1) / DN_THREADS;
        if (blocks > ctx->sm_count * 8) blocks = ctx->sm_count * 8;
        dens_sample_kernel<<<blocks, DN_THREADS, 0, st>>>(d.cum, a->F, d.W, d.n, a->capacity, a->rand, a->faces,
                                                         a->xv, a->Nv, a->tri, a->x, a->ng);
    }
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}
