// Storage order of the Gaussians (a layout step; the paper has no
// counterpart).  Every per-Gaussian kernel gathers records of the Gaussians'
// nearest mesh vertices (skinning: Eq. 1 over S_g; shading: the neighbours'
// visibility words; the backward passes: atomics into the vertices).  In an
// avatar whose Gaussians come in arbitrary order, the 32 Gaussians of a warp
// touch 32 unrelated vertices; stored in the order of their nearest vertex
// (the mesh's vertices are themselves laid out along its surface), a warp's
// Gaussians share their neighbours.  Results do not depend on the order.
//
//   avatar_gaussian_order   stable order of the Gaussians by nearest vertex
//                           (the device radix sort of the splatting path)
//   avatar_gather_columns   applies an order to structure-of-arrays columns
//                           (or to the rows of an array of small records)
#include "splat_dev.cuh"

namespace {

int order_grid(const avatar_ctx *ctx, long n)
{
    long b = (n + 255) / 256, cap = (long)ctx->sm_count * 8;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

__global__ void order_keys_kernel(const int32_t *__restrict__ nearest, int G, int Nv, uint32_t *__restrict__ keys,
                                  int32_t *__restrict__ vals, int32_t *__restrict__ count, int32_t *status)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G; i += gridDim.x * blockDim.x) {
        int v = __ldg(nearest + i);
        if ((unsigned)v >= (unsigned)Nv) {
            av_report(status, AVATAR_ERR_INDEX);
            v = Nv - 1;  // still a key of the sort's width; the order stays a permutation
        }
        keys[i] = (uint32_t)v;
        vals[i] = i;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = G;
}

template <class T>
__global__ void gather_columns_kernel(int rows, int n, const T *__restrict__ src, T *__restrict__ dst,
                                      const int32_t *__restrict__ order, int32_t *status)
{
    const size_t r = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j = __ldg(order + i);
        if ((unsigned)j >= (unsigned)n) {
            av_report(status, AVATAR_ERR_INDEX);
            dst[r * n + i] = T(0);
            continue;
        }
        dst[r * n + i] = __ldg(src + r * n + j);
    }
}

struct OrderWs {
    uint32_t *k0, *k1;
    int32_t *v1, *count;
    SortWs sort;
};

size_t order_ws_layout(int G, void *base, size_t cap, OrderWs *out)
{
    WsCarver c(base, cap);
    const size_t n = (size_t)(G > 0 ? G : 1);
    OrderWs w;
    w.k0 = c.take<uint32_t>(n);
    w.k1 = c.take<uint32_t>(n);
    w.v1 = c.take<int32_t>(n);
    w.count = c.take<int32_t>(1);
    w.sort.hist = c.take<int32_t>((size_t)OS_MAX_PASSES * RADIX + OS_MAX_PASSES);
    w.sort.desc = c.take<unsigned>(sort_desc_words(n));
    if (out) *out = w;
    return c.off;
}

}  // namespace

extern "C" size_t avatar_gaussian_order_workspace_size(int G)
{
    if (G < 0) return 0;
    return order_ws_layout(G, nullptr, 0, nullptr);
}

extern "C" int avatar_gaussian_order(avatar_ctx *ctx, int G, int Nv, const int32_t *nearest, int32_t *order,
                                     void *ws, size_t ws_bytes, int32_t *status, avatar_stream_t stream)
{
    if (!ctx || G < 0 || Nv < 1 || (G > 0 && (!nearest || !order))) return AVATAR_ERR_INVALID_ARG;
    if (G == 0) return AVATAR_OK;
    OrderWs w;
    if (!ws || (((uintptr_t)ws) & 255) || ws_bytes < order_ws_layout(G, nullptr, 0, nullptr))
        return AVATAR_ERR_WORKSPACE;
    order_ws_layout(G, ws, ws_bytes, &w);
    cudaStream_t st = (cudaStream_t)stream;
    const int bits = Nv > 1 ? 32 - __builtin_clz((unsigned)(Nv - 1)) : 1;
    const int passes = (bits + 7) / 8;
    // the sort ends in (k0, v0) after an even number of passes, in (k1, v1)
    // after an odd one: the caller's order is whichever holds the result
    int32_t *v0 = passes % 2 == 0 ? order : w.v1;
    int32_t *v1 = passes % 2 == 0 ? w.v1 : order;
    order_keys_kernel<<<order_grid(ctx, G), 256, 0, st>>>(nearest, G, Nv, w.k0, v0, w.count, status);
    AV_CHECK_LAUNCH();
    return radix_sort(w.k0, v0, w.k1, v1, passes * 8, w.count, G, w.sort, status, st, sort_spin_limit(ctx));
}

// A w-word element (w 32-bit words) copied as a unit.
template <int W>
struct Words {
    uint32_t v[W];
    __host__ __device__ Words() {}
    __host__ __device__ explicit Words(int) {
        for (int i = 0; i < W; ++i) v[i] = 0u;
    }
};

template <int W>
__global__ void gather_words_kernel(int rows, int n, const Words<W> *__restrict__ src, Words<W> *__restrict__ dst,
                                    const int32_t *__restrict__ order, int32_t *status)
{
    const size_t r = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j = __ldg(order + i);
        if ((unsigned)j >= (unsigned)n) {
            av_report(status, AVATAR_ERR_INDEX);
            dst[r * n + i] = Words<W>(0);
            continue;
        }
        dst[r * n + i] = src[r * n + j];
    }
}

extern "C" int avatar_gather_columns(avatar_ctx *ctx, int rows, int n, int elem_bytes, const void *src, void *dst,
                                     const int32_t *order, int32_t *status, avatar_stream_t stream)
{
    if (!ctx || rows < 0 || rows > 65535 || n < 0) return AVATAR_ERR_INVALID_ARG;
    if (elem_bytes != 2 && elem_bytes != 4 && elem_bytes != 8 && elem_bytes != 12 && elem_bytes != 16)
        return AVATAR_ERR_INVALID_ARG;
    if (rows == 0 || n == 0) return AVATAR_OK;
    if (!src || !dst || !order || src == dst) return AVATAR_ERR_INVALID_ARG;
    if ((((uintptr_t)src) | ((uintptr_t)dst)) & (elem_bytes == 2 ? 1 : 3)) return AVATAR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const dim3 grid(order_grid(ctx, n), rows);
    switch (elem_bytes) {
        case 2:
            gather_columns_kernel<uint16_t><<<grid, 256, 0, st>>>(rows, n, (const uint16_t *)src, (uint16_t *)dst,
                                                                  order, status);
            break;
        case 4:
            gather_columns_kernel<uint32_t><<<grid, 256, 0, st>>>(rows, n, (const uint32_t *)src, (uint32_t *)dst,
                                                                  order, status);
            break;
        case 8:
            gather_words_kernel<2><<<grid, 256, 0, st>>>(rows, n, (const Words<2> *)src, (Words<2> *)dst, order, status);
            break;
        case 12:
            gather_words_kernel<3><<<grid, 256, 0, st>>>(rows, n, (const Words<3> *)src, (Words<3> *)dst, order, status);
            break;
        default:
            gather_words_kernel<4><<<grid, 256, 0, st>>>(rows, n, (const Words<4> *)src, (Words<4> *)dst, order, status);
            break;
    }
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}
