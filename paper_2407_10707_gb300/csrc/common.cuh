// Shared device helpers of the sm_103a relit-avatar library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "avatar.h"

struct avatar_ctx {
    int device;
    int sm_count;
    int max_smem_optin;
    int cluster_ok;
    int tune[AVATAR_TUNE_COUNT];
};

#define AV_CHECK_LAUNCH()                                    \
    do {                                                     \
        if (cudaPeekAtLastError() != cudaSuccess) {          \
            (void)cudaGetLastError();                        \
            return AVATAR_ERR_CUDA;                          \
        }                                                    \
    } while (0)

#define AV_TRY(expr)                          \
    do {                                      \
        int _rc = (expr);                     \
        if (_rc != AVATAR_OK) return _rc;     \
    } while (0)

static inline size_t av_align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Carves aligned sub-buffers out of a caller workspace.
struct WsCarver {
    char *base;
    size_t off;
    size_t cap;
    __host__ WsCarver(void *p, size_t c) : base((char *)p), off(0), cap(c) {}
    template <class T>
    __host__ T *take(size_t n) {
        size_t bytes = av_align256(n * sizeof(T));
        T *r = base ? (T *)(base + off) : nullptr;
        off += bytes;
        return r;
    }
    __host__ bool ok() const { return base != nullptr && off <= cap; }
};

__device__ __forceinline__ void av_report(int32_t *status, int code)
{
    if (status) atomicCAS(status, 0, code);
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums of sixteen per-lane values over the warp at once, by recursive
// halving (a reduce-scatter): each step keeps half of the values, chosen by
// one lane bit, and adds the partner lane's copy of that half.  On return
// lanes 2i and 2i + 1 hold the total of v[i]: 16 shuffles instead of the 80
// of sixteen separate reductions.
__device__ __forceinline__ float warp_reduce_scatter16(const float (&v)[16])
{
    const unsigned lane = threadIdx.x & 31u;
    const bool b4 = lane & 16u, b3 = lane & 8u, b2 = lane & 4u, b1 = lane & 2u;
    float w[8], u[4], t[2];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        w[i] = (b4 ? v[8 + i] : v[i]) + __shfl_xor_sync(0xffffffffu, b4 ? v[i] : v[8 + i], 16);
#pragma unroll
    for (int i = 0; i < 4; ++i)
        u[i] = (b3 ? w[4 + i] : w[i]) + __shfl_xor_sync(0xffffffffu, b3 ? w[i] : w[4 + i], 8);
#pragma unroll
    for (int i = 0; i < 2; ++i)
        t[i] = (b2 ? u[2 + i] : u[i]) + __shfl_xor_sync(0xffffffffu, b2 ? u[i] : u[2 + i], 4);
    const float s = (b1 ? t[1] : t[0]) + __shfl_xor_sync(0xffffffffu, b1 ? t[0] : t[1], 2);
    return s + __shfl_xor_sync(0xffffffffu, s, 1);
}

// Warp sums of nine per-lane values: v[0..7] by recursive halving (lanes
// 4i .. 4i + 3 end with the total of v[i], i = lane / 4) and v[8] by a
// butterfly (every lane ends with its total): 14 shuffles, where padding to
// sixteen slots for warp_reduce_scatter16 takes 16 and twice the selects.
__device__ __forceinline__ float warp_reduce_scatter9(const float (&v)[9], float &tot8)
{
    const unsigned lane = threadIdx.x & 31u;
    const bool b4 = lane & 16u, b3 = lane & 8u, b2 = lane & 4u;
    float w[4], u[2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        w[i] = (b4 ? v[4 + i] : v[i]) + __shfl_xor_sync(0xffffffffu, b4 ? v[i] : v[4 + i], 16);
#pragma unroll
    for (int i = 0; i < 2; ++i)
        u[i] = (b3 ? w[2 + i] : w[i]) + __shfl_xor_sync(0xffffffffu, b3 ? w[i] : w[2 + i], 8);
    float t = (b2 ? u[1] : u[0]) + __shfl_xor_sync(0xffffffffu, b2 ? u[0] : u[1], 4);
    t += __shfl_xor_sync(0xffffffffu, t, 2);
    t += __shfl_xor_sync(0xffffffffu, t, 1);
    float e = v[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    tot8 = e;
    return t;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Element i of an attribute array stored as FP32 or BF16 (attr_dtype).
__device__ __forceinline__ float ld_attr(const void *p, size_t i, int dtype)
{
    return dtype == AVATAR_DTYPE_BF16 ? __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16 *>(p) + i))
                                      : __ldg(reinterpret_cast<const float *>(p) + i);
}

constexpr float AV_PI = 3.14159265358979323846f;
