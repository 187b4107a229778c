// Throughput probes of the CUDA-core pipes: the measured denominators of the
// roofline fractions that are bound by plain arithmetic (visibility: INT32;
// shading and blending: FP32).  Not part of the paper's method.
//
// Every thread runs `iters` rounds of 16 x 8 operations of one kind on eight
// chains; each operation reads its own chain and the next one, so the chains
// stay live and no round can be folded into a closed form, while eight
// independent operations per round keep the pipe, not the latency, the bound.
// The result is stored only if it equals a runtime seed (practically never),
// which keeps the work without a memory stream.
#include "common.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_ROUNDS = 16;   // unrolled rounds per loop trip: 128 operations

template <int KIND>
__global__ void __launch_bounds__(PROBE_THREADS) alu_probe_kernel(int iters, uint32_t seed, uint32_t *sink)
{
    uint32_t a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed * (2u * i + 1u) + threadIdx.x * 0x9E3779B9u + blockIdx.x;
    if (KIND == AVATAR_PROBE_FFMA) {
        float f[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) f[i] = __uint_as_float((a[i] & 0x007FFFFFu) | 0x3F800000u);   // [1, 2)
        const float c = __uint_as_float(0x3F7FFF00u | (seed & 0xFFu));                          // just below 1
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < PROBE_ROUNDS; ++r) {
#pragma unroll
                for (int i = 0; i < 8; ++i) f[i] = fmaf(f[i], c, f[(i + 1) & 7]);
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = __float_as_uint(f[i]);
    } else {
        const uint32_t k = seed ^ 0x5BD1E995u;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < PROBE_ROUNDS; ++r) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const uint32_t b = a[(i + 1) & 7];
                    if (KIND == AVATAR_PROBE_IADD3) a[i] = a[i] + b + k;
                    else if (KIND == AVATAR_PROBE_LOP3) a[i] = (a[i] & b) ^ k;
                    else a[i] = a[i] * b + k;   // AVATAR_PROBE_IMAD
                }
            }
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) x ^= a[i];
    if (x == seed) *sink = x;
}

template <int KIND>
void launch_probe(int blocks, int iters, uint32_t *sink, cudaStream_t st)
{
    alu_probe_kernel<KIND><<<blocks, PROBE_THREADS, 0, st>>>(iters, 0x2545F491u, sink);
}

}  // namespace

extern "C" int avatar_probe_alu(avatar_ctx *ctx, int kind, int iters, uint32_t *sink, long long *ops,
                                avatar_stream_t stream)
{
    if (!ctx || !sink || iters < 1 || kind < 0 || kind > AVATAR_PROBE_IMAD) return AVATAR_ERR_INVALID_ARG;
    const int blocks = ctx->sm_count * (2048 / PROBE_THREADS);   // a full wave of 2,048 threads per SM
    cudaStream_t st = (cudaStream_t)stream;
    switch (kind) {
        case AVATAR_PROBE_FFMA: launch_probe<AVATAR_PROBE_FFMA>(blocks, iters, sink, st); break;
        case AVATAR_PROBE_IADD3: launch_probe<AVATAR_PROBE_IADD3>(blocks, iters, sink, st); break;
        case AVATAR_PROBE_LOP3: launch_probe<AVATAR_PROBE_LOP3>(blocks, iters, sink, st); break;
        default: launch_probe<AVATAR_PROBE_IMAD>(blocks, iters, sink, st); break;
    }
    AV_CHECK_LAUNCH();
    if (ops) *ops = (long long)blocks * PROBE_THREADS * iters * (PROBE_ROUNDS * 8);
    return AVATAR_OK;
}
