// Context, status strings and the L1 image loss (Sec. 3.3, Eq. 5, L1 part).
#include <stdlib.h>

#include "common.cuh"

namespace {

__global__ void __launch_bounds__(256)
l1_loss_kernel(int64_t n, const float *__restrict__ img, const float *__restrict__ tgt, float *__restrict__ loss,
               float *__restrict__ d_img, float inv_n)
{
    float acc = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float d = img[i] - tgt[i];
        acc += fabsf(d);
        if (d_img) d_img[i] = d > 0.f ? inv_n : (d < 0.f ? -inv_n : 0.f);
    }
    acc = warp_sum(acc);
    __shared__ float ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.f;
        v = warp_sum(v);
        if (threadIdx.x == 0) atomicAdd(loss, v * inv_n);
    }
}

}  // namespace

extern "C" const char *avatar_status_string(int status)
{
    switch (status) {
        case AVATAR_OK: return "ok";
        case AVATAR_ERR_INVALID_ARG: return "invalid argument";
        case AVATAR_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case AVATAR_ERR_OVERFLOW: return "tile/Gaussian pair buffer overflow";
        case AVATAR_ERR_TIMEOUT: return "bounded device wait expired";
        case AVATAR_ERR_CUDA: return "CUDA runtime error";
        case AVATAR_ERR_UNSUPPORTED: return "unsupported device or configuration";
        case AVATAR_ERR_INDEX: return "index out of range";
        default: return "unknown status";
    }
}

extern "C" int avatar_version(void) { return 10000; }

extern "C" int avatar_ctx_create(avatar_ctx **out, int device)
{
    if (!out) return AVATAR_ERR_INVALID_ARG;
    *out = nullptr;
    int major = 0, minor = 0, sms = 0, smem = 0, cluster = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&cluster, cudaDevAttrClusterLaunch, device) != cudaSuccess) {
        (void)cudaGetLastError();
        return AVATAR_ERR_CUDA;
    }
    // The kernels are built for sm_103a only.
    if (major != 10 || minor != 3 || !cluster) return AVATAR_ERR_UNSUPPORTED;
    avatar_ctx *c = (avatar_ctx *)malloc(sizeof(avatar_ctx));
    if (!c) return AVATAR_ERR_INVALID_ARG;
    c->device = device;
    c->sm_count = sms;
    c->max_smem_optin = smem;
    c->cluster_ok = cluster;
    for (int i = 0; i < AVATAR_TUNE_COUNT; ++i) c->tune[i] = 0;
    c->tune[AVATAR_TUNE_BLEND_PPT] = 1;
    c->tune[AVATAR_TUNE_BLEND_BWD_PPT] = 1;
    c->tune[AVATAR_TUNE_BATCH_TILE] = 16;
    c->tune[AVATAR_TUNE_REGION_MASKS] = 1;
    *out = c;
    return AVATAR_OK;
}

extern "C" int avatar_ctx_destroy(avatar_ctx *ctx)
{
    free(ctx);
    return AVATAR_OK;
}

extern "C" int avatar_ctx_sm_count(const avatar_ctx *ctx) { return ctx ? ctx->sm_count : 0; }

extern "C" int avatar_l1_loss(avatar_ctx *ctx, int64_t n, const float *img, const float *target, float *loss,
                              float *d_img, avatar_stream_t stream)
{
    if (!ctx || n < 1 || !img || !target || !loss) return AVATAR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess) return AVATAR_ERR_CUDA;
    long blocks = (n + 255) / 256;
    if (blocks > ctx->sm_count * 4L) blocks = ctx->sm_count * 4L;
    l1_loss_kernel<<<(int)blocks, 256, 0, st>>>(n, img, target, loss, d_img, (float)(1.0 / (double)n));
    AV_CHECK_LAUNCH();
    return AVATAR_OK;
}

extern "C" int avatar_ctx_set_tuning(avatar_ctx *ctx, int key, int value)
{
    if (!ctx || key < 0 || key >= AVATAR_TUNE_COUNT) return AVATAR_ERR_INVALID_ARG;
    switch (key) {
        case AVATAR_TUNE_BLEND_PPT:
        case AVATAR_TUNE_BLEND_BWD_PPT:
            if (value != 1 && value != 2 && value != 4) return AVATAR_ERR_INVALID_ARG;
            break;
        case AVATAR_TUNE_BATCH_TILE:
            if (value != 8 && value != 16 && value != 32) return AVATAR_ERR_INVALID_ARG;
            break;
        case AVATAR_TUNE_VIS_CLUSTER:
            if (value != 0 && value != 2 && value != 4 && value != 8) return AVATAR_ERR_INVALID_ARG;
            break;
        case AVATAR_TUNE_WAIT_LIMIT:
            if (value < 0 || value > (1 << 30)) return AVATAR_ERR_INVALID_ARG;
            break;
        case AVATAR_TUNE_REGION_MASKS:
            if (value != 0 && value != 1) return AVATAR_ERR_INVALID_ARG;
            break;
        default: break;
    }
    ctx->tune[key] = value;
    return AVATAR_OK;
}

extern "C" int avatar_ctx_get_tuning(const avatar_ctx *ctx, int key)
{
    if (!ctx || key < 0 || key >= AVATAR_TUNE_COUNT) return -1;
    return ctx->tune[key];
}
