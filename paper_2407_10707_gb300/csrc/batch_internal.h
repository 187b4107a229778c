// Batched forms of the stage launchers, used by the batched render (batch.cu).
// Each runs one launch per step over the whole batch (grid y or z indexes the
// pose or view); the per-frame entry points call the same kernels with a
// batch of one.
#pragma once

#include <cuda_runtime.h>

#include "avatar.h"

#define AV_INTERNAL __attribute__((visibility("hidden")))

// (a) B poses: pose [B][J][3], bone [B][J][12], xp [3][B Nv], xd and nd
// [3][B G], cov [6][B G], records [B Nv]; ag, rg, pg, ubar ([.][G], pose
// independent) are written once.
AV_INTERNAL size_t av_skin_batch_workspace_size(const avatar_skin_args *a, int B);
AV_INTERNAL int av_skin_batch(avatar_ctx *ctx, const avatar_skin_args *a, int B, void *ws, size_t ws_bytes,
                              cudaStream_t st);
// Adjoint over the same batch: upstream d_xd (position, splat and shading
// summed), d_cov and d_nd per pose ([.][B G]); d_ag, d_rg, d_pg, d_ubar once
// ([.][G]); d_xd2 must be NULL.  Canonical gradients summed over the poses.
AV_INTERNAL size_t av_skin_batch_backward_workspace_size(const avatar_skin_args *a, int B);
AV_INTERNAL int av_skin_batch_backward(avatar_ctx *ctx, const avatar_skin_args *a, const avatar_skin_grads *g, int B,
                                       const void *fwd_ws, void *ws, size_t ws_bytes, cudaStream_t st);

// (b) B poses: xp [3][B Nv], bits [B Nv][OW].
AV_INTERNAL size_t av_visibility_batch_workspace_size(const avatar_vis_args *a, int B);
AV_INTERNAL int av_visibility_batch(avatar_ctx *ctx, const avatar_vis_args *a, int B, void *ws, size_t ws_bytes,
                                    cudaStream_t st);

// (c) V views of B poses: view v shades pose view_pose[v] from camera
// centre view_cc[v]; xd, nd [3][B G], bits [B Nv][OW], light_L [B][NL][3];
// color, radiance [3][V G], cull [V G]; gradients per view ([.][V G]) except
// d_light_L ([B][NL][3], accumulated: zero it first).
AV_INTERNAL int av_shade_batch(avatar_ctx *ctx, const avatar_shade_args *a, int B, int V, const int32_t *view_pose,
                               const float *view_cc, cudaStream_t st);
AV_INTERNAL int av_shade_batch_backward(avatar_ctx *ctx, const avatar_shade_args *a, const avatar_shade_grads *g,
                                        int B, int V, const int32_t *view_pose, const float *view_cc,
                                        cudaStream_t st);
