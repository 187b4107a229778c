/*
 * avatar.h - C ABI of the GB300 (sm_103a) relit-avatar render path.
 *
 * The per-frame path of "Interactive Rendering of Relightable and Animatable
 * Gaussian Avatars" (arXiv 2407.10707): for a novel pose and environment
 * light, (a) skin the canonical Gaussians and mesh (Sec. 3.1, Eq. 1),
 * (b) compute per-vertex visibility toward D directions by rasterising the
 * posed mesh into depth maps (Sec. 3.2, shadow-mapping form), (c) shade every
 * Gaussian with the discrete rendering equation (Eq. 2, BRDF of App. A), and
 * (d) splat the Gaussians with tile-binned, depth-sorted front-to-back alpha
 * blending (the 3DGS rasteriser of Sec. 3.1).  Backward calls give the
 * adjoints used by the training loop (Sec. 3.3).
 *
 * Conventions shared by every call
 *  - Every pointer is a DEVICE pointer owned by the caller, except where a
 *    field says "host".  Arrays are float32 structure-of-arrays: "[3][G]"
 *    means three contiguous planes of G floats.  Index arrays are int32.
 *  - Calls are asynchronous on the given stream (NULL = legacy default
 *    stream) and never synchronise the device; they allocate no device
 *    memory.  Scratch comes from a caller-provided workspace whose size the
 *    matching *_workspace_size query returns; workspaces must be 256-byte
 *    aligned.
 *  - The return value reports argument errors found on the host and launch
 *    failures.  Errors found on the device (index out of range, pair-buffer
 *    overflow, a bounded wait that expired) are written to the optional
 *    device word `status` (first error wins; the caller zeroes it), so that
 *    calls stay capturable in CUDA graphs.
 *  - Outputs are overwritten, never accumulated, unless a field says so.
 *  - The library is single-GPU: the context binds one device.
 */
#ifndef AVATAR_H
#define AVATAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t; declared opaquely so this header needs no CUDA include. */
typedef struct CUstream_st *avatar_stream_t;

enum avatar_status {
    AVATAR_OK = 0,
    AVATAR_ERR_INVALID_ARG = 1,  /* bad size, NULL pointer, out-of-range value */
    AVATAR_ERR_WORKSPACE = 2,    /* workspace missing, misaligned or too small */
    AVATAR_ERR_OVERFLOW = 3,     /* (tile, Gaussian) pairs exceed pair_capacity */
    AVATAR_ERR_TIMEOUT = 4,      /* a bounded device-side wait expired */
    AVATAR_ERR_CUDA = 5,         /* a CUDA runtime call or launch failed */
    AVATAR_ERR_UNSUPPORTED = 6,  /* device or configuration not supported */
    AVATAR_ERR_INDEX = 7         /* device: an index array entry is out of range */
};

/* Storage type of the learnable per-Gaussian / per-vertex attributes that a
 * struct marks "(attr_dtype)": albedo, roughness, specular tint, opacity,
 * log-scale and rotation.  Positions, displacements, LBS weights and the
 * light stay FP32 (a BF16 position step is ~4 mm at 1 m, a BF16 weight sum
 * is off by up to 2^-9).  All arithmetic is FP32 either way. */
enum avatar_dtype {
    AVATAR_DTYPE_F32 = 0,
    AVATAR_DTYPE_BF16 = 1        /* bfloat16, round-to-nearest-even from FP32 */
};

/* Static English description of a status code; never NULL. */
const char *avatar_status_string(int status);

/* Library version as major*10000 + minor*100 + patch. */
int avatar_version(void);

/* ------------------------------------------------------------------ */
/* Context: binds a device, caches its SM count and tuning choices.     */
/* ------------------------------------------------------------------ */
typedef struct avatar_ctx avatar_ctx;

/* Create a context for CUDA device `device` (host pointer out).  Fails with
 * AVATAR_ERR_UNSUPPORTED on devices other than compute capability 10.3. */
int avatar_ctx_create(avatar_ctx **out, int device);
int avatar_ctx_destroy(avatar_ctx *ctx);
/* Number of streaming multiprocessors of the context's device. */
int avatar_ctx_sm_count(const avatar_ctx *ctx);

/* Tuning knobs of a context (work split only: results do not depend on
 * them).  The library's autotuner (paper_2407_10707_gb300.autotune) times
 * the choices on the actual workload and sets the fastest. */
enum avatar_tune_key {
    AVATAR_TUNE_BLEND_PPT = 0,     /* pixels per thread in the blend: 1, 2 or 4 (default 1) */
    AVATAR_TUNE_BLEND_BWD_PPT = 1, /* pixels per thread in the blend backward: 1, 2 or 4 (default 1) */
    AVATAR_TUNE_BATCH_TILE = 2,    /* tile edge of the batched render when its desc says 0 (default 16) */
    AVATAR_TUNE_VIS_CLUSTER = 3,   /* CTAs per direction of avatar_visibility: 0 (default: 32 KB depth-map
                                      slabs, at most 8), 2, 4 or 8; raised where the slab would not fit */
    AVATAR_TUNE_WAIT_LIMIT = 4,    /* polls of one predecessor's word before a radix-sort look-back wait
                                      (splatting, batched render) gives up: 0 = default (2^22, far beyond
                                      any real wait), or 1..2^30.  A block whose wait expires writes
                                      AVATAR_ERR_TIMEOUT to the status word and counts its offsets from the
                                      earlier keys itself, so the result is unchanged, only slower.  The
                                      tensor-core kernels' completion waits keep their own fixed limit. */
    AVATAR_TUNE_REGION_MASKS = 5,  /* 1 (default): pair keys carry the mask of the tile regions a
                                      Gaussian's ellipse reaches and the blends test it; 0: rect test
                                      alone (the form past 2^24 tiles).  Keep it fixed from a bin to
                                      the blend and backward that use its lists. */
    AVATAR_TUNE_COUNT = 6
};
int avatar_ctx_set_tuning(avatar_ctx *ctx, int key, int value);
/* Current value of a knob, or -1 for an invalid key. */
int avatar_ctx_get_tuning(const avatar_ctx *ctx, int key);

/* ------------------------------------------------------------------ */
/* Pipe throughput probes (the paper has no counterpart): the measured   */
/* denominators of the roofline fractions of arithmetic-bound stages.    */
/* ------------------------------------------------------------------ */
enum avatar_probe_kind {
    AVATAR_PROBE_FFMA = 0,   /* FP32 fused multiply-add (2 flops each) */
    AVATAR_PROBE_IADD3 = 1,  /* three-input INT32 add */
    AVATAR_PROBE_LOP3 = 2,   /* three-input INT32 logic operation */
    AVATAR_PROBE_IMAD = 3    /* INT32 multiply-add */
};
/* Launches one full wave (2,048 threads per SM) in which every thread runs
 * `iters` (>= 1) rounds of 128 operations of `kind` on eight register chains
 * that feed one another (no memory traffic).  The caller times the launch on
 * `stream` (CUDA events) and divides *ops (host, written on success: the
 * operations the launch executes) by the time.  sink: one device uint32 that
 * the kernel writes only in the impossible case its result equals an internal
 * seed.  Errors: AVATAR_ERR_INVALID_ARG for a NULL ctx/sink, iters < 1 or an
 * unknown kind; AVATAR_ERR_CUDA if the launch fails. */
int avatar_probe_alu(avatar_ctx *ctx, int kind, int iters, uint32_t *sink, long long *ops,
                     avatar_stream_t stream);

/* ------------------------------------------------------------------ */
/* Storage order of the Gaussians (a layout step; the paper has no      */
/* counterpart).  The per-Gaussian kernels gather their nearest mesh     */
/* vertices' records; stored in the order of their nearest vertex, the  */
/* 32 Gaussians of a warp share those records.  No result depends on    */
/* the order: reorder every per-Gaussian array of an avatar with the    */
/* same order, once, before rendering.                                   */
/* ------------------------------------------------------------------ */
/* Workspace bytes of avatar_gaussian_order for G Gaussians (0 if G < 0). */
size_t avatar_gaussian_order_workspace_size(int G);
/* order [G] (device, written): the stable order of the Gaussians by their
 * nearest vertex nearest [G] (device; row 0 of the avatar's knn, each in
 * [0, Nv)): order[i] is the i-th Gaussian by (nearest, index).  A nearest
 * index outside [0, Nv) is reported in *status (AVATAR_ERR_INDEX) and sorts
 * as Nv - 1.  Errors: AVATAR_ERR_INVALID_ARG (NULL pointers, G < 0,
 * Nv < 1), AVATAR_ERR_WORKSPACE (missing, misaligned or too small). */
int avatar_gaussian_order(avatar_ctx *ctx, int G, int Nv, const int32_t *nearest, int32_t *order, void *ws,
                          size_t ws_bytes, int32_t *status, avatar_stream_t stream);
/* dst[r][i] = src[r][order[i]] for rows r < rows (<= 65535) of n elements
 * of elem_bytes (2, 4, 8, 12 or 16) bytes each - columns of a
 * structure-of-arrays, or records such as a light's 3 floats - both device
 * arrays [rows][n] aligned to 2 bytes (elem_bytes 2) or 4 (the others) that
 * must not overlap.  An order entry outside [0, n) is reported in *status
 * (AVATAR_ERR_INDEX) and writes zeros.  Errors: AVATAR_ERR_INVALID_ARG. */
int avatar_gather_columns(avatar_ctx *ctx, int rows, int n, int elem_bytes, const void *src, void *dst,
                          const int32_t *order, int32_t *status, avatar_stream_t stream);

/* ------------------------------------------------------------------ */
/* (a) Skinning - Sec. 3.1, Eq. 1                                       */
/*                                                                      */
/* Forward kinematics: bone_j = T_j * translate(-J_j) with               */
/*   T_j = T_parent(j) * [Rodrigues(pose_j) | J_j - J_parent(j)].         */
/* Vertices: A_v = sum_k w_vk bone_k, xp_v = A_v (x_v + dx_v).            */
/* Gaussians (Eq. 1): u_j = 1/max(|x_g - x_j|, 1e-8) over the K nearest   */
/*   vertices, ubar = u / sum u, *_g = sum_j ubar_j *_j for albedo,       */
/*   roughness, specular tint, normal, LBS weights and displacement;      */
/*   xbar = x_g + dx_g; A_g = sum_k w_gk bone_k (= sum_j ubar_j A_j);     */
/*   x_gd = A_g xbar; Sigma_gd = M Sigma M^T with Sigma = R(q) S^2 R(q)^T,*/
/*   S = diag(exp(logscale)); n_gd = normalize(M normalize(n_g)), M the   */
/*   linear part of A_g.                                                  */
/* ------------------------------------------------------------------ */
typedef struct {
    int G;                 /* Gaussians (>= 0) */
    int Nv;                /* mesh vertices (>= 1) */
    int K;                 /* neighbours per Gaussian, 1..8 (paper: 3) */
    int J;                 /* joints, 1..64 (SMPL: 24) */
    /* canonical Gaussians */
    const float *xg;       /* [3][G] positions */
    const void *logscale;  /* [3][G] log of the three axis scales (attr_dtype) */
    const void *quat;      /* [4][G] rotation quaternion (w,x,y,z), any norm > 0 (attr_dtype) */
    const int32_t *knn;    /* [K][G] indices of the K nearest vertices (S_g) */
    /* canonical mesh attributes */
    const float *xv;       /* [3][Nv] positions */
    const float *dxv;      /* [3][Nv] displacement, or NULL for zero */
    const float *wv;       /* [Nv][J] LBS weights, vertex-major */
    const void *av;        /* [3][Nv] albedo (attr_dtype) */
    const void *rv;        /* [Nv] roughness (attr_dtype) */
    const void *pv;        /* [Nv] specular tint (attr_dtype) */
    const float *nv;       /* [3][Nv] normals */
    /* skeleton */
    const int32_t *parents; /* [J] parent index, parents[j] < j, root -1 */
    const float *joints;   /* [J][3] rest joint positions */
    const float *pose;     /* [J][3] axis-angle joint rotations */
    /* outputs */
    float *bone;           /* [J][12] bone transforms, row-major 3x4 */
    float *xp;             /* [3][Nv] posed vertices */
    float *xd;             /* [3][G] posed Gaussian positions x_gd */
    float *cov;            /* [6][G] posed covariance (xx,xy,xz,yy,yz,zz) */
    float *nd;             /* [3][G] posed unit normals n_gd */
    float *ag;             /* [3][G] albedo */
    float *rg;             /* [G] roughness */
    float *pg;             /* [G] specular tint */
    float *ubar;           /* [K][G] normalised Eq. 1 weights */
    int32_t *status;       /* optional device status word */
    int attr_dtype;        /* storage of the (attr_dtype) inputs: AVATAR_DTYPE_F32 or _BF16 */
} avatar_skin_args;

/* Workspace for avatar_skin: per-vertex packed records (Nv*112 bytes).
 * avatar_skin_backward reads the records the forward left there, so keep
 * the workspace intact between the two calls. */
size_t avatar_skin_workspace_size(const avatar_skin_args *a);
int avatar_skin(avatar_ctx *ctx, const avatar_skin_args *a, void *ws, size_t ws_bytes,
                avatar_stream_t stream);

typedef struct {
    /* upstream gradients ([.][G]); NULL = zero.  d_xd2 is a second upstream
     * gradient of x_gd (splatting and shading both reach x_gd); it is added
     * to d_xd. */
    const float *d_xd, *d_cov, *d_nd, *d_ag, *d_rg, *d_pg, *d_ubar, *d_xd2;
    /* gradients written ([.][G] and [.][Nv]); NULL = not wanted */
    float *d_xg;           /* [3][G] */
    float *d_logscale;     /* [3][G] */
    float *d_quat;         /* [4][G] */
    float *d_wv;           /* [Nv][J] */
    float *d_av;           /* [3][Nv] */
    float *d_rv;           /* [Nv] */
    float *d_pv;           /* [Nv] */
    float *d_dxv;          /* [3][Nv] */
} avatar_skin_grads;

/* Backward workspace (per-vertex accumulators), disjoint from the forward's. */
size_t avatar_skin_backward_workspace_size(const avatar_skin_args *a);
int avatar_skin_backward(avatar_ctx *ctx, const avatar_skin_args *a, const avatar_skin_grads *g,
                         const void *fwd_ws, void *ws, size_t ws_bytes, avatar_stream_t stream);

/* ------------------------------------------------------------------ */
/* Nearest neighbours - the sets S_g of Eq. 1 (the K_g nearest mesh     */
/* vertices of each Gaussian, Sec. 3.1) and S_v of the visibility        */
/* filters (Sec. 3.2), recomputed on the device when the canonical      */
/* positions change (rebinding).                                        */
/*                                                                      */
/* knn[k][i] = the index of the k-th nearest reference point of query   */
/* point i, ascending (squared distance, index), where the squared      */
/* distance is the FP64 value of (d0 d0 + d1 d1) + d2 d2 of the FP32     */
/* coordinates, every operation rounded to nearest: the result is that  */
/* definition's exactly.  A uniform grid over the reference points and  */
/* one thread per query point searching shells of cells.                */
/* ------------------------------------------------------------------ */
typedef struct {
    int N;                 /* query points (>= 0) */
    int M;                 /* reference points (>= K) */
    int K;                 /* neighbours, 1..32 */
    const float *x;        /* [3][N] query points */
    const float *ref;      /* [3][M] reference points */
    int32_t *knn;          /* [K][N] output indices */
    float *dist2;          /* [K][N] optional output: the squared distances (rounded to FP32) */
    int32_t *status;       /* optional device status word */
} avatar_knn_args;

size_t avatar_knn_workspace_size(const avatar_knn_args *a);
int avatar_knn(avatar_ctx *ctx, const avatar_knn_args *a, void *ws, size_t ws_bytes, avatar_stream_t stream);

/* ------------------------------------------------------------------ */
/* (b) Visibility - Sec. 3.2, depth-map (shadow-mapping) form.          */
/*                                                                      */
/* Exact integer rules (any correct implementation gives the same bits):*/
/*  q = rint(x*2^13) - rint(center*2^13), |q_i| < 2^16                    */
/*  B = rint(frame*2^13); s = e1.q, t = e2.q; zd = floor(-(w.q)/2^10)     */
/*  H = rint(half_extent*2^26) with 16R < H <= 2^30; M = floor(R 2^35/H)  */
/*  X = floor((s+H) M / 2^32), Y from t: 1/16-pixel units, in the window  */
/*  iff 0 <= X,Y < 16R.  Triangles with a vertex outside the window or    */
/*  zero area are skipped; a triangle (either winding) covers pixel (i,j) */
/*  iff its three edge functions at (16i+8, 16j+8) are >= 0; its depth    */
/*  there is floor(sum w_i zd_i / area); the depth map keeps the minimum. */
/*  bit(v,d) = 1 iff v is outside the window, its pixel is empty, or      */
/*  zd_v <= depth[pixel(v)] + rint(bias*2^16).                            */
/* (cull_back = 1 keeps only triangles of positive area, see the field.) */
/* The faces are rasterised in chunks of AVATAR_VIS_FACE_CHUNK in array  */
/* order; the bits do not depend on the order of the faces, and an order  */
/* that permutes faces only within these chunks keeps every chunk's       */
/* vertex range (a chunk's vertices are projected once into a cache).     */
/* Output bit layout: vertex-major words.  With dmap == NULL the word     */
/* index is d>>5 over the D viewpoints ([Nv][D/32]); with a light->view   */
/* map dmap[NL] the bits are re-ordered per light: bit k of vertex v is  */
/* bit(v, dmap[k]) in words [Nv][ceil(NL/32)] (the form avatar_shade     */
/* reads).                                                              */
/* ------------------------------------------------------------------ */
enum { AVATAR_VIS_FACE_CHUNK = 1024 };

typedef struct {
    int Nv;                /* vertices */
    int F;                 /* triangles */
    int D;                 /* viewpoints, multiple of 32, <= 4096 */
    int R;                 /* depth-map resolution, 8..512 */
    const float *xp;       /* [3][Nv] posed vertices */
    const int32_t *faces;  /* [F][3] vertex indices */
    const float *frames;   /* [D][9] unit rows e1, e2, w (w points toward the light) */
    float center[3];       /* host value: window centre (world) */
    float half_extent;     /* host value: window half width (world) */
    float bias;            /* host value: depth bias (world units) */
    int NL;                /* lights for the re-ordered output (0: none) */
    const int32_t *dmap;   /* [NL] light -> viewpoint, or NULL */
    uint32_t *bits;        /* output, layout above */
    int32_t *status;       /* optional device status word */
    int cull_back;         /* host value: 0 = two-sided (the rules above); 1 = rasterise only
                            * triangles whose integer area (a->b->c) is positive, i.e. that face
                            * the light for outward winding.  For closed, consistently outward-
                            * wound meshes both give identical bits (the nearest surface along
                            * any ray toward the light faces it); 1 does about half the work. */
} avatar_vis_args;

size_t avatar_visibility_workspace_size(const avatar_vis_args *a);
int avatar_visibility(avatar_ctx *ctx, const avatar_vis_args *a, void *ws, size_t ws_bytes,
                      avatar_stream_t stream);

/* avatar_visibility without a caller workspace.  (The paper has no
 * counterpart: this is a convenience of this library.)  It is meant for
 * callers that cannot allocate device memory: code inside a host application
 * whose framework owns every device allocation, or a real-time loop where a
 * cudaMalloc (which may synchronise the device) is not allowed.  The caller
 * still passes all inputs and the output `bits`; the scratch is a fixed
 * array of avatar_visibility_static_scratch_bytes() (8 MiB) compiled into the
 * library, which every GPU that loads the library keeps until the process
 * exits.
 *  - Sizes whose workspace (avatar_visibility_workspace_size) exceeds that
 *    array are rejected with AVATAR_ERR_WORKSPACE before any launch.
 *  - The first call on a device looks up the array's device address (with the
 *    context's device made current for the lookup); make that first call
 *    before any stream capture on the device.  A call that finds the device's
 *    CUDA context replaced (after cudaDeviceReset, say) looks it up again.
 *  - All calls on a device share the one array and it keeps the previous
 *    call's contents: calls that may overlap on the GPU (different streams
 *    without ordering) race on it and must be serialised by the caller.
 *  - Results are identical to avatar_visibility; the function allocates
 *    nothing. */
size_t avatar_visibility_static_scratch_bytes(void);
int avatar_visibility_static_scratch(avatar_ctx *ctx, const avatar_vis_args *a, avatar_stream_t stream);

/* ------------------------------------------------------------------ */
/* (b') The paper's own visibility - Sec. 3.2, Eqs. 3-4                 */
/*                                                                      */
/* Per direction d, with the projection, window and coverage rules of   */
/* avatar_visibility: a triangle appears in the triangle-ID image iff   */
/* at some pixel it covers its depth is the least depth there (every    */
/* tied triangle appears), and V^d[v] = 1 iff a triangle incident to v  */
/* appears (or v lies outside the window).  Then                        */
/* Vbar^d = mean(median(median(V^d))), both filters                     */
/* over S_v, the Kv nearest vertices of v (v itself included): the      */
/* median of Kv binary values (Kv odd) is 1 iff at least (Kv+1)/2 are 1 */
/* and the mean is their count / Kv.  Output: the count Kv * Vbar, an   */
/* integer in 0..Kv, per vertex and light (light k uses direction       */
/* base.dmap[k], or direction k when base.dmap is NULL) - every step is */
/* integer, so the result is bit-exact.  One cluster of CTAs per         */
/* direction holds the depth map and a vertex bitmap in shared memory;  */
/* AVATAR_ERR_UNSUPPORTED when they do not fit (very large Nv).          */
/* A bad neighbour index is reported (AVATAR_ERR_INDEX) and skipped.    */
/* ------------------------------------------------------------------ */
typedef struct {
    avatar_vis_args base;  /* geometry as for avatar_visibility (bias unused); base.bits, if not
                              NULL, receives the unfiltered V, [Nv][D/32] in direction order */
    int Kv;                /* filter neighbourhood, odd, 1..63 (paper: 19) */
    const int32_t *knn_v;  /* [Kv][Nv] nearest vertices of each vertex */
    uint8_t *vis_count;    /* [Nv][NL] output (NL = base.NL, or D when base.dmap is NULL) */
} avatar_vis_soft_args;

size_t avatar_visibility_soft_workspace_size(const avatar_vis_soft_args *a);
int avatar_visibility_soft(avatar_ctx *ctx, const avatar_vis_soft_args *a, void *ws, size_t ws_bytes,
                           avatar_stream_t stream);

/* ------------------------------------------------------------------ */
/* (c) Shading - Eq. 2 with the BRDF of App. A, cull and gamma (Sec 3.1)*/
/*                                                                      */
/* cull: with d = C - x_gd (FP32), culled iff !(fma(n2,d2,fma(n1,d1,     */
/*   n0*d0)) > 0); culled Gaussians get colour 0 and are not splatted.   */
/* Otherwise, w_o = normalize(C - x_gd), c_o = max(n.w_o, 0), and over   */
/* lights k with c_i = n.w_k > 0:                                       */
/*   vis = sum_j ubar_j bit(S_j, k)                                      */
/*   f_s = D F / (4 (c_i(1-kk)+kk)(c_o(1-kk)+kk)),  alpha = gamma^2,      */
/*   kk = (gamma+1)^2/8, D = alpha^2/(pi((n.h)^2(alpha^2-1)+1)^2),       */
/*   F = 0.04 + 0.96*2^((-5.55473 w_o.h - 6.98316) w_o.h)                */
/*   L_o += L_k A_k vis c_i (a/pi + p f_s)                               */
/* colour = max(L_o, 1e-6)^(1/2.2).                                      */
/* Bits are light-ordered ([Nv][ceil(NL/32)], see avatar_visibility).   */
/* ------------------------------------------------------------------ */
typedef struct {
    int G, K, NL, Nv;
    const float *xd, *nd, *ag, *rg, *pg; /* skinning outputs */
    const float *ubar;     /* [K][G] */
    const int32_t *knn;    /* [K][G] */
    const uint32_t *bits;  /* [Nv][ceil(NL/32)] light-ordered visibility */
    const float *light_L;  /* [NL][3] radiance */
    const float *light_A;  /* [NL] solid angle */
    const float *light_w;  /* [NL][3] unit direction toward the light */
    float cam_center[3];   /* host value: camera centre (world) */
    float *color;          /* [3][G] output shading colour */
    float *radiance;       /* [3][G] output L_o before gamma (read by the backward) */
    uint8_t *cull;         /* [G] output, 1 = back-facing */
    int32_t *status;
    /* optional soft visibility of the paper's filters (avatar_visibility_soft):
     * when not NULL it replaces bits, vis = sum_j ubar_j vis_count[S_j][k] / vis_den */
    const uint8_t *vis_count; /* [Nv][NL] light order */
    int vis_den;           /* Kv of the filters, >= 1 */
} avatar_shade_args;

int avatar_shade(avatar_ctx *ctx, const avatar_shade_args *a, avatar_stream_t stream);

/* The cull flags of avatar_shade alone (the same FP32 rule on xd, nd and
 * cam_center; reads nothing else and writes only a->cull[G]): splatting
 * needs them before shading ends, so a caller can project and bin on one
 * stream while visibility and shading run on another.  For valid inputs the
 * flags equal the ones avatar_shade writes. */
int avatar_cull(avatar_ctx *ctx, const avatar_shade_args *a, avatar_stream_t stream);

/* Relighting under many environment lights at once (the relighting use of
 * Sec. 3.5 applied to Eq. 2): every light l shares the texel geometry of
 * `base` (light_w, light_A) and has its own radiance env_L[l].  Because the
 * sums of Eq. 2 are linear in the radiance,
 *   L_o[g,(l,c)] = a_gc/pi (D B)[g,(l,c)] + p_g (S B)[g,(l,c)],
 *   D = vis * max(0, n.w_k), S = D * f_s, B[k,(l,c)] = L^(l)_kc A_k,
 * which this call evaluates on the tensor cores (tcgen05, BF16 operands,
 * FP32 accumulation in TMEM); D and S are rounded to BF16 (relative error
 * 2^-9 per term).  Colours follow avatar_shade (gamma 2.2, culled -> 0);
 * `base.light_L` and `base.color` are not used, `base.cull` is written, and
 * with n_env == 1 a non-null `base.radiance` receives L_o before gamma (so
 * avatar_shade_backward can follow this call in a training step).
 * A first pass writes the culled colours and lists the live Gaussians in
 * the workspace, so the tensor-core tiles hold live rows only.
 * Requires NL a multiple of 64 and at most 2048, 1 <= n_env <= 32, and the
 * resident light matrix (3 n_env rounded up to 16, times NL, BF16) plus 64 KB
 * of tiles and 16 B per light within the shared memory of one SM;
 * otherwise AVATAR_ERR_UNSUPPORTED / AVATAR_ERR_INVALID_ARG. */
typedef struct {
    avatar_shade_args base;
    int n_env;             /* number of environment lights */
    const float *env_L;    /* [n_env][NL][3] radiance of each light */
    float *env_color;      /* [n_env][3][G] output colours */
    void *workspace;       /* device scratch, avatar_shade_multi_workspace_size bytes */
    size_t workspace_bytes;
} avatar_shade_multi_args;

/* Workspace bytes for avatar_shade_multi (depends on base.G only). */
size_t avatar_shade_multi_workspace_size(const avatar_shade_multi_args *a);
int avatar_shade_multi(avatar_ctx *ctx, const avatar_shade_multi_args *a, avatar_stream_t stream);

typedef struct {
    const float *d_color;  /* [3][G] upstream */
    float *d_xd;           /* [3][G] written (through w_o) */
    float *d_nd;           /* [3][G] written */
    float *d_ag;           /* [3][G] written */
    float *d_rg;           /* [G] written */
    float *d_pg;           /* [G] written */
    float *d_ubar;         /* [K][G] written (through vis) */
    float *d_light_L;      /* [NL][3] written */
} avatar_shade_grads;

int avatar_shade_backward(avatar_ctx *ctx, const avatar_shade_args *a, const avatar_shade_grads *g,
                          avatar_stream_t stream);

/* ------------------------------------------------------------------ */
/* (d) Splatting - the 3DGS rasteriser of Sec. 3.1, black background    */
/*                                                                      */
/* project: p = R x + t; valid iff not culled, p.z > 0.2, o > 1/255 and  */
/*   det > 0; mean = (fx p.x/p.z + cx, fy p.y/p.z + cy); Sigma' = T Sigma */
/*   T^T + 0.3 I with T = J R (EWA); conic = inverse(Sigma');            */
/*   rect = pixels whose centre (i+1/2) lies in the AABB of the ellipse   */
/*   q <= 2 ln(255 o) padded by 1 pixel (tile-size independent).         */
/* bin: one pair per tile that g's rect meets (num_pairs counts them);  */
/*   a tile's list holds the pairs whose ellipse q <= 2 ln(255 o) comes  */
/*   within one pixel of the tile (the others cannot reach its pixels),  */
/*   ordered by (depth bits, g) - a stable device radix sort.            */
/* blend: per pixel centre, front to back: alpha = min(0.99, o e^{-q/2}),*/
/*   skip alpha < 1/255, stop before T(1-alpha) < 1e-4, C += c alpha T.   */
/* ------------------------------------------------------------------ */
typedef struct {
    float fx, fy, cx, cy;  /* pinhole intrinsics (pixels) */
    float R[9];            /* world->camera rotation, row-major (x right, y down, z forward) */
    float t[3];            /* world->camera translation */
    int width, height;     /* image size, 1..16384 */
} avatar_camera;

typedef struct {
    int G;
    avatar_camera cam;     /* host value */
    int tile;              /* tile edge: 8, 16 or 32 pixels; 0 = 16 */
    const float *xd;       /* [3][G] */
    const float *cov;      /* [6][G] */
    const void *opacity;   /* [G] (attr_dtype) */
    const float *color;    /* [3][G] */
    const uint8_t *cull;   /* [G] or NULL */
    /* per-Gaussian projection (written by project) */
    float *mean2d;         /* [2][G] */
    float *conic;          /* [3][G] (a, b, c): q = a dx^2 + 2 b dx dy + c dy^2 */
    float *depth;          /* [G] camera-space z */
    int32_t *rect;         /* [4][G] inclusive pixel rect x0,y0,x1,y1 (x0 > x1: empty) */
    /* binning (written by bin) */
    int32_t *tile_range;   /* [ntiles][2] begin, end into pair_gauss */
    int32_t *pair_gauss;   /* [pair_capacity] Gaussian index of each sorted pair */
    int64_t pair_capacity; /* capacity of pair_gauss, >= 1 */
    int32_t *num_pairs;    /* [1] pairs emitted, listed or not (the required capacity on overflow) */
    /* image (written by blend) */
    float *image;          /* [3][H][W] */
    float *T_final;        /* [H][W] final transmittance */
    int32_t *n_last;       /* [H][W] list positions traversed up to the last contributor */
    int32_t *status;
    int attr_dtype;        /* storage of opacity: AVATAR_DTYPE_F32 or _BF16 */
} avatar_splat_args;

/* ntiles = ceil(W/tile) * ceil(H/tile). */
int avatar_splat_num_tiles(const avatar_splat_args *a);
/* Workspace shared by all splat calls of one frame; keep it intact from
 * avatar_splat to avatar_splat_backward. */
size_t avatar_splat_workspace_size(const avatar_splat_args *a);
/* The three steps, and all three in order.  project reads xd, cov, opacity
 * and cull; bin reads the projection buffers and opacity; only blend reads
 * color (it completes the per-Gaussian blend records), so project and bin
 * may run before shading has finished.  bin also leaves in the workspace the
 * order in which blend and the backward visit the tiles (longest lists
 * first); the image does not depend on it. */
int avatar_splat_project(avatar_ctx *ctx, const avatar_splat_args *a, void *ws, size_t ws_bytes,
                         avatar_stream_t stream);
int avatar_splat_bin(avatar_ctx *ctx, const avatar_splat_args *a, void *ws, size_t ws_bytes,
                     avatar_stream_t stream);
int avatar_splat_blend(avatar_ctx *ctx, const avatar_splat_args *a, void *ws, size_t ws_bytes,
                       avatar_stream_t stream);
int avatar_splat(avatar_ctx *ctx, const avatar_splat_args *a, void *ws, size_t ws_bytes,
                 avatar_stream_t stream);

typedef struct {
    const float *d_image;  /* [3][H][W] upstream */
    float *d_xd;           /* [3][G] written */
    float *d_cov;          /* [6][G] written */
    float *d_opacity;      /* [G] written */
    float *d_color;        /* [3][G] written */
} avatar_splat_grads;

int avatar_splat_backward(avatar_ctx *ctx, const avatar_splat_args *a, const avatar_splat_grads *g,
                          void *ws, size_t ws_bytes, avatar_stream_t stream);

/* ------------------------------------------------------------------ */
/* Batching: many poses, cameras and lights in one launch per step      */
/*                                                                      */
/* B poses of one avatar, each with its own environment light (Sec. 3.5 */
/* relighting under novel poses), seen by V cameras of any resolution.  */
/* Every stage runs once over the whole batch: skinning and visibility  */
/* over the poses, shading and projection over the views, one depth     */
/* sort and one tile sort over all views' Gaussians and pairs, and one  */
/* persistent blend whose CTAs take tiles of every view from a shared   */
/* counter (uneven resolutions and Gaussian-per-tile loads balance on   */
/* the device).  The calls are asynchronous and capturable in a CUDA    */
/* graph; each view's image equals what the per-frame calls produce.    */
/* ------------------------------------------------------------------ */
#define AVATAR_BATCH_MAX_VIEWS 4096

typedef struct {
    avatar_camera cam;     /* host value */
    int pose;              /* pose shown, 0..B-1 */
    float center[3];       /* host value: camera centre (world), the w_o origin of Eq. 2 */
} avatar_view;

typedef struct {
    /* the canonical avatar: G, Nv, K, J, the canonical arrays and
     * attr_dtype as in avatar_skin_args (its pose, outputs and status are
     * not used) */
    avatar_skin_args avatar;
    const void *opacity;   /* [G] (avatar.attr_dtype) */
    /* mesh and visibility geometry, as in avatar_vis_args */
    int F;
    const int32_t *faces;  /* [F][3] */
    int D, R;              /* viewpoints (multiple of 32), depth-map resolution */
    const float *frames;   /* [D][9] */
    float center[3];       /* host value */
    float half_extent;     /* host value */
    float bias;            /* host value */
    int cull_back;         /* host value, as in avatar_vis_args */
    /* light texels shared by every pose (Eq. 2) */
    int NL;
    const float *light_A;  /* [NL] */
    const float *light_w;  /* [NL][3] */
    const int32_t *dmap;   /* [NL] light -> viewpoint */
    /* the batch */
    int B;                 /* poses, 1..65535 */
    const float *poses;    /* [B][J][3] axis-angle */
    const float *light_L;  /* [B][NL][3] each pose's environment light */
    int V;                 /* views, 1..AVATAR_BATCH_MAX_VIEWS */
    const avatar_view *views; /* host array [V] */
    int tile;              /* 8, 16, 32, or 0 = the context's tuned tile (16 until tuned) */
    int64_t pair_capacity; /* (tile, Gaussian) pairs over all views, 1..2^31-1 */
    float *images;         /* output: the views' [3][H][W] images back to back in view order */
    int32_t *num_pairs;    /* [1] output: pairs over all views (required capacity on overflow) */
    int32_t *status;       /* optional device status word */
} avatar_batch_desc;

/* Workspace of the batched forward and backward (one buffer serves both;
 * keep it between the two calls).  0 on invalid sizes. */
size_t avatar_render_batch_workspace_size(const avatar_batch_desc *d);
int avatar_render_batch(avatar_ctx *ctx, const avatar_batch_desc *d, void *ws, size_t ws_bytes,
                        avatar_stream_t stream);

typedef struct {
    const float *d_images; /* upstream, laid out like images */
    /* outputs, FP32 whatever the storage type, summed over the batch */
    float *d_xg;           /* [3][G] */
    float *d_logscale;     /* [3][G] */
    float *d_quat;         /* [4][G] */
    float *d_opacity;      /* [G] */
    float *d_wv;           /* [Nv][J] */
    float *d_av;           /* [3][Nv] */
    float *d_rv;           /* [Nv] */
    float *d_pv;           /* [Nv] */
    float *d_light_L;      /* [B][NL][3] */
} avatar_batch_grads;

/* Adjoint of the last avatar_render_batch on the same workspace. */
int avatar_render_batch_backward(avatar_ctx *ctx, const avatar_batch_desc *d, const avatar_batch_grads *g,
                                 void *ws, size_t ws_bytes, avatar_stream_t stream);

/* Autotuner: times the batch on this GPU for each tile edge (8, 16, 32)
 * and each blend work split (pixels per thread, forward and backward, with
 * g non-NULL), keeps the fastest in the context (used when d->tile == 0
 * and by the per-frame blend) and writes the choices to tuned[3] =
 * {tile, blend pixels per thread, backward pixels per thread} if non-NULL.
 * Synchronous: it waits for the stream, so it must not run during graph
 * capture (AVATAR_ERR_INVALID_ARG).  Candidates whose pairs overflow
 * pair_capacity are skipped. */
int avatar_render_batch_autotune(avatar_ctx *ctx, const avatar_batch_desc *d, const avatar_batch_grads *g,
                                 void *ws, size_t ws_bytes, avatar_stream_t stream, int *tuned);

/* ------------------------------------------------------------------ */
/* Regularisers of Sec. 3.3 (the terms of Eq. 6 beside the image loss): */
/*   L_smooth = sum_i sum_{k in S_v^i} |a_i - a_k|_1 + |gamma_i -        */
/*              gamma_k| + |p_i - p_k|      (vertex materials)          */
/*   L_mdist  = sum_i sum_{k in S_g^i} || x_g^i - x_v^k ||_2             */
/*   L_disp   = sum_i || dx^i ||_2                                      */
/*   L_scale  = sum_i sum_c max(0, exp(logscale_ic) - s0)               */
/* loss (+)= w_smooth L_smooth + w_mdist L_mdist + w_disp L_disp +       */
/* w_scale L_scale (paper: 0.002, 0.1, 0.02, 10; s0 = 0.005).  The       */
/* gradients are ADDED to the given buffers (NULL: not wanted), so the  */
/* call follows the image-loss backward in a training step.  Subgradient */
/* 0 where a difference or a norm is 0.  Sums reduced in FP64.          */
/* ------------------------------------------------------------------ */
typedef struct {
    int G, Nv;             /* Gaussians, vertices */
    int Kg, Kv;            /* |S_g| (0..64), |S_v| (0..64) */
    const float *xg;       /* [3][G] canonical Gaussian positions */
    const void *logscale;  /* [3][G] (attr_dtype) */
    const int32_t *knn;    /* [Kg][G] S_g */
    const float *xv;       /* [3][Nv] canonical vertices */
    const void *av;        /* [3][Nv] albedo (attr_dtype) */
    const void *rv;        /* [Nv] roughness (attr_dtype) */
    const void *pv;        /* [Nv] specular tint (attr_dtype) */
    const int32_t *knn_v;  /* [Kv][Nv] S_v */
    const float *dxv;      /* [3][Nv] displacement, or NULL (no displacement term) */
    int attr_dtype;        /* AVATAR_DTYPE_F32 or _BF16 */
    float w_smooth, w_mdist, w_disp, w_scale;
    float s0;              /* scale threshold */
    int accumulate;        /* 0: *loss = total;  1: *loss += total */
    float *loss;           /* [1] device, or NULL */
    float *terms;          /* [4] device output of the unweighted sums (smooth, mdist, disp, scale), or NULL */
    float *d_xg, *d_logscale, *d_av, *d_rv, *d_pv, *d_dxv;  /* FP32 gradients, accumulated */
    int32_t *status;
} avatar_reg_args;

size_t avatar_regularizers_workspace_size(const avatar_reg_args *a);
int avatar_regularizers(avatar_ctx *ctx, const avatar_reg_args *a, void *ws, size_t ws_bytes,
                        avatar_stream_t stream);

/* ------------------------------------------------------------------ */
/* Pose-dependent displacement MLP (Sec. 3.1; design in Sec. 4: four    */
/* layers of width 256, ReLU, random Fourier features):                 */
/*   gamma(x) = [sin(2 pi B x), cos(2 pi B x)]     B: [64][3]            */
/*   h1 = relu(W1 [gamma(x); theta] + b1)          W1: [256][128 + P]    */
/*   h2 = relu(W2 h1 + b2),  h3 = relu(W3 h2 + b3) W2, W3: [256][256]    */
/*   dx = W4 h3 + b4                               W4: [3][256]          */
/* With T poses the output is the mean over them,                      */
/*   dx = (1/T) sum_t d(x, theta_t),                                    */
/* the average displacement over the training poses that replaces the   */
/* per-pose displacement when rendering novel poses (Sec. 4); T = 1 is  */
/* the displacement at one pose.  On the tensor cores with BF16         */
/* operands and FP32 accumulation: the features, the hidden activations */
/* and W1's feature part, W2, W3, W4 are rounded to bfloat16 (nearest   */
/* even); theta's part of layer 1, the biases and the mean stay FP32     */
/* (the mean sums the poses in order, deterministic).  All arrays are   */
/* FP32, row-major as shown.  The workspace (avatar_mlp_workspace_size, */
/* 256-byte aligned) receives the packed BF16 weights and the poses'    */
/* layer-1 biases on every call.  Asynchronous on the stream; an        */
/* accelerator wait that runs out sets AVATAR_ERR_TIMEOUT in *status.   */
/* ------------------------------------------------------------------ */
typedef struct {
    int N;                 /* points (0 allowed) */
    int P;                 /* pose dimensions, 0..128 */
    int T;                 /* poses, >= 1 */
    const float *x;        /* [3][N] points (canonical vertices) */
    const float *theta;    /* [T][P] poses */
    const float *Bf;       /* [64][3] Fourier frequencies */
    const float *W1, *b1;  /* [256][128 + P], [256] */
    const float *W2, *b2;  /* [256][256], [256] */
    const float *W3, *b3;  /* [256][256], [256] */
    const float *W4, *b4;  /* [3][256], [3] */
    float *dx;             /* [3][N] output */
    int32_t *status;       /* device status word, or NULL */
} avatar_mlp_args;

size_t avatar_mlp_workspace_size(const avatar_mlp_args *a);
int avatar_mlp(avatar_ctx *ctx, const avatar_mlp_args *a, void *ws, size_t ws_bytes, avatar_stream_t stream);

/* ------------------------------------------------------------------ */
/* Density-based densification (App. B, Alg. 1): positions of Gaussians */
/* to add on under-covered mesh triangles.                              */
/*   D_v[k] = number of Gaussians with k among their K_g nearest (S_g)   */
/*   d_f    = (D_v[a] + D_v[b] + D_v[c]) / (6 K_g) per triangle (a,b,c)  */
/*   P_f    = max(0, d0 - d_f),  N' = floor(p0 sum P)                    */
/*   N' draws of a triangle with probability P_f / sum P, each placed    */
/*   uniformly on its triangle of the canonical mesh.                   */
/* Exact form: d0 6 K_g must be an integer (paper: d0 = 1); the weights */
/* w_f = max(0, d0 6 K_g - S_f) are integers, W = sum w_f, and          */
/* N' = floor((p0 W) / (6 K_g)) in IEEE FP64 in that order.  Draw j uses */
/* three caller-supplied uniform words (rand, [3][capacity]): its       */
/* triangle is the smallest f whose inclusive prefix sum of w exceeds    */
/* floor(rand[0][j] W / 2^32); u = (rand[1][j] >> 8) 2^-24, v likewise  */
/* from rand[2][j], (u, v) -> (1 - u, 1 - v) when u + v > 1 (decided    */
/* exactly), x = a + u (b - a) + v (c - a).  *count receives N'; when it */
/* exceeds capacity only the first capacity draws are written and       */
/* AVATAR_ERR_OVERFLOW is set in *status.  An out-of-range index in knn */
/* or faces sets AVATAR_ERR_INDEX and is skipped.  Asynchronous; no     */
/* host synchronisation (the count stays on the device).                 */
/* ------------------------------------------------------------------ */
typedef struct {
    int G, Nv, F;          /* Gaussians (>= 0), vertices, triangles (>= 1) */
    int Kg;                /* |S_g|, 1..64 (paper: 3) */
    const int32_t *knn;    /* [Kg][G] S_g */
    const int32_t *faces;  /* [F][3] */
    const float *xv;       /* [3][Nv] canonical vertices */
    float d0;              /* density threshold (paper: 1) */
    double p0;             /* fraction of sum P added per call (paper: 0.02) */
    int capacity;          /* columns of rand, tri and x */
    const uint32_t *rand;  /* [3][capacity] uniform 32-bit words */
    int32_t *count;        /* [1] device: N' */
    int32_t *tri;          /* [capacity] triangle of each added Gaussian (draw order) */
    float *x;              /* [3][capacity] canonical positions of the added Gaussians */
    int32_t *Dv;           /* [Nv] D_v, or NULL (kept in the workspace) */
    float *df;             /* [F] d_f, or NULL */
    int32_t *ng;           /* [F] draws per triangle (the multinomial sample), or NULL */
    int32_t *status;       /* device status word, or NULL */
} avatar_densify_args;

size_t avatar_densify_workspace_size(const avatar_densify_args *a);
int avatar_densify(avatar_ctx *ctx, const avatar_densify_args *a, void *ws, size_t ws_bytes,
                   avatar_stream_t stream);

/* ------------------------------------------------------------------ */
/* Adam update of the trainable parameters (Kingma and Ba; the          */
/* optimiser of the 3DGS training the paper follows, which states no    */
/* update rule of its own).  Step t (>= 1) of every group in one launch: */
/*   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2                   */
/*   p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)         */
/* in FP32; a BF16 parameter is updated in FP32 and rounded back to      */
/* nearest even.  m and v (FP32, zero before step 1) and p are updated   */
/* in place.  Asynchronous; capturable.                                  */
/* ------------------------------------------------------------------ */
#define AVATAR_ADAM_MAX_GROUPS 16

typedef struct {
    int64_t n;             /* elements */
    void *param;           /* [n] AVATAR_DTYPE_F32 or _BF16 (dtype) */
    int dtype;
    const float *grad;     /* [n] */
    float *m, *v;          /* [n] moments */
    float lr;              /* learning rate of the group */
} avatar_adam_group;

typedef struct {
    int n_groups;          /* 0..AVATAR_ADAM_MAX_GROUPS */
    avatar_adam_group group[AVATAR_ADAM_MAX_GROUPS];
    float beta1, beta2, eps;  /* 3DGS: 0.9, 0.999, 1e-15 */
    int step;              /* t >= 1 */
} avatar_adam_args;

int avatar_adam(avatar_ctx *ctx, const avatar_adam_args *a, avatar_stream_t stream);

/* ------------------------------------------------------------------ */
/* Image loss of Eq. 5 (Sec. 3.3), the 3DGS form:                       */
/*   L = (1 - lambda) mean |img - target| + lambda (1 - mean SSIM),     */
/* SSIM per channel and pixel under an 11 x 11 Gaussian window (sigma   */
/* 1.5, zero padding at the border), C1 = 0.01^2, C2 = 0.03^2:          */
/*   (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 +   */
/*   s_y^2 + C2)); means over all C H W values.  The loss is reduced in  */
/* FP64 (deterministic); d_img = weight dL/dimg.                        */
/* ------------------------------------------------------------------ */
typedef struct {
    int C, H, W;           /* channels, rows, columns */
    const float *img;      /* [C][H][W] */
    const float *target;   /* [C][H][W] */
    float lambda;          /* D-SSIM weight in 0..1 (paper: 0.2) */
    float weight;          /* scale of the loss and its gradient (1 for one image) */
    int accumulate;        /* 0: *loss = weight L;  1: *loss += weight L (batches of images) */
    float *loss;           /* [1] device output */
    float *d_img;          /* [C][H][W] output, or NULL for the loss alone */
} avatar_image_loss_args;

size_t avatar_image_loss_workspace_size(const avatar_image_loss_args *a);
int avatar_image_loss(avatar_ctx *ctx, const avatar_image_loss_args *a, void *ws, size_t ws_bytes,
                      avatar_stream_t stream);

/* ------------------------------------------------------------------ */
/* Image loss - L1 part of Eq. 5 (Sec. 3.3): loss = mean |img - target|, */
/* d_img = sign(img - target) / n.  loss is a device float, d_img may be */
/* NULL.                                                                */
/* ------------------------------------------------------------------ */
int avatar_l1_loss(avatar_ctx *ctx, int64_t n, const float *img, const float *target, float *loss,
                   float *d_img, avatar_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* AVATAR_H */
