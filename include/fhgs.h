/*
 * fhgs.h -- C ABI of libfhgs.so, the GB300 (sm_103a) hot path of FHGS
 * feature splatting (arXiv 2505.19154).
 *
 * The library renders 3-D Gaussians that each carry an RGB colour (SH) and a
 * D-dimensional feature, with the tile-based depth-sorted rasterizer the
 * paper builds on (App. A), the front-to-back compositing of Eq. 4 applied to
 * colour and feature (the DRF path of Sec. 3.2), its hand-written derivative
 * (App. A.2), and the compositing-weight-normalised fusion of 2-D feature
 * maps into per-Gaussian features (Sec. 3.1).
 *
 * Conventions shared by every call
 *   - Every pointer marked "device" is caller-owned CUDA device memory; the
 *     library never allocates, frees or retains caller buffers.  Scratch that
 *     the library needs is owned by the context (fhgs_ctx) and grows on
 *     demand; fhgs_reserve() pre-sizes it (required before stream capture).
 *   - Host arrays (cameras, params, the fusion map pointer table) are read
 *     during the call only.
 *   - Every call is asynchronous on the given CUDA stream (cudaStream_t,
 *     passed as void*; NULL = legacy default stream) and returns an
 *     fhgs_status.  Errors that the host can see (bad sizes, NULL pointers,
 *     unsupported options, misaligned pointers) return immediately and
 *     launch nothing.  Errors found on the device (instance-buffer overflow,
 *     a bounded wait that ran out, non-finite inputs) latch into the
 *     context's device status word; fhgs_sync_status() synchronises the
 *     stream and reports them.  fhgs_last_error() gives a message.
 *   - Arrays are dense and row-major.  Images of several cameras are packed
 *     one after the other: camera c's pixel (x, y) is row
 *     pix_offset(c) + y * width(c) + x, pix_offset(c) = sum_{c'<c} W*H.
 *   - Tiles are 16 x 16 pixels (App. A).  The global tile id of camera c's
 *     tile (tx, ty) is tile_offset(c) + ty * ceil(W/16) + tx,
 *     tile_offset(c) = sum_{c'<c} ceil(W/16) * ceil(H/16).
 */
#ifndef FHGS_H
#define FHGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FHGS_ABI_VERSION 2
#define FHGS_MAX_CAMS 32 /* cameras per call */
#define FHGS_MAX_SH_DEGREE 3

typedef enum fhgs_status {
    FHGS_OK = 0,
    FHGS_ERR_INVALID_ARG = 1,  /* NULL pointer, negative size, bad camera */
    FHGS_ERR_UNSUPPORTED = 2,  /* D % 8 != 0, sh_degree > 3, tile != 16x16, too many cameras,
                                  a camera too large for binning */
    FHGS_ERR_ALIGNMENT = 3,    /* a pointer that needs 16-byte alignment is not */
    FHGS_ERR_CUDA = 4,         /* a CUDA runtime call failed (see fhgs_last_error) */
    FHGS_ERR_CAPACITY = 5,     /* more tile instances than the buffer holds */
    FHGS_ERR_TIMEOUT = 6,      /* a bounded device-side wait ran out */
    FHGS_ERR_NUMERIC = 7,      /* non-finite input values were found (and culled) */
    FHGS_ERR_NO_DEVICE = 8     /* no CUDA device, or not an sm_103 GPU */
} fhgs_status;

typedef struct fhgs_ctx fhgs_ctx;

/* Pinhole camera, OpenCV axes (x right, y down, z forward).  world_to_cam is
 * the 3x4 matrix [R|t] row by row: x_cam = R x_world + t (the matrix W of
 * Eq. 3).  width, height >= 1; fx, fy > 0.  Tile grid (16x16 tiles):
 * (tiles_x + 1) * (tiles_y + 1) <= 57344 and tiles_x <= 4096 (4K frames fit;
 * larger ones return FHGS_ERR_UNSUPPORTED). */
typedef struct fhgs_camera {
    int32_t width, height;
    float fx, fy, cx, cy;
    float world_to_cam[12];
} fhgs_camera;

/* Rasterizer parameters.  The paper fixes the tile size (16x16, App. A); it
 * gives no value for the others, which take the 3DGS-family defaults set by
 * fhgs_default_params(). */
typedef struct fhgs_params {
    int32_t tile_w, tile_h;  /* must be 16, 16 */
    int32_t sh_degree;       /* 0..3; sh holds (sh_degree+1)^2 coefficients per channel */
    int32_t path;            /* FHGS_PATH_* : which render kernels run */
    int32_t batch;           /* Gaussians per batch in the tensor-core kernels; 0 = auto */
    int32_t d_split;         /* feature columns per CTA in the tensor-core kernels; 0 = auto */
    float znear;             /* cull if view depth <= znear (0.2) */
    float dilation;          /* added to the screen covariance diagonal (0.3 px^2) */
    float alpha_min;         /* skip a Gaussian at a pixel if alpha < alpha_min (1/255) */
    float alpha_max;         /* alpha = min(alpha_max, op * G) (0.99) */
    float t_eps;             /* stop before a Gaussian that takes T below t_eps (1e-4) */
    float cutoff_sq;         /* skip a pixel outside the ellipse q2 > cutoff_sq (9) */
    float fov_clamp;         /* Jacobian uses x/z clamped to +-fov_clamp*W/(2 fx) (1.3) */
    float bg[3];             /* background colour behind the remaining transmittance */
    int32_t geometry;        /* FHGS_GEOM_*: the primitives' footprint model */
    int32_t list_cut;        /* 0: full tile lists; 1: lists cut where every pixel has stopped (see
                                fhgs_bin_sort); fhgs_default_params sets 0 */
} fhgs_params;

/* Footprint models.  FHGS_GEOM_EWA: 3-D Gaussians splatted to screen conics
 * (the 3DGS rasterizer the paper builds on, App. A).  FHGS_GEOM_SURFEL: the
 * 2DGS surfels of Sec. 3.1 (Eq. 1-3): the plane p + s_u t_u u + s_v t_v v
 * (t_u, t_v the first two columns of R(q); s_u, s_v = scales[i][0..1],
 * scales[i][2] is ignored and gets a zero gradient) with density
 * exp(-(u^2 + v^2)/2) at the point u(x) where the pixel's ray meets the
 * plane; binning follows the binary32 rule of the surfel footprint's
 * dual-conic box.  The surfel model runs fhgs_project, fhgs_bin_sort, the
 * render forward and backward (on the tensor cores for BF16 features and a
 * supported D, as for EWA: the feature blend and its transpose as tcgen05
 * products, the per-(pixel, surfel) footprint chain on the CUDA cores; else
 * FP32 on the CUDA cores) and the NDFD losses with their backward over
 * surfel weights (on the tensor cores for BF16 features at D = 512, else the
 * CUDA cores); fusion and the allocation-free backward return
 * FHGS_ERR_UNSUPPORTED. */
enum { FHGS_GEOM_EWA = 0, FHGS_GEOM_SURFEL = 1 };

enum {
    FHGS_PATH_AUTO = 0, /* tensor-core feature blend when D > 0 and features are BF16 */
    FHGS_PATH_FP32 = 1, /* plain FP32 per-pixel loop on the CUDA cores */
    FHGS_PATH_TC = 2    /* BF16 x BF16 -> FP32 blend on tcgen05 tensor cores (BF16 only) */
};

typedef enum fhgs_dtype { FHGS_F32 = 0, FHGS_BF16 = 1 } fhgs_dtype;

/* The Gaussian parameters of Eq. 1 in their 3-D (EWA) form; all device,
 * float32, n rows.  means [n][3]; scales [n][3] (linear, > 0); quats [n][4]
 * (w, x, y, z), normalised inside; opacities [n] in [0, 1] (already
 * activated); sh [n][(sh_degree+1)^2][3]. */
typedef struct fhgs_gaussians {
    const float *means, *scales, *quats, *opacities, *sh;
    int64_t n;
} fhgs_gaussians;

/* Depth-sorted per-tile lists produced by fhgs_bin_sort (App. A: Duplicate-
 * WithKeys, SortByKeys, IdentifyTileRanges).  All device, caller-owned.
 *   gids      [capacity]      Gaussian index of each tile instance, sorted by
 *                             (global tile id, depth, Gaussian index).
 *   keys      [capacity]      nullable; the 64-bit sort key of each instance:
 *                             global tile id << 32 | IEEE bits of the view
 *                             depth (positive, so the bits order like depth).
 *   ranges    [total_tiles][2] [start, end) of each tile's run in gids.
 *   n_instances [1]            number of instances emitted (may exceed
 *                             capacity; then FHGS_ERR_CAPACITY is latched). */
typedef struct fhgs_bins {
    uint32_t *gids;
    uint64_t *keys;
    uint32_t *ranges;
    int64_t *n_instances;
    int64_t capacity;
} fhgs_bins;

/* ---------------------------------------------------------------- context */
/* Create a context on CUDA device `device` (made current for the call).
 * Fails with FHGS_ERR_NO_DEVICE if the device is absent or not sm_103. */
fhgs_status fhgs_create(fhgs_ctx **ctx, int device);
void fhgs_destroy(fhgs_ctx *ctx);
const char *fhgs_last_error(const fhgs_ctx *ctx);
const char *fhgs_status_string(fhgs_status s);
int fhgs_abi_version(void);
void fhgs_default_params(fhgs_params *p);

/* Bytes of the per-(camera, Gaussian) projection buffer that fhgs_project
 * fills; the caller allocates it (16-byte aligned) and passes it on. */
int64_t fhgs_proj_bytes(int64_t n, int n_cams);
/* Number of tiles over all cameras (rows of fhgs_bins.ranges). */
int64_t fhgs_total_tiles(const fhgs_camera *cams, int n_cams);
/* Pre-size the context's scratch for up to max_n Gaussians seen by these
 * cameras, so later calls with at most that many Gaussians and the same
 * camera resolutions allocate nothing (required before stream capture). */
fhgs_status fhgs_reserve(fhgs_ctx *ctx, int64_t max_n, const fhgs_camera *cams, int n_cams);
/* Synchronise `stream`, then read and clear the context's device status
 * word.  Returns the first latched device-side error, or FHGS_OK. */
fhgs_status fhgs_sync_status(fhgs_ctx *ctx, void *stream);

/* ------------------------------------------------------------ hot path ---- */
/* EWA projection of every Gaussian into every camera and its SH
 * colour (Sec. 2.1 / App. A "Homogenization, 2DScreenGaussians").  Writes
 * the opaque projection buffer `proj` (fhgs_proj_bytes(n, n_cams) bytes):
 * screen mean, conic, opacity, colour, tile rectangle and depth key per
 * (camera, Gaussian).  Binning decisions follow the FP32 binning
 * specification exactly (single-rounded binary32 operations in a fixed
 * order).  Non-finite inputs are culled and latch FHGS_ERR_NUMERIC. */
fhgs_status fhgs_project(fhgs_ctx *ctx, const fhgs_gaussians *g, const fhgs_camera *cams, int n_cams,
                         const fhgs_params *p, void *proj, void *stream);

/* Duplicate each projected Gaussian into every 16x16 tile its
 * rectangle overlaps, sort the instances by (global tile id, depth,
 * Gaussian index) and find each tile's range (App. A).  Fills `bins`;
 * bins->keys may be NULL.  Uses context scratch.
 *
 * With p->list_cut = 1 (EWA geometry; otherwise the lists stay full) each
 * tile's list is cut after a point that every pixel of the tile provably never
 * passes: compositing stops before a Gaussian that would take T below t_eps,
 * and Gaussians whose alpha is at least a_lo at every pixel centre of the tile
 * (nested boxes inside the ellipses q2 <= 3 and q2 <= 1, alpha bounded by
 * min(alpha_max, op exp(-q/2)) with margins above FP32 rounding) each multiply
 * T by at most 1 - a_lo.  The cut falls at the end of the depth segment (of
 * the sort's segments of the depth order) in which the sum of -ln(1 - a_lo)
 * first passes -ln(t_eps).  Each cut list is a prefix of the full one, every
 * render, NDFD and fusion output over the cut lists equals the output over
 * the full lists, and n_instances counts the cut instances.  Cameras whose
 * tile grid exceeds (tiles_x + 1)(tiles_y + 1) = 28672 keep full lists. */
fhgs_status fhgs_bin_sort(fhgs_ctx *ctx, int64_t n, const void *proj, const fhgs_camera *cams, int n_cams,
                          const fhgs_params *p, const fhgs_bins *bins, void *stream);

/* Front-to-back compositing (Eq. 4) per tile of colour and features.
 *   features [n][D] device, FHGS_F32 or FHGS_BF16 (D % 8 == 0; D may be 0 and
 *            features NULL for colour only).  FHGS_PATH_TC needs BF16.
 *   rgb      [P][3]  out: sum_i w_i c_i + T_final * bg
 *   feat     [P][D]  out, nullable: sum_i w_i f_i (no background)
 *   T_final  [P]     out: transmittance after the last contributor
 *   last     [P]     out: (position in the tile's list of the last
 *                    contributor) + 1, 0 if none
 * P = total pixels of all cameras.  The tensor-core path rounds w_i to
 * BF16 for the feature blend and accumulates in FP32. */
fhgs_status fhgs_render_fwd(fhgs_ctx *ctx, int64_t n, const void *proj, const fhgs_bins *bins,
                            const void *features, fhgs_dtype ftype, int D, const fhgs_camera *cams,
                            int n_cams, const fhgs_params *p, float *rgb, float *feat, float *T_final,
                            int32_t *last, void *stream);

/* Derivative of L = sum_p grad_rgb[p] . rgb[p] + grad_feat[p] . feat[p]
 * (App. A.2: dL/dalpha_k = T_k dL/dw_k - (1/(1-alpha_k)) sum_{i>k} w_i
 * dL/dw_i, plus the background term), walking each tile back to front and
 * recovering each contributor's T from T_final: the FP32 path divides by
 * (1 - alpha) per contributor; the tensor-core path divides once per group
 * of Gaussians by the group's product of (1 - alpha) and rebuilds the T
 * inside the group from prefix products.  All gradient outputs are
 * OVERWRITTEN (not accumulated), device float32 with the shapes of the
 * inputs: grad_means [n][3], grad_scales [n][3], grad_quats [n][4],
 * grad_opac [n], grad_sh [n][K][3], grad_features [n][D] (nullable: skips
 * that contraction).  grad_feat may be NULL (treated as zero).  The
 * tensor-core path reads grad_feat through a TMA tensor map; if the driver
 * cannot encode it, the call returns FHGS_ERR_CUDA before the render
 * kernel and no gradient is valid. */
fhgs_status fhgs_render_bwd(fhgs_ctx *ctx, const fhgs_gaussians *g, const void *proj, const fhgs_bins *bins,
                            const void *features, fhgs_dtype ftype, int D, const fhgs_camera *cams,
                            int n_cams, const fhgs_params *p, const float *T_final, const int32_t *last,
                            const float *grad_rgb, const float *grad_feat, float *grad_means,
                            float *grad_scales, float *grad_quats, float *grad_opac, float *grad_sh,
                            float *grad_features, void *stream);

/* Non-differentiable feature fusion (Sec. 3.1, with the per-primitive
 * feature defined as the compositing-weight-normalised scatter over views):
 *   num[g][c] += sum_{v,p} w_g(v,p) maps[v][p][c],  den[g] += sum w_g(v,p),
 * with w the Eq. 4 weights of the forward render of view v.  maps is a HOST
 * array of n_views DEVICE pointers, each [H_v*W_v][D] float32.
 * flags: FHGS_FUSE_ACCUMULATE keeps num/den (else they are zeroed first);
 * FHGS_FUSE_FINALIZE then writes out[g][c] = num/den where den > 0, else 0;
 * FHGS_FUSE_NORMALIZE additionally L2-normalises each non-zero out row.
 * out may be NULL unless FINALIZE is set.  Uses context scratch; views are
 * processed in groups of up to 8 (fewer when the group's projection records
 * would pass 4 GiB), each group projected, binned and fused by one launch of
 * each kernel, with one host read of its instance count.  p->path: FHGS_PATH_FP32 sums on the CUDA cores;
 * FHGS_PATH_AUTO and FHGS_PATH_TC use the tensor cores when D % 64 == 0
 * (weights and maps as BF16 hi + lo, ~16-bit products, FP32 accumulation;
 * FHGS_PATH_TC with another D returns FHGS_ERR_UNSUPPORTED).  Each view's
 * lists follow p->list_cut as in fhgs_bin_sort (the sums are the same); the
 * projection of a view skips the SH colour, which fusion does not read. */
enum { FHGS_FUSE_ACCUMULATE = 1, FHGS_FUSE_FINALIZE = 2, FHGS_FUSE_NORMALIZE = 4 };
fhgs_status fhgs_fuse_features(fhgs_ctx *ctx, const fhgs_gaussians *g, const fhgs_camera *views, int n_views,
                               const float *const *maps, int D, const fhgs_params *p, float *num,
                               float *den, float *out, uint32_t flags, void *stream);

/* ------------------------------------------------------- point features -- */
/* The paper's point-to-feature assignment (Sec. 3.1; App. A,
 * "PointsFeatureFusion"): point i takes the feature of the pixel it projects
 * to in one view, drawn among the views that see it.  A view sees the point
 * when its camera depth exceeds p->znear and the projection (x, y) lies in
 * [0, W) x [0, H); the pixel is (floor x, floor y); the draw is the k-th
 * visible view in view order with k = floor(u[i] |M_i|) (clamped).  The
 * projection is binary32 with one rounding per operation in the order
 * c_r = ((R_r0 X + R_r1 Y) + R_r2 Z) + t_r, x = fx (c_x / c_z) + cx,
 * y = fy (c_y / c_z) + cy, so the choice is reproducible bit for bit.
 *   means  [n][3] device float32;  u [n] device float32 in [0, 1) (the
 *          caller's uniform draws);
 *   views  host array of n_views (1 .. FHGS_MAX_POINT_VIEWS) cameras;
 *   maps   host array of n_views DEVICE pointers, each [H_v*W_v][D] float32,
 *          16-byte aligned; D a positive multiple of 8;
 *   out    [n][D] device float32, 16-byte aligned: the feature (zeros for a
 *          point no view sees);
 *   view, pixel [n] device int32, nullable: the drawn view (-1 if none) and
 *          the pixel index y W + x in it (-1 if none).
 * Uses context scratch for the view table (copied from host memory on the
 * stream), so it is not for stream capture. */
#define FHGS_MAX_POINT_VIEWS 4096
fhgs_status fhgs_point_features(fhgs_ctx *ctx, int64_t n, const float *means, const fhgs_camera *views, int n_views,
                                const float *const *maps, int D, const float *u, const fhgs_params *p, float *out,
                                int32_t *view, int32_t *pixel, void *stream);

/* ------------------------------------------------------ training step -- */
/* The device side of one training iteration (App. A, Alg. 1 loop body,
 * with L = L_rgb + l1 L_gt + l2 L_cf of Sec. 3.3; the gradients of the
 * three terms come from fhgs_render_bwd and fhgs_ndfd_bwd and add).
 *
 * L1 photometric loss over m floats:  loss[0] += inv_count sum |a - b|
 * (device float[1], accumulated: zero it first), grad[i] = inv_count
 * sign(a[i] - b[i]) (0 where equal; grad nullable).  For the mean over P
 * pixels of RGB, m = 3 P and inv_count = 1 / (3 P). */
fhgs_status fhgs_l1_loss(fhgs_ctx *ctx, int64_t m, const float *a, const float *b, float inv_count, float *loss,
                         float *grad, void *stream);

/* Adam over the raw Gaussian parameters of the 3DGS family: means,
 * log-scales, unnormalised quaternions, opacity logits and SH (all device
 * float32, updated in place; the rasterizer reads means, quats and SH as
 * they are, and scales = exp(log-scales), opacities = sigmoid(logits)).
 * grads[0 .. n_grad_sets-1] (1 to FHGS_MAX_GRAD_SETS sets, host array of
 * device pointers) are gradients with respect to the ACTIVATED values, as
 * fhgs_render_bwd / fhgs_ndfd_bwd write them; the update adds the sets
 * element by element (the loss terms' gradients add, Sec. 3.3), takes the
 * sum to the raw parameters (d/dlog s = s d/ds, d/dlogit = op (1 - op)
 * d/dop), then
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   theta -= lr m / (1 - b1^t) / (sqrt(v / (1 - b2^t)) + eps).
 * state: fhgs_adam_state_floats(n, sh_degree) device floats, zeroed before
 * step 1 (m and v of each group).  scales_out [n][3] and opacities_out [n]
 * (nullable) receive the activated values of the updated parameters. */
typedef struct fhgs_adam {
    float lr[5];          /* means, log-scales, quaternions, opacity logits, SH */
    float beta1, beta2, eps;
    int32_t step;         /* t >= 1 of this update */
} fhgs_adam;
typedef struct fhgs_grads {
    const float *means, *scales, *quats, *opacities, *sh; /* device, [n][3], [n][3], [n][4], [n], [n][K][3] */
} fhgs_grads;
#define FHGS_MAX_GRAD_SETS 4
int64_t fhgs_adam_state_floats(int64_t n, int sh_degree);
fhgs_status fhgs_adam_gaussians(fhgs_ctx *ctx, int64_t n, int sh_degree, float *means, float *log_scales, float *quats,
                                float *logit_opacities, float *sh, const fhgs_grads *grads, int n_grad_sets,
                                float *state, const fhgs_adam *opt, float *scales_out, float *opacities_out,
                                void *stream);

/* The activated parameters the rasterizer reads, from the raw ones:
 * scales_out = exp(log_scales) [n][3], opacities_out = sigmoid(logits) [n]
 * (all device float32), the same values fhgs_adam_gaussians writes after an
 * update; for the first forward of a training run. */
fhgs_status fhgs_activate_gaussians(fhgs_ctx *ctx, int64_t n, const float *log_scales, const float *logit_opacities,
                                    float *scales_out, float *opacities_out, void *stream);

/* out[0] += sum of x[0 .. m-1] (device float32; out accumulated, zero it
 * first): the per-pixel NDFD loss maps' totals, L_gt and L_cf of Sec. 3.3,
 * in FP32 partial sums. */
fhgs_status fhgs_sum(fhgs_ctx *ctx, int64_t m, const float *x, float *out, void *stream);

/* ------------------------------------------------------------------ NDFD -- */
/* The walk's end state of an NDFD forward, which the backward can read
 * instead of rebuilding it front to back (App. A records F_{N-1} and W_{N-1}
 * for the same purpose): per pixel the feature sum F_N = sum_i w_i f_i over
 * all contributors [P][D] float32 (16-byte aligned), T after the walk [P]
 * float32 and the last contributor's list position + 1 [P] int32.  All
 * device, caller-owned.  Only the tensor-core NDFD kernels write and read it
 * (BF16 features, EWA at D = 256 or 512, surfels at D = 512); the CUDA-core
 * kernels ignore it.  fhgs_ndfd_bwd may be given it only after fhgs_ndfd_fwd
 * wrote it for the same Gaussians, lists, features, cameras and parameters. */
typedef struct fhgs_ndfd_state {
    float *F;
    float *T;
    int32_t *last;
} fhgs_ndfd_state;

/* Non-differentiable feature driving (Sec. 3.2; App. A "NDFD"): per pixel,
 * over the same depth-sorted tile lists, contributors and Eq. 4 weights
 * w_i = alpha_i T_i as fhgs_render_fwd (i = 1 nearest), with the pixel's
 * ground-truth feature f_gt(p):
 *   sigma_i = 1 / (1 + exp(k (cos<f_i, f_gt(p)> - lambda)))  (Sec. 3.3; the
 *             cosine is 0 where either vector is zero; the paper fixes
 *             k = 20, lambda = 0.5 in Sec. 4),
 *   L_gt(p) = sum_i w_i sigma_i                                   (Eq. 5),
 *   L_cf(p) = sum_i sigma_i w_i (W_{i-1} - F_{i-1} . f_i),
 *             W_n = sum_{j<=n} w_j, F_n = sum_{j<=n} w_j f_j  (Eq. 6, App. A.1).
 * L_cf uses the plain dot product f_i . f_j, which is the cosine for the unit
 * features the paper assumes: pass L2-normalised features.  No feature image
 * is rendered or stored.  Arguments as fhgs_render_fwd, plus
 *   feat_gt [P][D] device, the ground-truth feature of every pixel of every
 *           camera (packed like the images), same dtype as features,
 *           16-byte aligned;
 *   k, lambda  the activation's slope and threshold (finite);
 *   L_gt, L_cf [P] device float32, out;
 *   n_contrib  [P] device int32, out, nullable: the number of contributors
 *              (the i of the sums) of each pixel.
 * D must be 32, 64, 128, 256 or 512 (else FHGS_ERR_UNSUPPORTED).  With BF16
 * features and D = 256 or 512 and p->path AUTO or TC, the D-deep dot
 * products run on the tensor cores (BF16 operands, FP32 accumulation; the
 * weights and the running F as BF16 hi + lo pairs), split over a cluster of
 * D / 128 CTAs per half tile; otherwise (or with FHGS_PATH_FP32) they run in
 * FP32 on the CUDA cores.  p->path TC with any other dtype or D returns
 * FHGS_ERR_UNSUPPORTED.  A wait of the tensor-core kernel that runs out
 * latches FHGS_ERR_TIMEOUT (read by fhgs_sync_status).  With
 * p->geometry = FHGS_GEOM_SURFEL the weights are the 2DGS surfel render's
 * (the ray-plane solve of Sec. 3.1, the paper's own combination); the
 * tensor-core kernels then take BF16 features at D = 512 only (FHGS_PATH_TC
 * with any other D is FHGS_ERR_UNSUPPORTED).  save (nullable) receives the
 * walk's end state when the tensor-core kernels run (fhgs_ndfd_state). */
fhgs_status fhgs_ndfd_fwd(fhgs_ctx *ctx, int64_t n, const void *proj, const fhgs_bins *bins, const void *features,
                          const void *feat_gt, fhgs_dtype ftype, int D, const fhgs_camera *cams, int n_cams,
                          const fhgs_params *p, float k, float lambda, float *L_gt, float *L_cf, int32_t *n_contrib,
                          const fhgs_ndfd_state *save, void *stream);

/* Derivative of L = sum_p grad_Lgt[p] L_gt(p) + grad_Lcf[p] L_cf(p) with
 * respect to the Gaussian parameters, through the weights w only (features
 * and f_gt are constants, Sec. 3.2):
 *   dL/dw_k = grad_Lgt sigma_k + grad_Lcf (sigma_k (W_{k-1} - F_{k-1} . f_k)
 *             + sum_{i>k} sigma_i w_i (1 - f_i . f_k))            (Sec. 3.3),
 *   dL/dalpha_k = T_k dL/dw_k - (1/(1-alpha_k)) sum_{i>k} w_i dL/dw_i (App. A.2).
 * The walk recomputes F_N front to back, then goes back to front; nothing
 * from a forward call is needed, unless `saved` (nullable) holds the end
 * state fhgs_ndfd_fwd wrote with `save` for the same inputs: the tensor-core
 * kernels then read F_N, T and the last contributors instead of the front-to-
 * back walk (the gradients agree to the order of their float atomics).
 * grad_Lgt, grad_Lcf [P] device float32.  All
 * gradient outputs are OVERWRITTEN, device float32 with the shapes of
 * fhgs_render_bwd's: grad_means [n][3], grad_scales [n][3], grad_quats [n][4]
 * (16-byte aligned), grad_opac [n], grad_sh [n][K][3] (all zero: colour
 * does not enter the losses).  To train on L_rgb + l1 L_gt + l2 L_cf, scale
 * grad_Lgt and grad_Lcf and add these gradients to fhgs_render_bwd's.  For
 * surfels (FHGS_GEOM_SURFEL) the footprint chain is the surfel render
 * backward's (implicit differentiation of the ray-plane solve) and
 * grad_scales[i][2] is zero. */
fhgs_status fhgs_ndfd_bwd(fhgs_ctx *ctx, const fhgs_gaussians *g, const void *proj, const fhgs_bins *bins,
                          const void *features, const void *feat_gt, fhgs_dtype ftype, int D,
                          const fhgs_camera *cams, int n_cams, const fhgs_params *p, float k, float lambda,
                          const float *grad_Lgt, const float *grad_Lcf, float *grad_means, float *grad_scales,
                          float *grad_quats, float *grad_opac, float *grad_sh, const fhgs_ndfd_state *saved,
                          void *stream);

/* ----------------------------------------------------- allocation-free -- */
/* Largest n_cams * n accepted by fhgs_render_bwd_noalloc.  Its scratch is
 * 48 bytes per (camera, Gaussian): 12 MiB, reserved on every GPU that loads
 * the library until the process exits. */
#define FHGS_NOALLOC_MAX_ENTRIES 262144

/* The paper has no counterpart to this call.  It is fhgs_render_bwd for
 * callers that cannot allocate device memory (code inside a custom device
 * allocator or a memory pool's callback, which must not re-enter cudaMalloc;
 * plugin hosts that own every device allocation; loops that keep allocation
 * out of their steady state).  It needs no context and allocates nothing:
 * arguments, layouts and results are those of fhgs_render_bwd, on the
 * current CUDA device.
 *   - Its scratch (the per-(camera, Gaussian) footprint gradients) and a
 *     status word are file-scope device arrays of the library.
 *   - n_cams * n > FHGS_NOALLOC_MAX_ENTRIES returns FHGS_ERR_UNSUPPORTED and
 *     launches nothing; the other argument checks return as in
 *     fhgs_render_bwd (without a message: there is no context).
 *   - The first call on a device looks up the arrays' device addresses with
 *     that device current; make that first call before any stream capture.
 *   - Every call shares the arrays and clears the scratch first: calls that
 *     overlap on the GPU (several streams or threads) race on it, so order
 *     them on one stream.
 *   - A device-side error (a bounded wait that ran out) is latched in a
 *     status word of its own, shared like the scratch; read and clear it
 *     with fhgs_noalloc_sync_status. */
fhgs_status fhgs_render_bwd_noalloc(const fhgs_gaussians *g, const void *proj, const fhgs_bins *bins,
                                    const void *features, fhgs_dtype ftype, int D, const fhgs_camera *cams,
                                    int n_cams, const fhgs_params *p, const float *T_final, const int32_t *last,
                                    const float *grad_rgb, const float *grad_feat, float *grad_means,
                                    float *grad_scales, float *grad_quats, float *grad_opac, float *grad_sh,
                                    float *grad_features, void *stream);

/* The paper has no counterpart to this call either.  Status of the
 * allocation-free backward on the current device: synchronises `stream`,
 * reads the status word that fhgs_render_bwd_noalloc's kernels latch into,
 * clears it, and returns FHGS_ERR_TIMEOUT (a bounded device-side wait ran
 * out: the gradients of that call are incomplete), FHGS_ERR_NUMERIC,
 * FHGS_ERR_CAPACITY or FHGS_OK.  Allocates nothing; FHGS_ERR_CUDA if a
 * runtime call fails. */
fhgs_status fhgs_noalloc_sync_status(void *stream);

/* ------------------------------------------------ failure detection -- */
/* Debug probe of the bounded device-side waits, off (0) by default and
 * process-wide.  While ns > 0, every CTA of the tensor-core kernels
 * (render forward and backward, fusion) launched afterwards -- through a
 * context or the allocation-free call -- first waits at most ns nanoseconds
 * on an mbarrier that nothing arrives at, before it issues any copy or MMA
 * or allocates tensor memory.  The wait runs out, the CTA latches
 * FHGS_ERR_TIMEOUT into the status word of its call and returns, so those
 * launches compute nothing.  It exists to test that a wait which runs out
 * is reported (fhgs_sync_status, fhgs_noalloc_sync_status) and leaves the
 * context usable.  ns > 10 s returns FHGS_ERR_INVALID_ARG.  A launch
 * captured in a CUDA graph keeps the value it was captured with. */
fhgs_status fhgs_debug_wait_probe(uint64_t ns);

/* ----------------------------------------------------- instrumentation -- */
/* Kernel timing: while enabled, every kernel group the context launches is
 * bracketed by CUDA events recorded on the launch stream (a pool of 8192
 * events, created when first enabled).  fhgs_profile_read synchronises on
 * the recorded events, writes a JSON object {"name": [launches, total_ms],
 * ...} into buf (NUL-terminated, truncated to len) and clears the records.
 * Timing adds one event record before and after each launch. */
fhgs_status fhgs_profile_enable(fhgs_ctx *ctx, int enable);
fhgs_status fhgs_profile_read(fhgs_ctx *ctx, char *buf, int64_t len);
/* Measurement helper; the paper has no counterpart.  Launches an FP32
 * fused-multiply-add throughput probe on `stream` (blocks x 1024 threads,
 * iters rounds of 128 FMAs per thread, on the current device) and returns the
 * FLOPs it performs, or -1 on bad sizes or a failed launch.  The caller times
 * the launch with CUDA events; FLOPs / time is the measured FP32 peak that
 * the CUDA-core kernels' rooflines are reported against. */
int64_t fhgs_ffma_probe(int blocks, int iters, void *stream);
/* Number of kernels this library has launched in this process. */
int64_t fhgs_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* FHGS_H */
