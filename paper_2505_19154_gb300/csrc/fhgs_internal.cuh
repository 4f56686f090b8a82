// Internal declarations shared by the CUDA translation units of libfhgs.so.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "fhgs.h"

namespace fhgs {

constexpr int kTile = 16;          // tile edge in pixels (App. A)
constexpr int kTilePix = kTile * kTile;

// Device status word bits (latched by kernels, read by fhgs_sync_status).
enum : unsigned { ST_CAPACITY = 1u, ST_TIMEOUT = 2u, ST_NUMERIC = 4u };

// One camera as the kernels see it (passed by value inside CamSet).
struct DevCam {
    int W, H, tiles_x, tiles_y;
    int tile_off;       // first global tile id of this camera
    int pad0;
    long long pix_off;  // first packed pixel row of this camera
    float fx, fy, cx, cy;
    float R[9];         // world-to-camera rotation, row-major
    float t[3];         // world-to-camera translation
    float campos[3];    // camera centre in world space, -R^T t
    float pad1;
};

struct CamSet {
    int n;
    int total_tiles;
    long long total_pix;
    DevCam c[FHGS_MAX_CAMS];
};

struct Params {
    float znear, dil, amin, amax, teps, cut, fov;
    float bg0, bg1, bg2;
    int sh_deg, K;
    // Failure-detection probe of the tensor-core kernels (fhgs_debug_wait_probe):
    // 0 = off; else each CTA first waits at most this many ns on an mbarrier
    // that nothing arrives at, latches ST_TIMEOUT and returns.
    unsigned long long probe_ns;
    int geom;  // FHGS_GEOM_EWA or FHGS_GEOM_SURFEL
};

// Per (camera, Gaussian) screen-space record used by the render kernels.
//   a = (mean_x, mean_y, conic_A, conic_B)   q2 = A dx^2 + 2 B dx dy + C dy^2
//   b = (conic_C, opacity, r, g)
//   c = (b, view depth, bits of the colour clamp mask, 0)
struct __align__(16) GRec {
    float4 a, b, c;
};

// Per (camera, surfel) record of the 2DGS path (surfel.cu): the projected
// centre and M = T'^-1 of the surfel's centred projective map (per pixel
// u = (M00 dx + M01 dy) / w, v = (M10 dx + M11 dy) / w, w = M20 dx + M21 dy
// + M22), opacity, colour:
//   a = (x_c, y_c, M00, M01)   b = (M10, M11, M20, M21)
//   c = (M22, opacity, r, g)   d = (b, view depth, colour clamp mask bits, 0)
struct __align__(16) SRec {
    float4 a, b, c, d;
};
// floats per (camera, surfel) in the render-gradient scratch of the 2DGS
// path: d(x_c, y_c, M00, M01, M10, M11, M20, M21, M22, opacity, r, g, b)
constexpr int kSurfelG2d = 16;

// Largest tile grid of one camera: the per-segment count kernel keeps
// (tiles_x + 1) * (tiles_y + 1) ints in shared memory (224 KB), and the
// scatter keeps at least one row of tile counters per warp.
constexpr long long FHGS_MAX_TILE_CELLS = 57344;
constexpr int FHGS_MAX_TILES_X = 4096;

// Layout of the caller's projection buffer (fhgs_proj_bytes).
struct ProjView {
    GRec *rec;        // [C*N]
    int4 *trect;      // [C*N] tile rectangle (tx0, ty0, tx1, ty1), inclusive
    uint32_t *ntiles; // [C*N] tiles in the rectangle, 0 if culled
    uint32_t *dkey;   // [C*N] IEEE bits of the view depth, 0xFFFFFFFF if culled
    SRec *srec;       // [C*N] surfel records (2DGS geometry only)
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Lets `kernel` take up to the device's opt-in dynamic shared memory.  The
// attribute is per-device state, so it is set once per device for each call
// site (`done` holds one bit per device): the launches after the first then
// make no runtime call but the launch itself, which keeps them legal inside
// a stream capture.
template <typename K>
inline void allow_max_smem(std::atomic<unsigned long long> &done, K kernel) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return;
    cudaFuncAttributes fa;  // the opt-in limit covers static and dynamic shared memory together
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes) ==
        cudaSuccess)
        done.fetch_or(bit, std::memory_order_acq_rel);
}

inline size_t proj_bytes(long long cn) {
    return align_up(sizeof(GRec) * cn, 256) + align_up(sizeof(int4) * cn, 256) +
           2 * align_up(sizeof(uint32_t) * cn, 256) + align_up(sizeof(SRec) * cn, 256) + 256;
}

inline ProjView proj_view(void *base, long long cn) {
    char *p = (char *)align_up((size_t)base, 256);
    ProjView v;
    v.rec = (GRec *)p;
    p += align_up(sizeof(GRec) * cn, 256);
    v.trect = (int4 *)p;
    p += align_up(sizeof(int4) * cn, 256);
    v.ntiles = (uint32_t *)p;
    p += align_up(sizeof(uint32_t) * cn, 256);
    v.dkey = (uint32_t *)p;
    p += align_up(sizeof(uint32_t) * cn, 256);
    v.srec = (SRec *)p;
    return v;
}

// Camera index of a global tile id (cameras are few; linear scan).
__device__ __forceinline__ int cam_of_tile(const CamSet &cs, int tile) {
    int ci = 0;
#pragma unroll 1
    while (ci + 1 < cs.n && tile >= cs.c[ci + 1].tile_off) ++ci;
    return ci;
}

// Eq. 4's alpha at a pixel: q2 = A dx^2 + 2 B dx dy + C dy^2 with
// (dx, dy) = pixel centre - mean, G = exp(-q2/2), alpha = min(alpha_max,
// op G).  Written with explicit fused multiply-adds so the forward, backward
// and fusion kernels all take bit-identical per-pixel decisions.
__device__ __forceinline__ float eval_q2(float dx, float dy, float A, float B, float C) {
    const float t = __fmaf_rn(2.f * B, dy, __fmul_rn(A, dx));
    return __fmaf_rn(t, dx, __fmul_rn(__fmul_rn(C, dy), dy));
}

// u(x), v(x) of a 2DGS surfel at a pixel centre from its record's a, b and
// M22 (explicit roundings, so that the surfel render, its backward and the
// NDFD kernels take the same decisions): (dx, dy) = pixel centre - x_c,
// w = M20 dx + M21 dy + M22, u = (M00 dx + M01 dy) / w, v = (M10 dx + M11 dy)
// / w.  False when the pixel's ray meets the plane behind the camera (w <= 0)
// or outside the cutoff u^2 + v^2 <= cutoff_sq.
struct SurfelHit {
    float dx, dy, iw, u, v, r2;
};

__device__ __forceinline__ bool surfel_uv(const float4 &A, const float4 &B, float M22, float fpx, float fpy, float cut,
                                          SurfelHit &h) {
    h.dx = __fsub_rn(fpx, A.x);
    h.dy = __fsub_rn(fpy, A.y);
    const float w = __fmaf_rn(B.z, h.dx, __fmaf_rn(B.w, h.dy, M22));
    if (!(w > 0.f)) return false;
    const float nu = __fmaf_rn(A.z, h.dx, __fmul_rn(A.w, h.dy));
    const float nv = __fmaf_rn(B.x, h.dx, __fmul_rn(B.y, h.dy));
    h.iw = __frcp_rn(w);
    h.u = __fmul_rn(nu, h.iw);
    h.v = __fmul_rn(nv, h.iw);
    h.r2 = __fmaf_rn(h.u, h.u, __fmul_rn(h.v, h.v));
    return h.r2 <= cut;
}

__device__ __forceinline__ void latch(unsigned *status, unsigned bit) {
    if (status) atomicOr(status, bit);
}

// Counts kernel launches (fhgs_launch_count); defined in api.cu.
void note_launch(int k);

// Argument checks of the allocation-free backward (api.cu); ctx may be
// nullptr.  Fills the device camera set, parameters and the path choice.
fhgs_status check_bwd_args(fhgs_ctx *ctx, const fhgs_gaussians *g, const void *proj, const fhgs_bins *bins,
                           const void *features, fhgs_dtype ftype, int D, const fhgs_camera *cams, int n_cams,
                           const fhgs_params *p, const float *T_final, const int32_t *last, const float *grad_rgb,
                           const float *grad_feat, float *grad_means, float *grad_scales, float *grad_quats,
                           float *grad_opac, float *grad_sh, float *grad_features, CamSet &cs, Params &q, bool &tc);

// ---------------------------------------------------------------- launches
// projection (project.cu)
void launch_project(const fhgs_gaussians &g, const CamSet &cs, const Params &p, ProjView pv,
                    unsigned *status, cudaStream_t st);
void launch_project_bwd(const fhgs_gaussians &g, const CamSet &cs, const Params &p, ProjView pv,
                        const float *g2d, float *gmeans, float *gscales, float *gquats, float *gop,
                        float *gsh, cudaStream_t st);

// binning (binning.cu)
struct BinScratch {
    uint32_t *dk_a, *dv_a, *dk_b, *dv_b;  // depth sort [C*N]
    short4 *rect;                         // tile rectangles in sorted order [C*N]
    int4 *inner;                          // list cut: the nested boxes' tile ranges in sorted order [C*N]
    uint32_t *imass;                      // list cut: their opacity-mass units [C*N]
    uint32_t *table;                      // per (tile, segment) counts, then offsets
    uint32_t *mass;                       // list cut: per (tile, segment) opacity mass
    int *close;                           // list cut: per tile, the last segment it takes
    uint32_t *partials;                   // scan partials of the table
    uint32_t *hist;                       // radix histogram [256][G]
    uint32_t *kbits;                      // AND and OR of the live depth keys (passes that can be skipped)
    int seg, nseg, sm_count;              // segment size, segments per camera
};
size_t bin_scratch_bytes(long long N, int n_cams, int total_tiles, int sm_count);
BinScratch bin_scratch_view(void *base, long long N, int n_cams, int total_tiles, int sm_count);
// cut: the render rules of the list cut (EWA geometry), or nullptr for the
// full lists of the (tile, depth) sort.
void launch_bin_sort(long long N, int n_cams, const CamSet &cs, ProjView pv, const fhgs_bins &bins,
                     BinScratch sc, const Params *cut, unsigned *status, cudaStream_t st);
// Whether launch_bin_sort can cut the lists of these cameras (the count pass
// keeps two difference arrays of each camera's tile grid in shared memory).
bool bin_cut_fits(const CamSet &cs);

// render, FP32 CUDA-core path (render_fp32.cu)
void launch_render_fwd_fp32(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                            const void *feats, int bf16, int D, float *rgb, float *feat, float *T,
                            int32_t *last, cudaStream_t st);
void launch_render_bwd_fp32(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                            const void *feats, int bf16, int D, const float *T, const int32_t *last,
                            const float *grgb, const float *gfeat, float *g2d, float *gfeatures,
                            cudaStream_t st);
// The feature map of each camera of a fusion launch: [H*W, D] float32.
struct FuseMaps {
    const float *m[FHGS_MAX_CAMS];
};
void launch_fuse_fp32(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                      const FuseMaps &maps, int D, float *num, float *den, cudaStream_t st);
void launch_fuse_finalize(long long N, int D, const float *num, const float *den, float *out, int normalize,
                          cudaStream_t st);
// fusion on the tensor cores (render_tc.cu): D a multiple of 64
int fuse_tc_dn(int D);
void launch_fuse_tc(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                    const FuseMaps &maps, int D, float *num, float *den, unsigned *status, cudaStream_t st);

// render, tcgen05 tensor-core path (render_tc.cu)
int tc_supported(int D, int d_split);
void launch_render_fwd_tc(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                          const __nv_bfloat16 *feats, int D, int d_split, float *rgb, float *feat, float *T,
                          int32_t *last, unsigned *status, cudaStream_t st);
// false (nothing launched) when the tensor map of gfeat cannot be encoded
bool launch_render_bwd_tc(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                          const __nv_bfloat16 *feats, int D, int d_split, const float *T, const int32_t *last,
                          const float *grgb, const float *gfeat, float *g2d, float *gfeatures, unsigned *status,
                          cudaStream_t st);

// tcgen05 backward with dL/dF streamed through shared memory in 64-channel
// chunks (render_bwd_stream.cu): D % 128 == 0 and grad_feat given; false
// (nothing launched) otherwise or when the tensor map cannot be encoded
bool bwd_stream_supported(int D);
bool launch_render_bwd_stream(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                              const __nv_bfloat16 *feats, int D, const float *T, const int32_t *last,
                              const float *grgb, const float *gfeat, float *g2d, float *gfeatures, unsigned *status,
                              cudaStream_t st);

// The paper's point-to-feature assignment (points.cu).  One view as the
// kernel reads it: width, height, fx, fy, cx, cy, [R|t] row by row, and the
// view's feature map [H*W][D] (device).
struct PFView {
    float cam[18];
    int32_t pad[2];
    const float *map;
};
void launch_point_features(long long n, const float *means, const PFView *views, int n_views, float znear,
                           const float *u, int D, float *out, int32_t *view, int32_t *pixel, cudaStream_t st);

// 2DGS surfel geometry (surfel.cu): projection with the binary32 binning
// rule, the FP32 render forward and backward, and the projection backward;
// g2d holds kSurfelG2d floats per (camera, surfel)
void launch_project_surfel(const fhgs_gaussians &g, const CamSet &cs, const Params &p, ProjView pv, unsigned *status,
                           cudaStream_t st);
void launch_render_fwd_surfel(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                              const void *feats, int bf16, int D, float *rgb, float *feat, float *T, int32_t *last,
                              cudaStream_t st);
void launch_render_bwd_surfel(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                              const void *feats, int bf16, int D, const float *T, const int32_t *last,
                              const float *grgb, const float *gfeat, float *g2d, float *gfeatures, cudaStream_t st);
void launch_project_surfel_bwd(const fhgs_gaussians &g, const CamSet &cs, const Params &p, ProjView pv,
                               const float *g2d, float *gmeans, float *gscales, float *gquats, float *gop,
                               float *gsh, cudaStream_t st);

// training-step kernels (train.cu)
void launch_l1_loss(long long m, const float *a, const float *b, float inv_count, float *loss, float *grad,
                    int sm_count, cudaStream_t st);
void launch_adam_gaussians(long long n, int K, float *means, float *log_s, float *quats, float *logit, float *sh,
                           const fhgs_grads *grads, int n_sets, float *state, const fhgs_adam *opt, float *scales_out,
                           float *opac_out, cudaStream_t st);
void launch_activate(long long n, const float *log_s, const float *logit, float *scales, float *opac,
                     cudaStream_t st);
void launch_sum(long long m, const float *x, float *out, int sm_count, cudaStream_t st);

// NDFD losses and their backward (ndfd.cu): D in {32, 64, 128, 256, 512}
bool ndfd_supported(int D);
void launch_ndfd_fwd(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                     const void *feats, const void *fgt, int bf16, int D, float ks, float lam, float *Lgt,
                     float *Lcf, int32_t *nc, cudaStream_t st);
void launch_ndfd_bwd(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                     const void *feats, const void *fgt, int bf16, int D, float ks, float lam, const float *dLgt,
                     const float *dLcf, float *g2d, cudaStream_t st);

// NDFD on the tensor cores (ndfd_tc.cu): BF16 features and ground truth, D
// in {256, 512} (EWA) or 512 (surfels), split over a cluster of D / 128 CTAs;
// g2d has 12 (EWA) or kSurfelG2d (surfel) floats per (camera, primitive)
bool ndfd_tc_supported(int D, int geom);
// The walk's end state of the tensor-core NDFD forward (F == nullptr: none):
// F_N [P][D], T after the walk [P], last contributor + 1 [P].
struct NdfdState {
    float *F;
    float *T;
    int32_t *last;
};
void launch_ndfd_fwd_tc(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                        const __nv_bfloat16 *feats, const __nv_bfloat16 *fgt, int D, float ks, float lam, float *Lgt,
                        float *Lcf, int32_t *nc, NdfdState save, unsigned *status, cudaStream_t st);
// g2d: 12 floats per (camera, Gaussian), accumulated (zero it first);
// saved.F != nullptr: the forward's end state replaces the front-to-back rebuild
void launch_ndfd_bwd_tc(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                        const __nv_bfloat16 *feats, const __nv_bfloat16 *fgt, int D, float ks, float lam,
                        const float *dLgt, const float *dLcf, float *g2d, NdfdState saved, unsigned *status,
                        cudaStream_t st);

}  // namespace fhgs
