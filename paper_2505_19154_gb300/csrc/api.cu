// C ABI of libfhgs.so (declared in include/fhgs.h): argument checks, context
// scratch, camera/parameter marshalling and kernel dispatch.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "fhgs_internal.cuh"

using namespace fhgs;

// Most views a fusion call projects, bins and fuses together.
constexpr int kFuseGroup = 8;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
};

struct fhgs_ctx {
    int device = 0;
    bool prof = false;
    std::vector<cudaEvent_t> pool;  // profiling events, created on first enable
    size_t pool_next = 0;
    std::vector<ProfRec> recs;
    int sm_count = 0;
    std::string err;
    unsigned *status = nullptr;  // device status word
    DevBuf bin;                  // binning scratch
    DevBuf g2d;                  // per (camera, Gaussian) render gradients
    DevBuf fuse_proj, fuse_gids, fuse_ranges, fuse_count;  // fusion view scratch
    DevBuf pf_views;             // view table of the point-feature assignment
};

static std::atomic<long long> g_launches{0};
// the context's small device area: word 0 is the status word
constexpr size_t kStatusBytes = 64;
static std::atomic<unsigned long long> g_wait_probe_ns{0};

namespace fhgs {
void note_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
}  // namespace fhgs

namespace {

constexpr size_t kProfEvents = 8192;

// Brackets one kernel group with CUDA events on its stream while profiling.
struct Prof {
    fhgs_ctx *ctx;
    cudaStream_t st;
    ProfRec *rec = nullptr;
    Prof(fhgs_ctx *c, const char *name, cudaStream_t s) : ctx(c), st(s) {
        if (!ctx->prof || ctx->pool_next + 2 > ctx->pool.size()) return;
        ctx->recs.push_back({name, ctx->pool[ctx->pool_next], ctx->pool[ctx->pool_next + 1]});
        ctx->pool_next += 2;
        rec = &ctx->recs.back();
        cudaEventRecord(rec->a, st);
    }
    ~Prof() {
        if (rec) cudaEventRecord(rec->b, st);
    }
};

fhgs_status fail(fhgs_ctx *ctx, fhgs_status s, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return s;
}

fhgs_status cuda_fail(fhgs_ctx *ctx, cudaError_t e, const char *what) {
    if (ctx) ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
    return FHGS_ERR_CUDA;
}

#define FHGS_CUDA(ctx, call)                                      \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
    } while (0)

fhgs_status ensure(fhgs_ctx *ctx, DevBuf &b, size_t bytes) {
    if (b.bytes >= bytes) return FHGS_OK;
    if (b.p) {
        cudaError_t e = cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFree");
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
    b.p = p;
    b.bytes = bytes;
    return FHGS_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

fhgs_status check_params(fhgs_ctx *ctx, const fhgs_params *p) {
    if (!p) return fail(ctx, FHGS_ERR_INVALID_ARG, "params is NULL");
    if (p->tile_w != kTile || p->tile_h != kTile)
        return fail(ctx, FHGS_ERR_UNSUPPORTED, "only 16x16 tiles are supported");
    if (p->sh_degree < 0 || p->sh_degree > FHGS_MAX_SH_DEGREE)
        return fail(ctx, FHGS_ERR_UNSUPPORTED, "sh_degree must be 0..3");
    if (!(p->alpha_max > 0.f && p->alpha_max < 1.f) || !(p->alpha_min >= 0.f) || !(p->t_eps > 0.f) ||
        !(p->cutoff_sq > 0.f) || !(p->znear > 0.f) || !(p->dilation >= 0.f))
        return fail(ctx, FHGS_ERR_INVALID_ARG, "parameter out of range");
    if (p->path < FHGS_PATH_AUTO || p->path > FHGS_PATH_TC)
        return fail(ctx, FHGS_ERR_INVALID_ARG, "unknown path");
    if (p->geometry != FHGS_GEOM_EWA && p->geometry != FHGS_GEOM_SURFEL)
        return fail(ctx, FHGS_ERR_INVALID_ARG, "unknown geometry");
    if (p->list_cut != 0 && p->list_cut != 1) return fail(ctx, FHGS_ERR_INVALID_ARG, "list_cut must be 0 or 1");
    return FHGS_OK;
}

fhgs_status make_cams(fhgs_ctx *ctx, const fhgs_camera *cams, int n_cams, CamSet &cs) {
    if (!cams) return fail(ctx, FHGS_ERR_INVALID_ARG, "cams is NULL");
    if (n_cams < 1) return fail(ctx, FHGS_ERR_INVALID_ARG, "n_cams must be >= 1, got " + std::to_string(n_cams));
    if (n_cams > FHGS_MAX_CAMS) return fail(ctx, FHGS_ERR_UNSUPPORTED, "at most 32 cameras per call");
    memset(&cs, 0, sizeof(cs));
    cs.n = n_cams;
    long long tiles = 0, pix = 0;
    for (int i = 0; i < n_cams; ++i) {
        const fhgs_camera &c = cams[i];
        if (c.width < 1 || c.height < 1 || !(c.fx > 0.f) || !(c.fy > 0.f) || !std::isfinite(c.cx) ||
            !std::isfinite(c.cy))
            return fail(ctx, FHGS_ERR_INVALID_ARG, "camera " + std::to_string(i) + " is invalid");
        for (int k = 0; k < 12; ++k)
            if (!std::isfinite(c.world_to_cam[k]))
                return fail(ctx, FHGS_ERR_INVALID_ARG, "camera " + std::to_string(i) + " has a non-finite pose");
        DevCam &d = cs.c[i];
        d.W = c.width;
        d.H = c.height;
        d.tiles_x = (c.width + kTile - 1) / kTile;
        d.tiles_y = (c.height + kTile - 1) / kTile;
        if ((long long)(d.tiles_x + 1) * (d.tiles_y + 1) > FHGS_MAX_TILE_CELLS || d.tiles_x > FHGS_MAX_TILES_X)
            return fail(ctx, FHGS_ERR_UNSUPPORTED, "camera " + std::to_string(i) + " is too large for the binning "
                        "kernels ((tiles_x + 1) * (tiles_y + 1) <= 57344, tiles_x <= 4096)");
        d.tile_off = (int)tiles;
        d.pix_off = pix;
        d.fx = c.fx;
        d.fy = c.fy;
        d.cx = c.cx;
        d.cy = c.cy;
        for (int r = 0; r < 3; ++r) {
            for (int k = 0; k < 3; ++k) d.R[3 * r + k] = c.world_to_cam[4 * r + k];
            d.t[r] = c.world_to_cam[4 * r + 3];
        }
        for (int k = 0; k < 3; ++k) {
            double acc = 0.0;
            for (int r = 0; r < 3; ++r) acc += (double)d.R[3 * r + k] * (double)d.t[r];
            d.campos[k] = (float)(-acc);
        }
        tiles += (long long)d.tiles_x * d.tiles_y;
        pix += (long long)c.width * c.height;
    }
    if (tiles >= (1ll << 31)) return fail(ctx, FHGS_ERR_UNSUPPORTED, "too many tiles");
    cs.total_tiles = (int)tiles;
    cs.total_pix = pix;
    return FHGS_OK;
}

Params make_params(const fhgs_params *p) {
    Params q;
    q.znear = p->znear;
    q.dil = p->dilation;
    q.amin = p->alpha_min;
    q.amax = p->alpha_max;
    q.teps = p->t_eps;
    q.cut = p->cutoff_sq;
    q.fov = p->fov_clamp;
    q.bg0 = p->bg[0];
    q.bg1 = p->bg[1];
    q.bg2 = p->bg[2];
    q.sh_deg = p->sh_degree;
    q.K = (p->sh_degree + 1) * (p->sh_degree + 1);
    q.probe_ns = g_wait_probe_ns.load(std::memory_order_relaxed);
    q.geom = p->geometry;
    return q;
}

fhgs_status check_gaussians(fhgs_ctx *ctx, const fhgs_gaussians *g, bool need_sh) {
    if (!g) return fail(ctx, FHGS_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->n < 0 || g->n >= (1ll << 31)) return fail(ctx, FHGS_ERR_INVALID_ARG, "bad Gaussian count");
    if (g->n == 0) return FHGS_OK;
    if (!g->means || !g->scales || !g->quats || !g->opacities || (need_sh && !g->sh))
        return fail(ctx, FHGS_ERR_INVALID_ARG, "a Gaussian parameter pointer is NULL");
    if (!aligned16(g->quats)) return fail(ctx, FHGS_ERR_ALIGNMENT, "quats must be 16-byte aligned");
    return FHGS_OK;
}

fhgs_status check_bins(fhgs_ctx *ctx, const fhgs_bins *b) {
    if (!b || !b->gids || !b->ranges || !b->n_instances)
        return fail(ctx, FHGS_ERR_INVALID_ARG, "bins has a NULL buffer");
    if (b->capacity < 0 || b->capacity > 0xFFFFFFFFll)
        return fail(ctx, FHGS_ERR_INVALID_ARG, "bins capacity out of range");
    return FHGS_OK;
}

fhgs_status check_features(fhgs_ctx *ctx, const void *features, fhgs_dtype ft, int D, long long n) {
    if (D < 0) return fail(ctx, FHGS_ERR_INVALID_ARG, "D must be >= 0");
    if (D % 8) return fail(ctx, FHGS_ERR_UNSUPPORTED, "D must be a multiple of 8");
    if (ft != FHGS_F32 && ft != FHGS_BF16) return fail(ctx, FHGS_ERR_INVALID_ARG, "unknown feature dtype");
    if (n == 0) return FHGS_OK;  // no rows: the pointer is never read
    if (D > 0 && !features) return fail(ctx, FHGS_ERR_INVALID_ARG, "features is NULL with D > 0");
    if (D > 0 && !aligned16(features)) return fail(ctx, FHGS_ERR_ALIGNMENT, "features must be 16-byte aligned");
    return FHGS_OK;
}

fhgs_status ensure_bin_scratch(fhgs_ctx *ctx, long long N, int n_cams, int total_tiles) {
    const size_t bytes = bin_scratch_bytes(N, n_cams, total_tiles, ctx->sm_count);
    return bytes > ctx->bin.bytes ? ensure(ctx, ctx->bin, bytes) : FHGS_OK;
}

bool bwd_stream_enabled() {
    static const bool on = [] {
        const char *e = std::getenv("FHGS_BWD_STREAM");
        return e && e[0] == '1';
    }();
    return on;
}

bool use_tc(const fhgs_params *p, fhgs_dtype ft, int D) {
    if (D == 0) return false;
    if (p->path == FHGS_PATH_FP32) return false;
    if (ft != FHGS_BF16) return false;
    return tc_supported(D, p->d_split) != 0;
}

}  // namespace

namespace fhgs {
// Argument checks of the allocation-free backward (fhgs_render_bwd_noalloc);
// the same checks as fhgs_render_bwd, with ctx == nullptr (no message kept).
fhgs_status check_bwd_args(fhgs_ctx *ctx, const fhgs_gaussians *g, const void *proj, const fhgs_bins *bins,
                           const void *features, fhgs_dtype ftype, int D, const fhgs_camera *cams, int n_cams,
                           const fhgs_params *p, const float *T_final, const int32_t *last, const float *grad_rgb,
                           const float *grad_feat, float *grad_means, float *grad_scales, float *grad_quats,
                           float *grad_opac, float *grad_sh, float *grad_features, CamSet &cs, Params &q, bool &tc) {
    fhgs_status s = check_params(ctx, p);
    if (s == FHGS_OK) s = check_gaussians(ctx, g, true);
    if (s == FHGS_OK) s = check_bins(ctx, bins);
    if (s == FHGS_OK) s = check_features(ctx, features, ftype, D, g ? g->n : 0);
    if (s != FHGS_OK) return s;
    if (!proj || !T_final || !last || !grad_rgb) return fail(ctx, FHGS_ERR_INVALID_ARG, "NULL input buffer");
    if (g->n > 0 && (!grad_means || !grad_scales || !grad_quats || !grad_opac || !grad_sh))
        return fail(ctx, FHGS_ERR_INVALID_ARG, "NULL gradient buffer");
    if (!aligned16(grad_quats)) return fail(ctx, FHGS_ERR_ALIGNMENT, "grad_quats must be 16-byte aligned");
    if ((grad_feat && !aligned16(grad_feat)) || (grad_features && !aligned16(grad_features)))
        return fail(ctx, FHGS_ERR_ALIGNMENT, "feature gradients must be 16-byte aligned");
    if (p->path == FHGS_PATH_TC && D > 0 && !use_tc(p, ftype, D))
        return fail(ctx, FHGS_ERR_UNSUPPORTED, "tensor-core path needs BF16 features and a supported D");
    if (p->geometry != FHGS_GEOM_EWA) return fail(ctx, FHGS_ERR_UNSUPPORTED, "EWA geometry only");
    if ((s = make_cams(ctx, cams, n_cams, cs)) != FHGS_OK) return s;
    q = make_params(p);
    tc = D > 0 && use_tc(p, ftype, D) && (grad_feat || grad_features);
    return FHGS_OK;
}
}  // namespace fhgs

extern "C" {

int fhgs_abi_version(void) { return FHGS_ABI_VERSION; }

const char *fhgs_status_string(fhgs_status s) {
    switch (s) {
        case FHGS_OK: return "ok";
        case FHGS_ERR_INVALID_ARG: return "invalid argument";
        case FHGS_ERR_UNSUPPORTED: return "unsupported";
        case FHGS_ERR_ALIGNMENT: return "misaligned pointer";
        case FHGS_ERR_CUDA: return "CUDA error";
        case FHGS_ERR_CAPACITY: return "instance buffer overflow";
        case FHGS_ERR_TIMEOUT: return "device wait timed out";
        case FHGS_ERR_NUMERIC: return "non-finite input";
        case FHGS_ERR_NO_DEVICE: return "no sm_103 device";
    }
    return "unknown status";
}

void fhgs_default_params(fhgs_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->tile_w = p->tile_h = kTile;
    p->sh_degree = 0;
    p->path = FHGS_PATH_AUTO;
    p->batch = 0;
    p->d_split = 0;
    p->znear = 0.2f;
    p->dilation = 0.3f;
    p->alpha_min = 1.0f / 255.0f;
    p->alpha_max = 0.99f;
    p->t_eps = 1e-4f;
    p->cutoff_sq = 9.0f;
    p->fov_clamp = 1.3f;
}

fhgs_status fhgs_create(fhgs_ctx **out, int device) {
    if (!out) return FHGS_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return FHGS_ERR_NO_DEVICE;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return FHGS_ERR_NO_DEVICE;
    if (prop.major != 10 || prop.minor != 3) return FHGS_ERR_NO_DEVICE;
    if (cudaSetDevice(device) != cudaSuccess) return FHGS_ERR_NO_DEVICE;
    fhgs_ctx *ctx = new fhgs_ctx();
    ctx->device = device;
    ctx->sm_count = prop.multiProcessorCount;
    if (cudaMalloc(&ctx->status, kStatusBytes) != cudaSuccess || cudaMemset(ctx->status, 0, kStatusBytes) != cudaSuccess) {
        delete ctx;
        return FHGS_ERR_CUDA;
    }
    *out = ctx;
    return FHGS_OK;
}

void fhgs_destroy(fhgs_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    for (DevBuf *b : {&ctx->bin, &ctx->g2d, &ctx->fuse_proj, &ctx->fuse_gids, &ctx->fuse_ranges, &ctx->fuse_count})
        if (b->p) cudaFree(b->p);
    for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
    if (ctx->status) cudaFree(ctx->status);
    delete ctx;
}

const char *fhgs_last_error(const fhgs_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int64_t fhgs_proj_bytes(int64_t n, int n_cams) {
    if (n < 0 || n_cams < 1) return -1;
    return (int64_t)proj_bytes((long long)n * n_cams);
}

int64_t fhgs_total_tiles(const fhgs_camera *cams, int n_cams) {
    if (!cams || n_cams < 1) return -1;
    int64_t t = 0;
    for (int i = 0; i < n_cams; ++i)
        t += (int64_t)((cams[i].width + kTile - 1) / kTile) * ((cams[i].height + kTile - 1) / kTile);
    return t;
}

fhgs_status fhgs_reserve(fhgs_ctx *ctx, int64_t max_n, const fhgs_camera *cams, int n_cams) {
    if (!ctx) return FHGS_ERR_INVALID_ARG;
    if (max_n < 0 || max_n >= (1ll << 31)) return fail(ctx, FHGS_ERR_INVALID_ARG, "bad reserve size");
    CamSet cs;
    fhgs_status s = make_cams(ctx, cams, n_cams, cs);
    if (s != FHGS_OK) return s;
    FHGS_CUDA(ctx, cudaSetDevice(ctx->device));
    if ((s = ensure_bin_scratch(ctx, max_n, n_cams, cs.total_tiles)) != FHGS_OK) return s;
    return ensure(ctx, ctx->g2d, sizeof(float) * 12 * (size_t)max_n * n_cams + 256);
}

fhgs_status fhgs_debug_wait_probe(uint64_t ns) {
    if (ns > 10000000000ull) return FHGS_ERR_INVALID_ARG;  // at most 10 s
    g_wait_probe_ns.store(ns, std::memory_order_relaxed);
    return FHGS_OK;
}

fhgs_status fhgs_sync_status(fhgs_ctx *ctx, void *stream) {
    if (!ctx) return FHGS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    FHGS_CUDA(ctx, cudaStreamSynchronize(st));
    unsigned h = 0;
    FHGS_CUDA(ctx, cudaMemcpy(&h, ctx->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    FHGS_CUDA(ctx, cudaMemset(ctx->status, 0, sizeof(unsigned)));
    if (h & ST_CAPACITY) return fail(ctx, FHGS_ERR_CAPACITY, "tile instance buffer overflow");
    if (h & ST_TIMEOUT) return fail(ctx, FHGS_ERR_TIMEOUT, "a device-side wait ran out");
    if (h & ST_NUMERIC) return fail(ctx, FHGS_ERR_NUMERIC, "non-finite inputs were culled");
    return FHGS_OK;
}

fhgs_status fhgs_project(fhgs_ctx *ctx, const fhgs_gaussians *g, const fhgs_camera *cams, int n_cams,
                         const fhgs_params *p, void *proj, void *stream) {
    if (!ctx) return FHGS_ERR_INVALID_ARG;
    fhgs_status s = check_params(ctx, p);
    if (s == FHGS_OK) s = check_gaussians(ctx, g, true);
    if (s != FHGS_OK) return s;
    CamSet cs;
    if ((s = make_cams(ctx, cams, n_cams, cs)) != FHGS_OK) return s;
    if (!proj) return fail(ctx, FHGS_ERR_INVALID_ARG, "proj is NULL");
    if (!aligned16(proj)) return fail(ctx, FHGS_ERR_ALIGNMENT, "proj must be 16-byte aligned");
    FHGS_CUDA(ctx, cudaSetDevice(ctx->device));
    const Params q = make_params(p);
    {
        Prof pr(ctx, "project", (cudaStream_t)stream);
        if (p->geometry == FHGS_GEOM_SURFEL)
            launch_project_surfel(*g, cs, q, proj_view(proj, (long long)g->n * n_cams), ctx->status,
                                  (cudaStream_t)stream);
        else
            launch_project(*g, cs, q, proj_view(proj, (long long)g->n * n_cams), ctx->status, (cudaStream_t)stream);
    }
    FHGS_CUDA(ctx, cudaGetLastError());
    return FHGS_OK;
}

fhgs_status fhgs_bin_sort(fhgs_ctx *ctx, int64_t n, const void *proj, const fhgs_camera *cams, int n_cams,
                          const fhgs_params *p, const fhgs_bins *bins, void *stream) {
    if (!ctx) return FHGS_ERR_INVALID_ARG;
    fhgs_status s = check_params(ctx, p);
    if (s == FHGS_OK) s = check_bins(ctx, bins);
    if (s != FHGS_OK) return s;
    if (n < 0 || n >= (1ll << 31)) return fail(ctx, FHGS_ERR_INVALID_ARG, "bad Gaussian count");
    if (!proj) return fail(ctx, FHGS_ERR_INVALID_ARG, "proj is NULL");
    CamSet cs;
    if ((s = make_cams(ctx, cams, n_cams, cs)) != FHGS_OK) return s;
    if ((long long)n * n_cams >= (1ll << 32)) return fail(ctx, FHGS_ERR_UNSUPPORTED, "too many entries");
    FHGS_CUDA(ctx, cudaSetDevice(ctx->device));
    const long long cn = (long long)n * n_cams;
    if ((s = ensure_bin_scratch(ctx, n, n_cams, cs.total_tiles)) != FHGS_OK) return s;
    BinScratch sc = bin_scratch_view(ctx->bin.p, n, n_cams, cs.total_tiles, ctx->sm_count);
    const Params q = make_params(p);
    {
        Prof pr(ctx, p->list_cut ? "bin_sort_cut" : "bin_sort", (cudaStream_t)stream);
        launch_bin_sort(n, n_cams, cs, proj_view(const_cast<void *>(proj), cn), *bins, sc,
                        p->list_cut ? &q : nullptr, ctx->status, (cudaStream_t)stream);
    }
    FHGS_CUDA(ctx, cudaGetLastError());
    return FHGS_OK;
}

fhgs_status fhgs_render_fwd(fhgs_ctx *ctx, int64_t n, const void *proj, const fhgs_bins *bins, const void *features,
                            fhgs_dtype ftype, int D, const fhgs_camera *cams, int n_cams, const fhgs_params *p,
                            float *rgb, float *feat, float *T_final, int32_t *last, void *stream) {
    if (!ctx) return FHGS_ERR_INVALID_ARG;
    fhgs_status s = check_params(ctx, p);
    if (s == FHGS_OK) s = check_bins(ctx, bins);
    if (s == FHGS_OK) s = check_features(ctx, features, ftype, D, n);
    if (s != FHGS_OK) return s;
    if (n < 0 || !proj || !rgb || !T_final || !last)
        return fail(ctx, FHGS_ERR_INVALID_ARG, "NULL output or projection buffer");
    if (feat && !aligned16(feat)) return fail(ctx, FHGS_ERR_ALIGNMENT, "feat must be 16-byte aligned");
    if (p->path == FHGS_PATH_TC && D > 0 && !use_tc(p, ftype, D))
        return fail(ctx, FHGS_ERR_UNSUPPORTED, "tensor-core path needs BF16 features and a supported D");
    CamSet cs;
    if ((s = make_cams(ctx, cams, n_cams, cs)) != FHGS_OK) return s;
    FHGS_CUDA(ctx, cudaSetDevice(ctx->device));
    const Params q = make_params(p);
    ProjView pv = proj_view(const_cast<void *>(proj), (long long)n * n_cams);
    cudaStream_t st = (cudaStream_t)stream;
    const int Df = feat ? D : 0;
    const bool tc = Df > 0 && use_tc(p, ftype, D);
    if (p->geometry == FHGS_GEOM_SURFEL && !tc) {
        {
            Prof pr(ctx, "render_fwd_surfel", st);
            launch_render_fwd_surfel(n, cs, q, pv, *bins, features, ftype == FHGS_BF16, Df, rgb, feat, T_final, last,
                                     st);
        }
        FHGS_CUDA(ctx, cudaGetLastError());
        return FHGS_OK;
    }
    Prof pr(ctx, tc ? (p->geometry == FHGS_GEOM_SURFEL ? "render_fwd_tc_surfel" : "render_fwd_tc") : "render_fwd_fp32",
            st);
    if (tc)
        launch_render_fwd_tc(n, cs, q, pv, *bins, (const __nv_bfloat16 *)features, D, p->d_split, rgb, feat, T_final,
                             last, ctx->status, st);
    else
        launch_render_fwd_fp32(n, cs, q, pv, *bins, features, ftype == FHGS_BF16, Df, rgb, feat, T_final, last, st);
    FHGS_CUDA(ctx, cudaGetLastError());
    return FHGS_OK;
}

fhgs_status fhgs_render_bwd(fhgs_ctx *ctx, const fhgs_gaussians *g, const void *proj, const fhgs_bins *bins,
                            const void *features, fhgs_dtype ftype, int D, const fhgs_camera *cams, int n_cams,
                            const fhgs_params *p, const float *T_final, const int32_t *last, const float *grad_rgb,
                            const float *grad_feat, float *grad_means, float *grad_scales, float *grad_quats,
                            float *grad_opac, float *grad_sh, float *grad_features, void *stream) {
    if (!ctx) return FHGS_ERR_INVALID_ARG;
    fhgs_status s = check_params(ctx, p);
    if (s == FHGS_OK) s = check_gaussians(ctx, g, true);
    if (s == FHGS_OK) s = check_bins(ctx, bins);
    if (s == FHGS_OK) s = check_features(ctx, features, ftype, D, g ? g->n : 0);
    if (s != FHGS_OK) return s;
    if (!proj || !T_final || !last || !grad_rgb)
        return fail(ctx, FHGS_ERR_INVALID_ARG, "NULL input buffer");
    if (g->n > 0 && (!grad_means || !grad_scales || !grad_quats || !grad_opac || !grad_sh))
        return fail(ctx, FHGS_ERR_INVALID_ARG, "NULL gradient buffer");
    if (!aligned16(grad_quats)) return fail(ctx, FHGS_ERR_ALIGNMENT, "grad_quats must be 16-byte aligned");
    if ((grad_feat && !aligned16(grad_feat)) || (grad_features && !aligned16(grad_features)))
        return fail(ctx, FHGS_ERR_ALIGNMENT, "feature gradients must be 16-byte aligned");
    if (p->path == FHGS_PATH_TC && D > 0 && !use_tc(p, ftype, D))
        return fail(ctx, FHGS_ERR_UNSUPPORTED, "tensor-core path needs BF16 features and a supported D");
    CamSet cs;
    if ((s = make_cams(ctx, cams, n_cams, cs)) != FHGS_OK) return s;
    FHGS_CUDA(ctx, cudaSetDevice(ctx->device));
    const long long n = g->n, cn = n * n_cams;
    cudaStream_t st = (cudaStream_t)stream;
    if (p->geometry == FHGS_GEOM_SURFEL) {
        if ((s = ensure(ctx, ctx->g2d, sizeof(float) * kSurfelG2d * (size_t)cn + 256)) != FHGS_OK) return s;
        float *g2d = (float *)ctx->g2d.p;
        FHGS_CUDA(ctx, cudaMemsetAsync(g2d, 0, sizeof(float) * kSurfelG2d * (size_t)cn, st));
        if (grad_features && D > 0)
            FHGS_CUDA(ctx, cudaMemsetAsync(grad_features, 0, sizeof(float) * (size_t)n * D, st));
        const Params q = make_params(p);
        ProjView pv = proj_view(const_cast<void *>(proj), cn);
        const bool tc = D > 0 && use_tc(p, ftype, D) && (grad_feat || grad_features);
        if (tc) {
            Prof pr(ctx, "render_bwd_tc_surfel", st);
            if (!launch_render_bwd_tc(n, cs, q, pv, *bins, (const __nv_bfloat16 *)features, D, p->d_split, T_final,
                                      last, grad_rgb, grad_feat, g2d, grad_features, ctx->status, st))
                return fail(ctx, FHGS_ERR_CUDA, "could not encode the tensor map of grad_feat");
        } else {
            Prof pr(ctx, "render_bwd_surfel", st);
            launch_render_bwd_surfel(n, cs, q, pv, *bins, features, ftype == FHGS_BF16, D, T_final, last, grad_rgb,
                                     grad_feat, g2d, D > 0 ? grad_features : nullptr, st);
        }
        {
            Prof pb(ctx, "project_bwd", st);
            launch_project_surfel_bwd(*g, cs, q, pv, g2d, grad_means, grad_scales, grad_quats, grad_opac, grad_sh,
                                      st);
        }
        FHGS_CUDA(ctx, cudaGetLastError());
        return FHGS_OK;
    }
    if ((s = ensure(ctx, ctx->g2d, sizeof(float) * 12 * (size_t)cn + 256)) != FHGS_OK) return s;
    float *g2d = (float *)ctx->g2d.p;
    FHGS_CUDA(ctx, cudaMemsetAsync(g2d, 0, sizeof(float) * 12 * (size_t)cn, st));
    if (grad_features && D > 0) FHGS_CUDA(ctx, cudaMemsetAsync(grad_features, 0, sizeof(float) * (size_t)n * D, st));
    const Params q = make_params(p);
    ProjView pv = proj_view(const_cast<void *>(proj), cn);
    const bool tc = D > 0 && use_tc(p, ftype, D) && (grad_feat || grad_features);
    {
        Prof pr(ctx, tc ? "render_bwd_tc" : "render_bwd_fp32", st);
        // d_split 1: the streamed kernel (all D channels per item, dL/dF in
        // 64-channel chunks), when D % 128 == 0 and dL/dF is given; d_split 0
        // (auto) takes it only when FHGS_BWD_STREAM=1 is set in the environment
        const bool stream_ok = tc && grad_feat != nullptr && bwd_stream_supported(D) &&
                               (p->d_split == 1 || (p->d_split == 0 && bwd_stream_enabled()));
        if (stream_ok) {
            if (!launch_render_bwd_stream(n, cs, q, pv, *bins, (const __nv_bfloat16 *)features, D, T_final, last,
                                          grad_rgb, grad_feat, g2d, grad_features, ctx->status, st))
                return fail(ctx, FHGS_ERR_CUDA, "could not encode the tensor map of grad_feat");
        } else if (tc) {
            if (!launch_render_bwd_tc(n, cs, q, pv, *bins, (const __nv_bfloat16 *)features, D, p->d_split, T_final,
                                      last, grad_rgb, grad_feat, g2d, grad_features, ctx->status, st))
                return fail(ctx, FHGS_ERR_CUDA, "could not encode the tensor map of grad_feat");
        } else
            launch_render_bwd_fp32(n, cs, q, pv, *bins, features, ftype == FHGS_BF16, D, T_final, last, grad_rgb,
                                   grad_feat, g2d, D > 0 ? grad_features : nullptr, st);
    }
    {
        Prof pb(ctx, "project_bwd", st);
        launch_project_bwd(*g, cs, q, pv, g2d, grad_means, grad_scales, grad_quats, grad_opac, grad_sh, st);
    }
    FHGS_CUDA(ctx, cudaGetLastError());
    return FHGS_OK;
}

fhgs_status fhgs_point_features(fhgs_ctx *ctx, int64_t n, const float *means, const fhgs_camera *views, int n_views,
                                const float *const *maps, int D, const float *u, const fhgs_params *p, float *out,
                                int32_t *view, int32_t *pixel, void *stream) {
    if (!ctx) return FHGS_ERR_INVALID_ARG;
    fhgs_status s = check_params(ctx, p);
    if (s != FHGS_OK) return s;
    if (n < 0 || n >= (1ll << 31)) return fail(ctx, FHGS_ERR_INVALID_ARG, "bad point count");
    if (D <= 0 || D % 8) return fail(ctx, FHGS_ERR_UNSUPPORTED, "D must be a positive multiple of 8");
    if (!views || n_views < 1 || n_views > FHGS_MAX_POINT_VIEWS)
        return fail(ctx, FHGS_ERR_INVALID_ARG, "bad views");
    if (!maps) return fail(ctx, FHGS_ERR_INVALID_ARG, "maps is NULL");
    if (n > 0 && (!means || !u || !out)) return fail(ctx, FHGS_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned16(out)) return fail(ctx, FHGS_ERR_ALIGNMENT, "out must be 16-byte aligned");
    std::vector<PFView> tab((size_t)n_views);
    for (int v = 0; v < n_views; ++v) {
        const fhgs_camera &c = views[v];
        if (c.width < 1 || c.height < 1 || !(c.fx > 0.f) || !(c.fy > 0.f))
            return fail(ctx, FHGS_ERR_INVALID_ARG, "bad camera");
        if (!maps[v]) return fail(ctx, FHGS_ERR_INVALID_ARG, "a feature map is NULL");
        if (!aligned16(maps[v])) return fail(ctx, FHGS_ERR_ALIGNMENT, "feature maps must be 16-byte aligned");
        PFView &t = tab[v];
        t.cam[0] = (float)c.width;
        t.cam[1] = (float)c.height;
        t.cam[2] = c.fx;
        t.cam[3] = c.fy;
        t.cam[4] = c.cx;
        t.cam[5] = c.cy;
        for (int k = 0; k < 12; ++k) t.cam[6 + k] = c.world_to_cam[k];
        t.pad[0] = t.pad[1] = 0;
        t.map = maps[v];
    }
    FHGS_CUDA(ctx, cudaSetDevice(ctx->device));
    if ((s = ensure(ctx, ctx->pf_views, sizeof(PFView) * (size_t)n_views)) != FHGS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    PFView *dv = (PFView *)ctx->pf_views.p;
    // from pageable memory: staged before the call returns, so tab may go
    FHGS_CUDA(ctx, cudaMemcpyAsync(dv, tab.data(), sizeof(PFView) * (size_t)n_views, cudaMemcpyHostToDevice, st));
    {
        Prof pr(ctx, "point_features", st);
        launch_point_features(n, means, dv, n_views, p->znear, u, D, out, view, pixel, st);
    }
    FHGS_CUDA(ctx, cudaGetLastError());
    return FHGS_OK;
}

fhgs_status fhgs_l1_loss(fhgs_ctx *ctx, int64_t m, const float *a, const float *b, float inv_count, float *loss,
                         float *grad, void *stream) {
    if (!ctx) return FHGS_ERR_INVALID_ARG;
    if (m < 0) return fail(ctx, FHGS_ERR_INVALID_ARG, "negative size");
    if (!loss || (m > 0 && (!a || !b))) return fail(ctx, FHGS_ERR_INVALID_ARG, "NULL buffer");
    if (!std::isfinite(inv_count)) return fail(ctx, FHGS_ERR_INVALID_ARG, "inv_count must be finite");
    FHGS_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    {
        Prof pr(ctx, "l1_loss", st);
        launch_l1_loss(m, a, b, inv_count, loss, grad, ctx->sm_count, st);
    }
    FHGS_CUDA(ctx, cudaGetLastError());
    return FHGS_OK;
}

int64_t fhgs_adam_state_floats(int64_t n, int sh_degree) {
    if (n < 0 || sh_degree < 0 || sh_degree > 3) return -1;
    const int64_t K = (int64_t)(sh_degree + 1) * (sh_degree + 1);
    return 2 * n * (11 + 3 * K);
}

fhgs_status fhgs_adam_gaussians(fhgs_ctx *ctx, int64_t n, int sh_degree, float *means, float *log_scales, float *quats,
                                float *logit_opacities, float *sh, const fhgs_grads *grads, int n_grad_sets,
                                float *state, const fhgs_adam *opt, float *scales_out, float *opacities_out,
                                void *stream) {
    if (!ctx) return FHGS_ERR_INVALID_ARG;
    if (n < 0 || n >= (1ll << 31)) return fail(ctx, FHGS_ERR_INVALID_ARG, "bad Gaussian count");
    if (sh_degree < 0 || sh_degree > 3) return fail(ctx, FHGS_ERR_UNSUPPORTED, "sh_degree must be 0..3");
    if (!opt) return fail(ctx, FHGS_ERR_INVALID_ARG, "opt is NULL");
    if (opt->step < 1) return fail(ctx, FHGS_ERR_INVALID_ARG, "the Adam step number starts at 1");
    if (!(opt->beta1 >= 0.f && opt->beta1 < 1.f && opt->beta2 >= 0.f && opt->beta2 < 1.f && opt->eps >= 0.f))
        return fail(ctx, FHGS_ERR_INVALID_ARG, "bad Adam constants");
    if (n_grad_sets < 1 || n_grad_sets > FHGS_MAX_GRAD_SETS || !grads)
        return fail(ctx, FHGS_ERR_INVALID_ARG, "1..4 gradient sets");
    if (n > 0 && (!means || !log_scales || !quats || !logit_opacities || !sh || !state))
        return fail(ctx, FHGS_ERR_INVALID_ARG, "NULL buffer");
    for (int k = 0; k < n_grad_sets && n > 0; ++k)
        if (!grads[k].means || !grads[k].scales || !grads[k].quats || !grads[k].opacities || !grads[k].sh)
            return fail(ctx, FHGS_ERR_INVALID_ARG, "NULL gradient buffer");
    FHGS_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    {
        Prof pr(ctx, "adam", st);
        launch_adam_gaussians(n, (sh_degree + 1) * (sh_degree + 1), means, log_scales, quats, logit_opacities, sh,
                              grads, n_grad_sets, state, opt, scales_out, opacities_out, st);
    }
    FHGS_CUDA(ctx, cudaGetLastError());
    return FHGS_OK;
}

fhgs_status fhgs_activate_gaussians(fhgs_ctx *ctx, int64_t n, const float *log_scales, const float *logit_opacities,
                                    float *scales_out, float *opacities_out, void *stream) {
    if (!ctx) return FHGS_ERR_INVALID_ARG;
    if (n < 0 || n >= (1ll << 31)) return fail(ctx, FHGS_ERR_INVALID_ARG, "bad Gaussian count");
    if (n > 0 && (!log_scales || !logit_opacities || !scales_out || !opacities_out))
        return fail(ctx, FHGS_ERR_INVALID_ARG, "NULL buffer");
    FHGS_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    {
        Prof pr(ctx, "activate", st);
        launch_activate(n, log_scales, logit_opacities, scales_out, opacities_out, st);
    }
    FHGS_CUDA(ctx, cudaGetLastError());
    return FHGS_OK;
}

fhgs_status fhgs_sum(fhgs_ctx *ctx, int64_t m, const float *x, float *out, void *stream) {
    if (!ctx) return FHGS_ERR_INVALID_ARG;
    if (m < 0) return fail(ctx, FHGS_ERR_INVALID_ARG, "negative size");
    if (!out || (m > 0 && !x)) return fail(ctx, FHGS_ERR_INVALID_ARG, "NULL buffer");
    FHGS_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    {
        Prof pr(ctx, "sum", st);
        launch_sum(m, x, out, ctx->sm_count, st);
    }
    FHGS_CUDA(ctx, cudaGetLastError());
    return FHGS_OK;
}

// Shared argument checks of the two NDFD calls.
// The NDFD losses run on the tensor cores unless the FP32 path is asked for
// or the features are not BF16 with D in {256, 512}.
static bool ndfd_use_tc(const fhgs_params *p, fhgs_dtype ftype, int D) {
    return p->path != FHGS_PATH_FP32 && ftype == FHGS_BF16 && ndfd_tc_supported(D, p->geometry);
}

static fhgs_status check_ndfd(fhgs_ctx *ctx, long long n, const void *proj, const fhgs_bins *bins,
                              const void *features, const void *feat_gt, fhgs_dtype ftype, int D,
                              const fhgs_params *p, float k, float lambda) {
    fhgs_status s = check_params(ctx, p);
    if (s == FHGS_OK) s = check_bins(ctx, bins);
    if (s == FHGS_OK) s = check_features(ctx, features, ftype, D, n);
    if (s != FHGS_OK) return s;
    if (!ndfd_supported(D)) return fail(ctx, FHGS_ERR_UNSUPPORTED, "NDFD needs D in {32, 64, 128, 256, 512}");
    if (!proj) return fail(ctx, FHGS_ERR_INVALID_ARG, "NULL input buffer");
    if (!feat_gt) return fail(ctx, FHGS_ERR_INVALID_ARG, "feat_gt is NULL");
    if (!aligned16(feat_gt)) return fail(ctx, FHGS_ERR_ALIGNMENT, "feat_gt must be 16-byte aligned");
    if (!std::isfinite(k) || !std::isfinite(lambda))
        return fail(ctx, FHGS_ERR_INVALID_ARG, "the activation's slope and threshold must be finite");
    if (p->path == FHGS_PATH_TC && !ndfd_use_tc(p, ftype, D))
        return fail(ctx, FHGS_ERR_UNSUPPORTED,
                    "tensor-core NDFD needs BF16 features with D in {256, 512} (EWA) or D = 512 (surfels)");
    return FHGS_OK;
}

// An NDFD end state: NULL, or all three buffers (F 16-byte aligned).
static fhgs_status check_ndfd_state(fhgs_ctx *ctx, const fhgs_ndfd_state *st) {
    if (!st) return FHGS_OK;
    if (!st->F || !st->T || !st->last) return fail(ctx, FHGS_ERR_INVALID_ARG, "NDFD state has a NULL buffer");
    if (!aligned16(st->F)) return fail(ctx, FHGS_ERR_ALIGNMENT, "NDFD state F must be 16-byte aligned");
    return FHGS_OK;
}

static NdfdState ndfd_state(const fhgs_ndfd_state *st) {
    NdfdState r{nullptr, nullptr, nullptr};
    if (st) r = NdfdState{st->F, st->T, st->last};
    return r;
}

fhgs_status fhgs_ndfd_fwd(fhgs_ctx *ctx, int64_t n, const void *proj, const fhgs_bins *bins, const void *features,
                          const void *feat_gt, fhgs_dtype ftype, int D, const fhgs_camera *cams, int n_cams,
                          const fhgs_params *p, float k, float lambda, float *L_gt, float *L_cf, int32_t *n_contrib,
                          const fhgs_ndfd_state *save, void *stream) {
    if (!ctx) return FHGS_ERR_INVALID_ARG;
    if (n < 0 || n >= (1ll << 31)) return fail(ctx, FHGS_ERR_INVALID_ARG, "bad Gaussian count");
    fhgs_status s = check_ndfd(ctx, n, proj, bins, features, feat_gt, ftype, D, p, k, lambda);
    if (s == FHGS_OK) s = check_ndfd_state(ctx, save);
    if (s != FHGS_OK) return s;
    if (!L_gt || !L_cf) return fail(ctx, FHGS_ERR_INVALID_ARG, "NULL output buffer");
    CamSet cs;
    if ((s = make_cams(ctx, cams, n_cams, cs)) != FHGS_OK) return s;
    FHGS_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const Params q = make_params(p);
    ProjView pv = proj_view(const_cast<void *>(proj), n * n_cams);
    if (ndfd_use_tc(p, ftype, D)) {
        Prof pr(ctx, p->geometry == FHGS_GEOM_SURFEL ? "ndfd_fwd_tc_surfel" : "ndfd_fwd_tc", st);
        launch_ndfd_fwd_tc(n, cs, q, pv, *bins, (const __nv_bfloat16 *)features, (const __nv_bfloat16 *)feat_gt, D, k,
                           lambda, L_gt, L_cf, n_contrib, ndfd_state(save), ctx->status, st);
    } else {
        Prof pr(ctx, p->geometry == FHGS_GEOM_SURFEL ? "ndfd_fwd_surfel" : "ndfd_fwd", st);
        launch_ndfd_fwd(n, cs, q, pv, *bins, features, feat_gt, ftype == FHGS_BF16, D, k, lambda, L_gt, L_cf, n_contrib, st);
    }
    FHGS_CUDA(ctx, cudaGetLastError());
    return FHGS_OK;
}

fhgs_status fhgs_ndfd_bwd(fhgs_ctx *ctx, const fhgs_gaussians *g, const void *proj, const fhgs_bins *bins,
                          const void *features, const void *feat_gt, fhgs_dtype ftype, int D,
                          const fhgs_camera *cams, int n_cams, const fhgs_params *p, float k, float lambda,
                          const float *grad_Lgt, const float *grad_Lcf, float *grad_means, float *grad_scales,
                          float *grad_quats, float *grad_opac, float *grad_sh, const fhgs_ndfd_state *saved,
                          void *stream) {
    if (!ctx) return FHGS_ERR_INVALID_ARG;
    fhgs_status s = check_gaussians(ctx, g, true);
    if (s == FHGS_OK) s = check_ndfd(ctx, g->n, proj, bins, features, feat_gt, ftype, D, p, k, lambda);
    if (s == FHGS_OK) s = check_ndfd_state(ctx, saved);
    if (s != FHGS_OK) return s;
    if (!grad_Lgt || !grad_Lcf) return fail(ctx, FHGS_ERR_INVALID_ARG, "NULL input buffer");
    if (g->n > 0 && (!grad_means || !grad_scales || !grad_quats || !grad_opac || !grad_sh))
        return fail(ctx, FHGS_ERR_INVALID_ARG, "NULL gradient buffer");
    if (!aligned16(grad_quats)) return fail(ctx, FHGS_ERR_ALIGNMENT, "grad_quats must be 16-byte aligned");
    CamSet cs;
    if ((s = make_cams(ctx, cams, n_cams, cs)) != FHGS_OK) return s;
    FHGS_CUDA(ctx, cudaSetDevice(ctx->device));
    const long long n = g->n, cn = n * n_cams;
    const bool surfel = p->geometry == FHGS_GEOM_SURFEL;
    const size_t per = surfel ? kSurfelG2d : 12;  // footprint-gradient floats per (camera, primitive)
    if ((s = ensure(ctx, ctx->g2d, sizeof(float) * per * (size_t)cn + 256)) != FHGS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    float *g2d = (float *)ctx->g2d.p;
    FHGS_CUDA(ctx, cudaMemsetAsync(g2d, 0, sizeof(float) * per * (size_t)cn, st));
    const Params q = make_params(p);
    ProjView pv = proj_view(const_cast<void *>(proj), cn);
    if (ndfd_use_tc(p, ftype, D)) {
        Prof pr(ctx, surfel ? "ndfd_bwd_tc_surfel" : "ndfd_bwd_tc", st);
        launch_ndfd_bwd_tc(n, cs, q, pv, *bins, (const __nv_bfloat16 *)features, (const __nv_bfloat16 *)feat_gt, D, k,
                           lambda, grad_Lgt, grad_Lcf, g2d, ndfd_state(saved), ctx->status, st);
    } else {
        Prof pr(ctx, surfel ? "ndfd_bwd_surfel" : "ndfd_bwd", st);
        launch_ndfd_bwd(n, cs, q, pv, *bins, features, feat_gt, ftype == FHGS_BF16, D, k, lambda, grad_Lgt,
                        grad_Lcf, g2d, st);
    }
    {
        Prof pb(ctx, "project_bwd", st);
        if (surfel)
            launch_project_surfel_bwd(*g, cs, q, pv, g2d, grad_means, grad_scales, grad_quats, grad_opac, grad_sh, st);
        else
            launch_project_bwd(*g, cs, q, pv, g2d, grad_means, grad_scales, grad_quats, grad_opac, grad_sh, st);
    }
    FHGS_CUDA(ctx, cudaGetLastError());
    return FHGS_OK;
}

fhgs_status fhgs_fuse_features(fhgs_ctx *ctx, const fhgs_gaussians *g, const fhgs_camera *views, int n_views,
                               const float *const *maps, int D, const fhgs_params *p, float *num, float *den,
                               float *out, uint32_t flags, void *stream) {
    if (!ctx) return FHGS_ERR_INVALID_ARG;
    fhgs_status s = check_params(ctx, p);
    if (s == FHGS_OK) s = check_gaussians(ctx, g, true);
    if (s != FHGS_OK) return s;
    if (p->geometry != FHGS_GEOM_EWA) return fail(ctx, FHGS_ERR_UNSUPPORTED, "fusion runs on the EWA geometry");
    if (!views || n_views < 0) return fail(ctx, FHGS_ERR_INVALID_ARG, "bad views");
    if (n_views > 0 && !maps) return fail(ctx, FHGS_ERR_INVALID_ARG, "maps is NULL");
    if (D <= 0 || D % 8) return fail(ctx, FHGS_ERR_UNSUPPORTED, "D must be a positive multiple of 8");
    if (!num || !den) return fail(ctx, FHGS_ERR_INVALID_ARG, "num/den is NULL");
    if ((flags & FHGS_FUSE_FINALIZE) && !out) return fail(ctx, FHGS_ERR_INVALID_ARG, "out is NULL with FINALIZE");
    if (!aligned16(num) || (out && !aligned16(out))) return fail(ctx, FHGS_ERR_ALIGNMENT, "num/out must be 16-byte aligned");
    for (int v = 0; v < n_views; ++v) {
        if (!maps[v]) return fail(ctx, FHGS_ERR_INVALID_ARG, "map " + std::to_string(v) + " is NULL");
        if (!aligned16(maps[v])) return fail(ctx, FHGS_ERR_ALIGNMENT, "map " + std::to_string(v) + " is not 16-byte aligned");
        CamSet tmp;
        if ((s = make_cams(ctx, views + v, 1, tmp)) != FHGS_OK) return s;
    }
    FHGS_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const long long n = g->n;
    if (!(flags & FHGS_FUSE_ACCUMULATE)) {
        FHGS_CUDA(ctx, cudaMemsetAsync(num, 0, sizeof(float) * (size_t)n * D, st));
        FHGS_CUDA(ctx, cudaMemsetAsync(den, 0, sizeof(float) * (size_t)n, st));
    }
    const Params q = make_params(p);
    // tensor cores unless the FP32 path is asked for (needs D % 64 == 0)
    if (p->path == FHGS_PATH_TC && !fuse_tc_dn(D))
        return fail(ctx, FHGS_ERR_UNSUPPORTED, "tensor-core fusion needs D % 64 == 0");
    const bool fuse_tc = p->path != FHGS_PATH_FP32 && fuse_tc_dn(D) != 0;
    // fusion reads no colour: the projection skips the SH
    Params qp = q;
    qp.sh_deg = 0;
    qp.K = 0;
    // Views go through in groups: one projection, one binning pass and one
    // fusion launch per group.  The group shares the binning's fixed costs
    // (the depth sort's passes, the scans, the host read of the instance
    // count) and gives its latency-bound scatter several views' warps at
    // once.  The group is capped by the projection records it needs.
    int group = (int)std::max<long long>(1, std::min<long long>(kFuseGroup, (4ll << 30) / (long long)proj_bytes(n)));
    group = std::min(group, std::max(1, n_views));
    if ((s = ensure(ctx, ctx->fuse_proj, proj_bytes(n * group))) != FHGS_OK) return s;
    if ((s = ensure(ctx, ctx->fuse_count, 256)) != FHGS_OK) return s;
    for (int v0 = 0; v0 < n_views && n > 0;) {
        const int nv = std::min(group, n_views - v0);
        CamSet cs;
        make_cams(ctx, views + v0, nv, cs);
        FuseMaps fm{};
        for (int i = 0; i < nv; ++i) fm.m[i] = maps[v0 + i];
        if ((s = ensure(ctx, ctx->fuse_ranges, sizeof(uint32_t) * 2 * (size_t)cs.total_tiles)) != FHGS_OK) return s;
        ProjView pv = proj_view(ctx->fuse_proj.p, n * nv);
        {
            Prof pr(ctx, "fuse_project", st);
            launch_project(*g, cs, qp, pv, ctx->status, st);
        }
        if ((s = ensure_bin_scratch(ctx, n, nv, cs.total_tiles)) != FHGS_OK) return s;
        BinScratch sc = bin_scratch_view(ctx->bin.p, n, nv, cs.total_tiles, ctx->sm_count);
        fhgs_bins b;
        b.keys = nullptr;
        b.ranges = (uint32_t *)ctx->fuse_ranges.p;
        b.n_instances = (int64_t *)ctx->fuse_count.p;
        // instance capacity: grow until the group's instances fit (reads the
        // count on the host, so fusion is not meant for stream capture); a
        // group whose instances overflow 32-bit offsets is split
        bool split = false;
        for (int tries = 0;; ++tries) {
            if (tries > 3) return fail(ctx, FHGS_ERR_CAPACITY, "instance buffer did not converge");
            if ((s = ensure(ctx, ctx->fuse_gids, sizeof(uint32_t) * 1024)) != FHGS_OK) return s;
            b.gids = (uint32_t *)ctx->fuse_gids.p;
            b.capacity = (long long)(ctx->fuse_gids.bytes / sizeof(uint32_t));
            {
                Prof pr(ctx, "fuse_bin_sort", st);
                launch_bin_sort(n, nv, cs, pv, b, sc, p->list_cut ? &q : nullptr, nullptr, st);
            }
            int64_t count = 0;
            FHGS_CUDA(ctx, cudaMemcpyAsync(&count, b.n_instances, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            FHGS_CUDA(ctx, cudaStreamSynchronize(st));
            if (count <= b.capacity) {
                if (fuse_tc) {
                    Prof pr(ctx, "fuse_tc", st);
                    launch_fuse_tc(n, cs, q, pv, b, fm, D, num, den, ctx->status, st);
                } else {
                    Prof pr(ctx, "fuse_fp32", st);
                    launch_fuse_fp32(n, cs, q, pv, b, fm, D, num, den, st);
                }
                break;
            }
            if (count > 0xFFFFFFFFll) {
                if (nv == 1) return fail(ctx, FHGS_ERR_CAPACITY, "too many instances in one view");
                group = nv / 2;
                split = true;
                break;
            }
            if ((s = ensure(ctx, ctx->fuse_gids, sizeof(uint32_t) * (size_t)(count + count / 8 + 1024))) !=
                FHGS_OK)
                return s;
        }
        FHGS_CUDA(ctx, cudaGetLastError());
        if (!split) v0 += nv;
    }
    if (flags & FHGS_FUSE_FINALIZE) {
        Prof pr(ctx, "fuse_finalize", st);
        launch_fuse_finalize(n, D, num, den, out, (flags & FHGS_FUSE_NORMALIZE) != 0, st);
    }
    FHGS_CUDA(ctx, cudaGetLastError());
    return FHGS_OK;
}

fhgs_status fhgs_profile_enable(fhgs_ctx *ctx, int enable) {
    if (!ctx) return FHGS_ERR_INVALID_ARG;
    FHGS_CUDA(ctx, cudaSetDevice(ctx->device));
    if (enable && ctx->pool.empty()) {
        ctx->pool.resize(kProfEvents);
        for (size_t i = 0; i < kProfEvents; ++i) FHGS_CUDA(ctx, cudaEventCreate(&ctx->pool[i]));
    }
    ctx->prof = enable != 0;
    return FHGS_OK;
}

fhgs_status fhgs_profile_read(fhgs_ctx *ctx, char *buf, int64_t len) {
    if (!ctx || !buf || len < 3) return FHGS_ERR_INVALID_ARG;
    FHGS_CUDA(ctx, cudaSetDevice(ctx->device));
    std::map<std::string, std::pair<long long, double>> agg;
    for (const ProfRec &r : ctx->recs) {
        FHGS_CUDA(ctx, cudaEventSynchronize(r.b));
        float ms = 0.f;
        FHGS_CUDA(ctx, cudaEventElapsedTime(&ms, r.a, r.b));
        auto &e = agg[r.name];
        e.first += 1;
        e.second += ms;
    }
    ctx->recs.clear();
    ctx->pool_next = 0;
    std::string out = "{";
    for (auto &kv : agg) {
        char tmp[160];
        snprintf(tmp, sizeof(tmp), "%s\"%s\": [%lld, %.6f]", out.size() > 1 ? ", " : "", kv.first.c_str(),
                 kv.second.first, kv.second.second);
        out += tmp;
    }
    out += "}";
    strncpy(buf, out.c_str(), (size_t)len - 1);
    buf[len - 1] = 0;
    return FHGS_OK;
}

int64_t fhgs_launch_count(void) { return g_launches.load(); }

}  // extern "C"
