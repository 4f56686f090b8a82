// fhgs_render_bwd_noalloc: the backward for callers that cannot allocate
// device memory: code running inside a custom device allocator or a memory
// pool's callback (which must not re-enter cudaMalloc), plugin hosts that own
// every device allocation and forbid libraries from making their own, and
// steady-state loops that keep allocation out of their hot path.  It is
// fhgs_render_bwd without a context: its one piece of scratch, the per-
// (camera, Gaussian) footprint gradients (12 floats each), lives in the
// file-scope device array below, and so does its status word.  The caller
// still provides every input and output.
//
// The array is reserved by every GPU that loads the library, until the
// process exits; FHGS_NOALLOC_MAX_ENTRIES bounds it (cameras x Gaussians).
#include <mutex>

#include "fhgs_internal.cuh"

using namespace fhgs;

namespace {

__device__ __align__(256) float g_noalloc_g2d[12ll * FHGS_NOALLOC_MAX_ENTRIES];
__device__ __align__(256) unsigned g_noalloc_status;

constexpr int kMaxDevices = 64;

struct DeviceScratch {
    float *g2d = nullptr;
    unsigned *status = nullptr;
    bool ready = false;
};

std::mutex g_mu;
DeviceScratch g_scratch[kMaxDevices];

// Device addresses of the file-scope arrays for the current device.  In host
// code the symbols are host-side stand-ins, not device addresses, so they are
// looked up once per device with cudaGetSymbolAddress while it is current.
fhgs_status scratch_for_current_device(DeviceScratch &out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FHGS_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceScratch &d = g_scratch[dev];
    if (!d.ready) {
        void *g = nullptr, *st = nullptr;
        if (cudaGetSymbolAddress(&g, g_noalloc_g2d) != cudaSuccess) return FHGS_ERR_CUDA;
        if (cudaGetSymbolAddress(&st, g_noalloc_status) != cudaSuccess) return FHGS_ERR_CUDA;
        d.g2d = static_cast<float *>(g);
        d.status = static_cast<unsigned *>(st);
        d.ready = true;
    }
    out = d;
    return FHGS_OK;
}

}  // namespace

extern "C" fhgs_status fhgs_render_bwd_noalloc(const fhgs_gaussians *g, const void *proj, const fhgs_bins *bins,
                                               const void *features, fhgs_dtype ftype, int D,
                                               const fhgs_camera *cams, int n_cams, const fhgs_params *p,
                                               const float *T_final, const int32_t *last, const float *grad_rgb,
                                               const float *grad_feat, float *grad_means, float *grad_scales,
                                               float *grad_quats, float *grad_opac, float *grad_sh,
                                               float *grad_features, void *stream) {
    CamSet cs;
    Params q;
    bool tc = false;
    fhgs_status s = check_bwd_args(nullptr, g, proj, bins, features, ftype, D, cams, n_cams, p, T_final, last,
                                   grad_rgb, grad_feat, grad_means, grad_scales, grad_quats, grad_opac, grad_sh,
                                   grad_features, cs, q, tc);
    if (s != FHGS_OK) return s;
    const long long n = g->n, cn = n * n_cams;
    if (cn > FHGS_NOALLOC_MAX_ENTRIES) return FHGS_ERR_UNSUPPORTED;
    DeviceScratch d;
    if ((s = scratch_for_current_device(d)) != FHGS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // the array keeps the previous call's contents: clear what is accumulated
    if (cudaMemsetAsync(d.g2d, 0, sizeof(float) * 12 * (size_t)cn, st) != cudaSuccess) return FHGS_ERR_CUDA;
    if (grad_features && D > 0 &&
        cudaMemsetAsync(grad_features, 0, sizeof(float) * (size_t)n * D, st) != cudaSuccess)
        return FHGS_ERR_CUDA;
    ProjView pv = proj_view(const_cast<void *>(proj), cn);
    if (tc) {
        if (!launch_render_bwd_tc(n, cs, q, pv, *bins, (const __nv_bfloat16 *)features, D, p->d_split, T_final, last,
                                  grad_rgb, grad_feat, d.g2d, grad_features, d.status, st))
            return FHGS_ERR_CUDA;
    } else
        launch_render_bwd_fp32(n, cs, q, pv, *bins, features, ftype == FHGS_BF16, D, T_final, last, grad_rgb,
                               grad_feat, d.g2d, D > 0 ? grad_features : nullptr, st);
    launch_project_bwd(*g, cs, q, pv, d.g2d, grad_means, grad_scales, grad_quats, grad_opac, grad_sh, st);
    return cudaGetLastError() == cudaSuccess ? FHGS_OK : FHGS_ERR_CUDA;
}

// Reads and clears the allocation-free call's status word on the current
// device, after the stream's work is done.  Host memory only: a stack word.
extern "C" fhgs_status fhgs_noalloc_sync_status(void *stream) {
    DeviceScratch d;
    fhgs_status s = scratch_for_current_device(d);
    if (s != FHGS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned h = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FHGS_ERR_CUDA;
    if (cudaMemcpyAsync(&h, d.status, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return FHGS_ERR_CUDA;
    if (cudaMemsetAsync(d.status, 0, sizeof(unsigned), st) != cudaSuccess) return FHGS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FHGS_ERR_CUDA;
    if (h & ST_TIMEOUT) return FHGS_ERR_TIMEOUT;
    if (h & ST_NUMERIC) return FHGS_ERR_NUMERIC;
    if (h & ST_CAPACITY) return FHGS_ERR_CAPACITY;
    return FHGS_OK;
}
