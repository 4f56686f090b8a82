// The paper's point-to-feature assignment (Sec. 3.1; App. A,
// "PointsFeatureFusion"): every point takes the feature of the pixel it
// projects to in one view, drawn among the views that see it.
//
// A view sees a point when its camera depth exceeds znear and the projection
// lies inside the image; the pixel is (floor x, floor y).  The draw is the
// k-th visible view in view order, k = floor(u |M|) for the caller's uniform
// u.  The projection decides integers, so it is evaluated in binary32 with
// one rounding per operation in a fixed order (explicit _rn intrinsics, no
// contraction):  c_r = ((R_r0 X + R_r1 Y) + R_r2 Z) + t_r,
// x = fx (c_x / c_z) + cx,  y = fy (c_y / c_z) + cy.
//
// One thread per point projects it into every view twice (count, then the
// k-th); the paper's SfM spatial hash is not needed for O(N V) projections.
// The warp then copies its 32 points' feature rows one after another with
// float4 loads and stores, so that each row moves as contiguous bytes.
#include "fhgs_internal.cuh"

namespace fhgs {
namespace {

__device__ __forceinline__ bool pf_visible(const PFView &c, float X, float Y, float Z, float znear, int &pix) {
    const float *R = c.cam + 6;
    const float cx = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(R[0], X), __fmul_rn(R[1], Y)), __fmul_rn(R[2], Z)), R[3]);
    const float cy = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(R[4], X), __fmul_rn(R[5], Y)), __fmul_rn(R[6], Z)), R[7]);
    const float cz =
        __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(R[8], X), __fmul_rn(R[9], Y)), __fmul_rn(R[10], Z)), R[11]);
    if (!(cz > znear)) return false;
    const float x = __fadd_rn(__fmul_rn(c.cam[2], __fdiv_rn(cx, cz)), c.cam[4]);
    const float y = __fadd_rn(__fmul_rn(c.cam[3], __fdiv_rn(cy, cz)), c.cam[5]);
    if (!(x >= 0.f && x < c.cam[0] && y >= 0.f && y < c.cam[1])) return false;
    pix = (int)floorf(y) * (int)c.cam[0] + (int)floorf(x);
    return true;
}

__global__ void __launch_bounds__(256) k_point_features(long long n, const float *__restrict__ means,
                                                        const PFView *__restrict__ views, int n_views, float znear,
                                                        const float *__restrict__ u, int D, float *out,
                                                        int32_t *view_out, int32_t *pix_out) {
    const int lane = threadIdx.x & 31;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int view = -1, pix = -1;
    if (i < n) {
        const float X = means[3 * i], Y = means[3 * i + 1], Z = means[3 * i + 2];
        int count = 0, px;
        for (int v = 0; v < n_views; ++v) count += pf_visible(views[v], X, Y, Z, znear, px) ? 1 : 0;
        if (count > 0) {
            int k = (int)__fmul_rn(u[i], (float)count);
            k = min(max(k, 0), count - 1);
            for (int v = 0; v < n_views; ++v) {
                if (!pf_visible(views[v], X, Y, Z, znear, px)) continue;
                if (k-- == 0) {
                    view = v;
                    pix = px;
                    break;
                }
            }
        }
        if (view_out) view_out[i] = view;
        if (pix_out) pix_out[i] = pix;
    }
    const long long i0 = i - lane;
    const int q = D >> 2;  // float4 words per row
    for (int l = 0; l < 32; ++l) {
        const long long ii = i0 + l;
        if (ii >= n) break;  // warp-uniform
        const int vv = __shfl_sync(0xffffffffu, view, l), pp = __shfl_sync(0xffffffffu, pix, l);
        float4 *dst = reinterpret_cast<float4 *>(out + ii * D);
        if (vv < 0) {
            for (int c = lane; c < q; c += 32) dst[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            const float4 *src = reinterpret_cast<const float4 *>(views[vv].map + (long long)pp * D);
            for (int c = lane; c < q; c += 32) dst[c] = src[c];
        }
    }
}

}  // namespace

void launch_point_features(long long n, const float *means, const PFView *views, int n_views, float znear,
                           const float *u, int D, float *out, int32_t *view, int32_t *pixel, cudaStream_t st) {
    if (n == 0) return;
    note_launch(1);
    const unsigned blocks = (unsigned)((n + 255) / 256);
    k_point_features<<<blocks, 256, 0, st>>>(n, means, views, n_views, znear, u, D, out, view, pixel);
}

}  // namespace fhgs
