// Non-differentiable feature driving, NDFD (Sec. 3.2-3.3, App. A "NDFD"):
// the per-pixel losses
//   L_gt = sum_i w_i sigma_i                                     (Eq. 5)
//   L_cf = sum_i sigma_i w_i (W_{i-1} - F_{i-1} . f_i)          (Eq. 6, App. A.1)
// with sigma_i = 1 / (1 + exp(k (cos<f_i, f_gt(p)> - lambda))), over the same
// depth-sorted tile lists and Eq. 4 weights as the render (i = 1 nearest), and
// their derivative through w (Sec. 3.3, App. A.2).  No feature image is
// written: the D-dimensional running feature F lives in registers.
//
// Layout: a block of 8 warps owns one 16-pixel row of a tile; each warp owns
// two adjacent pixels, and lane l holds channels [l*DPL, (l+1)*DPL) of their
// F and f_gt (D = 32 DPL).  Gaussian records and feature rows are staged in
// shared memory 32 at a time.  Per contributor the warp forms the partial
// dot products f_gt . f_i and F . f_i of both pixels, sums them over the
// lanes in one reduce-scatter (10 shuffles for 4 values), and every lane
// then updates the pixel scalars identically.  W_{i-1} = 1 - T_i (the
// weights and the transmittance sum to one).
//
// The backward first walks front to back to rebuild F_N (and T_N, the last
// contributor), then back to front with F_{k-1} = F_k - w_k f_k and the
// suffix G_k = sum_{i>k} sigma_i w_i f_i:
//   dL/dw_k = c_gt sigma_k + c_cf (sigma_k (W_{k-1} - F_{k-1} . f_k)
//             + sum_{i>k} sigma_i w_i - G_k . f_k),
//   dL/dalpha_k = T_k dL/dw_k - (1/(1 - alpha_k)) sum_{i>k} w_i dL/dw_i,
// and the footprint chain of the render backward.  Per-Gaussian footprint
// gradients are summed over the block in shared memory, then added to the
// per-(camera, Gaussian) gradient array with one vector atomic per chunk.
#include "fhgs_internal.cuh"

namespace fhgs {
namespace {

constexpr int kNC = 32;       // Gaussians per shared-memory chunk
constexpr int kWarps = 8;     // warps per block: 16 pixels, one tile row
constexpr int kThreads = 32 * kWarps;

template <int DPL, int BF16>
__device__ __forceinline__ void load_slice(const void *row, int lane, float (&out)[DPL]) {
    if constexpr (BF16) {
        const __nv_bfloat16 *r = reinterpret_cast<const __nv_bfloat16 *>(row) + lane * DPL;
        if constexpr (DPL % 8 == 0) {
#pragma unroll
            for (int q = 0; q < DPL / 8; ++q) {
                const uint4 v = reinterpret_cast<const uint4 *>(r)[q];
                const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float2 f = __bfloat1622float2(h[i]);
                    out[8 * q + 2 * i] = f.x;
                    out[8 * q + 2 * i + 1] = f.y;
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < DPL; ++i) out[i] = __bfloat162float(r[i]);
        }
    } else {
        const float *r = reinterpret_cast<const float *>(row) + lane * DPL;
        if constexpr (DPL % 4 == 0) {
#pragma unroll
            for (int q = 0; q < DPL / 4; ++q) {
                const float4 v = reinterpret_cast<const float4 *>(r)[q];
                out[4 * q] = v.x;
                out[4 * q + 1] = v.y;
                out[4 * q + 2] = v.z;
                out[4 * q + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < DPL; ++i) out[i] = r[i];
        }
    }
}

template <int DPL>
__device__ __forceinline__ float dot_slice(const float (&a)[DPL], const float (&b)[DPL]) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) s = fmaf(a[i], b[i], s);
    return s;
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Sums v[0..3] over the warp; every lane receives the four totals.  Halving
// exchanges (xor 16: two values, xor 8: one) leave lane l with the partial
// of value 2*bit4(l) + bit3(l), which xor 4, 2, 1 complete; lane 8 j then
// holds the total of value j.
__device__ __forceinline__ void warp_allreduce4(float (&v)[4], int lane) {
    const bool u16 = (lane & 16) != 0, u8 = (lane & 8) != 0;
    float k0 = u16 ? v[2] : v[0], k1 = u16 ? v[3] : v[1];
    const float s0 = u16 ? v[0] : v[2], s1 = u16 ? v[1] : v[3];
    k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
    k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
    float k = u8 ? k1 : k0;
    k += __shfl_xor_sync(0xffffffffu, u8 ? k0 : k1, 8);
    k += __shfl_xor_sync(0xffffffffu, k, 4);
    k += __shfl_xor_sync(0xffffffffu, k, 2);
    k += __shfl_xor_sync(0xffffffffu, k, 1);
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = __shfl_sync(0xffffffffu, k, 8 * j);
}

// The same for eight values: lane 4 j holds the total of value j.
__device__ __forceinline__ void warp_allreduce8(float (&v)[8], int lane) {
    const bool u16 = (lane & 16) != 0, u8 = (lane & 8) != 0, u4 = (lane & 4) != 0;
    float a[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float keep = u16 ? v[4 + i] : v[i], send = u16 ? v[i] : v[4 + i];
        a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float b[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float keep = u8 ? a[2 + i] : a[i], send = u8 ? a[i] : a[2 + i];
        b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float k = u4 ? b[1] : b[0];
    k += __shfl_xor_sync(0xffffffffu, u4 ? b[0] : b[1], 4);
    k += __shfl_xor_sync(0xffffffffu, k, 2);
    k += __shfl_xor_sync(0xffffffffu, k, 1);
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __shfl_sync(0xffffffffu, k, 4 * j);
}

__device__ __forceinline__ float ndfd_sigma(float phi, float k, float lam) {
    return 1.f / (1.f + expf(k * (phi - lam)));
}

struct RowCtx {
    int ci;
    long long pix[2];
    bool inside[2];
    float fpx[2], fpy;
    uint32_t s, e;
};

__device__ __forceinline__ RowCtx row_ctx(const CamSet &cs, const uint32_t *ranges, int warp) {
    RowCtx r;
    const int tile = blockIdx.x >> 4, row = blockIdx.x & 15;
    r.ci = cam_of_tile(cs, tile);
    const DevCam &cam = cs.c[r.ci];
    const int lt = tile - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const int py = ty * kTile + row;
    r.fpy = py + 0.5f;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int px = tx * kTile + 2 * warp + p;
        r.inside[p] = px < cam.W && py < cam.H;
        r.pix[p] = cam.pix_off + (long long)py * cam.W + px;
        r.fpx[p] = px + 0.5f;
    }
    r.s = ranges[2 * tile];
    r.e = ranges[2 * tile + 1];
    return r;
}

// Stages Gaussians [base, base + nb) of the list: records, ids, feature rows
// and the inverse feature norms (0 for a zero row).
template <int DPL, int BF16>
__device__ __forceinline__ void stage_chunk(const GRec *rec, const uint32_t *gids, uint32_t base, int nb,
                                            const void *feats, char *sfeat, float4 *sa, float4 *sb, uint32_t *sg,
                                            float *sinv, int warp, int lane) {
    constexpr int D = 32 * DPL;
    constexpr int kRowBytes = D * (BF16 ? 2 : 4);
    constexpr int kRowQ = kRowBytes / 16;
    const int tid = threadIdx.x;
    if (tid < nb) {
        const uint32_t g = gids[base + tid];
        const GRec r = rec[g];
        sa[tid] = r.a;
        sb[tid] = r.b;
        sg[tid] = g;
    }
    for (int c = tid; c < nb * kRowQ; c += kThreads) {
        const int row = c / kRowQ, q = c - row * kRowQ;
        const uint4 *src = reinterpret_cast<const uint4 *>(reinterpret_cast<const char *>(feats) +
                                                           (size_t)gids[base + row] * kRowBytes);
        reinterpret_cast<uint4 *>(sfeat + row * kRowBytes)[q] = src[q];
    }
    __syncthreads();
    for (int row = warp; row < nb; row += kWarps) {
        float f[DPL];
        load_slice<DPL, BF16>(sfeat + row * kRowBytes, lane, f);
        const float n2 = warp_sum(dot_slice<DPL>(f, f));
        if (lane == 0) sinv[row] = n2 > 0.f ? 1.f / sqrtf(n2) : 0.f;
    }
    __syncthreads();
}

// alpha of one Gaussian at a pixel, exactly as the render takes it:
// q2 <= cutoff, alpha = min(alpha_max, op G) >= alpha_min.
__device__ __forceinline__ bool ndfd_alpha(const Params &p, float4 A, float4 B, float fpx, float fpy, float &a,
                                           float &G, float &rho) {
    const float dx = fpx - A.x, dy = fpy - A.y;
    const float q2 = eval_q2(dx, dy, A.z, A.w, B.x);
    if (q2 > p.cut) return false;
    G = __expf(-0.5f * q2);
    rho = B.y * G;
    a = fminf(p.amax, rho);
    return a >= p.amin;
}

template <int DPL, int BF16>
__global__ void __launch_bounds__(kThreads, 2) k_ndfd_fwd(long long N, CamSet cs, Params p, ProjView pv,
                                                        const uint32_t *__restrict__ gids,
                                                        const uint32_t *__restrict__ ranges, const void *feats,
                                                        const void *fgt, float ks, float lam, float *Lgt_out,
                                                        float *Lcf_out, int32_t *nc_out) {
    constexpr int D = 32 * DPL;
    constexpr int kRowBytes = D * (BF16 ? 2 : 4);
    extern __shared__ __align__(16) char sfeat[];
    __shared__ float4 sa[kNC], sb[kNC];
    __shared__ uint32_t sg[kNC];
    __shared__ float sinv[kNC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const RowCtx rc = row_ctx(cs, ranges, warp);
    const GRec *rec = pv.rec + (long long)rc.ci * N;

    float F[2][DPL], g[2][DPL], igt[2], T[2], Lgt[2], Lcf[2];
    int nc[2] = {0, 0};
    bool done[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        done[q] = !rc.inside[q];
        T[q] = 1.f;
        Lgt[q] = Lcf[q] = 0.f;
#pragma unroll
        for (int i = 0; i < DPL; ++i) F[q][i] = g[q][i] = 0.f;
        if (rc.inside[q]) load_slice<DPL, BF16>(reinterpret_cast<const char *>(fgt) + rc.pix[q] * kRowBytes, lane, g[q]);
        const float n2 = warp_sum(dot_slice<DPL>(g[q], g[q]));
        igt[q] = n2 > 0.f ? 1.f / sqrtf(n2) : 0.f;
    }

    for (uint32_t base = rc.s; base < rc.e; base += kNC) {
        if (__syncthreads_and(done[0] && done[1])) break;
        const int nb = (int)min((uint32_t)kNC, rc.e - base);
        stage_chunk<DPL, BF16>(rec, gids, base, nb, feats, sfeat, sa, sb, sg, sinv, warp, lane);
        for (int j = 0; j < nb; ++j) {
            if (done[0] && done[1]) break;
            const float4 A = sa[j], B = sb[j];
            bool c[2];
            float a[2], Tn[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                float G, rho;
                c[q] = !done[q] && ndfd_alpha(p, A, B, rc.fpx[q], rc.fpy, a[q], G, rho);
                if (c[q]) {
                    Tn[q] = T[q] * (1.f - a[q]);
                    if (Tn[q] < p.teps) {
                        done[q] = true;
                        c[q] = false;
                    }
                }
            }
            if (!c[0] && !c[1]) continue;
            float f[DPL];
            load_slice<DPL, BF16>(sfeat + j * kRowBytes, lane, f);
            float v[4] = {dot_slice<DPL>(g[0], f), dot_slice<DPL>(F[0], f), dot_slice<DPL>(g[1], f),
                          dot_slice<DPL>(F[1], f)};
            warp_allreduce4(v, lane);
            const float inv = sinv[j];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (!c[q]) continue;
                const float w = a[q] * T[q];
                const float sg_ = ndfd_sigma(v[2 * q] * inv * igt[q], ks, lam);
                Lgt[q] = fmaf(w, sg_, Lgt[q]);
                Lcf[q] = fmaf(sg_ * w, (1.f - T[q]) - v[2 * q + 1], Lcf[q]);
#pragma unroll
                for (int i = 0; i < DPL; ++i) F[q][i] = fmaf(w, f[i], F[q][i]);
                T[q] = Tn[q];
                ++nc[q];
            }
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 2; ++q)
            if (rc.inside[q]) {
                Lgt_out[rc.pix[q]] = Lgt[q];
                Lcf_out[rc.pix[q]] = Lcf[q];
                if (nc_out) nc_out[rc.pix[q]] = nc[q];
            }
    }
}

template <int DPL, int BF16>
__global__ void __launch_bounds__(kThreads, 1) k_ndfd_bwd(long long N, CamSet cs, Params p, ProjView pv,
                                                        const uint32_t *__restrict__ gids,
                                                        const uint32_t *__restrict__ ranges, const void *feats,
                                                        const void *fgt, float ks, float lam,
                                                        const float *__restrict__ dLgt,
                                                        const float *__restrict__ dLcf, float *g2d) {
    constexpr int D = 32 * DPL;
    constexpr int kRowBytes = D * (BF16 ? 2 : 4);
    extern __shared__ __align__(16) char sfeat[];
    __shared__ float4 sa[kNC], sb[kNC];
    __shared__ uint32_t sg[kNC];
    __shared__ float sinv[kNC];
    __shared__ __align__(16) float sacc[kNC][8];
    __shared__ int smax;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const RowCtx rc = row_ctx(cs, ranges, warp);
    const GRec *rec = pv.rec + (long long)rc.ci * N;
    float *g2dc = g2d + (long long)rc.ci * N * 12;

    float F[2][DPL], T[2];
    int last[2];
    bool done[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        done[q] = !rc.inside[q];
        T[q] = 1.f;
        last[q] = 0;
#pragma unroll
        for (int i = 0; i < DPL; ++i) F[q][i] = 0.f;
    }
    if (threadIdx.x == 0) smax = 0;
    for (int i = threadIdx.x; i < kNC * 8; i += kThreads) (&sacc[0][0])[i] = 0.f;

    // front to back: F_N, T_N and the last contributor of each pixel
    for (uint32_t base = rc.s; base < rc.e; base += kNC) {
        if (__syncthreads_and(done[0] && done[1])) break;
        const int nb = (int)min((uint32_t)kNC, rc.e - base);
        stage_chunk<DPL, BF16>(rec, gids, base, nb, feats, sfeat, sa, sb, sg, sinv, warp, lane);
        for (int j = 0; j < nb; ++j) {
            if (done[0] && done[1]) break;
            const float4 A = sa[j], B = sb[j];
            bool c[2];
            float a[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                float G, rho;
                c[q] = !done[q] && ndfd_alpha(p, A, B, rc.fpx[q], rc.fpy, a[q], G, rho);
                if (c[q] && T[q] * (1.f - a[q]) < p.teps) {
                    done[q] = true;
                    c[q] = false;
                }
            }
            if (!c[0] && !c[1]) continue;
            float f[DPL];
            load_slice<DPL, BF16>(sfeat + j * kRowBytes, lane, f);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (!c[q]) continue;
                const float w = a[q] * T[q];
#pragma unroll
                for (int i = 0; i < DPL; ++i) F[q][i] = fmaf(w, f[i], F[q][i]);
                T[q] *= 1.f - a[q];
                last[q] = (int)(base - rc.s) + j + 1;
            }
        }
    }

    // back to front
    float g[2][DPL], Gs[2][DPL], igt[2], cgt[2], ccf[2], Ss[2], Sw[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
#pragma unroll
        for (int i = 0; i < DPL; ++i) g[q][i] = Gs[q][i] = 0.f;
        cgt[q] = ccf[q] = 0.f;
        if (rc.inside[q]) {
            load_slice<DPL, BF16>(reinterpret_cast<const char *>(fgt) + rc.pix[q] * kRowBytes, lane, g[q]);
            cgt[q] = dLgt[rc.pix[q]];
            ccf[q] = dLcf[rc.pix[q]];
        }
        const float n2 = warp_sum(dot_slice<DPL>(g[q], g[q]));
        igt[q] = n2 > 0.f ? 1.f / sqrtf(n2) : 0.f;
        Ss[q] = Sw[q] = 0.f;
    }
    __syncthreads();
    if (lane == 0) atomicMax(&smax, max(last[0], last[1]));
    __syncthreads();
    const int Lmax = min(smax, (int)(rc.e - rc.s));
    for (int bend = Lmax; bend > 0; bend -= kNC) {
        const int bstart = max(0, bend - kNC), nb = bend - bstart;
        __syncthreads();
        stage_chunk<DPL, BF16>(rec, gids, rc.s + bstart, nb, feats, sfeat, sa, sb, sg, sinv, warp, lane);
        for (int j = nb - 1; j >= 0; --j) {
            const float4 A = sa[j], B = sb[j];
            bool c[2];
            float a[2], G[2], rho[2];
#pragma unroll
            for (int q = 0; q < 2; ++q)
                c[q] = bstart + j < last[q] && ndfd_alpha(p, A, B, rc.fpx[q], rc.fpy, a[q], G[q], rho[q]);
            if (!c[0] && !c[1]) continue;
            float f[DPL];
            load_slice<DPL, BF16>(sfeat + j * kRowBytes, lane, f);
            float w[2] = {0.f, 0.f};
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (!c[q]) continue;
                T[q] = T[q] / (1.f - a[q]);
                w[q] = a[q] * T[q];
#pragma unroll
                for (int i = 0; i < DPL; ++i) F[q][i] = fmaf(-w[q], f[i], F[q][i]);
            }
            float v[8] = {dot_slice<DPL>(g[0], f), dot_slice<DPL>(F[0], f), dot_slice<DPL>(Gs[0], f),
                          dot_slice<DPL>(g[1], f), dot_slice<DPL>(F[1], f), dot_slice<DPL>(Gs[1], f), 0.f, 0.f};
            warp_allreduce8(v, lane);
            const float inv = sinv[j];
            float geo[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (!c[q]) continue;
                const float sig = ndfd_sigma(v[3 * q] * inv * igt[q], ks, lam);
                const float gw = cgt[q] * sig + ccf[q] * (sig * ((1.f - T[q]) - v[3 * q + 1]) + Ss[q] - v[3 * q + 2]);
                const float oma = 1.f - a[q];
                const float dal = T[q] * gw - Sw[q] / oma;
                Sw[q] = fmaf(w[q], gw, Sw[q]);
                const float sw = sig * w[q];
                Ss[q] += sw;
#pragma unroll
                for (int i = 0; i < DPL; ++i) Gs[q][i] = fmaf(sw, f[i], Gs[q][i]);
                const float drho = rho[q] > p.amax ? 0.f : dal;
                const float dq2 = -0.5f * rho[q] * drho;
                const float dx = rc.fpx[q] - A.x, dy = rc.fpy - A.y;
                geo[0] -= (2.f * A.z * dx + 2.f * A.w * dy) * dq2;
                geo[1] -= (2.f * A.w * dx + 2.f * B.x * dy) * dq2;
                geo[2] += dx * dx * dq2;
                geo[3] += 2.f * dx * dy * dq2;
                geo[4] += dy * dy * dq2;
                geo[5] += G[q] * drho;
            }
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < 6; ++k) atomicAdd(&sacc[j][k], geo[k]);
            }
        }
        __syncthreads();
        if ((int)threadIdx.x < nb) {
            const int j = threadIdx.x;
            const float4 u = *reinterpret_cast<const float4 *>(&sacc[j][0]);
            const float2 t = *reinterpret_cast<const float2 *>(&sacc[j][4]);
            if (u.x != 0.f || u.y != 0.f || u.z != 0.f || u.w != 0.f || t.x != 0.f || t.y != 0.f) {
                float *dst = g2dc + 12 * (long long)sg[j];
                atomicAdd(reinterpret_cast<float4 *>(dst), u);
                atomicAdd(reinterpret_cast<float2 *>(dst + 4), t);
            }
            *reinterpret_cast<float4 *>(&sacc[j][0]) = make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float2 *>(&sacc[j][4]) = make_float2(0.f, 0.f);
        }
    }
}

template <int DPL, int BF16>
void launch_fwd_t(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                  const void *feats, const void *fgt, float ks, float lam, float *Lgt, float *Lcf, int32_t *nc,
                  cudaStream_t st) {
    static std::atomic<unsigned long long> smem_set{0};
    const int smem = kNC * 32 * DPL * (BF16 ? 2 : 4);
    allow_max_smem(smem_set, k_ndfd_fwd<DPL, BF16>);
    note_launch(1);
    k_ndfd_fwd<DPL, BF16><<<(unsigned)cs.total_tiles * 16, kThreads, smem, st>>>(
        N, cs, p, pv, bins.gids, bins.ranges, feats, fgt, ks, lam, Lgt, Lcf, nc);
}

template <int DPL, int BF16>
void launch_bwd_t(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                  const void *feats, const void *fgt, float ks, float lam, const float *dLgt, const float *dLcf,
                  float *g2d, cudaStream_t st) {
    static std::atomic<unsigned long long> smem_set{0};
    const int smem = kNC * 32 * DPL * (BF16 ? 2 : 4);
    allow_max_smem(smem_set, k_ndfd_bwd<DPL, BF16>);
    note_launch(1);
    k_ndfd_bwd<DPL, BF16><<<(unsigned)cs.total_tiles * 16, kThreads, smem, st>>>(
        N, cs, p, pv, bins.gids, bins.ranges, feats, fgt, ks, lam, dLgt, dLcf, g2d);
}

}  // namespace

bool ndfd_supported(int D) { return D == 32 || D == 64 || D == 128 || D == 256 || D == 512; }

#define FHGS_NDFD_CASES(X, BF) \
    X(1, BF) X(2, BF) X(4, BF) X(8, BF) X(16, BF)

void launch_ndfd_fwd(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                     const void *feats, const void *fgt, int bf16, int D, float ks, float lam, float *Lgt,
                     float *Lcf, int32_t *nc, cudaStream_t st) {
    if (cs.total_tiles == 0) return;
#define X(DPL, BF)                                                                            \
    if (D == 32 * DPL && bf16 == BF) {                                                        \
        launch_fwd_t<DPL, BF>(N, cs, p, pv, bins, feats, fgt, ks, lam, Lgt, Lcf, nc, st);     \
        return;                                                                               \
    }
    FHGS_NDFD_CASES(X, 0)
    FHGS_NDFD_CASES(X, 1)
#undef X
}

void launch_ndfd_bwd(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                     const void *feats, const void *fgt, int bf16, int D, float ks, float lam, const float *dLgt,
                     const float *dLcf, float *g2d, cudaStream_t st) {
    if (cs.total_tiles == 0) return;
#define X(DPL, BF)                                                                                  \
    if (D == 32 * DPL && bf16 == BF) {                                                              \
        launch_bwd_t<DPL, BF>(N, cs, p, pv, bins, feats, fgt, ks, lam, dLgt, dLcf, g2d, st);        \
        return;                                                                                     \
    }
    FHGS_NDFD_CASES(X, 0)
    FHGS_NDFD_CASES(X, 1)
#undef X
}

}  // namespace fhgs
