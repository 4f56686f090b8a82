// Non-differentiable feature driving, NDFD (Sec. 3.2-3.3, App. A "NDFD"):
// the per-pixel losses
//   L_gt = sum_i w_i sigma_i                                     (Eq. 5)
//   L_cf = sum_i sigma_i w_i (W_{i-1} - F_{i-1} . f_i)          (Eq. 6, App. A.1)
// with sigma_i = 1 / (1 + exp(k (cos<f_i, f_gt(p)> - lambda))), over the same
// depth-sorted tile lists and Eq. 4 weights as the render (i = 1 nearest), and
// their derivative through w (Sec. 3.3, App. A.2).  No feature image is
// written: the D-dimensional running feature F lives in registers.
//
// Layout.  A block of 8 warps owns one 16-pixel row of a tile; each warp owns
// two adjacent pixels.  Lane l holds channels {128 k + 4 l + r} (DPL = D/32
// of them) of the two pixels' F and f_gt, so that a warp's float4 reads of a
// feature row cover contiguous bytes.  Gaussian records and feature rows
// (converted to FP32) are staged in shared memory 32 at a time.
//
// Per chunk, lane j first decides alpha_j of entry j for both pixels (the
// render's cutoff, alpha_min and alpha_max rules); an inclusive prefix
// product over the lanes gives T_j, the stop rule (T_j (1 - alpha_j) < t_eps)
// becomes the first set bit of a ballot, and w_j = alpha_j T_j.  W_{i-1} =
// 1 - T_i (weights and transmittance sum to one).  The feature work then
// visits only the contributors, four at a time: per contributor each lane
// adds its channels' share of f_gt . f_i and F . f_i of both pixels to 16
// partial sums and updates F += w_i f_i; one 16-value reduce-scatter (16
// shuffles) completes the four contributors' dot products, and the lanes
// that hold them accumulate L_gt and L_cf.
//
// The backward runs one pixel per warp (16 warps per block, a register
// budget of 128 per thread).  It rebuilds F_N front to back the same way,
// then walks back to front, two contributors k at a time, with
// F_{k-1} = F_k - w_k f_k and the suffix G = sum_{i>k} sigma_i w_i f_i:
//   dL/dw_k = c_gt sigma_k + c_cf (sigma_k (W_{k-1} - F_{k-1} . f_k)
//             + sum_{i>k} sigma_i w_i - G . f_k),
//   dL/dalpha_k = T_k dL/dw_k - (1/(1 - alpha_k)) sum_{i>k} w_i dL/dw_i,
// and the footprint chain of the render backward.  Inside a pair the later
// contributor's share of G enters the earlier one's G . f_k through the
// pair's Gram entry f_i . f_k.  T_k comes from T after the chunk divided by a
// suffix product of (1 - alpha).  Per-Gaussian footprint gradients are summed
// over the block in shared memory, then added to the per-(camera, Gaussian)
// gradient array with one vector atomic per chunk.
#include "fhgs_internal.cuh"

namespace fhgs {
namespace {

constexpr int kNC = 32;       // Gaussians per shared-memory chunk (one per lane)
constexpr int kWarps = 8;     // warps per block: 16 pixels, one tile row
constexpr int kThreads = 32 * kWarps;
constexpr unsigned kFull = 0xffffffffu;

// Channel c of lane `lane`, slot i:  DPL >= 4: 128 (i/4) + 4 lane + i%4;
// DPL = 2: 2 lane + i;  DPL = 1: lane.
template <int DPL>
__device__ __forceinline__ int chan(int lane, int i) {
    if constexpr (DPL >= 4) return 128 * (i >> 2) + 4 * lane + (i & 3);
    else return DPL * lane + i;
}

// The lane's channels of an FP32 row (shared or global memory).
template <int DPL>
__device__ __forceinline__ void load_row_f32(const float *row, int lane, float (&out)[DPL]) {
    if constexpr (DPL >= 4) {
#pragma unroll
        for (int k = 0; k < DPL / 4; ++k) {
            const float4 v = *reinterpret_cast<const float4 *>(row + 128 * k + 4 * lane);
            out[4 * k] = v.x;
            out[4 * k + 1] = v.y;
            out[4 * k + 2] = v.z;
            out[4 * k + 3] = v.w;
        }
    } else if constexpr (DPL == 2) {
        const float2 v = *reinterpret_cast<const float2 *>(row + 2 * lane);
        out[0] = v.x;
        out[1] = v.y;
    } else {
        out[0] = row[lane];
    }
}

// The lane's channels of a global row of `features`' dtype.
template <int DPL, int BF16>
__device__ __forceinline__ void load_row_g(const void *row, int lane, float (&out)[DPL]) {
    if constexpr (!BF16) {
        load_row_f32<DPL>(reinterpret_cast<const float *>(row), lane, out);
    } else {
        const __nv_bfloat16 *r = reinterpret_cast<const __nv_bfloat16 *>(row);
        if constexpr (DPL >= 4) {
#pragma unroll
            for (int k = 0; k < DPL / 4; ++k) {
                const uint2 v = *reinterpret_cast<const uint2 *>(r + 128 * k + 4 * lane);
                const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.x));
                const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.y));
                out[4 * k] = a.x;
                out[4 * k + 1] = a.y;
                out[4 * k + 2] = b.x;
                out[4 * k + 3] = b.y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < DPL; ++i) out[i] = __bfloat162float(r[chan<DPL>(lane, i)]);
        }
    }
}

template <int DPL>
__device__ __forceinline__ float dot_slice(const float (&a)[DPL], const float (&b)[DPL]) {
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int i = 0; i < DPL; i += 2) {
        s0 = fmaf(a[i], b[i], s0);
        if (i + 1 < DPL) s1 = fmaf(a[i + 1], b[i + 1], s1);
    }
    return s0 + s1;
}

template <int DPL>
__device__ __forceinline__ void axpy_slice(float w, const float (&f)[DPL], float (&y)[DPL]) {
#pragma unroll
    for (int i = 0; i < DPL; ++i) y[i] = fmaf(w, f[i], y[i]);
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// One halving step of a reduce-scatter: lanes with `bit` set keep the upper
// half of v and send the lower half to their partner (lane ^ bit), which
// keeps the lower half.
template <int H>
__device__ __forceinline__ void rs_step(const float *v, float *out, int lane, int bit) {
    const bool up = (lane & bit) != 0;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const float keep = up ? v[H + i] : v[i], send = up ? v[i] : v[H + i];
        out[i] = keep + __shfl_xor_sync(kFull, send, bit);
    }
}

// Sums 16 per-lane values over the warp; lane l receives the total of value
// l >> 1 (16 shuffles).
__device__ __forceinline__ float warp_rs16(const float (&v)[16], int lane) {
    float a[8], b[4], c[2], d[1];
    rs_step<8>(v, a, lane, 16);
    rs_step<4>(a, b, lane, 8);
    rs_step<2>(b, c, lane, 4);
    rs_step<1>(c, d, lane, 2);
    return d[0] + __shfl_xor_sync(kFull, d[0], 1);
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

// Stages Gaussians [base, base + nb) of the list: records (a, b of the EWA
// record; a, b, c of the surfel record), ids, feature rows
// as FP32 (row-major, D floats per row) and the inverse feature norms (0 for
// a zero row).  Ends with a block barrier.
template <int DPL, int BF16, int GEOM, int NT = kThreads>
__device__ __forceinline__ void stage_chunk(const void *rec, const uint32_t *gids, uint32_t base, int nb,
                                            const void *feats, float *sf, float4 *sa, float4 *sb, float4 *sc,
                                            uint32_t *sg, float *sinv, int warp, int lane) {
    constexpr int D = 32 * DPL;
    constexpr int kRowQ = D * (BF16 ? 2 : 4) / 16;  // 16-byte words per source row
    const int tid = threadIdx.x;
    if (tid < nb) {
        const uint32_t g = gids[base + tid];
        if constexpr (GEOM == FHGS_GEOM_EWA) {
            const GRec r = static_cast<const GRec *>(rec)[g];
            sa[tid] = r.a;
            sb[tid] = r.b;
        } else {
            const SRec r = static_cast<const SRec *>(rec)[g];
            sa[tid] = r.a;
            sb[tid] = r.b;
            sc[tid] = r.c;
        }
        sg[tid] = g;
    }
    for (int c = tid; c < nb * kRowQ; c += NT) {
        const int row = c / kRowQ, q = c - row * kRowQ;
        const uint4 v = reinterpret_cast<const uint4 *>(reinterpret_cast<const char *>(feats) +
                                                        (size_t)gids[base + row] * (kRowQ * 16))[q];
        if constexpr (BF16) {
            float4 *dst = reinterpret_cast<float4 *>(sf + row * D + 8 * q);
            const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.x));
            const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.y));
            const float2 c2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.z));
            const float2 d = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.w));
            dst[0] = make_float4(a.x, a.y, b.x, b.y);
            dst[1] = make_float4(c2.x, c2.y, d.x, d.y);
        } else {
            reinterpret_cast<uint4 *>(sf + row * D)[q] = v;
        }
    }
    __syncthreads();
    for (int row = warp; row < nb; row += NT / 32) {
        float f[DPL];
        load_row_f32<DPL>(sf + row * D, lane, f);
        const float n2 = warp_sum(dot_slice<DPL>(f, f));
        if (lane == 0) sinv[row] = n2 > 0.f ? 1.f / sqrtf(n2) : 0.f;
    }
    __syncthreads();
}

// alpha of one primitive at a pixel, exactly as the render takes it: EWA,
// q2 <= cutoff on the conic; a 2DGS surfel, u^2 + v^2 <= cutoff at the
// ray-plane intersection (Sec. 3.1, Eq. 1-3); then G = exp(-r^2 / 2) and
// alpha = min(alpha_max, op G) >= alpha_min.
template <int GEOM>
__device__ __forceinline__ bool ndfd_alpha(const Params &p, float4 A, float4 B, float4 C, float fpx, float fpy,
                                           float &a, float &G, float &rho) {
    if constexpr (GEOM == FHGS_GEOM_EWA) {
        const float dx = fpx - A.x, dy = fpy - A.y;
        const float q2 = eval_q2(dx, dy, A.z, A.w, B.x);
        if (q2 > p.cut) return false;
        G = __expf(-0.5f * q2);
        rho = B.y * G;
    } else {
        SurfelHit h;
        if (!surfel_uv(A, B, C.x, fpx, fpy, p.cut, h)) return false;
        G = __expf(-0.5f * h.r2);
        rho = C.y * G;
    }
    a = fminf(p.amax, rho);
    return a >= p.amin;
}

// Front-to-back decisions of one chunk for pixel q, lane j <-> entry j:
// given contrib (alpha test passed, pixel not yet done) and alpha, returns
// the contributor mask (entries before the stop), this lane's weight w_j
// and transmittance before it T_j, and advances T / done.
__device__ __forceinline__ unsigned chunk_weights(bool contrib, float a, float teps, int lane, float &T, bool &done,
                                                  float &w, float &Tj) {
    float inc = contrib ? 1.f - a : 1.f;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const float t = __shfl_up_sync(kFull, inc, d);
        if (lane >= d) inc *= t;
    }
    float ex = __shfl_up_sync(kFull, inc, 1);
    if (lane == 0) ex = 1.f;
    Tj = T * ex;
    const unsigned stop = __ballot_sync(kFull, contrib && T * inc < teps);
    const unsigned before = stop ? (1u << (__ffs(stop) - 1)) - 1u : kFull;
    const unsigned m = __ballot_sync(kFull, contrib) & before;
    w = (m >> lane) & 1u ? a * Tj : 0.f;
    const float Tstop = __shfl_sync(kFull, Tj, stop ? __ffs(stop) - 1 : 0);
    const float Tall = __shfl_sync(kFull, inc, 31);
    if (stop) {
        done = true;
        T = Tstop;
    } else {
        T *= Tall;
    }
    return m;
}

template <int DPL, int BF16, int GEOM>
__global__ void __launch_bounds__(kThreads, 2) k_ndfd_fwd(long long N, CamSet cs, Params p, ProjView pv,
                                                        const uint32_t *__restrict__ gids,
                                                        const uint32_t *__restrict__ ranges, const void *feats,
                                                        const void *fgt, float ks, float lam, float *Lgt_out,
                                                        float *Lcf_out, int32_t *nc_out) {
    constexpr int D = 32 * DPL;
    constexpr int kGtRowBytes = D * (BF16 ? 2 : 4);
    extern __shared__ __align__(16) float sf[];
    __shared__ float4 sa[kNC], sb[kNC], sc[kNC];
    __shared__ uint32_t sg[kNC];
    __shared__ float sinv[kNC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const RowCtx rc = row_ctx(cs, ranges, warp);
    const void *rec = GEOM == FHGS_GEOM_EWA ? static_cast<const void *>(pv.rec + (long long)rc.ci * N)
                                            : static_cast<const void *>(pv.srec + (long long)rc.ci * N);

    float F0[DPL], F1[DPL], g0[DPL], g1[DPL], igt[2], T[2] = {1.f, 1.f};
    int nc[2] = {0, 0};
    bool done[2] = {!rc.inside[0], !rc.inside[1]};
#pragma unroll
    for (int i = 0; i < DPL; ++i) F0[i] = F1[i] = g0[i] = g1[i] = 0.f;
    if (rc.inside[0]) load_row_g<DPL, BF16>(reinterpret_cast<const char *>(fgt) + rc.pix[0] * kGtRowBytes, lane, g0);
    if (rc.inside[1]) load_row_g<DPL, BF16>(reinterpret_cast<const char *>(fgt) + rc.pix[1] * kGtRowBytes, lane, g1);
    {
        const float n0 = warp_sum(dot_slice<DPL>(g0, g0)), n1 = warp_sum(dot_slice<DPL>(g1, g1));
        igt[0] = n0 > 0.f ? 1.f / sqrtf(n0) : 0.f;
        igt[1] = n1 > 0.f ? 1.f / sqrtf(n1) : 0.f;
    }
    // lanes l with l % 4 == 0 accumulate the terms of pixel (l >> 2) & 1
    float acc_gt = 0.f, acc_cf = 0.f;
    const int my_slot = lane >> 3, my_q = (lane >> 2) & 1;

    for (uint32_t base = rc.s; base < rc.e; base += kNC) {
        if (__syncthreads_and(done[0] && done[1])) break;
        const int nb = (int)min((uint32_t)kNC, rc.e - base);
        stage_chunk<DPL, BF16, GEOM>(rec, gids, base, nb, feats, sf, sa, sb, sc, sg, sinv, warp, lane);
        float a[2] = {0.f, 0.f};
        bool c[2] = {false, false};
        if (lane < nb) {
            const float4 A = sa[lane], B = sb[lane], Cc = sc[lane];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                float G, rho;
                c[q] = !done[q] && ndfd_alpha<GEOM>(p, A, B, Cc, rc.fpx[q], rc.fpy, a[q], G, rho);
            }
        }
        float wl[2], Tl[2];
        unsigned m[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            m[q] = chunk_weights(c[q], a[q], p.teps, lane, T[q], done[q], wl[q], Tl[q]);
            nc[q] += __popc(m[q]);
        }
        unsigned U = m[0] | m[1];
        while (U) {
            int js[4];
            float ww[4][2];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                js[s] = U ? __ffs(U) - 1 : -1;
                U &= U - 1;
                const int src = js[s] < 0 ? 0 : js[s];
                const float w0 = __shfl_sync(kFull, wl[0], src), w1 = __shfl_sync(kFull, wl[1], src);
                ww[s][0] = js[s] < 0 ? 0.f : w0;   // an empty slot carries no weight
                ww[s][1] = js[s] < 0 ? 0.f : w1;
            }
            float v[16];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                if (js[s] >= 0) {
                    float f[DPL];
                    load_row_f32<DPL>(sf + js[s] * D, lane, f);
                    v[4 * s + 0] = dot_slice<DPL>(g0, f);
                    v[4 * s + 1] = dot_slice<DPL>(F0, f);
                    v[4 * s + 2] = dot_slice<DPL>(g1, f);
                    v[4 * s + 3] = dot_slice<DPL>(F1, f);
                    axpy_slice<DPL>(ww[s][0], f, F0);
                    axpy_slice<DPL>(ww[s][1], f, F1);
                } else {
                    v[4 * s] = v[4 * s + 1] = v[4 * s + 2] = v[4 * s + 3] = 0.f;
                }
            }
            // value 4 s + 2 q + t (t = 0: f_gt . f, t = 1: F . f) lands in lanes 8 s + 4 q + 2 t (+1)
            const float tot = warp_rs16(v, lane);
            const float X = __shfl_down_sync(kFull, tot, 2);
            int j = -1;
            float w = 0.f;
#pragma unroll
            for (int s = 0; s < 4; ++s)
                if (s == my_slot) {
                    j = js[s];
                    w = my_q ? ww[s][1] : ww[s][0];
                }
            const int src = j < 0 ? 0 : j;
            const float t0 = __shfl_sync(kFull, Tl[0], src), t1 = __shfl_sync(kFull, Tl[1], src);
            if ((lane & 3) == 0 && j >= 0 && w > 0.f) {
                const float sig = ndfd_sigma(tot * sinv[j] * (my_q ? igt[1] : igt[0]), ks, lam);
                acc_gt = fmaf(w, sig, acc_gt);
                acc_cf = fmaf(sig * w, (1.f - (my_q ? t1 : t0)) - X, acc_cf);
            }
        }
    }
    const float L0 = warp_sum(my_q ? 0.f : acc_gt), L1 = warp_sum(my_q ? acc_gt : 0.f);
    const float C0 = warp_sum(my_q ? 0.f : acc_cf), C1 = warp_sum(my_q ? acc_cf : 0.f);
    if (lane == 0) {
        if (rc.inside[0]) {
            Lgt_out[rc.pix[0]] = L0;
            Lcf_out[rc.pix[0]] = C0;
            if (nc_out) nc_out[rc.pix[0]] = nc[0];
        }
        if (rc.inside[1]) {
            Lgt_out[rc.pix[1]] = L1;
            Lcf_out[rc.pix[1]] = C1;
            if (nc_out) nc_out[rc.pix[1]] = nc[1];
        }
    }
}

// The backward runs one pixel per warp, 16 warps per block (the block's tile
// row), so that twice as many warps hide the latency of its dependent dot
// products and shuffles.
constexpr int kWarpsB = 16;
constexpr int kThreadsB = 32 * kWarpsB;

// Sums 8 per-lane values over the warp; lane l receives the total of value
// l >> 2 (9 shuffles).
__device__ __forceinline__ float warp_rs8(const float (&v)[8], int lane) {
    float a[4], b[2], c[1];
    rs_step<4>(v, a, lane, 16);
    rs_step<2>(a, b, lane, 8);
    rs_step<1>(b, c, lane, 4);
    const float t = c[0] + __shfl_xor_sync(kFull, c[0], 2);
    return t + __shfl_xor_sync(kFull, t, 1);
}

// Per-warp scalars of the chunk's entries (lane j writes entry j): alpha,
// T before the entry, G and rho.
struct EntryScalars {
    float a, T, G, rho;
};

// Footprint gradients per (camera, primitive): EWA, d(mean x, y; conic A,
// B, C; opacity) (6 of 12 floats, the render backward's layout); surfel,
// d(x_c, y_c, M00, M01, M10, M11, M20, M21, M22, opacity) (10 of 16).
template <int GEOM>
struct GeoG {
    static constexpr int kN = GEOM == FHGS_GEOM_EWA ? 6 : 10;     // components
    static constexpr int kPad = GEOM == FHGS_GEOM_EWA ? 8 : 12;   // shared-memory row
    static constexpr int kG2d = GEOM == FHGS_GEOM_EWA ? 12 : kSurfelG2d;
};

// dL/dalpha of one contributor -> its footprint gradient at the pixel,
// through alpha = min(alpha_max, op G), G = exp(-r^2/2) (the clamp passes no
// gradient): EWA r^2 = q2 of the conic at (dx, dy); surfel r^2 = u^2 + v^2
// with u = (M00 dx + M01 dy) / w, v = (M10 dx + M11 dy) / w, w = M20 dx +
// M21 dy + M22 (the ray-plane solve recomputed at the pixel).
template <int GEOM>
__device__ __forceinline__ void footprint_geo(float (&geo)[GeoG<GEOM>::kN], float4 A, float4 B, float4 C, float fpx,
                                              float fpy, const EntryScalars &e, float amax, float dal) {
    const float drho = e.rho > amax ? 0.f : dal;
    if constexpr (GEOM == FHGS_GEOM_EWA) {
        const float dq2 = -0.5f * e.rho * drho;
        const float dx = fpx - A.x, dy = fpy - A.y;
        geo[0] = -(2.f * A.z * dx + 2.f * A.w * dy) * dq2;
        geo[1] = -(2.f * A.w * dx + 2.f * B.x * dy) * dq2;
        geo[2] = dx * dx * dq2;
        geo[3] = 2.f * dx * dy * dq2;
        geo[4] = dy * dy * dq2;
        geo[5] = e.G * drho;
    } else {
        SurfelHit h;
        surfel_uv(A, B, C.x, fpx, fpy, 3.4e38f, h);  // a contributor: the ray meets the plane in front
        const float dr2 = -0.5f * e.rho * drho;
        const float du = 2.f * h.u * dr2, dv = 2.f * h.v * dr2;
        const float dnu = du * h.iw, dnv = dv * h.iw;
        const float dw = -(du * h.u + dv * h.v) * h.iw;
        geo[0] = -(dnu * A.z + dnv * B.x + dw * B.z);
        geo[1] = -(dnu * A.w + dnv * B.y + dw * B.w);
        geo[2] = dnu * h.dx;
        geo[3] = dnu * h.dy;
        geo[4] = dnv * h.dx;
        geo[5] = dnv * h.dy;
        geo[6] = dw * h.dx;
        geo[7] = dw * h.dy;
        geo[8] = dw;
        geo[9] = e.G * drho;
    }
}

template <int DPL, int BF16, int GEOM>
__global__ void __launch_bounds__(kThreadsB, 1) k_ndfd_bwd(long long N, CamSet cs, Params p, ProjView pv,
                                                         const uint32_t *__restrict__ gids,
                                                         const uint32_t *__restrict__ ranges, const void *feats,
                                                         const void *fgt, float ks, float lam,
                                                         const float *__restrict__ dLgt,
                                                         const float *__restrict__ dLcf, float *g2d) {
    constexpr int D = 32 * DPL;
    constexpr int kGtRowBytes = D * (BF16 ? 2 : 4);
    extern __shared__ __align__(16) float sf[];
    using GG = GeoG<GEOM>;
    __shared__ float4 sa[kNC], sb[kNC], sc[kNC];
    __shared__ uint32_t sg[kNC];
    __shared__ float sinv[kNC];
    __shared__ __align__(16) float sacc[kNC][GG::kPad];
    __shared__ __align__(16) EntryScalars sent[kWarpsB][kNC];
    __shared__ int smax;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // pixel `warp` of the block's tile row
    const int tile = blockIdx.x >> 4, row = blockIdx.x & 15;
    const int ci = cam_of_tile(cs, tile);
    const DevCam &cam = cs.c[ci];
    const int lt = tile - cam.tile_off;
    const int px = (lt % cam.tiles_x) * kTile + warp, py = (lt / cam.tiles_x) * kTile + row;
    const bool inside = px < cam.W && py < cam.H;
    const long long pix = cam.pix_off + (long long)py * cam.W + px;
    const float fpx = px + 0.5f, fpy = py + 0.5f;
    const uint32_t ls = ranges[2 * tile], le = ranges[2 * tile + 1];
    const void *rec = GEOM == FHGS_GEOM_EWA ? static_cast<const void *>(pv.rec + (long long)ci * N)
                                            : static_cast<const void *>(pv.srec + (long long)ci * N);
    float *g2dc = g2d + (long long)ci * N * GG::kG2d;

    float F[DPL], T = 1.f;
    int last = 0;
    bool done = !inside;
#pragma unroll
    for (int i = 0; i < DPL; ++i) F[i] = 0.f;
    if (threadIdx.x == 0) smax = 0;
    for (int i = threadIdx.x; i < kNC * GG::kPad; i += kThreadsB) (&sacc[0][0])[i] = 0.f;

    // front to back: F_N, T_N and the last contributor
    for (uint32_t base = ls; base < le; base += kNC) {
        if (__syncthreads_and(done)) break;
        const int nb = (int)min((uint32_t)kNC, le - base);
        stage_chunk<DPL, BF16, GEOM, kThreadsB>(rec, gids, base, nb, feats, sf, sa, sb, sc, sg, sinv, warp, lane);
        float a = 0.f;
        bool c = false;
        if (lane < nb) {
            float G, rho;
            c = !done && ndfd_alpha<GEOM>(p, sa[lane], sb[lane], sc[lane], fpx, fpy, a, G, rho);
        }
        float wl, Tl;
        const unsigned m = chunk_weights(c, a, p.teps, lane, T, done, wl, Tl);
        if (m) last = (int)(base - ls) + 32 - __clz(m);
        unsigned U = m;
        while (U) {
            const int j = __ffs(U) - 1;
            U &= U - 1;
            const float w = __shfl_sync(kFull, wl, j);
            float f[DPL];
            load_row_f32<DPL>(sf + j * D, lane, f);
            axpy_slice<DPL>(w, f, F);
        }
    }

    // back to front
    float g[DPL], Gs[DPL], igt, cgt = 0.f, ccf = 0.f, Ss = 0.f, Sw = 0.f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) g[i] = Gs[i] = 0.f;
    if (inside) {
        cgt = dLgt[pix];
        ccf = dLcf[pix];
        load_row_g<DPL, BF16>(reinterpret_cast<const char *>(fgt) + pix * kGtRowBytes, lane, g);
    }
    {
        const float n2 = warp_sum(dot_slice<DPL>(g, g));
        igt = n2 > 0.f ? 1.f / sqrtf(n2) : 0.f;
    }
    __syncthreads();
    if (lane == 0) atomicMax(&smax, last);
    __syncthreads();
    const int Lmax = min(smax, (int)(le - ls));
    EntryScalars *es = sent[warp];
    for (int bend = Lmax; bend > 0; bend -= kNC) {
        const int bstart = max(0, bend - kNC), nb = bend - bstart;
        __syncthreads();
        stage_chunk<DPL, BF16, GEOM, kThreadsB>(rec, gids, ls + bstart, nb, feats, sf, sa, sb, sc, sg, sinv, warp,
                                                lane);
        // alpha of entry `lane`, then T before it: T after the chunk divided
        // by the suffix product of (1 - alpha) from the entry on
        float a = 0.f, Gv = 0.f, rho = 0.f;
        bool c = false;
        if (lane < nb)
            c = bstart + lane < last && ndfd_alpha<GEOM>(p, sa[lane], sb[lane], sc[lane], fpx, fpy, a, Gv, rho);
        float suf = c ? 1.f - a : 1.f;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const float t = __shfl_down_sync(kFull, suf, d);
            if (lane + d < 32) suf *= t;
        }
        const float Tb = T / suf;
        T = __shfl_sync(kFull, Tb, 0);
        const unsigned m = __ballot_sync(kFull, c);
        es[lane] = EntryScalars{a, Tb, Gv, rho};
        __syncwarp();
        unsigned U = m;
        while (U) {
            // two contributors in walk order: j0 (farther), then j1
            const int j0 = 31 - __clz(U);
            U &= ~(1u << j0);
            const int j1 = U ? 31 - __clz(U) : -1;
            if (j1 >= 0) U &= ~(1u << j1);
            const EntryScalars e0 = es[j0];
            const EntryScalars e1 = es[j1 < 0 ? j0 : j1];
            const float w0 = e0.a * e0.T, w1 = j1 < 0 ? 0.f : e1.a * e1.T;
            float v[8], f[DPL], f1[DPL];
            load_row_f32<DPL>(sf + j0 * D, lane, f);
            axpy_slice<DPL>(-w0, f, F);   // F_{j0 - 1}
            v[0] = dot_slice<DPL>(g, f);
            v[1] = dot_slice<DPL>(F, f);
            v[2] = dot_slice<DPL>(Gs, f);
            if (j1 >= 0) {
                load_row_f32<DPL>(sf + j1 * D, lane, f1);
                axpy_slice<DPL>(-w1, f1, F);   // F_{j1 - 1}
                v[3] = dot_slice<DPL>(g, f1);
                v[4] = dot_slice<DPL>(F, f1);
                v[5] = dot_slice<DPL>(Gs, f1);
                v[6] = dot_slice<DPL>(f, f1);   // the pair's Gram entry
            } else {
#pragma unroll
                for (int i = 0; i < DPL; ++i) f1[i] = 0.f;
                v[3] = v[4] = v[5] = v[6] = 0.f;
            }
            v[7] = 0.f;
            const float tot = warp_rs8(v, lane);   // value i in lanes 4 i .. 4 i + 3
            const float phi0 = __shfl_sync(kFull, tot, 0), X0 = __shfl_sync(kFull, tot, 4);
            const float A0 = __shfl_sync(kFull, tot, 8), phi1 = __shfl_sync(kFull, tot, 12);
            const float X1 = __shfl_sync(kFull, tot, 16), A1 = __shfl_sync(kFull, tot, 20);
            const float gram = __shfl_sync(kFull, tot, 24);
            float geo0[GG::kN], geo1[GG::kN];
            const float sig0 = ndfd_sigma(phi0 * sinv[j0] * igt, ks, lam);
            const float gw0 = cgt * sig0 + ccf * (sig0 * ((1.f - e0.T) - X0) + Ss - A0);
            footprint_geo<GEOM>(geo0, sa[j0], sb[j0], sc[j0], fpx, fpy, e0, p.amax, e0.T * gw0 - Sw / (1.f - e0.a));
            Sw = fmaf(w0, gw0, Sw);
            const float sw0 = sig0 * w0;
            Ss += sw0;
            float sw1 = 0.f;
#pragma unroll
            for (int k = 0; k < GG::kN; ++k) geo1[k] = 0.f;
            if (j1 >= 0) {
                const float sig1 = ndfd_sigma(phi1 * sinv[j1] * igt, ks, lam);
                // G . f_j1: G at the pair's start plus j0's share
                const float Y = fmaf(sw0, gram, A1);
                const float gw1 = cgt * sig1 + ccf * (sig1 * ((1.f - e1.T) - X1) + Ss - Y);
                footprint_geo<GEOM>(geo1, sa[j1], sb[j1], sc[j1], fpx, fpy, e1, p.amax,
                                    e1.T * gw1 - Sw / (1.f - e1.a));
                Sw = fmaf(w1, gw1, Sw);
                sw1 = sig1 * w1;
                Ss += sw1;
            }
            axpy_slice<DPL>(sw0, f, Gs);
            axpy_slice<DPL>(sw1, f1, Gs);
            // lanes 0..kN-1 add j0's components, lanes 16..16+kN-1 j1's
            const int k = lane & 15;
            float val = 0.f;
#pragma unroll
            for (int kk = 0; kk < GG::kN; ++kk)
                if (kk == k) val = lane < 16 ? geo0[kk] : geo1[kk];
            const int j = lane < 16 ? j0 : j1;
            if (k < GG::kN && j >= 0 && inside && val != 0.f) atomicAdd(&sacc[j][k], val);
        }
        __syncthreads();
        if ((int)threadIdx.x < nb) {
            const int j = threadIdx.x;
            float *dst = g2dc + GG::kG2d * (long long)sg[j];
#pragma unroll
            for (int k = 0; k < GG::kN; k += 4) {
                if (k + 4 <= GG::kN) {
                    const float4 u = *reinterpret_cast<const float4 *>(&sacc[j][k]);
                    if (u.x != 0.f || u.y != 0.f || u.z != 0.f || u.w != 0.f)
                        atomicAdd(reinterpret_cast<float4 *>(dst + k), u);
                    *reinterpret_cast<float4 *>(&sacc[j][k]) = make_float4(0.f, 0.f, 0.f, 0.f);
                } else {
                    const float2 t = *reinterpret_cast<const float2 *>(&sacc[j][k]);
                    if (t.x != 0.f || t.y != 0.f) atomicAdd(reinterpret_cast<float2 *>(dst + k), t);
                    *reinterpret_cast<float2 *>(&sacc[j][k]) = make_float2(0.f, 0.f);
                }
            }
        }
    }
}

template <int DPL, int BF16, int GEOM>
void launch_fwd_t(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                  const void *feats, const void *fgt, float ks, float lam, float *Lgt, float *Lcf, int32_t *nc,
                  cudaStream_t st) {
    static std::atomic<unsigned long long> smem_set{0};
    const int smem = kNC * 32 * DPL * 4;
    allow_max_smem(smem_set, k_ndfd_fwd<DPL, BF16, GEOM>);
    note_launch(1);
    k_ndfd_fwd<DPL, BF16, GEOM><<<(unsigned)cs.total_tiles * 16, kThreads, smem, st>>>(
        N, cs, p, pv, bins.gids, bins.ranges, feats, fgt, ks, lam, Lgt, Lcf, nc);
}

template <int DPL, int BF16, int GEOM>
void launch_bwd_t(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                  const void *feats, const void *fgt, float ks, float lam, const float *dLgt, const float *dLcf,
                  float *g2d, cudaStream_t st) {
    static std::atomic<unsigned long long> smem_set{0};
    const int smem = kNC * 32 * DPL * 4;
    allow_max_smem(smem_set, k_ndfd_bwd<DPL, BF16, GEOM>);
    note_launch(1);
    k_ndfd_bwd<DPL, BF16, GEOM><<<(unsigned)cs.total_tiles * 16, kThreadsB, smem, st>>>(
        N, cs, p, pv, bins.gids, bins.ranges, feats, fgt, ks, lam, dLgt, dLcf, g2d);
}

}  // namespace

bool ndfd_supported(int D) { return D == 32 || D == 64 || D == 128 || D == 256 || D == 512; }

#define FHGS_NDFD_CASES(X, BF, G) \
    X(1, BF, G) X(2, BF, G) X(4, BF, G) X(8, BF, G) X(16, BF, G)

void launch_ndfd_fwd(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                     const void *feats, const void *fgt, int bf16, int D, float ks, float lam, float *Lgt,
                     float *Lcf, int32_t *nc, cudaStream_t st) {
    if (cs.total_tiles == 0) return;
#define X(DPL, BF, G)                                                                          \
    if (D == 32 * DPL && bf16 == BF && p.geom == G) {                                          \
        launch_fwd_t<DPL, BF, G>(N, cs, p, pv, bins, feats, fgt, ks, lam, Lgt, Lcf, nc, st);   \
        return;                                                                                \
    }
    FHGS_NDFD_CASES(X, 0, FHGS_GEOM_EWA)
    FHGS_NDFD_CASES(X, 1, FHGS_GEOM_EWA)
    FHGS_NDFD_CASES(X, 0, FHGS_GEOM_SURFEL)
    FHGS_NDFD_CASES(X, 1, FHGS_GEOM_SURFEL)
#undef X
}

void launch_ndfd_bwd(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                     const void *feats, const void *fgt, int bf16, int D, float ks, float lam, const float *dLgt,
                     const float *dLcf, float *g2d, cudaStream_t st) {
    if (cs.total_tiles == 0) return;
#define X(DPL, BF, G)                                                                                \
    if (D == 32 * DPL && bf16 == BF && p.geom == G) {                                                \
        launch_bwd_t<DPL, BF, G>(N, cs, p, pv, bins, feats, fgt, ks, lam, dLgt, dLcf, g2d, st);      \
        return;                                                                                      \
    }
    FHGS_NDFD_CASES(X, 0, FHGS_GEOM_EWA)
    FHGS_NDFD_CASES(X, 1, FHGS_GEOM_EWA)
    FHGS_NDFD_CASES(X, 0, FHGS_GEOM_SURFEL)
    FHGS_NDFD_CASES(X, 1, FHGS_GEOM_SURFEL)
#undef X
}

}  // namespace fhgs
