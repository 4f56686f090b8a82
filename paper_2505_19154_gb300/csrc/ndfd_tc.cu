// NDFD losses on the tensor cores (Sec. 3.2-3.3, Eq. 5-6, App. A.1):
//   L_gt(p) = sum_i w_i sigma_i,   L_cf(p) = sum_i sigma_i w_i (W_{i-1} - F_{i-1} . f_i)
// over the render's depth-sorted tile lists and Eq. 4 weights (i = 1 the
// nearest), sigma_i = 1 / (1 + exp(k (cos<f_i, f_gt(p)> - lambda))).
//
// Per chunk of 64 list entries and half tile of P = 128 pixels the D-deep
// work is four products:
//   Phi   = F_gt . F_c^T                     (P x 64)  f_gt . f_i
//   X     = F_start . F_c^T + W . Gs         (P x 64)  F_{i-1} . f_i
//   Gamma = F_c . F_c^T                      (64 x 64) the chunk's Gram matrix
//   F    += W . F_c                          (P x D)   the running feature
// where W holds the chunk's weights and Gs the strictly upper part of Gamma
// (Gs[j][i] = f_j . f_i for j < i), so that W . Gs adds the chunk's own
// earlier entries to F_{i-1} . f_i.  The weights are decided on the CUDA cores
// exactly as the tensor-core render decides them (FP32 alpha, transmittance
// and stop rule).  W, F and Gs enter the products as BF16 hi + lo pairs (the
// features themselves are BF16), so X carries ~16 mantissa bits.
//
// D = 128 NC is split over a cluster of NC CTAs (NC = 2 or 4), each owning
// 128 channels of every row: its F slice (FP32, 128 TMEM columns), the F_gt
// slice and the chunk's feature slice.  Every CTA decides all 128 pixels'
// weights itself: the same inputs and instructions give the same decisions,
// and recomputing them costs less than sending them (distributed shared
// memory carries only some 10 bytes per cycle per SM here).  Phi, X and the
// Gram diagonal (the squared feature norms) are partial sums over the
// channel slice; after every chunk each CTA sends the rows of pixel slice r
// (128 / NC pixels) to CTA r, which adds the NC partials and forms cos,
// sigma and the two loss terms of its pixels.  The exchange is paced by
// mbarriers with bounded waits (rows ready at the receiver, slots free at
// the sender).
//
// Tensor memory (512 columns): F [0, 128), F hi [128, 192), F lo [192, 256)
// (two channels per column: the A operand of X read from TMEM), Phi
// [256, 320), X [320, 384), Gamma [384, 448).
//
// Every wait is bounded (2 s of %globaltimer); on expiry the kernel latches
// FHGS_ERR_TIMEOUT, stops walking, waits (bounded) for its own MMAs, frees its
// tensor memory and meets its cluster once more before it returns.
#include <cuda.h>

#include <atomic>

#include "fhgs_internal.cuh"
#include "tc_ptx.cuh"

namespace fhgs {
namespace {

using namespace tc;

constexpr int kC = 64;  // list entries per chunk

constexpr int cal(int x, int a) { return (x + a - 1) / a * a; }

constexpr int kStashRow = 68;  // floats per own pixel in the weight stash (64 + 4: spreads the banks)

// The part of a projected record the NDFD kernels stage, per footprint
// model: EWA, GRec.a and .b (mean, conic, opacity); 2DGS surfel, SRec.a, .b
// and .c (centre, M = T'^-1, opacity).  alpha() takes the render's decision
// at a pixel: EWA q2 <= cutoff and alpha = min(alpha_max, op 2^(-q2 log2(e)/2));
// surfel u^2 + v^2 <= cutoff at the ray-plane hit and alpha = min(alpha_max,
// op exp(-(u^2 + v^2)/2)) (the surfel render's exponential).  Both return 0
// for a primitive that does not count, and G and rho = op G.
struct __align__(16) RecAB {
    float4 a, b;
};
struct __align__(16) RecABC {
    float4 a, b, c;
};
template <int GEOM>
struct NRec;
template <>
struct NRec<FHGS_GEOM_EWA> {
    using T = RecAB;
    using Src = GRec;
    static constexpr int kG2 = 12;   // footprint-gradient floats per (camera, Gaussian)
    static constexpr int kAcc = 8;   // shared accumulator row
    static constexpr int kN = 6;     // d(mean x, y; conic A, B, C; opacity)
    // adds the footprint gradient of dL/dalpha at a pixel to g[0..5] (the
    // clamp alpha = alpha_max passes none)
    __device__ static void footprint(const RecAB &r, float fpx, float fpy, float dal, const Params &p, float *g) {
        const float4 A = r.a, B = r.b;
        const float dx = fpx - A.x, dy = fpy - A.y;
        const float q2 = eval_q2(dx, dy, A.z, A.w, B.x);
        const float G = gauss_q2(q2), rho = B.y * G;
        const float drho = rho > p.amax ? 0.f : dal;
        const float dq2 = -0.5f * rho * drho;
        g[0] += -(2.f * A.z * dx + 2.f * A.w * dy) * dq2;
        g[1] += -(2.f * A.w * dx + 2.f * B.x * dy) * dq2;
        g[2] += dx * dx * dq2;
        g[3] += 2.f * dx * dy * dq2;
        g[4] += dy * dy * dq2;
        g[5] += G * drho;
    }
    __device__ static float alpha(const RecAB &r, float fpx, float fpy, const Params &p, float &G, float &rho) {
        const float dx = fpx - r.a.x, dy = fpy - r.a.y;
        const float q2 = eval_q2(dx, dy, r.a.z, r.a.w, r.b.x);
        G = gauss_q2(q2);
        rho = r.b.y * G;
        const float al = fminf(p.amax, rho);
        return (q2 <= p.cut && al >= p.amin) ? al : 0.f;
    }
};
template <>
struct NRec<FHGS_GEOM_SURFEL> {
    using T = RecABC;
    using Src = SRec;
    static constexpr int kG2 = kSurfelG2d;
    static constexpr int kAcc = 12;
    static constexpr int kN = 10;    // d(x_c, y_c, M00, M01, M10, M11, M20, M21, M22, opacity)
    // the surfel render backward's chain through u, v and w of the ray-plane hit
    __device__ static void footprint(const RecABC &r, float fpx, float fpy, float dal, const Params &p, float *g) {
        SurfelHit h;
        surfel_uv(r.a, r.b, r.c.x, fpx, fpy, 3.4e38f, h);  // a contributor: the ray meets the plane in front
        const float G = __expf(-0.5f * h.r2), rho = r.c.y * G;
        const float drho = rho > p.amax ? 0.f : dal;
        const float dr2 = -0.5f * rho * drho;
        const float du = 2.f * h.u * dr2, dv = 2.f * h.v * dr2;
        const float dnu = du * h.iw, dnv = dv * h.iw, dw = -(du * h.u + dv * h.v) * h.iw;
        g[0] -= dnu * r.a.z + dnv * r.b.x + dw * r.b.z;
        g[1] -= dnu * r.a.w + dnv * r.b.y + dw * r.b.w;
        g[2] += dnu * h.dx;
        g[3] += dnu * h.dy;
        g[4] += dnv * h.dx;
        g[5] += dnv * h.dy;
        g[6] += dw * h.dx;
        g[7] += dw * h.dy;
        g[8] += dw;
        g[9] += G * drho;
    }
    __device__ static float alpha(const RecABC &r, float fpx, float fpy, const Params &p, float &G, float &rho) {
        SurfelHit h;
        const bool hit = surfel_uv(r.a, r.b, r.c.x, fpx, fpy, p.cut, h);
        G = __expf(-0.5f * h.r2);
        rho = r.c.y * G;
        const float al = fminf(p.amax, rho);
        return (hit && al >= p.amin) ? al : 0.f;
    }
};

template <int NC, int GEOM = FHGS_GEOM_EWA>
struct NCfg {
    static constexpr int kNC = NC;
    using Rec = typename NRec<GEOM>::T;
    using RecSrc = typename NRec<GEOM>::Src;
    static constexpr int kGeom = GEOM;
    static constexpr int kFStages = 2;       // feature stages (chunk b + 1 loads under chunk b)
    static constexpr int kOwn = 128 / NC;    // pixels whose losses this CTA completes
    static constexpr int kTpp = 256 / kOwn;  // threads per own pixel in the loss pass
    static constexpr int kEpt = kC / kTpp;   // entries per thread in the loss pass
    static constexpr int kRow = 2 * kC + 4;  // floats per exchanged pixel row: Phi[64], X[64], 4 of padding
    // one sender's slot at a receiver: rows, then the Gram diagonal [64], then
    // the partial |f_gt|^2 of the receiver's pixels
    static constexpr int kSlotF = kOwn * kRow + kC + kOwn;
    static constexpr int kOffGt = 0;                        // [2][128 px][64 ch] BF16, K-major, swizzled
    static constexpr int kOffF = kOffGt + 2 * 128 * 128;    // [2 stages][2][64 g][64 ch] BF16
    static constexpr int kOffWh = kOffF + 2 * 2 * kC * 128;  // [128 px][64 g] BF16 weights, hi
    static constexpr int kOffWl = kOffWh + 128 * 128;       // lo
    static constexpr int kOffGh = kOffWl + 128 * 128;       // [64 i][64 j] BF16 strict Gram part, hi
    static constexpr int kOffGl = kOffGh + kC * 128;        // lo
    static constexpr int kOffRecv = kOffGl + kC * 128;      // [NC][kSlotF] floats
    static constexpr int kOffStash = kOffRecv + cal(NC * kSlotF * 4, 16);  // [kOwn][kStashRow] w, then T
    static constexpr int kOffRec = kOffStash + 2 * kOwn * kStashRow * 4;  // [2 stages][64] staged records
    static constexpr int kOffGid = kOffRec + 2 * kC * (int)sizeof(Rec);  // [3][64] ids
    static constexpr int kOffPix = kOffGid + 3 * kC * 4;           // per pixel: T, done, last, P0, L0, |f_gt|^2
    static constexpr int kOffDiag = kOffPix + 6 * 128 * 4;         // [64] Gram diagonal of the chunk
    static constexpr int kOffAcc = kOffDiag + kC * 4;              // [3][kOwn] L_gt, L_cf, count of own pixels
    static constexpr int kOffBar = cal(kOffAcc + 3 * kOwn * 4, 8);
    static constexpr int kSmem = 1024 + kOffBar + 64;  // 6 barriers and the TMEM slot
    static_assert(kSmem <= 232448, "NDFD CTA exceeds the opt-in shared memory");
    static_assert(8 * 32 * 20 * 4 <= kOffGh - kOffWh, "the row staging must fit in the weight operands");
    static_assert(8 * 32 * 36 * 4 <= kOffGh, "the saved state's tiles must fit in the operand stages");
    static constexpr uint32_t kColF = 0, kColFh = 128, kColFl = 192, kColPhi = 256, kColX = 320, kColGam = 384;
};

// BF16 hi + lo parts of x: hi = bf16(x), lo = bf16(x - hi).
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}
__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Byte offset of K-step ks (16 BF16 along K) inside a K-major operand whose
// 64-element K blocks are `blk` bytes apart.
__device__ __forceinline__ uint32_t kstep(int ks, uint32_t blk) { return (uint32_t)(ks >> 2) * blk + (uint32_t)(ks & 3) * 32u; }

// Everything a CTA needs to know about its item (tile, half) and its place
// in the cluster.
struct Item {
    int ci, tx, ty, half, q;
    uint32_t s, e;
    const DevCam *cam;
};

__device__ __forceinline__ Item make_item(const CamSet &cs, const uint32_t *ranges, int item, int q) {
    Item it;
    const int tile = item >> 1;
    it.half = item & 1;
    it.ci = cam_of_tile(cs, tile);
    it.cam = &cs.c[it.ci];
    const int lt = tile - it.cam->tile_off;
    it.tx = lt % it.cam->tiles_x;
    it.ty = lt / it.cam->tiles_x;
    it.s = ranges[2 * tile];
    it.e = ranges[2 * tile + 1];
    it.q = q;
    return it;
}

// Pixel `pidx` (0..127) of the item's half tile: (i, j) = (pidx % 16, pidx / 16).
__device__ __forceinline__ bool item_pixel(const Item &it, int pidx, long long &pix, float &fpx, float &fpy) {
    const int px = it.tx * kTile + (pidx & 15), py = it.ty * kTile + it.half * 8 + (pidx >> 4);
    pix = it.cam->pix_off + (long long)py * it.cam->W + px;
    fpx = px + 0.5f;
    fpy = py + 0.5f;
    return px < it.cam->W && py < it.cam->H;
}



// Per-pixel walk state in shared memory (one entry per pixel of the half tile).
struct PixState {
    float *T;   // transmittance entering the next chunk
    int *done;  // the pixel's walk has stopped
    int *last;  // list position after its last contributor
    float *P0;  // group 0's product of (1 - alpha) over its 32 entries
    int *L0;    // group 0's last entry with alpha > 0, or -1
};

// Front-to-back weights of one chunk (list entries [pos0, pos0 + nb), records
// R) for the half tile's 128 pixels, by the tensor-core render's rules: 256
// threads, group g = tid / 128 takes entries [32 g, 32 g + 32); both groups
// evaluate their alphas and running products of (1 - alpha) at once, then
// group 1 starts from T_in P_0 unless group 0 stops.  alpha = min(alpha_max,
// op G) counts when q2 <= cutoff and alpha >= alpha_min; the walk stops at
// the first counted entry j with T_j (1 - alpha_j) < t_eps, which itself does
// not contribute.  Every CTA of a cluster takes the same decisions (same
// inputs, same instructions), which costs less than exchanging them.  Writes
// w (negated when `neg`) as BF16 hi + lo into the K-major [128 px][64]
// operands, and w and T (before the entry) of the pixels [own0, own0 + own)
// into the stash.  Returns, uniformly over the CTA, whether every pixel has
// stopped after the chunk.
template <int GEOM>
__device__ __forceinline__ bool chunk_weights(const Params &p, const typename NRec<GEOM>::T *R, int nb, int pos0,
                                              int pidx, int grp,
                                              float fpx, float fpy, PixState ps, uint8_t *sWh, uint8_t *sWl,
                                              float *stash_w, float *stash_T, int own0, int own, bool neg) {
    const float T_in = ps.T[pidx];
    const bool done_in = ps.done[pidx] != 0;
    const int last_in = ps.last[pidx];
    float a[32], l[32];
    float P = 1.f;
    int lastc = -1;
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
        const int j = grp * 32 + jj;
        float G, rho;
        const float al = NRec<GEOM>::alpha(R[j], fpx, fpy, p, G, rho);
        a[jj] = j < nb ? al : 0.f;
        l[jj] = P;
        P *= 1.f - a[jj];
        lastc = a[jj] > 0.f ? jj : lastc;
    }
    if (grp == 0) {
        ps.P0[pidx] = P;
        ps.L0[pidx] = lastc;
    }
    __syncthreads();
    const float P0 = ps.P0[pidx];
    const bool stop0 = !done_in && T_in * P0 < p.teps;
    const float Ts = grp == 0 ? T_in : T_in * P0;
    bool done = grp == 0 ? done_in : (done_in || stop0);
    const bool owner = grp == 0 ? (done_in || stop0) : !(done_in || stop0);
    const int pl = pidx - own0;
    const bool mine = pl >= 0 && pl < own;
    float Tstop = 0.f;
    int lastw = -1;
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
        uint32_t hw[4], lw[4];
        float w8[8], T8[8];
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const int jj = 8 * qq + h;
            const float Tj = Ts * l[jj];
            const float Tn = Ts * (jj < 31 ? l[jj + 1] : P);
            bool okj = a[jj] > 0.f && !done;
            const bool stop = okj && Tn < p.teps;
            if (stop) Tstop = Tj;
            done = done || stop;
            okj = okj && !stop;
            w8[h] = okj ? a[jj] * Tj : 0.f;
            T8[h] = Tj;
            if (okj) lastw = jj;
        }
        if (mine) {
            float *dw = stash_w + pl * kStashRow + grp * 32 + 8 * qq, *dT = stash_T + pl * kStashRow + grp * 32 + 8 * qq;
            *reinterpret_cast<float4 *>(dw) = make_float4(w8[0], w8[1], w8[2], w8[3]);
            *reinterpret_cast<float4 *>(dw + 4) = make_float4(w8[4], w8[5], w8[6], w8[7]);
            *reinterpret_cast<float4 *>(dT) = make_float4(T8[0], T8[1], T8[2], T8[3]);
            *reinterpret_cast<float4 *>(dT + 4) = make_float4(T8[4], T8[5], T8[6], T8[7]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            __nv_bfloat16 h0, l0, h1, l1;
            split_bf16(neg ? -w8[2 * u] : w8[2 * u], h0, l0);
            split_bf16(neg ? -w8[2 * u + 1] : w8[2 * u + 1], h1, l1);
            hw[u] = pack2(h0, h1);
            lw[u] = pack2(l0, l1);
        }
        *reinterpret_cast<uint4 *>(sWh + swz(pidx, grp * 4 + qq)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(sWl + swz(pidx, grp * 4 + qq)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    if (owner) {  // exactly one group carries the pixel's state to the next chunk
        if (grp == 0) {
            ps.T[pidx] = done_in ? T_in : Tstop;
            ps.done[pidx] = 1;
            ps.last[pidx] = lastw >= 0 ? pos0 + lastw + 1 : last_in;
        } else {
            const int L0 = ps.L0[pidx];
            ps.T[pidx] = done ? Tstop : Ts * P;
            ps.done[pidx] = done ? 1 : 0;
            ps.last[pidx] = lastw >= 0 ? pos0 + 32 + lastw + 1 : (L0 >= 0 ? pos0 + L0 + 1 : last_in);
        }
    }
    return __syncthreads_and(grp == 0 || done) != 0;
}

// F (FP32, TMEM columns [colF, colF + 128)) -> BF16 hi + lo copies in TMEM,
// two channels per column (the layout of an A operand read from TMEM: lane =
// pixel, 8 columns per K step of 16).  Warp w converts channels
// [64 (w / 4), + 64) of its lane quadrant.
__device__ __forceinline__ void split_to_tmem(uint32_t taddr, uint32_t colF, uint32_t colH, uint32_t colL, int warp) {
    const uint32_t lq = (uint32_t)((warp & 3) * 32) << 16;
    const int h = warp >> 2;
#pragma unroll
    for (int part = 0; part < 2; ++part) {
        float v[32];
        tmem_ld32(taddr + lq + colF + 64 * h + 32 * part, v);
        uint32_t hi[16], lo[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            __nv_bfloat16 h0, l0, h1, l1;
            split_bf16(v[2 * i], h0, l0);
            split_bf16(v[2 * i + 1], h1, l1);
            hi[i] = pack2(h0, h1);
            lo[i] = pack2(l0, l1);
        }
        tmem_st16(taddr + lq + colH + 32 * h + 16 * part, hi);
        tmem_st16(taddr + lq + colL + 32 * h + 16 * part, lo);
    }
    tmem_st_wait();
}

// Gamma (TMEM lanes = entries i, columns = entries j) -> one masked part as a
// K-major B operand [64 rows i][64 j] (BF16 hi + lo): `before` keeps j < i
// (the entries before i), else j > i.  Warps 0, 1 (lanes = rows 0..63) take
// columns 0..31, warps 4, 5 columns 32..63; the warp holding column i also
// writes the diagonal entry.
__device__ __forceinline__ void gram_part(uint32_t taddr, uint32_t colG, int warp, int lane, bool before,
                                          uint8_t *sGh, uint8_t *sGl, float *diag) {
    const int i = (warp & 3) * 32 + lane, ch = warp >> 2;
    float g[32];
    tmem_ld32(taddr + ((uint32_t)((warp & 3) * 32) << 16) + colG + 32 * ch, g);
    float dg = 0.f;
    bool mine = false;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int h = 0; h < 8; h += 2) {
            float v2[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int jl = 8 * c + h + u, j = 32 * ch + jl;
                if (j == i) {
                    dg = g[jl];
                    mine = true;
                }
                v2[u] = (before ? j < i : j > i) ? g[jl] : 0.f;
            }
            __nv_bfloat16 h0, l0, h1, l1;
            split_bf16(v2[0], h0, l0);
            split_bf16(v2[1], h1, l1);
            hw[h >> 1] = pack2(h0, h1);
            lw[h >> 1] = pack2(l0, l1);
        }
        *reinterpret_cast<uint4 *>(sGh + swz(i, 4 * ch + c)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(sGl + swz(i, 4 * ch + c)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    if (mine) diag[i] = dg;
}

// Shared-memory views and loaders of one CTA's item, common to the forward
// and the backward.
template <class C>
struct ItemSmem {
    uint8_t *sm;
    uint32_t sm_s;
    __device__ typename C::Rec *rec(int b) const {
        return reinterpret_cast<typename C::Rec *>(sm + C::kOffRec + (b & 1) * kC * (int)sizeof(typename C::Rec));
    }
    __device__ uint32_t *gid(int b) const {
        return reinterpret_cast<uint32_t *>(sm + C::kOffGid + ((b % 3 + 3) % 3) * kC * 4);
    }
    __device__ uint32_t feat_s(int b) const {
        return sm_s + C::kOffF + (C::kFStages == 2 ? (uint32_t)(b & 1) : 0u) * (2 * kC * 128);
    }
    __device__ PixState pix() const {
        int *base = reinterpret_cast<int *>(sm + C::kOffPix);
        return PixState{reinterpret_cast<float *>(base), base + 128, base + 256, reinterpret_cast<float *>(base + 384),
                        base + 512};
    }
    __device__ float *ngt() const { return reinterpret_cast<float *>(sm + C::kOffPix) + 640; }
    __device__ float *diag() const { return reinterpret_cast<float *>(sm + C::kOffDiag); }
    __device__ float *recv() const { return reinterpret_cast<float *>(sm + C::kOffRecv); }
    __device__ float *stash_w() const { return reinterpret_cast<float *>(sm + C::kOffStash); }
    __device__ float *stash_T() const { return stash_w() + C::kOwn * kStashRow; }
    __device__ float *acc(int k) const { return reinterpret_cast<float *>(sm + C::kOffAcc) + k * C::kOwn; }
    __device__ uint64_t *bars() const { return reinterpret_cast<uint64_t *>(sm + C::kOffBar); }
};

// Every loader commits exactly one cp.async group in every thread, empty or
// not, so that the waits on group counts hold.  Chunk b of the item holds list
// entries [s + 64 b, s + 64 b + 64) of camera ci; `q` selects the CTA's 128
// channels.
template <class C>
struct Loader {
    static constexpr int NC = C::kNC;
    const ItemSmem<C> &S;
    const uint32_t *gids;
    const typename C::RecSrc *rec;
    const __nv_bfloat16 *feats;
    uint32_t s, e;
    int nchunks, q, tid;
    __device__ void gid(int b) const {
        if (b >= 0 && b < nchunks && tid < kC) {
            const uint32_t at = s + (uint32_t)b * kC + tid;
            cp_async4(smem_u32(S.gid(b) + tid), gids + (at < e ? at : s), at < e);
        }
        cp_async_commit();
    }
    __device__ void records(int b) const {
        if (b >= 0 && b < nchunks && tid < kC) {
            const bool v = s + (uint32_t)b * kC + tid < e;
            const uint32_t dst = smem_u32(S.rec(b) + tid);
            const float4 *src = reinterpret_cast<const float4 *>(rec + (v ? S.gid(b)[tid] : 0u));
#pragma unroll
            for (int w4 = 0; w4 < (int)(sizeof(typename C::Rec) / 16); ++w4) cp_async16(dst + 16 * w4, src + w4, v);
        }
        cp_async_commit();
    }
    __device__ void features(int b) const {
        if (b >= 0 && b < nchunks) {
            const int nb = (int)min((uint32_t)kC, e - (s + (uint32_t)b * kC));
            const uint32_t fb = S.feat_s(b);
            const uint32_t *ids = S.gid(b);
#pragma unroll
            for (int c = tid; c < kC * 16; c += 256) {
                const int g = c >> 4, cc = c & 15;
                const bool valid = g < nb;
                cp_async16(fb + (uint32_t)(cc >> 3) * (kC * 128) + swz(g, cc & 7),
                           feats + (size_t)(valid ? ids[g] : 0u) * (128 * NC) + 128 * q + cc * 8, valid);
            }
        }
        cp_async_commit();
    }
};

// Descriptors of the chunk's operands (address field = byte address / 16).
struct ChunkDesc {
    uint64_t FK, FM;  // chunk features as a K-major operand (rows = entries) and as an MN-major B (K = entries)
};
__device__ __forceinline__ ChunkDesc chunk_desc(uint32_t fb) {
    return ChunkDesc{sdesc(fb, 16, 1024), sdesc(fb, kC * 128, 1024)};
}
constexpr uint32_t kId64 = idesc_bf16(128, kC, false, false);    // P x 64 products, K-major A and B
constexpr uint32_t kId128 = idesc_bf16(128, 128, false, true);   // P x 128 channel update, MN-major B

// Gamma = F_c F_c^T: M = 128 rows of A read the chunk's 64 rows and the 64
// rows after them (lanes 64..127 of the result are never read).
__device__ __forceinline__ void issue_gram(uint32_t tG, const ChunkDesc &cd) {
#pragma unroll
    for (int ks = 0; ks < 8; ++ks) {
        const uint64_t o = (uint64_t)(kstep(ks, kC * 128) >> 4);
        mma_bf16(tG, cd.FK + o, cd.FK + o, kId64, ks > 0 ? 1u : 0u);
    }
}
// D (P x 64) [+]= A(P x 128 channels) F_c^T, A a K-major operand in shared memory with 64-channel blocks `blk` apart.
__device__ __forceinline__ void issue_rows_x_chunk(uint32_t tD, uint64_t a0, uint32_t blk, const ChunkDesc &cd,
                                                   bool acc) {
#pragma unroll
    for (int ks = 0; ks < 8; ++ks)
        mma_bf16(tD, a0 + (uint64_t)(kstep(ks, blk) >> 4), cd.FK + (uint64_t)(kstep(ks, kC * 128) >> 4), kId64,
                 (acc || ks > 0) ? 1u : 0u);
}
// D (P x 64) [+]= (hi + lo)(P x 128 channels, TMEM) F_c^T.
__device__ __forceinline__ void issue_tmem_x_chunk(uint32_t tD, uint32_t tH, uint32_t tL, const ChunkDesc &cd,
                                                   bool acc) {
#pragma unroll
    for (int ks = 0; ks < 8; ++ks)
        mma_bf16_ta(tD, tH + 8 * ks, cd.FK + (uint64_t)(kstep(ks, kC * 128) >> 4), kId64, (acc || ks > 0) ? 1u : 0u);
#pragma unroll
    for (int ks = 0; ks < 8; ++ks) mma_bf16_ta(tD, tL + 8 * ks, cd.FK + (uint64_t)(kstep(ks, kC * 128) >> 4), kId64, 1u);
}
// F (P x 128) [+]= (Wh + Wl)(P x 64) F_c(64 x 128).
__device__ __forceinline__ void issue_update(uint32_t tF, uint64_t wh, uint64_t wl, const ChunkDesc &cd, bool acc) {
#pragma unroll
    for (int ks = 0; ks < 4; ++ks)
        mma_bf16(tF, wh + (uint64_t)((ks * 32) >> 4), cd.FM + (uint64_t)((ks * 2048) >> 4), kId128,
                 (acc || ks > 0) ? 1u : 0u);
#pragma unroll
    for (int ks = 0; ks < 4; ++ks)
        mma_bf16(tF, wl + (uint64_t)((ks * 32) >> 4), cd.FM + (uint64_t)((ks * 2048) >> 4), kId128, 1u);
}
// D (P x 64) [+]= Wh Gh + Wl Gh + Wh Gl (the chunk's own Gram part).
__device__ __forceinline__ void issue_w_gram(uint32_t tD, uint64_t wh, uint64_t wl, uint64_t gh, uint64_t gl,
                                             bool acc) {
#pragma unroll
    for (int ks = 0; ks < 4; ++ks)
        mma_bf16(tD, wh + (uint64_t)((ks * 32) >> 4), gh + (uint64_t)((ks * 32) >> 4), kId64,
                 (acc || ks > 0) ? 1u : 0u);
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) mma_bf16(tD, wl + (uint64_t)((ks * 32) >> 4), gh + (uint64_t)((ks * 32) >> 4), kId64, 1u);
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) mma_bf16(tD, wh + (uint64_t)((ks * 32) >> 4), gl + (uint64_t)((ks * 32) >> 4), kId64, 1u);
}

// The partial Phi (warps 0..3) or X (warps 4..7) rows of this warp's lane
// quadrant -> the slot of this CTA at the receiver of those pixels, then one
// arrival per thread on the receiver's "data ready" barrier.  The rows go
// through a 2 KB staging tile per warp (`stage`, free shared memory), 16
// columns at a time, so that each remote store instruction writes 64
// contiguous bytes of 8 rows rather than 16 bytes of 32 rows.  Warps 0..3
// also send the pixels' partial |f_gt|^2, and the receiver's first X warp
// the chunk's Gram diagonal.
template <class C>
__device__ __forceinline__ void send_rows(const ItemSmem<C> &S, uint32_t taddr, uint32_t colA, uint32_t colB, int q,
                                          int warp, int lane, float *stage) {
    constexpr int NC = C::kNC;
    constexpr int kSR = 20;  // floats per staged row (16 + 4: spreads the banks)
    const int qd = warp & 3, dst = qd * NC / 4;
    const int row0 = qd * 32 - dst * C::kOwn;  // the warp's first row in the receiver's slot
    const uint32_t slot = mapa(smem_u32(S.recv() + q * C::kSlotF), (uint32_t)dst);
    const bool second = warp >= 4;
    float *st = stage + warp * 32 * kSR;
#pragma unroll
    for (int piece = 0; piece < 4; ++piece) {
        float v[16];
        tmem_ld16(taddr + ((uint32_t)(qd * 32) << 16) + (second ? colB : colA) + 16 * piece, v);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            *reinterpret_cast<float4 *>(st + lane * kSR + 4 * i) = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        __syncwarp();
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            const int r = 8 * it + (lane >> 2), c4 = (lane & 3) * 4;
            const float4 x = *reinterpret_cast<const float4 *>(st + r * kSR + c4);
            st_cluster_v4(slot + (uint32_t)((row0 + r) * C::kRow + (second ? kC : 0) + 16 * piece + c4) * 4u, x.x, x.y,
                          x.z, x.w);
        }
        __syncwarp();
    }
    const int row = row0 + lane;
    if (!second) {
        st_cluster_f32(slot + (uint32_t)(C::kOwn * C::kRow + kC + row) * 4u, S.ngt()[qd * 32 + lane]);
    } else if (qd == dst * (4 / NC)) {
        st_cluster_v2(slot + (uint32_t)(C::kOwn * C::kRow + 2 * lane) * 4u, S.diag()[2 * lane], S.diag()[2 * lane + 1]);
    }
    mbar_arrive_cluster(mapa(smem_u32(&S.bars()[2]), (uint32_t)dst));
}

// Stages the CTA's F_gt slice (BF16, K-major [2][128 px][64 ch]) of the
// item's pixels, zero outside the image; commits one cp.async group.
template <class C>
__device__ __forceinline__ void load_gt(const ItemSmem<C> &S, const Item &it, const __nv_bfloat16 *fgt, int q,
                                        int tid) {
    constexpr int NC = C::kNC;
    const uint32_t g0 = S.sm_s + C::kOffGt;
    for (int c = tid; c < 128 * 16; c += 256) {
        const int row = c >> 4, cc = c & 15;
        long long rp;
        float fx, fy;
        const bool v = item_pixel(it, row, rp, fx, fy);
        cp_async16(g0 + (uint32_t)(cc >> 3) * (128 * 128) + swz(row, cc & 7),
                   fgt + (size_t)(v ? rp : 0) * (128 * NC) + 128 * q + cc * 8, v);
    }
    cp_async_commit();
}

// Partial |f_gt|^2 over the CTA's channels of pixel tid (tid < 128).
template <class C>
__device__ __forceinline__ void gt_norm(const ItemSmem<C> &S, int tid) {
    if (tid >= 128) return;
    float s2 = 0.f;
#pragma unroll
    for (int cc = 0; cc < 16; ++cc) {
        const uint4 v = *reinterpret_cast<const uint4 *>(S.sm + C::kOffGt + (cc >> 3) * (128 * 128) + swz(tid, cc & 7));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float lo = __uint_as_float(w[u] << 16), hi = __uint_as_float(w[u] & 0xFFFF0000u);
            s2 = fmaf(lo, lo, s2);
            s2 = fmaf(hi, hi, s2);
        }
    }
    S.ngt()[tid] = s2;
}

// 1 / |f_i| of the chunk's entries (tid < 64) from the NC senders' Gram
// diagonals, 0 for a zero feature row, into `inv`.
template <class C>
__device__ __forceinline__ void entry_inv_norms(const ItemSmem<C> &S, int tid, float *inv) {
    constexpr int NC = C::kNC;
    if (tid >= kC) return;
    float n2 = 0.f;
#pragma unroll
    for (int sl = 0; sl < NC; ++sl) n2 += S.recv()[sl * C::kSlotF + C::kOwn * C::kRow + tid];
    inv[tid] = n2 > 0.f ? 1.f / sqrtf(n2) : 0.f;
}

// sigma = 1 / (1 + exp(k (phi - lambda))) with the fast exponential and
// reciprocal (relative error ~1e-6, far inside the loss bar).
__device__ __forceinline__ float sigma_fast(float phi, float k, float lam) {
    return __frcp_rn(1.f + __expf(k * (phi - lam)));
}

// The loss pass of the own pixels: kTpp threads per pixel, kEpt consecutive
// entries each; adds the NC senders' partial Phi and X, then sigma and the
// two loss terms of every contributor (w > 0).
template <class C>
__device__ __forceinline__ void own_losses(const ItemSmem<C> &S, int tid, float ks, float lam, const float *inv) {
    constexpr int NC = C::kNC;
    constexpr int E = C::kEpt;
    const int pl = tid / C::kTpp, k0 = (tid % C::kTpp) * E;
    const float *rv = S.recv();
    float ph[E], x[E];
#pragma unroll
    for (int k = 0; k < E; ++k) ph[k] = x[k] = 0.f;
    float n2 = 0.f;
#pragma unroll
    for (int sl = 0; sl < NC; ++sl) {
        const float *slot = rv + sl * C::kSlotF;
        n2 += slot[C::kOwn * C::kRow + kC + pl];
#pragma unroll
        for (int k = 0; k < E; k += 4) {
            const float4 a = *reinterpret_cast<const float4 *>(slot + pl * C::kRow + k0 + k);
            const float4 b = *reinterpret_cast<const float4 *>(slot + pl * C::kRow + kC + k0 + k);
            ph[k] += a.x; ph[k + 1] += a.y; ph[k + 2] += a.z; ph[k + 3] += a.w;
            x[k] += b.x; x[k + 1] += b.y; x[k + 2] += b.z; x[k + 3] += b.w;
        }
    }
    const float igt = n2 > 0.f ? 1.f / sqrtf(n2) : 0.f;
    float lg = 0.f, lc = 0.f, cnt = 0.f;
#pragma unroll
    for (int k = 0; k < E; k += 4) {
        const float4 w4 = *reinterpret_cast<const float4 *>(S.stash_w() + pl * kStashRow + k0 + k);
        const float4 T4 = *reinterpret_cast<const float4 *>(S.stash_T() + pl * kStashRow + k0 + k);
        const float4 i4 = *reinterpret_cast<const float4 *>(inv + k0 + k);
        const float wv[4] = {w4.x, w4.y, w4.z, w4.w}, Tv[4] = {T4.x, T4.y, T4.z, T4.w};
        const float iv[4] = {i4.x, i4.y, i4.z, i4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (wv[u] > 0.f) {
                const float sig = sigma_fast(ph[k + u] * iv[u] * igt, ks, lam);
                lg = fmaf(wv[u], sig, lg);
                lc = fmaf(sig * wv[u], (1.f - Tv[u]) - x[k + u], lc);
                cnt += 1.f;
            }
        }
    }
#pragma unroll
    for (int o = C::kTpp / 2; o > 0; o >>= 1) {
        lg += __shfl_xor_sync(0xffffffffu, lg, o);
        lc += __shfl_xor_sync(0xffffffffu, lc, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (tid % C::kTpp == 0) {
        S.acc(0)[pl] += lg;
        S.acc(1)[pl] += lc;
        S.acc(2)[pl] += cnt;
    }
}

template <int NC, int GEOM>
__global__ void __launch_bounds__(256, 1)
    k_ndfd_fwd_tc(long long N, CamSet cs, Params p, ProjView pv, const uint32_t *__restrict__ gids,
                  const uint32_t *__restrict__ ranges, const __nv_bfloat16 *__restrict__ feats,
                  const __nv_bfloat16 *__restrict__ fgt, float ks, float lam, float *Lgt_out, float *Lcf_out,
                  int32_t *nc_out, NdfdState save, unsigned *status) {
    using C = NCfg<NC, GEOM>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align_smem_1024(smem_raw);
    if (probe_wait_expired(p, sm, status)) return;  // uniform over the grid, before any cluster operation
    const ItemSmem<C> S{sm, smem_u32(sm)};
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = (int)cluster_rank();
    const Item it = make_item(cs, ranges, (int)(blockIdx.x / NC), q);
    // a wait that ran out anywhere in the grid makes the later CTAs skip their
    // walk (no waits), so that a fault of the exchange costs seconds, not a
    // wave of timeouts per CTA; a cluster's CTAs may disagree, which only
    // makes the walking ones' waits run out too
    const bool skip = (*(volatile unsigned *)status & ST_TIMEOUT) != 0;
    const int nchunks = skip ? 0 : (int)((it.e - it.s + kC - 1) / kC);
    uint64_t *bars = S.bars();  // [0] Gamma done, [1] chunk's MMAs done, [2] rows ready, [3] slots free
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 4);
    const PixState ps = S.pix();
    const int grp = tid >> 7, pidx = tid & 127, own0 = q * C::kOwn;
    long long pix;
    float fpx, fpy;
    const bool inside = item_pixel(it, pidx, pix, fpx, fpy);

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 256);  // NC senders x 256 / NC threads
        mbar_init(&bars[3], NC);   // one arrival per receiver
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(tslot, 512);
    if (grp == 0) {
        ps.T[pidx] = 1.f;
        ps.done[pidx] = inside ? 0 : 1;
        ps.last[pidx] = 0;
    }
    if (tid < C::kOwn) S.acc(0)[tid] = S.acc(1)[tid] = S.acc(2)[tid] = 0.f;
    const typename C::RecSrc *recs =
        reinterpret_cast<const typename C::RecSrc *>(GEOM == FHGS_GEOM_SURFEL ? (const void *)pv.srec
                                                                             : (const void *)pv.rec) +
        (long long)it.ci * N;
    const Loader<C> L{S, gids, recs, feats, it.s, it.e, nchunks, q, tid};
    load_gt<C>(S, it, fgt, q, tid);
    L.gid(0);
    L.gid(1);
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t taddr = *tslot;
    cluster_sync();  // every CTA's barriers are initialised before the first remote arrival
    cp_async_wait<1>();  // F_gt and the ids of chunk 0
    __syncthreads();
    L.records(0);
    L.features(0);
    gt_norm<C>(S, tid);

    const uint32_t sGt = S.sm_s + C::kOffGt, sWh = S.sm_s + C::kOffWh, sWl = S.sm_s + C::kOffWl;
    const uint32_t sGh = S.sm_s + C::kOffGh, sGl = S.sm_s + C::kOffGl;
    const uint64_t dGt = sdesc(sGt, 16, 1024), dWh = sdesc(sWh, 16, 1024), dWl = sdesc(sWl, 16, 1024);
    const uint64_t dGh = sdesc(sGh, 16, 1024), dGl = sdesc(sGl, 16, 1024);
    const uint32_t tF = taddr + C::kColF, tFh = taddr + C::kColFh, tFl = taddr + C::kColFl;
    const uint32_t tPhi = taddr + C::kColPhi, tX = taddr + C::kColX, tGam = taddr + C::kColGam;

    bool timeout = false, pending = false;
    int b = 0;
    for (; b < nchunks; ++b) {
        const uint32_t base = it.s + (uint32_t)b * kC;
        const int nb = (int)min((uint32_t)kC, it.e - base);
        cp_async_wait<0>();  // ids of b+1, records and features of b
        __syncthreads();
        L.gid(b + 2);
        L.records(b + 1);
        L.features(b + 1);  // its stage was last read by the MMAs of chunk b-1, complete
        const bool all_done = chunk_weights<GEOM>(p, S.rec(b), nb, (int)(base - it.s), pidx, grp, fpx, fpy, ps,
                                                  sm + C::kOffWh, sm + C::kOffWl, S.stash_w(), S.stash_T(), own0,
                                                  C::kOwn, false);
        if (b > 0) split_to_tmem(taddr, C::kColF, C::kColFh, C::kColFl, warp);  // F after chunk b-1
        fence_async_smem();
        tc_before();
        __syncthreads();
        const ChunkDesc cd = chunk_desc(S.feat_s(b));
        if (tid == 0) {
            tc_after();
            issue_gram(tGam, cd);
            mma_commit(&bars[0]);
            issue_rows_x_chunk(tPhi, dGt, 128 * 128, cd, false);
            if (b > 0) issue_tmem_x_chunk(tX, tFh, tFl, cd, false);
            issue_update(tF, dWh, dWl, cd, b > 0);
        }
        bool ok = true;
        if ((warp & 3) < 2) {
            ok = mbar_wait(&bars[0], (uint32_t)(b & 1));
            if (ok) {
                tc_after();
                gram_part(taddr, C::kColGam, warp, lane, true, sm + C::kOffGh, sm + C::kOffGl, S.diag());
            }
            fence_async_smem();
        }
        const bool tmo = __syncthreads_or(!ok) != 0;
        if (tid == 0) {
            tc_after();
            if (!tmo) issue_w_gram(tX, dWh, dWl, dGh, dGl, b > 0);
            mma_commit(&bars[1]);
        }
        pending = true;
        ok = mbar_wait(&bars[1], (uint32_t)(b & 1));
        if (__syncthreads_or(!ok) || tmo) {
            timeout = true;
            if (tid == 0) latch(status, ST_TIMEOUT);
            break;
        }
        pending = false;
        tc_after();
        // exchange: every receiver has consumed this CTA's slots of chunk b-1
        ok = b == 0 || mbar_wait_cluster(&bars[3], (uint32_t)((b - 1) & 1));
        if (__syncthreads_or(!ok)) {
            timeout = true;
            if (tid == 0) latch(status, ST_TIMEOUT);
            break;
        }
        // the weight operands are free until the next chunk's weights: 8 warps x 2.5 KB of staging
        send_rows<C>(S, taddr, C::kColPhi, C::kColX, q, warp, lane, reinterpret_cast<float *>(sm + C::kOffWh));
        ok = mbar_wait_cluster(&bars[2], (uint32_t)(b & 1));
        if (__syncthreads_or(!ok)) {
            timeout = true;
            if (tid == 0) latch(status, ST_TIMEOUT);
            break;
        }
        entry_inv_norms<C>(S, tid, S.diag());  // the diagonal itself was sent: reuse its buffer
        __syncthreads();
        own_losses<C>(S, tid, ks, lam, S.diag());
        __syncthreads();
        if (tid < NC) mbar_arrive_cluster(mapa(smem_u32(&bars[3]), (uint32_t)tid));  // this CTA's slots are read
        if (all_done) break;
    }
    cp_async_wait_all();
    if (timeout) {
        if (pending) mbar_wait(&bars[1], (uint32_t)(b & 1));
    } else if (tid < C::kOwn && !skip) {
        long long opix;
        float fx, fy;
        if (item_pixel(it, own0 + tid, opix, fx, fy)) {
            Lgt_out[opix] = S.acc(0)[tid];
            Lcf_out[opix] = S.acc(1)[tid];
            if (nc_out) nc_out[opix] = (int32_t)S.acc(2)[tid];
        }
    }
    if (save.F != nullptr && !timeout && !skip) {
        // the walk's end state for the backward: F_N of this CTA's 128
        // channels (TMEM lane = pixel; group g takes columns 64 g ..), and T
        // and the last contributor, which every CTA of the cluster holds alike
        // Each 32 x 32 block goes through the warp's padded tile in the operand
        // stages (free after the walk), so that lane l then stores 16 bytes of
        // pixel 4 i + l / 8: 128 contiguous bytes per pixel and store.
        tc_after();
        const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
        const int c0 = grp * 64, sub = lane >> 3, c4 = (lane & 7) * 4;
        float *tileb = reinterpret_cast<float *>(sm) + warp * (32 * 36);
        long long opix[8];
        bool oin[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float fx, fy;
            oin[i] = item_pixel(it, (warp & 3) * 32 + 4 * i + sub, opix[i], fx, fy);
        }
#pragma unroll 1
        for (int j = 0; j < 2; ++j) {
            float v[32];
            tmem_ld32(taddr + C::kColF + lanes + c0 + 32 * j, v);
#pragma unroll
            for (int i = 0; i < 8; ++i)
                *reinterpret_cast<float4 *>(tileb + lane * 36 + 4 * i) =
                    make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (oin[i])
                    *reinterpret_cast<float4 *>(save.F + opix[i] * (long long)(NC * 128) + q * 128 + c0 + 32 * j +
                                                c4) = *reinterpret_cast<const float4 *>(tileb + (4 * i + sub) * 36 + c4);
            __syncwarp();
        }
        if (q == 0 && grp == 0 && inside) {
            save.T[pix] = ps.T[pidx];
            save.last[pix] = ps.last[pidx];
        }
    }
    tc_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, 512);
    cluster_sync();  // no CTA leaves while another may still write to its shared memory
}

// ------------------------------------------------------------- backward
// The backward (App. A.2 with the NDFD terms of Sec. 3.3):
//   dL/dw_k = c_gt sigma_k + c_cf (sigma_k (W_{k-1} - F_{k-1} . f_k) + S_k - G_k . f_k),
//   S_k = sum_{i>k} sigma_i w_i,  G_k = sum_{i>k} sigma_i w_i f_i,
//   dL/dalpha_k = T_k dL/dw_k - Sw_k / (1 - alpha_k),  Sw_k = sum_{i>k} w_i dL/dw_i,
// then the footprint chain of the render backward.  Pass A rebuilds F_N
// front to back (weights and F += W F_c).  Pass B walks the chunks back to
// front; per chunk, with F_end and G_end the sums over the later entries:
//   X = F_end . F_c^T - W . Gs      (F_{k-1} . f_k plus w_k Gamma_kk)
//   Y = G_end . F_c^T + (sigma W) . Gs   (G_k . f_k)
//   F -= W . F_c,  G += (sigma W) . F_c
// with Gs[i][k] = f_i . f_k for i > k.  sigma needs the full Phi: the
// partial Phi rows go to the pixels' owner (round 1), which returns sigma w
// to every CTA (round 2); the partial X and Y rows then go to the owner
// (round 3), which runs the recursion for its pixels and adds their
// footprint gradients to the per-(camera, Gaussian) array.

template <int NC, int GEOM = FHGS_GEOM_EWA>
struct NBCfg {
    static constexpr int kNC = NC;
    using Rec = typename NRec<GEOM>::T;
    using RecSrc = typename NRec<GEOM>::Src;
    static constexpr int kGeom = GEOM;
    static constexpr int kG2 = NRec<GEOM>::kG2, kAcc = NRec<GEOM>::kAcc;
    static constexpr int kOwn = 128 / NC;  // the owner passes: warp w takes own pixels w, w + 8, ...
    static constexpr int kRow = 2 * kC + 4;
    static constexpr int kSlotF = kOwn * kRow + kC + kOwn;   // rows; Gram diagonal [64]; partial |f_gt|^2
    static constexpr int kFStages = 1;  // chunk b's features load under its weights
    static constexpr int kOffGt = 0;
    static constexpr int kOffF = kOffGt + 2 * 128 * 128;
    static constexpr int kOffWh = kOffF + kFStages * 2 * kC * 128;  // -W, then sigma W (hi)
    static constexpr int kOffWl = kOffWh + 128 * 128;
    static constexpr int kOffGh = kOffWl + 128 * 128;                // Gs: f_i . f_k for i > k (hi, lo)
    static constexpr int kOffGl = kOffGh + kC * 128;
    static constexpr int kOffRecv = kOffGl + kC * 128;
    static constexpr int kOffStash = kOffRecv + cal(NC * kSlotF * 4, 16);  // [3][kOwn][kStashRow]: alpha, T, sigma
    static constexpr int kOffRec = kOffStash + 3 * kOwn * kStashRow * 4;
    static constexpr int kOffGid = kOffRec + 2 * kC * (int)sizeof(Rec);
    // [9][128]: T, done, last, P0, L0, |f_gt|^2 per pixel, then 5 x kOwn scalars of the own pixels
    static constexpr int kOffPix = kOffGid + 3 * kC * 4;
    static constexpr int kOffDiag = kOffPix + 9 * 128 * 4;  // [2][64]: full Gram diagonal, inverse norms
    static constexpr int kOffAcc = kOffDiag + 2 * kC * 4;   // [64][kAcc] footprint gradients of the own pixels
    static constexpr int kOffBar = cal(kOffAcc + kC * kAcc * 4, 8);
    static constexpr int kSmem = 1024 + kOffBar + 128;      // 11 barriers, the TMEM slot, Lmax
    static_assert(kSmem <= 232448, "NDFD backward CTA exceeds the opt-in shared memory");
    static_assert(8 * 32 * 36 * 4 <= kOffRecv - kOffF, "the saved state's tiles must fit in the free stages");
    static constexpr uint32_t kColF = 0, kColG = 128, kColA = 256, kColB = 320, kColH = 384, kColL = 448;
};

// Back-to-front weights of one chunk for the 128 pixels.  The contributors
// are the entries before the pixel's last contributor (pos < last) that pass
// the alpha test; with T_end, the transmittance after the chunk, group 1
// (entries 32..63) starts from T_end / P_1 and group 0 from that / P_0 (P_g
// the product of (1 - alpha) over the group's contributors), then a forward
// running product gives T before each entry.  Writes -w (BF16 hi + lo) into
// the K-major weight operand, alpha and T of the own pixels into the stash,
// and T entering the chunk back into the state.
template <int GEOM>
__device__ __forceinline__ void chunk_weights_bwd(const Params &p, const typename NRec<GEOM>::T *R, int nb, int pos0,
                                                  int pidx, int grp,
                                                  float fpx, float fpy, PixState ps, uint8_t *sWh, uint8_t *sWl,
                                                  float *stash_a, float *stash_T, int own0, int own) {
    const float T_end = ps.T[pidx];
    const int last = ps.last[pidx];
    float a[32], l[32];
    float P = 1.f;
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
        const int j = grp * 32 + jj;
        float G, rho;
        const float al = NRec<GEOM>::alpha(R[j], fpx, fpy, p, G, rho);
        a[jj] = (j < nb && pos0 + j < last) ? al : 0.f;
        l[jj] = P;
        P *= 1.f - a[jj];
    }
    if (grp == 1) ps.P0[pidx] = P;
    __syncthreads();
    const float T1 = T_end / ps.P0[pidx];         // T entering group 1
    const float Ts = grp == 1 ? T1 : T1 / P;      // T entering this group
    const int pl = pidx - own0;
    const bool mine = pl >= 0 && pl < own;
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
        float w8[8], T8[8];
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const int jj = 8 * qq + h;
            T8[h] = Ts * l[jj];
            w8[h] = a[jj] * T8[h];
        }
        if (mine) {
            float *da = stash_a + pl * kStashRow + grp * 32 + 8 * qq, *dT = stash_T + pl * kStashRow + grp * 32 + 8 * qq;
            *reinterpret_cast<float4 *>(da) = make_float4(a[8 * qq], a[8 * qq + 1], a[8 * qq + 2], a[8 * qq + 3]);
            *reinterpret_cast<float4 *>(da + 4) = make_float4(a[8 * qq + 4], a[8 * qq + 5], a[8 * qq + 6], a[8 * qq + 7]);
            *reinterpret_cast<float4 *>(dT) = make_float4(T8[0], T8[1], T8[2], T8[3]);
            *reinterpret_cast<float4 *>(dT + 4) = make_float4(T8[4], T8[5], T8[6], T8[7]);
        }
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            __nv_bfloat16 h0, l0, h1, l1;
            split_bf16(-w8[2 * u], h0, l0);
            split_bf16(-w8[2 * u + 1], h1, l1);
            hw[u] = pack2(h0, h1);
            lw[u] = pack2(l0, l1);
        }
        *reinterpret_cast<uint4 *>(sWh + swz(pidx, grp * 4 + qq)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(sWl + swz(pidx, grp * 4 + qq)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    __syncthreads();  // T_end and P_1 are read before T is rewritten
    if (grp == 0) ps.T[pidx] = Ts;
}

// Half of a pixel row exchange: warps w and w + 4 (lane quadrant w % 4) send
// columns [32 (w / 4), + 32) of the TMEM accumulator at `col` into the
// `half` (0: first 64 floats, 1: second) of this CTA's slot at the owner of
// those pixels, through a 2.5 KB staging tile per warp; warps 0..3 add the
// partial |f_gt|^2 when `ngt`, the owner's first warp w >= 4 the Gram
// diagonal when `diag`; every thread then arrives once on the owner's
// barrier `bar` (unless `arrive` is false: a second call completes the
// exchange).  Without a staging tile (stage == nullptr) each thread stores
// its own row.
template <class C>
__device__ __forceinline__ void send_half(const ItemSmem<C> &S, uint32_t taddr, uint32_t col, int half, int q,
                                          int warp, int lane, float *stage, bool ngt, bool diag, const float *dvals,
                                          uint64_t *bar, bool arrive = true) {
    constexpr int NC = C::kNC;
    constexpr int kSR = 20;
    const int qd = warp & 3, dst = qd * NC / 4, h2 = warp >> 2;
    const int row0 = qd * 32 - dst * C::kOwn;
    const uint32_t slot = mapa(smem_u32(S.recv() + q * C::kSlotF), (uint32_t)dst);
#pragma unroll
    for (int piece = 0; piece < 2; ++piece) {
        float v[16];
        tmem_ld16(taddr + ((uint32_t)(qd * 32) << 16) + col + 32 * h2 + 16 * piece, v);
        if (stage == nullptr) {  // no free shared memory: each thread stores its own row
#pragma unroll
            for (int i = 0; i < 4; ++i)
                st_cluster_v4(slot + (uint32_t)((row0 + lane) * C::kRow + half * kC + 32 * h2 + 16 * piece + 4 * i) * 4u,
                              v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            continue;
        }
        float *st = stage + warp * 32 * kSR;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            *reinterpret_cast<float4 *>(st + lane * kSR + 4 * i) = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        __syncwarp();
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            const int r = 8 * it + (lane >> 2), c4 = (lane & 3) * 4;
            const float4 x = *reinterpret_cast<const float4 *>(st + r * kSR + c4);
            st_cluster_v4(slot + (uint32_t)((row0 + r) * C::kRow + half * kC + 32 * h2 + 16 * piece + c4) * 4u, x.x,
                          x.y, x.z, x.w);
        }
        __syncwarp();
    }
    if (ngt && h2 == 0) st_cluster_f32(slot + (uint32_t)(C::kOwn * C::kRow + kC + row0 + lane) * 4u, S.ngt()[qd * 32 + lane]);
    if (diag && h2 == 1 && qd == dst * (4 / NC))
        st_cluster_v2(slot + (uint32_t)(C::kOwn * C::kRow + 2 * lane) * 4u, dvals[2 * lane], dvals[2 * lane + 1]);
    if (arrive) mbar_arrive_cluster(mapa(smem_u32(bar), (uint32_t)dst));
}

// Round 1 at the owner: adds the NC partial Phi rows of its pixels, forms
// sigma of every contributor (w = alpha T > 0; 0 otherwise) into the stash
// and sends sigma w of its pixels to the second half of its slot in every
// CTA (round 2), one arrival per thread and CTA on their `bar`.  Warp w
// takes the own pixels w, w + 8, ...; lane l entries l and l + 32, so that
// each remote store writes 128 contiguous bytes.  inv holds the entries'
// inverse feature norms, igt the own pixels' inverse |f_gt|.
template <class C>
__device__ __forceinline__ void owner_sigma(const ItemSmem<C> &S, int warp, int lane, int q, float ks, float lam,
                                            const float *inv, const float *igt, const float *stash_a,
                                            const float *stash_T, float *stash_s, uint64_t *bar) {
    constexpr int NC = C::kNC;
    const float inv0 = inv[lane], inv1 = inv[lane + 32];
#pragma unroll
    for (int pl = warp; pl < C::kOwn; pl += 8) {
        float ph0 = 0.f, ph1 = 0.f;
#pragma unroll
        for (int sl = 0; sl < NC; ++sl) {
            const float *row = S.recv() + sl * C::kSlotF + pl * C::kRow;
            ph0 += row[lane];
            ph1 += row[lane + 32];
        }
        const float ig = igt[pl];
        const float w0 = stash_a[pl * kStashRow + lane] * stash_T[pl * kStashRow + lane];
        const float w1 = stash_a[pl * kStashRow + lane + 32] * stash_T[pl * kStashRow + lane + 32];
        const float s0 = w0 > 0.f ? sigma_fast(ph0 * inv0 * ig, ks, lam) : 0.f;
        const float s1 = w1 > 0.f ? sigma_fast(ph1 * inv1 * ig, ks, lam) : 0.f;
        stash_s[pl * kStashRow + lane] = s0;
        stash_s[pl * kStashRow + lane + 32] = s1;
        const uint32_t off = smem_u32(S.recv()) + (uint32_t)(q * C::kSlotF + pl * C::kRow + kC + lane) * 4u;
#pragma unroll
        for (int d = 0; d < NC; ++d) {
            const uint32_t dst = mapa(off, (uint32_t)d);
            st_cluster_f32(dst, s0 * w0);
            st_cluster_f32(dst + 128u, s1 * w1);
        }
    }
#pragma unroll
    for (int d = 0; d < NC; ++d) mbar_arrive_cluster(mapa(smem_u32(bar), (uint32_t)d));
}

// Round 2 at every CTA: sigma w of all 128 pixels (second halves of the
// owners' slots) -> the K-major [128 px][64] operand as BF16 hi + lo.
template <class C>
__device__ __forceinline__ void build_sigma_w(const ItemSmem<C> &S, int pidx, int grp, uint8_t *sWh, uint8_t *sWl) {
    const int r = pidx / C::kOwn, pl = pidx - r * C::kOwn;
    const float *row = S.recv() + r * C::kSlotF + pl * C::kRow + kC + grp * 32;
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
        const float4 a = *reinterpret_cast<const float4 *>(row + 8 * qq);
        const float4 b = *reinterpret_cast<const float4 *>(row + 8 * qq + 4);
        const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            __nv_bfloat16 h0, l0, h1, l1;
            split_bf16(v[2 * u], h0, l0);
            split_bf16(v[2 * u + 1], h1, l1);
            hw[u] = pack2(h0, h1);
            lw[u] = pack2(l0, l1);
        }
        *reinterpret_cast<uint4 *>(sWh + swz(pidx, grp * 4 + qq)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(sWl + swz(pidx, grp * 4 + qq)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
}

// Inclusive suffix sum over the lanes: lane l gets the sum of lanes l..31.
__device__ __forceinline__ float lane_suffix(float x, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const float t = __shfl_down_sync(0xffffffffu, x, d);
        if (lane + d < 32) x += t;
    }
    return x;
}

// Round 3 at the owner: X and Y of its pixels (sums of the NC partials), then
// back to front over the chunk, per pixel: S_k, dL/dw_k, Sw_k and dL/dalpha_k,
// and the footprint gradients (mean x, y; conic A, B, C; opacity) of every
// contributor.  Warp w takes the own pixels w, w + 8, ...; lane l entries l
// and l + 32 (entry l + 32 comes later in the walk), so the suffix sums are
// lane scans and each lane sums its two entries' gradients over its pixels
// in registers before one shared-memory atomic per component and warp into
// acc[entry][0..5].  own holds per own pixel: c_gt, c_cf, and S and Sw of the
// later chunks (updated).
template <class C>
__device__ __forceinline__ void owner_grads(const ItemSmem<C> &S, int warp, int lane, const Params &p,
                                            const typename C::Rec *R, const Item &it, int own0, const float *diag,
                                            const float *stash_a, const float *stash_T, const float *stash_s,
                                            float *own, float *acc) {
    constexpr int NC = C::kNC;
    using NR = NRec<C::kGeom>;
    const typename C::Rec rec0 = R[lane], rec1 = R[lane + 32];
    const float dg0 = diag[lane], dg1 = diag[lane + 32];
    float g0[NR::kN], g1[NR::kN];
#pragma unroll
    for (int c = 0; c < NR::kN; ++c) g0[c] = g1[c] = 0.f;
#pragma unroll 2
    for (int pl = warp; pl < C::kOwn; pl += 8) {
        long long pix;
        float fpx, fpy;
        const bool inside = item_pixel(it, own0 + pl, pix, fpx, fpy);
        float X0 = 0.f, X1 = 0.f, Y0 = 0.f, Y1 = 0.f;
#pragma unroll
        for (int sl = 0; sl < NC; ++sl) {
            const float *row = S.recv() + sl * C::kSlotF + pl * C::kRow;
            X0 += row[lane];
            X1 += row[lane + 32];
            Y0 += row[kC + lane];
            Y1 += row[kC + lane + 32];
        }
        const float a0 = stash_a[pl * kStashRow + lane], a1 = stash_a[pl * kStashRow + lane + 32];
        const float T0 = stash_T[pl * kStashRow + lane], T1 = stash_T[pl * kStashRow + lane + 32];
        const float s0 = stash_s[pl * kStashRow + lane], s1 = stash_s[pl * kStashRow + lane + 32];
        const float w0 = a0 * T0, w1 = a1 * T1;
        X0 -= w0 * dg0;  // F_{k-1} . f_k: the product took F after entry k
        X1 -= w1 * dg1;
        const float cgt = own[pl], ccf = own[C::kOwn + pl];
        const float Send = own[2 * C::kOwn + pl], Swend = own[3 * C::kOwn + pl];
        // S_k = S of the later chunks + sigma w of the chunk's later entries
        const float v0 = s0 * w0, v1 = s1 * w1;
        const float i1 = lane_suffix(v1, lane), i0 = lane_suffix(v0, lane);
        const float t1 = __shfl_sync(0xffffffffu, i1, 0), t0 = __shfl_sync(0xffffffffu, i0, 0);
        const float S1 = Send + (i1 - v1), S0 = Send + t1 + (i0 - v0);
        const float gw0 = cgt * s0 + ccf * (s0 * ((1.f - T0) - X0) + S0 - Y0);
        const float gw1 = cgt * s1 + ccf * (s1 * ((1.f - T1) - X1) + S1 - Y1);
        const float u0 = w0 * gw0, u1 = w1 * gw1;
        const float j1 = lane_suffix(u1, lane), j0 = lane_suffix(u0, lane);
        const float r1 = __shfl_sync(0xffffffffu, j1, 0), r0 = __shfl_sync(0xffffffffu, j0, 0);
        const float Sw1 = Swend + (j1 - u1), Sw0 = Swend + r1 + (j0 - u0);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float w = h ? w1 : w0;
            if (!(w > 0.f && inside)) continue;
            const float al = h ? a1 : a0, T = h ? T1 : T0, gw = h ? gw1 : gw0, Sw = h ? Sw1 : Sw0;
            const float dal = T * gw - Sw / (1.f - al);
            if (h) NR::footprint(rec1, fpx, fpy, dal, p, g1);
            else NR::footprint(rec0, fpx, fpy, dal, p, g0);
        }
        if (lane == 0) {  // the chunk's totals carry to the earlier chunks
            own[2 * C::kOwn + pl] = Send + t1 + t0;
            own[3 * C::kOwn + pl] = Swend + r1 + r0;
        }
    }
#pragma unroll
    for (int c = 0; c < NR::kN; ++c) {
        if (g0[c] != 0.f) atomicAdd(&acc[lane * NR::kAcc + c], g0[c]);
        if (g1[c] != 0.f) atomicAdd(&acc[(lane + 32) * NR::kAcc + c], g1[c]);
    }
}

template <int NC, int GEOM>
__global__ void __launch_bounds__(256, 1)
    k_ndfd_bwd_tc(long long N, CamSet cs, Params p, ProjView pv, const uint32_t *__restrict__ gids,
                  const uint32_t *__restrict__ ranges, const __nv_bfloat16 *__restrict__ feats,
                  const __nv_bfloat16 *__restrict__ fgt, float ks, float lam, const float *__restrict__ dLgt,
                  const float *__restrict__ dLcf, float *g2d, NdfdState saved, unsigned *status) {
    using C = NBCfg<NC, GEOM>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align_smem_1024(smem_raw);
    if (probe_wait_expired(p, sm, status)) return;  // uniform over the grid, before any cluster operation
    const ItemSmem<C> S{sm, smem_u32(sm)};
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, grp = tid >> 7, pidx = tid & 127;
    const int q = (int)cluster_rank(), own0 = q * C::kOwn;
    const Item it = make_item(cs, ranges, (int)(blockIdx.x / NC), q);
    const bool skip = (*(volatile unsigned *)status & ST_TIMEOUT) != 0;  // see the forward
    const int nlist = skip ? 0 : (int)((it.e - it.s + kC - 1) / kC);
    // [0] pass-A update, [1] Gamma + Phi, [2] X + F update, [3] Y + G update (local commits);
    // [4] round-1 rows, [5] round-2 sigma w, [6] round-3 rows (data ready here);
    // [7] round-2 data consumed, [8] round-3 rows consumed (at the senders)
    uint64_t *bars = S.bars();
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 9);
    int *sLmax = reinterpret_cast<int *>(bars + 10);
    const PixState ps = S.pix();
    float *own = S.ngt() + 128;  // [4][kOwn]: c_gt, c_cf, S, Sw of the own pixels; then [kOwn] inverse |f_gt|
    float *igt = own + 4 * C::kOwn;
    float *stash_a = reinterpret_cast<float *>(sm + C::kOffStash), *stash_T = stash_a + C::kOwn * kStashRow;
    float *stash_s = stash_T + C::kOwn * kStashRow;
    float *diag = reinterpret_cast<float *>(sm + C::kOffDiag), *inv = diag + kC;
    float *acc = reinterpret_cast<float *>(sm + C::kOffAcc);
    long long pix;
    float fpx, fpy;
    const bool inside = item_pixel(it, pidx, pix, fpx, fpy);

    if (tid == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(&bars[i], 1);
        mbar_init(&bars[4], 256);
        mbar_init(&bars[5], 256 * NC);
        mbar_init(&bars[6], 256);
        mbar_init(&bars[7], NC);
        mbar_init(&bars[8], NC);
        fence_mbar_init();
        *sLmax = 0;
    }
    if (warp == 0) tmem_alloc(tslot, 512);
    if (grp == 0) {
        ps.T[pidx] = 1.f;
        ps.done[pidx] = inside ? 0 : 1;
        ps.last[pidx] = 0;
    }
    if (tid < C::kOwn) {
        long long op;
        float fx, fy;
        const bool in = item_pixel(it, own0 + tid, op, fx, fy);
        own[tid] = in ? dLgt[op] : 0.f;
        own[C::kOwn + tid] = in ? dLcf[op] : 0.f;
        own[2 * C::kOwn + tid] = own[3 * C::kOwn + tid] = 0.f;
    }
    for (int i = tid; i < kC * C::kAcc; i += 256) acc[i] = 0.f;
    const typename C::RecSrc *recs =
        reinterpret_cast<const typename C::RecSrc *>(GEOM == FHGS_GEOM_SURFEL ? (const void *)pv.srec
                                                                             : (const void *)pv.rec) +
        (long long)it.ci * N;
    const Loader<C> L{S, gids, recs, feats, it.s, it.e, nlist, q, tid};
    float *g2dc = g2d + (long long)it.ci * N * C::kG2;
    load_gt<C>(S, it, fgt, q, tid);
    L.gid(0);
    L.gid(1);
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t taddr = *tslot;
    cluster_sync();  // every CTA's barriers are initialised before the first remote arrival
    cp_async_wait<1>();  // F_gt and the ids of chunk 0
    __syncthreads();
    L.records(0);
    gt_norm<C>(S, tid);

    const uint32_t sGt = S.sm_s + C::kOffGt, sWh = S.sm_s + C::kOffWh, sWl = S.sm_s + C::kOffWl;
    const uint32_t sGh = S.sm_s + C::kOffGh, sGl = S.sm_s + C::kOffGl;
    const uint64_t dGt = sdesc(sGt, 16, 1024), dWh = sdesc(sWh, 16, 1024), dWl = sdesc(sWl, 16, 1024);
    const uint64_t dGh = sdesc(sGh, 16, 1024), dGl = sdesc(sGl, 16, 1024);
    const uint32_t tF = taddr + C::kColF, tG = taddr + C::kColG, tA = taddr + C::kColA, tB = taddr + C::kColB;
    const uint32_t tH = taddr + C::kColH, tL = taddr + C::kColL;
    float *stage = reinterpret_cast<float *>(sm + C::kOffWh);  // row staging while the weight operands are free

    bool timeout = false;
    int pend = -1;  // a commit barrier whose phase `pend_ph` may still be in flight
    uint32_t pend_ph = 0;
    // ---- pass A: F_N, T after the walk and the last contributors, front to
    // back; or, when the forward saved them, read back
    if (saved.F != nullptr && !skip) {
        if (grp == 0) {
            ps.T[pidx] = inside ? saved.T[pix] : 1.f;
            ps.last[pidx] = inside ? saved.last[pix] : 0;
        }
        // Each 32 x 32 block of the warp's pixels and channels comes in as 128
        // contiguous bytes per pixel and load (lane l: 16 bytes of pixel
        // 4 i + l / 8), through the warp's padded tile in the feature, weight
        // and Gram stages (free until pass B), then row by row into TMEM.
        const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
        const int c0 = grp * 64, sub = lane >> 3, c4 = (lane & 7) * 4;
        float *tileb = reinterpret_cast<float *>(sm + C::kOffF) + warp * (32 * 36);
        long long ipix[8];
        bool iin[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float fx, fy;
            iin[i] = item_pixel(it, (warp & 3) * 32 + 4 * i + sub, ipix[i], fx, fy);
        }
#pragma unroll 1
        for (int j = 0; j < 2; ++j) {
            float4 x[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                x[i] = iin[i] ? *reinterpret_cast<const float4 *>(saved.F + ipix[i] * (long long)(NC * 128) + q * 128 +
                                                                  c0 + 32 * j + c4)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int i = 0; i < 8; ++i) *reinterpret_cast<float4 *>(tileb + (4 * i + sub) * 36 + c4) = x[i];
            __syncwarp();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t v[16];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float4 y = *reinterpret_cast<const float4 *>(tileb + lane * 36 + 16 * h + 4 * k);
                    v[4 * k] = __float_as_uint(y.x);
                    v[4 * k + 1] = __float_as_uint(y.y);
                    v[4 * k + 2] = __float_as_uint(y.z);
                    v[4 * k + 3] = __float_as_uint(y.w);
                }
                tmem_st16(tF + lanes + c0 + 32 * j + 16 * h, v);
            }
            __syncwarp();
        }
        tmem_st_wait();
        tc_before();  // the stores precede the MMAs on F after the barrier below
    }
    for (int b = 0; b < ((saved.F != nullptr) ? 0 : nlist); ++b) {
        const uint32_t base = it.s + (uint32_t)b * kC;
        const int nb = (int)min((uint32_t)kC, it.e - base);
        L.features(b);  // its stage was last read by the previous chunk's update, complete
        cp_async_wait<1>();  // ids of b+1 and records of b (the features of b are the newest group)
        __syncthreads();
        L.gid(b + 2);
        L.records(b + 1);
        const bool all_done = chunk_weights<GEOM>(p, S.rec(b), nb, (int)(base - it.s), pidx, grp, fpx, fpy, ps,
                                                  sm + C::kOffWh, sm + C::kOffWl, stash_a, stash_T, own0, C::kOwn,
                                                  false);
        cp_async_wait<2>();  // the features of b
        fence_async_smem();
        tc_before();
        __syncthreads();
        if (tid == 0) {
            tc_after();
            issue_update(tF, dWh, dWl, chunk_desc(S.feat_s(b)), b > 0);
            mma_commit(&bars[0]);
        }
        pend = 0;
        pend_ph = (uint32_t)(b & 1);
        const bool ok = mbar_wait(&bars[0], (uint32_t)(b & 1));  // the operands are reused by the next chunk
        if (__syncthreads_or(!ok)) {
            timeout = true;
            if (tid == 0) latch(status, ST_TIMEOUT);
            break;
        }
        pend = -1;
        if (all_done) break;
    }
    cp_async_wait_all();
    if (grp == 0) atomicMax(sLmax, ps.last[pidx]);
    tc_after();
    __syncthreads();
    const int nB = timeout ? 0 : (min(*sLmax, (int)(it.e - it.s)) + kC - 1) / kC;
    if (tid < C::kOwn) {  // inverse |f_gt| of the own pixels: the partial norms are exchanged in round 1
        igt[tid] = 0.f;
    }

    // ---- pass B: back to front
    if (nB > 0) {
        L.gid(nB - 1);
        L.gid(nB - 2);
        cp_async_wait<1>();
        __syncthreads();
        L.records(nB - 1);
    }
    for (int b = nB - 1, itn = 0; b >= 0; --b, ++itn) {
        const uint32_t ph = (uint32_t)(itn & 1);
        const uint32_t base = it.s + (uint32_t)b * kC;
        const int nb = (int)min((uint32_t)kC, it.e - base);
        L.features(b);
        cp_async_wait<1>();  // ids of b-1 and records of b (features of b are the newest group)
        __syncthreads();
        L.gid(b - 2);
        L.records(b - 1);
        chunk_weights_bwd<GEOM>(p, S.rec(b), nb, (int)(base - it.s), pidx, grp, fpx, fpy, ps, sm + C::kOffWh,
                                sm + C::kOffWl, stash_a, stash_T, own0, C::kOwn);
        split_to_tmem(taddr, C::kColF, C::kColH, C::kColL, warp);  // F_end
        cp_async_wait<2>();  // the features of b (the records of b-1 and ids of b-2 may be in flight)
        fence_async_smem();
        tc_before();
        __syncthreads();
        const ChunkDesc cd = chunk_desc(S.feat_s(b));
        if (tid == 0) {
            tc_after();
            issue_gram(tA, cd);
            issue_rows_x_chunk(tB, dGt, 128 * 128, cd, false);
            mma_commit(&bars[1]);
        }
        pend = 1;
        pend_ph = ph;
        bool ok = mbar_wait(&bars[1], ph);
        tc_after();
        if ((warp & 3) < 2 && ok) gram_part(taddr, C::kColA, warp, lane, false, sm + C::kOffGh, sm + C::kOffGl, diag);
        fence_async_smem();
        // round 1: every owner has consumed the round-3 rows of the previous chunk
        if (ok && itn > 0) ok = mbar_wait_cluster(&bars[8], (uint32_t)((itn - 1) & 1));
        if (__syncthreads_or(!ok)) {
            timeout = true;
            if (tid == 0) latch(status, ST_TIMEOUT);
            break;
        }
        pend = -1;
        // the weight operands still feed X and the F update: no staging tile
        send_half<C>(S, taddr, C::kColB, 0, q, warp, lane, nullptr, true, true, diag, &bars[4]);
        tc_before();
        __syncthreads();  // Gamma and Phi are read: their columns take X and Y
        if (tid == 0) {
            tc_after();
            issue_tmem_x_chunk(tA, tH, tL, cd, false);        // X = F_end F_c^T
            issue_w_gram(tA, dWh, dWl, dGh, dGl, true);       //   - W Gs
            issue_update(tF, dWh, dWl, cd, true);             // F -= W F_c
            mma_commit(&bars[2]);
        }
        pend = 2;
        pend_ph = ph;
        // round 1 at the owner: sigma of its pixels, sigma w to every CTA
        ok = mbar_wait_cluster(&bars[4], ph);
        if (__syncthreads_or(!ok)) {
            timeout = true;
            if (tid == 0) latch(status, ST_TIMEOUT);
            break;
        }
        if (tid < kC) {
            float d2 = 0.f;
#pragma unroll
            for (int sl = 0; sl < NC; ++sl) d2 += S.recv()[sl * C::kSlotF + C::kOwn * C::kRow + tid];
            diag[tid] = d2;
            inv[tid] = d2 > 0.f ? 1.f / sqrtf(d2) : 0.f;
        }
        if (itn == 0 && tid < C::kOwn) {
            float n2 = 0.f;
#pragma unroll
            for (int sl = 0; sl < NC; ++sl) n2 += S.recv()[sl * C::kSlotF + C::kOwn * C::kRow + kC + tid];
            igt[tid] = n2 > 0.f ? 1.f / sqrtf(n2) : 0.f;
        }
        __syncthreads();
        owner_sigma<C>(S, warp, lane, q, ks, lam, inv, igt, stash_a, stash_T, stash_s, &bars[5]);
        // X's reads of F hi/lo and of -W are done: G_end -> hi/lo, sigma w -> the weight operands
        ok = mbar_wait(&bars[2], ph);
        if (ok) {
            tc_after();
            if (itn > 0) split_to_tmem(taddr, C::kColG, C::kColH, C::kColL, warp);
        }
        if (ok) ok = mbar_wait_cluster(&bars[5], ph);
        if (__syncthreads_or(!ok)) {
            timeout = true;
            if (tid == 0) latch(status, ST_TIMEOUT);
            break;
        }
        build_sigma_w<C>(S, pidx, grp, sm + C::kOffWh, sm + C::kOffWl);
        fence_async_smem();
        tc_before();
        __syncthreads();
        if (tid < NC) mbar_arrive_cluster(mapa(smem_u32(&bars[7]), (uint32_t)tid));  // round-2 data consumed
        if (tid == 0) {
            tc_after();
            if (itn > 0) issue_tmem_x_chunk(tB, tH, tL, cd, false);   // Y = G_end F_c^T
            issue_w_gram(tB, dWh, dWl, dGh, dGl, itn > 0);            //   + sigma W Gs
            issue_update(tG, dWh, dWl, cd, itn > 0);                  // G += sigma W F_c
            mma_commit(&bars[3]);
        }
        pend = 3;
        pend_ph = ph;
        ok = mbar_wait(&bars[3], ph);
        if (ok) ok = mbar_wait_cluster(&bars[7], ph);  // every owner has built its sigma W operand
        if (__syncthreads_or(!ok)) {
            timeout = true;
            if (tid == 0) latch(status, ST_TIMEOUT);
            break;
        }
        pend = -1;
        tc_after();
        // round 3: X (first halves) and Y (second halves) to the owners
        send_half<C>(S, taddr, C::kColA, 0, q, warp, lane, stage, false, false, diag, &bars[6], false);
        send_half<C>(S, taddr, C::kColB, 1, q, warp, lane, stage, false, false, diag, &bars[6]);
        ok = mbar_wait_cluster(&bars[6], ph);
        if (__syncthreads_or(!ok)) {
            timeout = true;
            if (tid == 0) latch(status, ST_TIMEOUT);
            break;
        }
        owner_grads<C>(S, warp, lane, p, S.rec(b), it, own0, diag, stash_a, stash_T, stash_s, own, acc);
        __syncthreads();
        if (tid < NC) mbar_arrive_cluster(mapa(smem_u32(&bars[8]), (uint32_t)tid));  // round-3 rows consumed
        if (tid < kC && tid < nb) {  // the own pixels' footprint gradients of the chunk's primitives
            float *a = acc + tid * C::kAcc;
            float *dst = g2dc + C::kG2 * (long long)S.gid(b)[tid];
#pragma unroll
            for (int k = 0; k < NRec<GEOM>::kN; k += 4) {
                if (k + 4 <= NRec<GEOM>::kN) {
                    const float4 u = *reinterpret_cast<const float4 *>(a + k);
                    if (u.x != 0.f || u.y != 0.f || u.z != 0.f || u.w != 0.f)
                        atomicAdd(reinterpret_cast<float4 *>(dst + k), u);
                    *reinterpret_cast<float4 *>(a + k) = make_float4(0.f, 0.f, 0.f, 0.f);
                } else {
                    const float2 t = *reinterpret_cast<const float2 *>(a + k);
                    if (t.x != 0.f || t.y != 0.f) atomicAdd(reinterpret_cast<float2 *>(dst + k), t);
                    *reinterpret_cast<float2 *>(a + k) = make_float2(0.f, 0.f);
                }
            }
        }
    }
    cp_async_wait_all();
    if (timeout && pend >= 0) mbar_wait(&bars[pend], pend_ph);
    tc_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, 512);
    cluster_sync();  // no CTA leaves while another may still write to its shared memory
}

// Launches one cluster of NC CTAs per (tile, half): grid = 2 NC tiles.
template <int NC, typename... Args>
void launch_cluster(void (*kernel)(Args...), int smem, unsigned n_items, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_items * NC);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = NC;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    note_launch(1);
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int NC, int GEOM>
void launch_fwd_tc_t(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                     const __nv_bfloat16 *feats, const __nv_bfloat16 *fgt, float ks, float lam, float *Lgt,
                     float *Lcf, int32_t *nc, NdfdState save, unsigned *status, cudaStream_t st) {
    static std::atomic<unsigned long long> smem_set{0};
    allow_max_smem(smem_set, k_ndfd_fwd_tc<NC, GEOM>);
    launch_cluster<NC>(k_ndfd_fwd_tc<NC, GEOM>, NCfg<NC, GEOM>::kSmem, (unsigned)cs.total_tiles * 2u, st, N, cs, p, pv,
                       (const uint32_t *)bins.gids, (const uint32_t *)bins.ranges, feats, fgt, ks, lam, Lgt, Lcf, nc,
                       save, status);
}

template <int NC, int GEOM>
void launch_bwd_tc_t(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                     const __nv_bfloat16 *feats, const __nv_bfloat16 *fgt, float ks, float lam, const float *dLgt,
                     const float *dLcf, float *g2d, NdfdState saved, unsigned *status, cudaStream_t st) {
    static std::atomic<unsigned long long> smem_set{0};
    allow_max_smem(smem_set, k_ndfd_bwd_tc<NC, GEOM>);
    launch_cluster<NC>(k_ndfd_bwd_tc<NC, GEOM>, NBCfg<NC, GEOM>::kSmem, (unsigned)cs.total_tiles * 2u, st, N, cs, p, pv,
                       (const uint32_t *)bins.gids, (const uint32_t *)bins.ranges, feats, fgt, ks, lam, dLgt, dLcf,
                       g2d, saved, status);
}

}  // namespace

bool ndfd_tc_supported(int D, int geom) {
    return geom == FHGS_GEOM_SURFEL ? D == 512 : (D == 256 || D == 512);  // surfels: the 4-CTA layout only fits
}

void launch_ndfd_bwd_tc(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                        const __nv_bfloat16 *feats, const __nv_bfloat16 *fgt, int D, float ks, float lam,
                        const float *dLgt, const float *dLcf, float *g2d, NdfdState saved, unsigned *status,
                        cudaStream_t st) {
    if (cs.total_tiles == 0) return;
    if (p.geom == FHGS_GEOM_SURFEL) {
        if (D == 512)
            launch_bwd_tc_t<4, FHGS_GEOM_SURFEL>(N, cs, p, pv, bins, feats, fgt, ks, lam, dLgt, dLcf, g2d, saved,
                                                 status, st);
    } else if (D == 512) {
        launch_bwd_tc_t<4, FHGS_GEOM_EWA>(N, cs, p, pv, bins, feats, fgt, ks, lam, dLgt, dLcf, g2d, saved, status, st);
    } else if (D == 256) {
        launch_bwd_tc_t<2, FHGS_GEOM_EWA>(N, cs, p, pv, bins, feats, fgt, ks, lam, dLgt, dLcf, g2d, saved, status, st);
    }
}

void launch_ndfd_fwd_tc(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                        const __nv_bfloat16 *feats, const __nv_bfloat16 *fgt, int D, float ks, float lam, float *Lgt,
                        float *Lcf, int32_t *nc, NdfdState save, unsigned *status, cudaStream_t st) {
    if (cs.total_tiles == 0) return;
    if (p.geom == FHGS_GEOM_SURFEL) {
        if (D == 512)
            launch_fwd_tc_t<4, FHGS_GEOM_SURFEL>(N, cs, p, pv, bins, feats, fgt, ks, lam, Lgt, Lcf, nc, save, status,
                                                 st);
    } else if (D == 512) {
        launch_fwd_tc_t<4, FHGS_GEOM_EWA>(N, cs, p, pv, bins, feats, fgt, ks, lam, Lgt, Lcf, nc, save, status, st);
    } else if (D == 256) {
        launch_fwd_tc_t<2, FHGS_GEOM_EWA>(N, cs, p, pv, bins, feats, fgt, ks, lam, Lgt, Lcf, nc, save, status, st);
    }
}

}  // namespace fhgs
