// Tensor-core (tcgen05) render kernels for sm_103a.
//
// The feature half of Eq. 4, F(p) = sum_i w_i(p) f_i, is per tile a dense
// contraction: F(P x D) += W(P x B) . Fe(B x D) with W the compositing
// weights of a batch of B depth-sorted Gaussians.  One CTA owns a half tile
// (16 x 8 = 128 pixels, one pixel per thread = one TMEM lane) and a slice of
// DN feature columns.  Per batch its threads compute the weights on the CUDA
// cores (FP32 alpha, T and RGB exactly as the FP32 path), write them as BF16
// into shared memory in the UMMA 128-byte-swizzled K-major layout, while
// cp.async stages the batch's feature rows (BF16, MN-major, swizzled); one
// thread then issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) into a
// TMEM accumulator of 128 lanes x DN columns.  Two stages overlap the next
// batch's weights and loads with the running MMAs; tcgen05.commit on an
// mbarrier frees a stage.  After the last batch the accumulator is read with
// tcgen05.ld and written once to the feature image.
//
// The backward (App. A.2) walks each half tile back to front in batches of
// 64: G(P x B) = dF(P x DN) . Fe(B x DN)^T on the tensor cores (dF split
// into BF16 hi + lo parts, two MMAs, so G carries ~16 mantissa bits), then
// the scalar pass (alpha, T, dL/dalpha, footprint gradients) on the CUDA
// cores, then dFe(B x DN) = W^T(B x P) . dF(P x DN) (hi + lo) with M padded
// to 128 by a zero block, drained from TMEM into the feature gradient with
// vector atomics.  Transmittance is recovered without a divide per Gaussian:
// per 32-Gaussian sub-batch T_start = T_end / prod(1 - alpha), then a
// forward prefix product.  dL/dalpha is linear in g_i = dC.c_i + dF.f_i, so
// each DN slice adds its own share of the footprint gradients.
//
// Every mbarrier wait is bounded (2 s of %globaltimer); on expiry the kernel
// latches FHGS_ERR_TIMEOUT, waits once more (bounded) for its MMAs, frees its
// TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <type_traits>
#include <cstring>

#include "fhgs_internal.cuh"
#include "tc_ptx.cuh"

namespace fhgs {
namespace {

using namespace tc;

// ------------------------------------------------------------- forward
constexpr int kFB = 64;  // Gaussians per forward batch (MMA K)

// 256 threads: two groups of 4 warps share the half tile's 128 pixels; group g
// weighs Gaussians [32 g, 32 g + 32) of each batch.  Both groups evaluate
// their alphas and the running products of (1 - alpha) over their own 32 at
// once; after one exchange of group 0's product each group knows the
// transmittance entering its Gaussians (T decreases along the list, so group
// 0 stops inside the batch exactly when T_in P_0 < t_eps), and both
// finalise their weights in parallel.
//
// Loads run ahead of use: the ids of batch b+2, the records of batch b+1 and
// (once the MMA of batch b-1 has freed its stage) the feature rows of batch
// b+1 are in flight while batch b is weighed.  With one feature stage (DN =
// 512, two CTAs per SM) batch b's rows load under its own weights.
template <int DN, int GEOM = FHGS_GEOM_EWA>
struct FwdCfg {
    static constexpr int kWBytes = 128 * 128;            // 128 px x 64 BF16 weights
    static constexpr int kFBytes = kFB * DN * 2;         // 64 rows x DN BF16 features
    static constexpr int kNSub = DN > 256 ? DN / 256 : 1;
    static constexpr int kMmaN = DN > 256 ? 256 : DN;
    static constexpr int kRecBytes = kFB * (GEOM == FHGS_GEOM_SURFEL ? 64 : 48);  // GRec or SRec
    // two feature stages, except at DN = 512 where one keeps the CTA small
    // enough for two per SM (one CTA's epilogue then runs beside the other's
    // batches)
    static constexpr int kFStages = DN >= 512 ? 1 : 2;
    static constexpr int kOffF = 2 * kWBytes;
    static constexpr int kOffRec = kOffF + kFStages * kFBytes;
    static constexpr int kOffGid = kOffRec + 2 * kRecBytes;  // [3][64] Gaussian ids
    static constexpr int kOffX = kOffGid + 3 * kFB * 4;      // per-pixel exchange, 8 words per pixel
    static constexpr int kOffBar = kOffX + 128 * 8 * 4;
    static constexpr int kSmem = 1024 + kOffBar + 64;
    // epilogue: one padded 32 x 36 FP32 tile per warp in the weight and
    // feature stages
    static_assert(8 * 32 * 36 * 4 <= kOffRec, "epilogue tiles must fit in the weight and feature stages");
};

// alpha and colour of one record at a pixel, by the FP32 paths' rules: EWA,
// q2 <= cutoff on the conic, alpha = min(alpha_max, op 2^(-q2 log2(e) / 2));
// a 2DGS surfel (Sec. 3.1, Eq. 1-3), u^2 + v^2 <= cutoff at the ray-plane
// intersection and alpha = min(alpha_max, op exp(-(u^2 + v^2) / 2)) with the
// exponential of the surfel FP32 render, so that its backward (which reads
// this forward's T and last contributor) takes the same decisions.
template <int GEOM>
struct FwdRec;
template <>
struct FwdRec<FHGS_GEOM_EWA> {
    using T = GRec;
    __device__ static float alpha(const GRec &r, float fpx, float fpy, const Params &p) {
        const float dx = fpx - r.a.x, dy = fpy - r.a.y;
        const float q2 = eval_q2(dx, dy, r.a.z, r.a.w, r.b.x);
        const float al = fminf(p.amax, r.b.y * gauss_q2(q2));
        return (q2 <= p.cut && al >= p.amin) ? al : 0.f;
    }
    __device__ static float3 rgb(const GRec &r) { return make_float3(r.b.z, r.b.w, r.c.x); }
};
template <>
struct FwdRec<FHGS_GEOM_SURFEL> {
    using T = SRec;
    __device__ static float alpha(const SRec &r, float fpx, float fpy, const Params &p) {
        SurfelHit h;
        if (!surfel_uv(r.a, r.b, r.c.x, fpx, fpy, p.cut, h)) return 0.f;
        const float al = fminf(p.amax, r.c.y * __expf(-0.5f * h.r2));
        return al >= p.amin ? al : 0.f;
    }
    __device__ static float3 rgb(const SRec &r) { return make_float3(r.c.z, r.c.w, r.d.x); }
};

template <int DN, int GEOM = FHGS_GEOM_EWA>
__global__ void __launch_bounds__(256, 2)
    k_render_fwd_tc(long long N, CamSet cs, Params p, ProjView pv, const uint32_t *__restrict__ gids,
                    const uint32_t *__restrict__ ranges, const __nv_bfloat16 *__restrict__ feats, int D,
                    float *rgb, float *feat, float *Tout, int32_t *last_out, unsigned *status) {
    using C = FwdCfg<DN, GEOM>;
    using FR = FwdRec<GEOM>;
    using Rec = typename FR::T;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align_smem_1024(smem_raw);
    if (probe_wait_expired(p, sm, status)) return;
    uint8_t *sW = sm;                                            // [2][128 rows][128 B]
    float *xT = reinterpret_cast<float *>(sm + C::kOffX);        // [128] T entering the next batch
    int *xDone = reinterpret_cast<int *>(xT + 128);               // [128]
    int *xLast = xDone + 128;                                     // [128]
    float *xP0 = reinterpret_cast<float *>(xLast + 128);         // [128] group 0's product of (1 - alpha)
    int *xL0 = reinterpret_cast<int *>(xP0 + 128);                // [128] group 0's last alpha > 0, or -1
    float *xRgb = reinterpret_cast<float *>(xL0 + 128);          // [128][3]
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + C::kOffBar);  // [2]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 2);
    auto srec = [&](int b) { return reinterpret_cast<Rec *>(sm + C::kOffRec + (b & 1) * C::kRecBytes); };
    auto sgid = [&](int b) { return reinterpret_cast<uint32_t *>(sm + C::kOffGid + (b % 3) * kFB * 4); };

    const int tid = threadIdx.x, warp = tid >> 5, grp = tid >> 7, pidx = tid & 127;
    const int tile = blockIdx.x >> 1, half = blockIdx.x & 1, chunk = blockIdx.y;
    const int ci = cam_of_tile(cs, tile);
    const DevCam &cam = cs.c[ci];
    const int lt = tile - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const int px = tx * kTile + (pidx & 15), py = ty * kTile + half * 8 + (pidx >> 4);
    const bool inside = px < cam.W && py < cam.H;
    const long long pix = cam.pix_off + (long long)py * cam.W + px;
    const uint32_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
    const int nbatches = (int)((e - s + kFB - 1) / kFB);
    const int d0 = chunk * DN;
    const Rec *rec = (GEOM == FHGS_GEOM_SURFEL ? reinterpret_cast<const Rec *>(pv.srec)
                                              : reinterpret_cast<const Rec *>(pv.rec)) +
                     (long long)ci * N;

    // TMEM is allocated right before the first MMA and released after the
    // epilogue's last read of it: with two CTAs on an SM, one CTA's batches
    // run while the other's epilogue drains to global memory
    if (tid == 0) {
        mbar_init(&bar[0], C::kNSub);  // one arrival per accumulator half's issuer
        mbar_init(&bar[1], C::kNSub);
        fence_mbar_init();
    }
    if (grp == 0) {
        xT[pidx] = 1.f;
        xDone[pidx] = inside ? 0 : 1;
        xLast[pidx] = 0;
    }
    const uint32_t sW_s = smem_u32(sW), sF_s = smem_u32(sm + C::kOffF);
    constexpr uint32_t idesc = idesc_bf16(128, C::kMmaN, false, true);

    // Every load helper commits exactly one cp.async group in every thread,
    // empty or not, so that the wait_group counts below hold.
    auto load_gid = [&](int b) {  // ids of batch b
        if (b < nbatches && tid < kFB) {
            const uint32_t at = s + (uint32_t)b * kFB + tid;
            cp_async4(smem_u32(sgid(b) + tid), gids + (at < e ? at : s), at < e);
        }
        cp_async_commit();
    };
    auto load_rec = [&](int b) {  // records of batch b (its ids are in shared memory)
        if (b < nbatches && tid < kFB) {
            const bool v = s + (uint32_t)b * kFB + tid < e;
            const uint32_t dst = smem_u32(srec(b) + tid);
            const Rec *src = rec + (v ? sgid(b)[tid] : 0u);
#pragma unroll
            for (int w4 = 0; w4 < (int)(sizeof(Rec) / 16); ++w4)
                cp_async16(dst + 16 * w4, reinterpret_cast<const float4 *>(src) + w4, v);
        }
        cp_async_commit();
    };
    auto load_feat = [&](int b) {  // feature rows of batch b, zero-filled past the end
        if (b < nbatches) {
            const int nb = (int)min((uint32_t)kFB, e - (s + (uint32_t)b * kFB));
            constexpr int kCPR = DN / 8;
            const uint32_t fb = sF_s + (C::kFStages == 2 ? (b & 1) : 0) * C::kFBytes;
            const uint32_t *ids = sgid(b);
#pragma unroll 4
            for (int q = tid; q < kFB * kCPR; q += 256) {
                const int g = q / kCPR, c = q - g * kCPR;
                const bool valid = g < nb;
                cp_async16(fb + (c >> 3) * (kFB * 128) + swz(g, c & 7),
                           feats + (size_t)(valid ? ids[g] : 0u) * D + d0 + c * 8, valid);
            }
        }
        cp_async_commit();
    };

    __syncthreads();
    uint32_t taddr = 0;
    bool have_tmem = false;

    const float fpx = px + 0.5f, fpy = py + 0.5f;
    float cr = 0.f, cg = 0.f, cb = 0.f;  // this group's share of the colour
    uint32_t ph[2] = {0u, 0u};
    int nbatch = 0;
    bool timeout = false;
    // prologue: ids of batches 0 and 1; records and features of batch 0
    load_gid(0);
    load_gid(1);
    cp_async_wait<1>();
    __syncthreads();
    load_rec(0);
    load_feat(0);
    for (int b = 0; b < nbatches; ++b) {
        const int stg = b & 1;
        const uint32_t base = s + (uint32_t)b * kFB;
        const int nb = (int)min((uint32_t)kFB, e - base);
        // the newest groups are [ids b+1, records b, features b]: all but the
        // last have landed after this wait
        cp_async_wait<1>();
        __syncthreads();
        load_gid(b + 2);
        load_rec(b + 1);
        const float T_in = xT[pidx];
        const bool done_in = xDone[pidx] != 0;
        const int last_in = xLast[pidx];
        // alphas of this group's 32 Gaussians and the running product of (1 - alpha)
        const Rec *R = srec(b);
        float a[32], l[32];
        float P = 1.f;
        int lastc = -1;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
            const int j = grp * 32 + jj;
            const float al = FR::alpha(R[j], fpx, fpy, p);
            a[jj] = j < nb ? al : 0.f;
            l[jj] = P;
            P *= 1.f - a[jj];
            lastc = a[jj] > 0.f ? jj : lastc;
        }
        if (grp == 0) {
            xP0[pidx] = P;
            xL0[pidx] = lastc;
        }
        // two stages: the feature stage of batch b+1 is free once the MMA of
        // batch b-1 is done; one stage: that of batch b (batch 0's came with
        // the prologue)
        bool ok = true;
        if (b >= 1) {
            const int ps = stg ^ 1;
            ok = mbar_wait(&bar[ps], ph[ps]);
            if (ok) ph[ps] ^= 1u;
        }
        if (__syncthreads_or(!ok)) {
            timeout = true;
            break;
        }
        if (C::kFStages == 2) load_feat(b + 1);
        else if (b >= 1) load_feat(b);
        else cp_async_commit();
        // weights: group 1 starts from T_in P_0 unless group 0 stops
        const float P0 = xP0[pidx];
        const bool stop0 = !done_in && T_in * P0 < p.teps;
        const float Ts = grp == 0 ? T_in : T_in * P0;
        bool done = grp == 0 ? done_in : (done_in || stop0);
        const bool owner = grp == 0 ? (done_in || stop0) : !(done_in || stop0);
        float Tstop = 0.f;
        int lastw = -1;
        uint8_t *wb = sW + stg * C::kWBytes;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float w8[8];
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                const int jj = 8 * q + h, j = grp * 32 + jj;
                const float Tj = Ts * l[jj];
                const float Tn = Ts * (jj < 31 ? l[jj + 1] : P);
                bool okj = a[jj] > 0.f && !done;
                const bool stop = okj && Tn < p.teps;
                if (stop) Tstop = Tj;
                done = done || stop;
                okj = okj && !stop;
                const float w = okj ? a[jj] * Tj : 0.f;
                w8[h] = w;
                if (okj) {
                    const float3 c3 = FR::rgb(R[j]);
                    cr += w * c3.x;
                    cg += w * c3.y;
                    cb += w * c3.z;
                    lastw = jj;
                }
            }
            uint4 pk;
            pk.x = pack_bf16(w8[0], w8[1]);
            pk.y = pack_bf16(w8[2], w8[3]);
            pk.z = pack_bf16(w8[4], w8[5]);
            pk.w = pack_bf16(w8[6], w8[7]);
            *reinterpret_cast<uint4 *>(wb + swz(pidx, grp * 4 + q)) = pk;
        }
        if (owner) {  // exactly one group carries the pixel's state to the next batch
            const int pos0 = (int)(base - s);
            if (grp == 0) {
                xT[pidx] = done_in ? T_in : Tstop;
                xDone[pidx] = 1;
                xLast[pidx] = lastw >= 0 ? pos0 + lastw + 1 : last_in;
            } else {
                const int L0 = xL0[pidx];
                xT[pidx] = done ? Tstop : Ts * P;
                xDone[pidx] = done ? 1 : 0;
                xLast[pidx] = lastw >= 0 ? pos0 + 32 + lastw + 1 : (L0 >= 0 ? pos0 + L0 + 1 : last_in);
            }
        }
        // two stages: the newest groups are [ids b+2, records b+1, features
        // b+1] and this batch's features have landed after wait<3>; one stage:
        // this batch's features are the newest group
        if (C::kFStages == 2) cp_async_wait<3>();
        else cp_async_wait<0>();
        fence_async_smem();
        if (!have_tmem && warp == 0) tmem_alloc(tslot, DN);  // may wait for the other CTA's release
        const int all_done = __syncthreads_and(grp == 0 || done);
        if (!have_tmem) {
            tc_after();
            taddr = *tslot;
            have_tmem = true;
        }
        // each 256-column half of the accumulator has its own issuing thread
        // (threads 0 and 32): the halves are independent accumulators
        if (tid == 0 || (C::kNSub > 1 && tid == 32)) {
            tc_after();
            const int nh = tid >> 5;
            const uint32_t wa = sW_s + stg * C::kWBytes, fb = sF_s + (C::kFStages == 2 ? stg : 0) * C::kFBytes;
            // descriptors as a base plus constants (address field = byte address / 16)
            const uint64_t a0 = sdesc(wa, 16, 1024), b0 = sdesc(fb, kFB * 128, 1024);
#pragma unroll
            for (int ks = 0; ks < kFB / 16; ++ks)
                mma_bf16(taddr + nh * 256, a0 + (uint64_t)((ks * 32) >> 4),
                         b0 + (uint64_t)((nh * 4 * (kFB * 128) + ks * 2048) >> 4), idesc,
                         (nbatch > 0 || ks > 0) ? 1u : 0u);
            mma_commit(&bar[stg]);
        }
        ++nbatch;
        if (all_done) break;
    }
    cp_async_wait_all();

    if (nbatch > 0 && !timeout) {  // the last commit covers every MMA issued before it
        const int ls = (nbatch - 1) & 1;
        const bool ok = mbar_wait(&bar[ls], ph[ls]);
        if (__syncthreads_or(!ok)) timeout = true;
    }
    if (timeout) {
        if (tid == 0) latch(status, ST_TIMEOUT);
        if (nbatch > 0) {
            const int ls = (nbatch - 1) & 1;
            mbar_wait(&bar[ls], ph[ls]);
        }
    } else {
        tc_after();
        // accumulator -> global memory by plain 16-byte stores, no block-wide
        // step: warp w holds pixels 32 (w % 4) .. + 31 (its TMEM lanes) and
        // half of the columns; each 32 x 32 block goes through the warp's own
        // padded tile in shared memory (the weight and feature stages are
        // free), then lane l writes 16 bytes of pixel 4 i + l / 8 per step:
        // 128 contiguous bytes per pixel and store.  The stores are posted, so
        // the CTA leaves while the SM's write path drains them.
        const int lane = tid & 31, q = warp & 3, sub = lane >> 3, c4 = (lane & 7) * 4;
        float *tileb = reinterpret_cast<float *>(sm) + warp * (32 * 36);
        long long opix[8];
        bool oin[8];
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int prow = q * 32 + it * 4 + sub;
            const int ox = tx * kTile + (prow & 15), oy = ty * kTile + half * 8 + (prow >> 4);
            oin[it] = ox < cam.W && oy < cam.H;
            opix[it] = cam.pix_off + (long long)oy * cam.W + ox;
        }
#pragma unroll 1
        for (int cc = 0; cc < DN / 64; ++cc) {
            const int col = grp * (DN / 2) + cc * 32;
            float v[32];
            if (have_tmem) {
                tmem_ld32(taddr + ((uint32_t)(q * 32) << 16) + col, v);
            } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.f;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
                *reinterpret_cast<float4 *>(tileb + lane * 36 + 4 * i) =
                    make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            __syncwarp();
#pragma unroll
            for (int it = 0; it < 8; ++it)
                if (oin[it])
                    *reinterpret_cast<float4 *>(feat + opix[it] * D + d0 + col + c4) =
                        *reinterpret_cast<const float4 *>(tileb + (it * 4 + sub) * 36 + c4);
            __syncwarp();
        }
        // the accumulator has been read: release TMEM for the SM's other CTA
        tc_before();
        __syncthreads();
        if (have_tmem && warp == 0) tmem_dealloc(taddr, DN);
        have_tmem = false;
        if (chunk == 0) {
            if (grp == 1) {
                xRgb[3 * pidx] = cr;
                xRgb[3 * pidx + 1] = cg;
                xRgb[3 * pidx + 2] = cb;
            }
            __syncthreads();
            if (grp == 0 && inside) {
                const float T = xT[pidx];
                rgb[3 * pix + 0] = cr + xRgb[3 * pidx] + T * p.bg0;
                rgb[3 * pix + 1] = cg + xRgb[3 * pidx + 1] + T * p.bg1;
                rgb[3 * pix + 2] = cb + xRgb[3 * pidx + 2] + T * p.bg2;
                Tout[pix] = T;
                last_out[pix] = xLast[pidx];
            }
        }
    }
    tc_before();
    __syncthreads();
    if (have_tmem && warp == 0) tmem_dealloc(taddr, DN);  // only when the epilogue was skipped
}

// ------------------------------------------------------------- backward
constexpr int kBB = 64;  // Gaussians per backward batch

// One step of a warp reduce-scatter: lanes with bit `off` set keep the upper
// H values, the others the lower H, each adding its partner's copy.
template <int H>
__device__ __forceinline__ void rs_step(float *v, int lane, int off) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const float send = up ? v[i] : v[i + H];
        const float keep = up ? v[i + H] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
}

// Shared-memory plan of the backward CTA (byte offsets; atoms 1024-aligned):
//   W   [128 px][64 g] BF16 weights            (B of dFe^T, MN-major)
//   Dh  [DN/64][128 px][64] BF16 dF hi           (A of G, K-major; A of dFe^T, MN-major)
//   Dl  same, dF lo = bf16(dF - hi)
//   Th  [128 px][64 g] BF16 t = G dL/drho, hi    (A of the moments, MN-major)
//   Tl  same, lo
//   X   [2 K-blocks][16 rows][64 px] BF16       (B of the moments, K-major): rows 1, i, j, i^2, i j, j^2
//   F   [DN/64][64 g][64] BF16 feature rows      (B of G, K-major)
// Th is followed by Tl (and Dh by Dl): the M=128 MMAs with only 64 real rows
// (the moments; dFe^T at DN = 64) read their second M block from the next
// buffer and those rows are unused.
template <int DN, int kG, int GEOM = FHGS_GEOM_EWA>
struct BwdCfg {
    static constexpr bool kSurf = GEOM == FHGS_GEOM_SURFEL;
    static constexpr int kG2 = kSurf ? kSurfelG2d : 12;  // footprint-gradient floats per (camera, primitive)
    static constexpr int kThreads = 128 * kG;  // kG groups of 4 warps over the half tile's 128 pixels
    static constexpr int kJ = kBB / kG;        // Gaussians per thread and batch
    static constexpr int kRecStages = kG == 2 ? 3 : 2;  // with 2, the drain reads its records from global
    static constexpr int kNBlk = DN / 64;
    static constexpr int kOffW = 0;
    static constexpr int kOffDh = kOffW + 128 * 128;
    static constexpr int kOffDl = kOffDh + kNBlk * 128 * 128;
    static constexpr int kOffTh = kOffDl + kNBlk * 128 * 128;
    static constexpr int kOffTl = kOffTh + 128 * 128;
    static constexpr int kOffX = kOffTl + 128 * 128;
    static constexpr int kOffF = kOffX + 2 * 16 * 128;
    static constexpr int kOffRec = kOffF + kNBlk * kBB * 128;
    static constexpr int kRecBytes = kBB * 48;
    static constexpr int kOffGid = kOffRec + kRecStages * kRecBytes;  // record stages: (b-1 for the drain,) b, b+1
    // surfels: the records' a, b, c stages like a GRec, the blue colour (d.x) beside them
    static constexpr int kOffBlue = kOffGid + 4 * kBB * 4;   // ids of b-1 .. b+2
    static constexpr int kOffRgb = kOffBlue + (GEOM == FHGS_GEOM_SURFEL ? kRecStages * kBB * 4 : 0);
    static constexpr int kOffFlag = kOffRgb + 2 * kBB * 3 * 4;  // [2 batches][64][3] colour sums
    static constexpr int kOffXch = kOffFlag + 16;  // [2 batches][64 bits] masks; then per pixel: P, S of groups 1.., T, S
    static constexpr int kOffBar = kOffXch + 128 * 4 * (2 * (kG - 1) + 2);
    static constexpr int kSmem = 1024 + kOffBar + 64;
    static_assert(kSmem <= 232448, "backward CTA exceeds the opt-in shared memory");
    static constexpr int kTmemCols = 512;
    static constexpr int kColGl = 64;   // G's lo part (G's hi part at column 0)
    static constexpr int kColF = 128;   // dFe^T, 64 columns per block of 128 channels
    static constexpr int kColM = 256;   // moments, 16 columns
    static constexpr int kColDl = 384;  // dF lo: DN / 2 columns
    static_assert(kColDl + DN / 2 <= kTmemCols, "dF lo exceeds tensor memory");
};

// kG groups of 4 warps share the half tile's 128 pixels; group g handles
// Gaussians [kJ g, kJ g + kJ) of each batch.  Back to front, the last
// group's Gaussians come first: it runs the App. A.2 recursion with the true
// suffix sum S, while group g < kG-1 runs it from S = 0 and then subtracts
// G_k (S + S_>g) / (1 - alpha_k), with S_>g the sum of w g over the later
// groups' Gaussians; transmittance needs the later groups' products of
// (1 - alpha).
template <int DN, int kG, int GEOM = FHGS_GEOM_EWA>
__global__ void __launch_bounds__(128 * kG, 1)
    k_render_bwd_tc(long long N, CamSet cs, Params p, ProjView pv, const uint32_t *__restrict__ gids,
                    const uint32_t *__restrict__ ranges, const __nv_bfloat16 *__restrict__ feats, int D,
                    const float *__restrict__ Tfin, const int32_t *__restrict__ lastv,
                    const float *__restrict__ grgb, const float *__restrict__ gfeat,
                    const __grid_constant__ CUtensorMap dfm, float *g2d, float *gfeatures, unsigned *status,
                    int n_items) {
    using C = BwdCfg<DN, kG, GEOM>;
    constexpr int kJ = C::kJ;
    if ((int)blockIdx.x >= n_items) return;  // uniform over the CTA
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align_smem_1024(smem_raw);
    if (probe_wait_expired(p, sm, status)) return;
    uint8_t *sW = sm + C::kOffW;
    uint8_t *sDh = sm + C::kOffDh;
    uint8_t *sDl = sm + C::kOffDl;
    uint8_t *sTh = sm + C::kOffTh;
    uint8_t *sTl = sm + C::kOffTl;
    uint8_t *sX = sm + C::kOffX;
    auto sRgb = [&](int b) { return reinterpret_cast<float *>(sm + C::kOffRgb) + (b & 1) * kBB * 3; };
    auto sMask = [&](int b) { return reinterpret_cast<uint32_t *>(sm + C::kOffFlag) + (b & 1) * 2; };
    float *xP = reinterpret_cast<float *>(sm + C::kOffXch);  // [kG-1][128] group g's prod (1 - alpha), g >= 1
    float *xSg = xP + (kG - 1) * 128;                          // [kG-1][128] group g's sum w g, g >= 1
    float *xT = xSg + (kG - 1) * 128;                          // [128] T after the batch
    float *xS = xT + 128;                                      // [128] S after the batch
    // [0] G, [1] dFe + moments, [2] dF staging of pixels 0..63, [3] of pixels 64..127
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + C::kOffBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 4);
    // [2] per item parity: max over the CTA of (item counter << 32 | last); the
    // counter only grows, so no slot is ever reset, and a slot's next writer
    // is two items later, past at least one barrier of every thread
    unsigned long long *smax = reinterpret_cast<unsigned long long *>(bars + 5);
    auto srec = [&](int b) { return reinterpret_cast<GRec *>(sm + C::kOffRec + (b % C::kRecStages) * C::kRecBytes); };
    auto sblue = [&](int b) { return reinterpret_cast<float *>(sm + C::kOffBlue) + (b % C::kRecStages) * kBB; };
    // surfels: dL/drho of the batch, [64 surfels][128 px] FP32 with the pixel
    // index XOR (surfel % 32) (conflict-free both ways), in the t buffers;
    // the footprint-gradient sums of the batch, [64][12], in the X buffer
    float *sDr = reinterpret_cast<float *>(sTh);
    float *sGeo = reinterpret_cast<float *>(sX);
    auto sgid = [&](int b) { return reinterpret_cast<uint32_t *>(sm + C::kOffGid + (b & 3) * kBB * 4); };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, grp = tid >> 7, pidx = tid & 127;
    const bool want_fg = gfeatures != nullptr;
    const int nch = D / DN;  // D slices: items are (tile, half, slice), tile and half fastest
    const int n_half = n_items / nch;

    if (warp == 0) tmem_alloc(tslot, C::kTmemCols);
    if (tid == 0) {
        mbar_init(&bars[0], 2);  // G's hi and lo parts, two issuers
        mbar_init(&bars[1], (DN >= 256 ? 2 : 1) + 1);  // one issuer per feature-gradient block, one for the moments
        mbar_init(&bars[2], 1);
        mbar_init(&bars[3], 1);
        fence_mbar_init();
        smax[0] = smax[1] = 0ull;
    }
    if (tid < 2 * kBB) sRgb(0)[3 * tid] = sRgb(0)[3 * tid + 1] = sRgb(0)[3 * tid + 2] = 0.f;  // both slots
    if (tid < 4) sMask(0)[tid] = 0u;
    if constexpr (C::kSurf) {
        for (int q = tid; q < kBB * 12; q += C::kThreads) sGeo[q] = 0.f;
    } else {
        // pixel-moment rows of X: X[n][p] for p = i + 16 j
        for (int q = tid; q < 16 * 128; q += C::kThreads) {
            const int n = q >> 7, pp = q & 127;
            const float i = (float)(pp & 15), jv = (float)(pp >> 4);
            const float val = n == 0 ? 1.f : n == 1 ? i : n == 2 ? jv : n == 3 ? i * i : n == 4 ? i * jv
                                                       : n == 5 ? jv * jv : 0.f;
            *reinterpret_cast<__nv_bfloat16 *>(sX + (pp >> 6) * (16 * 128) + swz(n, (pp & 63) >> 3) +
                               2 * (pp & 7)) = __float2bfloat16_rn(val);
        }
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t taddr = *tslot;
    const uint32_t tG = taddr, tGl = taddr + C::kColGl, tM = taddr + C::kColM, tF = taddr + C::kColF;
    const uint32_t tDl = taddr + C::kColDl;
    const uint32_t sW_s = smem_u32(sW), sDh_s = smem_u32(sDh), sDl_s = smem_u32(sDl);
    const uint32_t sTh_s = smem_u32(sTh), sTl_s = smem_u32(sTl), sX_s = smem_u32(sX);
    const uint32_t sF_s = smem_u32(sm + C::kOffF);
    constexpr uint32_t idG = idesc_bf16(128, kBB, false, false);
    constexpr uint32_t idF = idesc_bf16(128, kBB, true, true);
    constexpr uint32_t idM = idesc_bf16(128, 16, true, false);
    // G = dF Fe^T in two accumulators, each with its own issuing thread: the
    // hi part reads dF hi from shared memory (thread 0); the lo part reads dF
    // lo from TMEM (thread 128), copied there once per item, so that the lo
    // buffer in shared memory can take the next item's staged dF.
    auto issue_dF_copy = [&]() {  // dF lo -> TMEM (thread 128, before its first G)
        const uint64_t cl0 = sdesc(sDl_s, 16, 1024);
#pragma unroll
        for (int ks = 0; ks < DN / 16; ++ks)
            tmem_cp_128x256b(tDl + ks * 8, cl0 + (uint64_t)(((ks >> 2) * (128 * 128) + (ks & 3) * 32) >> 4));
    };
    // Descriptors are a base plus a constant: the address field is the low 14
    // bits (byte address / 16) and no sum here reaches 256 KB.
    const uint64_t dF0 = sdesc(sF_s, 16, 1024), dW0 = sdesc(sW_s, 128 * 128, 1024);
    const uint64_t dDh0 = sdesc(sDh_s, 128 * 128, 1024), dTh0 = sdesc(sTh_s, 128 * 128, 1024);
    const uint64_t dX0 = sdesc(sX_s, 16, 1024);
    const uint64_t dDhK0 = sdesc(sDh_s, 16, 1024);  // dF hi as a K-major A operand
    auto issue_G = [&](bool lo) {  // G(px, g) = sum_d dF(px, d) Fe(g, d): hi (thread 0) or lo (thread 128)
        tc_after();
#pragma unroll
        for (int ks = 0; ks < DN / 16; ++ks) {
            const uint64_t bd = dF0 + (uint64_t)(((ks >> 2) * (kBB * 128) + (ks & 3) * 32) >> 4);
            if (lo) mma_bf16_ta(tGl, tDl + ks * 8, bd, idG, ks > 0 ? 1u : 0u);
            else mma_bf16(tG, dDhK0 + (uint64_t)(((ks >> 2) * (128 * 128) + (ks & 3) * 32) >> 4), bd, idG,
                          ks > 0 ? 1u : 0u);
        }
        mma_commit(&bars[0]);
    };
    // dFe^T = dF^T W, one M = 128 block of channels per MMA (TMEM lanes =
    // channels, columns = the batch's Gaussians); for DN = 64 lanes 64..127
    // read past the channel block and are never drained.  Block mb is issued
    // by thread 32 (1 + mb) (separate accumulators, so no order between them).
    constexpr int kFBlk = DN >= 128 ? DN / 128 : 1;
    auto issue_F = [&](int mb) {
        tc_after();
        if (want_fg) {
#pragma unroll
            for (int ks = 0; ks < 128 / 16; ++ks)
                mma_bf16(tF + mb * kBB, dDh0 + (uint64_t)((mb * 2 * (128 * 128) + ks * 2048) >> 4),
                         dW0 + (uint64_t)((ks * 2048) >> 4), idF, ks > 0 ? 1u : 0u);
        }
        mma_commit(&bars[1]);  // arrives at once when nothing was issued
    };
    // moments = T^T X with T hi in rows 0..63 and T lo in rows 64..127 of one
    // M = 128 operand (Tl follows Th): lanes 0..63 get the hi part, 64..127
    // the lo part.  Issued by thread 32 (1 + kFBlk).
    auto issue_M = [&]() {
        tc_after();
        if constexpr (!C::kSurf) {  // surfels: no moments (the commit arrives at once)
#pragma unroll
            for (int ks = 0; ks < 128 / 16; ++ks)
                mma_bf16(tM, dTh0 + (uint64_t)((ks * 2048) >> 4),
                         dX0 + (uint64_t)(((ks >> 2) * (16 * 128) + (ks & 3) * 32) >> 4), idM, ks > 0 ? 1u : 0u);
        }
        mma_commit(&bars[1]);
    };

    // the drain of batch db of an item (moments and colour sums into the
    // footprint gradients, the feature-gradient block into grad_features);
    // the item's geometry is passed in, it may be the previous item's
    auto drain = [&](int db, int dnbat_end, int dx0, int dy0, float *dg2dc, const GRec *drec, int dchunk, int dd0) {
        const int dbe = dnbat_end - db * kBB, dnb = dbe - max(0, dbe - kBB);
        const int q = warp & 3;
        // moments: lanes 0..63 hold the T-hi part of Gaussian (lane), read by
        // warps 0 and 1; lanes 64..127 the T-lo part, read by warps 6 and 7.
        // Both add their (linear) share; the colour sums go with the hi part.
        // (Surfels: their footprint and colour sums left with the batch.)
        if (!C::kSurf && ((grp == 0 && q < 2) || (grp == 1 && q >= 2))) {
            const bool hi = grp == 0;
            const int j = (q & 1) * 32 + lane;
            const uint32_t wmask = sMask(db)[q & 1] & (dnb >= (q & 1) * 32 + 32 ? 0xFFFFFFFFu
                                   : (dnb > (q & 1) * 32 ? (1u << (dnb - (q & 1) * 32)) - 1u : 0u));
            const bool mine = (wmask >> lane) & 1u;
            const uint32_t gid = sgid(db)[j];
            float m[16];
            tmem_ld16(tM + ((uint32_t)(q * 32) << 16), m);
            if (mine) {
                // the batch's records: still staged with three stages, else from global (L2)
                const GRec r = C::kRecStages == 3 ? srec(db)[j] : drec[gid];
                // moments about the pixel grid: dx = i - a, dy = j - b
                const float a = r.a.x - (float)dx0 - 0.5f, bb = r.a.y - (float)dy0 - 0.5f;
                const float M0 = m[0], Mi = m[1], Mj = m[2], Mii = m[3], Mij = m[4], Mjj = m[5];
                const float Sx = Mi - a * M0, Sy = Mj - bb * M0;
                const float Sxx = Mii - 2.f * a * Mi + a * a * M0;
                const float Sxy = Mij - a * Mj - bb * Mi + a * bb * M0;
                const float Syy = Mjj - 2.f * bb * Mj + bb * bb * M0;
                const float op = r.b.y, cA = r.a.z, cB = r.a.w, cC = r.b.x;
                float4 *dst = reinterpret_cast<float4 *>(dg2dc + C::kG2 * (long long)gid);
                atomicAdd(dst, make_float4(op * (cA * Sx + cB * Sy), op * (cB * Sx + cC * Sy),
                                           -0.5f * op * Sxx, -op * Sxy));
                atomicAdd(dst + 1, make_float4(-0.5f * op * Syy, M0, hi && dchunk == 0 ? sRgb(db)[3 * j] : 0.f,
                                               hi && dchunk == 1 % nch ? sRgb(db)[3 * j + 1] : 0.f));
                if (hi && dchunk == 2 % nch) atomicAdd(dg2dc + C::kG2 * (long long)gid + 8, sRgb(db)[3 * j + 2]);
            }
        }
        if (want_fg && (DN >= 128 || q < 2)) {
            // lane l of warp w holds channel 128 mb + 32 (w % 4) + l of every
            // Gaussian of its columns.  DN = 256: channel block g % 2 and
            // Gaussians [128 / kG * (g / 2), + 128 / kG); DN <= 128: Gaussians
            // [kJ g, kJ g + kJ).  Each kJ x 32 block goes through the warp's
            // share of the t buffers (free: the MMAs that read them are done),
            // so that each lane then adds 4 consecutive channels of one
            // Gaussian: 4 Gaussians x 128 contiguous bytes per vector reduction.
            const int mb = DN >= 256 ? (grp & 1) : 0;
            const int jn = DN >= 256 ? 128 / kG : kJ;
            const int j0 = DN >= 256 ? (grp >> 1) * jn : grp * kJ;
            const uint64_t vmask = dnb >= 64 ? ~0ull : ((1ull << dnb) - 1ull);
            const uint64_t msk = ((((uint64_t)sMask(db)[1] << 32) | sMask(db)[0]) & vmask) >> j0;
            float *stage = reinterpret_cast<float *>(sTh) + warp * (kJ * 32);
            const int sub = lane >> 3, q4 = (lane & 7) * 4;
            float *dst = gfeatures + dd0 + mb * 128 + q * 32 + q4;
            const uint32_t *ids = sgid(db) + j0;
#pragma unroll 1
            for (int h = 0; h < jn / kJ; ++h) {
                const uint32_t mh = (uint32_t)(msk >> (kJ * h)) & (kJ == 32 ? 0xFFFFFFFFu : 0xFFFFu);
                if (mh == 0u) continue;  // warp-uniform
                float v[kJ];
                if constexpr (kJ == 32) tmem_ld32(tF + mb * kBB + j0 + kJ * h + ((uint32_t)(q * 32) << 16), v);
                else tmem_ld16(tF + mb * kBB + j0 + kJ * h + ((uint32_t)(q * 32) << 16), v);
#pragma unroll
                for (int jj = 0; jj < kJ; ++jj) stage[jj * 32 + lane] = v[jj];
                __syncwarp();
#pragma unroll
                for (int it = 0; it < kJ / 4; ++it) {
                    const int jj = it * 4 + sub;
                    if ((mh >> jj) & 1u)
                        atomicAdd(reinterpret_cast<float4 *>(dst + (size_t)ids[kJ * h + jj] * D),
                                  *reinterpret_cast<const float4 *>(stage + jj * 32 + q4));
                }
                __syncwarp();
            }
        }
    };
    // where item `it` lives: tile, half, slice, camera and its first pixel
    struct ItemGeo {
        int tile, chunk, ci, x0, y0;
    };
    auto item_geo = [&](int it) {
        ItemGeo g;
        const int hx = it % n_half;
        g.chunk = it / n_half;
        g.tile = hx >> 1;
        g.ci = cam_of_tile(cs, g.tile);
        const DevCam &cm = cs.c[g.ci];
        const int lt = g.tile - cm.tile_off;
        g.x0 = (lt % cm.tiles_x) * kTile;
        g.y0 = (lt / cm.tiles_x) * kTile + (hx & 1) * 8;
        return g;
    };

    // dF arrives by TMA, staged row-major [64 px][DN] FP32 in two halves:
    // pixels 0..63 (image rows 0..3 of the half tile) in the Dl region, free
    // once Dl's copy into TMEM is done, so issued during the previous item;
    // pixels 64..127 in the Dh region, free once the previous item's last FM
    // has read it.  The tensor is dF as [total pixels][D]: one box of 16
    // pixels x DN channels per image row.  Pixels right of or below a
    // camera's image are read from the next row or camera (or as zero past
    // the end) and never used.  Called by warp 0.
    auto stage_half = [&](int item, int hf) {
        if (lane == 0) {
            uint64_t *bar = &bars[2 + hf];
            if (gfeat == nullptr) {
                mbar_arrive_expect_tx(bar, 0u);
            } else {
                const ItemGeo g = item_geo(item);
                const DevCam &c = cs.c[g.ci];
                const uint32_t dst = smem_u32(hf == 0 ? sDl : sDh);
                mbar_arrive_expect_tx(bar, 64u * DN * 4);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const long long row = c.pix_off + (long long)(g.y0 + hf * 4 + r) * c.W + g.x0;
                    tma_load_2d(dst + r * (16 * DN * 4), &dfm, g.chunk * DN, (int)row, bar);
                }
            }
        }
        __syncwarp();
    };
    uint32_t phA = 0, phB = 0;
    bool pendA = false, pendB = false;  // staging copies in flight (for the timeout exit)
    if (warp == 0) {
        stage_half(blockIdx.x, 0);
        stage_half(blockIdx.x, 1);
    }
    pendA = pendB = true;
    uint32_t ph0 = 0, ph1 = 0;
    bool pend0 = false, pend1 = false;
    bool timeout = false;
    // the previous item's last batch waits for its FM and drain until the
    // next item's loads are in flight
    bool have_prev = false;
    int prev_b = 0, prev_end = 0, prev_x0 = 0, prev_y0 = 0, prev_chunk = 0, prev_d0 = 0;
    float *prev_g2dc = g2d;
    const GRec *prev_rec = pv.rec;
    constexpr int kL = DN >= 128 ? DN / 128 : 1;
    int k = 0;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x, ++k) {
        const ItemGeo ig = item_geo(it);
        const int chunk = ig.chunk, ci = ig.ci, x0 = ig.x0, y0 = ig.y0;
        const DevCam &cam = cs.c[ci];
        const int px = x0 + (pidx & 15), py = y0 + (pidx >> 4);
        const bool inside = px < cam.W && py < cam.H;
        const long long pix = cam.pix_off + (long long)py * cam.W + px;
        const uint32_t s = ranges[2 * ig.tile], e = ranges[2 * ig.tile + 1];
        const int d0 = chunk * DN;
        const GRec *rec = pv.rec + (long long)ci * N;
        const SRec *srecg = C::kSurf ? pv.srec + (long long)ci * N : nullptr;  // surfels
        float *g2dc = g2d + (long long)ci * N * C::kG2;
        // the next item's pixels 0..63 go to Dl once this item's dF is in TMEM
        bool stageA_next = it + (int)gridDim.x < n_items;
        auto stage_next_A = [&]() {
            if (stageA_next) {
                if (warp == 0) stage_half(it + gridDim.x, 0);
                pendA = true;
                stageA_next = false;
            }
        };
        float T = 1.f, dC0 = 0.f, dC1 = 0.f, dC2 = 0.f;
        int lastp = 0;
        if (inside) {
            T = Tfin[pix];
            lastp = lastv[pix];
            dC0 = grgb[3 * pix];
            dC1 = grgb[3 * pix + 1];
            dC2 = grgb[3 * pix + 2];
        }
        // tail of the previous item: its last FM (Dh is then free for this
        // item's pixels 64..127), then its drain
        if (have_prev) {
            const bool ok = mbar_wait(&bars[1], ph1);
            if (ok) {
                ph1 ^= 1u;
                pend1 = false;
            }
            if (__syncthreads_or(!ok)) {
                timeout = true;
                break;
            }
            if (warp == 0) stage_half(it, 1);
            pendB = true;
            tc_after();
            drain(prev_b, prev_end, prev_x0, prev_y0, prev_g2dc, prev_rec, prev_chunk, prev_d0);
            tc_before();
            __syncthreads();
            if (tid < kBB) sRgb(prev_b)[3 * tid] = sRgb(prev_b)[3 * tid + 1] = sRgb(prev_b)[3 * tid + 2] = 0.f;
            if (tid < 2) sMask(prev_b)[tid] = 0u;
            have_prev = false;
        } else if (k > 0) {  // the previous item issued no MMA that reads Dh
            if (warp == 0) stage_half(it, 1);
            pendB = true;
        }
        if (grp == 0) atomicMax(&smax[k & 1], ((unsigned long long)k << 32) | (uint32_t)max(lastp, 0));
        __syncthreads();
        const int Lmax = (int)min((unsigned long long)(e - s), smax[k & 1] & 0xFFFFFFFFull);
        const int nbat = (Lmax + kBB - 1) / kBB;
    // Every load helper commits one cp.async group in every thread, empty or
    // not.  Ids run two batches ahead of use, records one (from ids already
    // in shared memory), so no thread waits on a dependent global load.
    auto load_gid = [&](int b) {  // ids of batch b (ring slot b & 3)
        if (b < nbat && tid < kBB) {
            const int be = Lmax - b * kBB, bs = max(0, be - kBB), nb = be - bs;
            cp_async4(smem_u32(sgid(b) + tid), gids + s + bs + (tid < nb ? tid : 0), tid < nb);
        }
        cp_async_commit();
    };
    auto load_rec = [&](int b) {  // records of batch b (its stage; its ids have landed)
        if (b < nbat) {
            const int be = Lmax - b * kBB, bs = max(0, be - kBB), nb = be - bs;
            if (tid < nb) {
                const uint32_t dst = smem_u32(srec(b) + tid);
                if constexpr (C::kSurf) {
                    const SRec *src = srecg + sgid(b)[tid];
                    cp_async16(dst, &src->a, true);
                    cp_async16(dst + 16, &src->b, true);
                    cp_async16(dst + 32, &src->c, true);
                    cp_async4(smem_u32(sblue(b) + tid), &src->d.x, true);
                } else {
                    const GRec *src = rec + sgid(b)[tid];
                    cp_async16(dst, &src->a, true);
                    cp_async16(dst + 16, &src->b, true);
                    cp_async16(dst + 32, &src->c, true);
                }
            }
        }
        cp_async_commit();
    };
    auto prefetch_feat = [&](int b) {  // feature rows (reads the staged ids)
        const int be = Lmax - b * kBB, bs = max(0, be - kBB), nb = be - bs;
        const uint32_t *ids = sgid(b);
        constexpr int kCPR = DN / 8;
#pragma unroll 4
        for (int q = tid; q < kBB * kCPR; q += C::kThreads) {
            const int g = q / kCPR, c = q - g * kCPR;
            cp_async16(sF_s + (c >> 3) * (kBB * 128) + swz(g, c & 7), feats + (size_t)ids[g] * D + d0 + c * 8,
                       g < nb);
        }
        cp_async_commit();
    };
        if (nbat > 0) {  // the ids' latency runs under the staging wait
            load_gid(0);
            load_gid(1);
        }
        // this item's staged dF: both halves are waited for also when the
        // item has no batch, so that the staging buffers are quiet before reuse
        {
            const bool okA = mbar_wait(&bars[2], phA);
            const bool okB = okA && mbar_wait(&bars[3], phB);
            if (okA) {
                phA ^= 1u;
                pendA = false;
            }
            if (okB) {
                phB ^= 1u;
                pendB = false;
            }
            if (__syncthreads_or(!okB)) {
                timeout = true;
                break;
            }
        }
        if (nbat == 0) stage_next_A();  // nothing reads Dl for this item
        if (nbat > 0) {
            // the staged rows -> registers, 32 / kG rows per warp; every thread
            // has read its share before any hi / lo write overwrites the staging
            constexpr int kRows = 32 / kG;  // staged rows per warp
            float4 vdf[kRows][kL];
#pragma unroll
            for (int rr = 0; rr < kRows; ++rr) {
                const int prow = warp * kRows + rr;
                const int qx = x0 + (prow & 15), qy = y0 + (prow >> 4);
                const bool qin = qx < cam.W && qy < cam.H && gfeat != nullptr;
                const uint8_t *row = (prow < 64 ? sDl : sDh) + (prow & 63) * (DN * 4);
#pragma unroll
                for (int li = 0; li < kL; ++li) {
                    const int f = li * 128 + lane * 4;
                    vdf[rr][li] = (qin && f < DN) ? *reinterpret_cast<const float4 *>(row + 4 * f)
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            cp_async_wait_all();
            __syncthreads();  // ids of batches 0 and 1 are staged; the staging has been read
            load_rec(0);
            prefetch_feat(0);
            // dF -> BF16 hi / lo, K-major swizzled
            {
#pragma unroll
                for (int rr = 0; rr < kRows; ++rr) {
                    const int prow = warp * kRows + rr;
#pragma unroll
                    for (int li = 0; li < kL; ++li) {
                        const int f = li * 128 + lane * 4;
                        if (f >= DN) continue;
                        const float4 x = vdf[rr][li];
                        const __nv_bfloat162 h01 = __floats2bfloat162_rn(x.x, x.y);
                        const __nv_bfloat162 h23 = __floats2bfloat162_rn(x.z, x.w);
                        const float2 b01 = __bfloat1622float2(h01), b23 = __bfloat1622float2(h23);
                        const __nv_bfloat162 l01 = __floats2bfloat162_rn(x.x - b01.x, x.y - b01.y);
                        const __nv_bfloat162 l23 = __floats2bfloat162_rn(x.z - b23.x, x.w - b23.y);
                        const uint32_t off = (f >> 6) * (128 * 128) + swz(prow, (f & 63) >> 3) + ((f & 7) ? 8 : 0);
                        uint2 hv, lv;
                        hv.x = *reinterpret_cast<const uint32_t *>(&h01);
                        hv.y = *reinterpret_cast<const uint32_t *>(&h23);
                        lv.x = *reinterpret_cast<const uint32_t *>(&l01);
                        lv.y = *reinterpret_cast<const uint32_t *>(&l23);
                        *reinterpret_cast<uint2 *>(sDh + off) = hv;
                        *reinterpret_cast<uint2 *>(sDl + off) = lv;
                    }
                }
            }
            fence_async_smem();
            __syncthreads();  // hi / lo written: their copies into TMEM run while records and features land
            if (tid == 128) issue_dF_copy();
            cp_async_wait_all();
            fence_async_smem();
            __syncthreads();
            if (tid == 0) issue_G(false);
            if (tid == 128) issue_G(true);  // the same thread as the copies: the MMAs follow them
            pend0 = true;
            if (nbat > 1) {  // G of batch 0 done: the feature stage takes batch 1
                const bool ok = mbar_wait(&bars[0], ph0);
                if (ok) {
                    ph0 ^= 1u;
                    pend0 = false;
                }
                if (__syncthreads_or(!ok)) {
                    timeout = true;
                    break;
                }
                prefetch_feat(1);
                stage_next_A();  // the copies into TMEM (before G) have read Dl
            }
        }

        const float fpx = px + 0.5f, fpy = py + 0.5f;
        // the colour part of dL/dw (and the background term) belongs to slice 0
        // only; every slice sums its own colour channels for the colour gradients
        const float rC0 = chunk == 0 ? dC0 : 0.f, rC1 = chunk == 0 ? dC1 : 0.f, rC2 = chunk == 0 ? dC2 : 0.f;
        float S = T * (rC0 * p.bg0 + rC1 * p.bg1 + rC2 * p.bg2);
        for (int b = 0; b < nbat; ++b) {
            const int be = Lmax - b * kBB, bs = max(0, be - kBB), nb = be - bs;
            const bool more = b + 1 < nbat;
            load_gid(b + 2);
            load_rec(b + 1);
            if (pend0) {  // only when this item has a single batch: later G's are waited after a recursion
                const bool ok = mbar_wait(&bars[0], ph0);
                if (ok) {
                    ph0 ^= 1u;
                    pend0 = false;
                }
                if (__syncthreads_or(!ok)) {
                    timeout = true;
                    break;
                }
                stage_next_A();
            }
            tc_after();
            const GRec *R = srec(b);
            float Gv[kJ];
            {  // G = hi part + lo part
                const uint32_t lq = ((uint32_t)((warp & 3) * 32) << 16) + grp * kJ;
                float gl[kJ];
                if constexpr (kJ == 32) {
                    tmem_ld32(tG + lq, Gv);
                    tmem_ld32(tGl + lq, gl);
                } else {
                    tmem_ld16(tG + lq, Gv);
                    tmem_ld16(tGl + lq, gl);
                }
#pragma unroll
                for (int jj = 0; jj < kJ; ++jj) Gv[jj] += gl[jj];
            }
            float al[kJ], gx[kJ], Tj[kJ];
            float P = 1.f;
            const int jlim = min(nb, lastp - bs);  // Gaussians past the batch or the pixel's last
#pragma unroll
            for (int jj = 0; jj < kJ; ++jj) {
                const int j = grp * kJ + jj;
                const float4 A4 = R[j].a, B4 = R[j].b;
                if constexpr (C::kSurf) {  // the surfel render's hit and exponential
                    SurfelHit h;
                    const bool hit = surfel_uv(A4, B4, R[j].c.x, fpx, fpy, p.cut, h);
                    const float G = __expf(-0.5f * h.r2);
                    const float rho = R[j].c.y * G;
                    const float aa = fminf(p.amax, rho);
                    const bool ok = (j < jlim) && hit && (aa >= p.amin);
                    al[jj] = ok ? aa : 0.f;
                    gx[jj] = (ok && rho <= p.amax) ? G : 0.f;
                } else {
                    const float dx = fpx - A4.x, dy = fpy - A4.y;
                    const float q2 = eval_q2(dx, dy, A4.z, A4.w, B4.x);
                    const float G = gauss_q2(q2);
                    const float rho = B4.y * G;
                    const float aa = fminf(p.amax, rho);
                    const bool ok = (j < jlim) && (q2 <= p.cut) && (aa >= p.amin);
                    al[jj] = ok ? aa : 0.f;
                    gx[jj] = (ok && rho <= p.amax) ? G : 0.f;
                }
                P *= 1.f - al[jj];
            }
            if (grp >= 1) xP[(grp - 1) * 128 + pidx] = P;
            // batch b+1's records and features (requested before this batch's
            // alphas) have landed, and this batch's G has left TMEM: G of batch
            // b+1 runs under the rest of batch b
            cp_async_wait_all();
            fence_async_smem();
            tc_before();
            __syncthreads();
            if (more) {
                if (tid == 0) issue_G(false);
                if (tid == 128) issue_G(true);
                pend0 = true;
            }
            // T after this group's Gaussians (the later groups' products of
            // (1 - alpha) divided out), then T before each of them
            float Pl = 1.f;
#pragma unroll
            for (int m = 1; m < kG; ++m)
                if (m > grp) Pl *= xP[(m - 1) * 128 + pidx];
            const float Tend = grp == kG - 1 ? T : __fdividef(T, Pl);
            const float Tstart = __fdividef(Tend, P);
            {
                float t = Tstart;
#pragma unroll
                for (int jj = 0; jj < kJ; ++jj) {
                    Tj[jj] = t;
                    t *= 1.f - al[jj];
                }
            }
            // App. A.2 back to front: dL/dalpha_k = T_k g_k - S_k / (1 - alpha_k);
            // Gv becomes t_k = G dL/drho (earlier groups: still without S + S_>g)
            float Sg = grp == kG - 1 ? S : 0.f;
            // the colour part of g only in slice 0 (rC is zero elsewhere)
            auto recurse = [&](auto with_colour) {
#pragma unroll
                for (int jj = kJ - 1; jj >= 0; --jj) {
                    const int j = grp * kJ + jj;
                    // selects, not products with zero: records past the batch end are stale
                    const bool c = al[jj] > 0.f;
                    const float w = al[jj] * Tj[jj];
                    float gc = Gv[jj];
                    if constexpr (decltype(with_colour)::value) {
                        if constexpr (C::kSurf) {
                            const float4 C4 = R[j].c;
                            gc += rC0 * C4.z + rC1 * C4.w + rC2 * sblue(b)[j];
                        } else {
                            const float4 B4 = R[j].b;
                            gc += rC0 * B4.z + rC1 * B4.w + rC2 * R[j].c.x;
                        }
                    }
                    const float g = c ? gc : 0.f;
                    const float dal = Tj[jj] * g - __fdividef(Sg, 1.f - al[jj]);
                    Sg = c ? Sg + w * g : Sg;
                    Gv[jj] = c ? gx[jj] * dal : 0.f;
                }
            };
            if (chunk == 0) recurse(std::true_type{});
            else recurse(std::false_type{});
            if (grp >= 1) xSg[(grp - 1) * 128 + pidx] = grp == kG - 1 ? Sg - S : Sg;
            // G of batch b+1 (issued after this batch's alphas) is done by now:
            // the feature stage takes batch b+2, a whole iteration ahead
            bool gok = true;
            if (more) {
                gok = mbar_wait(&bars[0], ph0);
                if (gok) {
                    ph0 ^= 1u;
                    pend0 = false;
                }
            }
            if (__syncthreads_or(!gok)) {
                timeout = true;
                break;
            }
            if (b + 2 < nbat) prefetch_feat(b + 2);
            else cp_async_commit();
            if (grp < kG - 1) {
                float Sb = S;  // suffix sum entering this group's Gaussians
#pragma unroll
                for (int m = 1; m < kG; ++m)
                    if (m > grp) Sb += xSg[(m - 1) * 128 + pidx];
#pragma unroll
                for (int jj = 0; jj < kJ; ++jj) Gv[jj] -= __fdividef(gx[jj] * Sb, 1.f - al[jj]);
                if (grp == 0) {
                    S = Sb + Sg;
                    T = Tstart;
                    xT[pidx] = T;
                    xS[pidx] = S;
                }
            }
            // FM of batch b-1 has finished: drain it, then its operands are free
            if (b >= 1) {
                const bool ok = mbar_wait(&bars[1], ph1);
                if (ok) {
                    ph1 ^= 1u;
                    pend1 = false;
                }
                if (__syncthreads_or(!ok)) {
                    timeout = true;
                    break;
                }
                tc_after();
                drain(b - 1, Lmax, x0, y0, g2dc, rec, chunk, d0);
                tc_before();
                __syncthreads();
                if (tid < kBB) sRgb(b - 1)[3 * tid] = sRgb(b - 1)[3 * tid + 1] = sRgb(b - 1)[3 * tid + 2] = 0.f;
                if (tid < 2) sMask(b - 1)[tid] = 0u;
            }
            // weights (B of dFe^T) and t hi/lo (A of the moments) of this group's Gaussians
#pragma unroll
            for (int q = 0; q < kJ / 8; ++q) {
                uint4 pw, ph, pl;
                uint32_t *pwv = &pw.x, *phv = &ph.x, *plv = &pl.x;
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int j0 = 8 * q + 2 * h;
                    pwv[h] = pack_bf16(al[j0] * Tj[j0], al[j0 + 1] * Tj[j0 + 1]);
                    if constexpr (!C::kSurf) {
                        const __nv_bfloat162 th = __floats2bfloat162_rn(Gv[j0], Gv[j0 + 1]);
                        const float2 tb = __bfloat1622float2(th);
                        phv[h] = *reinterpret_cast<const uint32_t *>(&th);
                        plv[h] = pack_bf16(Gv[j0] - tb.x, Gv[j0 + 1] - tb.y);
                    }
                }
                const uint32_t off = swz(pidx, grp * (kJ / 8) + q);
                *reinterpret_cast<uint4 *>(sW + off) = pw;
                if constexpr (!C::kSurf) {
                    *reinterpret_cast<uint4 *>(sTh + off) = ph;
                    *reinterpret_cast<uint4 *>(sTl + off) = pl;
                }
            }
            if constexpr (C::kSurf) {  // dL/drho = t / G of the unclamped contributors
#pragma unroll
                for (int jj = 0; jj < kJ; ++jj) {
                    const int j = grp * kJ + jj;
                    sDr[j * 128 + (pidx ^ (j & 31))] = gx[jj] > 0.f ? Gv[jj] / gx[jj] : 0.f;
                }
            }
            // which Gaussians contribute anywhere in the CTA: one OR per warp
            uint32_t cmask = 0;
#pragma unroll
            for (int jj = 0; jj < kJ; ++jj) cmask |= (al[jj] > 0.f ? 1u : 0u) << jj;
            cmask = __reduce_or_sync(0xffffffffu, cmask);
            if (lane == 0 && cmask) atomicOr(&sMask(b)[(grp * kJ) >> 5], cmask << ((grp * kJ) & 31));
            // colour sums sum_p w dC_p per Gaussian; channel c is summed by slice
            // c % (number of slices).  A reduce-scatter over the warp's 32 pixels
            // leaves lane l with the warp's sum for Gaussian kJ grp + l (32
            // per group), or lanes 2l and 2l+1 with that of kJ grp + l (16).
            if (cmask) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (c % nch != chunk) continue;
                    const float dc = c == 0 ? dC0 : (c == 1 ? dC1 : dC2);
                    float v[kJ];
#pragma unroll
                    for (int jj = 0; jj < kJ; ++jj) v[jj] = al[jj] * Tj[jj] * dc;
                    if constexpr (kJ == 32) {
                        rs_step<16>(v, lane, 16);
                        rs_step<8>(v, lane, 8);
                        rs_step<4>(v, lane, 4);
                        rs_step<2>(v, lane, 2);
                        rs_step<1>(v, lane, 1);
                        if (cmask & (1u << lane)) atomicAdd(&sRgb(b)[3 * (grp * kJ + lane) + c], v[0]);
                    } else {
                        rs_step<kJ / 2>(v, lane, 16);
                        rs_step<kJ / 4>(v, lane, 8);
                        rs_step<kJ / 8>(v, lane, 4);
                        rs_step<kJ / 16>(v, lane, 2);
                        v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
                        const int jl = lane >> 1;
                        if (!(lane & 1) && (cmask & (1u << jl))) atomicAdd(&sRgb(b)[3 * (grp * kJ + jl) + c], v[0]);
                    }
                }
            }
            fence_async_smem();  // weights and t (generic writes) -> the MMA operands
            __syncthreads();
            if (grp != 0) {
                T = xT[pidx];
                S = xS[pidx];
            }
            if (tid == 32) issue_F(0);
            if (kFBlk > 1 && tid == 64) issue_F(1);
            if (tid == 32 * (1 + kFBlk)) issue_M();
            pend1 = true;
            if constexpr (C::kSurf) {
                // surfels: footprint gradients d(x_c, y_c, M00, M01, M10, M11, M20,
                // M21, M22, opacity) of the batch, summed over the half tile's
                // pixels while the feature-gradient MMAs run.  Thread t takes
                // surfel t % 64 and pixels [P (t / 64), + P) (P = 128 / threads
                // per surfel), recomputes the ray-plane hit at each pixel with a
                // nonzero dL/drho and applies the surfel render backward's chain.
                constexpr int kTPG = C::kThreads / kBB, kPPT = 128 / kTPG;
                const int j = tid & (kBB - 1), qq = tid / kBB;
                if (j < nb) {
                    const float4 A4 = R[j].a, B4 = R[j].b, C4 = R[j].c;
                    float ga[10];
#pragma unroll
                    for (int c = 0; c < 10; ++c) ga[c] = 0.f;
#pragma unroll 4
                    for (int i = 0; i < kPPT; ++i) {
                        const int pp = qq * kPPT + i;
                        const float drho = sDr[j * 128 + (pp ^ (j & 31))];
                        if (drho == 0.f) continue;
                        SurfelHit h;
                        surfel_uv(A4, B4, C4.x, (float)(x0 + (pp & 15)) + 0.5f, (float)(y0 + (pp >> 4)) + 0.5f,
                                  3.4e38f, h);
                        const float G = __expf(-0.5f * h.r2), rho = C4.y * G;
                        const float dr2 = -0.5f * rho * drho;
                        const float du = 2.f * h.u * dr2, dv = 2.f * h.v * dr2;
                        const float dnu = du * h.iw, dnv = dv * h.iw, dw = -(du * h.u + dv * h.v) * h.iw;
                        ga[0] -= dnu * A4.z + dnv * B4.x + dw * B4.z;
                        ga[1] -= dnu * A4.w + dnv * B4.y + dw * B4.w;
                        ga[2] += dnu * h.dx;
                        ga[3] += dnu * h.dy;
                        ga[4] += dnv * h.dx;
                        ga[5] += dnv * h.dy;
                        ga[6] += dw * h.dx;
                        ga[7] += dw * h.dy;
                        ga[8] += dw;
                        ga[9] += G * drho;
                    }
#pragma unroll
                    for (int c = 0; c < 10; ++c)
                        if (ga[c] != 0.f) atomicAdd(&sGeo[j * 12 + c], ga[c]);
                }
                __syncthreads();
                if (tid < nb) {  // one set of vector reductions per surfel of the batch, with its colour sums
                    float *gs = sGeo + tid * 12;
                    const float r0 = chunk == 0 ? sRgb(b)[3 * tid] : 0.f;
                    const float r1 = chunk == 1 % nch ? sRgb(b)[3 * tid + 1] : 0.f;
                    const float r2 = chunk == 2 % nch ? sRgb(b)[3 * tid + 2] : 0.f;
                    bool any = r0 != 0.f || r1 != 0.f || r2 != 0.f;
#pragma unroll
                    for (int c = 0; c < 10; ++c) any = any || gs[c] != 0.f;
                    if (any) {
                        float *dst = g2dc + C::kG2 * (long long)sgid(b)[tid];
                        atomicAdd(reinterpret_cast<float4 *>(dst), make_float4(gs[0], gs[1], gs[2], gs[3]));
                        atomicAdd(reinterpret_cast<float4 *>(dst + 4), make_float4(gs[4], gs[5], gs[6], gs[7]));
                        atomicAdd(reinterpret_cast<float4 *>(dst + 8), make_float4(gs[8], gs[9], r0, r1));
                        if (r2 != 0.f) atomicAdd(dst + 12, r2);
                    }
#pragma unroll
                    for (int c = 0; c < 12; ++c) gs[c] = 0.f;
                }
            }
        }
        if (timeout) break;
        if (nbat > 0) {
            have_prev = true;
            prev_b = nbat - 1;
            prev_end = Lmax;
            prev_x0 = x0;
            prev_y0 = y0;
            prev_g2dc = g2dc;
            prev_rec = rec;
            prev_chunk = chunk;
            prev_d0 = d0;
        }
    }
    if (have_prev && !timeout) {  // the last item's last FM
        const bool ok = mbar_wait(&bars[1], ph1);
        if (ok) {
            ph1 ^= 1u;
            pend1 = false;
        }
        if (__syncthreads_or(!ok)) {
            timeout = true;
        } else {
            tc_after();
            drain(prev_b, prev_end, prev_x0, prev_y0, prev_g2dc, prev_rec, prev_chunk, prev_d0);
        }
    }
    if (timeout) {
        if (tid == 0) latch(status, ST_TIMEOUT);
        if (pend0) mbar_wait(&bars[0], ph0);
        if (pend1) mbar_wait(&bars[1], ph1);
        if (pendA) mbar_wait(&bars[2], phA);
        if (pendB) mbar_wait(&bars[3], phB);
    }
    cp_async_wait_all();
    tc_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, C::kTmemCols);
}

// ------------------------------------------------------------- fusion
// Feature fusion of one view (Sec. 3.1): num[g][c] += sum_p w_g(p) F(p)[c]
// and den[g] += sum_p w_g(p), with w the Eq. 4 weights.  Per half tile and
// slice of DN map columns the map tile (128 px x DN, FP32) is split once into
// BF16 hi + lo; per batch of 64 Gaussians the weights, walked front to back as
// in the forward, are split into BF16 hi + lo as well, and
//   num_b (64 g x DN) = Wh^T Mh + Wh^T Ml + Wl^T Mh,   den_b = (Wh + Wl)^T 1
// accumulate in TMEM (M = 128 with the batch's Gaussians in rows 0..63), so
// every product carries about 16 mantissa bits.  Batch b's block is drained
// into num/den (vector atomics on contiguous rows) while batch b+1 is weighed.
template <int DN>
struct FuseCfg {
    static constexpr int kNBlk = DN / 64;
    static constexpr int kOffWh = 0;                            // [128 px][64 g] BF16, MN-major A
    static constexpr int kOffWl = kOffWh + 128 * 128;           // (Wh's unused second M block reads it)
    static constexpr int kOffMh = kOffWl + 128 * 128;           // [DN/64][128 px][64] BF16, MN-major B
    static constexpr int kOffMl = kOffMh + kNBlk * 128 * 128;
    static constexpr int kOffOne = kOffMl + kNBlk * 128 * 128;  // [2 K-blocks][16 rows][64 px]: row 0 = 1
    static constexpr int kRecBytes = kFB * 48;
    static constexpr int kOffRec = kOffOne + 2 * 16 * 128;
    static constexpr int kOffGid = kOffRec + 2 * kRecBytes;      // [4][64] ids: the drain of b-1 reads them late
    static constexpr int kOffMask = kOffGid + 4 * kFB * 4;      // [2 batches][2 groups] contributors
    static constexpr int kOffX = kOffMask + 16;                  // per pixel: T, done, P0
    static constexpr int kOffBar = kOffX + 128 * 3 * 4;
    static constexpr int kSmem = 1024 + kOffBar + 64;
    static constexpr int kColDen = DN;                           // den in 16 columns after num
    static constexpr int kTmemCols = DN + 16 <= 128 ? 128 : (DN + 16 <= 256 ? 256 : 512);
    static_assert(kSmem <= 232448, "fusion CTA exceeds the opt-in shared memory");
};

template <int DN>
__global__ void __launch_bounds__(256, 1)
    k_fuse_tc(long long N, CamSet cs, Params p, ProjView pv, const uint32_t *__restrict__ gids,
              const uint32_t *__restrict__ ranges, const FuseMaps maps, int D, float *num, float *den,
              unsigned *status) {
    using C = FuseCfg<DN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align_smem_1024(smem_raw);
    if (probe_wait_expired(p, sm, status)) return;
    uint8_t *sWh = sm + C::kOffWh;
    uint8_t *sWl = sm + C::kOffWl;
    uint8_t *sMh = sm + C::kOffMh;
    uint8_t *sMl = sm + C::kOffMl;
    uint8_t *sOne = sm + C::kOffOne;
    float *xT = reinterpret_cast<float *>(sm + C::kOffX);
    int *xDone = reinterpret_cast<int *>(xT + 128);
    float *xP0 = reinterpret_cast<float *>(xDone + 128);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + C::kOffBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    auto srec = [&](int b) { return reinterpret_cast<GRec *>(sm + C::kOffRec + (b & 1) * C::kRecBytes); };
    auto sgid = [&](int b) { return reinterpret_cast<uint32_t *>(sm + C::kOffGid + (b & 3) * kFB * 4); };
    auto sMask = [&](int b) { return reinterpret_cast<uint32_t *>(sm + C::kOffMask) + (b & 1) * 2; };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, grp = tid >> 7, pidx = tid & 127;
    const int tile = blockIdx.x >> 1, half = blockIdx.x & 1, chunk = blockIdx.y;
    const int ci = cam_of_tile(cs, tile);
    const DevCam &cam = cs.c[ci];
    const int lt = tile - cam.tile_off;
    const int x0 = (lt % cam.tiles_x) * kTile, y0 = (lt / cam.tiles_x) * kTile + half * 8;
    const int px = x0 + (pidx & 15), py = y0 + (pidx >> 4);
    const bool inside = px < cam.W && py < cam.H;
    const uint32_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
    const int nbatches = (int)((e - s + kFB - 1) / kFB);
    const int d0 = chunk * DN;
    const GRec *rec = pv.rec + (long long)ci * N;
    const float *__restrict__ fmap = maps.m[ci];
    if (nbatches == 0) return;  // uniform over the CTA: nothing to fuse

    if (warp == 0) tmem_alloc(tslot, C::kTmemCols);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        fence_mbar_init();
    }
    if (grp == 0) {
        xT[pidx] = 1.f;
        xDone[pidx] = inside ? 0 : 1;
    }
    if (tid < 4) sMask(0)[tid] = 0u;  // both batch slots
    // ones operand: B (K = pixels, N = 16), K-major, row 0 = 1
    for (int q = tid; q < 16 * 128; q += 256) {
        const int n = q >> 7, pp = q & 127;
        *reinterpret_cast<__nv_bfloat16 *>(sOne + (pp >> 6) * (16 * 128) + swz(n, (pp & 63) >> 3) + 2 * (pp & 7)) =
            __float2bfloat16_rn(n == 0 ? 1.f : 0.f);
    }
    // map tile of this CTA's pixels -> BF16 hi / lo, MN-major swizzled
    {
        constexpr int kL = DN >= 128 ? DN / 128 : 1;
#pragma unroll 1
        for (int r0 = 0; r0 < 16; r0 += 8) {
            float4 v[8][kL];
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) {
                const int prow = warp * 16 + r0 + rr;
                const int qx = x0 + (prow & 15), qy = y0 + (prow >> 4);
                const bool qin = qx < cam.W && qy < cam.H;
                const float *src = fmap + ((long long)qy * cam.W + qx) * D + d0;
#pragma unroll
                for (int li = 0; li < kL; ++li) {
                    const int f = li * 128 + lane * 4;
                    v[rr][li] = (qin && f < DN) ? *reinterpret_cast<const float4 *>(src + f)
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) {
                const int prow = warp * 16 + r0 + rr;
#pragma unroll
                for (int li = 0; li < kL; ++li) {
                    const int f = li * 128 + lane * 4;
                    if (f >= DN) continue;
                    const float4 x = v[rr][li];
                    const __nv_bfloat162 h01 = __floats2bfloat162_rn(x.x, x.y);
                    const __nv_bfloat162 h23 = __floats2bfloat162_rn(x.z, x.w);
                    const float2 b01 = __bfloat1622float2(h01), b23 = __bfloat1622float2(h23);
                    const __nv_bfloat162 l01 = __floats2bfloat162_rn(x.x - b01.x, x.y - b01.y);
                    const __nv_bfloat162 l23 = __floats2bfloat162_rn(x.z - b23.x, x.w - b23.y);
                    const uint32_t off = (f >> 6) * (128 * 128) + swz(prow, (f & 63) >> 3) + ((f & 7) ? 8 : 0);
                    uint2 hv, lv;
                    hv.x = *reinterpret_cast<const uint32_t *>(&h01);
                    hv.y = *reinterpret_cast<const uint32_t *>(&h23);
                    lv.x = *reinterpret_cast<const uint32_t *>(&l01);
                    lv.y = *reinterpret_cast<const uint32_t *>(&l23);
                    *reinterpret_cast<uint2 *>(sMh + off) = hv;
                    *reinterpret_cast<uint2 *>(sMl + off) = lv;
                }
            }
        }
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t taddr = *tslot;
    const uint32_t tNum = taddr, tDen = taddr + C::kColDen;
    const uint32_t sWh_s = smem_u32(sWh), sWl_s = smem_u32(sWl), sMh_s = smem_u32(sMh), sMl_s = smem_u32(sMl);
    const uint32_t sOne_s = smem_u32(sOne);
    constexpr uint32_t idN = idesc_bf16(128, DN, true, true);
    constexpr uint32_t idD = idesc_bf16(128, 16, true, false);

    auto load_gid = [&](int b) {
        if (b < nbatches && tid < kFB) {
            const uint32_t at = s + (uint32_t)b * kFB + tid;
            cp_async4(smem_u32(sgid(b) + tid), gids + (at < e ? at : s), at < e);
        }
        cp_async_commit();
    };
    auto load_rec = [&](int b) {
        if (b < nbatches && tid < kFB) {
            const bool v = s + (uint32_t)b * kFB + tid < e;
            const uint32_t dst = smem_u32(srec(b) + tid);
            const GRec *src = rec + (v ? sgid(b)[tid] : 0u);
            cp_async16(dst, &src->a, v);
            cp_async16(dst + 16, &src->b, v);
            cp_async16(dst + 32, &src->c, v);
        }
        cp_async_commit();
    };
    auto issue = [&]() {  // num_b and den_b of the batch whose weights are staged
        tc_after();
#pragma unroll
        for (int ks = 0; ks < 128 / 16; ++ks) {
            const uint64_t ah = sdesc(sWh_s + ks * 2048, 128 * 128, 1024);
            const uint64_t al = sdesc(sWl_s + ks * 2048, 128 * 128, 1024);
            const uint64_t bh = sdesc(sMh_s + ks * 2048, 128 * 128, 1024);
            const uint64_t bl = sdesc(sMl_s + ks * 2048, 128 * 128, 1024);
            const uint64_t bo = sdesc(sOne_s + (ks >> 2) * (16 * 128) + (ks & 3) * 32, 16, 1024);
            mma_bf16(tNum, ah, bh, idN, ks > 0 ? 1u : 0u);
            mma_bf16(tNum, ah, bl, idN, 1u);
            mma_bf16(tNum, al, bh, idN, 1u);
            mma_bf16(tDen, ah, bo, idD, ks > 0 ? 1u : 0u);
            mma_bf16(tDen, al, bo, idD, 1u);
        }
        mma_commit(&bar[0]);
    };
    // batch db's block: den (slice 0) and num rows of the contributing Gaussians
    auto drain = [&](int db) {
        const int dnb = (int)min((uint32_t)kFB, e - (s + (uint32_t)db * kFB));
        if ((warp & 3) < 2) {
            const int h = warp & 1;
            const uint32_t wmask = sMask(db)[h] & (dnb >= h * 32 + 32 ? 0xFFFFFFFFu
                                   : (dnb > h * 32 ? (1u << (dnb - h * 32)) - 1u : 0u));
            const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
            if (grp == 0 && chunk == 0) {
                float dv[16];
                tmem_ld16(tDen + lanes, dv);
                if ((wmask >> lane) & 1u) atomicAdd(den + sgid(db)[h * 32 + lane], dv[0]);
            }
            if (wmask) {
                float *stage = reinterpret_cast<float *>(sWh) + (h + 2 * grp) * (32 * 36);
                const int sub = lane >> 3, q4 = (lane & 7) * 4;
#pragma unroll 1
                for (int cc = 0; cc < DN / 64; ++cc) {
                    float v[32];
                    tmem_ld32(tNum + lanes + grp * (DN / 2) + cc * 32, v);
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        *reinterpret_cast<float4 *>(stage + lane * 36 + 4 * i) =
                            make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                    __syncwarp();
#pragma unroll
                    for (int it = 0; it < 8; ++it) {
                        const int jj = it * 4 + sub;
                        if ((wmask >> jj) & 1u) {
                            const uint32_t g = sgid(db)[h * 32 + jj];
                            atomicAdd(reinterpret_cast<float4 *>(num + (size_t)g * D + d0 + grp * (DN / 2) +
                                                                 cc * 32 + q4),
                                      *reinterpret_cast<const float4 *>(stage + jj * 36 + q4));
                        }
                    }
                    __syncwarp();
                }
            }
        }
    };

    const float fpx = px + 0.5f, fpy = py + 0.5f;
    uint32_t ph = 0u;
    bool pend = false, timeout = false;
    int nb_done = 0;  // batches whose MMAs were issued
    load_gid(0);
    load_gid(1);
    cp_async_wait<1>();
    __syncthreads();
    load_rec(0);
    for (int b = 0; b < nbatches; ++b) {
        const uint32_t base = s + (uint32_t)b * kFB;
        const int nb = (int)min((uint32_t)kFB, e - base);
        // the newest groups are [ids b+1, records b] (and, from b = 1, the two
        // issued one batch ago): all have landed after this wait
        cp_async_wait<0>();
        __syncthreads();
        load_gid(b + 2);
        load_rec(b + 1);
        const float T_in = xT[pidx];
        const bool done_in = xDone[pidx] != 0;
        const GRec *R = srec(b);
        float a[32], l[32];
        float P = 1.f;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
            const int j = grp * 32 + jj;
            const float4 A4 = R[j].a, B4 = R[j].b;
            const float dx = fpx - A4.x, dy = fpy - A4.y;
            const float q2 = eval_q2(dx, dy, A4.z, A4.w, B4.x);
            const float al = fminf(p.amax, B4.y * gauss_q2(q2));
            a[jj] = (j < nb && q2 <= p.cut && al >= p.amin) ? al : 0.f;
            l[jj] = P;
            P *= 1.f - a[jj];
        }
        if (grp == 0) xP0[pidx] = P;
        // the previous batch's MMAs are done: drain their block
        bool ok = true;
        if (pend) {
            ok = mbar_wait(&bar[0], ph);
            if (ok) {
                ph ^= 1u;
                pend = false;
            }
        }
        if (__syncthreads_or(!ok)) {
            timeout = true;
            break;
        }
        if (b >= 1) {
            tc_after();
            drain(b - 1);
            tc_before();
        }
        __syncthreads();  // the drain's staging (in the weight buffers) is free again
        if (tid < 2) sMask(b - 1)[tid] = 0u;
        // weights: group 1 starts from T_in P_0 unless group 0 stops
        const float P0 = xP0[pidx];
        const bool stop0 = !done_in && T_in * P0 < p.teps;
        const float Ts = grp == 0 ? T_in : T_in * P0;
        bool done = grp == 0 ? done_in : (done_in || stop0);
        const bool owner = grp == 0 ? (done_in || stop0) : !(done_in || stop0);
        float Tstop = 0.f;
        uint32_t cmask = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float w8[8];
#pragma unroll
            for (int hh = 0; hh < 8; ++hh) {
                const int jj = 8 * q + hh;
                const float Tj = Ts * l[jj];
                const float Tn = Ts * (jj < 31 ? l[jj + 1] : P);
                bool okj = a[jj] > 0.f && !done;
                const bool stop = okj && Tn < p.teps;
                if (stop) Tstop = Tj;
                done = done || stop;
                okj = okj && !stop;
                w8[hh] = okj ? a[jj] * Tj : 0.f;
                cmask |= (okj ? 1u : 0u) << jj;
            }
            uint4 ph4, pl4;
            uint32_t *phv = &ph4.x, *plv = &pl4.x;
#pragma unroll
            for (int hh = 0; hh < 4; ++hh) {
                const __nv_bfloat162 hi = __floats2bfloat162_rn(w8[2 * hh], w8[2 * hh + 1]);
                const float2 hb = __bfloat1622float2(hi);
                phv[hh] = *reinterpret_cast<const uint32_t *>(&hi);
                plv[hh] = pack_bf16(w8[2 * hh] - hb.x, w8[2 * hh + 1] - hb.y);
            }
            const uint32_t off = swz(pidx, grp * 4 + q);
            *reinterpret_cast<uint4 *>(sWh + off) = ph4;
            *reinterpret_cast<uint4 *>(sWl + off) = pl4;
        }
        cmask = __reduce_or_sync(0xffffffffu, cmask);
        if (lane == 0 && cmask) atomicOr(&sMask(b)[grp], cmask);
        if (owner) {
            if (grp == 0) {
                xT[pidx] = done_in ? T_in : Tstop;
                xDone[pidx] = 1;
            } else {
                xT[pidx] = done ? Tstop : Ts * P;
                xDone[pidx] = done ? 1 : 0;
            }
        }
        fence_async_smem();
        const int all_done = __syncthreads_and(grp == 0 || done);
        if (tid == 0) issue();
        pend = true;
        ++nb_done;
        if (all_done) break;
    }
    cp_async_wait_all();
    if (!timeout && pend) {
        const bool ok = mbar_wait(&bar[0], ph);
        if (ok) {
            ph ^= 1u;
            pend = false;
        }
        if (__syncthreads_or(!ok)) {
            timeout = true;
        } else {
            tc_after();
            drain(nb_done - 1);
        }
    }
    if (timeout) {
        if (tid == 0) latch(status, ST_TIMEOUT);
        if (pend) mbar_wait(&bar[0], ph);
    }
    tc_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, C::kTmemCols);
}

int pick_fwd_dn(int D, int d_split) {
    if (d_split == 64 || d_split == 128 || d_split == 256 || d_split == 512) return (D % d_split == 0) ? d_split : 0;
    for (int dn = 512; dn >= 64; dn >>= 1)
        if (D % dn == 0) return dn;
    return 0;
}

int pick_bwd_dn(int D, int d_split) {
    if (d_split == 64 || d_split == 128 || d_split == 256) return (D % d_split == 0) ? d_split : 0;
    if (d_split == 512) return (D % 256 == 0) ? 256 : 0;
    if (D % 256 == 0) return 256;
    if (D % 128 == 0) return 128;
    if (D % 64 == 0) return 64;
    return 0;
}

}  // namespace

// Streaming multiprocessors of the current device, looked up once per device.
int sm_count_current() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n <= 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

int tc_supported(int D, int d_split) {
    return D > 0 && pick_fwd_dn(D, d_split) != 0 && pick_bwd_dn(D, d_split) != 0;
}

void launch_render_fwd_tc(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                          const __nv_bfloat16 *feats, int D, int d_split, float *rgb, float *feat, float *T,
                          int32_t *last, unsigned *status, cudaStream_t st) {
    const int dn = pick_fwd_dn(D, d_split);
    dim3 grid(cs.total_tiles * 2, D / dn);
    note_launch(1);
#define FHGS_FWD(DNV)                                                                                     \
    case DNV: {                                                                                           \
        if (p.geom == FHGS_GEOM_SURFEL) {                                                                 \
            static std::atomic<unsigned long long> smem_done{0};                                        \
            allow_max_smem(smem_done, k_render_fwd_tc<DNV, FHGS_GEOM_SURFEL>);                          \
            k_render_fwd_tc<DNV, FHGS_GEOM_SURFEL><<<grid, 256, FwdCfg<DNV, FHGS_GEOM_SURFEL>::kSmem, st>>>( \
                N, cs, p, pv, bins.gids, bins.ranges, feats, D, rgb, feat, T, last, status);              \
        } else {                                                                                          \
            static std::atomic<unsigned long long> smem_done{0};                                        \
            allow_max_smem(smem_done, k_render_fwd_tc<DNV>);                                            \
            k_render_fwd_tc<DNV><<<grid, 256, FwdCfg<DNV>::kSmem, st>>>(N, cs, p, pv, bins.gids, bins.ranges, \
                                                                       feats, D, rgb, feat, T, last, status); \
        }                                                                                                 \
        break;                                                                                            \
    }
    switch (dn) {
        FHGS_FWD(64)
        FHGS_FWD(128)
        FHGS_FWD(256)
        FHGS_FWD(512)
        default: break;
    }
#undef FHGS_FWD
}

// Gaussian groups of the backward CTA (4 warps each): FHGS_BWD_GROUPS = 2 or
// 4, default 4.
static int bwd_groups() {
    static const int g = [] {
        const char *e = getenv("FHGS_BWD_GROUPS");
        return (e && atoi(e) == 2) ? 2 : 4;
    }();
    return g;
}

// Tensor map of dL/dfeat as a [rows][D] FP32 matrix with boxes of 16 rows x
// dn columns (no swizzle; out-of-range elements read as zero).
static bool make_dF_tmap(CUtensorMap *m, const float *base, long long rows, int D, int dn) {
    return dn <= 256 && encode_f32_rows_tmap(m, base, rows, D, dn, 16);
}

bool launch_render_bwd_tc(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                          const __nv_bfloat16 *feats, int D, int d_split, const float *T, const int32_t *last,
                          const float *grgb, const float *gfeat, float *g2d, float *gfeatures, unsigned *status,
                          cudaStream_t st) {
    const int dn = pick_bwd_dn(D, d_split);
    CUtensorMap dfm;
    memset(&dfm, 0, sizeof(dfm));
    if (gfeat != nullptr && !make_dF_tmap(&dfm, gfeat, cs.total_pix, D, dn)) return false;
    // persistent: one CTA per SM walks the (tile, half, slice) items
    const int n_items = cs.total_tiles * 2 * (D / dn);
    const dim3 grid((unsigned)max(1, min(n_items, sm_count_current())));
    note_launch(1);
#define FHGS_BWD_G(DNV, GV, GEO)                                                                               \
    {                                                                                                          \
        static std::atomic<unsigned long long> smem_done{0};                                                 \
        allow_max_smem(smem_done, k_render_bwd_tc<DNV, GV, GEO>);                                            \
        k_render_bwd_tc<DNV, GV, GEO><<<grid, BwdCfg<DNV, GV, GEO>::kThreads, BwdCfg<DNV, GV, GEO>::kSmem, st>>>( \
            N, cs, p, pv, bins.gids, bins.ranges, feats, D, T, last, grgb, gfeat, dfm, g2d, gfeatures, status,  \
            n_items);                                                                                          \
    }
#define FHGS_BWD(DNV, GV)                                                                                      \
    case DNV * 8 + GV:                                                                                         \
        if (p.geom == FHGS_GEOM_SURFEL) FHGS_BWD_G(DNV, 4, FHGS_GEOM_SURFEL) /* kG = 2 has no room */         \
        else FHGS_BWD_G(DNV, GV, FHGS_GEOM_EWA)                                                                \
        break;
    switch (dn * 8 + bwd_groups()) {
        FHGS_BWD(64, 2)
        FHGS_BWD(128, 2)
        FHGS_BWD(256, 2)
        FHGS_BWD(64, 4)
        FHGS_BWD(128, 4)
        FHGS_BWD(256, 4)
        default: break;
    }
#undef FHGS_BWD
#undef FHGS_BWD_G
    return true;
}

int fuse_tc_dn(int D) {
    if (D % 256 == 0) return 256;
    if (D % 128 == 0) return 128;
    if (D % 64 == 0) return 64;
    return 0;
}

void launch_fuse_tc(long long N, const CamSet &cs, const Params &p, ProjView pv, const fhgs_bins &bins,
                    const FuseMaps &maps, int D, float *num, float *den, unsigned *status, cudaStream_t st) {
    const int dn = fuse_tc_dn(D);
    dim3 grid(cs.total_tiles * 2, D / dn);
    note_launch(1);
#define FHGS_FUSE(DNV)                                                                                         \
    case DNV: {                                                                                                \
        static std::atomic<unsigned long long> smem_done{0};                                                 \
        allow_max_smem(smem_done, k_fuse_tc<DNV>);                                                           \
        k_fuse_tc<DNV><<<grid, 256, FuseCfg<DNV>::kSmem, st>>>(N, cs, p, pv, bins.gids, bins.ranges, maps, D,  \
                                                               num, den, status);                            \
        break;                                                                                                 \
    }
    switch (dn) {
        FHGS_FUSE(64)
        FHGS_FUSE(128)
        FHGS_FUSE(256)
        default: break;
    }
#undef FHGS_FUSE
}

}  // namespace fhgs
