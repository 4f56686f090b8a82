// Tile binning (App. A: DuplicateWithKeys, SortByKeys, IdentifyTileRanges).
//
// The paper sorts one 64-bit key per tile instance, (tile id << 32 | depth
// bits), with ties left to the sort.  Every instance of a Gaussian shares its
// depth, and a view has only a few thousand tiles, so the same order is built
// here without sorting instances at all:
//   1. stable LSD radix sort of the C*N (camera, Gaussian) entries by the
//      32-bit depth bits (culled entries carry 0xFFFFFFFF and sort last), then
//      one stable pass by camera: entries are grouped by camera, in depth
//      order, ties by Gaussian index;
//   2. each camera's depth-ordered entries are cut into segments of SEG; per
//      segment the number of its Gaussians covering each tile comes from a 2-D
//      difference array over the tile grid in shared memory (4 corner updates
//      per rectangle, then row and column prefix sums);
//   3. one exclusive scan over the (tile, segment) count table gives, for each
//      tile, where each segment's run starts; the tile ranges are the
//      segment-0 offsets;
//   4. one warp per segment walks its Gaussians in depth order and writes each
//      one's Gaussian index into every tile of its rectangle at the tile's
//      running offset (kept in shared memory).
// The result equals the ascending sort of (tile << 32 | depth bits, index).
// Instances are written once, 4 bytes each; no kernel waits on another
// block, grids are fixed and counts live on the device, so the sequence can
// be captured in a CUDA graph.
#include "fhgs_internal.cuh"

namespace fhgs {
namespace {

constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixRounds = 8;
constexpr int kRadixTile = kRadixThreads * kRadixRounds;  // 2048
constexpr int kBuckets = 256;
constexpr int kRadixBlocksPerSM = 2;  // grid cap of the radix passes (the digit table is 256 x grid)

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048

// ---------------------------------------------------------------- radix
// A pass may be skipped when every key that matters shares its digit: kb
// (nullable) holds the AND and the OR of those keys' bits, and a skipped
// pass copies the keys in order (the sort stays stable).
__device__ __forceinline__ bool radix_skip(const uint32_t *kb, int shift, uint32_t mask) {
    return kb != nullptr && (((kb[0] ^ kb[1]) >> shift) & mask) == 0u;
}

// Per-block digit histogram of the block's contiguous segment.
__global__ void __launch_bounds__(kRadixThreads) k_radix_upsweep(const uint32_t *__restrict__ keys, long long n,
                                                                 int shift, uint32_t mask, uint32_t *hist,
                                                                 const uint32_t *__restrict__ kb) {
    if (radix_skip(kb, shift, mask)) return;
    __shared__ uint32_t h[kRadixWarps][kBuckets];
    for (int i = threadIdx.x; i < kRadixWarps * kBuckets; i += kRadixThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    const long long G = gridDim.x;
    const long long seg = (n + G - 1) / G;
    const long long s = blockIdx.x * seg, e = min(n, s + seg);
    const int w = threadIdx.x >> 5;
    for (long long i0 = s; i0 < e; i0 += kRadixTile) {
        uint32_t kk[kRadixRounds];  // the tile's keys requested together
#pragma unroll
        for (int r = 0; r < kRadixRounds; ++r) {
            const long long i = i0 + r * kRadixThreads + threadIdx.x;
            kk[r] = i < e ? keys[i] : 0u;
        }
#pragma unroll
        for (int r = 0; r < kRadixRounds; ++r) {
            const long long i = i0 + r * kRadixThreads + threadIdx.x;
            if (i < e) atomicAdd(&h[w][(kk[r] >> shift) & mask], 1u);
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kBuckets; d += kRadixThreads) {
        uint32_t t = 0;
#pragma unroll
        for (int k = 0; k < kRadixWarps; ++k) t += h[k][d];
        hist[(long long)d * G + blockIdx.x] = t;
    }
}

// In-place exclusive scan of a u32 array with one 1024-thread block.  Each
// step moves 16384 values: coalesced loads into shared memory, 16
// consecutive values per thread scanned there, coalesced stores back.  The
// step count, not the bandwidth, sets the time.  Optionally writes the total.
constexpr int kScanSmallItems = 16;
constexpr int kScanSmallStep = 1024 * kScanSmallItems;
constexpr int kScanSmallSmem = kScanSmallStep * 4 + kScanSmallStep / 32 * 4;  // values, then one pad word per 32
__device__ __forceinline__ int scan_small_slot(int i) { return i + (i >> 5); }  // pad: conflict-free per-thread rows
__global__ void __launch_bounds__(1024) k_scan_small(uint32_t *a, int total, int64_t *total_out,
                                                    const uint32_t *__restrict__ kb = nullptr, int shift = 0,
                                                    uint32_t mask = 0u) {
    if (radix_skip(kb, shift, mask)) return;
    extern __shared__ uint32_t sv[];
    __shared__ uint32_t carry;
    __shared__ uint32_t wsum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < total; base += kScanSmallStep) {
#pragma unroll
        for (int k = 0; k < kScanSmallItems; ++k) {
            const int i = k * 1024 + threadIdx.x;
            sv[scan_small_slot(i)] = base + i < total ? a[base + i] : 0u;
        }
        __syncthreads();
        const int r0 = threadIdx.x * kScanSmallItems;
        uint32_t v[kScanSmallItems], tsum = 0;
#pragma unroll
        for (int k = 0; k < kScanSmallItems; ++k) {
            v[k] = sv[scan_small_slot(r0 + k)];
            tsum += v[k];
        }
        uint32_t x = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t wv = wsum[threadIdx.x];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, wv, o);
                if (threadIdx.x >= o) wv += y;
            }
            wsum[threadIdx.x] = wv;
        }
        __syncthreads();
        uint32_t run = carry + (threadIdx.x >= 32 ? wsum[(threadIdx.x >> 5) - 1] : 0u) + x - tsum;
#pragma unroll
        for (int k = 0; k < kScanSmallItems; ++k) {
            sv[scan_small_slot(r0 + k)] = run;
            run += v[k];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kScanSmallItems; ++k) {
            const int i = k * 1024 + threadIdx.x;
            if (base + i < total) a[base + i] = sv[scan_small_slot(i)];
        }
        if (threadIdx.x == 1023) carry = run;
        __syncthreads();
    }
    if (total_out && threadIdx.x == 0) *total_out = (int64_t)carry;
}

// Stable scatter.  The block walks its segment in tiles of kRadixTile items;
// inside a tile, warp w owns items [w*256, w*256+256) visited in 8 rounds of
// 32 consecutive items, so (warp, round, lane) is memory order and ranks
// computed in that order keep the sort stable.  The tile is first reordered
// by digit in shared memory, then written out in that order: consecutive
// threads store consecutive slots of one digit's run, so each store
// instruction touches a few sectors instead of one per lane.
__global__ void __launch_bounds__(kRadixThreads) k_radix_downsweep(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, long long n, int shift, uint32_t mask, const uint32_t *__restrict__ hist,
    const uint32_t *__restrict__ kb) {
    __shared__ uint32_t run[kBuckets];                // next output slot per digit
    __shared__ uint32_t tot[kBuckets];                // this tile's count per digit
    __shared__ uint32_t tstart[kBuckets];             // first tile-local slot per digit
    __shared__ uint32_t wcnt[kRadixWarps][kBuckets];  // per-warp counts, then prefixes
    __shared__ uint32_t wsum[kRadixWarps];
    __shared__ uint32_t sk[kRadixTile], sv[kRadixTile];  // the tile in digit order
    const long long G = gridDim.x;
    const long long seg = (n + G - 1) / G;
    const long long s = blockIdx.x * seg, e = min(n, s + seg);
    if (radix_skip(kb, shift, mask)) {  // every key that matters has this digit: keep the order
        for (long long i = s + threadIdx.x; i < e; i += kRadixThreads) {
            kout[i] = kin[i];
            vout[i] = vin[i];
        }
        return;
    }
    for (int d = threadIdx.x; d < kBuckets; d += kRadixThreads) run[d] = hist[(long long)d * G + blockIdx.x];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (long long t0 = s; t0 < e; t0 += kRadixTile) {
        for (int d = lane; d < kBuckets; d += 32) wcnt[w][d] = 0;
        uint32_t key[kRadixRounds], val[kRadixRounds], rank[kRadixRounds];
        int dig[kRadixRounds];
#pragma unroll
        for (int r = 0; r < kRadixRounds; ++r) {  // loads first: all in flight together
            const long long i = t0 + w * (32 * kRadixRounds) + r * 32 + lane;
            key[r] = i < e ? kin[i] : 0u;
            val[r] = i < e ? vin[i] : 0u;
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < kRadixRounds; ++r) {
            const long long i = t0 + w * (32 * kRadixRounds) + r * 32 + lane;
            const bool valid = i < e;
            // invalid lanes get a private out-of-range digit: they match no one
            dig[r] = valid ? (int)((key[r] >> shift) & mask) : (kBuckets + lane);
            const unsigned peers = __match_any_sync(0xffffffffu, dig[r]);
            const uint32_t before = valid ? wcnt[w][dig[r]] : 0u;
            __syncwarp();
            if (valid && (peers & lt) == 0) wcnt[w][dig[r]] = before + __popc(peers);
            __syncwarp();
            rank[r] = before + __popc(peers & lt);
        }
        __syncthreads();
        static_assert(kBuckets == kRadixThreads, "one thread per digit");
        {
            const int d = threadIdx.x;
            uint32_t acc = 0;
#pragma unroll
            for (int k = 0; k < kRadixWarps; ++k) {
                const uint32_t c = wcnt[k][d];
                wcnt[k][d] = acc;
                acc += c;
            }
            tot[d] = acc;
            // exclusive scan of the digit totals over the block
            uint32_t x = acc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) wsum[w] = x;
            __syncthreads();
            uint32_t before = 0;
#pragma unroll
            for (int k = 0; k < kRadixWarps; ++k) before += k < w ? wsum[k] : 0u;
            tstart[d] = before + x - acc;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kRadixRounds; ++r) {
            if (dig[r] < kBuckets) {
                const uint32_t q = tstart[dig[r]] + wcnt[w][dig[r]] + rank[r];
                sk[q] = key[r];
                sv[q] = val[r];
            }
        }
        __syncthreads();
        const int tn = (int)min((long long)kRadixTile, e - t0);
#pragma unroll
        for (int r = 0; r < kRadixRounds; ++r) {
            const int q = r * kRadixThreads + threadIdx.x;
            if (q < tn) {
                const uint32_t k2 = sk[q];
                const int d = (int)((k2 >> shift) & mask);
                const uint32_t pos = run[d] + (uint32_t)q - tstart[d];
                kout[pos] = k2;
                vout[pos] = sv[q];
            }
        }
        __syncthreads();
        run[threadIdx.x] += tot[threadIdx.x];
        __syncthreads();
    }
}

// Keys and indices of the depth sort, and the AND / OR of the keys of the
// entries that are not culled (culled entries, key 0xFFFFFFFF, have empty
// rectangles, so their place in the order does not matter).
// Grid-stride: each thread folds its entries' keys, so the block issues one
// pair of global atomics however many entries it covers.
__global__ void k_iota_keys(const uint32_t *__restrict__ dkey, long long n, uint32_t *k, uint32_t *v,
                            uint32_t *kb) {
    uint32_t ta = 0xFFFFFFFFu, to = 0u;  // AND / OR of this thread's live keys
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const uint32_t key = dkey[i];
        k[i] = key;
        v[i] = (uint32_t)i;
        if (key != 0xFFFFFFFFu) {
            ta &= key;
            to |= key;
        }
    }
    __shared__ uint32_t ra[8], ro[8];  // one AND / OR per warp, then one pair of atomics per block
    const uint32_t a = __reduce_and_sync(0xffffffffu, ta);
    const uint32_t o = __reduce_or_sync(0xffffffffu, to);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        ra[w] = a;
        ro[w] = o;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t ba = 0xFFFFFFFFu, bo = 0u;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            ba &= ra[k];
            bo |= ro[k];
        }
        if (ba != 0xFFFFFFFFu || bo != 0u) {  // the block holds a live key
            atomicAnd(&kb[0], ba);
            atomicOr(&kb[1], bo);
        }
    }
}

__global__ void k_cam_keys(const uint32_t *__restrict__ order, long long n, long long N, uint32_t *k) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) k[i] = (uint32_t)(order[i] / N);
}

int radix_blocks(long long n, int sm_count) {
    long long g = (n + 4095) / 4096;
    if (g > (long long)kRadixBlocksPerSM * sm_count) g = (long long)kRadixBlocksPerSM * sm_count;
    return (int)(g < 1 ? 1 : g);
}

// Sorts (kA, vA) by the low `bits` bits of kA; returns true if the result is
// in (kB, vB) (odd number of passes), false if back in (kA, vA).
bool radix_sort_pairs(uint32_t *kA, uint32_t *vA, uint32_t *kB, uint32_t *vB, long long n, int bits,
                      uint32_t *hist, int G, cudaStream_t st, const uint32_t *kb = nullptr) {
    int shift = 0;
    bool a_to_b = true;
    while (shift < bits) {
        const int nb = min(8, bits - shift);
        const uint32_t mask = (1u << nb) - 1u;
        const uint32_t *ki = a_to_b ? kA : kB;
        const uint32_t *vi = a_to_b ? vA : vB;
        uint32_t *ko = a_to_b ? kB : kA;
        uint32_t *vo = a_to_b ? vB : vA;
        note_launch(3);
        k_radix_upsweep<<<G, kRadixThreads, 0, st>>>(ki, n, shift, mask, hist, kb);
        static std::atomic<unsigned long long> scan_done{0};
        allow_max_smem(scan_done, k_scan_small);
        k_scan_small<<<1, 1024, kScanSmallSmem, st>>>(hist, kBuckets * G, nullptr, kb, shift, mask);
        k_radix_downsweep<<<G, kRadixThreads, 0, st>>>(ki, vi, ko, vo, n, shift, mask, hist, kb);
        shift += nb;
        a_to_b = !a_to_b;
    }
    return !a_to_b;
}

// ------------------------------------------------------- tile counting
// One block per (segment, camera): per-tile counts of the segment's Gaussians
// via a 2-D difference array of the camera's tile grid.  Writes
// table[(tile_off + tile) * S + seg].
// Tile rectangles in sorted order (empty rectangle for culled entries), so
// that the per-segment passes below read them sequentially.
//
// List cut.  Compositing stops at a pixel once its transmittance would fall
// below t_eps, so the entries of a tile's list that follow the point where
// every pixel of the tile has stopped are never read.  A bound finds such a
// point without compositing: if a Gaussian's alpha is at least a_lo at every
// pixel centre of a tile, each pixel that has not stopped multiplies its T by
// at most (1 - a_lo), so once the sum of -ln(1 - a_lo) over such Gaussians
// passes -ln(t_eps) every pixel of the tile has stopped (a pixel that had not
// would hold T < t_eps).  Per sorted entry two nested boxes, inside the
// ellipses q2 <= 3 and q2 <= 1, give the tiles whose pixel centres all lie in
// them; on those tiles alpha >= min(alpha_max, op exp(-q/2)).  The bounds are
// shrunk by margins far above FP32 rounding, and a level whose bound falls
// below alpha_min counts nothing, so the cut only ever drops entries that no
// pixel reaches: every output is the one the full lists give.
constexpr float kCutUnits = 256.f;  // mass units per unit of -ln(1 - a)
__host__ __device__ constexpr float cut_level(int l) { return l == 0 ? 3.f : 1.f; }  // outer, inner q2

__device__ __forceinline__ uint32_t pack_range(int lo, int hi) {
    return (uint32_t)(lo & 0xFFFF) | ((uint32_t)(hi & 0xFFFF) << 16);
}

// Tile range of the pixel centres inside [m - h, m + h] (centres of tile k are
// 16 k + 0.5 .. 16 k + 15.5), within the rectangle's [lo, hi].
__device__ __forceinline__ uint32_t inner_range(float m, float h, int lo, int hi) {
    const float f0 = fminf(fmaxf(ceilf((m - h - 0.5f) * (1.f / kTile)), -1e6f), 1e6f);
    const float f1 = fminf(fmaxf(floorf((m + h - (kTile - 0.5f)) * (1.f / kTile)), -1e6f), 1e6f);
    const int k0 = max(lo, (int)f0), k1 = min(hi, (int)f1);
    return k0 <= k1 ? pack_range(k0, k1) : pack_range(1, 0);
}

__device__ __forceinline__ uint32_t cut_units(float op, float q, float amin, float amax) {
    const float alo = fminf(amax, op * expf(-0.5f * q)) * (1.f - 1e-3f);
    if (!(alo > 0.f) || alo < amin * (1.f + 1e-3f)) return 0u;
    return (uint32_t)floorf(-log1pf(-alo) * kCutUnits * (1.f - 1e-4f));
}

__global__ void __launch_bounds__(256) k_gather_rects(const uint32_t *__restrict__ order, ProjView pv, long long cn,
                                                      short4 *rect, int4 *inner, uint32_t *imass, Params p) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cn) return;
    const uint32_t e = order[i];
    const bool live = pv.ntiles[e] != 0u;
    const int4 r = live ? pv.trect[e] : make_int4(0, 0, -1, -1);
    rect[i] = make_short4((short)r.x, (short)r.y, (short)r.z, (short)r.w);  // tile coordinates fit in 16 bits
    if (inner == nullptr) return;
    // the two boxes |dx| <= a, |dy| <= b with b = a sqrt(A/C): their corners
    // give q2 = 2 a^2 (A + |B| sqrt(A/C)) = q
    uint32_t bx[2] = {pack_range(1, 0), pack_range(1, 0)}, by[2] = {pack_range(1, 0), pack_range(1, 0)};
    uint32_t u[2] = {0u, 0u};
    if (live) {
        const GRec g = pv.rec[e];
        const float A = g.a.z, B = g.a.w, C = g.b.x, op = g.b.y;
        if (A > 0.f && C > 0.f) {
            const float rr = sqrtf(A / C);
            const float den = 2.f * (A + fabsf(B) * rr);
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                const float q = cut_level(l);
                if (q > p.cut) continue;
                u[l] = cut_units(op, q, p.amin, p.amax);
                if (u[l] == 0u) continue;
                const float a0 = sqrtf(q / den);
                const float ha = a0 * (1.f - 1e-3f) - 1e-2f, hb = a0 * rr * (1.f - 1e-3f) - 1e-2f;
                if (!(ha > 0.f) || !(hb > 0.f)) {
                    u[l] = 0u;
                    continue;
                }
                bx[l] = inner_range(g.a.x, ha, r.x, r.z);
                by[l] = inner_range(g.a.y, hb, r.y, r.w);
            }
        }
    }
    if (u[1] < u[0]) u[1] = u[0];  // the inner box holds at least the outer bound
    inner[i] = make_int4((int)bx[0], (int)by[0], (int)bx[1], (int)by[1]);
    imass[i] = u[0] | ((u[1] - u[0]) << 16);
}

__device__ __forceinline__ void add_box(int *d, int pitch, uint32_t rx, uint32_t ry, int v) {
    const int x0 = (int)(rx & 0xFFFFu), x1 = (int)(rx >> 16), y0 = (int)(ry & 0xFFFFu), y1 = (int)(ry >> 16);
    if (v == 0 || x0 > x1 || y0 > y1) return;
    atomicAdd(&d[y0 * pitch + x0], v);
    atomicAdd(&d[y0 * pitch + x1 + 1], -v);
    atomicAdd(&d[(y1 + 1) * pitch + x0], -v);
    atomicAdd(&d[(y1 + 1) * pitch + x1 + 1], v);
}

// With the list cut (CUT) the same pass sums the segment's opacity mass per
// tile (a second difference array over the nested boxes) into mass[].
template <bool CUT>
__global__ void __launch_bounds__(256) k_seg_count(const short4 *__restrict__ rect, const int4 *__restrict__ inner,
                                                   const uint32_t *__restrict__ imass, long long N, int SEG, int S,
                                                   CamSet cs, uint32_t *table, uint32_t *mass) {
    extern __shared__ int diff[];
    const int seg = blockIdx.x, ci = blockIdx.y;
    const DevCam &cam = cs.c[ci];
    const int tx = cam.tiles_x, ty = cam.tiles_y, pitch = tx + 1;
    const int cells = pitch * (ty + 1);
    int *dm = diff + cells;
    for (int i = threadIdx.x; i < cells; i += blockDim.x) {
        diff[i] = 0;
        if (CUT) dm[i] = 0;
    }
    __syncthreads();
    const long long b0 = (long long)ci * N + (long long)seg * SEG;
    const long long b1 = min((long long)(ci + 1) * N, b0 + SEG);
    for (long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        const short4 sr = rect[i];
        const int4 r = make_int4(sr.x, sr.y, sr.z, sr.w);
        if (r.w < r.y) continue;
        atomicAdd(&diff[r.y * pitch + r.x], 1);
        atomicAdd(&diff[r.y * pitch + r.z + 1], -1);
        atomicAdd(&diff[(r.w + 1) * pitch + r.x], -1);
        atomicAdd(&diff[(r.w + 1) * pitch + r.z + 1], 1);
        if (CUT) {
            const int4 ib = inner[i];
            const uint32_t m = imass[i];
            add_box(dm, pitch, (uint32_t)ib.x, (uint32_t)ib.y, (int)(m & 0xFFFFu));
            add_box(dm, pitch, (uint32_t)ib.z, (uint32_t)ib.w, (int)(m >> 16));
        }
    }
    __syncthreads();
    for (int y = threadIdx.x; y < ty; y += blockDim.x) {  // prefix along x
        int acc = 0, am = 0;
        for (int x = 0; x < tx; ++x) {
            acc += diff[y * pitch + x];
            diff[y * pitch + x] = acc;
            if (CUT) {
                am += dm[y * pitch + x];
                dm[y * pitch + x] = am;
            }
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < tx; x += blockDim.x) {  // prefix along y
        int acc = 0, am = 0;
        for (int y = 0; y < ty; ++y) {
            acc += diff[y * pitch + x];
            diff[y * pitch + x] = acc;
            if (CUT) {
                am += dm[y * pitch + x];
                dm[y * pitch + x] = am;
            }
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < tx * ty; t += blockDim.x) {
        const int y = t / tx, x = t - y * tx;
        table[(long long)(cam.tile_off + t) * S + seg] = (uint32_t)diff[y * pitch + x];
        if (CUT) mass[(long long)(cam.tile_off + t) * S + seg] = (uint32_t)dm[y * pitch + x];
    }
}

// One warp per tile: the first segment by whose end the tile's opacity mass
// reaches thr closes the tile; the counts of all later segments become 0, so
// the scan and the scatter give the tile only the entries up to that segment.
// close[t] = S when the mass never reaches thr.
__global__ void __launch_bounds__(256) k_close_tiles(const uint32_t *__restrict__ mass, int S, int total_tiles,
                                                     uint32_t thr, uint32_t *table, int *close) {
    const int t = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (t >= total_tiles) return;
    const uint32_t *m = mass + (long long)t * S;
    uint32_t *c = table + (long long)t * S;
    uint32_t run = 0;
    int cs = S;
    for (int s0 = 0; s0 < S; s0 += 32) {
        const int s = s0 + lane;
        const uint32_t v = s < S ? min(m[s], thr) : 0u;  // capped: the sums stay far below 2^32
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t hit = __ballot_sync(0xffffffffu, run + incl >= thr);
        if (hit) {
            cs = s0 + __ffs(hit) - 1;
            break;
        }
        run += __shfl_sync(0xffffffffu, incl, 31);
    }
    for (int s = cs + 1 + lane; s < S; s += 32) c[s] = 0u;
    if (lane == 0) close[t] = cs;
}

// ------------------------------------------------------------- big scan
// Exclusive scan of a long u32 array: block sums, scan of the sums, then a
// block-local rescan with the offsets.
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ a, long long n,
                                                              uint32_t *partials) {
    const long long base = (long long)blockIdx.x * kScanTile;
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const long long j = base + i * kScanThreads + threadIdx.x;
        if (j < n) sum += a[j];
    }
    __shared__ uint32_t red[kScanThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) s += red[w];
        partials[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(uint32_t *a, long long n,
                                                            const uint32_t *__restrict__ partials) {
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t tsum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? a[base + i] : 0u;
        tsum += v[i];
    }
    uint32_t x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) >= o) x += y;
    }
    __shared__ uint32_t wsum[kScanThreads / 32];
    if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) wpre += wsum[w];
    uint32_t run = partials[blockIdx.x] + wpre + x - tsum;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) a[base + i] = run;
        run += v[i];
    }
}

// ------------------------------------------------------------- scatter
constexpr int kScatterWarps = 4;
constexpr int kStage = 128;  // entries staged in shared memory per step
constexpr int kScatterCtr = 8192;  // tile counters per warp at most: 145 KB per block
constexpr int kScatterStageWords = kStage * 7;  // staged rectangles, indices and prefix per warp

// One warp per (segment, camera, band of tile rows): walks the segment's
// Gaussians in depth order and writes each one into every tile of its
// rectangle that lies in the band, at the tile's running offset.  Long
// segments give each (tile, segment) run many consecutive entries (whole
// sectors per write burst); bands restore the parallelism.  Within one
// Gaussian all tiles differ, so the 32 lanes update distinct counters.
__global__ void __launch_bounds__(kScatterWarps * 32) k_seg_scatter(const uint32_t *__restrict__ order,
                                                                     const short4 *__restrict__ rect,
                                                                     long long N, int SEG, int S, int nband,
                                                                     int band_rows, CamSet cs,
                                                                     const uint32_t *__restrict__ table, uint32_t *gids,
                                                                     long long capacity) {
    extern __shared__ uint32_t sh[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long item = (long long)blockIdx.x * kScatterWarps + warp;
    const int ci = blockIdx.y;
    if (item >= (long long)S * nband) return;  // warp-uniform; the kernel uses no block barrier
    const int seg = (int)(item / nband), band = (int)(item - (long long)seg * nband);
    const DevCam &cam = cs.c[ci];
    const int tx = cam.tiles_x;
    const int by0 = band * band_rows, by1 = min(cam.tiles_y, by0 + band_rows);
    if (by0 >= by1) return;
    const int ctr_words = (band_rows * tx + 3) & ~3;
    uint32_t *ctr = sh + warp * (ctr_words + kScatterStageWords);
    int4 *st_r = reinterpret_cast<int4 *>(ctr + ctr_words);         // staged rectangles
    uint32_t *st_g = reinterpret_cast<uint32_t *>(st_r + kStage);  // staged Gaussian index
    uint32_t *st_p = st_g + kStage;                                 // exclusive prefix of their tile counts
    const int T = (by1 - by0) * tx;
    for (int t = lane; t < T; t += 32) ctr[t] = table[(long long)(cam.tile_off + by0 * tx + t) * S + seg];
    const long long b0 = (long long)ci * N + (long long)seg * SEG;
    const long long b1 = min((long long)(ci + 1) * N, b0 + SEG);
    for (long long c0 = b0; c0 < b1; c0 += kStage) {
        const int m = (int)min((long long)kStage, b1 - c0);
        __syncwarp();
        // stage only the Gaussians that touch the band, in order (ballot compaction)
        int mt = 0;
        // the stage's rectangles and indices are requested together
        short4 rs[kStage / 32];
        uint32_t es[kStage / 32];
#pragma unroll
        for (int u = 0; u < kStage / 32; ++u) {
            const int k = u * 32 + lane;
            rs[u] = k < m ? rect[c0 + k] : make_short4(0, 0, -1, -1);
            es[u] = k < m ? order[c0 + k] : 0u;
        }
#pragma unroll
        for (int u = 0; u < kStage / 32; ++u) {
            int4 r = make_int4(rs[u].x, rs[u].y, rs[u].z, rs[u].w);
            const uint32_t e = es[u];
            r.y = max(r.y, by0);
            r.w = min(r.w, by1 - 1);
            const bool touch = r.w >= r.y;
            const uint32_t bal = __ballot_sync(0xffffffffu, touch);
            if (touch) {
                const int at = mt + __popc(bal & ((1u << lane) - 1u));
                st_r[at] = r;
                st_g[at] = (uint32_t)(e - (long long)ci * N);
            }
            mt += __popc(bal);
        }
        __syncwarp();
        // the staged Gaussians' (Gaussian, tile) pairs, flattened in order:
        // lane l of step s takes pair 32 s + l.  Pairs of one step that hit
        // the same tile are ranked by lane, which is their depth order.
        uint32_t cnt[kStage / 32];
        uint32_t lsum = 0;
#pragma unroll
        for (int u = 0; u < kStage / 32; ++u) {
            const int k = lane * (kStage / 32) + u;
            cnt[u] = 0;
            if (k < mt) {
                const int4 r = st_r[k];
                cnt[u] = (uint32_t)((r.z - r.x + 1) * (r.w - r.y + 1));
            }
            lsum += cnt[u];
        }
        uint32_t incl = lsum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        uint32_t run = incl - lsum;
#pragma unroll
        for (int u = 0; u < kStage / 32; ++u) {
            st_p[lane * (kStage / 32) + u] = run;
            run += cnt[u];
        }
        __syncwarp();
        const uint32_t lt_mask = (1u << lane) - 1u;
        for (uint32_t i0 = 0; i0 < total; i0 += 32) {
            const uint32_t i = i0 + lane;
            const bool act = i < total;
            // the Gaussian of pair i: the last k with prefix[k] <= i
            int lo = 0, hi = mt - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (st_p[mid] <= i) lo = mid;
                else hi = mid - 1;
            }
            const int4 r = st_r[lo];
            const int w = r.z - r.x + 1;
            const uint32_t q = i - st_p[lo];
            // q / w via a float reciprocal: exact for q < 2^22 (q + 0.5 never lands on an integer)
            const int qy = (int)(((float)q + 0.5f) * (1.f / (float)w));
            const int qx = (int)q - qy * w;
            const int t = (r.y - by0 + qy) * tx + r.x + qx;
            const uint32_t same = __match_any_sync(0xffffffffu, act ? (uint32_t)t : (0x80000000u | (uint32_t)lane));
            const uint32_t rank = __popc(same & lt_mask);
            const uint32_t base = act ? ctr[t] : 0u;
            __syncwarp();
            if (act) {
                const uint32_t pos = base + rank;
                if (pos < capacity) gids[pos] = st_g[lo];
                if (rank == 0) ctr[t] = base + (uint32_t)__popc(same);
            }
            __syncwarp();
        }
    }
}

// The scatter of the list cut: one warp per (segment, camera, tile row).
// Tiles closed before this segment (close[t] < seg) take no entries.  The
// row's open tiles are listed in shared memory (olist; opre[x] = open tiles
// left of x), a staged Gaussian's pairs are the open tiles of its x range in
// order, and a warp whose row has no open tile leaves at once.
__global__ void __launch_bounds__(kScatterWarps * 32) k_seg_scatter_cut(const uint32_t *__restrict__ order,
                                                                         const short4 *__restrict__ rect, long long N,
                                                                         int SEG, int S, int max_ty, int row_words,
                                                                         CamSet cs, const int *__restrict__ close,
                                                                         const uint32_t *__restrict__ table,
                                                                         uint32_t *gids, long long capacity) {
    extern __shared__ uint32_t sh[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long item = (long long)blockIdx.x * kScatterWarps + warp;
    const int ci = blockIdx.y;
    if (item >= (long long)S * max_ty) return;  // warp-uniform; the kernel uses no block barrier
    const int seg = (int)(item / max_ty), row = (int)(item - (long long)seg * max_ty);
    const DevCam &cam = cs.c[ci];
    if (row >= cam.tiles_y) return;
    const int tx = cam.tiles_x;
    uint32_t *ctr = sh + warp * (3 * row_words + kScatterStageWords);
    uint32_t *opre = ctr + row_words;
    uint32_t *olist = opre + row_words;
    uint32_t *st_o = olist + row_words;  // staged: first open index, pair count, Gaussian, pair prefix
    uint32_t *st_c = st_o + kStage;
    uint32_t *st_g = st_c + kStage;
    uint32_t *st_p = st_g + kStage;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int tbase = cam.tile_off + row * tx;
    uint32_t nopen = 0;
    for (int x0 = 0; x0 < tx; x0 += 32) {
        const int x = x0 + lane;
        const bool open = x < tx && seg <= close[tbase + x];
        const uint32_t bal = __ballot_sync(0xffffffffu, open);
        const uint32_t at = nopen + __popc(bal & lt_mask);
        if (x < tx) opre[x] = at;
        if (open) {
            olist[at] = (uint32_t)x;
            ctr[x] = table[(long long)(tbase + x) * S + seg];
        }
        nopen += __popc(bal);
    }
    if (nopen == 0) return;
    if (lane == 0) opre[tx] = nopen;
    __syncwarp();
    const long long b0 = (long long)ci * N + (long long)seg * SEG;
    const long long b1 = min((long long)(ci + 1) * N, b0 + SEG);
    // a stage's rectangles and indices are requested together, and the next
    // stage's while this one's pairs are written: eight loads in flight
    short4 rs[kStage / 32];
    uint32_t es[kStage / 32];
    auto fetch = [&](long long c) {
#pragma unroll
        for (int u = 0; u < kStage / 32; ++u) {
            const long long k = c + u * 32 + lane;
            rs[u] = k < b1 ? rect[k] : make_short4(0, 0, -1, -1);
            es[u] = k < b1 ? order[k] : 0u;
        }
    };
    fetch(b0);
    for (long long c0 = b0; c0 < b1; c0 += kStage) {
        __syncwarp();
        int mt = 0;
        short4 rn[kStage / 32];
        uint32_t en[kStage / 32];
#pragma unroll
        for (int u = 0; u < kStage / 32; ++u) {
            rn[u] = rs[u];
            en[u] = es[u];
        }
        if (c0 + kStage < b1) fetch(c0 + kStage);
#pragma unroll
        for (int u = 0; u < kStage / 32; ++u) {
            uint32_t o0 = 0, cnt = 0;
            const short4 r = rn[u];
            const uint32_t e = en[u];
            if (r.y <= row && row <= r.w) {
                o0 = opre[r.x];
                cnt = opre[r.z + 1] - o0;
            }
            const bool touch = cnt > 0u;
            const uint32_t bal = __ballot_sync(0xffffffffu, touch);
            if (touch) {
                const int at = mt + __popc(bal & lt_mask);
                st_o[at] = o0;
                st_c[at] = cnt;
                st_g[at] = (uint32_t)(e - (long long)ci * N);
            }
            mt += __popc(bal);
        }
        __syncwarp();
        if (mt == 0) continue;
        uint32_t cnt[kStage / 32];
        uint32_t lsum = 0;
#pragma unroll
        for (int u = 0; u < kStage / 32; ++u) {
            const int k = lane * (kStage / 32) + u;
            cnt[u] = k < mt ? st_c[k] : 0u;
            lsum += cnt[u];
        }
        uint32_t incl = lsum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        uint32_t run = incl - lsum;
#pragma unroll
        for (int u = 0; u < kStage / 32; ++u) {
            st_p[lane * (kStage / 32) + u] = run;
            run += cnt[u];
        }
        __syncwarp();
        for (uint32_t i0 = 0; i0 < total; i0 += 32) {
            const uint32_t i = i0 + lane;
            const bool act = i < total;
            int lo = 0, hi = mt - 1;  // the staged Gaussian of pair i: the last k with prefix[k] <= i
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (st_p[mid] <= i) lo = mid;
                else hi = mid - 1;
            }
            const uint32_t x = act ? olist[st_o[lo] + (i - st_p[lo])] : 0u;
            const uint32_t same = __match_any_sync(0xffffffffu, act ? x : (0x80000000u | (uint32_t)lane));
            const uint32_t rank = __popc(same & lt_mask);
            const uint32_t base = act ? ctr[x] : 0u;
            __syncwarp();
            if (act) {
                const uint32_t pos = base + rank;
                if (pos < capacity) gids[pos] = st_g[lo];
                if (rank == 0) ctr[x] = base + (uint32_t)__popc(same);
            }
            __syncwarp();
        }
    }
}

__global__ void __launch_bounds__(256) k_table_ranges(const uint32_t *__restrict__ table, int S, int total_tiles,
                                                      const int64_t *total, long long capacity, uint32_t *ranges,
                                                      unsigned *status) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = *total;
    if (t == 0 && tot > capacity) latch(status, ST_CAPACITY);
    if (t >= total_tiles) return;
    const long long s = table[(long long)t * S];
    const long long e = (t + 1 < total_tiles) ? (long long)table[(long long)(t + 1) * S] : tot;
    const bool empty = e <= s;  // empty tiles read (0, 0)
    ranges[2 * (long long)t] = empty ? 0u : (uint32_t)min(s, capacity);
    ranges[2 * (long long)t + 1] = empty ? 0u : (uint32_t)min(e, capacity);
}

// 64-bit sort keys of the sorted instances (optional output).
__global__ void __launch_bounds__(256) k_keys64(const uint32_t *__restrict__ ranges, const uint32_t *__restrict__ gids,
                                                ProjView pv, long long N, CamSet cs, uint64_t *keys) {
    const int t = blockIdx.x;
    const int ci = cam_of_tile(cs, t);
    const uint32_t s = ranges[2 * t], e = ranges[2 * t + 1];
    for (uint32_t i = s + threadIdx.x; i < e; i += blockDim.x)
        keys[i] = ((uint64_t)t << 32) | pv.dkey[(long long)ci * N + gids[i]];
}

int seg_size(long long N, int total_tiles) {
    int seg = 256;
    while (seg < 4096 && (N + seg - 1) / seg > 256) seg <<= 1;
    while ((long long)total_tiles * ((N + seg - 1) / seg) > (32ll << 20) && seg < (1 << 20)) seg <<= 1;
    return seg;
}

}  // namespace

size_t bin_scratch_bytes(long long N, int n_cams, int total_tiles, int sm_count) {
    const long long cn = N * n_cams;
    const int SEG = seg_size(N, total_tiles);
    const long long S = (N + SEG - 1) / SEG;
    const long long tab = (long long)total_tiles * (S > 0 ? S : 1);
    const int G = kRadixBlocksPerSM * sm_count;
    return 5 * align_up(sizeof(uint32_t) * (cn + 1), 256) + align_up(sizeof(int4) * (cn + 1), 256) +
           align_up(sizeof(short4) * (cn + 1), 256) +
           2 * align_up(sizeof(uint32_t) * (tab + 1), 256) + align_up(sizeof(int) * (total_tiles + 1), 256) +
           align_up(sizeof(uint32_t) * ((tab + kScanTile - 1) / kScanTile + 1), 256) +
           align_up(sizeof(uint32_t) * kBuckets * (size_t)G, 256) + 256 + 256;
}

BinScratch bin_scratch_view(void *base, long long N, int n_cams, int total_tiles, int sm_count) {
    const long long cn = N * n_cams;
    const int SEG = seg_size(N, total_tiles);
    const long long S = (N + SEG - 1) / SEG;
    const long long tab = (long long)total_tiles * (S > 0 ? S : 1);
    char *p = (char *)align_up((size_t)base, 256);
    BinScratch s;
    auto take = [&](size_t bytes) {
        char *r = p;
        p += align_up(bytes, 256);
        return (uint32_t *)r;
    };
    s.dk_a = take(sizeof(uint32_t) * (cn + 1));
    s.dv_a = take(sizeof(uint32_t) * (cn + 1));
    s.dk_b = take(sizeof(uint32_t) * (cn + 1));
    s.dv_b = take(sizeof(uint32_t) * (cn + 1));
    s.rect = reinterpret_cast<short4 *>(take(sizeof(short4) * (cn + 1)));
    s.inner = reinterpret_cast<int4 *>(take(sizeof(int4) * (cn + 1)));
    s.imass = take(sizeof(uint32_t) * (cn + 1));
    s.table = take(sizeof(uint32_t) * (tab + 1));
    s.mass = take(sizeof(uint32_t) * (tab + 1));
    s.close = reinterpret_cast<int *>(take(sizeof(int) * (total_tiles + 1)));
    s.partials = take(sizeof(uint32_t) * ((tab + kScanTile - 1) / kScanTile + 1));
    s.hist = take(sizeof(uint32_t) * kBuckets * (size_t)(kRadixBlocksPerSM * sm_count));
    s.kbits = take(2 * sizeof(uint32_t));
    s.seg = SEG;
    s.nseg = (int)S;
    s.sm_count = sm_count;
    return s;
}

bool bin_cut_fits(const CamSet &cs) {
    for (int c = 0; c < cs.n; ++c)
        if (2ll * (cs.c[c].tiles_x + 1) * (cs.c[c].tiles_y + 1) > FHGS_MAX_TILE_CELLS) return false;
    return true;
}

namespace {

// 1. depth order of all (camera, Gaussian) entries, grouped by camera, and
// the tile rectangles (with the cut: the nested boxes) in that order.
uint32_t *sort_entries(long long N, int n_cams, ProjView pv, const BinScratch &sc, const Params *cut,
                       cudaStream_t st) {
    const long long cn = (long long)n_cams * N;
    const int G = radix_blocks(cn, sc.sm_count);
    cudaMemsetAsync(sc.kbits, 0xFF, sizeof(uint32_t), st);
    cudaMemsetAsync(sc.kbits + 1, 0, sizeof(uint32_t), st);
    note_launch(1);
    const long long iota_blocks = min((cn + 255) / 256, 8ll * sc.sm_count);
    k_iota_keys<<<(unsigned)iota_blocks, 256, 0, st>>>(pv.dkey, cn, sc.dk_a, sc.dv_a, sc.kbits);
    const bool in_b = radix_sort_pairs(sc.dk_a, sc.dv_a, sc.dk_b, sc.dv_b, cn, 32, sc.hist, G, st, sc.kbits);
    uint32_t *order = in_b ? sc.dv_b : sc.dv_a;
    if (n_cams > 1) {
        uint32_t *ck = in_b ? sc.dk_b : sc.dk_a;  // reuse the key buffer for camera ids
        note_launch(1);
        k_cam_keys<<<(unsigned)((cn + 255) / 256), 256, 0, st>>>(order, cn, N, ck);
        uint32_t *ok2 = in_b ? sc.dk_a : sc.dk_b, *ov2 = in_b ? sc.dv_a : sc.dv_b;
        int bits = 1;
        while ((1 << bits) < n_cams) ++bits;
        if (radix_sort_pairs(ck, order, ok2, ov2, cn, bits, sc.hist, G, st)) order = ov2;
    }
    Params q;
    memset(&q, 0, sizeof(q));
    if (cut) q = *cut;
    note_launch(1);
    k_gather_rects<<<(unsigned)((cn + 255) / 256), 256, 0, st>>>(order, pv, cn, sc.rect, cut ? sc.inner : nullptr,
                                                                 sc.imass, q);
    return order;
}

// 2. per-segment tile counts (and, with the cut, opacity masses)
void count_tiles(long long N, int n_cams, const CamSet &cs, const BinScratch &sc, bool cut, cudaStream_t st) {
    int max_cells = 0;
    for (int c = 0; c < n_cams; ++c) max_cells = max(max_cells, (cs.c[c].tiles_x + 1) * (cs.c[c].tiles_y + 1));
    const int count_smem = (cut ? 2 : 1) * max_cells * (int)sizeof(int);
    note_launch(1);
    if (cut) {
        static std::atomic<unsigned long long> count_done{0};
        allow_max_smem(count_done, k_seg_count<true>);
        k_seg_count<true><<<dim3(sc.nseg, n_cams), 256, count_smem, st>>>(sc.rect, sc.inner, sc.imass, N, sc.seg,
                                                                          sc.nseg, cs, sc.table, sc.mass);
    } else {
        static std::atomic<unsigned long long> count_done{0};
        allow_max_smem(count_done, k_seg_count<false>);
        k_seg_count<false><<<dim3(sc.nseg, n_cams), 256, count_smem, st>>>(sc.rect, nullptr, nullptr, N, sc.seg,
                                                                           sc.nseg, cs, sc.table, nullptr);
    }
}

// 3. exclusive scan of a (tile, segment) table in place, its total into *total
void scan_table(uint32_t *table, long long tab, uint32_t *partials, int64_t *total, cudaStream_t st) {
    const unsigned nparts = (unsigned)((tab + kScanTile - 1) / kScanTile);
    note_launch(3);
    k_scan_reduce<<<nparts, kScanThreads, 0, st>>>(table, tab, partials);
    static std::atomic<unsigned long long> scan_done{0};
    allow_max_smem(scan_done, k_scan_small);
    k_scan_small<<<1, 1024, kScanSmallSmem, st>>>(partials, (int)nparts, total);
    k_scan_down<<<nparts, kScanThreads, 0, st>>>(table, tab, partials);
}

void grid_extent(const CamSet &cs, int &max_tx, int &max_ty) {
    max_tx = max_ty = 0;
    for (int c = 0; c < cs.n; ++c) {
        max_ty = max(max_ty, cs.c[c].tiles_y);
        max_tx = max(max_tx, cs.c[c].tiles_x);
    }
}

// 4b. the list cut's scatter: each segment into the tiles that close[] leaves
// open, at the offsets of the scanned (tile, segment) table
void scatter_cut(long long N, const CamSet &cs, const BinScratch &sc, const uint32_t *order, const fhgs_bins &bins,
                 cudaStream_t st) {
    int max_tx, max_ty;
    grid_extent(cs, max_tx, max_ty);
    if (max_ty == 0) return;
    // one warp per (segment, tile row): counters, open prefix and open list
    const int row_words = (max_tx + 1 + 3) & ~3;
    const int scat_smem = kScatterWarps * (3 * row_words + kScatterStageWords) * (int)sizeof(uint32_t);
    static std::atomic<unsigned long long> scatter_done{0};
    allow_max_smem(scatter_done, k_seg_scatter_cut);
    note_launch(1);
    const long long items = (long long)sc.nseg * max_ty;
    k_seg_scatter_cut<<<dim3((unsigned)((items + kScatterWarps - 1) / kScatterWarps), cs.n), kScatterWarps * 32,
                        scat_smem, st>>>(order, sc.rect, N, sc.seg, sc.nseg, max_ty, row_words, cs, sc.close,
                                         sc.table, bins.gids, bins.capacity);
}

}  // namespace

void launch_bin_sort(long long N, int n_cams, const CamSet &cs, ProjView pv, const fhgs_bins &bins, BinScratch sc,
                     const Params *cutp, unsigned *status, cudaStream_t st) {
    const long long cn = (long long)n_cams * N;
    cudaMemsetAsync(bins.ranges, 0, sizeof(uint32_t) * 2 * (size_t)cs.total_tiles, st);
    cudaMemsetAsync(bins.n_instances, 0, sizeof(int64_t), st);
    if (cn == 0) return;
    // the list cut needs the EWA records, a stop threshold in (0, 1) and room
    // for two difference arrays per camera grid
    const bool cut = cutp != nullptr && cutp->geom == FHGS_GEOM_EWA && cutp->teps > 0.f && cutp->teps < 1.f &&
                     bin_cut_fits(cs);
    const uint32_t *order = sort_entries(N, n_cams, pv, sc, cut ? cutp : nullptr, st);
    const int S = sc.nseg;
    count_tiles(N, n_cams, cs, sc, cut, st);
    if (cut) {
        // tiles close once their mass passes -ln(t_eps) (one unit of margin
        // above the FP32 products of T)
        const uint32_t thr = (uint32_t)ceil(-log((double)cutp->teps) * kCutUnits) + 1u;
        note_launch(1);
        k_close_tiles<<<(cs.total_tiles + 7) / 8, 256, 0, st>>>(sc.mass, S, cs.total_tiles, thr, sc.table,
                                                                sc.close);
    }
    // 3. scan of the (tile, segment) table: segment offsets and the total
    const long long tab = (long long)cs.total_tiles * S;
    scan_table(sc.table, tab, sc.partials, bins.n_instances, st);
    // 4. tile ranges, then the scatter of Gaussian indices
    note_launch(1);
    k_table_ranges<<<(cs.total_tiles + 255) / 256, 256, 0, st>>>(sc.table, S, cs.total_tiles, bins.n_instances,
                                                                 bins.capacity, bins.ranges, status);
    if (cut) {
        scatter_cut(N, cs, sc, order, bins, st);
    } else {
        int max_tx, max_ty;
        grid_extent(cs, max_tx, max_ty);
        // bands of tile rows: enough (segment, band) warps to fill the GPU, at
        // most a few thousand counters each
        const long long want = 128ll * sc.sm_count;  // warps
        int nband = (int)min((long long)max_ty, (want + (long long)S * n_cams - 1) / ((long long)S * n_cams));
        nband = max(nband, 1);
        // at most kScatterCtr counters per warp (tiles_x <= 4096 keeps one row)
        const int band_rows = max(1, min((max_ty + nband - 1) / nband, kScatterCtr / max(max_tx, 1)));
        nband = (max_ty + band_rows - 1) / band_rows;
        const int ctr_words = (band_rows * max_tx + 3) & ~3;
        const int scat_smem = kScatterWarps * (ctr_words + kScatterStageWords) * (int)sizeof(uint32_t);
        static std::atomic<unsigned long long> scatter_done{0};
        allow_max_smem(scatter_done, k_seg_scatter);
        note_launch(1);
        const long long items = (long long)S * nband;
        k_seg_scatter<<<dim3((unsigned)((items + kScatterWarps - 1) / kScatterWarps), n_cams), kScatterWarps * 32,
                        scat_smem, st>>>(order, sc.rect, N, sc.seg, S, nband, band_rows, cs, sc.table, bins.gids,
                                         bins.capacity);
    }
    if (bins.keys) {
        note_launch(1);
        k_keys64<<<cs.total_tiles, 256, 0, st>>>(bins.ranges, bins.gids, pv, N, cs, bins.keys);
    }
}

}  // namespace fhgs
