// Tile binning (App. A: DuplicateWithKeys, SortByKeys, IdentifyTileRanges).
//
// The paper sorts one 64-bit key per tile instance, (tile id << 32 | depth
// bits).  Here the same order is reached in two stable stages, because every
// instance of one Gaussian shares its depth:
//   1. sort the C*N (camera, Gaussian) entries by their 32-bit depth bits
//      (stable LSD radix sort; ties stay in (camera, index) order);
//   2. emit the tile instances in that depth order and stable-sort them by
//      their 32-bit global tile id alone (only ceil(log2 tiles) bits).
// The result equals the ascending sort of (tile << 32 | depth, gid) while
// moving 8 bytes per instance per pass over a few passes instead of 12 bytes
// over six or more.  No kernel waits on another block: each radix pass is
// histogram -> scan -> scatter, all grids fixed, counts read on the device,
// so the sequence can be captured in a CUDA graph.
#include "fhgs_internal.cuh"

namespace fhgs {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048

constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixRounds = 8;                                   // items per thread per tile
constexpr int kRadixTile = kRadixThreads * kRadixRounds;          // 2048
constexpr int kBuckets = 256;

// ---------------------------------------------------------------- scan
// offsets[j] = sum_{j' < j} ntiles[order[j']] (exclusive), total -> *n_out.
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ ntiles,
                                                              const uint32_t *__restrict__ order, long long n,
                                                              uint32_t *partials) {
    const long long base = (long long)blockIdx.x * kScanTile;
    unsigned long long sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const long long j = base + i * kScanThreads + threadIdx.x;
        if (j < n) sum += ntiles[order[j]];
    }
    __shared__ unsigned long long red[kScanThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) s += red[w];
        partials[blockIdx.x] = (uint32_t)min(s, 0xFFFFFFFFull);
    }
}

// Exclusive scan of the block partials in place (one block); writes the total.
__global__ void __launch_bounds__(1024) k_scan_partials(uint32_t *partials, int nblocks, int64_t *n_out) {
    __shared__ unsigned long long carry;
    __shared__ unsigned long long wsum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nblocks; base += 1024) {
        const int i = base + threadIdx.x;
        unsigned long long v = i < nblocks ? partials[i] : 0;
        unsigned long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            unsigned long long w = wsum[threadIdx.x];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
                if (threadIdx.x >= o) w += y;
            }
            wsum[threadIdx.x] = w;
        }
        __syncthreads();
        const unsigned long long wpre = (threadIdx.x >= 32) ? wsum[(threadIdx.x >> 5) - 1] : 0;
        const unsigned long long excl = carry + wpre + x - v;
        if (i < nblocks) partials[i] = (uint32_t)min(excl, 0xFFFFFFFFull);
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_out = (int64_t)carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t *__restrict__ ntiles,
                                                            const uint32_t *__restrict__ order, long long n,
                                                            const uint32_t *__restrict__ partials,
                                                            uint32_t *offsets) {
    // each thread owns kScanItems consecutive entries (blocked), so a warp
    // scan over per-thread sums gives every entry's exclusive prefix
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t tsum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? ntiles[order[base + i]] : 0u;
        tsum += v[i];
    }
    uint32_t x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
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
        if (base + i < n) offsets[base + i] = run;
        run += v[i];
    }
}

// ---------------------------------------------------------------- emit
// Warp-cooperative duplication: each warp takes 32 depth-ordered entries and
// writes the tile instances of each one with all 32 lanes (coalesced).
__global__ void __launch_bounds__(256) k_emit(const uint32_t *__restrict__ order, const uint32_t *__restrict__ offsets,
                                              ProjView pv, long long N, long long n_entries, CamSet cs,
                                              uint32_t *tkey, uint32_t *tval, long long capacity,
                                              const int64_t *n_total, unsigned *status) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    uint32_t nt = 0, off = 0, g = 0;
    int4 tr = make_int4(0, 0, 0, 0);
    int tile_off = 0, tiles_x = 0;
    if (j < n_entries) {
        const uint32_t e = order[j];
        nt = pv.ntiles[e];
        if (nt) {
            const int ci = (int)(e / N);
            g = (uint32_t)(e - (long long)ci * N);
            tr = pv.trect[e];
            off = offsets[j];
            tile_off = cs.c[ci].tile_off;
            tiles_x = cs.c[ci].tiles_x;
        }
    }
    if (lane == 0 && blockIdx.x == 0 && threadIdx.x == 0 && *n_total > capacity) latch(status, ST_CAPACITY);
    for (int k = 0; k < 32; ++k) {
        const uint32_t n_k = __shfl_sync(0xffffffffu, nt, k);
        if (n_k == 0) continue;
        const uint32_t off_k = __shfl_sync(0xffffffffu, off, k);
        const uint32_t g_k = __shfl_sync(0xffffffffu, g, k);
        const int x0 = __shfl_sync(0xffffffffu, tr.x, k);
        const int y0 = __shfl_sync(0xffffffffu, tr.y, k);
        const int x1 = __shfl_sync(0xffffffffu, tr.z, k);
        const int to = __shfl_sync(0xffffffffu, tile_off, k);
        const int tx_n = __shfl_sync(0xffffffffu, tiles_x, k);
        const int w = x1 - x0 + 1;
        for (uint32_t t = lane; t < n_k; t += 32) {
            const long long pos = (long long)off_k + t;
            if (pos >= capacity) break;
            const int ly = (int)(t / (uint32_t)w), lx = (int)(t - (uint32_t)ly * w);
            tkey[pos] = (uint32_t)(to + (y0 + ly) * tx_n + x0 + lx);
            tval[pos] = g_k;
        }
    }
}

// ---------------------------------------------------------------- radix
__device__ __forceinline__ long long clamp_n(const int64_t *n_dev, long long n_host, long long cap) {
    long long n = n_dev ? (long long)*n_dev : n_host;
    return n < cap ? n : cap;
}

// Per-block digit histogram of the block's contiguous segment.
__global__ void __launch_bounds__(kRadixThreads) k_radix_upsweep(const uint32_t *__restrict__ keys,
                                                                 const int64_t *n_dev, long long n_host,
                                                                 long long cap, int shift, uint32_t mask,
                                                                 uint32_t *hist) {
    __shared__ uint32_t h[kRadixWarps][kBuckets];
    for (int i = threadIdx.x; i < kRadixWarps * kBuckets; i += kRadixThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    const long long n = clamp_n(n_dev, n_host, cap);
    const long long G = gridDim.x;
    const long long seg = (n + G - 1) / G;
    const long long s = blockIdx.x * seg, e = min(n, s + seg);
    const int w = threadIdx.x >> 5;
    const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
    for (long long i0 = s; i0 < e; i0 += kRadixThreads) {
        const long long i = i0 + threadIdx.x;
        const int d = i < e ? (int)((keys[i] >> shift) & mask) : (kBuckets + (int)(threadIdx.x & 31));
        // warp-aggregated: one shared-memory add per distinct digit
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (d < kBuckets && (peers & lt) == 0) atomicAdd(&h[w][d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kBuckets; d += kRadixThreads) {
        uint32_t t = 0;
#pragma unroll
        for (int k = 0; k < kRadixWarps; ++k) t += h[k][d];
        hist[(long long)d * G + blockIdx.x] = t;
    }
}

// Exclusive scan of hist (digit-major, block-minor) in place, one block.
__global__ void __launch_bounds__(1024) k_radix_scan(uint32_t *hist, int total) {
    __shared__ uint32_t carry;
    __shared__ uint32_t wsum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < total; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < total ? hist[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t wv = wsum[threadIdx.x];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, wv, o);
                if (threadIdx.x >= o) wv += y;
            }
            wsum[threadIdx.x] = wv;
        }
        __syncthreads();
        const uint32_t wpre = threadIdx.x >= 32 ? wsum[(threadIdx.x >> 5) - 1] : 0u;
        const uint32_t excl = carry + wpre + x - v;
        if (i < total) hist[i] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
}

// Stable scatter.  The block walks its segment in tiles of kRadixTile items;
// inside a tile, warp w owns items [w*256, w*256+256) visited in 8 rounds of
// 32 consecutive items, so (warp, round, lane) is memory order and ranks
// computed in that order keep the sort stable.
__global__ void __launch_bounds__(kRadixThreads) k_radix_downsweep(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, const int64_t *n_dev, long long n_host, long long cap, int shift, uint32_t mask,
    const uint32_t *__restrict__ hist) {
    __shared__ uint32_t run[kBuckets];                 // next output slot per digit
    __shared__ uint32_t tot[kBuckets];                 // this tile's count per digit
    __shared__ uint32_t wcnt[kRadixWarps][kBuckets];   // per-warp counts, then prefixes
    const long long n = clamp_n(n_dev, n_host, cap);
    const long long G = gridDim.x;
    const long long seg = (n + G - 1) / G;
    const long long s = blockIdx.x * seg, e = min(n, s + seg);
    for (int d = threadIdx.x; d < kBuckets; d += kRadixThreads) run[d] = hist[(long long)d * G + blockIdx.x];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (long long t0 = s; t0 < e; t0 += kRadixTile) {
        for (int d = lane; d < kBuckets; d += 32) wcnt[w][d] = 0;
        __syncwarp();
        uint32_t key[kRadixRounds], val[kRadixRounds], rank[kRadixRounds];
        int dig[kRadixRounds];
#pragma unroll
        for (int r = 0; r < kRadixRounds; ++r) {
            const long long i = t0 + w * (32 * kRadixRounds) + r * 32 + lane;
            const bool valid = i < e;
            key[r] = valid ? kin[i] : 0u;
            val[r] = valid ? vin[i] : 0u;
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
        // exclusive prefix over warps per digit; the sum is the tile total
        for (int d = threadIdx.x; d < kBuckets; d += kRadixThreads) {
            uint32_t acc = 0;
#pragma unroll
            for (int k = 0; k < kRadixWarps; ++k) {
                const uint32_t c = wcnt[k][d];
                wcnt[k][d] = acc;
                acc += c;
            }
            tot[d] = acc;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kRadixRounds; ++r) {
            if (dig[r] < kBuckets) {
                const uint32_t pos = run[dig[r]] + wcnt[w][dig[r]] + rank[r];
                kout[pos] = key[r];
                vout[pos] = val[r];
            }
        }
        __syncthreads();
        for (int d = threadIdx.x; d < kBuckets; d += kRadixThreads) run[d] += tot[d];
        __syncthreads();
    }
}

// ---------------------------------------------------------------- ranges
__global__ void __launch_bounds__(256) k_ranges(const uint32_t *__restrict__ tkey, const int64_t *n_dev, long long cap,
                                                uint32_t *ranges) {
    const long long n = clamp_n(n_dev, 0, cap);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t t = tkey[i];
        if (i == 0 || tkey[i - 1] != t) ranges[2 * (long long)t] = (uint32_t)i;
        if (i == n - 1 || tkey[i + 1] != t) ranges[2 * (long long)t + 1] = (uint32_t)(i + 1);
    }
}

__global__ void __launch_bounds__(256) k_keys64(const uint32_t *__restrict__ tkey, const uint32_t *__restrict__ gid,
                                                const int64_t *n_dev, long long cap, ProjView pv, long long N,
                                                CamSet cs, uint64_t *keys) {
    const long long n = clamp_n(n_dev, 0, cap);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t t = tkey[i];
        const int ci = cam_of_tile(cs, (int)t);
        keys[i] = ((uint64_t)t << 32) | pv.dkey[(long long)ci * N + gid[i]];
    }
}

void radix_sort_pairs(uint32_t *kA, uint32_t *vA, uint32_t *kB, uint32_t *vB, const int64_t *n_dev, long long n_host,
                      long long cap, int bits, uint32_t *hist, int G, cudaStream_t st) {
    // data starts in (kA, vA); passes alternate A->B, B->A
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
        k_radix_upsweep<<<G, kRadixThreads, 0, st>>>(ki, n_dev, n_host, cap, shift, mask, hist);
        k_radix_scan<<<1, 1024, 0, st>>>(hist, kBuckets * G);
        k_radix_downsweep<<<G, kRadixThreads, 0, st>>>(ki, vi, ko, vo, n_dev, n_host, cap, shift, mask, hist);
        shift += nb;
        a_to_b = !a_to_b;
    }
}

int radix_passes(int bits) { return (bits + 7) / 8; }

}  // namespace

size_t bin_scratch_bytes(long long cn, long long capacity, int radix_blocks) {
    const long long nparts = (cn + kScanTile - 1) / kScanTile + 1;
    return 5 * align_up(sizeof(uint32_t) * (cn + 1), 256) + align_up(sizeof(uint32_t) * nparts, 256) +
           align_up(sizeof(uint32_t) * kBuckets * (size_t)radix_blocks, 256) +
           3 * align_up(sizeof(uint32_t) * (capacity + 1), 256) + 256;
}

BinScratch bin_scratch_view(void *base, long long cn, long long capacity, int radix_blocks) {
    const long long nparts = (cn + kScanTile - 1) / kScanTile + 1;
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
    s.offsets = take(sizeof(uint32_t) * (cn + 1));
    s.partials = take(sizeof(uint32_t) * nparts);
    s.hist = take(sizeof(uint32_t) * kBuckets * (size_t)radix_blocks);
    s.tk_a = take(sizeof(uint32_t) * (capacity + 1));
    s.tk_b = take(sizeof(uint32_t) * (capacity + 1));
    s.tv_a = take(sizeof(uint32_t) * (capacity + 1));
    s.radix_blocks = radix_blocks;
    return s;
}

__global__ void k_iota_keys(const uint32_t *__restrict__ dkey, long long n, uint32_t *k, uint32_t *v) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        k[i] = dkey[i];
        v[i] = (uint32_t)i;
    }
}

void launch_bin_sort(long long N, int n_cams, const CamSet &cs, ProjView pv, const fhgs_bins &bins, BinScratch sc,
                     unsigned *status, int sm_count, cudaStream_t st) {
    const long long cn = (long long)n_cams * N;
    const int G = sc.radix_blocks;
    cudaMemsetAsync(bins.ranges, 0, sizeof(uint32_t) * 2 * (size_t)cs.total_tiles, st);
    if (cn == 0) {
        cudaMemsetAsync(bins.n_instances, 0, sizeof(int64_t), st);
        return;
    }
    // 1. depth order of all (camera, Gaussian) entries (culled ones last)
    note_launch(1);
    k_iota_keys<<<(unsigned)((cn + 255) / 256), 256, 0, st>>>(pv.dkey, cn, sc.dk_a, sc.dv_a);
    radix_sort_pairs(sc.dk_a, sc.dv_a, sc.dk_b, sc.dv_b, nullptr, cn, cn, 32, sc.hist, G, st);
    const uint32_t *order = sc.dv_a;  // 4 passes: result back in A
    // 2. instance offsets in depth order
    const unsigned nparts = (unsigned)((cn + kScanTile - 1) / kScanTile);
    note_launch(3);
    k_scan_reduce<<<nparts, kScanThreads, 0, st>>>(pv.ntiles, order, cn, sc.partials);
    k_scan_partials<<<1, 1024, 0, st>>>(sc.partials, (int)nparts, bins.n_instances);
    k_scan_down<<<nparts, kScanThreads, 0, st>>>(pv.ntiles, order, cn, sc.partials, sc.offsets);
    // 3. emit, then stable sort by global tile id into bins.gids
    int bits = 1;
    while ((1ll << bits) < (long long)cs.total_tiles) ++bits;
    const int passes = radix_passes(bits);
    uint32_t *k0 = (passes % 2 == 0) ? sc.tk_a : sc.tk_b;
    uint32_t *v0 = (passes % 2 == 0) ? bins.gids : sc.tv_a;
    uint32_t *k1 = (passes % 2 == 0) ? sc.tk_b : sc.tk_a;
    uint32_t *v1 = (passes % 2 == 0) ? sc.tv_a : bins.gids;
    note_launch(1);
    k_emit<<<(unsigned)((cn + 255) / 256), 256, 0, st>>>(order, sc.offsets, pv, N, cn, cs, k0, v0, bins.capacity,
                                                         bins.n_instances, status);
    radix_sort_pairs(k0, v0, k1, v1, bins.n_instances, 0, bins.capacity, bits, sc.hist, G, st);
    // final data is in (k0, v0) when passes is even, (k1, v1) when odd; both
    // choices put the values in bins.gids
    const uint32_t *tk = (passes % 2 == 0) ? k0 : k1;
    const int grid = sm_count * 8;
    note_launch(1);
    k_ranges<<<grid, 256, 0, st>>>(tk, bins.n_instances, bins.capacity, bins.ranges);
    if (bins.keys) note_launch(1);
    if (bins.keys) k_keys64<<<grid, 256, 0, st>>>(tk, bins.gids, bins.n_instances, bins.capacity, pv, N, cs, bins.keys);
}

}  // namespace fhgs
