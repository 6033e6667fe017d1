// Device-wide exclusive scan and stable LSD radix sort (8-bit counting-sort
// passes) used by the binning step (Sec. 2.1 step 1: partition) and by the
// longest-first work ordering.
//
// Radix pass = histogram per 2048-key tile -> exclusive scan of the
// digit-major histogram -> stable scatter (the tile is first placed in
// digit order in shared memory, so that the global writes of each digit's
// run are contiguous).  Stability inside a tile: warp w
// owns keys [256w, 256w+256) and walks them in rounds of 32; lanes holding
// the same digit find each other with __match_any_sync, rank by lane order,
// and a warp-private digit histogram in shared memory carries counts across
// rounds; a per-digit prefix over the 8 warps orders warps.  The resulting
// order is a pure function of the input: the sort is deterministic.
#include "sr_internal.h"

namespace sr {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int warp_inclusive_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan of one 2048-item tile (8 consecutive items per thread);
// writes the tile total to tile_sums[blockIdx.x].
__global__ void __launch_bounds__(kScanThreads) k_scan_tile(const int* __restrict__ in, int* out,
                                                             int n, int* tile_sums) {
    __shared__ int warp_sums[kScanThreads / 32];
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
    int local = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const long long idx = base + k;
        v[k] = idx < n ? in[idx] : 0;
        local += v[k];
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int incl = warp_inclusive_scan(local);
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
        w = warp_inclusive_scan(w);
        if (lane < kScanThreads / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    int run = (warp > 0 ? warp_sums[warp - 1] : 0) + incl - local;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const long long idx = base + k;
        if (idx < n) out[idx] = run;
        run += v[k];
    }
    if (threadIdx.x == 0 && tile_sums != nullptr) tile_sums[blockIdx.x] = warp_sums[kScanThreads / 32 - 1];
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(int* out, int n, const int* __restrict__ offs) {
    const int add = offs[blockIdx.x];
    const long long base = (long long)blockIdx.x * kScanTile;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const long long idx = base + k * kScanThreads + threadIdx.x;
        if (idx < n) out[idx] += add;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_radix_hist(const unsigned long long* __restrict__ keys,
                                                              int n, int shift, int* hist, int n_tiles) {
    __shared__ int h[kRadixBuckets];
    for (int i = threadIdx.x; i < kRadixBuckets; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kScanTile;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const long long idx = base + k * kScanThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & (kRadixBuckets - 1)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadixBuckets; d += blockDim.x) hist[(long long)d * n_tiles + blockIdx.x] = h[d];
}

__global__ void __launch_bounds__(kScanThreads) k_radix_scatter(
    const unsigned long long* __restrict__ kin, const int* __restrict__ vin,
    unsigned long long* __restrict__ kout, int* __restrict__ vout, int n, int shift,
    const int* __restrict__ hist_scan, int n_tiles, unsigned long long* check) {
    constexpr int kWarps = kScanThreads / 32;
    __shared__ int wh[kWarps][kRadixBuckets];
    __shared__ int gbase[kRadixBuckets];
    __shared__ int loff[kRadixBuckets];
    __shared__ int wsum[kWarps];
    __shared__ unsigned long long skey[kScanTile];
    __shared__ int sval[kScanTile];
    for (int i = threadIdx.x; i < kWarps * kRadixBuckets; i += blockDim.x) (&wh[0][0])[i] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long base = (long long)blockIdx.x * kScanTile + warp * (kScanItems * 32);
    unsigned long long key[kScanItems];
    int val[kScanItems], dig[kScanItems], rnk[kScanItems];
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        const long long idx = base + r * 32 + lane;
        const bool ok = idx < n;
        key[r] = ok ? kin[idx] : 0ull;
        val[r] = ok ? vin[idx] : 0;
        dig[r] = ok ? (int)((key[r] >> shift) & (kRadixBuckets - 1)) : kRadixBuckets;
        const unsigned peers = __match_any_sync(kFull, dig[r]);
        const int old = ok ? wh[warp][dig[r]] : 0;
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) wh[warp][dig[r]] = old + __popc(peers);
        __syncwarp();
        rnk[r] = old + __popc(peers & lt);
    }
    __syncthreads();
    // one digit per thread: prefix over the warps, the tile's count of the
    // digit, and (block scan) the digit's first position inside the tile
    static_assert(kRadixBuckets == kScanThreads, "one digit per thread");
    const int d = threadIdx.x;
    int run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const int t = wh[w][d];
        wh[w][d] = run;
        run += t;
    }
    gbase[d] = hist_scan[(long long)d * n_tiles + blockIdx.x];
    const int incl = warp_inclusive_scan(run);
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int v = lane < kWarps ? wsum[lane] : 0;
        v = warp_inclusive_scan(v);
        if (lane < kWarps) wsum[lane] = v;
    }
    __syncthreads();
    loff[d] = (warp > 0 ? wsum[warp - 1] : 0) + incl - run;
    __syncthreads();
    // the tile in digit order in shared memory (the same order as the
    // global output: warp, round, lane within each digit) ...
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        if (dig[r] < kRadixBuckets) {
            const int lp = loff[dig[r]] + wh[warp][dig[r]] + rnk[r];
            skey[lp] = key[r];
            sval[lp] = val[r];
        }
    }
    __syncthreads();
    // ... then written out by consecutive threads to consecutive addresses
    // of each digit's run
    const long long tile0 = (long long)blockIdx.x * kScanTile;
    const int cnt = (int)(n - tile0 < kScanTile ? n - tile0 : kScanTile);
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        const unsigned long long k = skey[t];
        const int dd = (int)((k >> shift) & (kRadixBuckets - 1));
        const int pos = gbase[dd] + (t - loff[dd]);
        if (!SR_BOUND(pos >= 0 && pos < n, check, kChkScatter)) continue;
        kout[pos] = k;
        vout[pos] = sval[t];
    }
}

inline int tiles_of(long long n) { return (int)((n + kScanTile - 1) / kScanTile); }

}  // namespace

int scan_alloc(ScanScratch& s, long long n) {
    scan_free(s);
    long long m = n;
    while (true) {
        const int t = tiles_of(m);
        int* buf = nullptr;
        cudaError_t e = cudaMalloc(&buf, sizeof(int) * (size_t)(t > 0 ? t : 1));
        if (e != cudaSuccess) return cuda_fail(e, "scan_alloc");
        s.partials.push_back(buf);
        s.sizes.push_back(t);
        if (t <= 1) break;
        m = t;
    }
    return SR_OK;
}

void scan_free(ScanScratch& s) {
    for (int* p : s.partials) cudaFree(p);
    s.partials.clear();
    s.sizes.clear();
}

static int scan_level(const int* in, int* out, int n, ScanScratch& s, size_t level, cudaStream_t st) {
    if (n <= 0) return SR_OK;
    const int t = tiles_of(n);
    if (level >= s.partials.size() || t > s.sizes[level]) return set_error(SR_ERR_CAPACITY, "scan scratch too small");
    k_scan_tile<<<t, kScanThreads, 0, st>>>(in, out, n, s.partials[level]);
    SR_LAUNCH_CHECK("k_scan_tile");
    if (t > 1) {
        int rc = scan_level(s.partials[level], s.partials[level], t, s, level + 1, st);
        if (rc) return rc;
        k_scan_add<<<t, kScanThreads, 0, st>>>(out, n, s.partials[level]);
        SR_LAUNCH_CHECK("k_scan_add");
    }
    return SR_OK;
}

int exclusive_scan(const int* in, int* out, int n, ScanScratch& s, cudaStream_t st) {
    return scan_level(in, out, n, s, 0, st);
}

int radix_alloc(RadixScratch& r, long long n) {
    radix_free(r);
    r.max_tiles = tiles_of(n > 0 ? n : 1);
    const size_t hn = (size_t)kRadixBuckets * r.max_tiles;
    cudaError_t e = cudaMalloc(&r.hist, sizeof(int) * hn);
    if (e != cudaSuccess) return cuda_fail(e, "radix_alloc");
    e = cudaMalloc(&r.hist_scan, sizeof(int) * hn);
    if (e != cudaSuccess) return cuda_fail(e, "radix_alloc");
    return scan_alloc(r.scan, (long long)hn);
}

void radix_free(RadixScratch& r) {
    if (r.hist) cudaFree(r.hist);
    if (r.hist_scan) cudaFree(r.hist_scan);
    r.hist = r.hist_scan = nullptr;
    r.max_tiles = 0;
    scan_free(r.scan);
}

int radix_sort_pairs(unsigned long long* keys[2], int* vals[2], int n, int key_bits,
                     RadixScratch& r, cudaStream_t st, int* which, unsigned long long* check) {
    int cur = 0;
    *which = 0;
    if (n <= 0) return SR_OK;
    const int t = tiles_of(n);
    if (t > r.max_tiles) return set_error(SR_ERR_CAPACITY, "radix scratch too small");
    const int hn = kRadixBuckets * t;
    for (int shift = 0; shift < key_bits; shift += kRadixBits) {
        k_radix_hist<<<t, kScanThreads, 0, st>>>(keys[cur], n, shift, r.hist, t);
        SR_LAUNCH_CHECK("k_radix_hist");
        int rc = exclusive_scan(r.hist, r.hist_scan, hn, r.scan, st);
        if (rc) return rc;
        k_radix_scatter<<<t, kScanThreads, 0, st>>>(keys[cur], vals[cur], keys[1 - cur], vals[1 - cur], n,
                                                    shift, r.hist_scan, t, check);
        SR_LAUNCH_CHECK("k_radix_scatter");
        cur = 1 - cur;
    }
    *which = cur;
    return SR_OK;
}

}  // namespace sr
