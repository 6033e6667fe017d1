// Device-wide exclusive scan and stable LSD radix sort (8-bit counting-sort
// passes) used by the binning step (Sec. 2.1 step 1: partition) and by the
// longest-first work ordering.
//
// The sort is single-sweep: one kernel counts every pass's digits over the
// whole key array at once (a digit's total does not depend on the order
// the earlier passes leave), then each pass is one kernel.  A pass ranks a
// 2048-key tile's digits (stable: warp w owns keys [256w, 256w+256) and
// walks them in rounds of 32; lanes holding the same digit find each other
// with __match_any_sync and rank by lane order; a warp-private digit
// histogram in shared memory carries counts across rounds; a per-digit
// prefix over the 8 warps orders warps), finds each digit's offset of the
// tile by a decoupled look-back over the tiles before it, places the tile
// in digit order in shared memory and writes each digit's run to
// consecutive addresses.  Tiles take ids in the order their blocks start
// (an atomic counter), so a tile waits only on tiles whose blocks are
// already running; every wait is bounded.  The resulting order is a pure
// function of the input: the sort is deterministic.
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

constexpr int kMaxPasses = 8;                          // 64-bit keys
constexpr unsigned long long kLbAggregate = 1ull << 62;  // look-back word: tile count of a digit
constexpr unsigned long long kLbPrefix = 2ull << 62;     // look-back word: inclusive prefix
constexpr int kLbMaxSpins = 1 << 20;                    // bound of one look-back wait
constexpr int kLbWindow = 8;                            // look-back words loaded at once

__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Every pass's digit totals at once: totals[p * 256 + d].
__global__ void __launch_bounds__(kScanThreads) k_radix_upsweep(const unsigned long long* __restrict__ keys,
                                                                int n, int passes, int* __restrict__ totals) {
    __shared__ int h[kMaxPasses][kRadixBuckets];
    for (int i = threadIdx.x; i < kMaxPasses * kRadixBuckets; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[idx];
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(k >> (8 * p)) & (kRadixBuckets - 1)], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadixBuckets; i += blockDim.x) {
        const int v = (&h[0][0])[i];
        if (v) atomicAdd(&totals[i], v);
    }
}

// One pass (digit at bit `shift`, pass tag 1..8 in bits 56-61 of the
// look-back words, which start cleared).  digit_total: this pass's 256
// totals; status: 256 look-back words per tile; tile_counter: this pass's
// tile-id counter.  A look-back wait that runs out sets bit 1 of *err.
__global__ void __launch_bounds__(kScanThreads) k_radix_onesweep(
    const unsigned long long* __restrict__ kin, const int* __restrict__ vin,
    unsigned long long* __restrict__ kout, int* __restrict__ vout, int n, int shift, int pass_tag,
    const int* __restrict__ digit_total, unsigned long long* status, unsigned* tile_counter, long long* err,
    unsigned long long* check) {
    constexpr int kWarps = kScanThreads / 32;
    __shared__ int wh[kWarps][kRadixBuckets];
    __shared__ int gbase[kRadixBuckets];
    __shared__ int loff[kRadixBuckets];
    __shared__ int wsum[kWarps];
    __shared__ int s_tile;
    __shared__ unsigned long long skey[kScanTile];
    __shared__ int sval[kScanTile];
    for (int i = threadIdx.x; i < kWarps * kRadixBuckets; i += blockDim.x) (&wh[0][0])[i] = 0;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(tile_counter, 1u);
    __syncthreads();
    const int tile = s_tile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long base = (long long)tile * kScanTile + warp * (kScanItems * 32);
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
    // one digit per thread: prefix over the warps and the tile's count of
    // the digit
    static_assert(kRadixBuckets == kScanThreads, "one digit per thread");
    const int d = threadIdx.x;
    int run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const int t = wh[w][d];
        wh[w][d] = run;
        run += t;
    }
    // the digit's offset of this tile: publish the tile's count, then add
    // the predecessors' words back to one that holds an inclusive prefix
    const unsigned long long tag = (unsigned long long)pass_tag << 56;
    unsigned long long* mine = status + (long long)tile * kRadixBuckets + d;
    long long excl = 0;
    if (tile == 0) {
        st_relaxed(mine, kLbPrefix | tag | (unsigned)run);
    } else {
        st_relaxed(mine, kLbAggregate | tag | (unsigned)run);
        // predecessors in windows of kLbWindow words loaded together (the
        // walk is a chain of dependent loads otherwise)
        int j = tile - 1, spins = 0;
        bool done = false;
        while (j >= 0 && !done) {
            unsigned long long w[kLbWindow];
            const int m = j + 1 < kLbWindow ? j + 1 : kLbWindow;
#pragma unroll
            for (int q = 0; q < kLbWindow; ++q)
                w[q] = q < m ? ld_relaxed(status + (long long)(j - q) * kRadixBuckets + d) : 0ull;
            int q = 0;
            for (; q < m; ++q) {
                if ((int)((w[q] >> 56) & 63) != pass_tag) break;        // not published yet
                excl += (unsigned)w[q];
                if ((w[q] >> 62) == 2ull) {                             // inclusive prefix reached
                    done = true;
                    break;
                }
            }
            if (done) break;
            j -= q;
            if (q < m) {                                                // wait for tile j
                if (++spins > kLbMaxSpins) {
                    if (err) atomicOr((unsigned long long*)err, 2ull);
                    break;
                }
                __nanosleep(32);
            }
        }
        st_relaxed(mine, kLbPrefix | tag | (unsigned)(excl + run));
    }
    // digit bases: exclusive scan of the pass's totals
    const int tot = digit_total[d];
    const int incl_t = warp_inclusive_scan(tot);
    if (lane == 31) wsum[warp] = incl_t;
    __syncthreads();
    if (warp == 0) {
        int v = lane < kWarps ? wsum[lane] : 0;
        v = warp_inclusive_scan(v);
        if (lane < kWarps) wsum[lane] = v;
    }
    __syncthreads();
    gbase[d] = (warp > 0 ? wsum[warp - 1] : 0) + incl_t - tot + (int)excl;
    __syncthreads();
    // the tile's digit offsets inside the tile
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
    const long long tile0 = (long long)tile * kScanTile;
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
    r.bytes = sizeof(int) * (kMaxPasses * kRadixBuckets + kMaxPasses) +
              sizeof(unsigned long long) * (size_t)kRadixBuckets * r.max_tiles;
    cudaError_t e = cudaMalloc(&r.region, r.bytes);
    if (e != cudaSuccess) return cuda_fail(e, "radix_alloc");
    return SR_OK;
}

void radix_free(RadixScratch& r) {
    if (r.region) cudaFree(r.region);
    r.region = nullptr;
    r.bytes = 0;
    r.max_tiles = 0;
}

int radix_sort_pairs(unsigned long long* keys[2], int* vals[2], int n, int key_bits,
                     RadixScratch& r, cudaStream_t st, int* which, unsigned long long* check, long long* err) {
    int cur = 0;
    *which = 0;
    if (n <= 0) return SR_OK;
    const int t = tiles_of(n);
    if (t > r.max_tiles) return set_error(SR_ERR_CAPACITY, "radix scratch too small");
    const int passes = (key_bits + kRadixBits - 1) / kRadixBits;
    if (passes > kMaxPasses) return set_error(SR_ERR_ARG, "radix keys wider than 64 bits");
    if (passes == 0) return SR_OK;
    // region: totals (passes x 256), tile counters (passes), look-back words (256 per tile)
    int* totals = static_cast<int*>(r.region);
    unsigned* counters = reinterpret_cast<unsigned*>(totals + kMaxPasses * kRadixBuckets);
    unsigned long long* status = reinterpret_cast<unsigned long long*>(
        static_cast<char*>(r.region) + sizeof(int) * (kMaxPasses * kRadixBuckets + kMaxPasses));
    const size_t used = sizeof(int) * (kMaxPasses * kRadixBuckets + kMaxPasses) +
                        sizeof(unsigned long long) * (size_t)kRadixBuckets * t;
    SR_CUDA_CHECK(cudaMemsetAsync(r.region, 0, used, st));
    const int ub = t < 1024 ? t : 1024;
    k_radix_upsweep<<<ub, kScanThreads, 0, st>>>(keys[0], n, passes, totals);
    SR_LAUNCH_CHECK("k_radix_upsweep");
    for (int p = 0; p < passes; ++p) {
        k_radix_onesweep<<<t, kScanThreads, 0, st>>>(keys[cur], vals[cur], keys[1 - cur], vals[1 - cur], n,
                                                     kRadixBits * p, p + 1, totals + kRadixBuckets * p, status,
                                                     counters + p, err, check);
        SR_LAUNCH_CHECK("k_radix_onesweep");
        cur = 1 - cur;
    }
    *which = cur;
    return SR_OK;
}

}  // namespace sr
