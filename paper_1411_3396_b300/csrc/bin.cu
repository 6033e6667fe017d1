// Binning: bit-exact cells, sub-cell Morton order and 32-particle chunks.
// This is step 1 of the paper's short-range timestep (Sec. 2.1: partition
// the volume into overlapping blocks of active particles whose passive
// neighbours lie within the cutoff).
//
// Spec (per volume of side L, n_c cells per axis, b sub-cell bits,
// M = n_c 2^b fine cells per axis, h = L / M in binary64):
//   fold      x < 0 -> x + L, then x >= L -> x - L     (inputs in [-L, 2L))
//   t = x / h (binary64, round to nearest), q = min(floor(t), M - 1)
//   cell = q >> b, sub = q & (2^b - 1), global cell id volume-major,
//   key = (cell << 3b) | morton(sub); order by key, ties by caller index
//   chunks = runs of <= 32 consecutive particles inside a cell
//   anchor qA = q of the chunk's first particle, offset = binary32(t - qA)
//
// The order is reached by a counting sort on the cell, then a sort of each
// cell on the composite (morton(sub) << ib) | caller index, ib = bits of a
// caller index:
//   k_keys           cell and Morton code per particle; per-cell counts
//                    taken with atomics give each particle a place in its
//                    cell (in no fixed order)
//   k_cell_scan      one pass over the cells (decoupled look-back): cell
//                    starts, chunk starts and each chunk's record (cell,
//                    first sorted row, count, volume); cells
//                    of 2..kWarpSeg particles are listed for a warp sort,
//                    larger ones up to kSegTile for a block sort, the rest
//                    as huge
//   k_scatter        each particle's composite into its cell's range
//   k_split          one block per huge cell splits it on the composite's
//                    top 8 bits into up to 256 buckets, which are listed
//   k_sort_segments  the listed ranges: a warp each (bitonic in registers
//                    up to kSmallCell, else stable LSD passes on the
//                    Morton code's 8-bit digits in the warp's shared memory
//                    and then each run of equal codes in caller-index
//                    order), then a block each for the block list (the same
//                    steps, through global memory above kSegTile)
//   k_chunk_fill     one warp per U chunks: slots from the sorted composites
// The composites of a cell are distinct (the caller index is part of
// them), so each cell ends in the spec's order whatever order the atomics
// left, and the result is a pure function of the input.
#include "sr_internal.h"

namespace sr {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long spread3(unsigned v) {
    unsigned long long x = v & 0x3ffu;               // up to 10 bits
    x = (x | (x << 16)) & 0x030000FFull;
    x = (x | (x << 8)) & 0x0300F00Full;
    x = (x | (x << 4)) & 0x030C30C3ull;
    x = (x | (x << 2)) & 0x09249249ull;
    return x;
}

__device__ __forceinline__ int volume_of_row(long long i, const long long* __restrict__ part_start,
                                             int n_vol) {
    // largest v with part_start[v] <= i  (part_start[0] = 0)
    int lo = 0, hi = n_vol;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (part_start[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int volume_of_cell(int cell, const int* __restrict__ cell_base, int n_vol) {
    int lo = 0, hi = n_vol;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (cell_base[mid] <= cell) lo = mid; else hi = mid;
    }
    return lo;
}

// x / h correctly rounded in binary64, for x in [0, box) and y = RN(1/h),
// by Markstein's fused multiply-add quotient correction (P. Markstein, IBM
// J. Res. Dev. 34(1), 1990).  The product x y can be 1.5 ulp from x / h,
// so one correction step first brings q within an ulp.  After that the
// residual x - h q is exact, and q + (x - h q) y rounds to the correctly
// rounded quotient.  Five binary64 operations replace a division; B300's
// binary64 rate makes that the cost of binning when h is not a power of
// two.  Below 2^-900 the residual could leave the normal range, so the
// division is taken there (x = 0 included).
__device__ __forceinline__ double quotient_rn_normal(double x, double h, double y) {   // x >= 2^-900
    double q = x * y;
    q = fma(fma(-q, h, x), y, q);
    return fma(fma(-q, h, x), y, q);
}

// The same correctly rounded quotient from the product alone and one exact
// integer step, for x in [2^-900, box) and h not a power of two.
// q0 = RN(x y) lies within 1.5 ulp of x / h, so RN(x / h) is q0 or one of
// its two neighbours: which one follows from comparing x / h with the
// midpoints next to q0, that is x = Mx 2^Ex with m h = (2 Mq +- 1) Mh
// 2^(Eq - 1 + Eh) (integer significands, products in 128 bits).  Below a
// power of two the lower neighbour is half an ulp away, so that midpoint is
// (4 Mq - 1) 2^(Eq - 2).  No midpoint can equal x / h exactly: Mh has an
// odd factor above 1 and 2 Mq +- 1 is odd and above 2^53, so their product
// is no 53-bit significand times a power of two.  One binary64 operation
// and integer arithmetic, against five binary64 operations for the
// corrections above (B300 runs binary64 at 1/64 of its binary32 rate).
__device__ __forceinline__ double quotient_rn_int(double x, double h, double y) {
    constexpr unsigned long long kMant = (1ull << 52) - 1ull, kHidden = 1ull << 52;
    const double q0 = x * y;
    const unsigned long long ux = (unsigned long long)__double_as_longlong(x);
    const unsigned long long uq = (unsigned long long)__double_as_longlong(q0);
    const unsigned long long uh = (unsigned long long)__double_as_longlong(h);
    const unsigned long long mx = (ux & kMant) | kHidden, mq = (uq & kMant) | kHidden;
    const unsigned long long mh = (uh & kMant) | kHidden;
    const int s = (int)(ux >> 52) - (int)(uq >> 52) - (int)(uh >> 52) + 1076;   // Ex - Eq - Eh + 1, in [52, 55]
    const unsigned long long xl = mx << s, xh = mx >> (64 - s);                  // x as Mx 2^s
    const unsigned long long a = 2ull * mq + 1ull;                                 // upper midpoint
    const unsigned long long pl = a * mh, ph = __umul64hi(a, mh);
    const bool up = xh > ph || (xh == ph && xl > pl);
    bool down;
    if (mq != kHidden) {                                                           // (2 Mq - 1) Mh = P - 2 Mh
        const unsigned long long d = 2ull * mh;
        const unsigned long long ll = pl - d, lh = ph - (pl < d ? 1ull : 0ull);
        down = xh < lh || (xh == lh && xl < ll);
    } else {                                                                       // q0 a power of two
        const unsigned long long b = 4ull * mq - 1ull;
        const unsigned long long ll = b * mh, lh = __umul64hi(b, mh);
        const unsigned long long yl = xl << 1, yh = (xh << 1) | (xl >> 63);
        down = yh < lh || (yh == lh && yl < ll);
    }
    return __longlong_as_double((long long)(uq + (up ? 1ull : 0ull) - (down ? 1ull : 0ull)));
}

__device__ __forceinline__ double quotient_rn(double x, double h, double y) {
    return x < 0x1p-900 ? x / h : quotient_rn_normal(x, h, y);
}

// The integer form of the binary64 steps for a spacing h that is not a
// power of two, as fine_axis_bits does for 2^-s: x in [0, box) checked on
// its bit pattern (x below 2^-900, x = 0 included, is left to the binary64
// code), t = x / h from quotient_rn, then floor(t) and t = mant 2^-F read
// off t's bits.  q is floor(t) before the clamp to M - 1 (t can round up to
// M for x just below box): the caller clamps the cell index, while the
// offset is taken from the unclamped t.  Returns false where the caller
// takes the binary64 code.
__device__ __forceinline__ bool fine_axis_quot(double x, unsigned long long ubox, double h, double y, int& q,
                                               unsigned long long& mant, int& F) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    if (u >= ubox || u < (123ull << 52)) return false;       // outside [2^-900, box)
    const double t = quotient_rn_int(x, h, y);
    const unsigned long long ut = (unsigned long long)__double_as_longlong(t);
    const int E = (int)(ut >> 52) - 1023;                     // t >= 0: sign bit clear
    if (E < 0) {                                              // t < 1 (zero or subnormal included)
        q = 0;
        mant = 0ull;
        F = -1;
        return true;
    }
    if (E > 52) return false;
    mant = (ut & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    F = 52 - E;
    q = (int)(mant >> F);
    return true;
}

// floor(x / h) alone (the cell and Morton code need nothing more), from
// one product t' = x y, y = RN(1/h), instead of the corrected quotient:
// t' carries two roundings of relative size 2^-53, so it lies within
// 2.5 ulp of RN(x / h), and floor(t') = floor(RN(x / h)) whenever t' is
// 16 ulps or more from every integer.  Returns false otherwise (and for
// whatever fine_axis_quot declines), and the caller takes the corrected
// quotient.
__device__ __forceinline__ bool fine_axis_floor(double x, unsigned long long ubox, double y, int& q) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    if (u >= ubox || u < (123ull << 52)) return false;       // outside [2^-900, box)
    const unsigned long long ut = (unsigned long long)__double_as_longlong(x * y);
    const int E = (int)(ut >> 52) - 1023;
    if (E < 0) {                                              // t' < 1
        if (ut >= 0x3FEFFFFFFFFFFFF0ull) return false;       // within 16 ulps of 1
        q = 0;
        return true;
    }
    if (E > 47) return false;
    const int F = 52 - E;
    const unsigned long long mant = (ut & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const unsigned long long frac = mant & ((1ull << F) - 1ull);
    if (frac < 16ull || frac > (1ull << F) - 16ull) return false;
    q = (int)(mant >> F);
    return true;
}

// Fine-grid coordinate of one axis; flags non-finite / out-of-range input.
__device__ __forceinline__ void fine_axis(double x, const VolDev& V, double& t, int& q, bool& bad) {
    const double box = V.box;
    const int M = V.M;
    if (!(x >= -box && x < 2.0 * box)) {  // also catches NaN
        bad = true;
        x = 0.0;
    }
    if (x < 0.0) x = x + box;
    if (x >= box) x = x - box;
    // x / h, correctly rounded; for h = 2^k the product with 2^-k is exact
    t = V.h_pow2 ? x * V.inv_h : quotient_rn(x, V.h, V.inv_h);
    int qq = (int)floor(t);
    if (qq > M - 1) qq = M - 1;
    if (qq < 0) qq = 0;
    q = qq;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

constexpr int kSmallCell = 128;                 // ranges sorted by one warp in registers (bitonic)
static_assert(kSmallCell <= 128, "a position in a small range takes 7 bits of the 32-bit sort key");
constexpr int kWarpSeg = 512;                   // ranges sorted by one warp in shared memory (LSD)
constexpr int kWarpRounds = kWarpSeg / 32;
constexpr int kSegTile = 2048;                  // elements a block-sort holds in shared memory
constexpr int kSegThreads = 256;                // one 8-bit digit per thread
constexpr int kSegWarps = kSegThreads / 32;
constexpr int kSegRounds = kSegTile / kSegThreads;
constexpr int kSegMaxPasses = 8;                // composites of up to 64 bits
constexpr int kTieRunMax = 32;                 // longest run of equal Morton codes fixed by one thread
// k_sort_segments' dynamic shared memory: two kWarpSeg halves per warp in
// the warp phase; kSegTile values and the pass histograms in the block phase
constexpr int kSortSmem = (int)sizeof(unsigned long long) * 2 * kSegWarps * kWarpSeg;
static_assert(sizeof(unsigned long long) * kSegTile + sizeof(int) * kSegMaxPasses * 256 <= (size_t)kSortSmem,
              "block phase fits in the warp phase's shared memory");
constexpr int kSplitThreads = 512;
constexpr int kSplitRounds = 8;                // elements per thread per round of k_split (loads in flight)
constexpr int kFillU1 = 2;                     // chunks per warp round of k_chunk_fill (32-slot chunks)
constexpr int kFillU2 = 2;                     // (64-slot chunks)
constexpr int kCellTile = kScanTile;            // cells per block of the cell scan
constexpr unsigned long long kLbAggregate = 1ull << 62;   // look-back word: the tile's own sums
constexpr unsigned long long kLbPrefix = 2ull << 62;      // look-back word: inclusive prefix
constexpr int kLbMaxSpins = 1 << 20;            // bound of one look-back wait

__device__ __forceinline__ int block_exclusive_scan256(int v, int* warp_tot) {
    // 256 threads, one value each; warp_tot: 8 ints of shared memory
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    int before = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) before += w < warp ? warp_tot[w] : 0;
    __syncthreads();
    return before + x - v;
}

// Bitonic sort of 32 S values held as v[s] at lane l (element l + 32 s),
// ascending.
template <int S, class T>
__device__ __forceinline__ void warp_bitonic(T (&v)[S]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32 * S; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int js = j >> 5;
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    if (s & js) continue;
                    const bool asc = ((lane + 32 * s) & k) == 0;
                    const T x = v[s], y = v[s | js];
                    if ((x > y) == asc) {
                        v[s] = y;
                        v[s | js] = x;
                    }
                }
            } else {
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const T y = __shfl_xor_sync(kFull, v[s], j);
                    const bool asc = ((lane + 32 * s) & k) == 0, lower = (lane & j) == 0;
                    const T lo = v[s] < y ? v[s] : y, hi = v[s] < y ? y : v[s];
                    v[s] = lower == asc ? lo : hi;
                }
            }
        }
    }
}

// The values of a range of at most kSmallCell (lane l: elements l + 32 s,
// ~0 past the end), loaded ahead of its sort; nothing for larger ranges.
__device__ __forceinline__ void load_small(const unsigned long long* src, int m, unsigned long long (&v)[4]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 0; s < 4; ++s) v[s] = m <= kSmallCell && lane + 32 * s < m ? src[lane + 32 * s] : ~0ull;
}

// Sorts the preloaded composites of a range of m <= 32 S values into dst:
// a bitonic sort of 32-bit keys (Morton code << 7 | position in the range:
// 3 b + 7 <= 31 bits) instead of the 64-bit composites, then each output
// takes its composite from the position in its key (S shuffles).  Equal
// Morton codes (particles in one fine cell) leave such a run ordered by
// position, not caller index; if the range has one, the gathered
// composites are sorted again in full.
template <int S>
__device__ __forceinline__ void warp_sort_store_s(const unsigned long long (&in)[4], unsigned long long* dst, int m,
                                                  int ib) {
    const int lane = threadIdx.x & 31;
    unsigned k[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int e = lane + 32 * s;
        k[s] = e < m ? ((unsigned)(in[s] >> ib) << 7) | (unsigned)e : 0xffffffffu;
    }
    warp_bitonic<S>(k);
    unsigned long long v[S];
    bool tie = false;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int p = (int)(k[s] & 127u);
        unsigned long long c = ~0ull;
#pragma unroll
        for (int t = 0; t < S; ++t) {
            const unsigned long long g = __shfl_sync(kFull, in[t], p & 31);
            if ((p >> 5) == t) c = g;
        }
        const int o = lane + 32 * s;
        v[s] = o < m ? c : ~0ull;
        const unsigned up = __shfl_up_sync(kFull, k[s], 1);
        const unsigned wrap = __shfl_sync(kFull, k[s > 0 ? s - 1 : 0], 31);
        const unsigned prev = lane > 0 ? up : wrap;
        tie = tie || (o < m && o > 0 && (prev >> 7) == (k[s] >> 7));
    }
    if (__any_sync(kFull, tie)) warp_bitonic<S>(v);
#pragma unroll
    for (int s = 0; s < S; ++s)
        if (lane + 32 * s < m) dst[lane + 32 * s] = v[s];
}

// Sorts the preloaded values of a range of m <= kSmallCell into dst.
__device__ __forceinline__ void warp_sort_store(const unsigned long long (&v)[4], unsigned long long* dst, int m,
                                                int ib) {
    if (m <= 32) warp_sort_store_s<1>(v, dst, m, ib);
    else if (m <= 64) warp_sort_store_s<2>(v, dst, m, ib);
    else warp_sort_store_s<4>(v, dst, m, ib);
}

// Shared-memory counters ctr[key] += 1 for every lane with ok, one atomic
// per distinct key of the warp; returns the counter's value before this
// lane's unit (lanes of one key in lane order).
__device__ __forceinline__ int warp_add(int* ctr, int key, bool ok) {
    const unsigned peers = __match_any_sync(kFull, ok ? key : -1);
    const int leader = __ffs(peers) - 1;
    int old = 0;
    if (ok && (threadIdx.x & 31) == leader) old = atomicAdd(ctr + key, __popc(peers));
    old = __shfl_sync(kFull, old, leader);
    return old + __popc(peers & lanemask_lt());
}

// Stable LSD passes of one warp over cur[0, m) (m <= kWarpSeg) on the 8-bit
// digits at shift0, shift0 + 8, ... (passes of them), through the other
// buffer nxt, with 256 counters in cnt; returns the buffer holding the
// result.  A pass ranks each value among the earlier ones of its digit (32
// at a time, lanes of one digit in lane order), scans the counts and
// scatters; passes whose digit is the same throughout are skipped.
__device__ unsigned long long* warp_lsd_passes(unsigned long long* cur, unsigned long long* nxt, int m, int shift0,
                                               int passes, int* cnt) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const int rounds = (m + 31) >> 5;
    for (int p = 0; p < passes; ++p) {
        const int shift = shift0 + 8 * p;
        for (int d = lane; d < 256; d += 32) cnt[d] = 0;
        __syncwarp();
        int rk[kWarpRounds];
#pragma unroll
        for (int r = 0; r < kWarpRounds; ++r) {
            rk[r] = 0;
            if (r < rounds) {
                const int e = r * 32 + lane;
                const bool ok = e < m;
                const int d = ok ? (int)((cur[e] >> shift) & 255ull) : 256;
                const unsigned peers = __match_any_sync(kFull, d);
                const int old = ok ? cnt[d] : 0;
                __syncwarp();
                if (ok && lane == __ffs(peers) - 1) cnt[d] = old + __popc(peers);
                __syncwarp();
                rk[r] = old + __popc(peers & lt);
            }
        }
        int loc[8], sum = 0;
        bool whole = false;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            loc[t] = cnt[8 * lane + t];
            sum += loc[t];
            whole = whole || loc[t] == m;
        }
        if (__any_sync(kFull, whole)) continue;          // one digit throughout: order kept
        int x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += t;
        }
        int run = x - sum;
        __syncwarp();
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            cnt[8 * lane + t] = run;
            run += loc[t];
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < kWarpRounds; ++r) {
            const int e = r * 32 + lane;
            if (r < rounds && e < m) {
                const unsigned long long v = cur[e];
                nxt[cnt[(int)((v >> shift) & 255ull)] + rk[r]] = v;
            }
        }
        __syncwarp();
        unsigned long long* t = cur;
        cur = nxt;
        nxt = t;
    }
    return cur;
}

// Length of the run of values equal to v[e] above bit ib (the Morton code
// of a composite) that starts at e, or 0 if e does not start one; lengths
// are counted up to kTieRunMax + 1.  Only the bits above ib are compared,
// and the tie fix permutes values only inside such runs, so the answer
// does not depend on fixes of other runs in progress.
__device__ __forceinline__ int tie_run_at(const unsigned long long* v, int e, int m, int ib) {
    const unsigned long long key = v[e] >> ib;
    if (e > 0 && (v[e - 1] >> ib) == key) return 0;
    int len = 1;
    while (e + len < m && len <= kTieRunMax && (v[e + len] >> ib) == key) ++len;
    return len;
}

// Insertion sort of v[0, len) (one thread; a run of equal Morton codes
// ordered by the whole composite, that is by caller index).
__device__ __forceinline__ void sort_run(unsigned long long* v, int len) {
    for (int i = 1; i < len; ++i) {
        const unsigned long long x = v[i];
        int j = i - 1;
        while (j >= 0 && v[j] > x) {
            v[j + 1] = v[j];
            --j;
        }
        v[j + 1] = x;
    }
}

// One warp sorts src[0, m) (m <= kWarpSeg) by the low `bits` bits into
// dst[0, m), in buf (2 kWarpSeg values) with 256 counters in cnt, all the
// warp's own shared memory.  The composites are (Morton << ib) | caller
// index: stable LSD passes on the Morton digits only (bits ib and up), then
// each run of equal Morton codes is put in caller-index order by one lane.
// A run longer than kTieRunMax (many particles in one fine cell) makes the
// warp sort the range on all `bits` bits instead.
__device__ void warp_lsd(const unsigned long long* src, unsigned long long* dst, int m, int bits, int ib,
                         unsigned long long* buf, int* cnt) {
    const int lane = threadIdx.x & 31;
    for (int e = lane; e < m; e += 32) buf[e] = src[e];
    __syncwarp();
    const int mpasses = bits > ib ? (bits - ib + 7) >> 3 : 0;
    unsigned long long* cur = warp_lsd_passes(buf, buf + kWarpSeg, m, ib, mpasses, cnt);
    bool long_run = false;
    for (int e = lane; e < m; e += 32) long_run = long_run || tie_run_at(cur, e, m, ib) > kTieRunMax;
    if (__any_sync(kFull, long_run)) {
        cur = warp_lsd_passes(cur, cur == buf ? buf + kWarpSeg : buf, m, 0, (bits + 7) >> 3, cnt);
    } else {
        for (int e = lane; e < m; e += 32) {
            const int len = tie_run_at(cur, e, m, ib);
            if (len > 1) sort_run(cur + e, len);
        }
        __syncwarp();
    }
    for (int e = lane; e < m; e += 32) dst[e] = cur[e];
}

// Cell and Morton code of every particle, and its place in its cell from
// the cell's count (warp-aggregated atomics: lanes of one cell take one
// atomic).
__global__ void __launch_bounds__(256) k_keys(const double* __restrict__ pos, int n,
                                              const VolDev* __restrict__ vols,
                                              const long long* __restrict__ part_start, int n_vol,
                                              int b, unsigned long long* __restrict__ keys,
                                              int* __restrict__ place, int* __restrict__ count,
                                              Counters* ctr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool ok = i < n;
    int cell = 0;
    unsigned long long m = 0ull;
    bool bad = false;
    if (ok) {
        const int v = n_vol > 1 ? volume_of_row(i, part_start, n_vol) : 0;
        const VolDev& V = vols[v];
        int q[3];
        const double x3[3] = {pos[3ll * i], pos[3ll * i + 1], pos[3ll * i + 2]};
        bool fast = true;
        {
            const unsigned long long ubox = (unsigned long long)__double_as_longlong(V.box);
            unsigned long long mant;
            int F;
            if (V.h_pow2) {
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) fast = fast && fine_axis_bits(x3[ax], ubox, V.inv_h_exp, q[ax], mant, F);
            } else {
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    fast = fast && fine_axis_floor(x3[ax], ubox, V.inv_h, q[ax]);
                    q[ax] = min(q[ax], V.M - 1);
                }
            }
        }
        if (!fast) {
            double t[3];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) fine_axis(x3[ax], V, t[ax], q[ax], bad);
        }
        const int mask = (1 << b) - 1;
        cell = V.cell_base + ((q[2] >> b) * V.n_c + (q[1] >> b)) * V.n_c + (q[0] >> b);
        m = spread3(q[0] & mask) | (spread3(q[1] & mask) << 1) | (spread3(q[2] & mask) << 2);
        ok = SR_BOUND(cell >= V.cell_base && cell < V.cell_base + V.n_c * V.n_c * V.n_c, &ctr->check,
                      kChkKeyCell);
    }
    const unsigned live = __ballot_sync(kFull, ok);
    if (!ok) return;
    const unsigned peers = __match_any_sync(live, cell);
    const int leader = __ffs(peers) - 1;
    int first = 0;
    if (lane == leader) first = atomicAdd(count + cell, __popc(peers));
    first = __shfl_sync(live, first, leader);
    keys[i] = ((unsigned long long)cell << (3 * b)) | m;
    place[i] = first + __popc(peers & lanemask_lt());
    if (bad) atomicOr((unsigned long long*)&ctr->err, 1ull);
}

// Cell starts and chunk starts from the counts (both exclusive scans, cell
// total_cells holding the totals), each chunk's record (cell, first sorted
// row, count, volume), and the lists of cells to sort by warp, by block or
// to split.  A tile of 2048 cells per block; the tile's
// prefix comes from the tiles before it by a decoupled look-back over
// words holding (flag, particle sum, chunk sum) in (2, 31, 31) bits.
__global__ void __launch_bounds__(kScanThreads) k_cell_scan(
    const int* __restrict__ count, int tc, int C, int* __restrict__ cell_start, int* __restrict__ ccs,
    int4* __restrict__ chunk_span, const int* __restrict__ vol_cell_base, int n_vol, long long max_chunks,
    int* __restrict__ huge, long long huge_cap,
    int4* __restrict__ wsegs, long long wseg_cap, int4* __restrict__ bsegs, long long bseg_cap, int sort_bits,
    BinCounters* bc, unsigned long long* status, long long* err, unsigned long long* check) {
    constexpr int kWarps = kScanThreads / 32;
    __shared__ int s_tile;
    __shared__ unsigned s_wa[kWarps], s_wb[kWarps];
    __shared__ unsigned s_pa, s_pb;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(&bc->tile, 1u);
    __syncthreads();
    const int tile = s_tile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long c0 = (long long)tile * kCellTile + (long long)threadIdx.x * kScanItems;
    int cnt[kScanItems];
    unsigned a = 0u, nb = 0u;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const long long c = c0 + k;
        cnt[k] = c < tc ? count[c] : 0;
        a += (unsigned)cnt[k];
        nb += (unsigned)((cnt[k] + C - 1) / C);
    }
    unsigned ia = a, ibn = nb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned ta = __shfl_up_sync(kFull, ia, o), tb = __shfl_up_sync(kFull, ibn, o);
        if (lane >= o) {
            ia += ta;
            ibn += tb;
        }
    }
    if (lane == 31) {
        s_wa[warp] = ia;
        s_wb[warp] = ibn;
    }
    __syncthreads();
    unsigned wa = 0u, wb = 0u, ta = 0u, tb = 0u;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        if (w < warp) {
            wa += s_wa[w];
            wb += s_wb[w];
        }
        ta += s_wa[w];
        tb += s_wb[w];
    }
    if (warp == 0) {
        unsigned long long pa = 0ull, pb = 0ull;
        const unsigned long long own = ((unsigned long long)ta << 31) | tb;
        if (tile == 0) {
            if (lane == 0) st_relaxed(status, kLbPrefix | own);
        } else {
            if (lane == 0) st_relaxed(status + tile, kLbAggregate | own);
            int j = tile - 1, spins = 0;
            while (true) {
                const int at = j - lane;
                const unsigned long long w = at >= 0 ? ld_relaxed(status + at) : kLbPrefix;
                const unsigned fl = (unsigned)(w >> 62);
                const unsigned pre = __ballot_sync(kFull, fl == 2u);
                const unsigned notr = __ballot_sync(kFull, fl == 0u);
                const int stop = pre ? __ffs(pre) - 1 : 31;             // lanes 0..stop are needed
                const unsigned need = stop == 31 ? kFull : ((2u << stop) - 1u);
                if (notr & need) {                                       // a needed tile has not published
                    if (++spins > kLbMaxSpins) {
                        if (lane == 0 && err) atomicOr((unsigned long long*)err, 2ull);
                        break;
                    }
                    __nanosleep(32);
                    continue;
                }
                const unsigned va = lane <= stop ? (unsigned)((w >> 31) & 0x7fffffffull) : 0u;
                const unsigned vb = lane <= stop ? (unsigned)(w & 0x7fffffffull) : 0u;
                pa += __reduce_add_sync(kFull, va);
                pb += __reduce_add_sync(kFull, vb);
                if (pre) break;
                j -= 32;
            }
            if (lane == 0) st_relaxed(status + tile, kLbPrefix | ((pa + ta) << 31) | (pb + tb));
        }
        if (lane == 0) {
            s_pa = (unsigned)pa;
            s_pb = (unsigned)pb;
        }
    }
    __syncthreads();
    unsigned ra = s_pa + wa + ia - a, rb = s_pb + wb + ibn - nb;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const long long c = c0 + k;
        if (c > tc) break;
        cell_start[c] = (int)ra;
        ccs[c] = (int)rb;
        if (c == tc) break;
        const int m = cnt[k], nch = (m + C - 1) / C;
        const int v = nch > 0 && n_vol > 1 ? volume_of_cell((int)c, vol_cell_base, n_vol) : 0;
        for (int j = 0; j < nch; ++j)
            if (SR_BOUND((long long)rb + j < max_chunks, check, kChkBinScan))
                chunk_span[rb + j] = make_int4((int)c, (int)ra + j * C, min(C, m - j * C), v);
        if (m > kSegTile) {
            const int h = atomicAdd(&bc->n_huge, 1);
            if (SR_BOUND(h < huge_cap, check, kChkBinScan)) huge[h] = (int)c;
        } else if (m > kWarpSeg) {
            const int s = atomicAdd(&bc->n_bseg, 1);
            if (SR_BOUND(s < bseg_cap, check, kChkBinScan)) bsegs[s] = make_int4((int)ra, m, 0, sort_bits);
        } else if (m > 1) {
            const int s = atomicAdd(&bc->n_wseg, 1);
            if (SR_BOUND(s < wseg_cap, check, kChkBinScan)) wsegs[s] = make_int4((int)ra, m, 0, sort_bits);
        }
        ra += (unsigned)m;
        rb += (unsigned)nch;
    }
}

// Each particle's composite (morton << ib) | caller index at its place in
// its cell's range.
__global__ void __launch_bounds__(256) k_scatter(const unsigned long long* __restrict__ keys,
                                                 const int* __restrict__ place, int n, int b, int ib,
                                                 const int* __restrict__ cell_start, int tc,
                                                 unsigned long long* __restrict__ comp, unsigned long long* check) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long k = keys[i];
    const long long cell = (long long)(k >> (3 * b));
    if (!SR_BOUND(cell < tc, check, kChkScatter)) return;
    const long long dest = (long long)cell_start[cell] + place[i];
    if (!SR_BOUND(dest >= 0 && dest < n, check, kChkScatter)) return;
    comp[dest] = ((k & ((1ull << (3 * b)) - 1ull)) << ib) | (unsigned long long)i;
}

// Huge cells, one block each (work queue): buckets on the composite's top 8
// bits (counted, then placed into scratch at the cell's offsets, both with
// warp-aggregated shared-memory atomics); buckets of more than one value
// are listed for k_sort_segments.  Bucket members share the top bits, so a
// bucket is sorted on the bits below them.
__global__ void __launch_bounds__(kSplitThreads) k_split(unsigned long long* __restrict__ comp,
                                                         unsigned long long* __restrict__ scratch,
                                                         const int* __restrict__ cell_start,
                                                         const int* __restrict__ huge, BinCounters* bc,
                                                         int4* __restrict__ wsegs, long long wseg_cap,
                                                         int4* __restrict__ bsegs, long long bseg_cap, int bits,
                                                         int n, unsigned long long* check) {
    __shared__ int hist[256], first[256], fill[256];
    __shared__ int warp_tot[8];
    __shared__ int s_item;
    const int top = bits > 8 ? bits - 8 : 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(&bc->next_huge, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= bc->n_huge) break;
        const int c = huge[item];
        const int base = cell_start[c], m = cell_start[c + 1] - base;
        const int mm = SR_BOUND(base >= 0 && m >= 0 && (long long)base + m <= n, check, kChkBinSort) ? m : 0;
        if (threadIdx.x < 256) hist[threadIdx.x] = 0;
        __syncthreads();
        for (int e0 = warp * 32 * kSplitRounds; e0 < mm; e0 += kSplitThreads * kSplitRounds) {
            unsigned long long v[kSplitRounds];          // the rounds' loads in flight together
#pragma unroll
            for (int r = 0; r < kSplitRounds; ++r) {
                const int e = e0 + 32 * r + lane;
                v[r] = e < mm ? comp[base + e] : 0ull;
            }
#pragma unroll
            for (int r = 0; r < kSplitRounds; ++r) {
                const int e = e0 + 32 * r + lane;
                warp_add(hist, (int)((v[r] >> top) & 255ull), e < mm);
            }
        }
        __syncthreads();
        // exclusive scan over the 256 buckets by the first 8 warps
        int ex = 0;
        if (threadIdx.x < 256) {
            const int h = hist[threadIdx.x];
            int x = h;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kFull, x, o);
                if (lane >= o) x += t;
            }
            if (lane == 31) warp_tot[warp] = x;
            ex = x - h;
        }
        __syncthreads();
        if (threadIdx.x < 256) {
            int before = 0;
#pragma unroll
            for (int w = 0; w < 8; ++w) before += w < warp ? warp_tot[w] : 0;
            first[threadIdx.x] = before + ex;
            fill[threadIdx.x] = before + ex;
        }
        __syncthreads();
        for (int e0 = warp * 32 * kSplitRounds; e0 < mm; e0 += kSplitThreads * kSplitRounds) {
            unsigned long long v[kSplitRounds];
#pragma unroll
            for (int r = 0; r < kSplitRounds; ++r) {
                const int e = e0 + 32 * r + lane;
                v[r] = e < mm ? comp[base + e] : 0ull;
            }
#pragma unroll
            for (int r = 0; r < kSplitRounds; ++r) {
                const int e = e0 + 32 * r + lane;
                const int at = warp_add(fill, (int)((v[r] >> top) & 255ull), e < mm);
                if (e < mm) scratch[base + at] = v[r];
            }
        }
        __syncthreads();
        // buckets: one value goes straight back, the rest are listed (a
        // bucket per thread of the first 8 warps)
        if (threadIdx.x < 256 && mm > 0) {
            const int sz = hist[threadIdx.x], o = base + first[threadIdx.x];
            if (sz == 1) {
                comp[o] = scratch[o];
            } else if (sz > 1 && sz <= kWarpSeg) {
                const int k = atomicAdd(&bc->n_wseg, 1);
                if (SR_BOUND(k < wseg_cap, check, kChkBinSort)) wsegs[k] = make_int4(o, sz, 1, top);
            } else if (sz > kWarpSeg) {
                const int k = atomicAdd(&bc->n_bseg, 1);
                if (SR_BOUND(k < bseg_cap, check, kChkBinSort)) bsegs[k] = make_int4(o, sz, 1, top);
            }
        }
        __syncthreads();
    }
}

// One stable LSD pass on the digit at `shift` of src[0, m) into dst (dst
// may be src when m <= kSegTile: every value is in registers before the
// first write).  run[d]: the digit's first destination, advanced past
// each tile.  Warp w takes a contiguous part of each tile, 32 at a time,
// so ties keep their order.
__device__ void seg_pass(const unsigned long long* src, unsigned long long* dst, int m, int shift, int* run,
                         int (*wh)[256], unsigned long long* check) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    for (int t0 = 0; t0 < m; t0 += kSegTile) {
        const int tm = min(kSegTile, m - t0);
        const int per = (tm + kSegThreads - 1) / kSegThreads * 32;     // elements per warp
        for (int i = threadIdx.x; i < kSegWarps * 256; i += kSegThreads) (&wh[0][0])[i] = 0;
        __syncthreads();
        unsigned long long v[kSegRounds];
        int dg[kSegRounds], rk[kSegRounds];
#pragma unroll
        for (int r = 0; r < kSegRounds; ++r) {
            v[r] = 0ull;
            dg[r] = 256;
            rk[r] = 0;
            if (r * 32 < per) {
                const int e = warp * per + r * 32 + lane;
                const bool ok = e < tm;
                if (ok) {
                    v[r] = src[t0 + e];
                    dg[r] = (int)((v[r] >> shift) & 255ull);
                }
                const unsigned peers = __match_any_sync(kFull, dg[r]);
                const int old = ok ? wh[warp][dg[r]] : 0;
                __syncwarp();
                if (ok && lane == __ffs(peers) - 1) wh[warp][dg[r]] = old + __popc(peers);
                __syncwarp();
                rk[r] = old + __popc(peers & lt);
            }
        }
        __syncthreads();
        {
            const int d = threadIdx.x;                 // one digit per thread
            int acc = run[d];
#pragma unroll
            for (int w = 0; w < kSegWarps; ++w) {
                const int t = wh[w][d];
                wh[w][d] = acc;
                acc += t;
            }
            run[d] = acc;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kSegRounds; ++r)
            if (dg[r] < 256) {
                const int at = wh[warp][dg[r]] + rk[r];
                if (SR_BOUND(at >= 0 && at < m, check, kChkBinSort)) dst[at] = v[r];
            }
        __syncthreads();
    }
}

// Stable LSD passes of the block over cur[0, mm) on the 8-bit digits at
// shift0, shift0 + 8, ... (passes of them; at most kSegMaxPasses).  In
// shared memory (in_smem, mm <= kSegTile) each pass goes back into cur;
// otherwise passes alternate between cur and alt.  Returns the buffer
// holding the result.  The digit counts of all passes come from one read;
// passes whose digit is the same for the whole range are skipped.
__device__ unsigned long long* block_lsd_passes(unsigned long long* cur, unsigned long long* alt, int mm, int shift0,
                                                int passes, bool in_smem, int (*hist)[256], int* run,
                                                int (*wh)[256], int* warp_tot, unsigned long long* check) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kSegMaxPasses * 256; i += kSegThreads) (&hist[0][0])[i] = 0;
    __syncthreads();
    for (int e0 = warp * 32; e0 < mm; e0 += kSegThreads) {
        const int e = e0 + lane;
        const bool in = e < mm;
        const unsigned long long v = in ? cur[e] : 0ull;
        for (int p = 0; p < passes; ++p) warp_add(hist[p], (int)((v >> (shift0 + 8 * p)) & 255ull), in);
    }
    __syncthreads();
    for (int p = 0; p < passes; ++p) {
        const int h = hist[p][threadIdx.x];
        if (__syncthreads_or(h == mm)) continue;             // one digit throughout: order kept
        run[threadIdx.x] = block_exclusive_scan256(h, warp_tot);
        __syncthreads();
        unsigned long long* dst = in_smem ? cur : alt;
        seg_pass(cur, dst, mm, shift0 + 8 * p, run, wh, check);
        if (!in_smem) {
            alt = cur;
            cur = dst;
        }
    }
    return cur;
}

// The listed ranges, sorted by the low `bits` bits into the composites
// array (from it, or from scratch where the split left a bucket).  PHASE 0,
// the warp list, one warp per range (dealt round robin): bitonic in
// registers up to kSmallCell, else warp_lsd in the warp's part of shared
// memory.  PHASE 1, the block list, one block per range: stable LSD passes
// on the Morton digits, in shared memory up to kSegTile values, else
// through the composites and scratch arrays in turn, then the runs of
// equal Morton codes in caller-index order (all bits for a range with a
// run longer than kTieRunMax); passes whose digit is the same for the
// whole range are skipped.
template <int PHASE>   // 0: the warp list, 1: the block list
__global__ void __launch_bounds__(kSegThreads, 3) k_sort_segments(unsigned long long* __restrict__ comp,
                                                               unsigned long long* __restrict__ scratch,
                                                               const int4* __restrict__ wsegs,
                                                               const int4* __restrict__ bsegs, BinCounters* bc,
                                                               int n, int ib, unsigned long long* check) {
    extern __shared__ unsigned long long sv[];   // see kSortSmem
    int (*hist)[256] = reinterpret_cast<int (*)[256]>(sv + kSegTile);   // block phase only
    __shared__ int wh[kSegWarps][256];
    __shared__ int run[256];
    __shared__ int warp_tot[8];
    __shared__ int s_item;
    const int warp = threadIdx.x >> 5;
    // warp list: items dealt round robin to the grid's warps; the entry two
    // items ahead and the values of the next small range are loaded while
    // the current range is sorted
    const int n_w = PHASE == 0 ? bc->n_wseg : 0, stride = gridDim.x * kSegWarps;
    auto entry = [&](int i) {
        int4 g = i < n_w ? wsegs[i] : make_int4(0, 0, 0, 0);
        if (!SR_BOUND(g.x >= 0 && g.y >= 0 && g.y <= kWarpSeg && (long long)g.x + g.y <= n && g.w >= 0 && g.w <= 64,
                      check, kChkBinSort))
            g = make_int4(0, 0, 0, 0);
        return g;
    };
    int item = blockIdx.x * kSegWarps + warp;
    int4 sg = entry(item), sn = entry(item + stride);
    unsigned long long pv[4];
    load_small((sg.z ? scratch : comp) + sg.x, sg.y, pv);
    while (item < n_w) {
        const int4 sn2 = entry(item + 2 * stride);
        unsigned long long nv[4];
        load_small((sn.z ? scratch : comp) + sn.x, sn.y, nv);
        if (sg.y <= kSmallCell) warp_sort_store(pv, comp + sg.x, sg.y, ib);
        else warp_lsd((sg.z ? scratch : comp) + sg.x, comp + sg.x, sg.y, sg.w, ib, sv + 2 * warp * kWarpSeg, wh[warp]);
        item += stride;
        sg = sn;
        sn = sn2;
#pragma unroll
        for (int t = 0; t < 4; ++t) pv[t] = nv[t];
    }
    if constexpr (PHASE == 1) {
        while (true) {
            // from the end of the list: the huge cells' buckets (appended
            // by k_split after the cell scan's ranges), the largest ranges,
            // start first
            if (threadIdx.x == 0) s_item = atomicAdd(&bc->next_bseg, 1);
            __syncthreads();
            const int taken = s_item;
            if (taken >= bc->n_bseg) break;
            const int4 sg = bsegs[bc->n_bseg - 1 - taken];
            const int off = sg.x, m = sg.y, bits = sg.w;
            const bool ok = SR_BOUND(off >= 0 && m >= 0 && (long long)off + m <= n && bits >= 0 && bits <= 64,
                                     check, kChkBinSort);
            const int mm = ok ? m : 0;
            unsigned long long* home = comp + off;
            unsigned long long* src = (sg.z ? scratch : comp) + off;
            const bool in_smem = mm <= kSegTile;
            unsigned long long* cur = in_smem ? sv : src;
            unsigned long long* alt = in_smem ? sv : (sg.z ? comp : scratch) + off;
            if (in_smem)
                for (int e = threadIdx.x; e < mm; e += kSegThreads) sv[e] = src[e];
            __syncthreads();
            // Morton digits first (stable), then runs of equal Morton codes in
            // caller-index order, as warp_lsd; a long run: all bits instead
            const int mpasses = bits > ib ? (bits - ib + 7) / 8 : 0;
            cur = block_lsd_passes(cur, alt, mm, ib, mpasses, in_smem, hist, run, wh, warp_tot, check);
            alt = in_smem ? sv : (cur == src ? (sg.z ? comp : scratch) + off : src);
            bool long_run = false;
            for (int e = threadIdx.x; e < mm; e += kSegThreads)
                long_run = long_run || tie_run_at(cur, e, mm, ib) > kTieRunMax;
            if (__syncthreads_or(long_run)) {
                cur = block_lsd_passes(cur, alt, mm, 0, (bits + 7) / 8, in_smem, hist, run, wh, warp_tot, check);
            } else {
                for (int e = threadIdx.x; e < mm; e += kSegThreads) {
                    const int len = tie_run_at(cur, e, mm, ib);
                    if (len > 1) sort_run(cur + e, len);
                }
                __syncthreads();
            }
            if (ok && cur != home)
                for (int e = threadIdx.x; e < mm; e += kSegThreads) home[e] = cur[e];
            __syncthreads();
        }
    }
}

// One chunk: slot offsets, indices and flags, anchor, bounding box and
// counts from the caller indices of its slots and their positions (lane l
// holds slots l + 32 s; x3 already loaded).
template <int K>
__device__ __forceinline__ void fill_chunk(
    long long k, int v, const int (&idx_in)[K], const bool (&valid_in)[K], const double (&x3)[K][3], int cnt,
    const VolDev* __restrict__ vols, float4* __restrict__ slot_pos, int* __restrict__ slot_idx,
    int4* __restrict__ chunk_meta, float4* __restrict__ chunk_lo, float4* __restrict__ chunk_hi,
    const unsigned char* __restrict__ active) {
    constexpr int C = 32 * K;
    const int lane = threadIdx.x & 31;
    const VolDev& V = vols[v];
    int orig[K], q[K][3], F[K][3];
    unsigned long long mant[K][3];
    double t[K][3];
    bool valid[K], fast[K];
    const unsigned long long ubox = (unsigned long long)__double_as_longlong(V.box);
#pragma unroll
    for (int s = 0; s < K; ++s) {
        valid[s] = valid_in[s];
        fast[s] = false;
        orig[s] = valid[s] ? idx_in[s] : -1;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) { q[s][ax] = 0; t[s][ax] = 0.0; F[s][ax] = -1; mant[s][ax] = 0ull; }
        if (valid[s]) {
            // the integer path needs t >= 1 on every axis for the offsets;
            // q holds the unclamped floor(t) there (the anchor is clamped)
            bool f = true;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax)
                f = f && (V.h_pow2 ? fine_axis_bits(x3[s][ax], ubox, V.inv_h_exp, q[s][ax], mant[s][ax], F[s][ax])
                                   : fine_axis_quot(x3[s][ax], ubox, V.h, V.inv_h, q[s][ax], mant[s][ax],
                                                    F[s][ax])) &&
                    F[s][ax] >= 0;
            fast[s] = f;
            if (!f) {
                bool bad = false;
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) fine_axis(x3[s][ax], V, t[s][ax], q[s][ax], bad);
            }
        }
    }
    int nact = 0;
#pragma unroll
    for (int s = 0; s < K; ++s) nact += __popc(__ballot_sync(kFull, valid[s] && (!active || active[orig[s]])));
    int qa[3];
    float bl[3], bh[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        qa[ax] = min(__shfl_sync(kFull, q[0][ax], 0), V.M - 1);   // slot 0 always exists
        bl[ax] = __int_as_float(0x7f800000);          // +inf
        bh[ax] = __int_as_float(0xff800000);          // -inf
    }
#pragma unroll
    for (int s = 0; s < K; ++s) {
        float off[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            off[ax] = !valid[s] ? kPad
                      : fast[s] ? offset_bits(mant[s][ax], F[s][ax], q[s][ax], qa[ax])
                                : __double2float_rn(t[s][ax] - (double)qa[ax]);
            if (valid[s]) {
                bl[ax] = fminf(bl[ax], off[ax]);
                bh[ax] = fmaxf(bh[ax], off[ax]);
            }
        }
        const long long slot = (long long)k * C + lane + 32 * s;
        const float w = !valid[s] ? 0.0f : (!active || active[orig[s]]) ? 1.0f : -1.0f;
        slot_pos[slot] = make_float4(off[0], off[1], off[2], w);
        slot_idx[slot] = orig[s];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            bl[ax] = fminf(bl[ax], __shfl_xor_sync(kFull, bl[ax], o));
            bh[ax] = fmaxf(bh[ax], __shfl_xor_sync(kFull, bh[ax], o));
        }
    }
    if (lane == 0) {
        chunk_meta[k] = make_int4(qa[0], qa[1], qa[2], v);
        chunk_lo[k] = make_float4(bl[0], bl[1], bl[2], __int_as_float(cnt));
        chunk_hi[k] = make_float4(bh[0], bh[1], bh[2], __int_as_float(nact));
    }
}

// One warp per group of U consecutive chunks: the caller indices of their
// slots from the sorted composites, then the chunks' slots and records;
// perm[sorted position] = caller index.  Each chunk's record (cell, first
// sorted row, count, volume) comes from the cell scan, so a chunk costs two
// dependent loads (composites, then positions); the U chunks' loads are
// issued together to keep more of them in flight.
template <int K, int U>
__global__ void __launch_bounds__(256, 3) k_chunk_fill(
    const double* __restrict__ pos, const unsigned long long* __restrict__ comp, int ib,
    const int4* __restrict__ chunk_span, const int* __restrict__ ccs, int total_cells,
    const VolDev* __restrict__ vols, int n_vol, float4* __restrict__ slot_pos, int* __restrict__ slot_idx,
    int4* __restrict__ chunk_meta, float4* __restrict__ chunk_lo, float4* __restrict__ chunk_hi,
    int* __restrict__ perm, const unsigned char* __restrict__ active, int n, long long max_chunks,
    unsigned long long* check) {
    [[maybe_unused]] constexpr int C = 32 * K;     // bounds checks only
    const int lane = threadIdx.x & 31;
    const int n_chunks = ccs[total_cells];
    const int warps = gridDim.x * (blockDim.x >> 5);
    const unsigned long long imask = (1ull << ib) - 1ull;
    for (int k0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * U; k0 < n_chunks; k0 += warps * U) {
        int4 sp[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k0 + u;
            sp[u] = make_int4(-1, 0, 0, 0);
            if (k < n_chunks && SR_BOUND(k < max_chunks, check, kChkChunkFill)) sp[u] = chunk_span[k];
            if (!SR_BOUND(sp[u].x < 0 || (sp[u].y >= 0 && sp[u].z > 0 && sp[u].z <= C &&
                                          (long long)sp[u].y + sp[u].z <= n && sp[u].w >= 0 && sp[u].w < n_vol),
                          check, kChkChunkFill))
                sp[u].x = -1;
        }
        int idx[U][K];
        bool valid[U][K];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int s = 0; s < K; ++s) {
                const int e = lane + 32 * s;
                valid[u][s] = sp[u].x >= 0 && e < sp[u].z;
                idx[u][s] = valid[u][s] ? (int)(comp[sp[u].y + e] & imask) : -1;
            }
        double x3[U][K][3];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int s = 0; s < K; ++s) {
                if (valid[u][s] && !SR_BOUND(idx[u][s] >= 0 && idx[u][s] < n, check, kChkChunkFill)) idx[u][s] = 0;
                const long long o = valid[u][s] ? 3ll * idx[u][s] : 0ll;
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) x3[u][s][ax] = valid[u][s] ? pos[o + ax] : 0.0;
            }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (sp[u].x < 0) continue;                   // warp-uniform
#pragma unroll
            for (int s = 0; s < K; ++s)
                if (valid[u][s]) perm[sp[u].y + lane + 32 * s] = idx[u][s];
            fill_chunk<K>(k0 + u, sp[u].w, idx[u], valid[u], x3[u], sp[u].z, vols, slot_pos, slot_idx, chunk_meta,
                          chunk_lo, chunk_hi, active);
        }
    }
}

}  // namespace

int bin_alloc(sr_plan* p) {
    BinScratch& B = p->bin;
    const long long tc = p->total_cells, cap = p->capacity;
    const long long tiles = (tc + 1 + kCellTile - 1) / kCellTile;
    const size_t off_status = 64, off_count = off_status + 8 * (size_t)tiles;
    B.clear_bytes = off_count + 4 * (size_t)(tc + 1);
    // list sizes: listed ranges are disjoint, each of at least 2 (warp list),
    // more than kWarpSeg (block list) or more than kSegTile (huge) elements
    B.huge_cap = cap / kSegTile + 1;
    B.bseg_cap = cap / kWarpSeg + 1;
    B.wseg_cap = cap / 2 + 1;
    cudaError_t e = cudaMalloc(&B.region, B.clear_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&B.huge, sizeof(int) * (size_t)B.huge_cap);
    if (e == cudaSuccess) e = cudaMalloc(&B.wsegs, sizeof(int4) * (size_t)B.wseg_cap);
    if (e == cudaSuccess) e = cudaMalloc(&B.bsegs, sizeof(int4) * (size_t)B.bseg_cap);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sort_segments<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSortSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sort_segments<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSortSmem);
    // one wave of resident blocks: every warp starts its share of the
    // round-robin warp list at once (a second wave would start late)
    for (int ph = 0; ph < 2 && e == cudaSuccess; ++ph) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, ph == 0 ? k_sort_segments<0> : k_sort_segments<1>, kSegThreads, kSortSmem);
        B.seg_blocks[ph] = (per_sm > 0 ? per_sm : 1) * p->sm_count;
    }
    if (e != cudaSuccess) return cuda_fail(e, "bin_alloc");
    char* r = static_cast<char*>(B.region);
    B.counters = reinterpret_cast<BinCounters*>(r);
    B.status = reinterpret_cast<unsigned long long*>(r + off_status);
    B.count = reinterpret_cast<int*>(r + off_count);
    return SR_OK;
}

void bin_free(sr_plan* p) {
    BinScratch& B = p->bin;
    cudaFree(B.region);
    cudaFree(B.huge);
    cudaFree(B.wsegs);
    cudaFree(B.bsegs);
    B = BinScratch{};
}

int launch_bin(sr_plan* p, const double* pos, long long n, cudaStream_t st, const unsigned char* active) {
    BinScratch& B = p->bin;
    const int b = p->sub_bits;
    const int ni = (int)n;
    const int tc = (int)p->total_cells;
    const int C = 32 * p->chunk_k;
    int ib = 1;                                   // bits of a caller index: n - 1 < 2^ib
    while ((1ll << ib) < n) ++ib;
    const int bits = 3 * b + ib;
    unsigned long long* check = &p->ctr->check;
    SR_CUDA_CHECK(cudaMemsetAsync(B.region, 0, B.clear_bytes, st));
    if (ni > 0) {
        k_keys<<<(ni + 255) / 256, 256, 0, st>>>(pos, ni, p->vols, p->vol_part_start, p->n_vol, b, p->keys[0],
                                                 p->vals[0], B.count, p->ctr);
        SR_LAUNCH_CHECK("k_keys");
    }
    const int tiles = (tc + 1 + kCellTile - 1) / kCellTile;
    k_cell_scan<<<tiles, kScanThreads, 0, st>>>(B.count, tc, C, p->cell_start, p->ccs, p->chunk_span, p->vol_cell_base,
                                                p->n_vol, p->max_chunks,
                                                B.huge, B.huge_cap, B.wsegs, B.wseg_cap, B.bsegs, B.bseg_cap, bits,
                                                B.counters, B.status,
                                                &p->ctr->err, check);
    SR_LAUNCH_CHECK("k_cell_scan");
    if (ni > 0) {
        k_scatter<<<(ni + 255) / 256, 256, 0, st>>>(p->keys[0], p->vals[0], ni, b, ib, p->cell_start, tc, p->keys[1],
                                                    check);
        SR_LAUNCH_CHECK("k_scatter");
        k_split<<<p->sm_count, kSplitThreads, 0, st>>>(p->keys[1], p->keys[0], p->cell_start, B.huge, B.counters,
                                                       B.wsegs, B.wseg_cap, B.bsegs, B.bseg_cap, bits, ni, check);
        SR_LAUNCH_CHECK("k_split");
        k_sort_segments<0><<<B.seg_blocks[0], kSegThreads, kSortSmem, st>>>(p->keys[1], p->keys[0], B.wsegs,
                                                                             B.bsegs, B.counters, ni, ib, check);
        SR_LAUNCH_CHECK("k_sort_segments<warp>");
        k_sort_segments<1><<<B.seg_blocks[1], kSegThreads, kSortSmem, st>>>(p->keys[1], p->keys[0], B.wsegs,
                                                                             B.bsegs, B.counters, ni, ib, check);
        SR_LAUNCH_CHECK("k_sort_segments<block>");
    }
    const int U = p->chunk_k == 2 ? kFillU2 : kFillU1;
    long long want = (p->max_chunks + 8 * U - 1) / (8 * U);
    long long cap = (long long)p->sm_count * 16;
    const int blocks = (int)(want < cap ? (want > 0 ? want : 1) : cap);
    if (p->chunk_k == 2)
        k_chunk_fill<2, kFillU2><<<blocks, 256, 0, st>>>(pos, p->keys[1], ib, p->chunk_span, p->ccs, tc, p->vols,
                                                         p->n_vol, p->slot_pos, p->slot_idx, p->chunk_meta,
                                                         p->chunk_lo, p->chunk_hi, p->vals[1], active, ni,
                                                         p->max_chunks, check);
    else
        k_chunk_fill<1, kFillU1><<<blocks, 256, 0, st>>>(pos, p->keys[1], ib, p->chunk_span, p->ccs, tc, p->vols,
                                                         p->n_vol, p->slot_pos, p->slot_idx, p->chunk_meta,
                                                         p->chunk_lo, p->chunk_hi, p->vals[1], active, ni,
                                                         p->max_chunks, check);
    SR_LAUNCH_CHECK("k_chunk_fill");
    p->sorted = 1;
    return launch_cost_and_order(p, st);
}

}  // namespace sr
