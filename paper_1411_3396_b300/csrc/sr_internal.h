// Internal declarations shared by the library's CUDA/C++ sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sr.h"

namespace sr {

constexpr int kMaxChunkK = 2;       // chunks hold 32 K particles, K = 1 or 2 (K per lane)

// Checks of the bounds-checked build (compiled with -DSR_CHECK): the code
// a failed check records in its error word.
enum CheckCode : int {
    kChkItem = 1,         // pair kernels: work item outside the chunk table
    kChkCell = 2,         // neighbour cell outside the cell table
    kChkChunk = 3,        // neighbour chunk outside the chunk table
    kChkRing = 4,         // pair kernel: staging ring over-filled
    kChkList = 5,         // flat enumeration: neighbour-chunk list over-filled
    kChkRow = 6,          // caller row of a slot outside [0, n)
    kChkGroupRing = 7,    // grouped kernel: staging or group ring over-filled
    kChkKeyCell = 8,      // binning: cell of a key outside the cell table
    kChkCellBounds = 9,   // binning: cell-start entry outside the cell table
    kChkChunkFill = 10,   // binning: sorted position, caller row or slot outside its array
    kChkScatter = 11,     // radix scatter: destination outside [0, n)
    kChkCenters = 12,     // center finder: slot or accumulator outside its halo's block
    kChkBinScan = 13,     // binning cell scan: chunk or list entry outside its table
    kChkBinSort = 14,     // binning: range to sort outside [0, n), or list over-filled
    kChkSelfTest = 99,    // sr_check_selftest
};

#ifdef __CUDACC__
#ifdef SR_CHECK
// A failed check records its code in *word (the first failure is kept) and
// yields false, so that the caller skips the access; nothing traps.
__device__ __forceinline__ bool check_bound(bool ok, unsigned long long* word, int code) {
    if (!ok && word) atomicCAS(word, 0ull, (unsigned long long)code);
    return ok;
}
#define SR_BOUND(cond, word, code) (sr::check_bound((cond), (word), (code)))
#else
// The release build evaluates nothing: the condition is not compiled.
#define SR_BOUND(cond, word, code) (true)
#endif
#endif
constexpr float kPad = 1.0e30f;     // coordinate of an empty slot: never within r_c

#ifdef __CUDACC__
// Integer forms of the exact binary64 steps that place a coordinate on a
// grid of spacing 2^-s (binning's fine grid, the PM mesh).  B300 runs
// binary64 arithmetic at a small fraction of its integer rate, and these
// few operations otherwise bound the kernels that use them.
//
// x in [0, box) (checked on its bit pattern: non-negative doubles order as
// their bits), so t = x * 2^s is exact and floor(t) can be read off the
// significand.  Returns false for anything else (negative or -0, >= box,
// NaN, inf), which the caller sends through its binary64 code.  On success:
// q = floor(t) and, when t >= 1, t = mant * 2^-F with F = 52 - E in
// [0, 52] (F = -1 when t < 1).
__device__ __forceinline__ bool fine_axis_bits(double x, unsigned long long ubox, int s, int& q,
                                               unsigned long long& mant, int& F) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    if (u >= ubox) return false;
    const int e = (int)(u >> 52);                 // biased exponent (sign bit clear)
    const int E = e - 1023 + s;                   // exponent of t
    if (e == 0 || E < 0) {                        // zero, subnormal x, or t < 1
        q = 0;
        mant = 0ull;
        F = -1;
        return true;
    }
    mant = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    if (E > 52) return false;                     // t >= 2^53: not a grid coordinate here
    F = 52 - E;
    q = (int)(mant >> F);
    return true;
}

// Round the positive integer a (< 2^63) to nb significant bits, to nearest
// with ties to even; the result keeps a's scale.  *msb is the position of the
// leading bit before and after (it moves up by one when the rounding carries).
__device__ __forceinline__ unsigned long long round_bits(unsigned long long a, int nb, int* msb) {
    const int sh = *msb - (nb - 1);
    if (sh <= 0) return a;
    unsigned long long m = a >> sh;
    const unsigned long long rem = a & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) {
        ++m;
        if (m == (1ull << nb)) {
            m >>= 1;
            ++*msb;
            return m << (sh + 1);
        }
    }
    return m << sh;
}

// binary32(binary64(t - qa)) for t = mant * 2^-F (F in [30, 52]), q =
// floor(t) and |q - qa| < 2^30: the difference held exactly as the integer
// d = (t - qa) 2^F, rounded to 53 significant bits (the binary64 subtraction)
// and then to 24 (the conversion), both to nearest even.
__device__ __forceinline__ float offset_bits(unsigned long long mant, int F, int q, int qa) {
    const unsigned long long frac = mant & ((1ull << F) - 1ull);
    const long long d = (long long)(q - qa) * (1ll << F) + (long long)frac;
    if (d == 0) return 0.0f;
    const unsigned int sgn = d < 0 ? 0x80000000u : 0u;
    unsigned long long a = d < 0 ? (unsigned long long)(-d) : (unsigned long long)d;
    int msb = 63 - __clzll((long long)a);
    a = round_bits(a, 53, &msb);
    a = round_bits(a, 24, &msb);
    const unsigned int m24 = (unsigned int)(msb >= 23 ? a >> (msb - 23) : a << (23 - msb));
    const int ex = msb - F + 127;                 // |t - qa| in [2^-52, 2^31): a normal binary32
    return __uint_as_float(sgn | ((unsigned int)ex << 23) | (m24 & 0x7FFFFFu));
}

// binary32 rounding (to nearest even) of the fraction t - floor(t), for
// t = mant * 2^-F, F in [0, 52]; the binary64 subtraction is exact.
__device__ __forceinline__ float fraction_bits(unsigned long long mant, int F) {
    unsigned long long a = F ? (mant & ((1ull << F) - 1ull)) : 0ull;
    if (a == 0ull) return 0.0f;
    int msb = 63 - __clzll((long long)a);
    a = round_bits(a, 24, &msb);
    const unsigned int m24 = (unsigned int)(msb >= 23 ? a >> (msb - 23) : a << (23 - msb));
    const int ex = msb - F + 127;                 // fraction in [2^-52, 1)
    return __uint_as_float(((unsigned int)ex << 23) | (m24 & 0x7FFFFFu));
}
#endif  // __CUDACC__

constexpr int kScanItems = 8;       // items per thread in scans / radix passes
constexpr int kScanThreads = 256;
constexpr int kScanTile = kScanItems * kScanThreads;
constexpr int kRadixBits = 8;
constexpr int kRadixBuckets = 1 << kRadixBits;
constexpr int kGroupedFirst = 15;   // force-kernel variants 0..14: one 32-lane i-group per chunk
constexpr int kGroupedVariants = 2; // 15, 16: several smaller i-groups per chunk (force_grp.cu)
constexpr int kVariants = kGroupedFirst + kGroupedVariants;

// Per-volume constants, device resident, read once per work item.
// Lengths inside kernels are in units of the fine grid h = L / (n_c 2^b).
struct VolDev {
    double box;          // L
    double h;            // fine cell side, L / M
    double inv_h;        // 1/h, used instead of a division when h is a power of two
    int h_pow2;          // 1 if h is an exact power of two (then x * inv_h == x / h)
    int inv_h_exp;       // s with inv_h = 2^s (when h_pow2)
    long long part_start;  // first caller row of the volume
    long long part_end;
    int n_c;             // cells per axis
    int M;               // fine cells per axis, n_c << sub_bits
    int cell_base;       // global id of the volume's first cell
    int sub_bits;
    float eps2u;         // binary32(eps^2 / h^2)
    float rc2u;          // binary32((r_c^2 + eps^2) / h^2): in-range iff s' < rc2u
    float rcm2u;         // culling radius^2 (r_c^2/h^2 with a relative margin)
    float rcm;           // its square root
    float scale_a;       // 1/h^2: unit sums -> accelerations
    float scale_g;       // 1/h^3: unit sums -> position cotangents
    float nq[6];         // -q(x) = sum nq[m] x^m, x = s' (units); f_u = r^3 - q(x)
    float ndq[5];        // -q'(x) = sum ndq[m] x^m
    float pad0;
};

// Device-side counters (one per plan).
struct Counters {
    long long queue;          // next work item of the persistent kernels
    long long err;            // bit 0: bad position seen by sr_bin
    unsigned long long cost_total;
    unsigned long long evals;         // counting variant: candidate (i, j) evaluations, valid i only
    unsigned long long lane_evals;    // counting variant: candidate evaluations x 32 lanes
    long long n_items;                // work items of the pair kernels: chunks holding an active particle
    unsigned long long check;         // bounds-checked build: code of the first failed check (0 = none)
    long long reserved;
};

// Work counters of one binning (bin.cu), cleared with the cell counts
// before each sr_bin.
struct BinCounters {
    unsigned tile;        // next tile of the cell scan
    int n_huge;           // cells listed for the split
    int n_wseg;           // ranges listed for a warp sort
    int n_bseg;           // ranges listed for a block sort
    int next_huge;        // work-queue positions
    int next_wseg;
    int next_bseg;
    int pad;
};

// Binning workspace: one region cleared per sr_bin (counters, the cell
// scan's look-back words, the per-cell counts) and the two work lists.
struct BinScratch {
    void* region = nullptr;
    size_t clear_bytes = 0;
    BinCounters* counters = nullptr;
    unsigned long long* status = nullptr;
    int* count = nullptr;                 // total_cells + 1
    int* huge = nullptr;                  // cells to split
    long long huge_cap = 0;
    int4* wsegs = nullptr;                // ranges to sort by warp: offset, size, source (1 = scratch), key bits
    long long wseg_cap = 0;
    int4* bsegs = nullptr;                // ranges to sort by block, same fields
    long long bseg_cap = 0;
    int seg_blocks[2] = {0, 0};           // resident blocks of the two segment-sort phases
};

struct ScanScratch {
    std::vector<int*> partials;   // one buffer per recursion level
    std::vector<int> sizes;
};

struct RadixScratch {
    void* region = nullptr;       // digit totals, tile counters, look-back words (radix.cu)
    size_t bytes = 0;
    int max_tiles = 0;
};

}  // namespace sr

struct sr_plan {
    int device = 0;
    int n_vol = 0;
    long long capacity = 0;
    long long n_binned = 0;
    bool binned = false;
    int sub_bits = 6;
    int chunk_k = 1;                       // particles per lane; chunk size = 32 * chunk_k
    int key_bits = 0;
    long long total_cells = 0;
    long long max_chunks = 0;
    double coef[6] = {0, 0, 0, 0, 0, 0};
    sr_params phys{};
    std::vector<sr::VolDev> vols_h;
    std::vector<long long> vol_n;

    // device workspace
    sr::VolDev* vols = nullptr;
    long long* vol_part_start = nullptr;   // n_vol + 1
    int* vol_cell_base = nullptr;          // n_vol + 1
    unsigned long long* keys[2] = {nullptr, nullptr};
    int* vals[2] = {nullptr, nullptr};
    int sorted = 0;                        // buffer index holding the sorted result
    int* cell_start = nullptr;             // total_cells + 1
    int* ccs = nullptr;                    // cell -> first chunk, total_cells + 1
    int4* chunk_span = nullptr;            // chunk -> cell, first sorted row, particle count, volume
    int4* chunk_meta = nullptr;            // anchor qx, qy, qz, volume
    float4* chunk_lo = nullptr;            // bbox min, w = count (int bits)
    float4* chunk_hi = nullptr;
    unsigned* cost = nullptr;
    unsigned long long* lpt_keys[2] = {nullptr, nullptr};
    int* lpt_vals[2] = {nullptr, nullptr};
    int* order = nullptr;                  // points into lpt_vals[sorted_lpt]
    float4* slot_pos = nullptr;
    int* slot_idx = nullptr;
    float4* slot_g = nullptr;
    sr::Counters* ctr = nullptr;
    double* inv_partials = nullptr;
    sr::RadixScratch rs_chunks;
    sr::BinScratch bin;

    // captured whole-step graph (sr_graph_capture)
    cudaGraphExec_t graph_exec = nullptr;
    long long graph_kernels = 0;       // library kernels in the captured graph

    // staging for sr_step_host
    double* h_pos_dev = nullptr;
    float* h_vel_dev = nullptr;
    float* h_acc_dev = nullptr;
    cudaStream_t h_side = nullptr;      // sr_step_host: velocity upload beside the binning
    cudaEvent_t h_fork = nullptr, h_join = nullptr;

    // staging for sr_step_host_submit: two sets used in turn, so that one
    // step's uploads run while the step before it computes
    double* q_pos[2] = {nullptr, nullptr};
    float* q_vel[2] = {nullptr, nullptr};
    float* q_acc[2] = {nullptr, nullptr};
    cudaStream_t q_up = nullptr, q_down = nullptr;    // host-to-device and device-to-host copies
    cudaEvent_t q_loaded[2] = {nullptr, nullptr};     // a set's uploads done
    cudaEvent_t q_computed[2] = {nullptr, nullptr};   // its step's force and kick done
    cudaEvent_t q_freed[2] = {nullptr, nullptr};      // its downloads done: the set may be refilled
    bool q_used[2] = {false, false};
    int q_next = 0;

    int sm_count = 0;
    int variant = 0;                       // pair-kernel variant (launch bounds), see force.cu
    int force_blocks = 0;
    int force_blocks_v[sr::kVariants] = {};
    int vjp_blocks = 0;
    int count_blocks = 0;
    int grp_count_blocks[sr::kGroupedVariants] = {};   // counting mode of the grouped variants
    int warps_per_block = 8;               // of the selected force variant
};

namespace sr {

// error handling ------------------------------------------------------------
int set_error(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
void note_launch(int k = 1);
#define SR_CUDA_CHECK(call)                                  \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) return sr::cuda_fail(_e, #call); \
    } while (0)
#define SR_LAUNCH_CHECK(what)                                \
    do {                                                     \
        sr::note_launch();                                   \
        cudaError_t _e = cudaGetLastError();                 \
        if (_e != cudaSuccess) return sr::cuda_fail(_e, what); \
    } while (0)

// host-side fit (fit.cpp)
int fit_poly(double rc, double sigma, double eps, int mode, double c[6]);

// scans and sorts (radix.cu)
int scan_alloc(ScanScratch& s, long long n);
void scan_free(ScanScratch& s);
int exclusive_scan(const int* in, int* out, int n, ScanScratch& s, cudaStream_t st);
int radix_alloc(RadixScratch& r, long long n);
void radix_free(RadixScratch& r);
// Sorts (keys[0], vals[0]) stably by the low key_bits bits; returns in *which
// the index (0/1) of the buffer pair that holds the result.
// A look-back wait that runs out sets bit 1 of *err (nullable).
int radix_sort_pairs(unsigned long long* keys[2], int* vals[2], int n, int key_bits,
                     RadixScratch& r, cudaStream_t st, int* which, unsigned long long* check = nullptr,
                     long long* err = nullptr);

// binning (bin.cu)
int bin_alloc(sr_plan* p);
void bin_free(sr_plan* p);
int launch_bin(sr_plan* p, const double* pos, long long n, cudaStream_t st,
               const unsigned char* active = nullptr);

// force, cost, order, vjp (force.cu)
int launch_cost_and_order(sr_plan* p, cudaStream_t st);
int launch_force(sr_plan* p, float* acc, unsigned long long* pairs, int* per_particle,
                 cudaStream_t st, float* vel = nullptr, float kdt = 0.f);
int launch_vjp(sr_plan* p, const float* g_acc, float* g_pos, float g_scale, int accumulate,
               cudaStream_t st);
int force_occupancy(sr_plan* p);
// grouped pair kernel (force_grp.cu), 32-particle chunks only
int grouped_occupancy(sr_plan* p, int* blocks, int* count_blocks);
int launch_force_grouped(sr_plan* p, float* acc, unsigned long long* pairs, int* per_particle,
                         cudaStream_t st, float* vel, float kdt);

// plain kernel (plain.cu)
int launch_force_plain(sr_plan* p, float* acc, cudaStream_t st);

// elementwise (kick.cu)
int launch_kick(long long n, const float* acc, float* vel, float dt, cudaStream_t st);
int launch_drift(sr_plan* p, double* pos, const float* vel, double dt, long long n,
                 cudaStream_t st);
int launch_invariants(long long n, const float* vel, const float* acc, double* out,
                      double* partials, cudaStream_t st);
constexpr int kInvBlocks = 1184;   // 8 * 148
int launch_check_selftest(sr_plan* p, cudaStream_t st);

}  // namespace sr
