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
//   key = (cell << 3b) | morton(sub);  stable sort by key (LSD radix)
//   chunks = runs of <= 32 consecutive particles inside a cell
//   anchor qA = q of the chunk's first particle, offset = binary32(t - qA)
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
    const double t = quotient_rn_normal(x, h, y);
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

__global__ void __launch_bounds__(256) k_keys(const double* __restrict__ pos, int n,
                                              const VolDev* __restrict__ vols,
                                              const long long* __restrict__ part_start, int n_vol,
                                              int b, unsigned long long* __restrict__ keys,
                                              int* __restrict__ vals, Counters* ctr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int v = n_vol > 1 ? volume_of_row(i, part_start, n_vol) : 0;
    const VolDev& V = vols[v];
    bool bad = false;
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
                fast = fast && fine_axis_quot(x3[ax], ubox, V.h, V.inv_h, q[ax], mant, F);
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
    const int cell = V.cell_base + ((q[2] >> b) * V.n_c + (q[1] >> b)) * V.n_c + (q[0] >> b);
    const unsigned long long m = spread3(q[0] & mask) | (spread3(q[1] & mask) << 1) |
                                 (spread3(q[2] & mask) << 2);
    if (!SR_BOUND(cell >= V.cell_base && cell < V.cell_base + V.n_c * V.n_c * V.n_c, &ctr->check, kChkKeyCell))
        return;
    keys[i] = ((unsigned long long)cell << (3 * b)) | m;
    vals[i] = i;
    if (bad) atomicOr((unsigned long long*)&ctr->err, 1ull);
}

__global__ void __launch_bounds__(256) k_cell_bounds(const unsigned long long* __restrict__ keys, int n,
                                                     int shift, int total_cells, int* __restrict__ cell_start,
                                                     unsigned long long* check) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > n) return;
    const int c_prev = p > 0 ? (int)(keys[p - 1] >> shift) : -1;
    const int c_cur = p < n ? (int)(keys[p] >> shift) : total_cells;
    if (!SR_BOUND(c_prev >= -1 && c_cur <= total_cells, check, kChkCellBounds)) return;
    for (int c = c_prev + 1; c <= c_cur; ++c) cell_start[c] = p;
}

__global__ void __launch_bounds__(256) k_cell_nch(const int* __restrict__ cell_start, int total_cells,
                                                  int chunk, int* __restrict__ nch) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > total_cells) return;
    nch[c] = c < total_cells ? (cell_start[c + 1] - cell_start[c] + chunk - 1) / chunk : 0;
}

// chunk -> cell map: thread per cell writes its chunk range.
__global__ void __launch_bounds__(256) k_chunk_cell(const int* __restrict__ ccs, int total_cells,
                                                    int* __restrict__ chunk_cell) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= total_cells) return;
    for (int k = ccs[c]; k < ccs[c + 1]; ++k) chunk_cell[k] = c;
}

// One warp per chunk of C = 32 K slots (lane l fills slots l + 32 s):
// slot positions / indices, anchor, bounding box.  active (caller order,
// nullable = every particle active) marks the particles whose forces are
// wanted: slot w = 1 (active), -1 (passive, a neighbour only) or 0 (empty);
// chunk_hi.w = the chunk's count of active particles (int bits).
template <int K>
__global__ void __launch_bounds__(256) k_chunk_fill(
    const double* __restrict__ pos, const int* __restrict__ perm, const int* __restrict__ cell_start,
    const int* __restrict__ ccs, const int* __restrict__ chunk_cell, int total_cells,
    const VolDev* __restrict__ vols, const int* __restrict__ vol_cell_base, int n_vol,
    float4* __restrict__ slot_pos, int* __restrict__ slot_idx, int4* __restrict__ chunk_meta,
    float4* __restrict__ chunk_lo, float4* __restrict__ chunk_hi, const unsigned char* __restrict__ active,
    int n, long long max_chunks, unsigned long long* check) {
    constexpr int C = 32 * K;
    const int lane = threadIdx.x & 31;
    const int n_chunks = ccs[total_cells];
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < n_chunks; k += warps) {
        const int cell = chunk_cell[k];
        if (!SR_BOUND(k < max_chunks && cell >= 0 && cell < total_cells, check, kChkChunkFill)) continue;
        const int r0 = (k - ccs[cell]) * C;
        const int n_cell = cell_start[cell + 1] - cell_start[cell];
        const int v = n_vol > 1 ? volume_of_cell(cell, vol_cell_base, n_vol) : 0;
        const VolDev& V = vols[v];
        int orig[K], q[K][3], F[K][3];
        unsigned long long mant[K][3];
        double t[K][3];
        bool valid[K], fast[K];
        const unsigned long long ubox = (unsigned long long)__double_as_longlong(V.box);
#pragma unroll
        for (int s = 0; s < K; ++s) {
            const int rank = r0 + lane + 32 * s;
            valid[s] = rank < n_cell;
            fast[s] = false;
            orig[s] = -1;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) { q[s][ax] = 0; t[s][ax] = 0.0; F[s][ax] = -1; mant[s][ax] = 0ull; }
            if (valid[s] && !SR_BOUND(cell_start[cell] + rank < n, check, kChkChunkFill)) valid[s] = false;
            if (valid[s]) {
                orig[s] = perm[cell_start[cell] + rank];
                if (!SR_BOUND(orig[s] >= 0 && orig[s] < n, check, kChkChunkFill)) orig[s] = 0;
                const double x3[3] = {pos[3ll * orig[s]], pos[3ll * orig[s] + 1], pos[3ll * orig[s] + 2]};
                // the integer path needs t >= 1 on every axis for the offsets;
                // q holds the unclamped floor(t) there (the anchor is clamped)
                bool f = true;
#pragma unroll
                for (int ax = 0; ax < 3; ++ax)
                    f = f && (V.h_pow2 ? fine_axis_bits(x3[ax], ubox, V.inv_h_exp, q[s][ax], mant[s][ax], F[s][ax])
                                       : fine_axis_quot(x3[ax], ubox, V.h, V.inv_h, q[s][ax], mant[s][ax],
                                                        F[s][ax])) &&
                        F[s][ax] >= 0;
                fast[s] = f;
                if (!f) {
                    bool bad = false;
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) fine_axis(x3[ax], V, t[s][ax], q[s][ax], bad);
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
            qa[ax] = min(__shfl_sync(kFull, q[0][ax], 0), V.M - 1);   // slot 0 (rank r0) always exists
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
            const int cnt = min(C, n_cell - r0);
            chunk_meta[k] = make_int4(qa[0], qa[1], qa[2], v);
            chunk_lo[k] = make_float4(bl[0], bl[1], bl[2], __int_as_float(cnt));
            chunk_hi[k] = make_float4(bh[0], bh[1], bh[2], __int_as_float(nact));
        }
    }
}

}  // namespace

int launch_bin(sr_plan* p, const double* pos, long long n, cudaStream_t st, const unsigned char* active) {
    const int b = p->sub_bits;
    const int ni = (int)n;
    if (ni > 0) {
        k_keys<<<(ni + 255) / 256, 256, 0, st>>>(pos, ni, p->vols, p->vol_part_start, p->n_vol, b,
                                                 p->keys[0], p->vals[0], p->ctr);
        SR_LAUNCH_CHECK("k_keys");
    }
    int which = 0;
    int rc = radix_sort_pairs(p->keys, p->vals, ni, p->key_bits, p->rs_particles, st, &which, &p->ctr->check,
                              &p->ctr->err);
    if (rc) return rc;
    p->sorted = which;
    const int tc = (int)p->total_cells;
    k_cell_bounds<<<(ni + 1 + 255) / 256, 256, 0, st>>>(p->keys[which], ni, 3 * b, tc, p->cell_start,
                                                        &p->ctr->check);
    SR_LAUNCH_CHECK("k_cell_bounds");
    k_cell_nch<<<(tc + 1 + 255) / 256, 256, 0, st>>>(p->cell_start, tc, 32 * p->chunk_k, p->cell_nch);
    SR_LAUNCH_CHECK("k_cell_nch");
    rc = exclusive_scan(p->cell_nch, p->ccs, tc + 1, p->scan_cells, st);
    if (rc) return rc;
    k_chunk_cell<<<(tc + 255) / 256, 256, 0, st>>>(p->ccs, tc, p->chunk_cell);
    SR_LAUNCH_CHECK("k_chunk_cell");
    long long want = (p->max_chunks + 7) / 8;
    long long cap = (long long)p->sm_count * 16;
    const int blocks = (int)(want < cap ? (want > 0 ? want : 1) : cap);
    if (p->chunk_k == 2)
        k_chunk_fill<2><<<blocks, 256, 0, st>>>(pos, p->vals[which], p->cell_start, p->ccs, p->chunk_cell, tc,
                                                p->vols, p->vol_cell_base, p->n_vol, p->slot_pos, p->slot_idx,
                                                p->chunk_meta, p->chunk_lo, p->chunk_hi, active, ni, p->max_chunks,
                                                &p->ctr->check);
    else
        k_chunk_fill<1><<<blocks, 256, 0, st>>>(pos, p->vals[which], p->cell_start, p->ccs, p->chunk_cell, tc,
                                                p->vols, p->vol_cell_base, p->n_vol, p->slot_pos, p->slot_idx,
                                                p->chunk_meta, p->chunk_lo, p->chunk_hi, active, ni, p->max_chunks,
                                                &p->ctr->check);
    SR_LAUNCH_CHECK("k_chunk_fill");
    return launch_cost_and_order(p, st);
}

}  // namespace sr
