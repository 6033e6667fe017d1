// Halo center finder: potential of every halo member and the most bound
// particle of each halo (Sec. 2.2: center at the potential minimum, from a
// direct pair sum over the halo's members).
//
//   phi_i = - sum_{j in halo(i), j != i} (|d_ij|^2 + eps^2)^(-1/2)
//
// Pipeline (all on the device, one stream, no host synchronisation):
//   1. keys = label (or n_halos for "no halo"), stable radix sort of
//      (key, caller index) -> members of each halo contiguous, in caller order;
//   2. per-halo first/last member, 32-member blocks, I-tiles of 4 blocks;
//      scans give each halo's first padded slot, its first tile row and
//      each row's first work item;
//   3. members written as binary32 offsets from the halo's first member
//      (binary64 minimum image), padded to whole blocks with far-away slots;
//   4. pair sums (one of two kernels), into 64-bit fixed-point accumulators;
//   5. phi scattered back to caller order; per-halo argmin.
//
// The symmetric kernel evaluates each unordered pair once and credits both
// members; its cost is one MUFU rsqrt per unordered pair, and the MUFU unit
// (16 results per clock per SM) bounds it.  A warp owns an I-tile of 128
// members (4 per lane) and streams 32-member J blocks through shared memory;
// arithmetic is packed (f32x2) over pairs of J members; the I side
// accumulates in registers, the J side is written per lane to a padded
// shared row and summed down the columns once per block.  The plain kernel
// gives each member one thread that sums over its whole halo (gather, two
// rsqrt per unordered pair).
#include "sr_internal.h"
#include "sr_centers.h"

#include <cmath>

namespace {

constexpr int kBlk = 32;               // members per block (one per lane)
constexpr int kTileRows = 4;           // blocks per I-tile (members per lane)
constexpr int kTile = kBlk * kTileRows;
constexpr int kJMax = 32;              // J blocks per work item
constexpr int kWarps = 8;              // warps per block of the pair kernels
constexpr int kThreads = kWarps * 32;
constexpr int kRedStride = 36;         // padded row of the J-side partial sums
constexpr unsigned kFull = 0xffffffffu;

struct CtrDev {
    unsigned long long queue;          // next work item of the symmetric kernel
    unsigned long long bad_labels;
    unsigned long long wide;
    unsigned long long members;        // labelled particles
    unsigned long long max_members;
    unsigned long long pairs;          // sum N_h (N_h - 1) / 2
    unsigned long long evaluated;      // unordered pair terms the symmetric kernel evaluates
    unsigned long long check;          // bounds-checked build: code of the first failed check
};

typedef unsigned long long f2;

__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ float rsqrt_mufu(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// 1/sqrt of both halves; +inf (a pad partner) gives +0.
__device__ __forceinline__ f2 f2_rsqrt(f2 s) {
    float a, b;
    f2_unpack(s, a, b);
    return f2_pack(rsqrt_mufu(a), rsqrt_mufu(b));
}

// binary32 partial sum -> fixed point with scale 2^S (exact power-of-two
// scaling; rounding only below the fixed-point resolution).
__device__ __forceinline__ long long to_fixed(float v, float scale) {
    return __float2ll_rn(v * scale);
}

// -- 1. keys ------------------------------------------------------------------
__global__ void k_ctr_reset(CtrDev* c, long long n) {
    c->queue = 0;
    c->bad_labels = 0;
    c->wide = 0;
    c->members = (unsigned long long)n;
    c->max_members = 0;
    c->pairs = 0;
    c->evaluated = 0;
    c->check = 0;
}

__global__ void k_ctr_keys(const int* __restrict__ labels, long long n, int nh,
                           unsigned long long* __restrict__ keys, int* __restrict__ vals, CtrDev* c) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = labels[i];
    const bool ok = l >= 0 && l < nh;
    if (!ok && l != -1) atomicAdd(&c->bad_labels, 1ull);
    keys[i] = ok ? (unsigned long long)l : (unsigned long long)nh;
    vals[i] = (int)i;
}

// -- 2. halo bounds, blocks, rows, items --------------------------------------
__global__ void k_ctr_bounds(const unsigned long long* __restrict__ keys, long long n, int nh,
                             int* __restrict__ start, int* __restrict__ end, CtrDev* c) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long k = keys[i];
    const unsigned long long prev = i > 0 ? keys[i - 1] : ~0ull;
    if (k < (unsigned long long)nh) {
        if (prev != k) start[k] = (int)i;
        if (i == n - 1 || keys[i + 1] != k) end[k] = (int)(i + 1);
    } else if (prev != k) {
        c->members = (unsigned long long)i;     // first unlabelled position
    }
}

// Per halo: blocks nb = ceil(N/32), tile rows ceil(nb/4); entry nh is the
// zero sentinel that makes the exclusive scans' last entry the total.
__global__ void k_ctr_halos(int nh, const int* __restrict__ start, const int* __restrict__ end,
                            int* __restrict__ nblk, int* __restrict__ nrow, CtrDev* c) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h > nh) return;
    if (h == nh) {
        nblk[h] = 0;
        nrow[h] = 0;
        return;
    }
    const int cnt = end[h] - start[h];
    const int nb = (cnt + kBlk - 1) / kBlk;
    nblk[h] = nb;
    nrow[h] = (nb + kTileRows - 1) / kTileRows;
    if (cnt > 0) {
        atomicMax(&c->max_members, (unsigned long long)cnt);
        atomicAdd(&c->pairs, (unsigned long long)cnt * (unsigned long long)(cnt - 1) / 2ull);
    }
}

// Row r = (halo h, I-tile t) covers J blocks [4t, nb): ceil((nb - 4t)/kJMax)
// items.  Rows past the total get 0 items so the scan's tail is the total.
__global__ void k_ctr_rows(int nh, int rows_cap, const int* __restrict__ row0,
                           const int* __restrict__ nblk, int2* __restrict__ row_tab,
                           int* __restrict__ row_nitem, CtrDev* c) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > rows_cap) return;
    const int rows = row0[nh];
    if (r >= rows) {
        row_nitem[r] = 0;
        return;
    }
    int lo = 0, hi = nh;                       // row0[lo] <= r < row0[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (row0[mid] <= r) lo = mid; else hi = mid;
    }
    const int t = r - row0[lo];
    const int rem = nblk[lo] - kTileRows * t;
    row_tab[r] = make_int2(lo, t);
    row_nitem[r] = (rem + kJMax - 1) / kJMax;
    atomicAdd(&c->evaluated, (unsigned long long)kTile * kBlk * (unsigned long long)rem);
}

// -- 3. member slots ------------------------------------------------------------
// Sorted member m of halo h goes to slot 32 pblk[h] + (m - start[h]) as its
// binary32 offset from the halo's first member.
__global__ void k_ctr_fill(const double* __restrict__ pos, const unsigned long long* __restrict__ keys,
                           const int* __restrict__ vals, int nh, const int* __restrict__ start,
                           const int* __restrict__ pblk, double box, float4* __restrict__ slot_pos,
                           int* __restrict__ slot_idx, CtrDev* c) {
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= (long long)c->members) return;
    const int h = (int)keys[m];
    const int s0 = start[h];
    const long long slot = (long long)pblk[h] * kBlk + (m - s0);
    const int i = vals[m];
    const int a = vals[s0];
    const double quarter = 0.25 * box;
    double d[3];
    bool wide = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double v = pos[3LL * i + k] - pos[3LL * a + k];
        v -= box * rint(v / box);
        wide |= !(fabs(v) <= quarter);
        d[k] = v;
    }
    if (wide) atomicAdd(&c->wide, 1ull);
    slot_pos[slot] = make_float4((float)d[0], (float)d[1], (float)d[2], 0.f);
    slot_idx[slot] = i;
}

// The unused tail slots of each halo's last block: far away, index -1.
__global__ void k_ctr_pad(int nh, const int* __restrict__ start, const int* __restrict__ end,
                          const int* __restrict__ pblk, const int* __restrict__ nblk,
                          float4* __restrict__ slot_pos, int* __restrict__ slot_idx) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long h = g / kBlk;
    const int lane = (int)(g % kBlk);
    if (h >= nh) return;
    const int cnt = end[h] - start[h];
    const int nb = nblk[h];
    if (nb == 0) return;
    const int r = (nb - 1) * kBlk + lane;
    if (r < cnt) return;
    const long long slot = (long long)pblk[h] * kBlk + r;
    slot_pos[slot] = make_float4(sr::kPad, sr::kPad, sr::kPad, 0.f);
    slot_idx[slot] = -1;
}

// Zero the accumulators of every member slot (pads are never read).
__global__ void k_ctr_zero(const unsigned long long* __restrict__ keys, const int* __restrict__ start,
                           const int* __restrict__ pblk, unsigned long long* __restrict__ psi,
                           const CtrDev* c) {
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= (long long)c->members) return;
    const int h = (int)keys[m];
    psi[(long long)pblk[h] * kBlk + (m - start[h])] = 0ull;
}

__global__ void k_ctr_queue_reset(CtrDev* c) { c->queue = 0; }

// -- 4a. symmetric pair kernel --------------------------------------------------
// Shared memory of one warp: the J block as three coordinate rows, and the
// J-side partial sums, one row of 32 per lane (row stride 36 floats: the
// 16-byte stores of each quarter warp and the column reads are both free of
// bank conflicts).
struct WarpSmem {
    float x[kBlk], y[kBlk], z[kBlk];
    float red[kBlk * kRedStride];
};

// J members k and k+1 against the lane's 4 I members.  Arithmetic is packed
// over the two J members: (x_k, x_k+1) - (x_i, x_i).  DIAG applies the
// triangle of the tile's own blocks: with dr = q - 4t, I row r keeps the
// whole block if r < dr, members k > lane if r == dr, nothing if r > dr.
template <bool DIAG>
__device__ __forceinline__ f2 pair_terms2(const WarpSmem& sm, int k, const f2 (&XI)[kTileRows],
                                          const f2 (&YI)[kTileRows], const f2 (&ZI)[kTileRows], f2 E2,
                                          f2 (&P)[kTileRows], int lane, int dr) {
    const float2 X = *reinterpret_cast<const float2*>(&sm.x[k]);
    const float2 Y = *reinterpret_cast<const float2*>(&sm.y[k]);
    const float2 Z = *reinterpret_cast<const float2*>(&sm.z[k]);
    const f2 XJ = f2_pack(X.x, X.y), YJ = f2_pack(Y.x, Y.y), ZJ = f2_pack(Z.x, Z.y);
    f2 J = 0ull;
#pragma unroll
    for (int r = 0; r < kTileRows; ++r) {
        const f2 DX = f2_sub(XJ, XI[r]), DY = f2_sub(YJ, YI[r]), DZ = f2_sub(ZJ, ZI[r]);
        const f2 S = f2_fma(DZ, DZ, f2_fma(DY, DY, f2_fma(DX, DX, E2)));
        f2 R = f2_rsqrt(S);
        if (DIAG) {
            const float m0 = (r < dr || (r == dr && k > lane)) ? 1.f : 0.f;
            const float m1 = (r < dr || (r == dr && k + 1 > lane)) ? 1.f : 0.f;
            R = f2_mul(R, f2_pack(m0, m1));
        }
        P[r] = f2_add(P[r], R);
        J = r == 0 ? R : f2_add(J, R);
    }
    return J;
}

template <bool DIAG>
__device__ __forceinline__ void block_terms(WarpSmem& sm, const f2 (&XI)[kTileRows], const f2 (&YI)[kTileRows],
                                            const f2 (&ZI)[kTileRows], f2 E2, f2 (&P)[kTileRows], int lane,
                                            int dr) {
    // J pairs stay in registers until the block is done: stores into shared
    // memory between the loads of the J rows would order every later load
    // behind them
    f2 Jb[kBlk / 2];
#pragma unroll
    for (int k = 0; k < kBlk; k += 2) Jb[k >> 1] = pair_terms2<DIAG>(sm, k, XI, YI, ZI, E2, P, lane, dr);
    ulonglong2* row = reinterpret_cast<ulonglong2*>(&sm.red[lane * kRedStride]);
#pragma unroll
    for (int m = 0; m < kBlk / 4; ++m) row[m] = make_ulonglong2(Jb[2 * m], Jb[2 * m + 1]);
}

__global__ void __launch_bounds__(kThreads, 2)
k_ctr_pairs(const float4* __restrict__ slot_pos, unsigned long long* __restrict__ psi,
            const int2* __restrict__ row_tab, const int* __restrict__ row_item0,
            const int* __restrict__ row0, const int* __restrict__ pblk, const int* __restrict__ nblk,
            const int* __restrict__ start, const int* __restrict__ end, int nh, float eps2,
            float scale, CtrDev* c, long long slot_max) {
    __shared__ WarpSmem smem[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem& sm = smem[warp];
    const int n_rows = row0[nh];
    const int n_items = row_item0[n_rows];
    const f2 E2 = f2_pack(eps2, eps2);

    while (true) {
        int item = 0;
        if (lane == 0) item = (int)atomicAdd(&c->queue, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= n_items) break;
        // row of the item: 32-way search, row_item0[lo] <= item < row_item0[hi]
        int lo = 0, hi = n_rows;
        while (hi - lo > 1) {
            const int stride = (hi - lo + kBlk - 1) / kBlk;
            const int probe = lo + lane * stride;
            const bool le = probe < hi && row_item0[probe] <= item;
            const unsigned bal = __ballot_sync(kFull, le);
            const int L = 31 - __clz(bal);
            lo = lo + L * stride;
            hi = min(hi, lo + stride);
        }
        const int2 rt = row_tab[lo];
        const int h = rt.x, t = rt.y;
        const int nb = nblk[h];
        const int cnt = end[h] - start[h];
        const long long base = (long long)pblk[h] * kBlk;
        const int q0 = kTileRows * t + (item - row_item0[lo]) * kJMax;
        const int q1 = min(q0 + kJMax, nb);
        // the halo's blocks lie inside the slot arrays, and its members inside its blocks
        if (!SR_BOUND(base >= 0 && base + (long long)nb * kBlk <= slot_max && cnt <= nb * kBlk && q0 < nb,
                      &c->check, sr::kChkCenters))
            continue;

        f2 XI[kTileRows], YI[kTileRows], ZI[kTileRows], P[kTileRows];
        long long acc[kTileRows];
#pragma unroll
        for (int r = 0; r < kTileRows; ++r) {
            const int b = kTileRows * t + r;
            float4 v = make_float4(sr::kPad, sr::kPad, sr::kPad, 0.f);
            if (b < nb) v = slot_pos[base + (long long)b * kBlk + lane];
            XI[r] = f2_pack(v.x, v.x);
            YI[r] = f2_pack(v.y, v.y);
            ZI[r] = f2_pack(v.z, v.z);
            acc[r] = 0;
        }

        float4 nxt = slot_pos[base + (long long)q0 * kBlk + lane];
        for (int q = q0; q < q1; ++q) {
            const float4 pj = nxt;
            if (q + 1 < q1) nxt = slot_pos[base + (long long)(q + 1) * kBlk + lane];
            __syncwarp();
            sm.x[lane] = pj.x;
            sm.y[lane] = pj.y;
            sm.z[lane] = pj.z;
            __syncwarp();
#pragma unroll
            for (int r = 0; r < kTileRows; ++r) P[r] = 0ull;
            const int dr = q - kTileRows * t;
            if (dr < kTileRows)
                block_terms<true>(sm, XI, YI, ZI, E2, P, lane, dr);
            else
                block_terms<false>(sm, XI, YI, ZI, E2, P, lane, dr);
            // I side: this block's partials into the fixed-point registers
#pragma unroll
            for (int r = 0; r < kTileRows; ++r) {
                float lo2, hi2;
                f2_unpack(P[r], lo2, hi2);
                acc[r] += to_fixed(lo2 + hi2, scale);
            }
            // J side: lane k sums column k of the warp's partial rows
            __syncwarp();
            float col = 0.f;
#pragma unroll
            for (int l = 0; l < kBlk; ++l) col += sm.red[l * kRedStride + lane];
            const int jm = q * kBlk + lane;
            if (jm < cnt) atomicAdd(&psi[base + jm], (unsigned long long)to_fixed(col, scale));
        }
#pragma unroll
        for (int r = 0; r < kTileRows; ++r) {
            const int im = (kTileRows * t + r) * kBlk + lane;
            if (im < cnt) atomicAdd(&psi[base + im], (unsigned long long)acc[r]);
        }
    }
}

// -- 4b. plain pair kernel --------------------------------------------------------
// Thread per member: sum over every other member of its halo (broadcast
// loads from global memory), binary32 partials of 32 terms into fixed point.
__global__ void __launch_bounds__(256)
k_ctr_plain(const float4* __restrict__ slot_pos, unsigned long long* __restrict__ psi,
            const unsigned long long* __restrict__ keys, const int* __restrict__ start,
            const int* __restrict__ end, const int* __restrict__ pblk, float eps2, float scale,
            const CtrDev* c) {
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= (long long)c->members) return;
    const int h = (int)keys[m];
    const int s0 = start[h], cnt = end[h] - s0;
    const long long base = (long long)pblk[h] * kBlk;
    const int me = (int)(m - s0);
    const float4 xi = slot_pos[base + me];
    long long acc = 0;
    for (int j0 = 0; j0 < cnt; j0 += kBlk) {
        const int j1 = min(j0 + kBlk, cnt);
        float part = 0.f;
        for (int j = j0; j < j1; ++j) {
            const float4 xj = slot_pos[base + j];
            const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
            const float s = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
            part += j != me ? rsqrt_mufu(s) : 0.f;
        }
        acc += to_fixed(part, scale);
    }
    psi[base + me] = (unsigned long long)acc;
}

// -- 5. outputs ------------------------------------------------------------------
__global__ void k_ctr_phi(const unsigned long long* __restrict__ keys, const int* __restrict__ vals,
                          const int* __restrict__ start, const int* __restrict__ pblk,
                          const unsigned long long* __restrict__ psi, double inv_scale,
                          double* __restrict__ phi, const CtrDev* c) {
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= (long long)c->members) return;
    const int h = (int)keys[m];
    const long long slot = (long long)pblk[h] * kBlk + (m - start[h]);
    phi[vals[m]] = -(double)(long long)psi[slot] * inv_scale;
}

// Block per halo (grid-stride): largest fixed-point sum, ties to the smaller
// caller index.
__global__ void __launch_bounds__(256)
k_ctr_argmin(int nh, const int* __restrict__ start, const int* __restrict__ end,
             const int* __restrict__ pblk, const unsigned long long* __restrict__ psi,
             const int* __restrict__ slot_idx, double inv_scale, long long* __restrict__ center,
             double* __restrict__ center_phi) {
    __shared__ long long sv[8];
    __shared__ int si[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int h = blockIdx.x; h < nh; h += gridDim.x) {
        const int cnt = end[h] - start[h];
        const long long base = (long long)pblk[h] * kBlk;
        long long bv = -1;
        int bi = 0x7fffffff;
        for (int m = threadIdx.x; m < cnt; m += blockDim.x) {
            const long long v = (long long)psi[base + m];
            const int i = slot_idx[base + m];
            if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long ov = __shfl_xor_sync(kFull, bv, o);
            const int oi = __shfl_xor_sync(kFull, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if (lane == 0) { sv[warp] = bv; si[warp] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (sv[w] > bv || (sv[w] == bv && si[w] < bi)) { bv = sv[w]; bi = si[w]; }
            if (center) center[h] = cnt > 0 ? (long long)bi : -1LL;
            if (center_phi) center_phi[h] = cnt > 0 ? -(double)bv * inv_scale : (double)INFINITY;
        }
        __syncthreads();
    }
}

inline unsigned grid_for(long long n, int threads) {
    return (unsigned)((n + threads - 1) / threads);
}

}  // namespace

struct sr_centers {
    long long n_max = 0;
    int nh_max = 0;
    long long slot_max = 0;
    int rows_cap = 0;
    unsigned long long* keys[2] = {nullptr, nullptr};
    int* vals[2] = {nullptr, nullptr};
    int sorted = 0;
    sr::RadixScratch rs;
    sr::ScanScratch scan_h;
    sr::ScanScratch scan_r;
    int* start = nullptr;
    int* end = nullptr;
    int* nblk = nullptr;
    int* pblk = nullptr;
    int* nrow = nullptr;
    int* row0 = nullptr;
    int2* row_tab = nullptr;
    int* row_nitem = nullptr;
    int* row_item0 = nullptr;
    float4* slot_pos = nullptr;
    int* slot_idx = nullptr;
    unsigned long long* psi = nullptr;
    CtrDev* ctr = nullptr;
    int variant = SR_CENTERS_SYMMETRIC;
    int pair_blocks = 0;
    int fixed_shift = 0;
    float eps2 = 0.f;
    bool prepared = false;                 // sr_centers_prepare done
    bool psi_valid = false;                // sr_centers_potential done since
    long long last_n = 0;
    int last_nh = 0;
    cudaStream_t last_stream = nullptr;
};

namespace {

int centers_free(sr_centers* c) {
    for (int k = 0; k < 2; ++k) {
        cudaFree(c->keys[k]);
        cudaFree(c->vals[k]);
    }
    sr::radix_free(c->rs);
    sr::scan_free(c->scan_h);
    sr::scan_free(c->scan_r);
    void* bufs[] = {c->start, c->end, c->nblk, c->pblk, c->nrow, c->row0, c->row_tab,
                    c->row_nitem, c->row_item0, c->slot_pos, c->slot_idx, c->psi, c->ctr};
    for (void* p : bufs) cudaFree(p);
    delete c;
    return SR_OK;
}

template <class T>
int dalloc(T** p, long long count, const char* what) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)(count > 0 ? count : 1));
    if (e != cudaSuccess) return sr::cuda_fail(e, what);
    return SR_OK;
}

// Largest S with (n - 1)/eps * 2^S < 2^61: no fixed-point sum can overflow.
int fixed_shift_for(long long n, double eps) {
    const double bound = (double)(n > 1 ? n - 1 : 1) / eps;
    int s = (int)std::floor(61.0 - std::log2(bound));
    if (s > 52) s = 52;
    if (s < 0) s = 0;
    return s;
}

}  // namespace

extern "C" {

int sr_centers_create(int64_t n_max, int32_t n_halos_max, sr_centers** out) {
    if (!out) return sr::set_error(SR_ERR_ARG, "sr_centers_create: null out");
    *out = nullptr;
    if (n_max < 1 || n_max > (1LL << 30))
        return sr::set_error(SR_ERR_ARG, "sr_centers_create: n_max must be in [1, 2^30]");
    if (n_halos_max < 1 || n_halos_max > (1 << 26))
        return sr::set_error(SR_ERR_ARG, "sr_centers_create: n_halos_max must be in [1, 2^26]");
    sr_centers* c = new sr_centers();
    c->n_max = n_max;
    c->nh_max = n_halos_max;
    // blocks: sum ceil(N_h/32) <= n/32 + n_h; rows: sum ceil(nb/4) <= blocks/4 + n_h
    const long long blocks_cap = n_max / kBlk + n_halos_max;
    c->slot_max = blocks_cap * kBlk;
    c->rows_cap = (int)(blocks_cap / kTileRows + n_halos_max + 1);
    int rc = SR_OK;
    for (int k = 0; k < 2 && !rc; ++k) {
        rc = dalloc(&c->keys[k], n_max, "sr_centers_create keys");
        if (!rc) rc = dalloc(&c->vals[k], n_max, "sr_centers_create vals");
    }
    if (!rc) rc = sr::radix_alloc(c->rs, n_max);
    if (!rc) rc = sr::scan_alloc(c->scan_h, (long long)n_halos_max + 1);
    if (!rc) rc = sr::scan_alloc(c->scan_r, (long long)c->rows_cap + 1);
    const long long hn = (long long)n_halos_max + 1;
    if (!rc) rc = dalloc(&c->start, hn, "sr_centers_create start");
    if (!rc) rc = dalloc(&c->end, hn, "sr_centers_create end");
    if (!rc) rc = dalloc(&c->nblk, hn, "sr_centers_create nblk");
    if (!rc) rc = dalloc(&c->pblk, hn, "sr_centers_create pblk");
    if (!rc) rc = dalloc(&c->nrow, hn, "sr_centers_create nrow");
    if (!rc) rc = dalloc(&c->row0, hn, "sr_centers_create row0");
    if (!rc) rc = dalloc(&c->row_tab, (long long)c->rows_cap + 1, "sr_centers_create row_tab");
    if (!rc) rc = dalloc(&c->row_nitem, (long long)c->rows_cap + 1, "sr_centers_create row_nitem");
    if (!rc) rc = dalloc(&c->row_item0, (long long)c->rows_cap + 1, "sr_centers_create row_item0");
    if (!rc) rc = dalloc(&c->slot_pos, c->slot_max, "sr_centers_create slot_pos");
    if (!rc) rc = dalloc(&c->slot_idx, c->slot_max, "sr_centers_create slot_idx");
    if (!rc) rc = dalloc(&c->psi, c->slot_max, "sr_centers_create psi");
    if (!rc) rc = dalloc(&c->ctr, 1, "sr_centers_create ctr");
    if (!rc) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ctr_pairs, kThreads, 0);
        if (e != cudaSuccess) rc = sr::cuda_fail(e, "sr_centers_create occupancy");
        c->pair_blocks = sms * (per_sm > 0 ? per_sm : 1);
    }
    if (rc) {
        centers_free(c);
        return rc;
    }
    *out = c;
    return SR_OK;
}

int sr_centers_destroy(sr_centers* c) {
    if (!c) return SR_OK;
    return centers_free(c);
}

int sr_centers_set_variant(sr_centers* c, int variant) {
    if (!c) return sr::set_error(SR_ERR_ARG, "sr_centers_set_variant: null workspace");
    if (variant != SR_CENTERS_SYMMETRIC && variant != SR_CENTERS_PLAIN)
        return sr::set_error(SR_ERR_ARG, "sr_centers_set_variant: unknown variant");
    c->variant = variant;
    return SR_OK;
}

int sr_centers_prepare(sr_centers* c, const double* pos, const int32_t* labels, int64_t n,
                       int32_t n_halos, double box, double eps, void* stream) {
    if (!c || (!pos && n > 0) || (!labels && n > 0))
        return sr::set_error(SR_ERR_ARG, "sr_centers_prepare: null workspace, pos or labels");
    if (n < 0 || n_halos < 0) return sr::set_error(SR_ERR_ARG, "sr_centers_prepare: negative size");
    if (!(box > 0.0) || !std::isfinite(box) || !(eps > 0.0) || !std::isfinite(eps))
        return sr::set_error(SR_ERR_ARG, "sr_centers_prepare: box and eps must be finite and > 0");
    if (n > c->n_max || n_halos > c->nh_max)
        return sr::set_error(SR_ERR_CAPACITY, "sr_centers_prepare: n or n_halos above the workspace maxima");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nh = n_halos;
    const int T = 256;
    c->prepared = false;

    k_ctr_reset<<<1, 1, 0, st>>>(c->ctr, (long long)n);
    SR_LAUNCH_CHECK("k_ctr_reset");
    if (nh > 0) {
        SR_CUDA_CHECK(cudaMemsetAsync(c->start, 0, sizeof(int) * (size_t)nh, st));
        SR_CUDA_CHECK(cudaMemsetAsync(c->end, 0, sizeof(int) * (size_t)nh, st));
    }
    if (n > 0) {
        k_ctr_keys<<<grid_for(n, T), T, 0, st>>>(labels, (long long)n, nh, c->keys[0], c->vals[0], c->ctr);
        SR_LAUNCH_CHECK("k_ctr_keys");
        int key_bits = 1;
        while ((1LL << key_bits) <= (long long)nh) ++key_bits;
        int rc = sr::radix_sort_pairs(c->keys, c->vals, (int)n, key_bits, c->rs, st, &c->sorted);
        if (rc) return rc;
        k_ctr_bounds<<<grid_for(n, T), T, 0, st>>>(c->keys[c->sorted], (long long)n, nh, c->start,
                                                   c->end, c->ctr);
        SR_LAUNCH_CHECK("k_ctr_bounds");
    }
    const unsigned long long* keys = c->keys[c->sorted];
    const int* vals = c->vals[c->sorted];
    k_ctr_halos<<<grid_for((long long)nh + 1, T), T, 0, st>>>(nh, c->start, c->end, c->nblk, c->nrow, c->ctr);
    SR_LAUNCH_CHECK("k_ctr_halos");
    int rc = sr::exclusive_scan(c->nblk, c->pblk, nh + 1, c->scan_h, st);
    if (!rc) rc = sr::exclusive_scan(c->nrow, c->row0, nh + 1, c->scan_h, st);
    if (rc) return rc;
    if (n > 0) {
        k_ctr_fill<<<grid_for(n, T), T, 0, st>>>(pos, keys, vals, nh, c->start, c->pblk, box, c->slot_pos,
                                                 c->slot_idx, c->ctr);
        SR_LAUNCH_CHECK("k_ctr_fill");
    }
    if (nh > 0) {
        k_ctr_pad<<<grid_for((long long)nh * kBlk, T), T, 0, st>>>(nh, c->start, c->end, c->pblk, c->nblk,
                                                                   c->slot_pos, c->slot_idx);
        SR_LAUNCH_CHECK("k_ctr_pad");
    }
    k_ctr_rows<<<grid_for((long long)c->rows_cap + 1, T), T, 0, st>>>(nh, c->rows_cap, c->row0, c->nblk,
                                                                      c->row_tab, c->row_nitem, c->ctr);
    SR_LAUNCH_CHECK("k_ctr_rows");
    rc = sr::exclusive_scan(c->row_nitem, c->row_item0, c->rows_cap + 1, c->scan_r, st);
    if (rc) return rc;
    c->fixed_shift = fixed_shift_for(n, eps);
    c->eps2 = (float)(eps * eps);
    c->prepared = true;
    c->psi_valid = false;
    c->last_n = n;
    c->last_nh = nh;
    c->last_stream = st;
    return SR_OK;
}

int sr_centers_potential(sr_centers* c, void* stream) {
    if (!c) return sr::set_error(SR_ERR_ARG, "sr_centers_potential: null workspace");
    if (!c->prepared) return sr::set_error(SR_ERR_STATE, "sr_centers_potential: call sr_centers_prepare first");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long n = c->last_n;
    const int nh = c->last_nh;
    const float scale = std::ldexp(1.0f, c->fixed_shift);
    const int T = 256;
    if (n > 0 && nh > 0) {
        // accumulators start from zero on every call (the pair kernels add)
        k_ctr_zero<<<grid_for(n, T), T, 0, st>>>(c->keys[c->sorted], c->start, c->pblk, c->psi, c->ctr);
        SR_LAUNCH_CHECK("k_ctr_zero");
        if (c->variant == SR_CENTERS_SYMMETRIC) {
            k_ctr_queue_reset<<<1, 1, 0, st>>>(c->ctr);
            SR_LAUNCH_CHECK("k_ctr_queue_reset");
            k_ctr_pairs<<<c->pair_blocks, kThreads, 0, st>>>(c->slot_pos, c->psi, c->row_tab, c->row_item0,
                                                             c->row0, c->pblk, c->nblk, c->start, c->end,
                                                             nh, c->eps2, scale, c->ctr, c->slot_max);
            SR_LAUNCH_CHECK("k_ctr_pairs");
        } else {
            k_ctr_plain<<<grid_for(n, T), T, 0, st>>>(c->slot_pos, c->psi, c->keys[c->sorted], c->start,
                                                      c->end, c->pblk, c->eps2, scale, c->ctr);
            SR_LAUNCH_CHECK("k_ctr_plain");
        }
    }
    c->psi_valid = true;
    c->last_stream = st;
    return SR_OK;
}

int sr_centers_finish(sr_centers* c, double* phi, int64_t* center, double* center_phi, void* stream) {
    if (!c) return sr::set_error(SR_ERR_ARG, "sr_centers_finish: null workspace");
    if (!c->psi_valid) return sr::set_error(SR_ERR_STATE, "sr_centers_finish: call sr_centers_potential first");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long n = c->last_n;
    const int nh = c->last_nh;
    const double inv_scale = std::ldexp(1.0, -c->fixed_shift);
    const int T = 256;
    if (phi && n > 0) {
        SR_CUDA_CHECK(cudaMemsetAsync(phi, 0, sizeof(double) * (size_t)n, st));
        k_ctr_phi<<<grid_for(n, T), T, 0, st>>>(c->keys[c->sorted], c->vals[c->sorted], c->start, c->pblk,
                                                c->psi, inv_scale, phi, c->ctr);
        SR_LAUNCH_CHECK("k_ctr_phi");
    }
    if ((center || center_phi) && nh > 0) {
        const int blocks = nh < 148 * 16 ? nh : 148 * 16;
        k_ctr_argmin<<<blocks, T, 0, st>>>(nh, c->start, c->end, c->pblk, c->psi, c->slot_idx, inv_scale,
                                           reinterpret_cast<long long*>(center), center_phi);
        SR_LAUNCH_CHECK("k_ctr_argmin");
    }
    c->last_stream = st;
    return SR_OK;
}

int sr_centers_run(sr_centers* c, const double* pos, const int32_t* labels, int64_t n,
                   int32_t n_halos, double box, double eps, double* phi, int64_t* center,
                   double* center_phi, void* stream) {
    int rc = sr_centers_prepare(c, pos, labels, n, n_halos, box, eps, stream);
    if (!rc) rc = sr_centers_potential(c, stream);
    if (!rc) rc = sr_centers_finish(c, phi, center, center_phi, stream);
    return rc;
}

int sr_centers_get_info(sr_centers* c, sr_centers_info* out) {
    if (!c || !out) return sr::set_error(SR_ERR_ARG, "sr_centers_get_info: null argument");
    if (!c->prepared) return sr::set_error(SR_ERR_STATE, "sr_centers_get_info: nothing prepared yet");
    SR_CUDA_CHECK(cudaStreamSynchronize(c->last_stream));
    CtrDev h{};
    SR_CUDA_CHECK(cudaMemcpy(&h, c->ctr, sizeof(CtrDev), cudaMemcpyDeviceToHost));
    int rows = 0, items = 0;
    SR_CUDA_CHECK(cudaMemcpy(&rows, c->row0 + c->last_nh, sizeof(int), cudaMemcpyDeviceToHost));
    if (c->variant == SR_CENTERS_SYMMETRIC)
        SR_CUDA_CHECK(cudaMemcpy(&items, c->row_item0 + rows, sizeof(int), cudaMemcpyDeviceToHost));
    out->n_particles = c->last_n;
    out->n_members = (int64_t)h.members;
    out->n_halos = c->last_nh;
    out->max_members = (int64_t)h.max_members;
    out->pairs = (int64_t)h.pairs;
    out->items = c->variant == SR_CENTERS_SYMMETRIC ? items : 0;
    out->evaluated = c->variant == SR_CENTERS_SYMMETRIC ? (int64_t)h.evaluated : 0;
    out->fixed_shift = c->fixed_shift;
    out->variant = c->variant;
    out->bad_labels = (int64_t)h.bad_labels;
    out->wide_members = (int64_t)h.wide;
    out->check_code = (int64_t)h.check;
    return SR_OK;
}

}  // extern "C"
