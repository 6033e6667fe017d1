// Device helpers shared by the pair kernels (force.cu: one i-group of 32 or
// 64 slots per chunk; force_grp.cu: several smaller i-groups per chunk):
// kernel arguments, the work item, neighbour-chunk enumeration with cell and
// chunk culling, and the binary32 pair arithmetic (scalar and packed f32x2).
//
// Units: offsets are in units of the fine grid h; shifts between chunks are
// exact integers (anchor differences plus image multiples of M).  With
// x = s' = |d|^2 + eps^2 (in units):  f_u(x) = x^(-3/2) - q(x) where
// q(x) = h^3 p(h^2 (x - eps_u^2)); a = h^-2 sum d f_u.
#pragma once

#include "sr_internal.h"

namespace sr {
namespace {

constexpr unsigned kFull = 0xffffffffu;

enum Mode { kForce = 0, kForceCount = 1, kVjp = 2 };

struct Args {
    const int* ccs;
    const int* cell_start;
    int total_cells;
    const int4* meta;
    const float4* clo;
    const float4* chi;
    const float4* slot_pos;
    const int* slot_idx;
    const float4* slot_g;
    const VolDev* vols;
    const int* order;
    Counters* ctr;
    float* out;                       // acc (force) or g_pos (vjp), float4 rows
    int* per_particle;
    unsigned long long* pair_total;
    int accumulate;
    float* vel;                       // force: nullable, fused kick vel += acc * kdt
    float kdt;
    long long n_rows;                 // caller rows of the binning (bounds of slot_idx entries)
};

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// 1/sqrt(x) as one MUFU operation.  The argument s' = |d|^2 + eps^2/h^2 is
// always a normal binary32 number (>= eps^2/h^2 > 0), so the flush-to-zero
// variant gives the same value as the denormal-safe library routine.
__device__ __forceinline__ float rsqrt_mufu(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// (px, py, pz) += f * (dx, dy, dz) only where s < rc2: one compare and three
// predicated FMAs (no select instructions).
__device__ __forceinline__ void masked_axpy3(float s, float rc2, float f, float dx, float dy, float dz,
                                             float& px, float& py, float& pz) {
    asm("{\n\t.reg .pred p;\n\t"
        "setp.lt.f32 p, %3, %4;\n\t"
        "@p fma.rn.f32 %0, %5, %6, %0;\n\t"
        "@p fma.rn.f32 %1, %5, %7, %1;\n\t"
        "@p fma.rn.f32 %2, %5, %8, %2;\n\t}"
        : "+f"(px), "+f"(py), "+f"(pz)
        : "f"(s), "f"(rc2), "f"(f), "f"(dx), "f"(dy), "f"(dz));
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Active chunk description, warp-uniform.
struct Item {
    int q[3];          // anchor
    int vol;
    int cnt;
    float lo[3], hi[3];
};

__device__ __forceinline__ Item load_item(const Args& a, int I) {
    Item it;
    const int4 m = a.meta[I];
    const float4 lo = a.clo[I];
    const float4 hi = a.chi[I];
    it.q[0] = m.x; it.q[1] = m.y; it.q[2] = m.z; it.vol = m.w;
    it.cnt = __float_as_int(lo.w);
    it.lo[0] = lo.x; it.lo[1] = lo.y; it.lo[2] = lo.z;
    it.hi[0] = hi.x; it.hi[1] = hi.y; it.hi[2] = hi.z;
    return it;
}

// Neighbour-cell offsets the chunk's box reaches: -1 if the box comes within
// the culling radius of the lower wall, +1 of the upper wall.
__device__ __forceinline__ void cell_range(const Item& it, const VolDev& V, int c[3], int olo[3], int ohi[3]) {
    const int b = V.sub_bits;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        c[ax] = it.q[ax] >> b;
        const float wall_lo = (float)((c[ax] << b) - it.q[ax]);
        const float wall_hi = wall_lo + (float)(1 << b);
        olo[ax] = (it.lo[ax] - V.rcm < wall_lo) ? -1 : 0;
        ohi[ax] = (it.hi[ax] + V.rcm > wall_hi) ? 1 : 0;
    }
}

// Calls visit(J, Sx, Sy, Sz, pj, gj) for every chunk J whose box comes
// within the culling radius of the item's box, in a fixed order (cells z, y,
// x ascending offsets; chunks ascending); pj[k] / gj[k] are the lane's slots
// lane + 32 k of chunk J (positions, and cotangents when WITH_G).
// Warp-uniform control flow.  (Holding the next group's records in
// registers to hide load latency was measured slower: it raises register
// pressure across the pair batches.)
template <int K, bool WITH_G, class Visit>
__device__ __forceinline__ void for_each_neighbour_chunk(const Args& a, const Item& it, const VolDev& V,
                                                         Visit&& visit) {
    constexpr int C = 32 * K;
    const int lane = threadIdx.x & 31;
    int c[3], olo[3], ohi[3];
    cell_range(it, V, c, olo, ohi);
    for (int oz = olo[2]; oz <= ohi[2]; ++oz) {
        int nz = c[2] + oz, kz = 0;
        if (nz < 0) { nz += V.n_c; kz = -1; } else if (nz >= V.n_c) { nz -= V.n_c; kz = 1; }
        for (int oy = olo[1]; oy <= ohi[1]; ++oy) {
            int ny = c[1] + oy, ky = 0;
            if (ny < 0) { ny += V.n_c; ky = -1; } else if (ny >= V.n_c) { ny -= V.n_c; ky = 1; }
            for (int ox = olo[0]; ox <= ohi[0]; ++ox) {
                int nx = c[0] + ox, kx = 0;
                if (nx < 0) { nx += V.n_c; kx = -1; } else if (nx >= V.n_c) { nx -= V.n_c; kx = 1; }
                const int cell = V.cell_base + (nz * V.n_c + ny) * V.n_c + nx;
                if (!SR_BOUND(cell >= 0 && cell < a.total_cells, &a.ctr->check, kChkCell)) continue;
                const int j0 = a.ccs[cell], j1 = a.ccs[cell + 1];
                const int bx = kx * V.M - it.q[0];
                const int by = ky * V.M - it.q[1];
                const int bz = kz * V.M - it.q[2];
                for (int jb = j0; jb < j1; jb += 32) {
                    const int J = jb + lane;
                    bool pass = false;
                    float Sx = 0.f, Sy = 0.f, Sz = 0.f;
                    if (J < j1 && SR_BOUND(J >= 0 && J < a.ccs[a.total_cells], &a.ctr->check, kChkChunk)) {
                        const int4 mj = a.meta[J];
                        const float4 lj = a.clo[J];
                        const float4 hj = a.chi[J];
                        Sx = (float)(mj.x + bx);
                        Sy = (float)(mj.y + by);
                        Sz = (float)(mj.z + bz);
                        const float gx = fmaxf(fmaxf(lj.x + Sx - it.hi[0], it.lo[0] - (hj.x + Sx)), 0.f);
                        const float gy = fmaxf(fmaxf(lj.y + Sy - it.hi[1], it.lo[1] - (hj.y + Sy)), 0.f);
                        const float gz = fmaxf(fmaxf(lj.z + Sz - it.hi[2], it.lo[2] - (hj.z + Sz)), 0.f);
                        pass = gx * gx + gy * gy + gz * gz < V.rcm2u;
                    }
                    unsigned mask = __ballot_sync(kFull, pass);
                    while (mask) {
                        const int l = __ffs(mask) - 1;
                        mask &= mask - 1;
                        float4 pj[K], gj[K];
#pragma unroll
                        for (int k = 0; k < K; ++k) {
                            const long long js = (long long)(jb + l) * C + lane + 32 * k;
                            pj[k] = a.slot_pos[js];
                            if (WITH_G) gj[k] = a.slot_g[js];
                        }
                        visit(jb + l, __shfl_sync(kFull, Sx, l), __shfl_sync(kFull, Sy, l),
                              __shfl_sync(kFull, Sz, l), pj, gj);
                    }
                }
            }
        }
    }
}

// The same chunks, in the same order, with the same visit calls as
// for_each_neighbour_chunk, enumerated with more loads in flight.  At about
// one particle per unit volume a cell holds two or three chunks, and the
// cell-by-cell loop above spends a chain of dependent loads (cell range,
// chunk records, slots) per cell with two or three of its 32 lanes busy.
// Here:
//   1. one lane per neighbour cell (at most 27) loads the cell's chunk
//      range: one round of loads for all cells;
//   2. the candidate chunks of all cells are numbered by a warp prefix sum
//      of their counts, and each lane takes one candidate (the owning cell
//      found by a binary search over the lanes' prefix values): chunk
//      records and box culling for 32 candidates per round, whatever the
//      cells' sizes; the passing chunks (index, shift) go to a per-warp
//      list in shared memory (list, CAP entries);
//   3. the list is visited in order, the slots of the next chunk loaded
//      before the current one is visited.
template <int K, bool WITH_G, int CAP, class Visit>
__device__ __forceinline__ void for_each_neighbour_chunk_flat(const Args& a, const Item& it, const VolDev& V,
                                                              int4* __restrict__ list, Visit&& visit) {
    static_assert(CAP >= 64, "the list takes a round of 32 candidates after a flush at CAP - 32");
    constexpr int C = 32 * K;
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    int c[3], olo[3], ohi[3];
    cell_range(it, V, c, olo, ohi);
    const int wx = ohi[0] - olo[0] + 1, wy = ohi[1] - olo[1] + 1;
    const int ncell = wx * wy * (ohi[2] - olo[2] + 1);
    int j0 = 0, cnt = 0, bx = 0, by = 0, bz = 0;
    if (lane < ncell) {                        // lane k: k-th cell in z, y, x order of ascending offsets
        int nx = c[0] + olo[0] + lane % wx, kx = 0;
        int ny = c[1] + olo[1] + (lane / wx) % wy, ky = 0;
        int nz = c[2] + olo[2] + lane / (wx * wy), kz = 0;
        if (nx < 0) { nx += V.n_c; kx = -1; } else if (nx >= V.n_c) { nx -= V.n_c; kx = 1; }
        if (ny < 0) { ny += V.n_c; ky = -1; } else if (ny >= V.n_c) { ny -= V.n_c; ky = 1; }
        if (nz < 0) { nz += V.n_c; kz = -1; } else if (nz >= V.n_c) { nz -= V.n_c; kz = 1; }
        const int cell = V.cell_base + (nz * V.n_c + ny) * V.n_c + nx;
        if (SR_BOUND(cell >= 0 && cell < a.total_cells, &a.ctr->check, kChkCell)) {
            j0 = a.ccs[cell];
            cnt = a.ccs[cell + 1] - j0;
        }
        bx = kx * V.M - it.q[0];
        by = ky * V.M - it.q[1];
        bz = kz * V.M - it.q[2];
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    const int excl = incl - cnt;
    int n = 0;                                 // list entries
    auto visit_list = [&]() {
        __syncwarp();
        float4 pn[K], gn[K];
        if (n > 0) {
            const long long js = (long long)list[0].x * C + lane;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                pn[k] = a.slot_pos[js + 32 * k];
                if (WITH_G) gn[k] = a.slot_g[js + 32 * k];
            }
        }
        for (int e = 0; e < n; ++e) {
            const int4 cur = list[e];
            float4 pj[K], gj[K];
#pragma unroll
            for (int k = 0; k < K; ++k) { pj[k] = pn[k]; gj[k] = gn[k]; }
            if (e + 1 < n) {                   // the next chunk's slots, in flight during this visit
                const long long js = (long long)list[e + 1].x * C + lane;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    pn[k] = a.slot_pos[js + 32 * k];
                    if (WITH_G) gn[k] = a.slot_g[js + 32 * k];
                }
            }
            visit(cur.x, __int_as_float(cur.y), __int_as_float(cur.z), __int_as_float(cur.w), pj, gj);
        }
        __syncwarp();
        n = 0;
    };
    for (int base = 0; base < total; base += 32) {
        const int t = base + lane;
        int k = 0;                             // the cell holding candidate t: largest k with excl_k <= t
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int cand = k + step;
            const int e = __shfl_sync(kFull, excl, cand & 31);
            if (cand < ncell && e <= t) k = cand;
        }
        const int jk = __shfl_sync(kFull, j0, k), ek = __shfl_sync(kFull, excl, k);
        const int bxk = __shfl_sync(kFull, bx, k), byk = __shfl_sync(kFull, by, k), bzk = __shfl_sync(kFull, bz, k);
        bool pass = false;
        int J = 0;
        float Sx = 0.f, Sy = 0.f, Sz = 0.f;
        if (t < total) {
            J = jk + (t - ek);
        }
        if (t < total && SR_BOUND(J >= 0 && J < a.ccs[a.total_cells], &a.ctr->check, kChkChunk)) {
            const int4 mj = a.meta[J];
            const float4 lj = a.clo[J];
            const float4 hj = a.chi[J];
            Sx = (float)(mj.x + bxk);
            Sy = (float)(mj.y + byk);
            Sz = (float)(mj.z + bzk);
            const float gx = fmaxf(fmaxf(lj.x + Sx - it.hi[0], it.lo[0] - (hj.x + Sx)), 0.f);
            const float gy = fmaxf(fmaxf(lj.y + Sy - it.hi[1], it.lo[1] - (hj.y + Sy)), 0.f);
            const float gz = fmaxf(fmaxf(lj.z + Sz - it.hi[2], it.lo[2] - (hj.z + Sz)), 0.f);
            pass = gx * gx + gy * gy + gz * gz < V.rcm2u;
        }
        const unsigned m = __ballot_sync(kFull, pass);
        if (pass && SR_BOUND(n + __popc(m & lt) < CAP, &a.ctr->check, kChkList))
            list[n + __popc(m & lt)] = make_int4(J, __float_as_int(Sx), __float_as_int(Sy), __float_as_int(Sz));
        n += __popc(m);
        if (n > CAP - 32) visit_list();
    }
    if (n > 0) visit_list();
}

struct Consts {
    float eps2, rc2, rcm2, scale;
    float n0, n1, n2, n3, n4, n5;      // -q coefficients
    float d0, d1, d2, d3, d4;          // -q' coefficients
};

__device__ __forceinline__ Consts load_consts(const VolDev& V, bool vjp) {
    Consts k;
    k.eps2 = V.eps2u; k.rc2 = V.rc2u; k.rcm2 = V.rcm2u;
    k.scale = vjp ? V.scale_g : V.scale_a;
    k.n0 = V.nq[0]; k.n1 = V.nq[1]; k.n2 = V.nq[2]; k.n3 = V.nq[3]; k.n4 = V.nq[4]; k.n5 = V.nq[5];
    k.d0 = V.ndq[0]; k.d1 = V.ndq[1]; k.d2 = V.ndq[2]; k.d3 = V.ndq[3]; k.d4 = V.ndq[4];
    return k;
}

// Force on one particle from one ring entry (already in the active chunk's frame).
template <bool COUNT>
__device__ __forceinline__ void pair_force(const float4 q, float xi, float yi, float zi, const Consts& K,
                                           float& px, float& py, float& pz, int& npair) {
    const float dx = q.x - xi;
    const float dy = q.y - yi;
    const float dz = q.z - zi;
    float s = fmaf(dx, dx, K.eps2);
    s = fmaf(dy, dy, s);
    s = fmaf(dz, dz, s);
    const float r = rsqrt_mufu(s);
    const float r2 = r * r;
    const float nq = fmaf(fmaf(fmaf(fmaf(fmaf(K.n5, s, K.n4), s, K.n3), s, K.n2), s, K.n1), s, K.n0);
    const float f = fmaf(r2, r, nq);
    masked_axpy3(s, K.rc2, f, dx, dy, dz, px, py, pz);
    if (COUNT) npair += (s < K.rc2) ? 1 : 0;
}

__device__ __forceinline__ void pair_vjp(const float4 q, const float4 gj, float xi, float yi, float zi,
                                         float gx, float gy, float gz, const Consts& K, float& px,
                                         float& py, float& pz) {
    const float dx = q.x - xi;
    const float dy = q.y - yi;
    const float dz = q.z - zi;
    float s = fmaf(dx, dx, K.eps2);
    s = fmaf(dy, dy, s);
    s = fmaf(dz, dz, s);
    const float r = rsqrt_mufu(s);
    const float r2 = r * r;
    const float r3 = r2 * r;
    const float nq = fmaf(fmaf(fmaf(fmaf(fmaf(K.n5, s, K.n4), s, K.n3), s, K.n2), s, K.n1), s, K.n0);
    const float f = r3 + nq;                                     // f_u
    const float nd = fmaf(fmaf(fmaf(fmaf(K.d4, s, K.d3), s, K.d2), s, K.d1), s, K.d0);
    const float fp = fmaf(-1.5f * r2, r3, nd);                   // f_u'
    const float ex = gj.x - gx, ey = gj.y - gy, ez = gj.z - gz;
    const float dot = fmaf(dz, ez, fmaf(dy, ey, dx * ex));
    const float w = 2.0f * fp * dot;
    if (s < K.rc2) {
        px = fmaf(w, dx, fmaf(f, ex, px));
        py = fmaf(w, dy, fmaf(f, ey, py));
        pz = fmaf(w, dz, fmaf(f, ez, pz));
    }
}

// Packed binary32 pairs (Blackwell f32x2 arithmetic): two values in one
// 64-bit register pair, low half = even ring entry, high half = odd entry.
// Each f32x2 operation is two IEEE binary32 operations (same rounding as the
// scalar ones) in one instruction issue.
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

struct PConsts {
    f2 e2, n0, n1, n2, n3, n4, n5;
    f2 d0, d1, d2, d3, d4;             // -q' coefficients (VJP only)
    float rc2;
};

template <bool VJP>
__device__ __forceinline__ PConsts pack_consts(const Consts& K) {
    PConsts P;
    P.e2 = f2_pack(K.eps2, K.eps2);
    P.n0 = f2_pack(K.n0, K.n0); P.n1 = f2_pack(K.n1, K.n1); P.n2 = f2_pack(K.n2, K.n2);
    P.n3 = f2_pack(K.n3, K.n3); P.n4 = f2_pack(K.n4, K.n4); P.n5 = f2_pack(K.n5, K.n5);
    if (VJP) {
        P.d0 = f2_pack(K.d0, K.d0); P.d1 = f2_pack(K.d1, K.d1); P.d2 = f2_pack(K.d2, K.d2);
        P.d3 = f2_pack(K.d3, K.d3); P.d4 = f2_pack(K.d4, K.d4);
    }
    P.rc2 = K.rc2;
    return P;
}

// Two ring entries against one particle for the VJP: on each half the same
// binary32 operations, in the same order, as pair_vjp.  Out-of-range pairs
// select f = w = 0 (fma(0, finite, p) = p exactly).
__device__ __forceinline__ void pair_vjp2(f2 X, f2 Y, f2 Z, f2 GJX, f2 GJY, f2 GJZ, f2 XI, f2 YI, f2 ZI,
                                          f2 GXI, f2 GYI, f2 GZI, const PConsts& P, f2& PX, f2& PY, f2& PZ) {
    const f2 DX = f2_sub(X, XI), DY = f2_sub(Y, YI), DZ = f2_sub(Z, ZI);
    f2 S = f2_fma(DX, DX, P.e2);
    S = f2_fma(DY, DY, S);
    S = f2_fma(DZ, DZ, S);
    float s0, s1;
    f2_unpack(S, s0, s1);
    const f2 R = f2_pack(rsqrt_mufu(s0), rsqrt_mufu(s1));
    const f2 R2 = f2_mul(R, R);
    const f2 R3 = f2_mul(R2, R);
    f2 H = f2_fma(P.n5, S, P.n4);
    H = f2_fma(H, S, P.n3);
    H = f2_fma(H, S, P.n2);
    H = f2_fma(H, S, P.n1);
    H = f2_fma(H, S, P.n0);
    const f2 F = f2_add(R3, H);                                      // f_u
    f2 ND = f2_fma(P.d4, S, P.d3);
    ND = f2_fma(ND, S, P.d2);
    ND = f2_fma(ND, S, P.d1);
    ND = f2_fma(ND, S, P.d0);
    const f2 M15 = f2_mul(f2_pack(-1.5f, -1.5f), R2);
    const f2 FP = f2_fma(M15, R3, ND);                               // f_u'
    const f2 EX = f2_sub(GJX, GXI), EY = f2_sub(GJY, GYI), EZ = f2_sub(GJZ, GZI);
    const f2 DOT = f2_fma(DZ, EZ, f2_fma(DY, EY, f2_mul(DX, EX)));
    const f2 W = f2_mul(f2_mul(f2_pack(2.0f, 2.0f), FP), DOT);
    const bool in0 = s0 < P.rc2, in1 = s1 < P.rc2;
    float f0, f1, w0, w1;
    f2_unpack(F, f0, f1);
    f2_unpack(W, w0, w1);
    const f2 Fm = f2_pack(in0 ? f0 : 0.f, in1 ? f1 : 0.f);
    const f2 Wm = f2_pack(in0 ? w0 : 0.f, in1 ? w1 : 0.f);
    PX = f2_fma(Wm, DX, f2_fma(Fm, EX, PX));
    PY = f2_fma(Wm, DY, f2_fma(Fm, EY, PY));
    PZ = f2_fma(Wm, DZ, f2_fma(Fm, EZ, PZ));
}

// Two ring entries against one particle; the same binary32 operations as
// pair_force on each half.  An out-of-range pair contributes f = 0, and
// fma(0, d, p) = p exactly, as the scalar path's skipped update.
template <bool COUNT>
__device__ __forceinline__ void pair_force2(f2 X, f2 Y, f2 Z, f2 XI, f2 YI, f2 ZI, const PConsts& P,
                                            f2& PX, f2& PY, f2& PZ, int& npair) {
    const f2 DX = f2_sub(X, XI), DY = f2_sub(Y, YI), DZ = f2_sub(Z, ZI);
    f2 S = f2_fma(DX, DX, P.e2);
    S = f2_fma(DY, DY, S);
    S = f2_fma(DZ, DZ, S);
    float s0, s1;
    f2_unpack(S, s0, s1);
    const f2 R = f2_pack(rsqrt_mufu(s0), rsqrt_mufu(s1));
    const f2 R2 = f2_mul(R, R);
    f2 H = f2_fma(P.n5, S, P.n4);
    H = f2_fma(H, S, P.n3);
    H = f2_fma(H, S, P.n2);
    H = f2_fma(H, S, P.n1);
    H = f2_fma(H, S, P.n0);
    float f0, f1;
    f2_unpack(f2_fma(R2, R, H), f0, f1);
    const bool in0 = s0 < P.rc2, in1 = s1 < P.rc2;
    const f2 F = f2_pack(in0 ? f0 : 0.f, in1 ? f1 : 0.f);
    PX = f2_fma(F, DX, PX);
    PY = f2_fma(F, DY, PY);
    PZ = f2_fma(F, DZ, PZ);
    if (COUNT) npair += (in0 ? 1 : 0) + (in1 ? 1 : 0);
}

inline Args make_args(sr_plan* p) {
    Args a{};
    a.ccs = p->ccs;
    a.cell_start = p->cell_start;
    a.total_cells = (int)p->total_cells;
    a.meta = p->chunk_meta;
    a.clo = p->chunk_lo;
    a.chi = p->chunk_hi;
    a.slot_pos = p->slot_pos;
    a.slot_idx = p->slot_idx;
    a.slot_g = p->slot_g;
    a.vols = p->vols;
    a.order = p->order;
    a.ctr = p->ctr;
    a.n_rows = p->n_binned;
    return a;
}

}  // namespace
}  // namespace sr
