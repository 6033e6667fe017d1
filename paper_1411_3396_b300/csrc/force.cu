// Short-range pair kernels: cost estimate + longest-first order, the
// persistent force kernel and its vector-Jacobian product.
//
// Work decomposition (Sec. 2.1): every chunk (C = 32 K particles of one
// cell, K = 1 or 2) is an "active" block; its "passive" particles are all
// particles within r_c, read from the 27 neighbouring cells (periodic
// images included).  Only active particles are written (the reconcile step
// is implicit).  Load balance follows the same section: per-block cost
// estimates, and the largest blocks are handed out first (longest-
// processing-time order) to a fixed pool of workers -- one warp each --
// pulling from an atomic queue.
//
// Per work item (one warp, lane l owns active slots l, l+32, ..., K of them):
//   1. cell culling   : neighbour cells only where the chunk's box comes
//                       within r_c of the cell wall;
//   2. chunk culling  : 32 candidate chunks at a time, one per lane, by
//                       box-to-box distance (ballot);
//   3. particle cull  : each surviving chunk's particles are shifted into
//                       the active chunk's frame and tested against its
//                       box; survivors are compacted into a per-warp ring
//                       in shared memory;
//   4. pair loop      : every full batch of 32 ring entries is broadcast
//                       from shared memory to all lanes; each entry meets
//                       the lane's K particles; each lane sums d f(s) over
//                       the batch in binary32 and adds the batch partial
//                       into a Kahan-compensated accumulator.
#include "pairs.cuh"

namespace sr {
namespace {

constexpr int kWarpsPerBlock = 8;
constexpr int kThreads = kWarpsPerBlock * 32;
constexpr int kRing = 256;        // per-warp ring of staged neighbours (packed batches take 128)
constexpr int kList = 64;         // per-warp list of neighbour chunks (flat enumeration, FLAGS bit 3)
constexpr int kVjpMinBlocks = 1;   // VJP kernel: 256-thread blocks, at least this many per SM
constexpr int vjp_flags(int k) { return k == 1 ? 2 : 0; }   // packed loop for 32-particle chunks
constexpr int kVjpFlat = 8;        // VJP with the flat neighbour enumeration (FLAGS bit 3)

// Per-lane state: K active particles.
template <int MODE, int K>
struct WarpState {
    float x[K], y[K], z[K];
    float gx[K], gy[K], gz[K];
    float sx[K], sy[K], sz[K], cx[K], cy[K], cz[K];
    int npair[K];
    int nevals;
    int wr, rd;
};

// FLAGS bit 0: two partial-sum sets (even / odd ring entries) to halve the
// dependent FMA chain of the accumulation; summed before the Kahan update.
// FLAGS bit 1: packed f32x2 pair loop over the pair-interleaved ring (see
// ring_put); its partial sums split even / odd entries like bit 0, over
// batches of 128 neighbours (one Kahan update per 128; 64 was 2% faster
// than 32, and 128 1% faster than 64).
template <int MODE, int K, int FLAGS>
__device__ __forceinline__ void run_batch_packed(float4* __restrict__ ring, float4* __restrict__ gring, int base,
                                                 int cnt, WarpState<MODE, K>& w, const PConsts& P) {
    constexpr bool kFull128 = (FLAGS & 4) == 0;     // full batches hold 128 entries (else 64)
    constexpr bool CNT = MODE == kForceCount;
    const ulonglong2* A = reinterpret_cast<const ulonglong2*>(ring);
    const f2* B = reinterpret_cast<const f2*>(ring + kRing / 2);
    if (cnt & 1) {                                   // pad to an even count with an inert entry
        const int p = (base + cnt) & (kRing - 1);
        float* Af = reinterpret_cast<float*>(ring);
        float* Bf = reinterpret_cast<float*>(ring + kRing / 2);
        if ((threadIdx.x & 31) == 0) {
            Af[(p >> 1) * 4 + (p & 1)] = kPad;
            Af[(p >> 1) * 4 + 2 + (p & 1)] = kPad;
            Bf[(p >> 1) * 2 + (p & 1)] = kPad;
            if (MODE == kVjp) {                      // a finite cotangent: the pad's terms are selected away
                float* Gf = reinterpret_cast<float*>(gring);
                float* Hf = reinterpret_cast<float*>(gring + kRing / 2);
                Gf[(p >> 1) * 4 + (p & 1)] = 0.f;
                Gf[(p >> 1) * 4 + 2 + (p & 1)] = 0.f;
                Hf[(p >> 1) * 2 + (p & 1)] = 0.f;
            }
        }
        __syncwarp();
    }
    const int m0 = base >> 1;
    const int npairs = (cnt + 1) >> 1;
    f2 XI[K], YI[K], ZI[K], PX[K], PY[K], PZ[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        XI[k] = f2_pack(w.x[k], w.x[k]);
        YI[k] = f2_pack(w.y[k], w.y[k]);
        ZI[k] = f2_pack(w.z[k], w.z[k]);
        PX[k] = PY[k] = PZ[k] = 0ull;                // (+0, +0)
    }
    if (MODE != kVjp && kFull128 && npairs == 64) {
#pragma unroll
        for (int m = 0; m < 64; ++m) {
            const ulonglong2 a = A[m0 + m];
            const f2 z = B[m0 + m];
#pragma unroll
            for (int k = 0; k < K; ++k)
                pair_force2<CNT>(a.x, a.y, z, XI[k], YI[k], ZI[k], P, PX[k], PY[k], PZ[k], w.npair[k]);
        }
    } else if (MODE == kVjp) {
        const ulonglong2* G = reinterpret_cast<const ulonglong2*>(gring);
        const f2* Hz = reinterpret_cast<const f2*>(gring + kRing / 2);
        f2 GXI[K], GYI[K], GZI[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            GXI[k] = f2_pack(w.gx[k], w.gx[k]);
            GYI[k] = f2_pack(w.gy[k], w.gy[k]);
            GZI[k] = f2_pack(w.gz[k], w.gz[k]);
        }
#pragma unroll 4
        for (int m = 0; m < npairs; ++m) {
            const ulonglong2 a = A[m0 + m], g = G[m0 + m];
            const f2 z = B[m0 + m], gz = Hz[m0 + m];
#pragma unroll
            for (int k = 0; k < K; ++k)
                pair_vjp2(a.x, a.y, z, g.x, g.y, gz, XI[k], YI[k], ZI[k], GXI[k], GYI[k], GZI[k], P, PX[k], PY[k],
                          PZ[k]);
        }
    } else if (npairs == 32) {
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            const ulonglong2 a = A[m0 + m];
            const f2 z = B[m0 + m];
#pragma unroll
            for (int k = 0; k < K; ++k)
                pair_force2<CNT>(a.x, a.y, z, XI[k], YI[k], ZI[k], P, PX[k], PY[k], PZ[k], w.npair[k]);
        }
    } else if (npairs == 16) {
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const ulonglong2 a = A[m0 + m];
            const f2 z = B[m0 + m];
#pragma unroll
            for (int k = 0; k < K; ++k)
                pair_force2<CNT>(a.x, a.y, z, XI[k], YI[k], ZI[k], P, PX[k], PY[k], PZ[k], w.npair[k]);
        }
    } else {
        for (int m = 0; m < npairs; ++m) {
            const ulonglong2 a = A[m0 + m];
            const f2 z = B[m0 + m];
#pragma unroll
            for (int k = 0; k < K; ++k)
                pair_force2<CNT>(a.x, a.y, z, XI[k], YI[k], ZI[k], P, PX[k], PY[k], PZ[k], w.npair[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float e, o;
        f2_unpack(PX[k], e, o); kahan_add(w.sx[k], w.cx[k], e + o);
        f2_unpack(PY[k], e, o); kahan_add(w.sy[k], w.cy[k], e + o);
        f2_unpack(PZ[k], e, o); kahan_add(w.sz[k], w.cz[k], e + o);
    }
    if (MODE == kForceCount) w.nevals += cnt;
}

template <int MODE, int K, int FLAGS>
__device__ __forceinline__ void run_batch(const float4* __restrict__ rp, const float4* __restrict__ rg, int cnt,
                                          WarpState<MODE, K>& w, const Consts& C) {
    float px[K], py[K], pz[K];
#pragma unroll
    for (int k = 0; k < K; ++k) px[k] = py[k] = pz[k] = 0.f;
    if (MODE != kVjp && (FLAGS & 1)) {
        constexpr bool CNT = MODE == kForceCount;
        float qx[K], qy[K], qz[K];
#pragma unroll
        for (int k = 0; k < K; ++k) qx[k] = qy[k] = qz[k] = 0.f;
        if (cnt == 32) {
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
                const float4 a0 = rp[j], a1 = rp[j + 1];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    pair_force<CNT>(a0, w.x[k], w.y[k], w.z[k], C, px[k], py[k], pz[k], w.npair[k]);
                    pair_force<CNT>(a1, w.x[k], w.y[k], w.z[k], C, qx[k], qy[k], qz[k], w.npair[k]);
                }
            }
        } else {
            for (int j = 0; j < cnt; ++j) {
                const float4 a0 = rp[j];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    if (j & 1) pair_force<CNT>(a0, w.x[k], w.y[k], w.z[k], C, qx[k], qy[k], qz[k], w.npair[k]);
                    else pair_force<CNT>(a0, w.x[k], w.y[k], w.z[k], C, px[k], py[k], pz[k], w.npair[k]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            px[k] += qx[k];
            py[k] += qy[k];
            pz[k] += qz[k];
            kahan_add(w.sx[k], w.cx[k], px[k]);
            kahan_add(w.sy[k], w.cy[k], py[k]);
            kahan_add(w.sz[k], w.cz[k], pz[k]);
        }
        if (MODE == kForceCount) w.nevals += cnt;
        return;
    }
    if (MODE == kVjp) {
        if (cnt == 32) {
#pragma unroll 8
            for (int j = 0; j < 32; ++j) {
                const float4 q = rp[j], g = rg[j];
#pragma unroll
                for (int k = 0; k < K; ++k)
                    pair_vjp(q, g, w.x[k], w.y[k], w.z[k], w.gx[k], w.gy[k], w.gz[k], C, px[k], py[k], pz[k]);
            }
        } else {
            for (int j = 0; j < cnt; ++j) {
                const float4 q = rp[j], g = rg[j];
#pragma unroll
                for (int k = 0; k < K; ++k)
                    pair_vjp(q, g, w.x[k], w.y[k], w.z[k], w.gx[k], w.gy[k], w.gz[k], C, px[k], py[k], pz[k]);
            }
        }
    } else {
        constexpr bool CNT = MODE == kForceCount;
        if (cnt == 32) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float4 q = rp[j];
#pragma unroll
                for (int k = 0; k < K; ++k) pair_force<CNT>(q, w.x[k], w.y[k], w.z[k], C, px[k], py[k], pz[k], w.npair[k]);
            }
        } else {
            for (int j = 0; j < cnt; ++j) {
                const float4 q = rp[j];
#pragma unroll
                for (int k = 0; k < K; ++k) pair_force<CNT>(q, w.x[k], w.y[k], w.z[k], C, px[k], py[k], pz[k], w.npair[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        kahan_add(w.sx[k], w.cx[k], px[k]);
        kahan_add(w.sy[k], w.cy[k], py[k]);
        kahan_add(w.sz[k], w.cz[k], pz[k]);
    }
    if (MODE == kForceCount) w.nevals += cnt;
}

// SINGLE: one-volume plans read the volume constants from the kernel
// parameter (constant bank, no registers); batches read them per item.
template <int MODE, int K, int WARPS, int MINB, int FLAGS, bool SINGLE>
__global__ void __launch_bounds__(WARPS * 32, MINB) k_pairs(const Args a, const VolDev v0) {
    constexpr int C = 32 * K;
    constexpr bool PACKED = (FLAGS & 2) != 0;
    constexpr int kPackedBatch = (FLAGS & 4) ? 64 : 128;   // staged neighbours per packed batch
    __shared__ float4 ring_p[WARPS][kRing];
    __shared__ float4 ring_g[MODE == kVjp ? WARPS : 1][kRing];
    __shared__ int4 nlist[(FLAGS & 8) ? WARPS : 1][kList];   // flat enumeration: passing neighbour chunks
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    float4* rp = ring_p[warp];
    float4* rg = ring_g[MODE == kVjp ? warp : 0];
    const int n_items = (int)a.ctr->n_items;       // chunks holding an active particle, in a.order
    while (true) {
        int it_idx = 0;
        if (lane == 0) it_idx = (int)atomicAdd((unsigned long long*)&a.ctr->queue, 1ull);
        it_idx = __shfl_sync(kFull, it_idx, 0);
        if (it_idx >= n_items) break;
        const int I = a.order[it_idx];
        if (!SR_BOUND(I >= 0 && I < a.ccs[a.total_cells], &a.ctr->check, kChkItem)) continue;
        const Item it = load_item(a, I);
        const VolDev& V = SINGLE ? v0 : a.vols[it.vol];
        const Consts KC = load_consts(V, MODE == kVjp);
        const PConsts PK = PACKED ? pack_consts<MODE == kVjp>(KC) : PConsts{};
        WarpState<MODE, K> w;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const long long sl = (long long)I * C + lane + 32 * k;
            const float4 pi = a.slot_pos[sl];
            w.x[k] = pi.x; w.y[k] = pi.y; w.z[k] = pi.z;
            w.gx[k] = w.gy[k] = w.gz[k] = 0.f;
            if (MODE == kVjp) {
                const float4 gi = a.slot_g[sl];
                w.gx[k] = gi.x; w.gy[k] = gi.y; w.gz[k] = gi.z;
            }
            w.sx[k] = w.sy[k] = w.sz[k] = w.cx[k] = w.cy[k] = w.cz[k] = 0.f;
            w.npair[k] = 0;
        }
        w.nevals = 0;
        w.wr = 0; w.rd = 0;
        auto stage = [&](int J, float Sx, float Sy, float Sz, const float4* pjs, const float4* gjs) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float4 pj = pjs[k];
                const float xj = pj.x + Sx, yj = pj.y + Sy, zj = pj.z + Sz;
                const float gx = fmaxf(fmaxf(xj - it.hi[0], it.lo[0] - xj), 0.f);
                const float gy = fmaxf(fmaxf(yj - it.hi[1], it.lo[1] - yj), 0.f);
                const float gz = fmaxf(fmaxf(zj - it.hi[2], it.lo[2] - zj), 0.f);
                const bool keep = gx * gx + gy * gy + gz * gz < KC.rcm2;
                const unsigned m = __ballot_sync(kFull, keep);
                if (keep && SR_BOUND(w.wr + __popc(m & lt) - w.rd < kRing, &a.ctr->check, kChkRing)) {
                    const int slot = (w.wr + __popc(m & lt)) & (kRing - 1);
                    if (PACKED) {
                        // pair-interleaved ring: entry p -> x, y at float4 p/2 lanes
                        // (p&1) and 2+(p&1); z in the second half at float2 p/2
                        float* Af = reinterpret_cast<float*>(rp);
                        float* Bf = reinterpret_cast<float*>(rp + kRing / 2);
                        Af[(slot >> 1) * 4 + (slot & 1)] = xj;
                        Af[(slot >> 1) * 4 + 2 + (slot & 1)] = yj;
                        Bf[(slot >> 1) * 2 + (slot & 1)] = zj;
                    } else {
                        rp[slot] = make_float4(xj, yj, zj, 0.f);
                    }
                    if (MODE == kVjp) {
                        if (PACKED) {                        // the same pair interleaving as positions
                            float* Gf = reinterpret_cast<float*>(rg);
                            float* Hf = reinterpret_cast<float*>(rg + kRing / 2);
                            Gf[(slot >> 1) * 4 + (slot & 1)] = gjs[k].x;
                            Gf[(slot >> 1) * 4 + 2 + (slot & 1)] = gjs[k].y;
                            Hf[(slot >> 1) * 2 + (slot & 1)] = gjs[k].z;
                        } else {
                            rg[slot] = gjs[k];
                        }
                    }
                }
                w.wr += __popc(m);
                __syncwarp();
                if (w.wr - w.rd >= (PACKED ? kPackedBatch : 32)) {
                    const int base = w.rd & (kRing - 1);
                    if (PACKED) run_batch_packed<MODE, K, FLAGS>(rp, rg, base, kPackedBatch, w, PK);
                    else run_batch<MODE, K, FLAGS>(rp + base, rg + base, 32, w, KC);
                    w.rd += PACKED ? kPackedBatch : 32;
                    __syncwarp();
                }
            }
        };
        if constexpr ((FLAGS & 8) != 0) for_each_neighbour_chunk_flat<K, MODE == kVjp, kList>(a, it, V, nlist[warp], stage);
        else for_each_neighbour_chunk<K, MODE == kVjp>(a, it, V, stage);
        if (w.wr > w.rd) {
            const int base = w.rd & (kRing - 1);
            if (PACKED) run_batch_packed<MODE, K, FLAGS>(rp, rg, base, w.wr - w.rd, w, PK);
            else run_batch<MODE, K, FLAGS>(rp + base, rg + base, w.wr - w.rd, w, KC);
            __syncwarp();
        }
        int cpairs = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = lane + 32 * k;
            // active particles only (slot w = 1; a passive neighbour's row is left untouched)
            if (l < it.cnt && a.slot_pos[(long long)I * C + l].w > 0.f) {
                const int orig = a.slot_idx[(long long)I * C + l];
                if (!SR_BOUND(orig >= 0 && orig < a.n_rows, &a.ctr->check, kChkRow)) continue;
                const float ox = (w.sx[k] - w.cx[k]) * KC.scale;
                const float oy = (w.sy[k] - w.cy[k]) * KC.scale;
                const float oz = (w.sz[k] - w.cz[k]) * KC.scale;
                float4* dst = reinterpret_cast<float4*>(a.out) + orig;
                if (MODE == kVjp && a.accumulate) {
                    const float4 prev = *dst;
                    *dst = make_float4(prev.x + ox, prev.y + oy, prev.z + oz, 0.f);
                } else {
                    *dst = make_float4(ox, oy, oz, 0.f);
                }
                if (MODE != kVjp && a.vel) {                  // fused kick, same arithmetic as sr_kick
                    float4* v = reinterpret_cast<float4*>(a.vel) + orig;
                    float4 vv = *v;
                    vv.x = fmaf(ox, a.kdt, vv.x);
                    vv.y = fmaf(oy, a.kdt, vv.y);
                    vv.z = fmaf(oz, a.kdt, vv.z);
                    *v = vv;
                }
                if (MODE == kForceCount) {
                    if (a.per_particle) a.per_particle[orig] = w.npair[k] - 1;   // minus the self pair
                    cpairs += w.npair[k] - 1;
                }
            }
        }
        if (MODE == kForceCount && a.pair_total) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cpairs += __shfl_xor_sync(kFull, cpairs, o);
            if (lane == 0) {
                atomicAdd(a.pair_total, (unsigned long long)cpairs);
                atomicAdd(&a.ctr->evals, (unsigned long long)w.nevals * (unsigned long long)it.cnt);
                atomicAdd(&a.ctr->lane_evals, (unsigned long long)w.nevals * (unsigned long long)C);
            }
        }
    }
}

// Cost estimate of each work item, for the longest-first order: the
// chunk's particle count times the population of the neighbour cells its
// box reaches (the same cell culling as the pair kernel).  One thread per
// chunk; chunks beyond the current count, and chunks without an active
// particle, get the key after every other (they are never work items);
// the work items are counted into ctr->n_items.
__global__ void __launch_bounds__(256) k_cost(const Args a, int max_chunks, unsigned* __restrict__ cost,
                                              unsigned long long* __restrict__ keys, int* __restrict__ vals) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_chunks = a.ccs[a.total_cells];
    unsigned long long cst = 0;
    const bool item = I < n_chunks && __float_as_int(a.chi[I].w) > 0;
    if (I < max_chunks && !item) {
        keys[I] = 255ull;
        vals[I] = I;
        if (I < n_chunks) cost[I] = 0u;
    } else if (item) {
        const Item it = load_item(a, I);
        const VolDev& V = a.vols[it.vol];
        int c[3], olo[3], ohi[3];
        cell_range(it, V, c, olo, ohi);
        unsigned long long sum = 0;
        for (int oz = olo[2]; oz <= ohi[2]; ++oz) {
            int nz = c[2] + oz;
            nz += nz < 0 ? V.n_c : (nz >= V.n_c ? -V.n_c : 0);
            for (int oy = olo[1]; oy <= ohi[1]; ++oy) {
                int ny = c[1] + oy;
                ny += ny < 0 ? V.n_c : (ny >= V.n_c ? -V.n_c : 0);
                for (int ox = olo[0]; ox <= ohi[0]; ++ox) {
                    int nx = c[0] + ox;
                    nx += nx < 0 ? V.n_c : (nx >= V.n_c ? -V.n_c : 0);
                    const int cell = V.cell_base + (nz * V.n_c + ny) * V.n_c + nx;
                    if (!SR_BOUND(cell >= 0 && cell < a.total_cells, &a.ctr->check, kChkCell)) continue;
                    sum += (unsigned)(a.cell_start[cell + 1] - a.cell_start[cell]);
                }
            }
        }
        cst = sum * (unsigned long long)it.cnt;
        if (cst > 0xffffffffull) cst = 0xffffffffull;
        cost[I] = (unsigned)cst;
        // quarter-octave bucket of the cost, largest first
        const unsigned long long x = cst + 1;
        const int msb = 63 - __clzll((long long)x);
        const int frac = msb >= 2 ? (int)((x >> (msb - 2)) & 3) : (int)((x << (2 - msb)) & 3);
        int bucket = msb * 4 + frac;
        if (bucket > 254) bucket = 254;
        keys[I] = (unsigned long long)(254 - bucket);
        vals[I] = I;
    }
    // the total: a warp sum first, one atomic per warp (every lane of the
    // launch is alive here; lanes past the chunks add 0)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cst += __shfl_xor_sync(kFull, cst, o);
    const int items = __popc(__ballot_sync(kFull, item));
    if ((threadIdx.x & 31) == 0) {
        if (cst) atomicAdd(&a.ctr->cost_total, cst);
        if (items) atomicAdd((unsigned long long*)&a.ctr->n_items, (unsigned long long)items);
    }
}

__global__ void __launch_bounds__(256) k_gather_g(const float* __restrict__ g, const int* __restrict__ slot_idx,
                                                  const int* __restrict__ ccs, int total_cells, int chunk,
                                                  float scale, float4* __restrict__ slot_g, long long n_rows,
                                                  unsigned long long* check) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n_slots = (long long)ccs[total_cells] * chunk;
    if (s >= n_slots) return;
    const int idx = slot_idx[s];
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (idx >= 0 && SR_BOUND(idx < n_rows, check, kChkRow)) {
        const float4 x = reinterpret_cast<const float4*>(g)[idx];
        v = make_float4(x.x * scale, x.y * scale, x.z * scale, 0.f);
    }
    slot_g[s] = v;
}


template <int MODE, int K, int WARPS, int MINB, int FLAGS, bool SINGLE>
int occ(sr_plan* p) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, k_pairs<MODE, K, WARPS, MINB, FLAGS, SINGLE>, WARPS * 32, 0);
    if (e != cudaSuccess) return -1;
    return (per_sm < 1 ? 1 : per_sm) * p->sm_count;
}

// Force-kernel variants (warps per block, min blocks per SM, flags):
//   0: 8 x 1   1: 8 x 2   2: 8 x 3   3: 8 x 4   (register budgets 255, 128, 85, 64)
//   4: 4 x 6   5: 4 x 7   6: 4 x 8              (85, 73, 64)
//   7: 8 x 3 with split partial sums (even / odd neighbours)
//   8..11: packed f32x2 pair loop (split partial sums, batches of 128): 8 x 2, 8 x 3, 4 x 6, 8 x 4
//   12: the packed loop in batches of 64, 8 x 4 (faster at near-uniform density)
//   13, 14: 11 and 12 with the flat neighbour enumeration (FLAGS bit 3)
// 64-particle chunks (K = 2) use variants 0..3 only.
#define SR_FORCE_VARIANTS(X) \
    X(0, 8, 1, 0) X(1, 8, 2, 0) X(2, 8, 3, 0) X(3, 8, 4, 0) \
    X(4, 4, 6, 0) X(5, 4, 7, 0) X(6, 4, 8, 0) X(7, 8, 3, 1) \
    X(8, 8, 2, 3) X(9, 8, 3, 3) X(10, 4, 6, 3) X(11, 8, 4, 3) X(12, 8, 4, 7) \
    X(13, 8, 4, 11) X(14, 8, 4, 15)

template <int K, bool SINGLE>
int occupancy_k(sr_plan* p) {
    int v[kVariants];
#define SR_OCC(I, W, B, F) \
    if constexpr (K == 1 || I < 4) v[I] = occ<kForce, K, W, B, F, SINGLE>(p); else v[I] = 0;
    SR_FORCE_VARIANTS(SR_OCC)
#undef SR_OCC
    const int c = occ<kForceCount, K, 8, 1, 0, SINGLE>(p), g = occ<kVjp, K, 8, kVjpMinBlocks, vjp_flags(K), SINGLE>(p);
    for (int i = 0; i < kGroupedFirst; ++i)
        if (v[i] < 0) return set_error(SR_ERR_CUDA, "occupancy query failed");   // 0 = not built for this K
    if (c < 0 || g < 0) return set_error(SR_ERR_CUDA, "occupancy query failed");
    if (K == 1) {
        if (int rc = grouped_occupancy(p, v + kGroupedFirst, p->grp_count_blocks)) return rc;
    } else {
        for (int i = kGroupedFirst; i < kVariants; ++i) v[i] = 0;          // grouped: 32-particle chunks only
    }
    for (int i = 0; i < kVariants; ++i) p->force_blocks_v[i] = v[i];
    p->count_blocks = c;
    p->vjp_blocks = g;
    return SR_OK;
}

template <int K, bool SINGLE>
void launch_force_k(sr_plan* p, const Args& a, cudaStream_t st) {
    const int blocks = p->force_blocks_v[p->variant];
    const VolDev& v0 = p->vols_h[0];
    switch (p->variant) {
#define SR_LAUNCH(I, W, B, F) \
    case I: if constexpr (K == 1 || I < 4) k_pairs<kForce, K, W, B, F, SINGLE><<<blocks, W * 32, 0, st>>>(a, v0); break;
        SR_FORCE_VARIANTS(SR_LAUNCH)
#undef SR_LAUNCH
        default: break;
    }
}

template <int MODE, int K>
void launch_mode(sr_plan* p, const Args& a, int blocks, cudaStream_t st) {
    const VolDev& v0 = p->vols_h[0];
    if (p->n_vol == 1) k_pairs<MODE, K, 8, 1, 0, true><<<blocks, kThreads, 0, st>>>(a, v0);
    else k_pairs<MODE, K, 8, 1, 0, false><<<blocks, kThreads, 0, st>>>(a, v0);
}

// The VJP kernel: packed f32x2 pair loop for 32-particle chunks, the scalar
// loop for 64-particle chunks.
// The VJP follows the selected force variant (the autotuner's reading of
// the density): the flat neighbour enumeration with variants 13-16, and
// packed batches of 64 staged neighbours with variants 12, 14-16 (else
// 128).  The enumeration does not change the bits; the batch size groups
// the compensated sums differently.
template <int K, int FLAGS>
void launch_vjp_f(sr_plan* p, const Args& a, int blocks, cudaStream_t st) {
    const VolDev& v0 = p->vols_h[0];
    if (p->n_vol == 1) k_pairs<kVjp, K, 8, kVjpMinBlocks, FLAGS, true><<<blocks, kThreads, 0, st>>>(a, v0);
    else k_pairs<kVjp, K, 8, kVjpMinBlocks, FLAGS, false><<<blocks, kThreads, 0, st>>>(a, v0);
}

template <int K>
void launch_vjp(sr_plan* p, const Args& a, int blocks, cudaStream_t st) {
    if constexpr (K == 1) {
        const int v = p->variant;
        const bool flat = v >= 13;
        const bool b64 = v == 12 || v >= 14;
        constexpr int F = vjp_flags(K);
        if (flat && b64) launch_vjp_f<K, F | kVjpFlat | 4>(p, a, blocks, st);
        else if (flat) launch_vjp_f<K, F | kVjpFlat>(p, a, blocks, st);
        else if (b64) launch_vjp_f<K, F | 4>(p, a, blocks, st);
        else launch_vjp_f<K, F>(p, a, blocks, st);
    } else {
        launch_vjp_f<K, vjp_flags(K)>(p, a, blocks, st);
    }
}

}  // namespace

// Pair-kernel variants selectable per plan (the autotuner times them).
int force_occupancy(sr_plan* p) {
    const bool single = p->n_vol == 1;
    const int rc = p->chunk_k == 2 ? (single ? occupancy_k<2, true>(p) : occupancy_k<2, false>(p))
                                   : (single ? occupancy_k<1, true>(p) : occupancy_k<1, false>(p));
    if (rc) return rc;
    p->force_blocks = p->force_blocks_v[p->variant];
    p->warps_per_block = kWarpsPerBlock;
    return SR_OK;
}

int launch_cost_and_order(sr_plan* p, cudaStream_t st) {
    Args a = make_args(p);
    SR_CUDA_CHECK(cudaMemsetAsync(&p->ctr->cost_total, 0, sizeof(unsigned long long), st));
    SR_CUDA_CHECK(cudaMemsetAsync(&p->ctr->n_items, 0, sizeof(long long), st));
    const long long mc = p->max_chunks;
    k_cost<<<(int)((mc + 255) / 256), 256, 0, st>>>(a, (int)mc, p->cost, p->lpt_keys[0], p->lpt_vals[0]);
    SR_LAUNCH_CHECK("k_cost");
    int which = 0;
    int rc = radix_sort_pairs(p->lpt_keys, p->lpt_vals, (int)mc, 8, p->rs_chunks, st, &which, &p->ctr->check,
                              &p->ctr->err);
    if (rc) return rc;
    p->order = p->lpt_vals[which];
    return SR_OK;
}

int launch_force(sr_plan* p, float* acc, unsigned long long* pairs, int* per_particle, cudaStream_t st,
                 float* vel, float kdt) {
    if (p->variant >= kGroupedFirst) return launch_force_grouped(p, acc, pairs, per_particle, st, vel, kdt);
    Args a = make_args(p);
    a.out = acc;
    a.vel = vel;
    a.kdt = kdt;
    a.per_particle = per_particle;
    a.pair_total = pairs;
    SR_CUDA_CHECK(cudaMemsetAsync(&p->ctr->queue, 0, sizeof(long long), st));
    if (pairs || per_particle) {
        SR_CUDA_CHECK(cudaMemsetAsync(&p->ctr->evals, 0, 2 * sizeof(unsigned long long), st));
        if (p->chunk_k == 2) launch_mode<kForceCount, 2>(p, a, p->count_blocks, st);
        else launch_mode<kForceCount, 1>(p, a, p->count_blocks, st);
        SR_LAUNCH_CHECK("k_pairs<count>");
        return SR_OK;
    }
    const bool single = p->n_vol == 1;
    if (p->chunk_k == 2) { if (single) launch_force_k<2, true>(p, a, st); else launch_force_k<2, false>(p, a, st); }
    else { if (single) launch_force_k<1, true>(p, a, st); else launch_force_k<1, false>(p, a, st); }
    SR_LAUNCH_CHECK("k_pairs<force>");
    return SR_OK;
}

int launch_vjp(sr_plan* p, const float* g_acc, float* g_pos, float g_scale, int accumulate, cudaStream_t st) {
    const int C = 32 * p->chunk_k;
    const long long n_slots = p->max_chunks * C;
    k_gather_g<<<(int)((n_slots + 255) / 256), 256, 0, st>>>(g_acc, p->slot_idx, p->ccs, (int)p->total_cells,
                                                             C, g_scale, p->slot_g, p->n_binned, &p->ctr->check);
    SR_LAUNCH_CHECK("k_gather_g");
    Args a = make_args(p);
    a.out = g_pos;
    a.accumulate = accumulate;
    SR_CUDA_CHECK(cudaMemsetAsync(&p->ctr->queue, 0, sizeof(long long), st));
    if (p->chunk_k == 2) launch_vjp<2>(p, a, p->vjp_blocks, st);
    else launch_vjp<1>(p, a, p->vjp_blocks, st);
    SR_LAUNCH_CHECK("k_pairs<vjp>");
    return SR_OK;
}

}  // namespace sr
