// Grouped pair kernel: smaller i-groups for low particle density.
//
// At about one particle per unit volume and r_c = 3 a particle has some 110
// neighbours within r_c, but the box of a 32-slot chunk grown by r_c holds
// four to five times as many, and the 32-lane kernel (force.cu) evaluates
// every staged neighbour for every slot of the chunk: about a fifth of its
// evaluations are in range.  Sec. 2.1 sizes the blocks to the local load;
// here each chunk is cut into NG = 32 / G i-groups of G consecutive slots
// (Morton order inside a cell, so each group is spatially compact), and
// every group gets a neighbour ring culled against its own, smaller box.
//
// Per work item (one warp, one chunk):
//   1. pass 1, as force.cu (flat enumeration): cell and chunk culling
//      against the chunk's box, each surviving chunk's particles shifted
//      into the chunk's frame and tested against its box; survivors go to a
//      64-entry staging ring;
//   2. pass 2, every 32 staging entries (one per lane): each entry is
//      tested against the NG group boxes and appended to the ring of every
//      group whose box it comes within the culling radius of;
//   3. group batches: when a group's ring holds kBatch entries, all 32
//      lanes evaluate them together.  Lane = il + G * jp takes slot il of
//      the group against ring entries 2 jp, 2 jp + 1, 2 (jp + J), ...
//      (J = 32 / G lanes per slot, two entries per packed f32x2 step).  The
//      J partial sums of a slot are added in a fixed tree order and the
//      lane that owns the slot (lane = slot) adds the batch total into its
//      Kahan-compensated accumulator.
//
// The shift of a neighbour into the chunk's frame, the differences, s' and
// the in-range predicate are the same binary32 operations as in force.cu,
// so per-particle pair counts are identical; only the grouping of the force
// sum differs.  No float atomics: results are run-to-run identical.
#include "pairs.cuh"

namespace sr {
namespace {

constexpr int kStage = 64;           // staging ring (pass 1), float4 entries
constexpr int kList = 64;            // neighbour-chunk list of the flat enumeration, int4 entries

// Shared memory of one warp, in float4 units: staging ring, neighbour-chunk
// list, the chunk's 32 slot positions, NG group boxes (lo, hi), NG group
// rings of RING entries
// (pair-interleaved: RING/2 float4 (x0, x1, y0, y1) then RING/2 float2
// (z0, z1)).
template <int NG, int RING>
__host__ __device__ constexpr int warp_f4() { return kStage + kList + 32 + 2 * NG + NG * (RING / 2 + RING / 4); }

template <int G, int RING>
constexpr int grp_smem_bytes(int warps) { return warps * warp_f4<32 / G, RING>() * 16; }

// Entry p of a pair-interleaved ring: x, y in float4 p/2 at lanes (p&1) and
// 2+(p&1); z in float2 p/2 at lane (p&1).
__device__ __forceinline__ void ring_put(float* A, float* B, int p, float x, float y, float z) {
    A[(p >> 1) * 4 + (p & 1)] = x;
    A[(p >> 1) * 4 + 2 + (p & 1)] = y;
    B[(p >> 1) * 2 + (p & 1)] = z;
}

template <int MODE, int G, int WARPS, int MINB, int RING, bool SINGLE>
__global__ void __launch_bounds__(WARPS * 32, MINB) k_pairs_grp(const Args a, const VolDev v0) {
    constexpr int NG = 32 / G;           // groups per chunk
    constexpr int J = 32 / G;            // lanes per slot in a group batch
    constexpr int kBatch = RING - 32;    // full group batch (a pass-2 step adds <= 32 per group)
    static_assert(kBatch % (2 * J) == 0, "a full group batch splits evenly over the lanes");
    constexpr bool CNT = MODE == kForceCount;
    extern __shared__ float4 smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    float4* const base = smem + warp * warp_f4<NG, RING>();
    float4* const stage = base;                                   // kStage
    int4* const nlist = reinterpret_cast<int4*>(base + kStage);   // kList
    float4* const islot = base + kStage + kList;                  // 32
    float4* const gbox = islot + 32;                              // 2 NG: lo, hi
    float4* const gA = gbox + 2 * NG;                             // NG x RING/2
    float2* const gB = reinterpret_cast<float2*>(gA + NG * (RING / 2));   // NG x RING/2
    const int il = lane & (G - 1);
    const int jp = lane / G;
    const int mygrp = lane / G;          // the group that slot `lane` belongs to
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
        const Consts KC = load_consts(V, false);
        const PConsts PK = pack_consts<false>(KC);

        // the chunk's slots (empty ones hold kPad) and the group boxes
        const float4 pi = a.slot_pos[(long long)I * 32 + lane];
        const bool valid = lane < it.cnt;
        islot[lane] = pi;
        float lx = valid ? pi.x : INFINITY, ly = valid ? pi.y : INFINITY, lz = valid ? pi.z : INFINITY;
        float hx = valid ? pi.x : -INFINITY, hy = valid ? pi.y : -INFINITY, hz = valid ? pi.z : -INFINITY;
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            lx = fminf(lx, __shfl_xor_sync(kFull, lx, o));
            ly = fminf(ly, __shfl_xor_sync(kFull, ly, o));
            lz = fminf(lz, __shfl_xor_sync(kFull, lz, o));
            hx = fmaxf(hx, __shfl_xor_sync(kFull, hx, o));
            hy = fmaxf(hy, __shfl_xor_sync(kFull, hy, o));
            hz = fmaxf(hz, __shfl_xor_sync(kFull, hz, o));
        }
        if (il == 0) {
            gbox[2 * mygrp] = make_float4(lx, ly, lz, 0.f);
            gbox[2 * mygrp + 1] = make_float4(hx, hy, hz, 0.f);
        }
        const int ng = (it.cnt + G - 1) / G;                       // groups holding particles
        float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;   // slot `lane`
        int npair = 0;
        unsigned long long ev_valid = 0, ev_lane = 0;                // counting mode statistics
        int wg[NG], rg[NG];
#pragma unroll
        for (int g = 0; g < NG; ++g) wg[g] = rg[g] = 0;
        int w1 = 0, r1 = 0;
        __syncwarp();

        // Evaluate n entries of group g's ring from position rd (even): all
        // lanes, then the batch total of each slot goes to its owner lane.
        auto batch = [&](int g, int rd, int n) {
            float* A = reinterpret_cast<float*>(gA + g * (RING / 2));
            float* B = reinterpret_cast<float*>(gB + g * (RING / 2));
            const int padded = (n + 2 * J - 1) / (2 * J) * (2 * J);
            if (lane < padded - n) ring_put(A, B, (rd + n + lane) & (RING - 1), kPad, kPad, kPad);
            __syncwarp();
            const float4 q = islot[g * G + il];
            const f2 XI = f2_pack(q.x, q.x), YI = f2_pack(q.y, q.y), ZI = f2_pack(q.z, q.z);
            f2 PX = 0ull, PY = 0ull, PZ = 0ull;
            int np = 0;
            const ulonglong2* A2 = reinterpret_cast<const ulonglong2*>(A);
            const f2* B2 = reinterpret_cast<const f2*>(B);
            const int m0 = (rd >> 1) + jp;
            // one loop for full and partial batches (a small instruction
            // footprint: the batch is inlined at three call sites)
            const int iters = padded / (2 * J);
#pragma unroll 4
            for (int t = 0; t < iters; ++t) {
                const int m = (m0 + J * t) & (RING / 2 - 1);
                const ulonglong2 e = A2[m];
                pair_force2<CNT>(e.x, e.y, B2[m], XI, YI, ZI, PK, PX, PY, PZ, np);
            }
            float e0, o0;
            f2_unpack(PX, e0, o0); float px = e0 + o0;
            f2_unpack(PY, e0, o0); float py = e0 + o0;
            f2_unpack(PZ, e0, o0); float pz = e0 + o0;
#pragma unroll
            for (int o = G; o < 32; o <<= 1) {                       // the J lanes of slot il
                px += __shfl_xor_sync(kFull, px, o);
                py += __shfl_xor_sync(kFull, py, o);
                pz += __shfl_xor_sync(kFull, pz, o);
                if (CNT) np += __shfl_xor_sync(kFull, np, o);
            }
            if (mygrp == g) {
                kahan_add(sx, cx, px);
                kahan_add(sy, cy, py);
                kahan_add(sz, cz, pz);
                if (CNT) npair += np;
            }
            if (CNT) {
                const int cg = min(G, it.cnt - g * G);
                ev_valid += (unsigned long long)n * cg;
                ev_lane += (unsigned long long)n * G;
            }
            __syncwarp();
        };

        // Pass 2 over n staging entries from r1: each into the rings of the
        // groups whose box it reaches; full group rings are evaluated.
        auto distribute = [&](int n) {
            float4 e = make_float4(kPad, kPad, kPad, 0.f);
            if (lane < n) e = stage[(r1 + lane) & (kStage - 1)];
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                if (g < ng) {
                    const float4 lo = gbox[2 * g], hi = gbox[2 * g + 1];
                    const float gx = fmaxf(fmaxf(lo.x - e.x, e.x - hi.x), 0.f);
                    const float gy = fmaxf(fmaxf(lo.y - e.y, e.y - hi.y), 0.f);
                    const float gz = fmaxf(fmaxf(lo.z - e.z, e.z - hi.z), 0.f);
                    const bool in = lane < n && gx * gx + gy * gy + gz * gz < KC.rcm2;
                    const unsigned m = __ballot_sync(kFull, in);
                    if (in && SR_BOUND(wg[g] + __popc(m & lt) - rg[g] < RING, &a.ctr->check, kChkGroupRing)) {
                        float* A = reinterpret_cast<float*>(gA + g * (RING / 2));
                        float* B = reinterpret_cast<float*>(gB + g * (RING / 2));
                        ring_put(A, B, (wg[g] + __popc(m & lt)) & (RING - 1), e.x, e.y, e.z);
                    }
                    wg[g] += __popc(m);
                }
            }
            __syncwarp();
            unsigned full = 0;                                      // groups holding a full batch
#pragma unroll
            for (int g = 0; g < NG; ++g)
                if (wg[g] - rg[g] >= kBatch) full |= 1u << g;
            while (full) {
                const int g = __ffs(full) - 1;
                full &= full - 1;
                int rd = 0;
#pragma unroll
                for (int q = 0; q < NG; ++q)
                    if (q == g) { rd = rg[q]; rg[q] += kBatch; }
                batch(g, rd & (RING - 1), kBatch);
            }
        };

        auto stage1 = [&](int, float Sx, float Sy, float Sz, const float4* pjs, const float4*) {
            const float4 pj = pjs[0];
            const float xj = pj.x + Sx, yj = pj.y + Sy, zj = pj.z + Sz;
            const float gx = fmaxf(fmaxf(xj - it.hi[0], it.lo[0] - xj), 0.f);
            const float gy = fmaxf(fmaxf(yj - it.hi[1], it.lo[1] - yj), 0.f);
            const float gz = fmaxf(fmaxf(zj - it.hi[2], it.lo[2] - zj), 0.f);
            const bool keep = gx * gx + gy * gy + gz * gz < KC.rcm2;
            const unsigned m = __ballot_sync(kFull, keep);
            if (keep && SR_BOUND(w1 + __popc(m & lt) - r1 < kStage, &a.ctr->check, kChkGroupRing))
                stage[(w1 + __popc(m & lt)) & (kStage - 1)] = make_float4(xj, yj, zj, 0.f);
            w1 += __popc(m);
            __syncwarp();
            if (w1 - r1 >= 32) {
                distribute(32);
                r1 += 32;
            }
        };
        for_each_neighbour_chunk_flat<1, false, kList>(a, it, V, nlist, stage1);
        if (w1 > r1) distribute(w1 - r1);
        // the rest of every group's ring (fewer than kBatch entries: pass 2
        // evaluates a group as soon as it holds kBatch)
        unsigned left = 0;
#pragma unroll
        for (int g = 0; g < NG; ++g)
            if (wg[g] > rg[g]) left |= 1u << g;
        while (left) {
            const int g = __ffs(left) - 1;
            left &= left - 1;
            int rd = 0, n = 0;
#pragma unroll
            for (int q = 0; q < NG; ++q)
                if (q == g) { rd = rg[q]; n = wg[q] - rg[q]; }
            batch(g, rd & (RING - 1), n);
        }

        int cpairs = 0;
        const int orig = a.slot_idx[(long long)I * 32 + lane];
        // active particles only (slot w = 1; a passive neighbour's row is left untouched)
        if (valid && pi.w > 0.f && SR_BOUND(orig >= 0 && orig < a.n_rows, &a.ctr->check, kChkRow)) {
            const float ox = (sx - cx) * KC.scale;
            const float oy = (sy - cy) * KC.scale;
            const float oz = (sz - cz) * KC.scale;
            float4* dst = reinterpret_cast<float4*>(a.out) + orig;
            *dst = make_float4(ox, oy, oz, 0.f);
            if (a.vel) {                                            // fused kick, same arithmetic as sr_kick
                float4* v = reinterpret_cast<float4*>(a.vel) + orig;
                float4 vv = *v;
                vv.x = fmaf(ox, a.kdt, vv.x);
                vv.y = fmaf(oy, a.kdt, vv.y);
                vv.z = fmaf(oz, a.kdt, vv.z);
                *v = vv;
            }
            if (CNT) {
                if (a.per_particle) a.per_particle[orig] = npair - 1;   // minus the self pair
                cpairs = npair - 1;
            }
        }
        if (CNT && a.pair_total) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cpairs += __shfl_xor_sync(kFull, cpairs, o);
            if (lane == 0) {
                atomicAdd(a.pair_total, (unsigned long long)cpairs);
                atomicAdd(&a.ctr->evals, ev_valid);
                atomicAdd(&a.ctr->lane_evals, ev_lane);
            }
        }
        __syncwarp();
    }
}

// Grouped variants (index - kGroupedFirst): group size, warps per block,
// blocks per SM, group ring entries.
#define SR_GROUPED_VARIANTS(X) X(0, 8, 8, 3, 128) X(1, 16, 8, 3, 128)

template <int MODE, int G, int WARPS, int MINB, int RING, bool SINGLE>
int grp_prepare(sr_plan* p, int* blocks) {
    auto k = k_pairs_grp<MODE, G, WARPS, MINB, RING, SINGLE>;
    const int bytes = grp_smem_bytes<G, RING>(WARPS);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_pairs_grp)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, WARPS * 32, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy of k_pairs_grp");
    *blocks = (per_sm < 1 ? 1 : per_sm) * p->sm_count;
    return SR_OK;
}

template <int MODE, bool SINGLE>
int grp_prepare_all(sr_plan* p, int* blocks) {
#define SR_GRP_PREP(I, G, W, B, R) \
    if (int rc = grp_prepare<MODE, G, W, B, R, SINGLE>(p, &blocks[I])) return rc;
    SR_GROUPED_VARIANTS(SR_GRP_PREP)
#undef SR_GRP_PREP
    return SR_OK;
}

template <int MODE, bool SINGLE>
void grp_launch(int v, int blocks, const Args& a, const VolDev& v0, cudaStream_t st) {
    switch (v) {
#define SR_GRP_LAUNCH(I, G, W, B, R)                                                                   \
    case I:                                                                                            \
        k_pairs_grp<MODE, G, W, B, R, SINGLE><<<blocks, W * 32, grp_smem_bytes<G, R>(W), st>>>(a, v0); \
        break;
        SR_GROUPED_VARIANTS(SR_GRP_LAUNCH)
#undef SR_GRP_LAUNCH
        default: break;
    }
}

}  // namespace

// Occupancy (and the dynamic shared-memory opt-in) of the grouped variants,
// for 32-particle chunks: blocks[i] and count_blocks[i] for variant
// kGroupedFirst + i in force and counting mode.
int grouped_occupancy(sr_plan* p, int* blocks, int* count_blocks) {
    if (p->n_vol == 1) {
        if (int rc = grp_prepare_all<kForce, true>(p, blocks)) return rc;
        return grp_prepare_all<kForceCount, true>(p, count_blocks);
    }
    if (int rc = grp_prepare_all<kForce, false>(p, blocks)) return rc;
    return grp_prepare_all<kForceCount, false>(p, count_blocks);
}

// sr_force / sr_force_kick with a grouped variant (p->variant >= kGroupedFirst):
// the counting mode when pairs or per_particle is given, as launch_force.
int launch_force_grouped(sr_plan* p, float* acc, unsigned long long* pairs, int* per_particle, cudaStream_t st,
                         float* vel, float kdt) {
    const int v = p->variant - kGroupedFirst;
    if (v < 0 || v >= kGroupedVariants || p->chunk_k != 1) return set_error(SR_ERR_ARG, "not a grouped variant");
    Args a = make_args(p);
    a.out = acc;
    a.vel = vel;
    a.kdt = kdt;
    a.per_particle = per_particle;
    a.pair_total = pairs;
    const VolDev& v0 = p->vols_h[0];
    const bool single = p->n_vol == 1;
    SR_CUDA_CHECK(cudaMemsetAsync(&p->ctr->queue, 0, sizeof(long long), st));
    if (pairs || per_particle) {
        SR_CUDA_CHECK(cudaMemsetAsync(&p->ctr->evals, 0, 2 * sizeof(unsigned long long), st));
        const int blocks = p->grp_count_blocks[v];
        if (single) grp_launch<kForceCount, true>(v, blocks, a, v0, st);
        else grp_launch<kForceCount, false>(v, blocks, a, v0, st);
        SR_LAUNCH_CHECK("k_pairs_grp<count>");
        return SR_OK;
    }
    const int blocks = p->force_blocks_v[p->variant];
    if (single) grp_launch<kForce, true>(v, blocks, a, v0, st);
    else grp_launch<kForce, false>(v, blocks, a, v0, st);
    SR_LAUNCH_CHECK("k_pairs_grp<force>");
    return SR_OK;
}

}  // namespace sr
