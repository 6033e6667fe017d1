// Short-range pair kernels: cost estimate + longest-first order, the
// persistent force kernel and its vector-Jacobian product.
//
// Work decomposition (Sec. 2.1): every chunk (<= 32 particles of one cell)
// is an "active" block; its "passive" particles are all particles within
// r_c, read from the 27 neighbouring cells (periodic images included).
// Only active particles are written (the reconcile step is implicit).
// Load balance follows the same section: per-block cost estimates, and the
// largest blocks are handed out first (longest-processing-time order) to
// a fixed pool of workers -- one warp each -- pulling from an atomic queue.
//
// Per work item (one warp, lane = one active particle):
//   1. cell culling   : neighbour cells only where the chunk's box comes
//                       within r_c of the cell wall;
//   2. chunk culling  : 32 candidate chunks at a time, one per lane, by
//                       box-to-box distance (ballot);
//   3. particle cull  : each surviving chunk's particles are shifted into
//                       the active chunk's frame and tested against its
//                       box; survivors are compacted into a per-warp ring
//                       in shared memory;
//   4. pair loop      : every full batch of 32 ring entries is broadcast
//                       from shared memory to all lanes; each lane sums
//                       d f(s) over the batch in binary32 and adds the batch
//                       partial into a Kahan-compensated accumulator.
//
// Units: offsets are in units of the fine grid h; shifts between chunks are
// exact integers (anchor differences plus image multiples of M).  With
// x = s' = |d|^2 + eps^2 (in units):  f_u(x) = x^(-3/2) - q(x) where
// q(x) = h^3 p(h^2 (x - eps_u^2)); a = h^-2 sum d f_u.
#include "sr_internal.h"

namespace sr {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerBlock = 8;
constexpr int kThreads = kWarpsPerBlock * 32;
constexpr int kRing = 64;

enum Mode { kForce = 0, kForceCount = 1, kVjp = 2 };

struct Args {
    const int* ccs;
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
};

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
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

// Calls visit(J, Sx, Sy, Sz, cntJ) for every chunk J whose box comes within
// the culling radius of the item's box, in a fixed order (cells z, y, x
// ascending offsets; chunks ascending).  Warp-uniform control flow.
template <class Visit>
__device__ __forceinline__ void for_each_neighbour_chunk(const Args& a, const Item& it, const VolDev& V,
                                                         Visit&& visit) {
    const int lane = threadIdx.x & 31;
    const int b = V.sub_bits;
    const int side = 1 << b;
    int c[3], olo[3], ohi[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        c[ax] = it.q[ax] >> b;
        const float wall_lo = (float)((c[ax] << b) - it.q[ax]);
        const float wall_hi = wall_lo + (float)side;
        olo[ax] = (it.lo[ax] - V.rcm < wall_lo) ? -1 : 0;
        ohi[ax] = (it.hi[ax] + V.rcm > wall_hi) ? 1 : 0;
    }
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
                const int j0 = a.ccs[cell], j1 = a.ccs[cell + 1];
                const int bx = kx * V.M - it.q[0];
                const int by = ky * V.M - it.q[1];
                const int bz = kz * V.M - it.q[2];
                for (int jb = j0; jb < j1; jb += 32) {
                    const int J = jb + lane;
                    bool pass = false;
                    float Sx = 0.f, Sy = 0.f, Sz = 0.f;
                    int cj = 0;
                    if (J < j1) {
                        const int4 mj = a.meta[J];
                        const float4 lj = a.clo[J];
                        const float4 hj = a.chi[J];
                        Sx = (float)(mj.x + bx);
                        Sy = (float)(mj.y + by);
                        Sz = (float)(mj.z + bz);
                        cj = __float_as_int(lj.w);
                        const float gx = fmaxf(fmaxf(lj.x + Sx - it.hi[0], it.lo[0] - (hj.x + Sx)), 0.f);
                        const float gy = fmaxf(fmaxf(lj.y + Sy - it.hi[1], it.lo[1] - (hj.y + Sy)), 0.f);
                        const float gz = fmaxf(fmaxf(lj.z + Sz - it.hi[2], it.lo[2] - (hj.z + Sz)), 0.f);
                        pass = gx * gx + gy * gy + gz * gz < V.rcm2u;
                    }
                    unsigned mask = __ballot_sync(kFull, pass);
                    while (mask) {
                        const int l = __ffs(mask) - 1;
                        mask &= mask - 1;
                        visit(jb + l, __shfl_sync(kFull, Sx, l), __shfl_sync(kFull, Sy, l),
                              __shfl_sync(kFull, Sz, l), __shfl_sync(kFull, cj, l));
                    }
                }
            }
        }
    }
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

// Force on one lane's particle from one ring entry (x, y, z already in the
// active chunk's frame).
template <bool COUNT>
__device__ __forceinline__ void pair_force(const float4 q, float xi, float yi, float zi, const Consts& K,
                                           float& px, float& py, float& pz, int& npair) {
    const float dx = q.x - xi;
    const float dy = q.y - yi;
    const float dz = q.z - zi;
    float s = fmaf(dx, dx, K.eps2);
    s = fmaf(dy, dy, s);
    s = fmaf(dz, dz, s);
    const float r = rsqrtf(s);
    const float r2 = r * r;
    const float nq = fmaf(fmaf(fmaf(fmaf(fmaf(K.n5, s, K.n4), s, K.n3), s, K.n2), s, K.n1), s, K.n0);
    const float f = fmaf(r2, r, nq);
    if (s < K.rc2) {
        px = fmaf(f, dx, px);
        py = fmaf(f, dy, py);
        pz = fmaf(f, dz, pz);
        if (COUNT) ++npair;
    }
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
    const float r = rsqrtf(s);
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

template <int MODE>
struct WarpState {
    float xi, yi, zi;
    float gx, gy, gz;
    float sx, sy, sz, cx, cy, cz;
    int npair;
    int wr, rd;
};

template <int MODE>
__device__ __forceinline__ void run_batch(const float4* __restrict__ rp, const float4* __restrict__ rg, int cnt,
                                          WarpState<MODE>& w, const Consts& K) {
    float px = 0.f, py = 0.f, pz = 0.f;
    if (MODE == kVjp) {
        if (cnt == 32) {
#pragma unroll 8
            for (int j = 0; j < 32; ++j) pair_vjp(rp[j], rg[j], w.xi, w.yi, w.zi, w.gx, w.gy, w.gz, K, px, py, pz);
        } else {
            for (int j = 0; j < cnt; ++j) pair_vjp(rp[j], rg[j], w.xi, w.yi, w.zi, w.gx, w.gy, w.gz, K, px, py, pz);
        }
    } else {
        constexpr bool C = MODE == kForceCount;
        if (cnt == 32) {
#pragma unroll
            for (int j = 0; j < 32; ++j) pair_force<C>(rp[j], w.xi, w.yi, w.zi, K, px, py, pz, w.npair);
        } else {
            for (int j = 0; j < cnt; ++j) pair_force<C>(rp[j], w.xi, w.yi, w.zi, K, px, py, pz, w.npair);
        }
    }
    kahan_add(w.sx, w.cx, px);
    kahan_add(w.sy, w.cy, py);
    kahan_add(w.sz, w.cz, pz);
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_pairs(const Args a) {
    __shared__ float4 ring_p[kWarpsPerBlock][kRing];
    __shared__ float4 ring_g[MODE == kVjp ? kWarpsPerBlock : 1][kRing];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    float4* rp = ring_p[warp];
    float4* rg = ring_g[MODE == kVjp ? warp : 0];
    const int n_items = a.ccs[a.total_cells];
    while (true) {
        int it_idx = 0;
        if (lane == 0) it_idx = (int)atomicAdd((unsigned long long*)&a.ctr->queue, 1ull);
        it_idx = __shfl_sync(kFull, it_idx, 0);
        if (it_idx >= n_items) break;
        const int I = a.order[it_idx];
        const Item it = load_item(a, I);
        const VolDev& V = a.vols[it.vol];
        const Consts K = load_consts(V, MODE == kVjp);
        WarpState<MODE> w;
        const float4 pi = a.slot_pos[(long long)I * kChunk + lane];
        w.xi = pi.x; w.yi = pi.y; w.zi = pi.z;
        w.gx = w.gy = w.gz = 0.f;
        if (MODE == kVjp) {
            const float4 gi = a.slot_g[(long long)I * kChunk + lane];
            w.gx = gi.x; w.gy = gi.y; w.gz = gi.z;
        }
        w.sx = w.sy = w.sz = w.cx = w.cy = w.cz = 0.f;
        w.npair = 0;
        w.wr = 0; w.rd = 0;
        for_each_neighbour_chunk(a, it, V, [&](int J, float Sx, float Sy, float Sz, int) {
            const long long js = (long long)J * kChunk + lane;
            const float4 pj = a.slot_pos[js];
            const float xj = pj.x + Sx, yj = pj.y + Sy, zj = pj.z + Sz;
            const float gx = fmaxf(fmaxf(xj - it.hi[0], it.lo[0] - xj), 0.f);
            const float gy = fmaxf(fmaxf(yj - it.hi[1], it.lo[1] - yj), 0.f);
            const float gz = fmaxf(fmaxf(zj - it.hi[2], it.lo[2] - zj), 0.f);
            const bool keep = gx * gx + gy * gy + gz * gz < K.rcm2;
            const unsigned m = __ballot_sync(kFull, keep);
            if (keep) {
                const int slot = (w.wr + __popc(m & lt)) & (kRing - 1);
                rp[slot] = make_float4(xj, yj, zj, 0.f);
                if (MODE == kVjp) rg[slot] = a.slot_g[js];
            }
            w.wr += __popc(m);
            __syncwarp();
            if (w.wr - w.rd >= 32) {
                const int base = w.rd & (kRing - 1);
                run_batch<MODE>(rp + base, rg + base, 32, w, K);
                w.rd += 32;
                __syncwarp();
            }
        });
        if (w.wr > w.rd) {
            const int base = w.rd & (kRing - 1);
            run_batch<MODE>(rp + base, rg + base, w.wr - w.rd, w, K);
            __syncwarp();
        }
        if (lane < it.cnt) {
            const int orig = a.slot_idx[(long long)I * kChunk + lane];
            const float ox = (w.sx - w.cx) * K.scale;
            const float oy = (w.sy - w.cy) * K.scale;
            const float oz = (w.sz - w.cz) * K.scale;
            float4* dst = reinterpret_cast<float4*>(a.out) + orig;
            if (MODE == kVjp && a.accumulate) {
                const float4 prev = *dst;
                *dst = make_float4(prev.x + ox, prev.y + oy, prev.z + oz, 0.f);
            } else {
                *dst = make_float4(ox, oy, oz, 0.f);
            }
            if (MODE == kForceCount && a.per_particle) a.per_particle[orig] = w.npair - 1;
        }
        if (MODE == kForceCount && a.pair_total) {
            int c = lane < it.cnt ? w.npair - 1 : 0;      // minus the self pair
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
            if (lane == 0) atomicAdd(a.pair_total, (unsigned long long)c);
        }
    }
}

// Cost estimate (pairs the item will evaluate, from chunk-level culling)
// and the longest-first sort key.  One warp per chunk.
__global__ void __launch_bounds__(kThreads) k_cost(const Args a, int max_chunks, unsigned* __restrict__ cost,
                                                   unsigned long long* __restrict__ keys, int* __restrict__ vals) {
    const int lane = threadIdx.x & 31;
    const int n_chunks = a.ccs[a.total_cells];
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int I = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); I < max_chunks; I += warps) {
        if (I >= n_chunks) {
            if (lane == 0) { keys[I] = 255ull; vals[I] = I; }
            continue;
        }
        const Item it = load_item(a, I);
        const VolDev& V = a.vols[it.vol];
        unsigned long long sum = 0;
        for_each_neighbour_chunk(a, it, V, [&](int, float, float, float, int cj) { sum += (unsigned)cj; });
        if (lane == 0) {
            unsigned long long c = sum * (unsigned long long)it.cnt;
            if (c > 0xffffffffull) c = 0xffffffffull;
            cost[I] = (unsigned)c;
            atomicAdd(&a.ctr->cost_total, c);
            // quarter-octave bucket of the cost, largest first
            const unsigned long long x = c + 1;
            const int msb = 63 - __clzll((long long)x);
            const int frac = msb >= 2 ? (int)((x >> (msb - 2)) & 3) : (int)((x << (2 - msb)) & 3);
            int bucket = msb * 4 + frac;
            if (bucket > 254) bucket = 254;
            keys[I] = (unsigned long long)(254 - bucket);
            vals[I] = I;
        }
    }
}

__global__ void __launch_bounds__(256) k_gather_g(const float* __restrict__ g, const int* __restrict__ slot_idx,
                                                  const int* __restrict__ ccs, int total_cells, float scale,
                                                  float4* __restrict__ slot_g) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n_slots = (long long)ccs[total_cells] * kChunk;
    if (s >= n_slots) return;
    const int idx = slot_idx[s];
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (idx >= 0) {
        const float4 x = reinterpret_cast<const float4*>(g)[idx];
        v = make_float4(x.x * scale, x.y * scale, x.z * scale, 0.f);
    }
    slot_g[s] = v;
}

Args make_args(sr_plan* p) {
    Args a{};
    a.ccs = p->ccs;
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
    return a;
}

template <int MODE>
int occupancy_blocks(sr_plan* p) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pairs<MODE>, kThreads, 0);
    if (e != cudaSuccess) return -(int)e;
    if (per_sm < 1) per_sm = 1;
    return per_sm * p->sm_count;
}

}  // namespace

int force_occupancy(sr_plan* p) {
    int b0 = occupancy_blocks<kForce>(p);
    int b1 = occupancy_blocks<kForceCount>(p);
    int b2 = occupancy_blocks<kVjp>(p);
    if (b0 < 0 || b1 < 0 || b2 < 0) return set_error(SR_ERR_CUDA, "cudaOccupancyMaxActiveBlocksPerMultiprocessor failed");
    p->force_blocks = b0;
    p->count_blocks = b1;
    p->vjp_blocks = b2;
    p->warps_per_block = kWarpsPerBlock;
    return SR_OK;
}

int launch_cost_and_order(sr_plan* p, cudaStream_t st) {
    Args a = make_args(p);
    SR_CUDA_CHECK(cudaMemsetAsync(&p->ctr->cost_total, 0, sizeof(unsigned long long), st));
    const long long mc = p->max_chunks;
    long long want = (mc + kWarpsPerBlock - 1) / kWarpsPerBlock;
    long long cap = (long long)p->sm_count * 8;
    const int blocks = (int)(want < cap ? (want > 0 ? want : 1) : cap);
    k_cost<<<blocks, kThreads, 0, st>>>(a, (int)mc, p->cost, p->lpt_keys[0], p->lpt_vals[0]);
    SR_LAUNCH_CHECK("k_cost");
    int which = 0;
    int rc = radix_sort_pairs(p->lpt_keys, p->lpt_vals, (int)mc, 8, p->rs_chunks, st, &which);
    if (rc) return rc;
    p->order = p->lpt_vals[which];
    return SR_OK;
}

int launch_force(sr_plan* p, float* acc, unsigned long long* pairs, int* per_particle, cudaStream_t st) {
    Args a = make_args(p);
    a.out = acc;
    a.per_particle = per_particle;
    a.pair_total = pairs;
    SR_CUDA_CHECK(cudaMemsetAsync(&p->ctr->queue, 0, sizeof(long long), st));
    if (pairs || per_particle) {
        k_pairs<kForceCount><<<p->count_blocks, kThreads, 0, st>>>(a);
        SR_LAUNCH_CHECK("k_pairs<count>");
    } else {
        k_pairs<kForce><<<p->force_blocks, kThreads, 0, st>>>(a);
        SR_LAUNCH_CHECK("k_pairs<force>");
    }
    return SR_OK;
}

int launch_vjp(sr_plan* p, const float* g_acc, float* g_pos, float g_scale, int accumulate, cudaStream_t st) {
    const long long n_slots = p->max_chunks * kChunk;
    k_gather_g<<<(int)((n_slots + 255) / 256), 256, 0, st>>>(g_acc, p->slot_idx, p->ccs, (int)p->total_cells,
                                                             g_scale, p->slot_g);
    SR_LAUNCH_CHECK("k_gather_g");
    Args a = make_args(p);
    a.out = g_pos;
    a.accumulate = accumulate;
    SR_CUDA_CHECK(cudaMemsetAsync(&p->ctr->queue, 0, sizeof(long long), st));
    k_pairs<kVjp><<<p->vjp_blocks, kThreads, 0, st>>>(a);
    SR_LAUNCH_CHECK("k_pairs<vjp>");
    return SR_OK;
}

}  // namespace sr
