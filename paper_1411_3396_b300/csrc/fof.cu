// Friends-of-friends halo finding (Sec. 2.2, Sec. 3.3) on a binned plan.
//
// 1. parent[i] = i for every caller index.
// 2. k_fof_pairs: persistent warps take the plan's chunks in its cost order;
//    for chunk I, the neighbour cells its box comes within the linking
//    length of, and in them the chunks J >= I whose boxes do (each
//    unordered chunk pair once; inside I only slot pairs i < j).  Each lane
//    first tests its slot of J against I's box (the same margined radius),
//    and lane i then tests its particle against the surviving slots of J,
//    broadcast by shuffles, with a binary32 predicate in fine-grid units (exact integer
//    shifts between chunk anchors); pairs within a relative 2^-10 of link^2
//    are decided again from the binary64 positions with the exact rounding
//    sequence of the definition.  Each friend pair found is appended to a
//    per-warp link buffer in shared memory (as the lane's cached group root
//    and the friend's index); when the buffer is nearly full, and at the end
//    of every item, the 32 lanes resolve the buffered links together, so the
//    union-find's memory round trips overlap instead of stalling the test
//    loop one at a time.  The union-find is lock-free: find with path
//    halving, link by CAS of the larger root under the smaller, retried
//    until the roots agree, so the final roots (each group's smallest index)
//    do not depend on the order of the links.  Every loop has an
//    iteration bound (2^24 unless the caller sets another) that sets an
//    error flag instead of spinning on; the host reads it as SR_ERR_TIMEOUT.
// 3. Roots (the smallest index of each group) and group sizes; a scan over
//    the roots of groups with at least min_members particles numbers the
//    halos in increasing root order; labels in caller order.
#include "sr_internal.h"
#include "sr_fof.h"

#include <cmath>

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kFofThreads = 256;
constexpr int kLinkCap = 256;              // per-warp link buffer (entries)
constexpr long long kDefaultMaxIter = 1 << 24;   // default bound of every union-find loop
constexpr double kBand = 1.0 / 1024.0;    // relative band of link^2 sent to the binary64 test

struct FofCtr {
    unsigned long long queue;
    unsigned long long links;
    unsigned long long band;
    unsigned long long err;
    unsigned long long members;
    unsigned long long max_members;
    unsigned long long tests;
    unsigned long long reserved;
};

__device__ __forceinline__ double fold(double v, double box) {
    if (v < 0.0 || v >= box) {
        if (v >= -box && v < 2.0 * box) {
            v = v < 0.0 ? v + box : v - box;
        } else {
            v = fmod(v, box);
            if (v < 0.0) v += box;
        }
        if (v >= box) v = 0.0;
    }
    return v;
}

// The friendship test of the definition, every operation rounded in binary64
// in the stated order (no contraction into fused multiply-adds).
__device__ bool friends_exact(const double* __restrict__ pos, int i, int j, double box, double link2) {
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double xi = fold(pos[3LL * i + a], box);
        const double xj = fold(pos[3LL * j + a], box);
        double d = __dsub_rn(xj, xi);
        d = __dsub_rn(d, __dmul_rn(box, rint(__ddiv_rn(d, box))));
        const double sq = __dmul_rn(d, d);
        s = a == 0 ? sq : __dadd_rn(s, sq);
    }
    return s < link2;
}

// Root of x.  Parent pointers only ever move to smaller indices (to an
// ancestor), so the halving store is safe against concurrent finds and
// links; loads bypass L1 so that a link made on another SM is seen.
__device__ int find_root(int* parent, int x, FofCtr* c, long long max_iter) {
    for (long long it = 0; it < max_iter; ++it) {
        const int p = __ldcg(parent + x);
        if (p == x) return x;
        const int gp = __ldcg(parent + p);
        if (gp != p) __stcg(parent + x, gp);
        x = gp;
    }
    atomicOr(&c->err, 1ull);
    return x;
}

__device__ void unite(int* parent, int a, int b, FofCtr* c, long long max_iter) {
    for (long long it = 0; it < max_iter; ++it) {
        const int ra = find_root(parent, a, c, max_iter), rb = find_root(parent, b, c, max_iter);
        if (ra == rb) return;
        const int hi = ra > rb ? ra : rb, lo = ra > rb ? rb : ra;
        if (atomicCAS(parent + hi, hi, lo) == hi) return;
        a = hi;
        b = lo;
    }
    atomicOr(&c->err, 1ull);
}

// The warp's buffered links (a, b) joined: lane l takes entries l, l + 32,
// ...; nl <= kLinkCap.  a is a cached group root (an ancestor of it): when
// b's root is a, the two are already in one group and nothing is written.
// Then every lane's cached roots move up to the current roots.
template <int K>
__device__ __forceinline__ void flush_links(const int2* buf, int nl, int* parent, FofCtr* c, long long max_iter,
                                            int (&ri)[K]) {
    __syncwarp();
    for (int e = (threadIdx.x & 31); e < nl; e += 32) {
        const int2 l = buf[e];
        const int rb = find_root(parent, l.y, c, max_iter);
        if (rb != l.x) unite(parent, l.x, rb, c, max_iter);
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
        if (ri[k] >= 0) ri[k] = find_root(parent, ri[k], c, max_iter);
    __syncwarp();
}

__global__ void k_fof_init(int n, int* __restrict__ parent, int* __restrict__ size) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    parent[i] = i;
    size[i] = 0;
}

template <int K>
__global__ void __launch_bounds__(kFofThreads, 4)
k_fof_pairs(const int* __restrict__ ccs, int total_cells, const int4* __restrict__ meta,
            const float4* __restrict__ clo, const float4* __restrict__ chi, const float4* __restrict__ slot_pos,
            const int* __restrict__ slot_idx, const sr::VolDev* __restrict__ vols, const int* __restrict__ order,
            const double* __restrict__ pos, double link, double link2, int* parent, FofCtr* c,
            long long max_iter) {
    constexpr int C = 32 * K;
    __shared__ int2 links_buf[kFofThreads / 32][kLinkCap];
    const int lane = threadIdx.x & 31;
    int2* lbuf = links_buf[threadIdx.x >> 5];
    const unsigned lt = (1u << lane) - 1u;
    const int n_items = ccs[total_cells];
    unsigned long long my_links = 0, my_band = 0, my_tests = 0;
    while (true) {
        int item = 0;
        if (lane == 0) item = (int)atomicAdd(&c->queue, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= n_items) break;
        const int I = order[item];
        const int4 m = meta[I];
        const float4 lo = clo[I], hi = chi[I];
        const sr::VolDev& V = vols[m.w];
        const double lu = link / V.h;                           // linking length in fine units
        const float lo_thr = (float)(lu * lu * (1.0 - kBand));
        const float hi_thr = (float)(lu * lu * (1.0 + kBand));
        const float cull = (float)(lu * (1.0 + kBand)) * (1.0f + 1.0f / 512.0f);
        const float cull2 = cull * cull;
        const int q[3] = {m.x, m.y, m.z};
        const float ilo[3] = {lo.x, lo.y, lo.z}, ihi[3] = {hi.x, hi.y, hi.z};
        float4 pi[K];
        int ii[K], ri[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            pi[k] = slot_pos[(long long)I * C + lane + 32 * k];
            ii[k] = slot_idx[(long long)I * C + lane + 32 * k];
            // the particle's group root as last seen (an ancestor of it);
            // links are buffered from it, which shortens their finds
            ri[k] = ii[k] >= 0 ? find_root(parent, ii[k], c, max_iter) : -1;
        }
        int nl = 0;                                              // buffered links (warp-uniform)
        const int b = V.sub_bits;
        int cc[3], olo[3], ohi[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            cc[ax] = q[ax] >> b;
            const float wall_lo = (float)((cc[ax] << b) - q[ax]);
            const float wall_hi = wall_lo + (float)(1 << b);
            olo[ax] = (ilo[ax] - cull < wall_lo) ? -1 : 0;
            ohi[ax] = (ihi[ax] + cull > wall_hi) ? 1 : 0;
        }
        for (int oz = olo[2]; oz <= ohi[2]; ++oz) {
            int nz = cc[2] + oz, kz = 0;
            if (nz < 0) { nz += V.n_c; kz = -1; } else if (nz >= V.n_c) { nz -= V.n_c; kz = 1; }
            for (int oy = olo[1]; oy <= ohi[1]; ++oy) {
                int ny = cc[1] + oy, ky = 0;
                if (ny < 0) { ny += V.n_c; ky = -1; } else if (ny >= V.n_c) { ny -= V.n_c; ky = 1; }
                for (int ox = olo[0]; ox <= ohi[0]; ++ox) {
                    int nx = cc[0] + ox, kx = 0;
                    if (nx < 0) { nx += V.n_c; kx = -1; } else if (nx >= V.n_c) { nx -= V.n_c; kx = 1; }
                    const int cell = V.cell_base + (nz * V.n_c + ny) * V.n_c + nx;
                    const int j0 = ccs[cell], j1 = ccs[cell + 1];
                    const int bx = kx * V.M - q[0], by = ky * V.M - q[1], bz = kz * V.M - q[2];
                    for (int jb = j0; jb < j1; jb += 32) {
                        const int J = jb + lane;
                        bool pass = false;
                        float Sx = 0.f, Sy = 0.f, Sz = 0.f;
                        if (J < j1 && J >= I) {
                            const int4 mj = meta[J];
                            const float4 lj = clo[J], hj = chi[J];
                            Sx = (float)(mj.x + bx);
                            Sy = (float)(mj.y + by);
                            Sz = (float)(mj.z + bz);
                            const float gx = fmaxf(fmaxf(lj.x + Sx - ihi[0], ilo[0] - (hj.x + Sx)), 0.f);
                            const float gy = fmaxf(fmaxf(lj.y + Sy - ihi[1], ilo[1] - (hj.y + Sy)), 0.f);
                            const float gz = fmaxf(fmaxf(lj.z + Sz - ihi[2], ilo[2] - (hj.z + Sz)), 0.f);
                            pass = gx * gx + gy * gy + gz * gz < cull2;
                        }
                        unsigned mask = __ballot_sync(kFull, pass);
                        while (mask) {
                            const int l = __ffs(mask) - 1;
                            mask &= mask - 1;
                            const int Jl = jb + l;
                            const float sx = __shfl_sync(kFull, Sx, l), sy = __shfl_sync(kFull, Sy, l),
                                        sz = __shfl_sync(kFull, Sz, l);
                            float4 pj[K];
                            int jj[K];
#pragma unroll
                            for (int k = 0; k < K; ++k) {
                                pj[k] = slot_pos[(long long)Jl * C + lane + 32 * k];
                                jj[k] = slot_idx[(long long)Jl * C + lane + 32 * k];
                            }
#pragma unroll
                            for (int kk = 0; kk < K; ++kk) {
                                // particle cull: only slots of J within the (margined) linking
                                // length of I's box can have a friend in I
                                bool near = false;
                                {
                                    const float xj = pj[kk].x + sx, yj = pj[kk].y + sy, zj = pj[kk].z + sz;
                                    const float gx = fmaxf(fmaxf(xj - ihi[0], ilo[0] - xj), 0.f);
                                    const float gy = fmaxf(fmaxf(yj - ihi[1], ilo[1] - yj), 0.f);
                                    const float gz = fmaxf(fmaxf(zj - ihi[2], ilo[2] - zj), 0.f);
                                    near = jj[kk] >= 0 && gx * gx + gy * gy + gz * gz < cull2;
                                }
                                for (unsigned sm = __ballot_sync(kFull, near); sm; sm &= sm - 1) {
                                    const int sl = __ffs(sm) - 1;
                                    const float xj = __shfl_sync(kFull, pj[kk].x, sl) + sx;
                                    const float yj = __shfl_sync(kFull, pj[kk].y, sl) + sy;
                                    const float zj = __shfl_sync(kFull, pj[kk].z, sl) + sz;
                                    const int jidx = __shfl_sync(kFull, jj[kk], sl);
                                    const int js = sl + 32 * kk;
#pragma unroll
                                    for (int k = 0; k < K; ++k) {
                                        const int is = lane + 32 * k;
                                        bool f = false;
                                        if (ii[k] >= 0 && jidx >= 0 && !(Jl == I && js <= is)) {
                                            ++my_tests;
                                            const float dx = xj - pi[k].x, dy = yj - pi[k].y, dz = zj - pi[k].z;
                                            const float s = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                                            if (s < hi_thr) {
                                                f = s < lo_thr;
                                                if (!f) {
                                                    ++my_band;
                                                    f = friends_exact(pos, ii[k], jidx, V.box, link2);
                                                }
                                            }
                                        }
                                        const unsigned fm = __ballot_sync(kFull, f);
                                        if (f) {
                                            ++my_links;
                                            lbuf[nl + __popc(fm & lt)] = make_int2(ri[k], jidx);
                                        }
                                        nl += __popc(fm);
                                        if (nl > kLinkCap - 32) {
                                            flush_links<K>(lbuf, nl, parent, c, max_iter, ri);
                                            nl = 0;
                                        }
                                    }
                                }
                            }
                        }
                    }
                }
            }
        }
        if (nl > 0) flush_links<K>(lbuf, nl, parent, c, max_iter, ri);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_links += __shfl_xor_sync(kFull, my_links, o);
        my_band += __shfl_xor_sync(kFull, my_band, o);
        my_tests += __shfl_xor_sync(kFull, my_tests, o);
    }
    if (lane == 0) {
        if (my_links) atomicAdd(&c->links, my_links);
        if (my_band) atomicAdd(&c->band, my_band);
        if (my_tests) atomicAdd(&c->tests, my_tests);
    }
}

__global__ void k_fof_roots(int n, int* parent, int* __restrict__ root, int* __restrict__ size, FofCtr* c,
                            long long max_iter) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = find_root(parent, i, c, max_iter);
    root[i] = r;
    // lanes with the same root add their count once (members of a group are
    // often neighbours in caller order; one address would otherwise take a
    // serialised atomic per member)
    const unsigned peers = __match_any_sync(__activemask(), r);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&size[r], __popc(peers));
}

// flag[i] = 1 for the root of a halo; flag[n] = 0 (the scan's total).
__global__ void k_fof_flags(int n, int min_members, const int* __restrict__ root, const int* __restrict__ size,
                            int* __restrict__ flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    flag[i] = (i < n && root[i] == i && size[i] >= min_members) ? 1 : 0;
}

__global__ void k_fof_labels(int n, const int* __restrict__ root, const int* __restrict__ size,
                             const int* __restrict__ flag, const int* __restrict__ hid, int* __restrict__ labels,
                             int* __restrict__ halo_sizes, FofCtr* c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = root[i];
    const bool halo = flag[r] != 0;
    labels[i] = halo ? hid[r] : -1;
    if (halo && r == i) {
        if (halo_sizes) halo_sizes[hid[i]] = size[i];
        atomicAdd(&c->members, (unsigned long long)size[i]);
        atomicMax(&c->max_members, (unsigned long long)size[i]);
    }
}

inline unsigned grid_for(long long n, int threads) {
    return (unsigned)((n + threads - 1) / threads);
}

}  // namespace

struct sr_fof {
    long long n_max = 0;
    long long max_iter = kDefaultMaxIter;
    int* parent = nullptr;
    int* root = nullptr;
    int* size = nullptr;
    int* flag = nullptr;
    int* hid = nullptr;
    FofCtr* ctr = nullptr;
    sr::ScanScratch scan;
    int blocks[2] = {0, 0};
    bool ran = false;
    long long last_n = 0;
    cudaStream_t last_stream = nullptr;
};

namespace {

int fof_free(sr_fof* f) {
    void* bufs[] = {f->parent, f->root, f->size, f->flag, f->hid, f->ctr};
    for (void* b : bufs) cudaFree(b);
    sr::scan_free(f->scan);
    delete f;
    return SR_OK;
}

}  // namespace

extern "C" {

int sr_fof_create(int64_t n_max, sr_fof** out) {
    if (!out) return sr::set_error(SR_ERR_ARG, "sr_fof_create: null out");
    *out = nullptr;
    if (n_max < 1 || n_max > 2147483646LL) return sr::set_error(SR_ERR_ARG, "sr_fof_create: bad n_max");
    sr_fof* f = new sr_fof();
    f->n_max = n_max;
    cudaError_t e = cudaMalloc(&f->parent, sizeof(int) * (size_t)n_max);
    if (e == cudaSuccess) e = cudaMalloc(&f->root, sizeof(int) * (size_t)n_max);
    if (e == cudaSuccess) e = cudaMalloc(&f->size, sizeof(int) * (size_t)n_max);
    if (e == cudaSuccess) e = cudaMalloc(&f->flag, sizeof(int) * (size_t)(n_max + 1));
    if (e == cudaSuccess) e = cudaMalloc(&f->hid, sizeof(int) * (size_t)(n_max + 1));
    if (e == cudaSuccess) e = cudaMalloc(&f->ctr, sizeof(FofCtr));
    int rc = e == cudaSuccess ? SR_OK : sr::cuda_fail(e, "sr_fof_create");
    if (!rc) rc = sr::scan_alloc(f->scan, n_max + 1);
    if (!rc) {
        int dev = 0, sms = 0, b1 = 0, b2 = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_fof_pairs<1>, kFofThreads, 0);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_fof_pairs<2>, kFofThreads, 0);
        if (e != cudaSuccess) rc = sr::cuda_fail(e, "sr_fof_create occupancy");
        f->blocks[0] = sms * (b1 > 0 ? b1 : 1);
        f->blocks[1] = sms * (b2 > 0 ? b2 : 1);
    }
    if (rc) {
        fof_free(f);
        return rc;
    }
    *out = f;
    return SR_OK;
}

int sr_fof_destroy(sr_fof* f) {
    if (!f) return SR_OK;
    return fof_free(f);
}

int sr_fof_run(sr_fof* f, sr_plan* p, const double* pos, int64_t n, double link, int min_members,
               int32_t* labels, int32_t* halo_sizes, void* stream) {
    if (!f || !p || ((!pos || !labels) && n > 0)) return sr::set_error(SR_ERR_ARG, "sr_fof_run: null argument");
    if (n < 0) return sr::set_error(SR_ERR_ARG, "sr_fof_run: n must be >= 0");
    if (!(link > 0.0) || !std::isfinite(link) || min_members < 1)
        return sr::set_error(SR_ERR_ARG, "sr_fof_run: link must be > 0 and min_members >= 1");
    if (n > f->n_max) return sr::set_error(SR_ERR_CAPACITY, "sr_fof_run: n above the workspace maximum");
    if (!p->binned || p->n_binned != n)
        return sr::set_error(SR_ERR_STATE, "sr_fof_run: the plan must be binned with these n positions");
    for (const sr::VolDev& v : p->vols_h) {
        const double side = v.h * (double)(1 << v.sub_bits);
        if (link * (1.0 + kBand) * (1.0 + 1.0 / 256.0) > side)
            return sr::set_error(SR_ERR_ARG, "sr_fof_run: linking length not below the plan's cell side");
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int N = (int)n;
    SR_CUDA_CHECK(cudaMemsetAsync(f->ctr, 0, sizeof(FofCtr), st));
    if (N > 0) {
        k_fof_init<<<grid_for(N, 256), 256, 0, st>>>(N, f->parent, f->size);
        SR_LAUNCH_CHECK("k_fof_init");
        if (p->chunk_k == 2)
            k_fof_pairs<2><<<f->blocks[1], kFofThreads, 0, st>>>(
                p->ccs, (int)p->total_cells, p->chunk_meta, p->chunk_lo, p->chunk_hi, p->slot_pos, p->slot_idx,
                p->vols, p->order, pos, link, link * link, f->parent, f->ctr, f->max_iter);
        else
            k_fof_pairs<1><<<f->blocks[0], kFofThreads, 0, st>>>(
                p->ccs, (int)p->total_cells, p->chunk_meta, p->chunk_lo, p->chunk_hi, p->slot_pos, p->slot_idx,
                p->vols, p->order, pos, link, link * link, f->parent, f->ctr, f->max_iter);
        SR_LAUNCH_CHECK("k_fof_pairs");
        k_fof_roots<<<grid_for(N, 256), 256, 0, st>>>(N, f->parent, f->root, f->size, f->ctr, f->max_iter);
        SR_LAUNCH_CHECK("k_fof_roots");
    }
    k_fof_flags<<<grid_for((long long)N + 1, 256), 256, 0, st>>>(N, min_members, f->root, f->size, f->flag);
    SR_LAUNCH_CHECK("k_fof_flags");
    int rc = sr::exclusive_scan(f->flag, f->hid, N + 1, f->scan, st);
    if (rc) return rc;
    if (N > 0) {
        k_fof_labels<<<grid_for(N, 256), 256, 0, st>>>(N, f->root, f->size, f->flag, f->hid, labels, halo_sizes,
                                                      f->ctr);
        SR_LAUNCH_CHECK("k_fof_labels");
    }
    f->ran = true;
    f->last_n = n;
    f->last_stream = st;
    return SR_OK;
}

int sr_fof_set_iteration_limit(sr_fof* f, int64_t max_iter) {
    if (!f) return sr::set_error(SR_ERR_ARG, "sr_fof_set_iteration_limit: null workspace");
    if (max_iter < 0) return sr::set_error(SR_ERR_ARG, "sr_fof_set_iteration_limit: negative limit");
    f->max_iter = max_iter == 0 ? kDefaultMaxIter : max_iter;
    return SR_OK;
}

int sr_fof_get_info(sr_fof* f, sr_fof_info* out) {
    if (!f || !out) return sr::set_error(SR_ERR_ARG, "sr_fof_get_info: null argument");
    if (!f->ran) return sr::set_error(SR_ERR_STATE, "sr_fof_get_info: no run yet");
    SR_CUDA_CHECK(cudaStreamSynchronize(f->last_stream));
    FofCtr h{};
    SR_CUDA_CHECK(cudaMemcpy(&h, f->ctr, sizeof(FofCtr), cudaMemcpyDeviceToHost));
    int nh = 0;
    SR_CUDA_CHECK(cudaMemcpy(&nh, f->hid + f->last_n, sizeof(int), cudaMemcpyDeviceToHost));
    out->n_particles = f->last_n;
    out->n_halos = nh;
    out->n_members = (int64_t)h.members;
    out->max_members = (int64_t)h.max_members;
    out->links = (int64_t)h.links;
    out->band_checks = (int64_t)h.band;
    out->tests = (int64_t)h.tests;
    out->error = h.err ? 1 : 0;
    if (h.err)
        return sr::set_error(SR_ERR_TIMEOUT, "sr_fof_run: a union-find loop reached its iteration limit; labels invalid");
    return SR_OK;
}

}  // extern "C"
