// The plain short-range kernel: one launch per z-slab of cells, one thread
// per particle slot, neighbour particles loaded straight from global memory
// for all 27 neighbour cells (no box culling, no shared-memory staging, no
// work queue).  Same pair arithmetic and the same per-chunk Kahan grouping
// as the persistent kernel, so both meet the same accuracy bar; it is the
// reference point for the persistent kernel's speed-up.
#include <vector>

#include "sr_internal.h"

namespace sr {
namespace {

__global__ void __launch_bounds__(128) k_plain(const int* __restrict__ ccs, const int4* __restrict__ meta,
                                               const float4* __restrict__ clo,
                                               const float4* __restrict__ slot_pos,
                                               const int* __restrict__ slot_idx,
                                               const VolDev* __restrict__ vols, int chunk, long long slot_begin,
                                               long long slot_end, float4* __restrict__ acc) {
    const long long s = slot_begin + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= slot_end) return;
    const int I = (int)(s / chunk);
    const int lane = (int)(s % chunk);
    const int4 mi = meta[I];
    const int cnt = __float_as_int(clo[I].w);
    if (lane >= cnt) return;
    const VolDev& V = vols[mi.w];
    const float4 pi = slot_pos[s];
    if (pi.w <= 0.f) return;                           // a passive neighbour: its row is not written
    const int b = V.sub_bits;
    const int cx = mi.x >> b, cy = mi.y >> b, cz = mi.z >> b;
    const float eps2 = V.eps2u, rc2 = V.rc2u;
    const float n0 = V.nq[0], n1 = V.nq[1], n2 = V.nq[2], n3 = V.nq[3], n4 = V.nq[4], n5 = V.nq[5];
    float sx = 0.f, sy = 0.f, sz = 0.f, kx = 0.f, ky = 0.f, kz = 0.f;
    for (int oz = -1; oz <= 1; ++oz) {
        int nz = cz + oz, wz = 0;
        if (nz < 0) { nz += V.n_c; wz = -1; } else if (nz >= V.n_c) { nz -= V.n_c; wz = 1; }
        for (int oy = -1; oy <= 1; ++oy) {
            int ny = cy + oy, wy = 0;
            if (ny < 0) { ny += V.n_c; wy = -1; } else if (ny >= V.n_c) { ny -= V.n_c; wy = 1; }
            for (int ox = -1; ox <= 1; ++ox) {
                int nx = cx + ox, wx = 0;
                if (nx < 0) { nx += V.n_c; wx = -1; } else if (nx >= V.n_c) { nx -= V.n_c; wx = 1; }
                const int cell = V.cell_base + (nz * V.n_c + ny) * V.n_c + nx;
                for (int J = ccs[cell]; J < ccs[cell + 1]; ++J) {
                    const int4 mj = meta[J];
                    const int cj = __float_as_int(clo[J].w);
                    const float Sx = (float)(mj.x + wx * V.M - mi.x);
                    const float Sy = (float)(mj.y + wy * V.M - mi.y);
                    const float Sz = (float)(mj.z + wz * V.M - mi.z);
                    float px = 0.f, py = 0.f, pz = 0.f;
                    for (int l = 0; l < cj; ++l) {
                        const float4 pj = slot_pos[(long long)J * chunk + l];
                        const float dx = (pj.x + Sx) - pi.x;
                        const float dy = (pj.y + Sy) - pi.y;
                        const float dz = (pj.z + Sz) - pi.z;
                        float q = fmaf(dx, dx, eps2);
                        q = fmaf(dy, dy, q);
                        q = fmaf(dz, dz, q);
                        float r;
                        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(q));
                        const float r2 = r * r;
                        const float nq = fmaf(fmaf(fmaf(fmaf(fmaf(n5, q, n4), q, n3), q, n2), q, n1), q, n0);
                        const float f = fmaf(r2, r, nq);
                        if (q < rc2) {
                            px = fmaf(f, dx, px);
                            py = fmaf(f, dy, py);
                            pz = fmaf(f, dz, pz);
                        }
                    }
                    float y = px - kx, t = sx + y; kx = (t - sx) - y; sx = t;
                    y = py - ky; t = sy + y; ky = (t - sy) - y; sy = t;
                    y = pz - kz; t = sz + y; kz = (t - sz) - y; sz = t;
                }
            }
        }
    }
    const int orig = slot_idx[s];
    acc[orig] = make_float4((sx - kx) * V.scale_a, (sy - ky) * V.scale_a, (sz - kz) * V.scale_a, 0.f);
}

}  // namespace

int launch_force_plain(sr_plan* p, float* acc, cudaStream_t st) {
    const long long tc = p->total_cells;
    std::vector<int> ccs(tc + 1);
    SR_CUDA_CHECK(cudaMemcpyAsync(ccs.data(), p->ccs, sizeof(int) * (tc + 1), cudaMemcpyDeviceToHost, st));
    SR_CUDA_CHECK(cudaStreamSynchronize(st));
    const int C = 32 * p->chunk_k;
    for (const VolDev& V : p->vols_h) {
        const long long slab = (long long)V.n_c * V.n_c;
        for (int cz = 0; cz < V.n_c; ++cz) {
            const long long c0 = V.cell_base + cz * slab, c1 = c0 + slab;
            const long long s0 = (long long)ccs[c0] * C, s1 = (long long)ccs[c1] * C;
            if (s1 <= s0) continue;
            const int blocks = (int)((s1 - s0 + 127) / 128);
            k_plain<<<blocks, 128, 0, st>>>(p->ccs, p->chunk_meta, p->chunk_lo, p->slot_pos, p->slot_idx,
                                            p->vols, C, s0, s1, reinterpret_cast<float4*>(acc));
            SR_LAUNCH_CHECK("k_plain");
        }
    }
    return SR_OK;
}

}  // namespace sr
