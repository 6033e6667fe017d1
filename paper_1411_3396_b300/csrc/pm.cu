// Long-range side of the force split (Sec. 2: spectrally filtered PM on a
// uniform grid) and the on-the-fly power spectrum (Sec. 4.1: CIC deposit,
// FFT, |delta(k)|^2 binned in |k|, divided by the CIC window).
//
// Grid n^3 (n a power of two), [x][y][z] with z fastest, spacing D = L/n.
//
//   deposit   thread per particle: cell and fraction in binary64, the 8
//             corner weights in binary32, added as 64-bit fixed point (2^S
//             scale, no overflow for n_max particles in one cell), so the
//             grid is independent of the order of the atomics;
//   delta     counts / nbar - 1 into a binary32 complex grid;
//   FFT       three passes, one per axis; n/16 threads per pencil, each
//             holding 16 points in registers; Stockham stages of radix 16
//             (then 2, 4 or 8 for the remaining factor) run in registers,
//             with one padded shared-memory exchange between stages; the
//             first stage reads and the last writes global memory in the
//             same coalesced pattern (along z for the z pass, T consecutive
//             z columns for the y and x passes); twiddles come from a table
//             computed in binary64 on the host;
//   P(k)      modes sorted once (at creation) by shell with the library's
//             stable radix sort; each block sums binary32 terms
//             |delta_k|^2 / W^2 of a fixed segment of one shell in binary64
//             and a final pass adds a shell's segments in order:
//             deterministic; the mean |k| per shell is a table;
//   force     a(k) = i k (4 pi / k^2) exp(-k^2 sigma^2) C(k) / W^2 for two
//             components at once (a_x + i a_y is the transform of two real
//             fields), inverse FFT, then a_z; CIC interpolation to the
//             particles.
#include "sr_internal.h"
#include "sr_pm.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace {

constexpr int kThreads = 256;
constexpr int kSegModes = 4096;        // modes per power-spectrum segment

inline unsigned grid_for(long long n, int threads) {
    return (unsigned)((n + threads - 1) / threads);
}

// Pencils per FFT block: 256 threads at n/16 threads per pencil, at most n
// (the y and x passes take T consecutive z columns of one row).
inline int fft_pencils(int n) {
    const int t = kThreads / (n / 16);
    return t > n ? n : t;
}

__host__ __device__ constexpr int pencil_stride(int n);

inline size_t fft_smem(int n) {
    return sizeof(float2) * (size_t)fft_pencils(n) * (size_t)pencil_stride(n);
}

// x mod L in [0, L) (fmod, then + L for a negative remainder, a result of
// L itself to 0); inputs in [-L, 2L) take one exact
// add or subtract, others the binary64 fmod.
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

constexpr int kNotPow2 = 1 << 30;      // inv_s when n / L is not a power of two

// Base cell and binary32 fractions of one particle (the cell and the
// fraction are formed in binary64; the weights that use the fraction run
// in binary32).  When inv_d = n / L = 2^inv_s and x lies in [0, L), the same
// values come from the bit pattern (exact scaling, floor and the exact
// fraction rounded once to binary32); otherwise, and for u < 1, binary64
// arithmetic.
__device__ __forceinline__ void cic_cell(const double* __restrict__ pos, long long i, double box, double inv_d,
                                         int inv_s, int n, int (&c)[3], float (&f)[3]) {
    const unsigned long long ubox = (unsigned long long)__double_as_longlong(box);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double x = pos[3 * i + a];
        int q, F;
        unsigned long long mant;
        if (inv_s != kNotPow2 && sr::fine_axis_bits(x, ubox, inv_s, q, mant, F) && F >= 0) {
            f[a] = sr::fraction_bits(mant, F);
            c[a] = q >= n ? q - n : q;
        } else {
            const double u = fold(x, box) * inv_d;
            const double fl = floor(u);
            f[a] = (float)(u - fl);
            const int ci = (int)fl;
            c[a] = ci >= n ? ci - n : ci;
        }
    }
}

// visit(ix, iy, iz, v) for the 8 CIC corners of a particle in base cell c
// with fractions f: v is the corner's binary32 weight in fixed point.  The
// one definition of the deposited integers, shared by both deposit kernels.
template <class Visit>
__device__ __forceinline__ void for_each_cic_corner(const int (&c)[3], const float (&f)[3], int n, float scale,
                                                    Visit&& visit) {
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
        const float wx = dx ? f[0] : 1.f - f[0];
        const int ix = c[0] + dx == n ? 0 : c[0] + dx;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const float wxy = wx * (dy ? f[1] : 1.f - f[1]);
            const int iy = c[1] + dy == n ? 0 : c[1] + dy;
#pragma unroll
            for (int dz = 0; dz < 2; ++dz) {
                const float w = wxy * (dz ? f[2] : 1.f - f[2]);
                const int iz = c[2] + dz == n ? 0 : c[2] + dz;
                visit(ix, iy, iz, (unsigned long long)__float2ll_rn(w * scale));
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads)
k_cic_deposit(const double* __restrict__ pos, long long np, double box, double inv_d, int inv_s, int n,
              float scale, unsigned long long* __restrict__ grid) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    int c[3];
    float f[3];
    cic_cell(pos, i, box, inv_d, inv_s, n, c, f);
    for_each_cic_corner(c, f, n, scale, [&](int ix, int iy, int iz, unsigned long long v) {
        atomicAdd(&grid[((long long)ix * n + iy) * n + iz], v);
    });
}

// The same deposit over the short-range binning's order: one warp per
// chunk (at most 32 particles of one binning cell).  The chunk's corners lie
// in the cell's mesh points plus one layer (ratio = mesh cells per binning
// cell), so the warp adds them into a shared-memory tile of that region
// first (at most 32 lanes contend for a point, where the caller-order
// deposit has every particle of a halo core contend for a few points of the
// mesh), then adds the tile's nonzero points to the mesh.  A corner outside
// the tile (the binary64 floors of the two grids can put a particle one mesh
// cell past its binning cell) goes straight to the mesh.  Integer sums
// commute: the mesh is the same bits as k_cic_deposit's.
constexpr int kDepWarps = 8;
constexpr int kDepTileMax = 512;       // tile points per warp (8 warps: 32 KB)

// 64-bit fixed-point add into a tile point held as two 32-bit words, with
// native 32-bit shared-memory atomics: the low word's carry is detected from
// the value it held before the add.  A point's sum stays below 2^64.
__device__ __forceinline__ void tile_add(unsigned* lo, unsigned* hi, unsigned long long v) {
    const unsigned vl = (unsigned)v, vh = (unsigned)(v >> 32);
    const unsigned old = atomicAdd(lo, vl);
    const unsigned carry = old > 0xffffffffu - vl ? 1u : 0u;
    if (vh + carry) atomicAdd(hi, vh + carry);
}

__global__ void __launch_bounds__(kDepWarps * 32)
k_cic_deposit_chunks(const double* __restrict__ pos, const int* __restrict__ ccs, int total_cells,
                     const int4* __restrict__ chunk_span, const int* __restrict__ slot_idx, int chunk, int n_c,
                     double ratio, int wt, double box, double inv_d, int inv_s, int n, float scale,
                     unsigned long long* __restrict__ grid) {
    __shared__ unsigned tlo[kDepWarps][kDepTileMax], thi[kDepWarps][kDepTileMax];
    unsigned* lo = tlo[threadIdx.x >> 5];
    unsigned* hi = thi[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int n_chunks = ccs[total_cells];
    const int tsize = wt * wt * wt;
    const int warps = gridDim.x * kDepWarps;
    for (int k = blockIdx.x * kDepWarps + (threadIdx.x >> 5); k < n_chunks; k += warps) {
        const int cell = chunk_span[k].x;
        const int cx = cell % n_c, cy = (cell / n_c) % n_c, cz = cell / (n_c * n_c);
        const int x0 = (int)floor(cx * ratio), y0 = (int)floor(cy * ratio), z0 = (int)floor(cz * ratio);
        for (int i = lane; i < tsize; i += 32) lo[i] = hi[i] = 0u;
        __syncwarp();
        for (int l = lane; l < chunk; l += 32) {
            const int orig = slot_idx[(long long)k * chunk + l];
            if (orig < 0) continue;                   // empty slot
            int c[3];
            float f[3];
            cic_cell(pos, orig, box, inv_d, inv_s, n, c, f);
            for_each_cic_corner(c, f, n, scale, [&](int ix, int iy, int iz, unsigned long long v) {
                int dx = ix - x0, dy = iy - y0, dz = iz - z0;   // in (-n, n]: one wrap at most
                dx += dx < 0 ? n : (dx >= n ? -n : 0);
                dy += dy < 0 ? n : (dy >= n ? -n : 0);
                dz += dz < 0 ? n : (dz >= n ? -n : 0);
                if (dx < wt && dy < wt && dz < wt) {
                    const int t = (dx * wt + dy) * wt + dz;
                    tile_add(&lo[t], &hi[t], v);
                } else {
                    atomicAdd(&grid[((long long)ix * n + iy) * n + iz], v);
                }
            });
        }
        __syncwarp();
        for (int i = lane; i < tsize; i += 32) {
            const unsigned long long v = ((unsigned long long)hi[i] << 32) | lo[i];
            if (!v) continue;
            const int dz = i % wt, dy = (i / wt) % wt, dx = i / (wt * wt);
            const int gx = (x0 + dx) % n, gy = (y0 + dy) % n, gz = (z0 + dz) % n;
            atomicAdd(&grid[((long long)gx * n + gy) * n + gz], v);
        }
        __syncwarp();
    }
}

// delta = counts / nbar - 1 as a complex grid (imaginary part 0).
__global__ void k_pm_delta(const unsigned long long* __restrict__ fx, long long n3, double inv_scale,
                           double inv_nbar, float2* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    const double cnt = (double)(long long)fx[i] * inv_scale;
    out[i] = make_float2((float)(cnt * inv_nbar - 1.0), 0.f);
}

__global__ void k_pm_counts(const unsigned long long* __restrict__ fx, long long n3, double inv_scale,
                            double* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    out[i] = (double)(long long)fx[i] * inv_scale;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// cos and sin of 2 pi q / 16, q = 0..7 (decimal expansions; q is a
// compile-time constant at every use, so these fold into immediates).
__device__ __forceinline__ constexpr float c16(int q) {
    return q == 0 ? 1.f : q == 1 ? 0.92387953251128674f : q == 2 ? 0.70710678118654752f
         : q == 3 ? 0.38268343236508977f : q == 4 ? 0.f : q == 5 ? -0.38268343236508977f
         : q == 6 ? -0.70710678118654752f : -0.92387953251128674f;
}
__device__ __forceinline__ constexpr float s16(int q) {
    return q == 0 ? 0.f : q == 1 ? 0.38268343236508977f : q == 2 ? 0.70710678118654752f
         : q == 3 ? 0.92387953251128674f : q == 4 ? 1.f : q == 5 ? 0.92387953251128674f
         : q == 6 ? 0.70710678118654752f : 0.38268343236508977f;
}

// x * exp(-+ 2 pi i q / 16), q = 0..15, with the trivial factors spelled out
template <bool INV>
__device__ __forceinline__ float2 rot16(int q, float2 x) {
    if (q >= 8) {                                   // exp(-i pi) = -1
        x = make_float2(-x.x, -x.y);
        q -= 8;
    }
    if (q == 0) return x;
    if (q == 4) return INV ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
    const float c = c16(q), sn = INV ? s16(q) : -s16(q);
    return make_float2(fmaf(c, x.x, -sn * x.y), fmaf(c, x.y, sn * x.x));
}

// 4-point DFT in place on (a, b, c, d) = x[0], x[1], x[2], x[3].
template <bool INV>
__device__ __forceinline__ void dft4(float2& a, float2& b, float2& c, float2& d) {
    const float2 t0 = make_float2(a.x + c.x, a.y + c.y), t1 = make_float2(a.x - c.x, a.y - c.y);
    const float2 t2 = make_float2(b.x + d.x, b.y + d.y), t3 = make_float2(b.x - d.x, b.y - d.y);
    // forward: X1 = t1 - i t3, X3 = t1 + i t3 (inverse: the other way)
    const float2 it3 = INV ? make_float2(-t3.y, t3.x) : make_float2(t3.y, -t3.x);
    a = make_float2(t0.x + t2.x, t0.y + t2.y);
    c = make_float2(t0.x - t2.x, t0.y - t2.y);
    b = make_float2(t1.x + it3.x, t1.y + it3.y);
    d = make_float2(t1.x - it3.x, t1.y - it3.y);
}

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
    const float2 t = a;
    a = make_float2(t.x + b.x, t.y + b.y);
    b = make_float2(t.x - b.x, t.y - b.y);
}

// In-register R-point DFT (R = 2, 4, 8, 16) on v[u + m G], m < R, G = 16/R,
// output in natural order in the same registers.  R = 16 and 8 are split
// as 4 x 4 and 2 x 4 (inner DFTs over the stride-4 or stride-2 subsets,
// twiddles W_R^{n2 k1}, outer DFTs).
template <int R, bool INV>
__device__ __forceinline__ void dft_r(float2 (&v)[16], int u) {
    constexpr int G = 16 / R;
    if constexpr (R == 2) {
        dft2<INV>(v[u], v[u + G]);
    } else if constexpr (R == 4) {
        dft4<INV>(v[u], v[u + G], v[u + 2 * G], v[u + 3 * G]);
    } else if constexpr (R == 8) {
        // x[n2 + 2 n1], n2 < 2, n1 < 4 -> y[n2][k1] -> X[k1 + 4 k2]
        float2 y[2][4];
#pragma unroll
        for (int n2 = 0; n2 < 2; ++n2) {
#pragma unroll
            for (int n1 = 0; n1 < 4; ++n1) y[n2][n1] = v[u + (n2 + 2 * n1) * G];
            dft4<INV>(y[n2][0], y[n2][1], y[n2][2], y[n2][3]);
        }
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            y[1][k1] = rot16<INV>(2 * k1, y[1][k1]);     // W8^{k1} = W16^{2 k1}
            dft2<INV>(y[0][k1], y[1][k1]);
            v[u + k1 * G] = y[0][k1];
            v[u + (k1 + 4) * G] = y[1][k1];
        }
    } else {
        float2 y[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
#pragma unroll
            for (int n1 = 0; n1 < 4; ++n1) y[n2][n1] = v[u + n2 + 4 * n1];
            dft4<INV>(y[n2][0], y[n2][1], y[n2][2], y[n2][3]);
        }
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            y[1][k1] = rot16<INV>(k1, y[1][k1]);
            y[2][k1] = rot16<INV>(2 * k1, y[2][k1]);
            y[3][k1] = rot16<INV>((3 * k1) & 15, y[3][k1]);
            dft4<INV>(y[0][k1], y[1][k1], y[2][k1], y[3][k1]);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[u + k1 + 4 * k2] = y[k2][k1];
        }
    }
}

// Stockham stage of radix R at stride S on a length-N transform: register
// v[e] holds element t + e N/16; butterfly j = t + u N/16 (u < 16/R) takes
// elements j + m N/R (registers u + m 16/R), multiplies by
// W_{S R}^{(j mod S) m}, and its output m belongs at
// (j / S) S R + (j mod S) + m S.
template <int N, int R, int S, bool INV>
__device__ __forceinline__ void fft_stage(float2 (&v)[16], int t, const float2* __restrict__ tw) {
    constexpr int G = 16 / R;
#pragma unroll
    for (int u = 0; u < G; ++u) {
        if (S > 1) {
            const int p = (t + u * (N / 16)) & (S - 1);
#pragma unroll
            for (int m = 1; m < R; ++m) {
                float2 w = __ldg(&tw[p * m * (N / (S * R))]);
                if (INV) w.y = -w.y;
                v[u + m * G] = cmul(w, v[u + m * G]);
            }
        }
        dft_r<R, INV>(v, u);
    }
}

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

// Shared-memory stride between a block's pencils: one slot per 16 points
// plus one, an odd number of 8-byte slots, so that the 16 pencils a half
// warp touches in the y and x passes fall in different banks.
__host__ __device__ constexpr int pencil_stride(int n) { return n + n / 16 + 1; }

// Outputs of stage (R, S) to shared memory, then element t + e N/16 back
// into register e.
template <int N, int R, int S>
__device__ __forceinline__ void exchange(float2 (&v)[16], int t, float2* __restrict__ buf) {
    constexpr int G = 16 / R;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < G; ++u) {
        const int j = t + u * (N / 16);
        const int base = (j / S) * S * R + (j & (S - 1));
#pragma unroll
        for (int m = 0; m < R; ++m) buf[pad16(base + m * S)] = v[u + m * G];
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = buf[pad16(t + e * (N / 16))];
}

// One FFT pass along `axis` (0 = x, stride n^2; 1 = y, stride n; 2 = z,
// stride 1) over T pencils per block, N/16 threads per pencil.  Radix-16
// stages first, the remaining factor (2, 4 or 8) last; global memory is
// read by the first stage and written by the last, in the same coalesced
// pattern (z pass: along z; y and x passes: T consecutive z columns).
template <int N, bool INV>
__global__ void __launch_bounds__(kThreads)
k_fft_pass(float2* __restrict__ data, int axis, int T, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    constexpr int P = N / 16;                 // threads per pencil
    int q, t;
    if (axis == 2) { t = threadIdx.x % P; q = threadIdx.x / P; }
    else { q = threadIdx.x % T; t = threadIdx.x / T; }
    const long long nn = (long long)N * N;
    long long base0, pstride, estride;
    if (axis == 2) {
        base0 = (long long)blockIdx.x * T * N;
        pstride = N;
        estride = 1;
    } else {
        const int per = N / T;
        const long long outer = blockIdx.x / per;
        const long long z0 = (long long)(blockIdx.x % per) * T;
        base0 = (axis == 1 ? outer * nn : outer * N) + z0;
        pstride = 1;
        estride = axis == 1 ? N : nn;
    }
    const long long pb = base0 + q * pstride;
    float2* buf = sm + q * pencil_stride(N);
    float2 v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = data[pb + (long long)(t + e * P) * estride];
    fft_stage<N, 16, 1, INV>(v, t, tw);
    if constexpr (N > 16) {
        constexpr int R2 = N >= 256 ? 16 : N / 16;
        exchange<N, 16, 1>(v, t, buf);
        fft_stage<N, R2, 16, INV>(v, t, tw);
        if constexpr (N > 256) {
            constexpr int R3 = N / 256;
            exchange<N, 16, 16>(v, t, buf);
            fft_stage<N, R3, 256, INV>(v, t, tw);
        }
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) data[pb + (long long)(t + e * P) * estride] = v[e];
}

// Shell of every mode (b = round(|m|); n/2 + 1 for modes outside 1..n/2)
// as sort keys, the mode index as value.
__global__ void k_pm_mode_keys(int n, long long n3, unsigned long long* __restrict__ keys, int* __restrict__ vals) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    const int z = (int)(i % n), y = (int)((i / n) % n), x = (int)(i / ((long long)n * n));
    const int h = n >> 1;
    const long long mx = x < h ? x : x - n, my = y < h ? y : y - n, mz = z < h ? z : z - n;
    const long long m2 = mx * mx + my * my + mz * mz;
    const int b = (int)rint(sqrt((double)m2));
    keys[i] = (unsigned long long)((b >= 1 && b <= h) ? b : h + 1);
    vals[i] = (int)i;
}

// Per segment: sum over its modes of |delta_k|^2 / W^2 (terms in binary32,
// the sum in binary64, fixed order).
__global__ void __launch_bounds__(kThreads)
k_pm_power_seg(const float2* __restrict__ dk, const int* __restrict__ perm, const int* __restrict__ seg_start,
               const int* __restrict__ seg_len, const float* __restrict__ inv_w2, int n,
               double* __restrict__ psum) {
    __shared__ double sp[kThreads];
    const int s = blockIdx.x;
    const int st = seg_start[s], len = seg_len[s];
    double ap = 0.0;
    for (int t = threadIdx.x; t < len; t += blockDim.x) {
        const int i = perm[st + t];
        const int z = i % n, y = (i / n) % n, x = i / (n * n);
        const float2 v = dk[i];
        const float p2 = fmaf(v.x, v.x, v.y * v.y) * (inv_w2[x] * inv_w2[y] * inv_w2[z]);
        ap += (double)p2;
    }
    sp[threadIdx.x] = ap;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sp[threadIdx.x] += sp[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) psum[s] = sp[0];
}

// Per shell: add its segments in order; |k| means come from the table
// made at creation (they do not depend on the particles).
__global__ void k_pm_power_final(int nb, const int* __restrict__ bin_seg0, const int* __restrict__ bin_modes,
                                 const double* __restrict__ psum, const double* __restrict__ kmean_tab,
                                 double pnorm, double* __restrict__ k_mean, double* __restrict__ power,
                                 long long* __restrict__ modes) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    double p = 0.0;
    for (int s = bin_seg0[b]; s < bin_seg0[b + 1]; ++s) p += psum[s];
    const long long m = bin_modes[b];
    if (k_mean) k_mean[b] = kmean_tab[b];
    if (power) power[b] = m ? pnorm * p / (double)m : NAN;
    if (modes) modes[b] = m;
}

// Spectrum of two acceleration components packed as one complex field:
// out = A_a(k) + i A_b(k), A(k) = i k G(k) C(k), C = nbar * delta_k, with
// the inverse-transform normalisation 1/(n^3 D^3) folded in.  For a single
// component pass b = -1.
__global__ void k_pm_green(const float2* __restrict__ dk, int n, long long n3, float kf, float sig2,
                           const float* __restrict__ inv_w2, float coef, int ca, int cb,
                           float2* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    const int z = (int)(i % n), y = (int)((i / n) % n), x = (int)(i / ((long long)n * n));
    const int h = n >> 1;
    const int mx = x < h ? x : x - n, my = y < h ? y : y - n, mz = z < h ? z : z - n;
    const float kx = kf * mx, ky = kf * my, kz = kf * mz;
    const float k2 = kx * kx + ky * ky + kz * kz;
    if (i == 0) {
        out[i] = make_float2(0.f, 0.f);
        return;
    }
    const float g = coef * expf(-k2 * sig2) / k2 * inv_w2[x] * inv_w2[y] * inv_w2[z];
    const float gx = x == h ? 0.f : kx, gy = y == h ? 0.f : ky, gz = z == h ? 0.f : kz;
    const float ka = ca == 0 ? gx : (ca == 1 ? gy : gz);
    const float kb = cb == 0 ? gx : (cb == 1 ? gy : gz);
    const float2 c = dk[i];
    // i k_a g c = (-k_a g c.y, k_a g c.x)
    const float2 A = make_float2(-ka * g * c.y, ka * g * c.x);
    float2 r = A;
    if (cb >= 0) {
        const float2 B = make_float2(-kb * g * c.y, kb * g * c.x);
        r = make_float2(A.x - B.y, A.y + B.x);   // A + i B
    }
    out[i] = r;
}

// Real (and imaginary) parts of the inverse transform into the float4
// acceleration grid.
__global__ void k_pm_extract(const float2* __restrict__ w, long long n3, int ca, int cb,
                             float4* __restrict__ accg) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    const float2 v = w[i];
    float4 a = accg[i];
    if (ca == 0) a.x = v.x; else if (ca == 1) a.y = v.x; else a.z = v.x;
    if (cb == 0) a.x = v.y; else if (cb == 1) a.y = v.y; else if (cb == 2) a.z = v.y;
    a.w = 0.f;
    accg[i] = a;
}

__global__ void __launch_bounds__(kThreads)
k_cic_interp(const double* __restrict__ pos, long long np, double box, double inv_d, int inv_s, int n,
             const float4* __restrict__ accg, float4* __restrict__ acc, int accumulate) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    int c[3];
    float f[3];
    cic_cell(pos, i, box, inv_d, inv_s, n, c, f);
    float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
        const float wx = dx ? f[0] : 1.f - f[0];
        const long long ix = c[0] + dx == n ? 0 : c[0] + dx;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const float wxy = wx * (dy ? f[1] : 1.f - f[1]);
            const long long iy = c[1] + dy == n ? 0 : c[1] + dy;
#pragma unroll
            for (int dz = 0; dz < 2; ++dz) {
                const float w = wxy * (dz ? f[2] : 1.f - f[2]);
                const long long iz = c[2] + dz == n ? 0 : c[2] + dz;
                const float4 g = __ldg(&accg[(ix * n + iy) * n + iz]);
                ax = fmaf(w, g.x, ax);
                ay = fmaf(w, g.y, ay);
                az = fmaf(w, g.z, az);
            }
        }
    }
    float4 o = accumulate ? acc[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    o.x += ax;
    o.y += ay;
    o.z += az;
    acc[i] = o;
}

}  // namespace

struct sr_pm {
    int n = 0;
    int logn = 0;
    long long n3 = 0;
    double box = 0.0;
    double sigma = 0.0;
    long long n_max = 0;
    int fixed_shift = 0;
    unsigned long long* fx = nullptr;   // fixed-point CIC counts
    float2* dk = nullptr;               // FFT of delta
    float2* work = nullptr;             // inverse-transform scratch
    float4* accg = nullptr;             // acceleration grid
    float2* tw = nullptr;               // exp(-2 pi i k / n), k < n
    float* inv_w2 = nullptr;            // 1 / sinc^4(pi m / n) per axis index
    double* kmean = nullptr;            // mean |k| per shell
    int* perm = nullptr;                // modes sorted by shell (shells 1..n/2 first)
    int* seg_start = nullptr;
    int* seg_len = nullptr;
    int* bin_seg0 = nullptr;            // first segment of each shell (n/2 + 1)
    int* bin_modes = nullptr;
    double* psum = nullptr;
    int n_seg = 0;
    long long last_np = 0;
    bool deposited = false;
    bool transformed = false;
    bool accel_valid = false;
};

namespace {
// s with n / L = 2^s, or kNotPow2 (the CIC kernels' integer path needs it).
int mesh_exp(const sr_pm* pm) {
    int ex = 0;
    const double m = std::frexp(pm->n / pm->box, &ex);
    return m == 0.5 ? ex - 1 : kNotPow2;
}
}  // namespace

namespace {

template <class T>
int dalloc(T** p, long long count, const char* what) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)(count > 0 ? count : 1));
    if (e != cudaSuccess) return sr::cuda_fail(e, what);
    return SR_OK;
}

int pm_free(sr_pm* p) {
    void* bufs[] = {p->fx, p->dk, p->work, p->accg, p->tw, p->inv_w2, p->kmean, p->perm, p->seg_start,
                    p->seg_len, p->bin_seg0, p->bin_modes, p->psum};
    for (void* b : bufs) cudaFree(b);
    delete p;
    return SR_OK;
}

template <int N, bool INV>
int fft3_n(float2* data, const float2* tw, cudaStream_t st) {
    const int T = fft_pencils(N);
    const unsigned threads = (unsigned)(T * (N / 16));
    const unsigned blocks = (unsigned)((long long)N * N / T);
    for (int axis = 2; axis >= 0; --axis) {
        k_fft_pass<N, INV><<<blocks, threads, fft_smem(N), st>>>(data, axis, T, tw);
        SR_LAUNCH_CHECK("k_fft_pass");
    }
    return SR_OK;
}

template <bool INV>
int fft3_dir(int n, float2* data, const float2* tw, cudaStream_t st) {
    switch (n) {
        case 16: return fft3_n<16, INV>(data, tw, st);
        case 32: return fft3_n<32, INV>(data, tw, st);
        case 64: return fft3_n<64, INV>(data, tw, st);
        case 128: return fft3_n<128, INV>(data, tw, st);
        case 256: return fft3_n<256, INV>(data, tw, st);
        case 512: return fft3_n<512, INV>(data, tw, st);
        case 1024: return fft3_n<1024, INV>(data, tw, st);
        default: return sr::set_error(SR_ERR_ARG, "fft: unsupported size");
    }
}

int fft3(sr_pm* p, float2* data, float sign, cudaStream_t st) {
    return sign < 0.f ? fft3_dir<false>(p->n, data, p->tw, st) : fft3_dir<true>(p->n, data, p->tw, st);
}

template <int N, bool INV>
cudaError_t fft_attr() {
    return cudaFuncSetAttribute(k_fft_pass<N, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem(N));
}

cudaError_t fft_attrs(int n) {
    switch (n) {
        case 16: { cudaError_t e = fft_attr<16, false>(); return e ? e : fft_attr<16, true>(); }
        case 32: { cudaError_t e = fft_attr<32, false>(); return e ? e : fft_attr<32, true>(); }
        case 64: { cudaError_t e = fft_attr<64, false>(); return e ? e : fft_attr<64, true>(); }
        case 128: { cudaError_t e = fft_attr<128, false>(); return e ? e : fft_attr<128, true>(); }
        case 256: { cudaError_t e = fft_attr<256, false>(); return e ? e : fft_attr<256, true>(); }
        case 512: { cudaError_t e = fft_attr<512, false>(); return e ? e : fft_attr<512, true>(); }
        default: { cudaError_t e = fft_attr<1024, false>(); return e ? e : fft_attr<1024, true>(); }
    }
}

// Mode permutation by shell and the segment tables (once, synchronous).
int build_shells(sr_pm* p) {
    const long long n3 = p->n3;
    unsigned long long* keys[2] = {nullptr, nullptr};
    int* vals[2] = {nullptr, nullptr};
    sr::RadixScratch rs;
    int rc = SR_OK;
    for (int k = 0; k < 2 && !rc; ++k) {
        rc = dalloc(&keys[k], n3, "sr_pm_create keys");
        if (!rc) rc = dalloc(&vals[k], n3, "sr_pm_create vals");
    }
    if (!rc) rc = sr::radix_alloc(rs, n3);
    int which = 0;
    if (!rc) {
        k_pm_mode_keys<<<grid_for(n3, kThreads), kThreads>>>(p->n, n3, keys[0], vals[0]);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = sr::cuda_fail(e, "k_pm_mode_keys");
    }
    int kb = 1;
    while ((1 << kb) <= p->n / 2 + 1) ++kb;
    if (!rc) rc = sr::radix_sort_pairs(keys, vals, (int)n3, kb, rs, nullptr, &which);
    // modes and mean |k| per shell, on the host with the same classification
    std::vector<int> modes(p->n / 2 + 2, 0);
    std::vector<double> ksum(p->n / 2 + 2, 0.0);
    if (!rc) {
        const int n = p->n, h = n / 2;
        const double kf = 2.0 * 3.14159265358979323846 / p->box;
        std::vector<long long> sq(n);
        for (int i = 0; i < n; ++i) {
            const long long m = i < h ? i : i - n;
            sq[i] = m * m;
        }
        for (int x = 0; x < n; ++x)
            for (int y = 0; y < n; ++y)
                for (int z = 0; z < n; ++z) {
                    const double r = std::sqrt((double)(sq[x] + sq[y] + sq[z]));
                    const int b = (int)std::rint(r);
                    const int sh = (b >= 1 && b <= h) ? b : h + 1;
                    modes[sh]++;
                    ksum[sh] += kf * r;
                }
    }
    if (!rc) {
        const int nb = p->n / 2;
        std::vector<int> seg_start, seg_len, bin_seg0(nb + 1, 0);
        long long off = 0;
        for (int b = 1; b <= nb; ++b) {
            bin_seg0[b - 1] = (int)seg_start.size();
            for (int s = 0; s < modes[b]; s += kSegModes) {
                seg_start.push_back((int)(off + s));
                seg_len.push_back(std::min(kSegModes, modes[b] - s));
            }
            off += modes[b];
        }
        bin_seg0[nb] = (int)seg_start.size();
        p->n_seg = (int)seg_start.size();
        std::vector<int> bm(modes.begin() + 1, modes.begin() + 1 + nb);
        std::vector<double> km(nb);
        for (int b = 1; b <= nb; ++b) km[b - 1] = ksum[b] / modes[b];
        rc = dalloc(&p->perm, n3, "sr_pm_create perm");
        if (!rc) rc = dalloc(&p->seg_start, p->n_seg, "seg_start");
        if (!rc) rc = dalloc(&p->seg_len, p->n_seg, "seg_len");
        if (!rc) rc = dalloc(&p->bin_seg0, nb + 1, "bin_seg0");
        if (!rc) rc = dalloc(&p->bin_modes, nb, "bin_modes");
        if (!rc) rc = dalloc(&p->psum, p->n_seg, "psum");
        if (!rc) rc = dalloc(&p->kmean, nb, "kmean");
        cudaError_t e = cudaSuccess;
        if (!rc) e = cudaMemcpy(p->perm, vals[which], sizeof(int) * n3, cudaMemcpyDeviceToDevice);
        if (!rc && e == cudaSuccess)
            e = cudaMemcpy(p->seg_start, seg_start.data(), sizeof(int) * p->n_seg, cudaMemcpyHostToDevice);
        if (!rc && e == cudaSuccess)
            e = cudaMemcpy(p->seg_len, seg_len.data(), sizeof(int) * p->n_seg, cudaMemcpyHostToDevice);
        if (!rc && e == cudaSuccess)
            e = cudaMemcpy(p->bin_seg0, bin_seg0.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice);
        if (!rc && e == cudaSuccess) e = cudaMemcpy(p->bin_modes, bm.data(), sizeof(int) * nb, cudaMemcpyHostToDevice);
        if (!rc && e == cudaSuccess) e = cudaMemcpy(p->kmean, km.data(), sizeof(double) * nb, cudaMemcpyHostToDevice);
        if (!rc && e != cudaSuccess) rc = sr::cuda_fail(e, "sr_pm_create tables");
    }
    for (int k = 0; k < 2; ++k) {
        cudaFree(keys[k]);
        cudaFree(vals[k]);
    }
    sr::radix_free(rs);
    return rc;
}

}  // namespace

extern "C" {

int sr_pm_create(int n_grid, double box, double sigma, int64_t n_max, sr_pm** out) {
    if (!out) return sr::set_error(SR_ERR_ARG, "sr_pm_create: null out");
    *out = nullptr;
    int logn = 0;
    while ((1 << logn) < n_grid) ++logn;
    if (n_grid < 16 || n_grid > 1024 || (1 << logn) != n_grid)
        return sr::set_error(SR_ERR_ARG, "sr_pm_create: n_grid must be a power of two in [16, 1024]");
    if (!(box > 0.0) || !std::isfinite(box) || !(sigma >= 0.0) || !std::isfinite(sigma))
        return sr::set_error(SR_ERR_ARG, "sr_pm_create: box must be > 0 and sigma >= 0");
    if (n_max < 1 || n_max > 2147483647LL) return sr::set_error(SR_ERR_ARG, "sr_pm_create: bad n_max");
    sr_pm* p = new sr_pm();
    p->n = n_grid;
    p->logn = logn;
    p->n3 = (long long)n_grid * n_grid * n_grid;
    p->box = box;
    p->sigma = sigma;
    p->n_max = n_max;
    // no cell can hold more than n_max particles: n_max 2^S < 2^62
    int bits = 0;
    while ((1LL << bits) <= n_max) ++bits;
    p->fixed_shift = 62 - bits;
    if (p->fixed_shift > 52) p->fixed_shift = 52;
    int rc = dalloc(&p->fx, p->n3, "sr_pm_create grid");
    if (!rc) rc = dalloc(&p->dk, p->n3, "sr_pm_create dk");
    if (!rc) rc = dalloc(&p->work, p->n3, "sr_pm_create work");
    if (!rc) rc = dalloc(&p->accg, p->n3, "sr_pm_create accel grid");
    if (!rc) rc = dalloc(&p->tw, n_grid, "sr_pm_create twiddles");
    if (!rc) rc = dalloc(&p->inv_w2, n_grid, "sr_pm_create window");
    if (!rc) {
        std::vector<float2> tw(n_grid);
        const double pi = 3.14159265358979323846;
        for (int k = 0; k < n_grid; ++k) {
            const double a = -2.0 * pi * k / n_grid;
            tw[k] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
        std::vector<float> iw(n_grid);
        for (int i = 0; i < n_grid; ++i) {
            const int m = i < n_grid / 2 ? i : i - n_grid;
            const double hh = pi * m / n_grid;
            const double s = m == 0 ? 1.0 : std::sin(hh) / hh;
            iw[i] = (float)(1.0 / (s * s * s * s));
        }
        cudaError_t e = cudaMemcpy(p->tw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(p->inv_w2, iw.data(), sizeof(float) * n_grid, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = sr::cuda_fail(e, "sr_pm_create tables");
    }
    if (!rc) {
        cudaError_t e = fft_attrs(n_grid);
        if (e != cudaSuccess) rc = sr::cuda_fail(e, "sr_pm_create fft smem");
    }
    if (!rc) rc = build_shells(p);
    if (rc) {
        pm_free(p);
        return rc;
    }
    *out = p;
    return SR_OK;
}

int sr_pm_destroy(sr_pm* pm) {
    if (!pm) return SR_OK;
    return pm_free(pm);
}

int sr_pm_deposit(sr_pm* pm, const double* pos, int64_t n, void* stream) {
    if (!pm || !pos) return sr::set_error(SR_ERR_ARG, "sr_pm_deposit: null workspace or pos");
    if (n < 1) return sr::set_error(SR_ERR_ARG, "sr_pm_deposit: n must be >= 1");
    if (n > pm->n_max) return sr::set_error(SR_ERR_CAPACITY, "sr_pm_deposit: n above n_max");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double scale = std::ldexp(1.0, pm->fixed_shift);
    SR_CUDA_CHECK(cudaMemsetAsync(pm->fx, 0, sizeof(unsigned long long) * (size_t)pm->n3, st));
    k_cic_deposit<<<grid_for(n, kThreads), kThreads, 0, st>>>(pos, (long long)n, pm->box, pm->n / pm->box,
                                                              mesh_exp(pm), pm->n, (float)scale, pm->fx);
    SR_LAUNCH_CHECK("k_cic_deposit");
    pm->last_np = n;
    pm->deposited = true;
    pm->transformed = false;
    pm->accel_valid = false;
    return SR_OK;
}

int sr_pm_deposit_binned(sr_pm* pm, const sr_plan* plan, const double* pos, int64_t n, void* stream) {
    if (!pm || !plan || !pos) return sr::set_error(SR_ERR_ARG, "sr_pm_deposit_binned: null argument");
    if (!plan->binned) return sr::set_error(SR_ERR_STATE, "sr_pm_deposit_binned: the plan holds no binning");
    if (plan->n_vol != 1) return sr::set_error(SR_ERR_ARG, "sr_pm_deposit_binned: a one-volume plan is needed");
    if (n != plan->n_binned) return sr::set_error(SR_ERR_ARG, "sr_pm_deposit_binned: n differs from the plan's binning");
    if (n < 1) return sr::set_error(SR_ERR_ARG, "sr_pm_deposit_binned: n must be >= 1");
    if (n > pm->n_max) return sr::set_error(SR_ERR_CAPACITY, "sr_pm_deposit_binned: n above n_max");
    const sr::VolDev& V = plan->vols_h[0];
    if (V.box != pm->box) return sr::set_error(SR_ERR_ARG, "sr_pm_deposit_binned: the plan's box differs");
    // the tile: a binning cell's mesh points plus one layer per axis
    const int n_c = V.n_c;
    const double ratio = (double)pm->n / (double)n_c;          // mesh cells per binning cell
    const int wt = (int)std::ceil(ratio) + 2;
    if ((long long)wt * wt * wt > kDepTileMax) return sr_pm_deposit(pm, pos, n, stream);   // cells too coarse
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double scale = std::ldexp(1.0, pm->fixed_shift);
    SR_CUDA_CHECK(cudaMemsetAsync(pm->fx, 0, sizeof(unsigned long long) * (size_t)pm->n3, st));
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (plan->max_chunks + kDepWarps - 1) / kDepWarps;
    const int blocks = (int)std::max(1LL, std::min(want, 8LL * sms));
    k_cic_deposit_chunks<<<blocks, kDepWarps * 32, 0, st>>>(
        pos, plan->ccs, (int)plan->total_cells, plan->chunk_span, plan->slot_idx, 32 * plan->chunk_k, n_c, ratio,
        wt, pm->box, pm->n / pm->box, mesh_exp(pm), pm->n, (float)scale, pm->fx);
    SR_LAUNCH_CHECK("k_cic_deposit_chunks");
    pm->last_np = n;
    pm->deposited = true;
    pm->transformed = false;
    pm->accel_valid = false;
    return SR_OK;
}

int sr_pm_transform(sr_pm* pm, void* stream) {
    if (!pm) return sr::set_error(SR_ERR_ARG, "sr_pm_transform: null workspace");
    if (!pm->deposited) return sr::set_error(SR_ERR_STATE, "sr_pm_transform: call sr_pm_deposit first");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double inv_nbar = (double)pm->n3 / (double)pm->last_np;
    k_pm_delta<<<grid_for(pm->n3, kThreads), kThreads, 0, st>>>(pm->fx, pm->n3, std::ldexp(1.0, -pm->fixed_shift),
                                                                inv_nbar, pm->dk);
    SR_LAUNCH_CHECK("k_pm_delta");
    int rc = fft3(pm, pm->dk, -1.f, st);
    if (rc) return rc;
    pm->transformed = true;
    pm->accel_valid = false;
    return SR_OK;
}

int sr_pm_power(sr_pm* pm, double* k_mean, double* power, int64_t* modes, void* stream) {
    if (!pm) return sr::set_error(SR_ERR_ARG, "sr_pm_power: null workspace");
    if (!pm->transformed) return sr::set_error(SR_ERR_STATE, "sr_pm_power: call sr_pm_transform first");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double n6 = (double)pm->n3 * (double)pm->n3;
    const double pnorm = pm->box * pm->box * pm->box / n6;
    k_pm_power_seg<<<pm->n_seg, kThreads, 0, st>>>(pm->dk, pm->perm, pm->seg_start, pm->seg_len, pm->inv_w2, pm->n,
                                                   pm->psum);
    SR_LAUNCH_CHECK("k_pm_power_seg");
    const int nb = pm->n / 2;
    k_pm_power_final<<<grid_for(nb, 128), 128, 0, st>>>(nb, pm->bin_seg0, pm->bin_modes, pm->psum, pm->kmean, pnorm,
                                                        k_mean, power, reinterpret_cast<long long*>(modes));
    SR_LAUNCH_CHECK("k_pm_power_final");
    return SR_OK;
}

int sr_pm_force(sr_pm* pm, const double* pos, int64_t n, float* acc, int accumulate, void* stream) {
    if (!pm || !pos || !acc) return sr::set_error(SR_ERR_ARG, "sr_pm_force: null argument");
    if (!pm->transformed) return sr::set_error(SR_ERR_STATE, "sr_pm_force: call sr_pm_transform first");
    if (n < 1) return sr::set_error(SR_ERR_ARG, "sr_pm_force: n must be >= 1");
    if (n > pm->n_max) return sr::set_error(SR_ERR_CAPACITY, "sr_pm_force: n above n_max");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!pm->accel_valid) {
        const double d = pm->box / pm->n;
        const double nbar = (double)pm->last_np / (double)pm->n3;
        // C = nbar delta_k; a(x) = ifft(.) / D^3 = (1 / (n^3 D^3)) sum_k ...
        const float coef = (float)(4.0 * 3.14159265358979323846 * nbar / ((double)pm->n3 * d * d * d));
        const float kf = (float)(2.0 * 3.14159265358979323846 / pm->box);
        const float sig2 = (float)(pm->sigma * pm->sigma);
        const unsigned g = grid_for(pm->n3, kThreads);
        k_pm_green<<<g, kThreads, 0, st>>>(pm->dk, pm->n, pm->n3, kf, sig2, pm->inv_w2, coef, 0, 1, pm->work);
        SR_LAUNCH_CHECK("k_pm_green");
        int rc = fft3(pm, pm->work, 1.f, st);
        if (rc) return rc;
        k_pm_extract<<<g, kThreads, 0, st>>>(pm->work, pm->n3, 0, 1, pm->accg);
        SR_LAUNCH_CHECK("k_pm_extract");
        k_pm_green<<<g, kThreads, 0, st>>>(pm->dk, pm->n, pm->n3, kf, sig2, pm->inv_w2, coef, 2, -1, pm->work);
        SR_LAUNCH_CHECK("k_pm_green");
        rc = fft3(pm, pm->work, 1.f, st);
        if (rc) return rc;
        k_pm_extract<<<g, kThreads, 0, st>>>(pm->work, pm->n3, 2, -1, pm->accg);
        SR_LAUNCH_CHECK("k_pm_extract");
        pm->accel_valid = true;
    }
    k_cic_interp<<<grid_for(n, kThreads), kThreads, 0, st>>>(pos, (long long)n, pm->box, pm->n / pm->box,
                                                             mesh_exp(pm), pm->n, pm->accg,
                                                             reinterpret_cast<float4*>(acc), accumulate);
    SR_LAUNCH_CHECK("k_cic_interp");
    return SR_OK;
}

int sr_pm_fft(sr_pm* pm, float* data, int inverse, void* stream) {
    if (!pm || !data) return sr::set_error(SR_ERR_ARG, "sr_pm_fft: null argument");
    return fft3(pm, reinterpret_cast<float2*>(data), inverse ? 1.f : -1.f, static_cast<cudaStream_t>(stream));
}

int sr_pm_copy(sr_pm* pm, int what, void* dst, void* stream) {
    if (!pm || !dst) return sr::set_error(SR_ERR_ARG, "sr_pm_copy: null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (what == SR_PM_EXPORT_COUNTS || what == SR_PM_EXPORT_DELTA_K) {
        if (!pm->deposited || (what == SR_PM_EXPORT_DELTA_K && !pm->transformed))
            return sr::set_error(SR_ERR_STATE, "sr_pm_copy: nothing deposited or transformed");
        if (what == SR_PM_EXPORT_COUNTS) {
            k_pm_counts<<<grid_for(pm->n3, kThreads), kThreads, 0, st>>>(pm->fx, pm->n3,
                                                                         std::ldexp(1.0, -pm->fixed_shift),
                                                                         static_cast<double*>(dst));
            SR_LAUNCH_CHECK("k_pm_counts");
        } else {
            SR_CUDA_CHECK(cudaMemcpyAsync(dst, pm->dk, sizeof(float2) * (size_t)pm->n3, cudaMemcpyDeviceToDevice, st));
        }
        return SR_OK;
    }
    if (what == SR_PM_EXPORT_ACCEL) {
        if (!pm->accel_valid) return sr::set_error(SR_ERR_STATE, "sr_pm_copy: no acceleration grid yet");
        SR_CUDA_CHECK(cudaMemcpyAsync(dst, pm->accg, sizeof(float4) * (size_t)pm->n3, cudaMemcpyDeviceToDevice, st));
        return SR_OK;
    }
    return sr::set_error(SR_ERR_ARG, "sr_pm_copy: unknown selector");
}

}  // extern "C"
