// Elementwise kernels that close the step: the kick v += a dt, the drift
// x <- fold(x + v dt), and deterministic binary64 global sums (momentum,
// net force, kinetic energy) used as run-health invariants.
#include "sr_internal.h"

namespace sr {
namespace {

__global__ void __launch_bounds__(256) k_kick(long long n, const float4* __restrict__ acc,
                                              float4* __restrict__ vel, float dt) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float4 a = acc[i];
        float4 v = vel[i];
        v.x = fmaf(a.x, dt, v.x);
        v.y = fmaf(a.y, dt, v.y);
        v.z = fmaf(a.z, dt, v.z);
        vel[i] = v;
    }
}

__global__ void __launch_bounds__(256) k_drift(long long n, double* __restrict__ pos,
                                               const float4* __restrict__ vel, double dt,
                                               const VolDev* __restrict__ vols,
                                               const long long* __restrict__ part_start, int n_vol) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int lo = 0, hi = n_vol;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (part_start[mid] <= i) lo = mid; else hi = mid;
        }
        const double box = vols[lo].box;
        const float4 v = vel[i];
        const double vv[3] = {(double)v.x, (double)v.y, (double)v.z};
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            // x + v dt as two correctly rounded operations (no fused multiply-add)
            double x = __dadd_rn(pos[3 * i + ax], __dmul_rn(vv[ax], dt));
            if (x < 0.0) x = x + box;
            if (x >= box) x = x - box;
            pos[3 * i + ax] = x;
        }
    }
}

// Stage 1: each block reduces a fixed, contiguous range of rows (so the
// association order depends only on n), writing 7 partial sums.
// Error-free transformations in binary32 (no contraction: explicit
// round-to-nearest intrinsics): s + e == a + b exactly (TwoSum, Knuth), and
// p + e == a * a exactly (TwoProduct by an FMA).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) += x for a sum held as an unevaluated pair of binary32 numbers:
// TwoSum of hi and x, its exact error added to lo, then the pair
// renormalised (Fast2Sum of the sum and the error terms), so that lo stays
// below about an ulp of hi and the pair keeps close to 48 significant bits
// however many terms it takes.
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
    float s, e;
    two_sum(hi, x, s, e);
    e = __fadd_rn(e, lo);
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

constexpr int kInvRows = 4;        // rows whose loads a thread issues together

// Block partial sums of the seven invariants.  B300 runs binary64 at 1/64
// of its binary32 rate, and binary64 adds per term bound this kernel (about
// 20 binary64 operations per row when every term was added in binary64,
// 3.5 when binary32 pairs were folded into binary64 every 8 rows).  Each
// thread now sums all of its rows as renormalised binary32 pairs, the
// squares split exactly by an FMA, and converts its seven pairs to binary64
// once at the end.  An emulation of the scheme on random sets of mixed
// magnitudes (tests/test_invariants_scheme.py) bounds its error against
// the exact sum.
__global__ void __launch_bounds__(256, 4) k_inv_partial(long long n, const float4* __restrict__ vel,
                                                     const float4* __restrict__ acc,
                                                     double* __restrict__ partials) {
    __shared__ double sh[7][256];
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long b0 = (long long)blockIdx.x * per;
    const long long b1 = b0 + per < n ? b0 + per : n;
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    float hi[7] = {0, 0, 0, 0, 0, 0, 0}, lo[7] = {0, 0, 0, 0, 0, 0, 0};
    // rows in the same order as one row per loop trip, with the loads of
    // kInvRows rows issued together (the sums' dependency chains would
    // otherwise leave one row's loads in flight per thread)
    for (long long i0 = b0 + threadIdx.x; i0 < b1; i0 += (long long)kInvRows * blockDim.x) {
        float4 vr[kInvRows], ar[kInvRows];
#pragma unroll
        for (int r = 0; r < kInvRows; ++r) {
            const long long i = i0 + (long long)r * blockDim.x;
            vr[r] = vel && i < b1 ? vel[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            ar[r] = acc && i < b1 ? acc[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < kInvRows; ++r) {
            if (i0 + (long long)r * blockDim.x >= b1) break;
            if (vel) {
                const float4 v = vr[r];
                df_add(hi[0], lo[0], v.x);
                df_add(hi[1], lo[1], v.y);
                df_add(hi[2], lo[2], v.z);
                const float px = __fmul_rn(v.x, v.x), py = __fmul_rn(v.y, v.y), pz = __fmul_rn(v.z, v.z);
                df_add(hi[6], lo[6], px);
                df_add(hi[6], lo[6], py);
                df_add(hi[6], lo[6], pz);
                // the products' exact rounding errors (tiny: one plain add each)
                lo[6] = __fadd_rn(lo[6], __fadd_rn(__fmaf_rn(v.x, v.x, -px),
                                                   __fadd_rn(__fmaf_rn(v.y, v.y, -py), __fmaf_rn(v.z, v.z, -pz))));
            }
            if (acc) {
                const float4 a = ar[r];
                df_add(hi[3], lo[3], a.x);
                df_add(hi[4], lo[4], a.y);
                df_add(hi[5], lo[5], a.z);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 7; ++c) s[c] += (double)hi[c] + (double)lo[c];
    s[6] *= 0.5;
#pragma unroll
    for (int k = 0; k < 7; ++k) sh[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int k = 0; k < 7; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x < 7) partials[(long long)blockIdx.x * 7 + threadIdx.x] = sh[threadIdx.x][0];
}

// The blocks' partial sums added by one block: each thread sums a fixed
// strided subset, then a fixed tree; deterministic (a single thread walking
// all partials in order was latency-bound: some 1,200 dependent binary64
// adds per sum).
__global__ void __launch_bounds__(256) k_inv_final(const double* __restrict__ partials, int blocks,
                                                   double* __restrict__ out) {
    __shared__ double sh[7][256];
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < blocks; b += blockDim.x) {
#pragma unroll
        for (int k = 0; k < 7; ++k) s[k] += partials[(long long)b * 7 + k];
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) sh[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int k = 0; k < 7; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x < 7) out[threadIdx.x] = sh[threadIdx.x][0];
}

int grid_for(long long n) {
    long long g = (n + 255) / 256;
    if (g > 148 * 16) g = 148 * 16;
    return (int)(g > 0 ? g : 1);
}

// One thread evaluates a bounds check whose condition is false, with no
// memory access behind it: exercises the error word of the bounds-checked
// build and its report by sr_plan_status (the release build records nothing).
__global__ void k_check_selftest(Counters* ctr) {
    if (!SR_BOUND(false, &ctr->check, kChkSelfTest)) return;
}

}  // namespace

int launch_kick(long long n, const float* acc, float* vel, float dt, cudaStream_t st) {
    if (n == 0) return SR_OK;
    k_kick<<<grid_for(n), 256, 0, st>>>(n, reinterpret_cast<const float4*>(acc), reinterpret_cast<float4*>(vel), dt);
    SR_LAUNCH_CHECK("k_kick");
    return SR_OK;
}

int launch_drift(sr_plan* p, double* pos, const float* vel, double dt, long long n, cudaStream_t st) {
    if (n == 0) return SR_OK;
    k_drift<<<grid_for(n), 256, 0, st>>>(n, pos, reinterpret_cast<const float4*>(vel), dt, p->vols,
                                         p->vol_part_start, p->n_vol);
    SR_LAUNCH_CHECK("k_drift");
    return SR_OK;
}

int launch_invariants(long long n, const float* vel, const float* acc, double* out, double* partials,
                      cudaStream_t st) {
    k_inv_partial<<<kInvBlocks, 256, 0, st>>>(n, reinterpret_cast<const float4*>(vel),
                                              reinterpret_cast<const float4*>(acc), partials);
    SR_LAUNCH_CHECK("k_inv_partial");
    k_inv_final<<<1, 256, 0, st>>>(partials, kInvBlocks, out);
    SR_LAUNCH_CHECK("k_inv_final");
    return SR_OK;
}

int launch_check_selftest(sr_plan* p, cudaStream_t st) {
    k_check_selftest<<<1, 1, 0, st>>>(p->ctr);
    SR_LAUNCH_CHECK("k_check_selftest");
    return SR_OK;
}

}  // namespace sr
