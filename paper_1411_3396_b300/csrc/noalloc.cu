// Run-health invariants without a plan and without any device allocation.
//
// sr_invariants needs a plan because its two-stage reduction keeps partial
// sums in plan-owned device memory.  Some callers cannot create that memory:
// code that runs while another component owns the whole device memory
// budget (a pooling allocator that must not be bypassed), monitoring hooks
// called from inside a time-stepping loop that is not allowed to allocate or
// to synchronise the device (cudaMalloc may do both), and tools that only
// want to check momentum or energy of buffers they were handed, without
// building the binning workspace of a plan.  sr_invariants_noalloc serves
// them: its partial sums live in a fixed file-scope device array that is
// loaded with the library, so the call itself never allocates.
#include <mutex>
#include <unordered_map>

#include "sr_internal.h"

namespace sr {
namespace {

constexpr int kNaThreads = 256;
constexpr long long kNaRowsPerBlock = 16384;       // rows reduced by one block
constexpr int kNaMaxBlocks = 4096;                  // partial-sum slots
constexpr long long kNaMaxRows = kNaRowsPerBlock * kNaMaxBlocks;   // 67,108,864 rows

// Partial sums, 7 doubles per block: 4096 x 7 x 8 B = 224 KiB, held by every
// device that loads the library until the process exits.
static __device__ __align__(256) double g_na_partials[kNaMaxBlocks * 7];

std::mutex g_na_mutex;
std::unordered_map<unsigned long long, double*> g_na_addr;   // context id -> address of g_na_partials

// Driver calls reached through the runtime's entry-point query, so the
// library needs no link-time dependency on the driver library.
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);

// Process-unique id of the current CUDA context (cuCtxGetId: ids are never
// reused, unlike context handles and device ordinals).  Called with
// g_na_mutex held.
int na_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !f)
            return set_error(SR_ERR_CUDA, "driver entry point cuCtxGetCurrent not found");
        void* g = nullptr;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !g)
            return set_error(SR_ERR_CUDA, "driver entry point cuCtxGetId not found");
        get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        get_id = reinterpret_cast<CtxGetIdFn>(g);
    }
    void* ctx = nullptr;
    if (get_current(&ctx) != 0) return set_error(SR_ERR_CUDA, "cuCtxGetCurrent failed");
    if (!ctx) {
        // no context bound to this thread yet: bind the current device's
        // primary context, as the runtime's first call would
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
        e = cudaSetDevice(dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
        if (get_current(&ctx) != 0 || !ctx) return set_error(SR_ERR_CUDA, "no current CUDA context");
    }
    if (get_id(ctx, id) != 0) return set_error(SR_ERR_CUDA, "cuCtxGetId failed");
    return SR_OK;
}

// Device address of g_na_partials in the current context, looked up once
// per context (the symbol name is only a host-side handle, not a device
// address).  Keyed by the context's id, so a device reset, which makes a new
// context, also makes a new lookup instead of reusing a stale address.
int na_scratch(double** out) {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    unsigned long long id = 0;
    const int rc = na_context_id(&id);
    if (rc) return rc;
    auto it = g_na_addr.find(id);
    if (it != g_na_addr.end()) {
        *out = it->second;
        return SR_OK;
    }
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_na_partials);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_na_partials)");
    g_na_addr[id] = static_cast<double*>(ptr);
    *out = static_cast<double*>(ptr);
    return SR_OK;
}

// Block b sums rows [b R, min(n, (b+1) R)) and always writes its 7 slots, so
// a call never reads partials left by an earlier call.
__global__ void __launch_bounds__(kNaThreads) k_na_partial(long long n, const float4* __restrict__ vel,
                                                           const float4* __restrict__ acc,
                                                           double* __restrict__ partials) {
    __shared__ double sh[7][kNaThreads];
    const long long b0 = (long long)blockIdx.x * kNaRowsPerBlock;
    const long long b1 = b0 + kNaRowsPerBlock < n ? b0 + kNaRowsPerBlock : n;
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (long long i = b0 + threadIdx.x; i < b1; i += kNaThreads) {
        if (vel) {
            const float4 v = vel[i];
            s[0] += v.x; s[1] += v.y; s[2] += v.z;
            s[6] += 0.5 * ((double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z);
        }
        if (acc) {
            const float4 a = acc[i];
            s[3] += a.x; s[4] += a.y; s[5] += a.z;
        }
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) sh[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = kNaThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int k = 0; k < 7; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x < 7) partials[(long long)blockIdx.x * 7 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_na_final(const double* __restrict__ partials, int blocks, double* __restrict__ out) {
    if (threadIdx.x < 7) {
        double s = 0.0;
        for (int b = 0; b < blocks; ++b) s += partials[(long long)b * 7 + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

}  // namespace
}  // namespace sr

using namespace sr;

extern "C" int sr_invariants_noalloc(int64_t n, const float* vel, const float* acc, double* out, void* stream) {
    if (!out) return set_error(SR_ERR_ARG, "out is null");
    if (n < 0) return set_error(SR_ERR_ARG, "n must be >= 0");
    if (n > kNaMaxRows)
        return set_error(SR_ERR_CAPACITY,
                         "sr_invariants_noalloc: n exceeds the 67,108,864-row limit of its static scratch "
                         "(use sr_invariants with a plan)");
    double* scratch = nullptr;
    int rc = na_scratch(&scratch);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int blocks = (int)((n + kNaRowsPerBlock - 1) / kNaRowsPerBlock);
    if (blocks < 1) blocks = 1;
    k_na_partial<<<blocks, kNaThreads, 0, st>>>(n, reinterpret_cast<const float4*>(vel),
                                                reinterpret_cast<const float4*>(acc), scratch);
    SR_LAUNCH_CHECK("k_na_partial");
    k_na_final<<<1, 32, 0, st>>>(scratch, blocks, out);
    SR_LAUNCH_CHECK("k_na_final");
    return SR_OK;
}
