// C ABI: plan lifecycle, argument checking, error reporting and the thin
// wrappers that enqueue the kernels of bin.cu, force.cu, plain.cu, kick.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sr_internal.h"

namespace sr {
namespace {
thread_local std::string g_last_error;

int variant_warps(int v) { return (v >= 4 && v <= 6) || v == 10 ? 4 : 8; }
std::atomic<long long> g_launches{0};

constexpr double kSideMargin = 1.0 + 1.0 / (1 << 20);   // cell side must exceed r_c by this factor
constexpr double kCullMargin = 1.0 + 1.0 / 512.0;       // culling radius^2 relative margin

template <class T>
int dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    return SR_OK;
}

void free_plan(sr_plan* p) {
    if (!p) return;
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    cudaFree(p->vols);
    cudaFree(p->vol_part_start);
    cudaFree(p->vol_cell_base);
    for (int k = 0; k < 2; ++k) {
        cudaFree(p->keys[k]);
        cudaFree(p->vals[k]);
        cudaFree(p->lpt_keys[k]);
        cudaFree(p->lpt_vals[k]);
    }
    cudaFree(p->cell_start);
    cudaFree(p->ccs);
    cudaFree(p->chunk_span);
    cudaFree(p->chunk_meta);
    cudaFree(p->chunk_lo);
    cudaFree(p->chunk_hi);
    cudaFree(p->cost);
    cudaFree(p->slot_pos);
    cudaFree(p->slot_idx);
    cudaFree(p->slot_g);
    cudaFree(p->ctr);
    cudaFree(p->inv_partials);
    cudaFree(p->h_pos_dev);
    cudaFree(p->h_vel_dev);
    cudaFree(p->h_acc_dev);
    if (p->h_side) cudaStreamDestroy(p->h_side);
    if (p->h_fork) cudaEventDestroy(p->h_fork);
    if (p->h_join) cudaEventDestroy(p->h_join);
    for (int k = 0; k < 2; ++k) {
        cudaFree(p->q_pos[k]);
        cudaFree(p->q_vel[k]);
        cudaFree(p->q_acc[k]);
        if (p->q_loaded[k]) cudaEventDestroy(p->q_loaded[k]);
        if (p->q_computed[k]) cudaEventDestroy(p->q_computed[k]);
        if (p->q_freed[k]) cudaEventDestroy(p->q_freed[k]);
    }
    if (p->q_up) cudaStreamDestroy(p->q_up);
    if (p->q_down) cudaStreamDestroy(p->q_down);
    radix_free(p->rs_chunks);
    bin_free(p);
    delete p;
}

int check_physics(const sr_params& q) {
    if (!(q.r_c > 0) || !std::isfinite(q.r_c)) return set_error(SR_ERR_ARG, "r_c must be positive and finite");
    if (!(q.eps > 0) || !std::isfinite(q.eps)) return set_error(SR_ERR_ARG, "eps must be positive and finite");
    if (!(q.sigma > 0) || !std::isfinite(q.sigma)) return set_error(SR_ERR_ARG, "sigma must be positive and finite");
    if (q.fit_mode != SR_FIT_CONSTRAINED && q.fit_mode != SR_FIT_UNCONSTRAINED)
        return set_error(SR_ERR_ARG, "bad fit_mode");
    if (q.chunk_size != 0 && q.chunk_size != 32 && q.chunk_size != 64)
        return set_error(SR_ERR_ARG, "chunk_size must be 0, 32 or 64");
    if (q.sub_bits < 0 || q.sub_bits > 8) return set_error(SR_ERR_ARG, "sub_bits must be in 0..8");
    return SR_OK;
}

// Cells per axis when the caller leaves it open: the side nearest to 4
// (in units of the mean spacing) that is at least min_side.  Near one
// particle per unit volume sides of 3.8 to 4.3 gave the fastest pair
// kernel (the 64-volume batch: 6.77 ms against 6.89 ms with the side
// rounded up from 4 to as much as 4.6, and 7.25 ms at 3.3 to 3.7).
int default_cells(double box, double min_side) {
    const double target = min_side > 4.0 ? min_side : 4.0;
    int n_c = (int)std::floor(box / target + 0.5);
    while (n_c > 1 && box / n_c < min_side) --n_c;
    return n_c < 1 ? 1 : n_c;
}

// Geometry and unit constants of one volume.
int make_volume(const sr_params& q, const double coef[6], int b, int cell_base, VolDev* V, int* n_c_out) {
    if (!(q.box > 2.0 * q.r_c) || !std::isfinite(q.box))
        return set_error(SR_ERR_ARG, "box must be finite and exceed 2 r_c (unique minimum image)");
    const double min_side = q.r_c * kSideMargin;
    int n_c = q.n_cells;
    if (n_c == 0) n_c = default_cells(q.box, min_side);
    if (n_c < 1) return set_error(SR_ERR_ARG, "n_cells must be >= 0");
    if (q.box / n_c < min_side) return set_error(SR_ERR_ARG, "cell side L/n_cells must exceed r_c");
    if ((long long)n_c << b >= (1ll << 23)) return set_error(SR_ERR_ARG, "n_cells * 2^sub_bits too large");
    std::memset(V, 0, sizeof(VolDev));
    V->box = q.box;
    V->n_c = n_c;
    V->M = n_c << b;
    V->sub_bits = b;
    V->cell_base = cell_base;
    const double h = q.box / V->M;
    V->h = h;
    int ex = 0;
    V->h_pow2 = (std::frexp(h, &ex) == 0.5) ? 1 : 0;
    V->inv_h = 1.0 / h;        // RN(1/h): exact scale when h = 2^k, else the binning's quotient correction
    V->inv_h_exp = V->h_pow2 ? 1 - ex : 0;            // h = 2^(ex - 1)
    const double h2 = h * h;
    const double e64 = q.eps * q.eps;
    V->eps2u = (float)(e64 / h2);
    V->rc2u = (float)((q.r_c * q.r_c + e64) / h2);
    const double rcm2 = (q.r_c * q.r_c / h2) * kCullMargin;
    V->rcm2u = (float)rcm2;
    V->rcm = (float)std::sqrt(rcm2);
    V->scale_a = (float)(1.0 / h2);
    V->scale_g = (float)(1.0 / (h2 * h));
    // q(x) = h^3 p(h^2 (x - e_u)) expanded in powers of x.
    const double eu = e64 / h2;
    double qm[6];
    for (int m = 0; m <= 5; ++m) {
        double s = 0.0;
        for (int k = m; k <= 5; ++k) {
            double binom = 1.0;
            for (int t = 0; t < m; ++t) binom = binom * (k - t) / (t + 1);
            s += coef[k] * std::pow(h2, k) * binom * std::pow(-eu, k - m);
        }
        qm[m] = h2 * h * s;
    }
    for (int m = 0; m <= 5; ++m) V->nq[m] = (float)(-qm[m]);
    for (int m = 0; m < 5; ++m) V->ndq[m] = (float)(-(m + 1) * qm[m + 1]);
    *n_c_out = n_c;
    return SR_OK;
}

int build_plan(const sr_params* params, const long long* n, int n_vol, bool batch, sr_plan** out) {
    *out = nullptr;
    if (!params || !n || n_vol < 1) return set_error(SR_ERR_ARG, "null parameters");
    int rc = check_physics(params[0]);
    if (rc) return rc;
    for (int v = 1; v < n_vol; ++v) {
        const sr_params& q = params[v];
        if ((rc = check_physics(q))) return rc;
        if (q.r_c != params[0].r_c || q.eps != params[0].eps || q.sigma != params[0].sigma ||
            q.fit_mode != params[0].fit_mode || q.sub_bits != params[0].sub_bits ||
            q.chunk_size != params[0].chunk_size)
            return set_error(SR_ERR_ARG, "batch volumes must share r_c, eps, sigma, fit_mode, sub_bits, chunk_size");
    }
    long long cap = 0;
    for (int v = 0; v < n_vol; ++v) {
        if (n[v] < (batch ? 0 : 1)) return set_error(SR_ERR_ARG, "particle count must be positive");
        cap += n[v];
    }
    if (cap < 1 || cap > (1ll << 30)) return set_error(SR_ERR_ARG, "particle count must be in [1, 2^30]");

    sr_plan* p = new sr_plan();
    p->phys = params[0];
    p->n_vol = n_vol;
    p->capacity = cap;
    p->sub_bits = params[0].sub_bits ? params[0].sub_bits : 6;
    p->chunk_k = params[0].chunk_size == 64 ? 2 : 1;
    const long long C = 32 * p->chunk_k;
    if ((rc = fit_poly(params[0].r_c, params[0].sigma, params[0].eps, params[0].fit_mode, p->coef))) {
        delete p;
        return rc;
    }
    long long cells = 0, start = 0;
    std::vector<long long> part_start(n_vol + 1);
    std::vector<int> cell_base(n_vol + 1);
    for (int v = 0; v < n_vol; ++v) {
        VolDev V;
        int n_c = 0;
        if ((rc = make_volume(params[v], p->coef, p->sub_bits, (int)cells, &V, &n_c))) { delete p; return rc; }
        V.part_start = start;
        V.part_end = start + n[v];
        part_start[v] = start;
        cell_base[v] = (int)cells;
        start += n[v];
        cells += (long long)n_c * n_c * n_c;
        if (cells >= (1ll << 30)) { delete p; return set_error(SR_ERR_ARG, "too many cells"); }
        p->vols_h.push_back(V);
        p->vol_n.push_back(n[v]);
    }
    part_start[n_vol] = start;
    cell_base[n_vol] = (int)cells;
    p->total_cells = cells;
    int cell_bits = 0;
    while ((1ll << cell_bits) < cells) ++cell_bits;
    p->key_bits = cell_bits + 3 * p->sub_bits;
    p->max_chunks = (cap + C - 1) / C + (cap < cells ? cap : cells);
    if (p->max_chunks * C >= (1ll << 31)) { delete p; return set_error(SR_ERR_CAPACITY, "too many slots"); }

    cudaError_t ge = cudaGetDevice(&p->device);
    if (ge == cudaSuccess) ge = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
    if (ge != cudaSuccess) {
        delete p;
        return cuda_fail(ge, "device query");
    }
    const long long mc = p->max_chunks, slots = mc * C;
#define SR_ALLOC(ptr, cnt)                                 \
    do {                                                   \
        if ((rc = dalloc(&(ptr), (size_t)(cnt)))) {        \
            free_plan(p);                                  \
            return rc;                                     \
        }                                                  \
    } while (0)
    SR_ALLOC(p->vols, n_vol);
    SR_ALLOC(p->vol_part_start, n_vol + 1);
    SR_ALLOC(p->vol_cell_base, n_vol + 1);
    for (int k = 0; k < 2; ++k) {
        SR_ALLOC(p->keys[k], cap);
        SR_ALLOC(p->vals[k], cap);
        SR_ALLOC(p->lpt_keys[k], mc);
        SR_ALLOC(p->lpt_vals[k], mc);
    }
    SR_ALLOC(p->cell_start, cells + 1);
    SR_ALLOC(p->ccs, cells + 1);
    SR_ALLOC(p->chunk_span, mc);
    SR_ALLOC(p->chunk_meta, mc);
    SR_ALLOC(p->chunk_lo, mc);
    SR_ALLOC(p->chunk_hi, mc);
    SR_ALLOC(p->cost, mc);
    SR_ALLOC(p->slot_pos, slots);
    SR_ALLOC(p->slot_idx, slots);
    SR_ALLOC(p->slot_g, slots);
    SR_ALLOC(p->ctr, 1);
    SR_ALLOC(p->inv_partials, (size_t)kInvBlocks * 7);
#undef SR_ALLOC
    if ((rc = radix_alloc(p->rs_chunks, mc)) || (rc = bin_alloc(p))) {
        free_plan(p);
        return rc;
    }
    cudaError_t e = cudaMemcpy(p->vols, p->vols_h.data(), sizeof(VolDev) * n_vol, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->vol_part_start, part_start.data(), sizeof(long long) * (n_vol + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->vol_cell_base, cell_base.data(), sizeof(int) * (n_vol + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->ctr, 0, sizeof(Counters));
    // an empty ccs table until the first sr_bin: zero chunks
    if (e == cudaSuccess) e = cudaMemset(p->ccs, 0, sizeof(int) * (cells + 1));
    if (e != cudaSuccess) {
        free_plan(p);
        return cuda_fail(e, "plan initialisation");
    }
    if ((rc = force_occupancy(p))) {
        free_plan(p);
        return rc;
    }
    p->order = p->lpt_vals[0];
    *out = p;
    return SR_OK;
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

int set_error(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return SR_ERR_CUDA;
}

thread_local long long t_launches = 0;     // this thread's launches (a capture's own count)
void note_launch(int k) {
    g_launches.fetch_add(k, std::memory_order_relaxed);
    t_launches += k;
}

}  // namespace sr

using namespace sr;

extern "C" {

int sr_fit_poly(double r_c, double sigma, double eps, int mode, double c_out[6]) {
    return fit_poly(r_c, sigma, eps, mode, c_out);
}

int sr_plan_create(const sr_params* params, int64_t n_max, sr_plan** out) {
    if (!out) return set_error(SR_ERR_ARG, "out is null");
    long long n = n_max;
    return build_plan(params, &n, 1, false, out);
}

int sr_plan_batch(const sr_params* params, const int64_t* n, int n_vol, sr_plan** out) {
    if (!out) return set_error(SR_ERR_ARG, "out is null");
    if (!n || n_vol < 1) return set_error(SR_ERR_ARG, "bad volume list");
    std::vector<long long> nn(n, n + n_vol);
    return build_plan(params, nn.data(), n_vol, true, out);
}

int sr_plan_destroy(sr_plan* plan) {
    if (!plan) return SR_OK;
    cudaDeviceSynchronize();
    free_plan(plan);
    return SR_OK;
}

int sr_plan_get_info(sr_plan* p, sr_plan_info* info) {
    if (!p || !info) return set_error(SR_ERR_ARG, "null argument");
    std::memset(info, 0, sizeof(*info));
    info->n_particles = p->binned ? p->n_binned : p->capacity;
    info->capacity = p->capacity;
    info->n_volumes = p->n_vol;
    info->total_cells = p->total_cells;
    info->max_chunks = p->max_chunks;
    int nch = 0;
    SR_CUDA_CHECK(cudaMemcpy(&nch, p->ccs + p->total_cells, sizeof(int), cudaMemcpyDeviceToHost));
    info->n_chunks = nch;
    info->sub_bits = p->sub_bits;
    info->key_bits = p->key_bits;
    info->workers = p->force_blocks * p->warps_per_block;
    info->warps_per_block = p->warps_per_block;
    info->variant = p->variant;
    info->chunk_size = 32 * p->chunk_k;
    info->warps_per_block = variant_warps(p->variant);
    info->workers = p->force_blocks_v[p->variant] * info->warps_per_block;
    for (int k = 0; k < 6; ++k) info->coef[k] = p->coef[k];
    return SR_OK;
}

int sr_plan_volume_info(const sr_plan* p, int v, int64_t* n, double* box, int* n_cells, double* h) {
    if (!p || v < 0 || v >= p->n_vol) return set_error(SR_ERR_ARG, "bad plan or volume index");
    if (n) *n = p->vol_n[v];
    if (box) *box = p->vols_h[v].box;
    if (n_cells) *n_cells = p->vols_h[v].n_c;
    if (h) *h = p->vols_h[v].h;
    return SR_OK;
}

int sr_bin_active(sr_plan* p, const double* pos, const uint8_t* active, int64_t n, void* stream) {
    if (!p) return set_error(SR_ERR_ARG, "plan is null");
    if (!pos && n > 0) return set_error(SR_ERR_ARG, "pos is null");
    if (n < 0) return set_error(SR_ERR_ARG, "n must be >= 0");
    if (n > p->capacity) return set_error(SR_ERR_CAPACITY, "n exceeds the plan capacity");
    if (p->n_vol > 1 && n != p->capacity)
        return set_error(SR_ERR_CAPACITY, "a batch plan bins exactly the sum of its volume counts");
    int rc = launch_bin(p, pos, n, as_stream(stream), active);
    if (rc) return rc;
    p->n_binned = n;
    p->binned = true;
    return SR_OK;
}

int sr_bin(sr_plan* p, const double* pos, int64_t n, void* stream) {
    return sr_bin_active(p, pos, nullptr, n, stream);
}

int sr_force(sr_plan* p, float* acc, unsigned long long* pair_count, int* per_particle, void* stream) {
    if (!p) return set_error(SR_ERR_ARG, "plan is null");
    if (!p->binned) return set_error(SR_ERR_STATE, "sr_force before sr_bin");
    if (!acc && p->n_binned > 0) return set_error(SR_ERR_ARG, "acc is null");
    return launch_force(p, acc, pair_count, per_particle, as_stream(stream));
}

int sr_force_kick(sr_plan* p, float* acc, float* vel, float dt, void* stream) {
    if (!p) return set_error(SR_ERR_ARG, "plan is null");
    if (!p->binned) return set_error(SR_ERR_STATE, "sr_force_kick before sr_bin");
    if ((!acc || !vel) && p->n_binned > 0) return set_error(SR_ERR_ARG, "acc or vel is null");
    return launch_force(p, acc, nullptr, nullptr, as_stream(stream), vel, dt);
}

int sr_leapfrog(sr_plan* p, double* pos, float* vel, float* acc, double dt, int steps, int64_t n, void* stream) {
    if (!p) return set_error(SR_ERR_ARG, "plan is null");
    if ((!pos || !vel || !acc) && n > 0) return set_error(SR_ERR_ARG, "null buffer");
    if (steps < 0) return set_error(SR_ERR_ARG, "steps must be >= 0");
    if (n < 0 || n > p->capacity) return set_error(SR_ERR_CAPACITY, "n exceeds the plan capacity");
    if (p->n_vol > 1 && n != p->capacity)
        return set_error(SR_ERR_CAPACITY, "a batch plan steps exactly the sum of its volume counts");
    if (steps == 0) return SR_OK;
    cudaStream_t st = as_stream(stream);
    const float half = (float)(0.5 * dt);
    int rc = launch_kick(n, acc, vel, half, st);                  // opening half kick
    for (int k = 0; k < steps && !rc; ++k) {
        rc = launch_drift(p, pos, vel, dt, n, st);
        if (!rc) rc = launch_bin(p, pos, n, st);
        // interior half kicks merge: v += a dt, closing half kick on the last step
        if (!rc) rc = launch_force(p, acc, nullptr, nullptr, st, vel, k + 1 < steps ? (float)dt : half);
    }
    if (rc) return rc;
    p->n_binned = n;
    p->binned = true;
    return SR_OK;
}

int sr_force_plain(sr_plan* p, float* acc, void* stream) {
    if (!p) return set_error(SR_ERR_ARG, "plan is null");
    if (!p->binned) return set_error(SR_ERR_STATE, "sr_force_plain before sr_bin");
    if (!acc && p->n_binned > 0) return set_error(SR_ERR_ARG, "acc is null");
    return launch_force_plain(p, acc, as_stream(stream));
}

int sr_force_vjp(sr_plan* p, const float* g_acc, float* g_pos, float g_scale, int accumulate, void* stream) {
    if (!p) return set_error(SR_ERR_ARG, "plan is null");
    if (!p->binned) return set_error(SR_ERR_STATE, "sr_force_vjp before sr_bin");
    if ((!g_acc || !g_pos) && p->n_binned > 0) return set_error(SR_ERR_ARG, "null cotangent pointer");
    return launch_vjp(p, g_acc, g_pos, g_scale, accumulate ? 1 : 0, as_stream(stream));
}

int sr_kick(int64_t n, const float* acc, float* vel, float dt, void* stream) {
    if (n < 0) return set_error(SR_ERR_ARG, "n must be >= 0");
    if (n > 0 && (!acc || !vel)) return set_error(SR_ERR_ARG, "null pointer");
    return launch_kick(n, acc, vel, dt, as_stream(stream));
}

int sr_drift(sr_plan* p, double* pos, const float* vel, double dt, int64_t n, void* stream) {
    if (!p) return set_error(SR_ERR_ARG, "plan is null");
    if (n < 0) return set_error(SR_ERR_ARG, "n must be >= 0");
    if (n > 0 && (!pos || !vel)) return set_error(SR_ERR_ARG, "null pointer");
    if (n > p->capacity) return set_error(SR_ERR_CAPACITY, "n exceeds the plan capacity");
    return launch_drift(p, pos, vel, dt, n, as_stream(stream));
}

int sr_invariants(sr_plan* p, int64_t n, const float* vel, const float* acc, double* out, void* stream) {
    if (!p) return set_error(SR_ERR_ARG, "plan is null");
    if (!out) return set_error(SR_ERR_ARG, "out is null");
    if (n < 0) return set_error(SR_ERR_ARG, "n must be >= 0");
    if (n > p->capacity) return set_error(SR_ERR_CAPACITY, "n exceeds the plan capacity");
    return launch_invariants(n, vel, acc, out, p->inv_partials, as_stream(stream));
}

int sr_plan_status(sr_plan* p, void* stream) {
    if (!p) return set_error(SR_ERR_ARG, "plan is null");
    long long err = 0;
    cudaStream_t st = as_stream(stream);
    SR_CUDA_CHECK(cudaMemcpyAsync(&err, &p->ctr->err, sizeof(long long), cudaMemcpyDeviceToHost, st));
    SR_CUDA_CHECK(cudaStreamSynchronize(st));
    unsigned long long chk = 0;
    SR_CUDA_CHECK(cudaMemcpyAsync(&chk, &p->ctr->check, sizeof(chk), cudaMemcpyDeviceToHost, st));
    SR_CUDA_CHECK(cudaStreamSynchronize(st));
    if (chk) {
        SR_CUDA_CHECK(cudaMemsetAsync(&p->ctr->check, 0, sizeof(chk), st));
        SR_CUDA_CHECK(cudaStreamSynchronize(st));
        return set_error(SR_ERR_CHECK, "bounds check " + std::to_string(chk) +
                                           " failed (bounds-checked build); the access was skipped");
    }
    if (err & 2) {
        SR_CUDA_CHECK(cudaMemsetAsync(&p->ctr->err, 0, sizeof(long long), st));
        SR_CUDA_CHECK(cudaStreamSynchronize(st));
        return set_error(SR_ERR_TIMEOUT, "a wait of the binning's radix sort ran out (the order is not valid)");
    }
    if (err & 1) {
        SR_CUDA_CHECK(cudaMemsetAsync(&p->ctr->err, 0, sizeof(long long), st));
        SR_CUDA_CHECK(cudaStreamSynchronize(st));
        return set_error(SR_ERR_RANGE, "sr_bin saw a non-finite position or one outside [-L, 2L)");
    }
    return SR_OK;
}

int sr_build_checked(void) {
#ifdef SR_CHECK
    return 1;
#else
    return 0;
#endif
}

int sr_check_selftest(sr_plan* p, void* stream) {
    if (!p) return set_error(SR_ERR_ARG, "plan is null");
    return launch_check_selftest(p, as_stream(stream));
}

int sr_plan_copy(sr_plan* p, int which, void* dst, int64_t bytes, void* stream) {
    if (!p || !dst || bytes < 0) return set_error(SR_ERR_ARG, "null argument");
    const void* src = nullptr;
    long long avail = 0;
    const long long mc = p->max_chunks, cells = p->total_cells, C = 32 * p->chunk_k;
    switch (which) {
        case SR_EXPORT_PERM: src = p->vals[p->sorted]; avail = 4 * p->capacity; break;
        case SR_EXPORT_CELL_START: src = p->cell_start; avail = 4 * (cells + 1); break;
        case SR_EXPORT_CELL_CHUNK_START: src = p->ccs; avail = 4 * (cells + 1); break;
        case SR_EXPORT_SLOT_POS: src = p->slot_pos; avail = 16 * mc * C; break;
        case SR_EXPORT_SLOT_IDX: src = p->slot_idx; avail = 4 * mc * C; break;
        case SR_EXPORT_CHUNK_META: src = p->chunk_meta; avail = 16 * mc; break;
        case SR_EXPORT_CHUNK_LO: src = p->chunk_lo; avail = 16 * mc; break;
        case SR_EXPORT_CHUNK_HI: src = p->chunk_hi; avail = 16 * mc; break;
        case SR_EXPORT_ORDER: src = p->order; avail = 4 * mc; break;
        case SR_EXPORT_COST: src = p->cost; avail = 4 * mc; break;
        case SR_EXPORT_COUNTERS: src = p->ctr; avail = sizeof(Counters); break;
        default: return set_error(SR_ERR_ARG, "unknown export selector");
    }
    if (bytes > avail) return set_error(SR_ERR_ARG, "bytes exceeds the array size");
    if (bytes == 0) return SR_OK;
    SR_CUDA_CHECK(cudaMemcpyAsync(dst, src, (size_t)bytes, cudaMemcpyDefault, as_stream(stream)));
    return SR_OK;
}

int sr_step_host(sr_plan* p, const double* pos, float* vel, float* acc, float dt, int64_t n, void* stream) {
    if (!p) return set_error(SR_ERR_ARG, "plan is null");
    if ((!pos || !vel) && n > 0) return set_error(SR_ERR_ARG, "null host buffer");
    if (n < 0 || n > p->capacity) return set_error(SR_ERR_CAPACITY, "n exceeds the plan capacity");
    cudaStream_t st = as_stream(stream);
    int rc;
    if ((!p->h_pos_dev && (rc = dalloc(&p->h_pos_dev, (size_t)p->capacity * 3))) ||
        (!p->h_vel_dev && (rc = dalloc(&p->h_vel_dev, (size_t)p->capacity * 4))) ||
        (!p->h_acc_dev && (rc = dalloc(&p->h_acc_dev, (size_t)p->capacity * 4))))
        return rc;
    if (!p->h_side) SR_CUDA_CHECK(cudaStreamCreateWithFlags(&p->h_side, cudaStreamNonBlocking));
    if (!p->h_fork) SR_CUDA_CHECK(cudaEventCreateWithFlags(&p->h_fork, cudaEventDisableTiming));
    if (!p->h_join) SR_CUDA_CHECK(cudaEventCreateWithFlags(&p->h_join, cudaEventDisableTiming));
    // The velocity upload runs on a side stream after the position upload
    // (both share the host link, and the binning needs the positions first),
    // beside the binning; the force kernel (which reads the velocities in the
    // fused kick) waits for it.
    if (n > 0) SR_CUDA_CHECK(cudaMemcpyAsync(p->h_pos_dev, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    SR_CUDA_CHECK(cudaEventRecord(p->h_fork, st));
    SR_CUDA_CHECK(cudaStreamWaitEvent(p->h_side, p->h_fork, 0));
    if (n > 0)
        SR_CUDA_CHECK(cudaMemcpyAsync(p->h_vel_dev, vel, sizeof(float) * 4 * n, cudaMemcpyHostToDevice, p->h_side));
    SR_CUDA_CHECK(cudaEventRecord(p->h_join, p->h_side));
    rc = sr_bin(p, p->h_pos_dev, n, stream);
    cudaError_t we = cudaStreamWaitEvent(st, p->h_join, 0);       // join even when sr_bin failed
    if (rc) return rc;
    if (we != cudaSuccess) return cuda_fail(we, "sr_step_host");
    if ((rc = launch_force(p, p->h_acc_dev, nullptr, nullptr, st, p->h_vel_dev, dt))) return rc;
    if (n > 0) {
        SR_CUDA_CHECK(cudaMemcpyAsync(vel, p->h_vel_dev, sizeof(float) * 4 * n, cudaMemcpyDeviceToHost, st));
        if (acc) SR_CUDA_CHECK(cudaMemcpyAsync(acc, p->h_acc_dev, sizeof(float) * 4 * n, cudaMemcpyDeviceToHost, st));
    }
    SR_CUDA_CHECK(cudaStreamSynchronize(st));
    return SR_OK;
}

int sr_step_host_submit(sr_plan* p, const double* pos, float* vel, float* acc, float dt, int64_t n, void* stream) {
    if (!p) return set_error(SR_ERR_ARG, "plan is null");
    if ((!pos || !vel) && n > 0) return set_error(SR_ERR_ARG, "null host buffer");
    if (n < 0 || n > p->capacity) return set_error(SR_ERR_CAPACITY, "n exceeds the plan capacity");
    cudaStream_t st = as_stream(stream);
    int rc;
    if (!p->q_up) {                      // first call; a failed one is resumed where it stopped
        for (int k = 0; k < 2; ++k) {
            if ((!p->q_pos[k] && (rc = dalloc(&p->q_pos[k], (size_t)p->capacity * 3))) ||
                (!p->q_vel[k] && (rc = dalloc(&p->q_vel[k], (size_t)p->capacity * 4))) ||
                (!p->q_acc[k] && (rc = dalloc(&p->q_acc[k], (size_t)p->capacity * 4))))
                return rc;
            if (!p->q_loaded[k]) SR_CUDA_CHECK(cudaEventCreateWithFlags(&p->q_loaded[k], cudaEventDisableTiming));
            if (!p->q_computed[k]) SR_CUDA_CHECK(cudaEventCreateWithFlags(&p->q_computed[k], cudaEventDisableTiming));
            if (!p->q_freed[k]) SR_CUDA_CHECK(cudaEventCreateWithFlags(&p->q_freed[k], cudaEventDisableTiming));
        }
        if (!p->q_down) SR_CUDA_CHECK(cudaStreamCreateWithFlags(&p->q_down, cudaStreamNonBlocking));
        SR_CUDA_CHECK(cudaStreamCreateWithFlags(&p->q_up, cudaStreamNonBlocking));
    }
    const int s = p->q_next;
    // uploads into set s once the step that used it last has been read back
    if (p->q_used[s]) SR_CUDA_CHECK(cudaStreamWaitEvent(p->q_up, p->q_freed[s], 0));
    if (n > 0) {
        SR_CUDA_CHECK(cudaMemcpyAsync(p->q_pos[s], pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, p->q_up));
        SR_CUDA_CHECK(cudaMemcpyAsync(p->q_vel[s], vel, sizeof(float) * 4 * n, cudaMemcpyHostToDevice, p->q_up));
    }
    SR_CUDA_CHECK(cudaEventRecord(p->q_loaded[s], p->q_up));
    // binning and force on the caller's stream, after the step before (the
    // plan's workspace) and after this set's uploads
    SR_CUDA_CHECK(cudaStreamWaitEvent(st, p->q_loaded[s], 0));
    if ((rc = sr_bin(p, p->q_pos[s], n, stream))) return rc;
    if ((rc = launch_force(p, p->q_acc[s], nullptr, nullptr, st, p->q_vel[s], dt))) return rc;
    SR_CUDA_CHECK(cudaEventRecord(p->q_computed[s], st));
    SR_CUDA_CHECK(cudaStreamWaitEvent(p->q_down, p->q_computed[s], 0));
    if (n > 0) {
        SR_CUDA_CHECK(cudaMemcpyAsync(vel, p->q_vel[s], sizeof(float) * 4 * n, cudaMemcpyDeviceToHost, p->q_down));
        if (acc)
            SR_CUDA_CHECK(cudaMemcpyAsync(acc, p->q_acc[s], sizeof(float) * 4 * n, cudaMemcpyDeviceToHost, p->q_down));
    }
    SR_CUDA_CHECK(cudaEventRecord(p->q_freed[s], p->q_down));
    p->q_used[s] = true;
    p->q_next = 1 - s;
    return SR_OK;
}

int sr_step_host_wait(sr_plan* p) {
    if (!p) return set_error(SR_ERR_ARG, "plan is null");
    // the uploads too: a submit that failed after enqueuing them has no
    // read-back that would wait for them
    if (p->q_up) SR_CUDA_CHECK(cudaStreamSynchronize(p->q_up));
    if (p->q_down) SR_CUDA_CHECK(cudaStreamSynchronize(p->q_down));
    return SR_OK;
}

int sr_plan_set_variant(sr_plan* p, int variant) {
    if (!p || variant < 0 || variant >= kVariants) return set_error(SR_ERR_ARG, "variant out of range");
    if (p->force_blocks_v[variant] <= 0) return set_error(SR_ERR_ARG, "variant not available for this chunk size");
    p->variant = variant;
    p->force_blocks = p->force_blocks_v[variant];
    return SR_OK;
}

int sr_variant_count(void) { return kVariants; }

int sr_autotune(sr_plan* p, float* acc, int reps, float* ms_out, void* stream) {
    if (!p) return set_error(SR_ERR_ARG, "plan is null");
    if (!p->binned) return set_error(SR_ERR_STATE, "sr_autotune before sr_bin");
    if (!acc || reps < 1) return set_error(SR_ERR_ARG, "acc is null or reps < 1");
    cudaStream_t st = as_stream(stream);
    cudaEvent_t e0, e1;
    SR_CUDA_CHECK(cudaEventCreate(&e0));
    SR_CUDA_CHECK(cudaEventCreate(&e1));
    float best = 1e30f, msv[kVariants];
    int best_v = p->variant;
    int rc = SR_OK;
    for (int v = 0; v < kVariants && rc == SR_OK; ++v) {
        msv[v] = 0.f;
        if (ms_out) ms_out[v] = 0.f;
        if (p->force_blocks_v[v] <= 0) continue;       // not built for this chunk size
        p->variant = v;
        if ((rc = launch_force(p, acc, nullptr, nullptr, st))) break;   // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && rc == SR_OK; ++r) rc = launch_force(p, acc, nullptr, nullptr, st);
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) { rc = cuda_fail(e, "sr_autotune"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        msv[v] = ms;
        if (ms_out) ms_out[v] = ms;
        if (ms < best) { best = ms; best_v = v; }
    }
    // The two fastest variants are often within the run-to-run spread of a
    // single timing (about 1%): when they are within 3%, time them again,
    // alternating one launch of each over 2 reps + 1 rounds, so that clock
    // or power drift weighs on both alike, and keep the faster total.
    int second = -1;
    for (int v = 0; v < kVariants && rc == SR_OK; ++v)
        if (v != best_v && msv[v] > 0.f && (second < 0 || msv[v] < msv[second])) second = v;
    if (rc == SR_OK && second >= 0 && msv[second] < 1.03f * best) {
        const int cand[2] = {best_v, second};
        float tot[2] = {0.f, 0.f};
        for (int r = 0; r < 2 * reps + 1 && rc == SR_OK; ++r) {
            for (int c = 0; c < 2 && rc == SR_OK; ++c) {
                p->variant = cand[c];
                cudaEventRecord(e0, st);
                rc = launch_force(p, acc, nullptr, nullptr, st);
                cudaEventRecord(e1, st);
                cudaError_t e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) { rc = cuda_fail(e, "sr_autotune"); break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                tot[c] += ms;
            }
        }
        if (rc == SR_OK && tot[1] < tot[0]) best_v = second;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->variant = best_v;
    p->force_blocks = p->force_blocks_v[best_v];
    return rc;
}

int sr_plan_tune(const sr_params* params, int64_t n_max, const double* pos, int64_t n, int reps, sr_plan** out,
                 sr_tune_entry* entries, int* n_entries, void* stream) {
    if (!out) return set_error(SR_ERR_ARG, "out is null");
    *out = nullptr;
    if (n_entries) *n_entries = 0;
    if (!params || (!pos && n > 0) || reps < 1) return set_error(SR_ERR_ARG, "null params or pos, or reps < 1");
    if (n < 1 || n > n_max) return set_error(SR_ERR_CAPACITY, "n must be in [1, n_max]");
    int rc = check_physics(*params);
    if (rc) return rc;
    const double min_side = params->r_c * kSideMargin;
    const int nc0 = default_cells(params->box, min_side);
    std::vector<int> cells;
    for (int nc : {nc0, (int)std::floor(nc0 * 4.0 / 3.0), (int)std::floor(nc0 * 3.0 / 4.0)}) {
        if (nc < 1 || params->box / nc < min_side) continue;
        if (std::find(cells.begin(), cells.end(), nc) == cells.end()) cells.push_back(nc);
    }
    float* acc = nullptr;
    cudaError_t e = cudaMalloc(&acc, sizeof(float) * 4 * (size_t)n);
    if (e != cudaSuccess) return cuda_fail(e, "sr_plan_tune scratch");
    std::vector<float> ms(kVariants);
    sr_plan* best = nullptr;
    float best_ms = 1e30f;
    int k = 0;
    for (int chunk : {32, 64}) {
        for (int nc : cells) {
            sr_params q = *params;
            q.chunk_size = chunk;
            q.n_cells = nc;
            sr_plan* p = nullptr;
            rc = sr_plan_create(&q, n_max, &p);
            if (!rc) rc = sr_bin(p, pos, n, stream);
            if (!rc) rc = sr_autotune(p, acc, reps, ms.data(), stream);
            if (rc) {
                if (p) sr_plan_destroy(p);
                break;
            }
            const float t = ms[p->variant];
            if (entries) entries[k] = sr_tune_entry{chunk, nc, p->variant, t};
            ++k;
            if (t < best_ms) {
                if (best) sr_plan_destroy(best);
                best = p;
                best_ms = t;
            } else {
                sr_plan_destroy(p);
            }
        }
        if (rc) break;
    }
    cudaFree(acc);
    if (n_entries) *n_entries = k;
    if (rc) {
        if (best) sr_plan_destroy(best);
        return rc;
    }
    *out = best;
    return SR_OK;
}

int sr_graph_capture(sr_plan* p, const double* pos, float* vel, float* acc, float dt, int64_t n, void* stream) {
    if (!p) return set_error(SR_ERR_ARG, "plan is null");
    if (!pos || !vel || !acc) return set_error(SR_ERR_ARG, "null buffer");
    if (!stream) return set_error(SR_ERR_ARG, "the legacy default stream cannot be captured");
    if (n < 0 || n > p->capacity) return set_error(SR_ERR_CAPACITY, "n exceeds the plan capacity");
    if (p->n_vol > 1 && n != p->capacity)
        return set_error(SR_ERR_CAPACITY, "a batch plan bins exactly the sum of its volume counts");
    cudaStream_t st = as_stream(stream);
    SR_CUDA_CHECK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const long long t0 = t_launches;
    int rc = launch_bin(p, pos, n, st);
    if (!rc) rc = launch_force(p, acc, nullptr, nullptr, st, vel, dt);      // kick fused into the epilogue
    const long long captured = t_launches - t0;
    // captured kernels run at each sr_graph_launch, not now
    g_launches.fetch_sub(captured, std::memory_order_relaxed);
    t_launches = t0;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    p->graph_exec = ex;
    p->graph_kernels = captured;
    p->n_binned = n;
    p->binned = true;
    return SR_OK;
}

int sr_graph_launch(sr_plan* p, void* stream) {
    if (!p) return set_error(SR_ERR_ARG, "plan is null");
    if (!p->graph_exec) return set_error(SR_ERR_STATE, "no captured graph");
    SR_CUDA_CHECK(cudaGraphLaunch(p->graph_exec, as_stream(stream)));
    note_launch((int)p->graph_kernels);
    return SR_OK;
}

const char* sr_last_error(void) { return g_last_error.c_str(); }

int64_t sr_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
