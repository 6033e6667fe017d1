/*
 * sr.h -- C ABI of the B300 short-range particle-particle force library.
 *
 * The library evaluates the short-range half of a split long/short-range
 * gravity solver (the paper's Sec. 2: a spectrally filtered PM long-range
 * force plus direct particle-particle sums inside a cutoff r_c), with the
 * on-node work decomposition of Sec. 2.1 (partition into overlapping blocks
 * with active and passive particles, evolve, reconcile) and the kick that
 * ends the step.  Force law (unit masses, G = 1, periodic box of side L):
 *
 *   a_i = sum_{j != i, |d_ij| < r_c} d_ij f_SR(|d_ij|^2),   d_ij = x_j - x_i (minimum image)
 *   f_SR(s) = (s + eps^2)^(-3/2) - p(s),
 *
 * p a degree-5 polynomial least-squares fit of the Gaussian-split long-range
 * force F_long(r)/r, F_long(r) = (1/r^2)[erf(r/2 sigma) - (r/(sigma sqrt pi)) exp(-r^2/4 sigma^2)].
 *
 * Conventions for every entry point:
 *  - Return value: SR_OK (0) or an SR_ERR_* code; the message of the last
 *    failure on the calling thread is returned by sr_last_error().  Nothing
 *    is thrown across the ABI.
 *  - "device" pointers are CUDA global-memory pointers on the current
 *    device; "host" pointers are CPU memory.  The caller owns every buffer it
 *    passes; the plan owns its workspace.
 *  - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Entry points that take a stream only enqueue work: they do not
 *    allocate, free or synchronise, so they can be captured into a CUDA
 *    graph (sr_force_plain is the exception, see there).
 *  - Positions are binary64 arrays of N rows (x, y, z), row-major (AoS).
 *    Velocities, accelerations and their cotangents are binary32 arrays of
 *    N rows (x, y, z, w) (16-byte float4 rows; w is ignored on input and
 *    written as 0 on output).  Rows follow the caller's particle order; for a
 *    batch plan, volumes are concatenated in plan order.
 */
#ifndef SR_H
#define SR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define SR_OK            0
#define SR_ERR_ARG       1   /* invalid argument (null pointer, bad size or parameter) */
#define SR_ERR_CUDA      2   /* a CUDA runtime call failed (message has the CUDA error) */
#define SR_ERR_CAPACITY  3   /* n exceeds the plan's capacity */
#define SR_ERR_STATE     4   /* call order violated (e.g. sr_force before sr_bin) */
#define SR_ERR_RANGE     5   /* a position was non-finite or outside [-L, 2L) */
#define SR_ERR_TIMEOUT   6   /* a bounded device-side loop ran out of iterations (see the call) */
#define SR_ERR_CHECK     7   /* bounds-checked build: an index check failed (the access was skipped) */

/* Polynomial fit modes. */
#define SR_FIT_CONSTRAINED    0  /* least squares with p(r_c^2) = (r_c^2+eps^2)^(-3/2): f_SR(r_c^2) = 0 */
#define SR_FIT_UNCONSTRAINED  1  /* plain least squares */

/* Export selectors for sr_plan_copy (all refer to the last sr_bin). */
#define SR_EXPORT_PERM              0  /* int32[n]: sorted position -> caller index */
#define SR_EXPORT_CELL_START        1  /* int32[total_cells+1]: first sorted position of each cell */
#define SR_EXPORT_CELL_CHUNK_START  2  /* int32[total_cells+1]: first chunk of each cell */
#define SR_EXPORT_SLOT_POS          3  /* float[4*C*n_chunks]: chunk-relative offsets (units of h), C = chunk size;
                                              w = 1 active, -1 passive (sr_bin_active), 0 empty slot */
#define SR_EXPORT_SLOT_IDX          4  /* int32[C*n_chunks]: caller index per slot, -1 = empty */
#define SR_EXPORT_CHUNK_META        5  /* int32[4*n_chunks]: anchor (qx, qy, qz) and volume */
#define SR_EXPORT_CHUNK_LO          6  /* float[4*n_chunks]: bbox min (x,y,z), w = particle count (int bits) */
#define SR_EXPORT_CHUNK_HI          7  /* float[4*n_chunks]: bbox max (x,y,z), w = active particles (int bits) */
#define SR_EXPORT_ORDER             8  /* int32[n_chunks]: work order of the persistent kernel */
#define SR_EXPORT_COST              9  /* uint32[n_chunks]: estimated pair evaluations per chunk */
#define SR_EXPORT_COUNTERS         10  /* int64[8]: queue head, error bits, cost total, candidate evaluations
                                              (valid i), evaluations x lanes, work items, 2 reserved */

/* Physics and binning parameters of one periodic volume (lengths in the
 * same unit as the positions; the workloads use the mean inter-particle
 * spacing). */
typedef struct sr_params {
    double box;       /* L > 2 r_c: periodic box side                                  */
    double r_c;       /* cutoff radius (> 0)                                           */
    double eps;       /* Plummer softening (> 0)                                       */
    double sigma;     /* Gaussian split scale (> 0)                                    */
    int    fit_mode;  /* SR_FIT_CONSTRAINED or SR_FIT_UNCONSTRAINED                    */
    int    n_cells;   /* cells per axis; 0 = automatic (side close to 4, >= r_c)        */
    int    sub_bits;  /* Morton bits per axis inside a cell (1..8); 0 = automatic (6)  */
    int    chunk_size;/* particles per chunk: 32 or 64; 0 = automatic (32)             */
} sr_params;

/* Read-only description of a plan (sizes of the exportable arrays). */
typedef struct sr_plan_info {
    int64_t n_particles;   /* particles of the last sr_bin (capacity before the first)  */
    int64_t capacity;      /* maximum particles                                        */
    int64_t n_volumes;
    int64_t total_cells;   /* sum over volumes of n_cells^3                            */
    int64_t max_chunks;    /* capacity of the chunk arrays                             */
    int64_t n_chunks;      /* chunks of the last sr_bin (reads device memory; syncs)   */
    int32_t sub_bits;
    int32_t key_bits;      /* significant bits of the sort key                         */
    int32_t workers;       /* resident warps of the persistent force kernel            */
    int32_t warps_per_block;
    int32_t variant;       /* selected pair-kernel variant (see sr_plan_set_variant)   */
    int32_t chunk_size;    /* particles per chunk (32 or 64)                           */
    double  coef[6];       /* fitted p(s) = sum_k coef[k] s^k (binary64)               */
} sr_plan_info;

typedef struct sr_plan sr_plan;

/*
 * sr_fit_poly -- fit p(s) = sum_k c_out[k] s^k to F_long(sqrt s)/sqrt s on
 * [0, r_c^2] (host only; no GPU needed).  Reading of the fit (the paper,
 * Sec. 2, names the filtered split but prints no polynomial): 4096 midpoint
 * samples s_k = r_c^2 (k + 1/2)/4096, unweighted least squares in the basis
 * (s/r_c^2)^m solved by Householder QR in binary64; mode CONSTRAINED also
 * imposes p(r_c^2) = (r_c^2 + eps^2)^(-3/2).
 * c_out: host array of 6 doubles, written on success.
 * Errors: SR_ERR_ARG for non-positive r_c or sigma, negative eps, bad mode
 * or null c_out.
 */
int sr_fit_poly(double r_c, double sigma, double eps, int mode, double c_out[6]);

/*
 * sr_plan_create -- plan for one periodic volume holding at most n_max
 * particles.  Allocates all device workspace (about 100 bytes per particle
 * plus 8 bytes per cell) on the current device; no later call allocates.
 * Binning (Sec. 2.1 step 1, "partition into overlapping blocks"): cells of
 * side L/n_cells >= r_c; each cell's particles in Morton order of their
 * sub-cell (2^sub_bits per axis); chunks of <= chunk_size (32 or 64)
 * consecutive particles per cell are the work units, each with a binary64
 * anchor and binary32 offsets.
 * Errors: SR_ERR_ARG (bad parameters, n_max < 1 or > 2^30), SR_ERR_CUDA
 * (allocation failed).  *out is NULL on failure.
 */
int sr_plan_create(const sr_params* params, int64_t n_max, sr_plan** out);

/*
 * sr_plan_batch -- plan for n_vol independent periodic volumes evaluated
 * together (one binning, one persistent force launch).  params[v].box and
 * n_cells may differ per volume; r_c, eps, sigma, fit_mode, sub_bits and
 * chunk_size must be equal.  n[v] (host array) is volume v's particle count; sr_bin
 * then takes the concatenation, sum n[v] rows.
 * Errors: as sr_plan_create, plus SR_ERR_ARG for mismatched physics.
 */
int sr_plan_batch(const sr_params* params, const int64_t* n, int n_vol, sr_plan** out);

/* sr_plan_destroy -- free a plan and its workspace (synchronises the device). */
int sr_plan_destroy(sr_plan* plan);

/* sr_plan_get_info -- fill *info (host). Synchronises to read n_chunks. */
int sr_plan_get_info(sr_plan* plan, sr_plan_info* info);

/*
 * sr_plan_volume_info -- geometry of volume v (host outputs, each nullable):
 * its particle count (capacity for a single-volume plan), box side, cells
 * per axis, and fine-grid side h = L / (n_cells 2^sub_bits).
 * Errors: SR_ERR_ARG for a null plan or v out of range.
 */
int sr_plan_volume_info(const sr_plan* plan, int v, int64_t* n, double* box, int* n_cells,
                        double* h);

/*
 * sr_bin -- bit-exact cell binning and stable counting sort (Sec. 2.1
 * step 1).  pos: device, n rows of binary64 (x, y, z).  Positions in
 * [-L, 2L) are folded into [0, L) (x<0: x+L, then x>=L: x-L); the fine
 * grid is h = L/(n_cells 2^sub_bits), q = min(floor(x/h), M-1); sort key
 * (cell << 3 sub_bits) | morton(sub-cell), ties by caller index; chunk
 * offsets binary32(x/h - qA).  Also computes each chunk's cost estimate and
 * the longest-first work order for sr_force.
 * Errors: SR_ERR_ARG (null pos), SR_ERR_CAPACITY (n > capacity; for a batch
 * plan n must equal the sum of n[v]).  Out-of-range or non-finite
 * positions do not fail the call: they are binned as 0 and flagged, and
 * sr_plan_status then returns SR_ERR_RANGE.
 */
int sr_bin(sr_plan* plan, const double* pos, int64_t n, void* stream);

/*
 * sr_bin_active -- sr_bin with a mask of the particles whose forces are
 * wanted (Sec. 2.1: a node evolves its active particles; the passive ones,
 * the overload copies of its neighbours' particles, are read-only).
 * active: device, n bytes in caller order, nonzero = active; NULL makes
 * every particle active (sr_bin).  Every particle is binned and serves as a
 * neighbour; the pair kernels (sr_force, sr_force_kick, sr_force_vjp and
 * the counting mode) take as work items only the chunks that hold an active
 * particle, and write only active particles' rows: the acc, vel, g_pos and
 * per_particle rows of passive particles are left untouched, and
 * pair_count adds the active particles' pairs only.  The mask is read
 * during this call only.  Errors as sr_bin.
 */
int sr_bin_active(sr_plan* plan, const double* pos, const uint8_t* active, int64_t n, void* stream);

/*
 * sr_force -- short-range accelerations of every binned particle (Sec. 2,
 * direct particle-particle sums; Sec. 2.1 steps 2-3: each chunk is an
 * active block reading its passive neighbours within r_c, and only active
 * particles are written).  One persistent launch: each warp repeatedly takes
 * the next chunk from the longest-first order, culls neighbour chunks and
 * particles by bounding boxes, stages the survivors through shared memory
 * and accumulates per-batch binary32 partial sums (32 neighbours; 128 in the
 * packed loop) into a Kahan (compensated) sum.  No float atomics: results
 * are run-to-run identical.
 * acc: device, n rows float4 (written, caller order).
 * pair_count: device uint64, nullable: if given, the kernel also counts the
 *   ordered in-range pairs (i != j) under the binary32 predicate
 *   s' = fma(dz,dz,fma(dy,dy,fma(dx,dx,eps^2/h^2))) < (r_c^2+eps^2)/h^2
 *   and ADDS the total to *pair_count.
 * per_particle: device int32[n], nullable: per-particle in-range counts
 *   (written, caller order); counting mode runs a slower kernel variant.
 * Errors: SR_ERR_STATE before the first sr_bin, SR_ERR_ARG (null acc while the plan holds particles).
 */
int sr_force(sr_plan* plan, float* acc, unsigned long long* pair_count,
             int* per_particle, void* stream);

/*
 * sr_force_kick -- sr_force with the kick fused into its epilogue: writes
 * acc (device float4 rows, caller order) and applies vel += acc * dt to the
 * same rows (device float4 rows, x, y, z; w untouched), with the
 * arithmetic of sr_kick, so the result equals sr_force then sr_kick bit for
 * bit, without re-reading acc.  The step either side of the pair sum in
 * the paper's timestep (Sec. 2.1: the evolved active particles are
 * updated).  Errors: SR_ERR_STATE before the first sr_bin, SR_ERR_ARG.
 */
int sr_force_kick(sr_plan* plan, float* acc, float* vel, float dt, void* stream);

/*
 * sr_leapfrog -- `steps` kick-drift-kick leapfrog steps of the short-range
 * dynamics: per step v += a dt/2, x <- fold(x + v dt), re-bin, a = a(x),
 * v += a dt/2.  Interior half kicks are merged (v += a dt in the fused
 * force epilogue), so a step costs one drift, one sr_bin and one fused
 * force-kick launch.  pos: device binary64 rows (updated); vel, acc:
 * device float4 rows; acc must hold a(x) of the input positions (e.g. from
 * sr_bin + sr_force) and holds a(x_K) on return.  n as for sr_bin.
 * Errors: SR_ERR_ARG, SR_ERR_CAPACITY, SR_ERR_CUDA.
 */
int sr_leapfrog(sr_plan* plan, double* pos, float* vel, float* acc, double dt, int steps, int64_t n,
                void* stream);

/*
 * sr_force_plain -- the same accelerations from the plain kernel: one
 * launch per z-slab of cells, one thread per particle slot, neighbour
 * particles read straight from global memory over the 27 neighbour cells,
 * no culling and no work queue.  It is the reference point for the
 * persistent kernel's speed-up.  Unlike the other calls it copies the
 * cell-to-chunk table to the host (one synchronisation) to size its
 * launches, so it cannot be captured into a CUDA graph.
 */
int sr_force_plain(sr_plan* plan, float* acc, void* stream);

/*
 * sr_force_vjp -- vector-Jacobian product of the accelerations with respect
 * to the positions, gather form (no atomics):
 *   xbar_i (+)= g_scale * sum_j [ f(s)(g_j - g_i) + 2 f'(s) (d.(g_j - g_i)) d ],
 *   d = x_j - x_i, f'(s) = -3/2 (s+eps^2)^(-5/2) - p'(s),
 * for the positions of the last sr_bin.  g_acc: device float4 rows (the
 * cotangent on acc); g_pos: device float4 rows, overwritten (accumulate = 0)
 * or added to (accumulate = 1).  Plans with 32-particle chunks run the
 * packed two-wide binary32 pair loop (each term the same binary32
 * operations as the scalar loop; even and odd neighbours summed separately
 * over batches of 128 before the compensated update); 64-particle chunks the
 * scalar loop.  Deterministic.
 * Errors: SR_ERR_STATE before the first sr_bin, SR_ERR_ARG (null pointers while the plan holds particles).
 */
int sr_force_vjp(sr_plan* plan, const float* g_acc, float* g_pos, float g_scale,
                 int accumulate, void* stream);

/*
 * sr_kick -- v += a * dt for n float4 rows (x, y, z; w untouched).
 * acc, vel: device.  Errors: SR_ERR_ARG (null pointers, n < 0).
 */
int sr_kick(int64_t n, const float* acc, float* vel, float dt, void* stream);

/*
 * sr_drift -- x <- fold(x + v dt) in binary64 for the plan's volumes
 * (t = double(v) * dt and x + t, each rounded once (no fused multiply-add),
 * then x<0: x+L, x>=L: x-L).  pos: device binary64
 * rows (x, y, z), updated in place; vel: device float4 rows; n as for
 * sr_bin.  Errors: SR_ERR_ARG, SR_ERR_CAPACITY.
 */
int sr_drift(sr_plan* plan, double* pos, const float* vel, double dt, int64_t n, void* stream);

/*
 * sr_invariants -- binary64 global sums of n float4 rows, in a fixed
 * reduction order (deterministic): out[0..2] = sum v, out[3..5] = sum a,
 * out[6] = sum |v|^2 / 2 (unit masses).  vel, acc: device; out: device
 * double[7], overwritten.  Either input may be NULL (its sums are 0).  The
 * plan provides the reduction workspace; n must not exceed its capacity.
 */
int sr_invariants(sr_plan* plan, int64_t n, const float* vel, const float* acc, double* out,
                  void* stream);

/*
 * sr_invariants_noalloc -- the same seven binary64 sums as sr_invariants
 * (sum v, sum a, sum |v|^2 / 2 of n float4 rows; vel or acc may be NULL),
 * for callers that cannot allocate device memory: no plan is needed and
 * nothing is allocated per call.  The paper has no counterpart; this entry
 * point exists for code that must not call cudaMalloc (an application whose
 * allocator owns the device memory, or a monitoring hook inside a step loop
 * that may neither allocate nor synchronise).
 * Scratch: a fixed 224 KiB device array inside the library (one per device
 * that loads it, held until the process exits), enough for n up to
 * 67,108,864 rows; larger n fails with SR_ERR_CAPACITY.  The first call in
 * each CUDA context looks up that array's device address (a CUDA runtime
 * query; a context made after a device reset gets its own lookup), so make
 * the first call on a device before any stream capture.  Under CUDA's lazy
 * module loading (the default) that first call is also what loads this
 * library's device code on the device, and the load allocates the array and
 * the code there: callers whose allocator must own all device memory from
 * some point on should warm the entry point up before it, for example with
 * n = 0 (which writes seven zeros to out).  Later calls allocate nothing.  All calls
 * share the array: calls whose kernels overlap on the GPU (different
 * streams, no ordering between them) race and may return wrong sums; calls
 * on one stream are safe.  Every call rewrites all partial sums it reads.
 * The summation order differs from sr_invariants, so results agree to
 * rounding (about 1e-15 relative), not bit for bit.
 * Errors: SR_ERR_ARG (null out, n < 0), SR_ERR_CAPACITY, SR_ERR_CUDA.
 */
int sr_invariants_noalloc(int64_t n, const float* vel, const float* acc, double* out, void* stream);

/*
 * sr_plan_status -- synchronise the stream and report device-side flags of
 * the last calls: SR_ERR_CHECK if a bounds check of the checked build failed,
 * else SR_ERR_TIMEOUT if a bounded wait of sr_bin's radix sort ran out (its
 * order is then not valid), else SR_ERR_RANGE if sr_bin saw a non-finite or
 * out-of-range position (the reported flag is then cleared), else SR_OK.
 */
int sr_plan_status(sr_plan* plan, void* stream);

/*
 * The bounds-checked build (libsr_b300_check.so, compiled with -DSR_CHECK;
 * same entry points, slower).  Its pair kernels, binning kernels, radix
 * scatter and center finder check every work-item, cell, chunk, ring, list,
 * caller-row and slot index before the access; a failed check records its
 * code in the plan's error word (the first one is kept), skips the access
 * and never traps, and sr_plan_status then returns SR_ERR_CHECK with the
 * code in sr_last_error (sr_centers_info.check_code for the center
 * finder).  The release build compiles none of the checks.
 * sr_build_checked -- 1 in the bounds-checked build, 0 in the release build.
 * sr_check_selftest -- records check code 99 without any memory access (a
 * check whose condition is false), so that the next sr_plan_status returns
 * SR_ERR_CHECK in the bounds-checked build; in the release build it does
 * nothing.  Enqueued on stream.  Errors: SR_ERR_ARG (null plan).
 */
int sr_build_checked(void);
int sr_check_selftest(sr_plan* plan, void* stream);

/*
 * sr_plan_copy -- copy one internal array of the last sr_bin (selector
 * SR_EXPORT_*) into dst (device or host memory, cudaMemcpyDefault), at most
 * bytes bytes, on stream.  For inspection and tests.
 */
int sr_plan_copy(sr_plan* plan, int which, void* dst, int64_t bytes, void* stream);

/*
 * sr_step_host -- one whole step from host buffers (end-to-end form): copy
 * pos (host binary64 rows) and vel (host float4 rows) to plan-owned device
 * buffers, sr_bin, sr_force_kick, copy acc (host float4 rows, nullable)
 * and the updated vel back, and wait for completion.  The velocity upload
 * runs on a plan-owned side stream after the position upload, beside the
 * binning (the force waits for it).  Host buffers should be page-locked for
 * overlap.  The first call allocates the staging buffers, the side stream
 * and two events.  n = 0 copies nothing (the buffers may then be null).
 */
int sr_step_host(sr_plan* plan, const double* pos, float* vel, float* acc, float dt,
                 int64_t n, void* stream);

/*
 * sr_step_host_submit / sr_step_host_wait -- the step of sr_step_host for a
 * stream of independent inputs (one short-range step of Sec. 2.1 per
 * input), pipelined: submit enqueues the step and returns without waiting,
 * so the uploads of one step run while the step before it computes, and
 * its read-back while the next one computes.
 *   submit: copy pos (host binary64 rows) and vel (host float4 rows) to one
 *           of two plan-owned staging sets (used in turn) on a plan-owned
 *           upload stream; sr_bin and sr_force_kick on `stream` once those
 *           copies are done; copy the updated vel and, if acc is not null,
 *           the accelerations (host float4 rows) back on a plan-owned
 *           download stream.  Steps run on `stream` in submission order
 *           (they share the plan's workspace), so every submit to a plan
 *           must name the same stream, as must other calls on the plan
 *           while steps are in flight.  The results are the same bits as
 *           sr_step_host's for the same inputs.
 *   wait:   blocks until every submitted step's read-back is done, and
 *           every upload, also those of a submit that returned an error
 *           after enqueuing them (its host buffers are read until then).
 * The host buffers of a step must stay valid and unchanged until its
 * read-back is done (sr_step_host_wait, or two submits later, when its
 * staging set is reused); pos is read, vel is read and then overwritten.
 * Page-locked host buffers are needed for the copies to overlap.  The first
 * submit allocates the two staging sets (2 x 56 bytes per particle of the
 * plan's capacity), two streams and six events.  n = 0 copies nothing (the
 * buffers may then be null).  Errors: SR_ERR_ARG (null plan, or a null
 * buffer with n > 0), SR_ERR_CAPACITY (n above the capacity), those of
 * sr_bin and sr_force_kick, SR_ERR_CUDA.
 */
int sr_step_host_submit(sr_plan* plan, const double* pos, float* vel, float* acc, float dt,
                        int64_t n, void* stream);
int sr_step_host_wait(sr_plan* plan);

/*
 * sr_plan_set_variant -- select the pair-kernel variant used by sr_force
 * (same arithmetic and summation order, different launch shape):
 *   0..3: 256-thread blocks, at least 1, 2, 3, 4 resident per SM
 *         (register budgets 255, 128, 85, 64 per thread);
 *   4..6: 128-thread blocks, at least 6, 7, 8 resident per SM
 *         (register budgets 85, 73, 64);
 *   7:    as 2, with split partial sums;
 *   8..11: packed two-wide binary32 pair loop (split partial sums,
 *         batches of 128 neighbours), launch shapes as 1, 2, 4, 3;
 *   12:   the packed loop in batches of 64, launch shape as 3;
 *   13, 14: variants 11 and 12 with the neighbour chunks enumerated for
 *         all cells at once (one lane per cell, then one lane per candidate
 *         chunk) and the next chunk's slots loaded during the current one:
 *         the same chunks in the same order, bit-identical to 11 and 12;
 *   15, 16: grouped kernel for low density: each chunk's 32 slots form
 *         i-groups of G consecutive slots (15: G = 8, 16: G = 16), each
 *         with a neighbour ring culled against its own box, evaluated by
 *         all 32 lanes (32 / G lanes per slot, packed loop, group batches
 *         of 96); 256-thread blocks, 3 per SM.
 * Variants 0..6 are bit-identical (batches of 32 neighbours); so are 8..11
 * and 13 (packed, batches of 128), and 12 and 14.  Split partial sums add even and odd neighbours
 * of a batch separately before the compensated update; variant 7 does so
 * over batches of 32 and variant 12 over batches of 64.  Variants of
 * different groups differ in the last bits.  All variants evaluate the same
 * binary32 pair terms and count the same pairs.
 * Plans with 64-particle chunks support variants 0..3.
 * The counting mode of sr_force (pair_count or per_particle given) runs the
 * grouped kernel when a grouped variant is selected, else one fixed
 * variant-0-order kernel.
 * Errors: SR_ERR_ARG (out of range or not available for the chunk size).
 */
int sr_plan_set_variant(sr_plan* plan, int variant);

/* sr_variant_count -- the number of pair-kernel variants (17: 0..16). */
int sr_variant_count(void);

/* One candidate geometry timed by sr_plan_tune. */
typedef struct sr_tune_entry {
    int32_t chunk_size;    /* particles per chunk (the i-tile of the 32-lane kernels)   */
    int32_t n_cells;       /* cells per axis                                          */
    int32_t variant;       /* the fastest pair-kernel variant on this geometry         */
    float ms;              /* its mean time per launch (ms)                            */
} sr_tune_entry;

/*
 * sr_plan_tune -- per-plan autotuner over the tile shape and the cell
 * geometry, then the kernel variant (Sec. 2.1 sizes the blocks to the
 * load; here the sizes are chosen by timing).  Candidates: chunk size 32
 * or 64, and cells per axis: the automatic count, and counts giving about
 * 3/4 and 4/3 of its cell side where the side stays above r_c.  For each,
 * a plan for n_max particles is created, pos (device, n rows of binary64
 * x, y, z) binned, and every pair-kernel variant timed (sr_autotune, reps
 * launches each); the plan of the fastest candidate is returned in *out,
 * the others are destroyed.  params->n_cells and params->chunk_size are
 * ignored (the candidates set them).  One volume only.
 * entries: host array of at least 6 (nullable), receives each candidate's
 * geometry, best variant and time; *n_entries (nullable) their count.
 * A set-up call: it allocates, synchronises, and must not be captured.
 * Errors: as sr_plan_create and sr_bin; SR_ERR_ARG (null out or pos,
 * reps < 1).
 */
int sr_plan_tune(const sr_params* params, int64_t n_max, const double* pos, int64_t n, int reps,
                 sr_plan** out, sr_tune_entry* entries, int* n_entries, void* stream);

/*
 * sr_autotune -- time each pair-kernel variant on the data of the last
 * sr_bin (reps launches each, CUDA events on stream, synchronising) and
 * keep the fastest.  When the second fastest is within 3% of it, the two
 * are timed again, one launch of each in turn over 2 reps + 1 rounds, and
 * the faster total is kept.  acc: device float4 rows used as scratch output.
 * ms_out: host float[sr_variant_count()], nullable, receives the mean time
 * per variant of the first pass (0 for variants not available for the
 * plan's chunk size).
 * This is a set-up call: it synchronises and must not be captured.
 * Errors: SR_ERR_STATE before the first sr_bin, SR_ERR_ARG, SR_ERR_CUDA.
 */
int sr_autotune(sr_plan* plan, float* acc, int reps, float* ms_out, void* stream);

/*
 * sr_graph_capture -- record one whole step (sr_bin of pos, then
 * sr_force_kick into acc and vel by dt, for n particles) on stream into a CUDA graph
 * owned by the plan, replacing any earlier one.  Nothing runs during the
 * capture.  pos, vel, acc: device buffers that every replay reads and
 * writes in place (refill their contents, keep the pointers).  stream must
 * not be the legacy default stream (NULL), which cannot be captured.
 * Errors: SR_ERR_ARG (null pointers or stream), SR_ERR_CAPACITY, SR_ERR_CUDA.
 */
int sr_graph_capture(sr_plan* plan, const double* pos, float* vel, float* acc, float dt, int64_t n,
                     void* stream);

/* sr_graph_launch -- replay the captured step on stream (one graph launch).
 * Errors: SR_ERR_STATE if nothing was captured, SR_ERR_CUDA. */
int sr_graph_launch(sr_plan* plan, void* stream);

/* sr_last_error -- message of the last failure on this thread ("" if none). */
const char* sr_last_error(void);

/* sr_launch_count -- number of kernels this library has launched so far
 * (process-wide, all threads).  The kernels of a graph made by
 * sr_graph_capture count at each sr_graph_launch, not at the capture.
 * Kernels captured by the caller's own stream capture count once, when
 * they are captured. */
int64_t sr_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SR_H */
