/*
 * sr_centers.h -- C ABI of the halo center finder.
 *
 * After halos have been identified, the paper's in-situ analysis (Sec. 2.2)
 * locates each halo's center at its potential minimum, the "most bound
 * particle", with a direct pair sum over the halo's members run on the GPU.
 * Reading used here (the paper gives no formula): unit masses, G = 1, each
 * halo treated as isolated, Plummer softening eps, minimum image in the
 * periodic box of side L:
 *
 *   phi_i = - sum_{j in halo(i), j != i} (|d_ij|^2 + eps^2)^(-1/2),   d_ij = x_j - x_i,
 *   center(h) = argmin_{i in h} phi_i, ties to the smaller caller index.
 *
 * Conventions are those of sr.h: SR_* status codes, sr_last_error() for the
 * message, caller-owned device buffers, stream as void*, calls that only
 * enqueue (no allocation, free or synchronisation) unless stated.
 *
 * Numerics: pair terms in binary32 with the hardware reciprocal square
 * root; each halo's members are stored as binary32 offsets from the halo's
 * first member (its smallest caller index), computed in binary64 with the
 * minimum image; per-tile binary32 partial sums are added as 64-bit fixed
 * point (scale 2^S, S chosen from n and eps so that no sum can overflow), so
 * the result does not depend on the order in which tiles finish.
 */
#ifndef SR_CENTERS_H
#define SR_CENTERS_H

#include <stdint.h>

#include "sr.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Kernels of sr_centers_run (sr_centers_set_variant). */
#define SR_CENTERS_SYMMETRIC  0  /* one rsqrt per unordered pair, both members updated (default) */
#define SR_CENTERS_PLAIN      1  /* one thread per member summing over its whole halo (gather) */

/* Workspace: sorted member table, per-halo and per-tile tables, fixed-point
 * accumulators.  Owned by the library. */
typedef struct sr_centers sr_centers;

/* Work counts of the last sr_centers_run (host; sr_centers_info synchronises). */
typedef struct sr_centers_info {
    int64_t n_particles;      /* n of the last run                                   */
    int64_t n_members;        /* particles with a label in [0, n_halos)               */
    int64_t n_halos;          /* halos of the last run (including empty ones)         */
    int64_t max_members;      /* largest halo                                         */
    int64_t pairs;            /* sum over halos of N_h (N_h - 1) / 2: unordered pairs */
    int64_t items;            /* work items of the symmetric kernel                   */
    int64_t evaluated;        /* unordered pair terms the symmetric kernel evaluates  */
    int32_t fixed_shift;      /* S of the fixed-point accumulators                    */
    int32_t variant;          /* SR_CENTERS_*                                         */
    int64_t bad_labels;       /* labels < -1 or >= n_halos (treated as -1)            */
    int64_t wide_members;     /* members farther than L/4 from their halo's first one */
    int64_t check_code;       /* bounds-checked build (sr_build_checked): code of the
                                 first failed bounds check of the last run, 0 = none */
} sr_centers_info;

/*
 * sr_centers_create -- workspace for up to n_max particles and n_halos_max
 * halos (device memory of about 90 bytes per particle plus 64 per halo).
 * Errors: SR_ERR_ARG (n_max < 1 or > 2^30, n_halos_max < 1 or > 2^26),
 * SR_ERR_CUDA (allocation failed).
 */
int sr_centers_create(int64_t n_max, int32_t n_halos_max, sr_centers** out);

int sr_centers_destroy(sr_centers* c);

/*
 * sr_centers_set_variant -- choose the kernel of later runs (SR_CENTERS_*).
 * Errors: SR_ERR_ARG (unknown variant).
 */
int sr_centers_set_variant(sr_centers* c, int variant);

/*
 * sr_centers_run -- potentials and most-bound particles of n_halos halos.
 *   pos:    device, n rows (x, y, z) binary64; any finite values (the
 *           minimum image makes positions outside [0, L) harmless).
 *   labels: device, n int32: halo id in [0, n_halos), or -1 for a particle
 *           in no halo.  Out-of-range labels are counted (bad_labels) and
 *           treated as -1.
 *   phi:        device, n binary64 out, nullable: phi_i in caller order,
 *               0 for particles in no halo.
 *   center:     device, n_halos int64 out, nullable: caller index of each
 *               halo's most bound member, -1 for a halo without members.
 *   center_phi: device, n_halos binary64 out, nullable: its potential
 *               (+infinity for an empty halo).
 * Precondition: every member lies within L/4 (per axis, minimum image) of
 * its halo's first member, so that offset differences are minimum images;
 * members beyond are counted (wide_members, sr_centers_info) and their
 * halo's potentials are not reliable.
 * Errors: SR_ERR_ARG (null workspace/pos/labels, n < 0, n_halos < 0,
 * box <= 0, eps <= 0, non-finite box or eps), SR_ERR_CAPACITY (n or
 * n_halos above the workspace's maxima), SR_ERR_CUDA (launch failure).
 */
int sr_centers_run(sr_centers* c, const double* pos, const int32_t* labels, int64_t n,
                   int32_t n_halos, double box, double eps, double* phi, int64_t* center,
                   double* center_phi, void* stream);

/*
 * The three stages of sr_centers_run, for callers that time or repeat them
 * separately (same arguments, same errors; each only enqueues):
 *   sr_centers_prepare   -- sort members by halo, build the member slots,
 *                           tile rows and work items (steps 1-3);
 *   sr_centers_potential -- the pair sums of the selected kernel (step 4),
 *                           from zeroed accumulators, so it can be repeated;
 *   sr_centers_finish    -- phi in caller order and the per-halo argmin
 *                           (step 5); phi, center, center_phi nullable.
 * Errors beyond sr_centers_run's: SR_ERR_STATE when a stage is called
 * before the one it depends on.
 */
int sr_centers_prepare(sr_centers* c, const double* pos, const int32_t* labels, int64_t n,
                       int32_t n_halos, double box, double eps, void* stream);
int sr_centers_potential(sr_centers* c, void* stream);
int sr_centers_finish(sr_centers* c, double* phi, int64_t* center, double* center_phi, void* stream);

/*
 * sr_centers_get_info -- counts of the last prepared input; synchronises the
 * stream of the last stage.  Errors: SR_ERR_ARG (null), SR_ERR_STATE (nothing
 * prepared yet).
 */
int sr_centers_get_info(sr_centers* c, sr_centers_info* out);

#ifdef __cplusplus
}
#endif

#endif /* SR_CENTERS_H */
