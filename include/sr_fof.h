/*
 * sr_fof.h -- C ABI of the friends-of-friends (FOF) halo finder.
 *
 * The paper finds halos with FOF (Sec. 2.2, Sec. 3.3): two particles are
 * friends when closer than the linking length (b times the mean
 * inter-particle spacing, b = 0.168 fiducial or 0.2), and halos are the
 * groups connected by friendship, kept down to 40 particles; the halo
 * catalogue then feeds the center finder (sr_centers.h).  Readings:
 *
 *   friends iff s < link^2, d = x_j - x_i with both positions folded into
 *   [0, L) (the modulo that takes a remainder's sign from L), then
 *   d <- d - L rint(d / L) per axis, s = (dx dx + dy dy) + dz dz, every
 *   operation rounded to binary64 in that order; the device decides most
 *   pairs with a binary32 predicate in the plan's fine-grid units and sends
 *   the pairs within a relative 2^-10 of link^2 to the binary64 test, so the
 *   decisions, and the labels, are exact;
 *   a group's tag is its smallest particle index; groups of at least
 *   min_members particles become halos 0, 1, ... in increasing tag order;
 *   other particles get label -1.
 *
 * The finder works on a plan binned (sr_bin) with the same positions: it
 * visits the plan's chunks and their neighbour chunks within the linking
 * length and joins friends in a lock-free union-find over caller indices
 * (a root is only ever linked under a smaller root, so every group's root
 * is its tag whatever the order of the links).  Conventions are those of
 * sr.h.
 */
#ifndef SR_FOF_H
#define SR_FOF_H

#include <stdint.h>

#include "sr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sr_fof sr_fof;

typedef struct sr_fof_info {
    int64_t n_particles;   /* n of the last run                                   */
    int64_t n_halos;       /* groups with at least min_members particles          */
    int64_t n_members;     /* particles in those halos                            */
    int64_t max_members;   /* largest halo                                        */
    int64_t links;         /* friend pairs found (each unordered pair once)       */
    int64_t band_checks;   /* pairs decided by the binary64 test                  */
    int64_t tests;         /* particle pairs tested with the binary32 predicate   */
    int64_t error;         /* 0, or 1 if a union-find loop hit its iteration bound */
} sr_fof_info;

/*
 * sr_fof_create -- workspace for up to n_max particles (5 int32 per particle).
 * Errors: SR_ERR_ARG (n_max < 1 or > 2^31 - 1), SR_ERR_CUDA.
 */
int sr_fof_create(int64_t n_max, sr_fof** out);

int sr_fof_destroy(sr_fof* f);

/*
 * sr_fof_run -- FOF groups of the n particles the plan was last binned with.
 *   pos:         device, the same n rows (x, y, z) binary64 given to sr_bin;
 *   link:        linking length (> 0, and below the plan's cell side so that
 *                the 27 neighbour cells hold every friend);
 *   labels:      device int32[n] out, caller order: halo id or -1;
 *   halo_sizes:  device int32[n] out, nullable: entry h is the size of halo h
 *                (h < n_halos of sr_fof_get_info); the rest is unspecified.
 * Errors: SR_ERR_ARG (null pointers with n > 0, link out of range, min_members < 1),
 * SR_ERR_STATE (plan not binned, or binned with a different n),
 * SR_ERR_CAPACITY (n > n_max).
 */
int sr_fof_run(sr_fof* f, sr_plan* plan, const double* pos, int64_t n, double link, int min_members,
               int32_t* labels, int32_t* halo_sizes, void* stream);

/*
 * sr_fof_get_info -- counts of the last run; synchronises its stream.
 * Errors: SR_ERR_ARG, SR_ERR_STATE (no run yet), SR_ERR_TIMEOUT (out is
 * filled; a union-find loop of that run reached its iteration limit, the
 * labels are not valid; the workspace stays usable).
 */
int sr_fof_get_info(sr_fof* f, sr_fof_info* out);

/*
 * sr_fof_set_iteration_limit -- bound of every union-find loop of later
 * runs (0 restores the default, 2^24).  A small limit makes the loops run
 * out on purpose, which exercises the timeout path without any device
 * fault.  Errors: SR_ERR_ARG (null, negative).
 */
int sr_fof_set_iteration_limit(sr_fof* f, int64_t max_iter);

#ifdef __cplusplus
}
#endif

#endif /* SR_FOF_H */
