/*
 * sr_pm.h -- C ABI of the long-range side: cloud-in-cell (CIC) deposit,
 * 3-d FFT, CIC-compensated power spectrum and the Gaussian-filtered
 * particle-mesh (PM) acceleration.
 *
 * Sec. 2 computes the long-range force with a spectrally filtered PM solver
 * on a uniform grid; Sec. 4.1 measures the matter power spectrum on the fly
 * by depositing the particles onto the PM grid with CIC, Fourier
 * transforming, binning |delta(k)|^2 in |k| and dividing by the CIC
 * window.  Readings (the paper prints no formulas):
 *
 *   grid      n_g^3 points at (i, j, k) D, D = L / n_g, periodic; arrays are
 *             indexed [x][y][z] with z fastest;
 *   CIC       u = fold(x) / D, i0 = floor(u), f = u - i0, weights (1-f, f)
 *             per axis to i0 and i0+1, products to the 8 corners;
 *   delta     counts / nbar - 1, nbar = n / n_g^3;
 *   FFT       delta_k = sum_x delta(x) exp(-i k.x), k = 2 pi m / L;
 *   P(k)      (L^3 / n_g^6) |delta_k|^2 / W(k)^2, W = prod_a sinc^2(k_a D / 2),
 *             binned by b = round(|m|), b = 1 .. n_g/2 (both k and -k count);
 *   force     a(k) = i k (4 pi / k^2) exp(-k^2 sigma^2) C(k) / W(k)^2,
 *             C the DFT of the CIC counts, the gradient's Nyquist
 *             component 0, a(x) = ifft(a(k)) / D^3, CIC interpolation to
 *             the particles (G = 1, unit masses; sigma the split scale of
 *             the short-range force law, so the two halves sum to Newton).
 *
 * Conventions are those of sr.h (status codes, sr_last_error(), caller-owned
 * device buffers, stream as void*, enqueue-only calls unless stated).
 * Numerics: CIC cells and fractions in binary64, corner weights in
 * binary32, summed as 64-bit fixed point (the density grid does not depend
 * on the order of the atomics); FFT and k-space arithmetic in binary32
 * complex with twiddle tables computed in binary64; power-spectrum terms in
 * binary32 summed in binary64 in a fixed order.
 */
#ifndef SR_PM_H
#define SR_PM_H

#include <stdint.h>

#include "sr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sr_pm sr_pm;

/* Export selectors for sr_pm_copy (device destination). */
#define SR_PM_EXPORT_COUNTS   0  /* binary64[n_g^3]: CIC counts of the last deposit            */
#define SR_PM_EXPORT_DELTA_K  1  /* float2[n_g^3]: FFT of delta of the last transform            */
#define SR_PM_EXPORT_ACCEL    2  /* float4[n_g^3]: long-range acceleration on the grid (x,y,z,0) */

/*
 * sr_pm_create -- workspace for an n_g^3 grid (n_g a power of two in
 * [16, 1024]) of a periodic box of side box, split scale sigma, for up to
 * n_max particles.  Device memory: about 48 n_g^3 bytes plus a mode
 * permutation built once here (it synchronises).
 * Errors: SR_ERR_ARG (bad n_g, box <= 0, sigma < 0, n_max < 1 or > 2^31-1),
 * SR_ERR_CUDA.
 */
int sr_pm_create(int n_grid, double box, double sigma, int64_t n_max, sr_pm** out);

int sr_pm_destroy(sr_pm* pm);

/*
 * sr_pm_deposit -- CIC counts of n particles (pos: device, n rows (x,y,z)
 * binary64, any finite values, folded into [0, L)).
 * Errors: SR_ERR_ARG (null, n < 1), SR_ERR_CAPACITY (n > n_max).
 */
int sr_pm_deposit(sr_pm* pm, const double* pos, int64_t n, void* stream);

/*
 * sr_pm_deposit_binned -- the same CIC counts, bit for bit, computed over
 * the cell order of a one-volume short-range plan that binned these n
 * positions with the same box (Sec. 2: both halves of the force split read
 * the same particles; the short-range binning is reused).  Each warp
 * deposits one chunk (at most 32 particles of one binning cell) into a
 * shared-memory tile of the cell's mesh points first and then adds the
 * tile to the mesh, so most of the 8 atomics per particle stay on chip.
 * pos: device, the n rows the plan binned (caller order).  If the plan's
 * cells hold too many mesh points for a tile, this falls back to
 * sr_pm_deposit (more than 6 mesh cells per binning cell along an axis).
 * Errors: SR_ERR_ARG (null argument, a batch plan, n different from the
 * plan's binning, another box), SR_ERR_STATE (plan not binned),
 * SR_ERR_CAPACITY (n > n_max).
 */
int sr_pm_deposit_binned(sr_pm* pm, const sr_plan* plan, const double* pos, int64_t n, void* stream);

/*
 * sr_pm_transform -- delta of the last deposit and its forward FFT, the
 * input of sr_pm_power and sr_pm_force.  Errors: SR_ERR_STATE before a
 * deposit.
 */
int sr_pm_transform(sr_pm* pm, void* stream);

/*
 * sr_pm_power -- the power spectrum of the last transform: k_mean, power
 * (binary64) and modes (int64) per shell b = 1 .. n_g/2, device arrays of
 * n_g/2 entries each (nullable individually).  Errors: SR_ERR_STATE before a
 * transform.
 */
int sr_pm_power(sr_pm* pm, double* k_mean, double* power, int64_t* modes, void* stream);

/*
 * sr_pm_force -- long-range accelerations of the last transform's density,
 * interpolated at the n particles pos (usually the deposited ones) into
 * acc (device, float4 rows (x, y, z, w)); accumulate = 0 overwrites x, y, z
 * and sets w = 0, accumulate = 1 adds to x, y, z (e.g. onto the short-range
 * accelerations of sr_force).  Errors: SR_ERR_STATE before a transform,
 * SR_ERR_ARG, SR_ERR_CAPACITY.
 */
int sr_pm_force(sr_pm* pm, const double* pos, int64_t n, float* acc, int accumulate, void* stream);

/*
 * sr_pm_fft -- in-place 3-d FFT of a device float2[n_g^3] array ([x][y][z],
 * z fastest) with the workspace's size: inverse = 0 computes
 * sum_x f(x) exp(-i k.x), inverse = 1 sum_k F(k) exp(+i k.x) (no 1/n_g^3).
 */
int sr_pm_fft(sr_pm* pm, float* data, int inverse, void* stream);

/*
 * sr_pm_copy -- copy an internal grid (SR_PM_EXPORT_*) to the device buffer
 * dst.  Errors: SR_ERR_ARG (unknown selector), SR_ERR_STATE (not computed).
 */
int sr_pm_copy(sr_pm* pm, int what, void* dst, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SR_PM_H */
