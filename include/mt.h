/*
 * mt.h -- C ABI of the GB300 null-geodesic ray tracer.
 *
 * The method is the one of Breton & Reverdy, arXiv 2111.08744
 * ("Magrathea-Pathfinder"): photons are integrated backward from an observer
 * on the null geodesics of the weakly perturbed FLRW metric (Eq. 1),
 *     ds^2 = a^2(eta) [ -(1 + 2 phi) d eta^2 + (1 - 2 phi) dx^2 ],
 * with the geodesic equations (Eqs. 2-3) and d phi / d lambda from the chain
 * rule (Eq. 4), by classical RK4 in the affine parameter with N steps per
 * AMR cell (Sect. 2.2); phi and grad phi are CIC-interpolated (Eq. 8) from an
 * octree with the level fallback of Sect. 2.2 / Fig. 1; per ray the library
 * returns the end point on an iso-eta surface and the redshift decomposition
 * of Eqs. (23)-(28) with no velocity terms.
 *
 * Units: c = 1, lengths and conformal time in h^-1 Mpc, phi = Phi / c^2.
 *
 * Ownership: every buffer passed in stays owned by the caller; the library
 * owns what mt_build_octree allocates until mt_free.  All GPU work is
 * enqueued on the CUDA stream given as `stream` (a cudaStream_t, NULL for the
 * legacy default stream); functions return once the work is enqueued unless
 * stated otherwise.  Calls that use the same octree must be ordered on one
 * stream (they share the octree's small device work area).
 *
 * Errors: functions return an mt_status.  Host-side validation failures
 * return MT_ERR_INVALID_ARG (or the specific code below) before any GPU work
 * is enqueued.  Per-ray outcomes are in the `status` output; kernel-level
 * faults (a hash probe run that exceeds the table) set a device flag read by
 * mt_device_status.
 */
#ifndef MT_H
#define MT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MT_OK = 0,
  MT_ERR_INVALID_ARG = 1,   /* a pointer, size, layout or parameter is invalid */
  MT_ERR_OOM = 2,           /* device memory allocation failed */
  MT_ERR_CUDA = 3,          /* a CUDA runtime call failed (no device, launch failure, ...) */
  MT_ERR_NOT_FULL_TREE = 4, /* keys unsorted, an octet incomplete or a parent missing (Sect. 2.1) */
  MT_ERR_TIMEOUT = 5,       /* a device-side iteration bound was reached */
  MT_ERR_OOB = 6,           /* a device-side index check failed */
  MT_ERR_UNSUPPORTED = 7    /* valid request this build does not handle (limits below) */
} mt_status;

/* field precision of the octree records */
enum { MT_FIELD_FP64 = 0, MT_FIELD_FP32 = 1 };

/* per-ray status values */
enum { MT_RAY_OK = 0, MT_RAY_LEFT_DOMAIN = 1, MT_RAY_MAX_STEPS = 2, MT_RAY_NONFINITE = 3 };

/* level-data residency */
enum { MT_HOST = 0, MT_DEVICE_COPY = 1, MT_DEVICE_BORROW = 2 };

/* limits of this build */
#define MT_MAX_LEVELS 8    /* refined levels above the coarse grid */
#define MT_MAX_SLICES 16   /* time slices */
#define MT_MAX_CONES 256   /* light cones (observers) per trace call */

typedef struct mt_octree mt_octree; /* opaque, library-owned */

/*
 * Grid description (Sect. 2.1).  Level l has N_l = n_coarse * 2^l cells per
 * axis of size dx_l = box / N_l; n_coarse must be a power of two and
 * N_{n_levels} <= 2^21, and no level may hold more than 2^32 cells (the
 * kernels address records by 32-bit rows, so N_0 <= 1024).  Cell (i, j, k)
 * of level l has the Morton key with bit 3b = bit b of i, bit 3b+1 = bit b
 * of j, bit 3b+2 = bit b of k, so the 8 children of a cell with key K have
 * keys 8K .. 8K+7.
 */
typedef struct {
  double box;               /* comoving side of the (periodic) box, > 0 */
  int32_t n_coarse;         /* N_0, power of two in [1, 1024] */
  int32_t n_levels;         /* refined levels, 0 .. MT_MAX_LEVELS */
  int32_t periodic;         /* 1: positions wrap into the box; 0: rays stop at the box edge */
  int32_t n_slices;         /* time slices, 1 .. MT_MAX_SLICES */
  const double* slice_eta;  /* host [n_slices], strictly ascending conformal times */
  int32_t precision;        /* MT_FIELD_FP64 (double records) or MT_FIELD_FP32 (float records) */
  int32_t pad;
} mt_grid_desc;

/*
 * Cells of one level.  Level 0 must hold all N_0^3 cells in Morton order
 * (keys 0 .. N_0^3 - 1; `keys` may be NULL there).  A refined level holds
 * whole octets: count is a multiple of 8, keys strictly ascending, each
 * octet's keys are 8K .. 8K+7, and its parent K exists on the level below
 * (the full-tree rule of Sect. 2.1).
 * records: [count][n_slices][4] of double (FP64) or float (FP32):
 *          phi, d phi/dx, d phi/dy, d phi/dz per cell and slice.
 */
typedef struct {
  const uint64_t* keys;   /* [count] */
  const void* records;    /* [count][n_slices][4] */
  int64_t count;
  int32_t residency;      /* MT_HOST, MT_DEVICE_COPY, or MT_DEVICE_BORROW (device data kept by
                             reference; it must outlive the octree and must not change) */
  int32_t pad;
} mt_level_data;

/*
 * mt_build_octree -- validate a full octree and build the device structure:
 * per-level record arrays in Morton order, the coarse level directly indexed,
 * each refined level behind an open-addressing hash from the parent key to its
 * octet (Sect. 2.1: flattened AMR with a unique binary index per cell).
 *
 * bg_table: host [bg_n][4] nodes (eta_j, a_j, H_j, dH/deta_j) of the
 * background (H = a'/a), strictly ascending and uniformly spaced in eta
 * (Sect. 2.2: a(eta) and a'(eta) from external pre-computed tables); the last
 * node is the observer's time eta_o (a = 1).  The library interpolates
 * a(eta) and H(eta) by cubic Hermite with slopes a H and dH/deta.
 *
 * levels: [n_levels + 1].  On success *out receives the handle.  Synchronous:
 * returns after the device structure is built and validated.
 * Errors: MT_ERR_INVALID_ARG (descriptor), MT_ERR_NOT_FULL_TREE, MT_ERR_OOM,
 * MT_ERR_CUDA.  On error *out is NULL and nothing stays allocated.
 */
mt_status mt_build_octree(const mt_grid_desc* grid, const mt_level_data* levels, const double* bg_table,
                          int32_t bg_n, void* stream, mt_octree** out);

/*
 * Interpolation of phi and grad phi at the photon (Sect. 2.2, Eqs. 7-9), each with the level
 * fallback of Sect. 2.2: start at the most refined level containing the photon and go one level
 * coarser while one of the cells the scheme needs is absent.
 *   NGP: the containing cell itself (no fallback needed);
 *   CIC: the 8 cells around the point, trilinear weights prod(1 - |r_i|);
 *   TSC: the containing cell and its 26 neighbours (the same 27 cells anywhere inside it),
 *        weights prod W_TSC(r_i), W_TSC = 3/4 - r^2 (|r| < 1/2), (3/2 - |r|)^2 / 2 (< 3/2).
 * The reverse mode of mt_trace_rays_adjoint (dL_dxi) supports CIC only.
 */
typedef enum { MT_INTERP_CIC = 0, MT_INTERP_NGP = 1, MT_INTERP_TSC = 2 } mt_interp;

/*
 * Trace parameters.  Rays [ray_begin[c], ray_begin[c+1]) belong to cone c
 * with observer observer[c] at eta_o and stop on the iso-eta surface
 * eta_stop(c) = eta(a = 1 / (1 + z_max[c])) (Sects. 2.3.2 and 2.4: the stop criterion, here
 * p = eta), found by bisection on the background interpolant.
 */
typedef struct {
  int32_t n_cones;          /* 1 .. MT_MAX_CONES */
  int32_t steps_per_cell;   /* N >= 1 (Sect. 2.2; 4 in common settings) */
  int32_t gravity_on;       /* 0: phi = 0 (FLRW / Born trajectories, Sect. 2.2), 1: full equations */
  int32_t interp;           /* weighting function of Sect. 2.2: MT_INTERP_CIC (0, Eq. 8),
                               MT_INTERP_NGP (Eq. 7) or MT_INTERP_TSC (Eq. 9) */
  const double* observer;   /* host [n_cones][3] */
  const double* z_max;      /* host [n_cones], >= 0 */
  const int64_t* ray_begin; /* host [n_cones + 1], ray_begin[0] = 0, non-decreasing */
  int64_t max_steps;        /* per-ray step cap (> 0); reaching it sets MT_RAY_MAX_STEPS */
} mt_trace_params;

/*
 * Per-ray outputs, caller-owned DEVICE buffers of length N (x: [3][N],
 * k: [4][N]).  Any pointer may be NULL to skip that output.
 *   x       end position, unwrapped comoving coordinates
 *   k       end wave vector k^0, k^1, k^2, k^3 (k^0 < 0: past-directed)
 *   eta     end conformal time; lambda: affine parameter reached
 *   chi     |x - x_o|; path: integral of |k| d lambda
 *   z0, z1, z4, z5   Eqs. (23), (24), (27), (28) with v = 0 (a_o = 1)
 *   d_a     a_s chi; d_l = (1 + z5)^2 d_a
 *   phi_o, phi_s     interpolated potential at the observer / end point
 *   isw     integral of d phi / d eta over eta from eta_s to eta_o (Eq. 27)
 *   n_steps RK4 steps taken; level: most refined level containing the end point
 *   status  MT_RAY_*
 */
typedef struct {
  double* x;
  double* k;
  double* eta;
  double* lambda;
  double* chi;
  double* path;
  double* z0;
  double* z1;
  double* z4;
  double* z5;
  double* d_a;
  double* d_l;
  double* phi_o;
  double* phi_s;
  double* isw;
  int32_t* n_steps;
  int32_t* level;
  int32_t* status;
  double* xi;   /* [3][N] end point moved along k onto the stop surface:
                   xi = x - (k / k0) (eta - eta_stop) */
} mt_ray_out;

/*
 * mt_trace_rays -- integrate n_rays null geodesics (Sect. 2.2).
 * dirs: device [3][n_rays] unit observed directions n (the ray starts with
 * k^0 = -1, k^i = n sqrt((1 + 2 phi_o)/(1 - 2 phi_o)), the null condition).
 * One persistent launch serves every cone; warps pull rays from a device
 * queue as rays finish.  FP64 octrees integrate and interpolate in double;
 * FP32 octrees interpolate in float and keep the ray state in double.
 * Errors: MT_ERR_INVALID_ARG (parameters, NULL tree/dirs), MT_ERR_CUDA.
 */
mt_status mt_trace_rays(const mt_octree* tree, const mt_trace_params* params, const double* dirs, int64_t n_rays,
                        const mt_ray_out* out, void* stream);

/*
 * mt_trace_rays_adjoint -- derivatives of the ray map (Sect. 2.3 distortion matrix, and the
 * gradient of a loss on the end points with respect to the gridded potential).
 *
 * The end point of a ray is taken on its iso-eta stop surface:
 *     xi = x - (k / k0) (eta - eta_stop).
 * Forward mode (jac or lens non-NULL): two tangents of the FP64 RK4 map along the observer's
 * screen vectors e_1 = (-sin t1, cos t1, 0), e_2 = (-cos t1 cos t2, -sin t1 cos t2, sin t2)
 * (t1, t2 the azimuth and polar angle of the direction; Sect. 2.3.2) give
 *     A_ab = (d xi / d theta_b) . e~_a / chi,   chi = |xi - x_o|,
 * with e~ the beta-screen of the end point (Eq. 21 in the limit of an infinitesimal beam,
 * without neighbouring rays).  jac: device [4][N] = A11, A12, A21, A22.  lens: device
 * [5][N] = kappa, gamma_1, gamma_2, omega, det A (= 1/mu) from Eq. (11).  Asynchronous.
 *
 * Reverse mode (dL_dxi and dL_drec non-NULL): given dL/dxi (device [3][N]), ACCUMULATES
 * (+=) dL/d(record) into dL_drec[l] (device FP64 buffers [count_l][n_slices][4], one per
 * level 0..n_levels, same layout as the records; a NULL entry skips that level), through the
 * exact adjoint of the discrete map (RK4 stages, CIC weights, time slices, step-size and
 * last-step dependence, and phi at the observer).  States are checkpointed every
 * checkpoint_every (1..64) steps and each segment is recomputed.  Synchronous: the call
 * counts each ray's steps, allocates temporary buffers (the checkpoints, 8 doubles each; the
 * step counts; on FP32 octrees also 9 doubles per ray that the forward pass leaves for the
 * sweep), runs the forward pass and the sweep and frees them.  Rays that do not end with
 * MT_RAY_OK add nothing.
 *
 * Both modes integrate each ray as mt_trace_rays does and differentiate that map: FP64
 * arithmetic on an FP64 octree; on an FP32 octree the mixed step (FP32 stages, FP64 state) with
 * FP32 stage derivatives and an FP64 tangent / cotangent state (reverse mode: per-lane FP32
 * accumulation of the record cotangents, added to dL_drec with FP64 atomics).  Reverse mode
 * supports MT_INTERP_CIC only (others: MT_ERR_UNSUPPORTED).  Both write the ray outputs `out`
 * (NULL pointers skip an output) of their integration.  checkpoint_every sets the checkpoint
 * memory (8 doubles per checkpoint) and the length of the segments the sweep holds at a time;
 * every step is integrated once more in the sweep whatever its value.
 * Errors: as mt_trace_rays; MT_ERR_INVALID_ARG if neither mode is requested or reverse-mode
 * arguments are incomplete; MT_ERR_OOM if the checkpoint buffer cannot be allocated.
 */
mt_status mt_trace_rays_adjoint(const mt_octree* tree, const mt_trace_params* params, const double* dirs,
                                int64_t n_rays, const mt_ray_out* out, double* jac, double* lens,
                                const double* dL_dxi, double* const* dL_drec, int32_t checkpoint_every,
                                void* stream);

/*
 * mt_trace_rays_jvp -- forward-mode derivative of the end points with respect to the gridded
 * potential records: dxi = J v for the map records -> xi (xi = x - (k / k0)(eta - eta_stop), the
 * end point on the iso-eta surface), the Jacobian-vector product whose transpose the reverse mode
 * of mt_trace_rays_adjoint applies.  The same differentiable discrete map: RK4 stages of Eqs.
 * (2)-(4), CIC weights (Eq. 8) at the level and slices the trace uses, the step size and the
 * shortened last step, and phi at the observer in the initial wave vector.
 * d_rec: [n_levels + 1] device FP64 buffers [count_l][n_slices][4] (same layout as the records; a
 * NULL entry is a zero perturbation on that level).  dxi: device [3][N], overwritten (0 for rays
 * that do not end with MT_RAY_OK).  `out` receives the rays' outputs (NULL pointers skip them).
 * FP64 arithmetic, records of the octree's precision; MT_INTERP_CIC only (others:
 * MT_ERR_UNSUPPORTED).  Asynchronous on `stream`; allocates nothing.
 * Errors: as mt_trace_rays; MT_ERR_INVALID_ARG for NULL d_rec or dxi.
 */
mt_status mt_trace_rays_jvp(const mt_octree* tree, const mt_trace_params* params, const double* dirs, int64_t n_rays,
                            const mt_ray_out* out, const double* const* d_rec, double* dxi, void* stream);

/*
 * mt_trace_rays_lensing -- the infinitesimal-beam distortion matrix of Sect. 2.3.1 along each
 * traced ray (Eq. 12):
 *   A_ab = delta_ab - 2 int_0^chi_s dchi (chi_s - chi) chi / chi_s  d_a d_b phi(eta(chi), x(chi)),
 * the Cartesian Hessian of phi from central differences of the interpolated grad phi with the
 * step h = size of the most refined cell containing the photon (Eq. 13; d_i d_j = d_j d_i), its
 * screen components at the photon's angular position seen from the observer (Eqs. 14-16, on the
 * basis e_1 = e_phi, e_2 = -e_theta also used by the finite beams and mt_trace_rays_adjoint), and
 * the trapezoidal rule over the ray's step points (chi = |x - x_o|).  A is symmetric (no
 * rotation).  With params->gravity_on = 0 the rays follow FLRW trajectories: the Born
 * approximation of Sect. 2.3.1.  The rays advance exactly as in mt_trace_rays (same step, same
 * precision rules) and `out` receives their outputs.
 * jac: device [4][N] = A11, A12, A21, A22; lens: device [5][N] = kappa, gamma_1, gamma_2,
 * omega (= 0), det A (= 1/mu); at least one non-NULL.  Asynchronous on `stream`.
 * Errors: as mt_trace_rays; MT_ERR_INVALID_ARG if jac and lens are both NULL.
 */
mt_status mt_trace_rays_lensing(const mt_octree* tree, const mt_trace_params* params, const double* dirs,
                                int64_t n_rays, const mt_ray_out* out, double* jac, double* lens, void* stream);

/*
 * mt_trace_beams -- the finite-beam distortion matrix of Sect. 2.3.2 (Eqs. 17-21) for each of
 * n_beams central directions dirs[:, i]: the central ray and four rays at semi-aperture eps,
 * along n +- tan(eps) e_1 (A, B) and n -+ tan(eps) e_2 (C, D) (normalised; e_1 = e_phi,
 * e_2 = -e_theta of n), all stopped on the cone's iso-eta surface with their end points moved
 * along k onto it (xi).  With the screen basis (e~_1, e~_2) of v = xi_central - x_o
 * (screen = 0, beta-screen) or of the central ray's end wave vector (screen = 1, Sachs screen)
 * and chi = |xi_central - x_o|:
 *   A_a1 = (xi_A - xi_B) . e~_a / (2 chi tan eps),  A_a2 = (xi_D - xi_C) . e~_a / (2 chi tan eps)
 * (the second column as xi_D - xi_C, so that A is the identity without gravity).  jac: device
 * [4][N] = A11, A12, A21, A22; lens: device [5][N] = kappa, gamma_1, gamma_2, omega, det A
 * (Eq. 11); at least one non-NULL.  `out` receives the central rays' outputs.  The rays advance
 * as in mt_trace_rays (same step and precision rules, params->interp honoured); each GPU lane
 * integrates one beam's five rays in turn, so nothing is allocated.  Asynchronous.
 * Errors: as mt_trace_rays; MT_ERR_INVALID_ARG if eps is not in (0, 0.5) rad, screen is not 0 or
 * 1, or jac and lens are both NULL.
 */
mt_status mt_trace_beams(const mt_octree* tree, const mt_trace_params* params, const double* dirs, int64_t n_beams,
                         double eps, int32_t screen, const mt_ray_out* out, double* jac, double* lens, void* stream);

/*
 * mt_find_geodesics -- geodesic finder (Sect. 2.5): for each source at comoving position
 * src[:, i] (device [3][N], absolute box coordinates; source i belongs to the cone of params,
 * whose observer x_o it uses; z_max is ignored), the observed direction theta at x_o whose ray,
 * stopped on the sphere |x - x_o| = chi_s = |src - x_o| (the end point moved back along k onto it),
 * is seen from x_o in the source's direction beta.  Newton on the screen (e_phi, -e_theta) of the
 * current direction, theta_{i+1} = theta_i - A^{-1} (beta_i - beta) (Eq. 22), with A the exact
 * derivative of the discrete map (forward tangents) from the first iteration, until |beta_i - beta|
 * < tol (rad); after max_newton (1..100) iterations, up to max_grid (0..64) rounds of a 5 x 5 grid
 * around the best direction, halving its spacing each round.  Rays advance as in the trace calls;
 * the background table's first node bounds them.  Outputs (device, length N): theta [3][N];
 * jac [4][N] (A11, A12, A21, A22 at the solution, or NULL); resid [N] (|beta_i - beta|, or NULL);
 * iters [N] (Newton iterations + grid rounds + 1, or NULL); status [N]: 0 converged by Newton, 1 by the grid,
 * 2 not converged (theta is the best found), 3 the ray failed; `out` receives the solution ray's
 * outputs at the sphere (x on it; z0..z5, phi_s, isw at that point).  Asynchronous.
 * Errors: as mt_trace_rays's parameter checks; MT_ERR_INVALID_ARG for tol <= 0, out-of-range
 * iteration limits or NULL required arrays.
 */
mt_status mt_find_geodesics(const mt_octree* tree, const mt_trace_params* params, const double* src, int64_t n_src,
                            double tol, int32_t max_newton, int32_t max_grid, const mt_ray_out* out, double* theta,
                            double* jac, double* resid, int32_t* iters, int32_t* status, void* stream);

/*
 * mt_healpix_bin -- HEALPix maps of per-ray quantities (Sect. 2.4 map products: lensing,
 * lensing_born, deflection, phi, isw, steps, relative differences...).  Each direction
 * dirs[:, i] (device [3][n], any length) gets its pixel at resolution nside (a power of two,
 * <= 2^28) in the NESTED (nest = 1) or RING (nest = 0) numbering of Gorski et al. (2005), and
 * values[q][i] (device [k][n]) is ADDED to sums[q][pix] (device [k][12 nside^2]); counts[pix]
 * (device [12 nside^2], may be NULL) gains 1 per ray; ipix (device [n], may be NULL) receives the
 * pixels.  The map of quantity q is sums[q] / counts.  FP64 atomics: the sums' rounding order is
 * not fixed.  Rays shot at pixel centres map one to one.  Asynchronous on `stream`.
 * Errors: MT_ERR_INVALID_ARG (nside, nest, NULL arrays), MT_ERR_CUDA.
 */
mt_status mt_healpix_bin(const double* dirs, int64_t n, const double* values, int32_t k, int64_t nside, int32_t nest,
                         double* sums, double* counts, int64_t* ipix, void* stream);

/*
 * mt_deflection -- the deflection angle of Sect. 2.4, alpha = theta - beta, for rays traced with
 * params (the cone table gives each ray's observer): theta = dirs[:, i] (observed direction),
 * beta = the direction of xi[:, i] - x_o (xi: end points on the stop surface, device [3][N], as
 * written by the trace calls).  alpha: device [3][N] = the components of theta^ - beta^ on the
 * screen (e_phi, -e_theta) of theta, and the angle between theta and beta (rad).  Asynchronous.
 * Errors: as mt_trace_rays's parameter checks; MT_ERR_INVALID_ARG for NULL arrays.
 */
mt_status mt_deflection(const mt_octree* tree, const mt_trace_params* params, const double* dirs, int64_t n_rays,
                        const double* xi, double* alpha, void* stream);

/*
 * mt_pullback_coarse_phi -- dL/dphi_0 on the coarse grid from record cotangents dL_drec
 * (as accumulated by mt_trace_rays_adjoint), through this library's field model:
 *   coarse records  = w_s (phi_0, D phi_0), D the periodic 5-point central difference
 *                     (f[i-2] - 8 f[i-1] + 8 f[i+1] - f[i+2]) / (12 dx_0);
 *   refined records = w_s (I_0[phi_0](x_c), I_0[D phi_0](x_c)) + terms that do not depend
 *                     on phi_0, with I_0 trilinear interpolation of the periodic,
 *                     cell-centred coarse grid at the refined cell's centre x_c;
 *   w_s = slice_weight[s] (host [n_slices]), the time-slice scaling of the potential.
 * dL_dphi0: device [N_0^3] FP64 in the coarse records' (Morton) order, overwritten.
 * Uses a temporary device buffer (4 doubles per coarse cell); synchronous.
 * The paper differentiates nothing; this is the "gradient with respect to the gridded
 * phi" of the differentiable form of the method.
 */
mt_status mt_pullback_coarse_phi(const mt_octree* tree, double* const* dL_drec, const double* slice_weight,
                                 double* dL_dphi0, void* stream);

/*
 * mt_field_from_coarse_phi -- the forward map of the field model of mt_pullback_coarse_phi: the
 * records of every level from the coarse potential phi0 (device [N_0^3] FP64, Morton order), written
 * to records[l] (device FP64 [count_l][n_slices][4], the octree's row order; overwritten):
 *   records_0[c][s] = w_s (phi_0[c], (D phi_0)[c]) + base_0[c][s],
 *   records_l[c][s] = w_s (I_0[phi_0](x_c), I_0[D phi_0](x_c)) + base_l[c][s],
 * with D, I_0 and w_s as there; base[l] (device, same layout; NULL or a NULL entry: zero) holds the
 * terms that do not depend on phi_0 (the records at phi_0 = 0).  The octree supplies the geometry
 * (keys, counts), not its records.  Uses a temporary device buffer (4 doubles per coarse cell);
 * synchronous.  Errors: MT_ERR_INVALID_ARG, MT_ERR_OOM, MT_ERR_CUDA.
 */
mt_status mt_field_from_coarse_phi(const mt_octree* tree, const double* phi0, const double* slice_weight,
                                   const double* const* base, double* const* records, void* stream);

/*
 * mt_trace_rays_noalloc -- the same trace as mt_trace_rays, for callers that must not
 * allocate GPU memory.  The paper has no counterpart: this is a property of this
 * library's interface, not of the method.
 *
 * Who needs it: code that traces from inside a host application whose device memory is
 * owned by another allocator (a framework's caching allocator that has reserved the
 * GPU, or a serving process with a fixed device-memory budget), where a cudaMalloc would
 * fail or is not allowed, and loops that cannot afford cudaMalloc/cudaFree, which may
 * synchronise the whole device.  mt_trace_rays allocates nothing per call either, but its
 * scratch lives in the octree; this entry point's scratch (the ray-queue counter and the
 * cone table) is a static device array of this library, about 160 KiB, present on every
 * GPU that loads the library until the process exits.  It calls no cudaMalloc, cudaFree
 * or other allocating routine.
 *
 * Arguments, outputs and results are those of mt_trace_rays.  Because the cone table sits
 * in the static array instead of the kernel's parameters, up to MT_NOALLOC_MAX_CONES cones
 * are accepted; more return MT_ERR_UNSUPPORTED before any GPU work.
 *
 * The first call on a device looks up the static array's device address
 * (cudaGetSymbolAddress, once per device, with the octree's device current).  Every call
 * clears the queue counter and rewrites the cone table on `stream`, copying the table from
 * pageable host memory, so the call waits for earlier work on `stream` before it returns.
 * All calls share the one array: calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  Device-side faults are flagged in the octree's status word
 * (mt_device_status).
 */
#define MT_NOALLOC_MAX_CONES 4096
mt_status mt_trace_rays_noalloc(const mt_octree* tree, const mt_trace_params* params, const double* dirs,
                                int64_t n_rays, const mt_ray_out* out, void* stream);

/*
 * mt_set_launch_config -- launch shape of mt_trace_rays on this octree (tuning only; results
 * do not depend on it): block_size 64, 128 or 256 threads (0: default 128), blocks_per_sm
 * >= 1 to cap the persistent grid at num_SMs x blocks_per_sm (0: as many as fit).
 * Errors: MT_ERR_INVALID_ARG.
 */
mt_status mt_set_launch_config(mt_octree* tree, int32_t block_size, int32_t blocks_per_sm);

/*
 * mt_set_trace_options -- further tuning of mt_trace_rays on this octree (results do not depend on
 * it): ray_chunk = ray ids a warp claims from the queue at a time (a multiple of 32 in [32, 1024];
 * 0: default 32); staging (FP32 octrees, CIC) = 1: each ray's 8 CIC records of both slices are
 * staged in shared memory and reused while the ray stays in that neighbourhood, 2: read through L1
 * at every stage (no shared memory), 0: default (1).  Errors: MT_ERR_INVALID_ARG.
 */
mt_status mt_set_trace_options(mt_octree* tree, int32_t ray_chunk, int32_t staging);

/*
 * mt_device_status -- synchronise `stream` and return the device-side flag of
 * the last kernels on this octree (MT_OK, MT_ERR_OOB, MT_ERR_TIMEOUT), then
 * clear it.
 */
mt_status mt_device_status(const mt_octree* tree, void* stream);

/*
 * mt_probe_fp64_fma_rate -- measured FP64 fused multiply-add rate of the current device, in
 * lane-operations per second (one FMA of one thread = 1): the denominator of the FP64-pipe
 * roofline reported for the trace kernels.  Not part of the method (the paper has no
 * counterpart): a calibration kernel of independent FMA chains, `iters` per chain, launched
 * num_SMs x (resident blocks) times `repeats` + 1 on `stream` (the first launch warms up), timed
 * with CUDA events; *fma_per_s receives the best rate.  Synchronous; allocates nothing.
 * Errors: MT_ERR_INVALID_ARG (NULL output, iters < 1, repeats < 1), MT_ERR_CUDA.
 */
mt_status mt_probe_fp64_fma_rate(int64_t iters, int32_t repeats, double* fma_per_s, void* stream);

/* mt_free -- release everything mt_build_octree allocated (NULL is ignored).
 * The caller must make sure no enqueued work still uses the octree. */
void mt_free(mt_octree* tree);

/* mt_status_str -- static description of a status code. */
const char* mt_status_str(mt_status s);

/* mt_octree_info -- level counts and device bytes held (for reporting). */
mt_status mt_octree_info(const mt_octree* tree, int64_t* cells_per_level /* [n_levels+1] or NULL */,
                         int64_t* device_bytes /* or NULL */);

#ifdef __cplusplus
}
#endif

#endif /* MT_H */
