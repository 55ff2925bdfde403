// Per-ray device code of the geodesic integrator (Sect. 2.2), shared by the trace kernels.
//
// State per ray: y = (x[3], eta, k0, k[3], I, s) in double, plus lambda.
//   Field precision double: interpolation and right-hand side in double.
//   Field precision float : in-cell fractions, weights, interpolation and the
//     gravitational terms of the right-hand side in float; the background terms,
//     the RK4 combination and the state stay double.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mt_internal.cuh"
#include "mt_mixed.cuh"

namespace mt {

struct OutPtrs {
  double *x, *k, *eta, *lambda, *chi, *path, *z0, *z1, *z4, *z5, *d_a, *d_l, *phi_o, *phi_s, *isw;
  int32_t *n_steps, *level, *status;
  double* xi;
};

struct TraceArgs {
  int steps_per_cell;
  int gravity_on;
  long long max_steps;
  long long n_rays;
  int interp;     // MT_INTERP_*
  int ray_chunk;  // trace kernels: ray ids a warp claims per refill (a multiple of 32)
};

// The octree's field as a kernel argument, carrying the trace's interpolation scheme.
inline DevField launch_field(const mt_octree* tree, const TraceArgs& A) {
  DevField f = tree->f;
  f.interp = A.interp;
  return f;
}

constexpr int kBlock = 128;

// Geodesic right-hand side.  Returns false outside a non-periodic domain.  When lf is
// non-null it receives the most refined level containing the point.
template <class T, int IP = MT_INTERP_CIC>
__device__ __forceinline__ bool geodesic_rhs(const DevField& F, bool grav, const double* y, double* dy, int* lf,
                                             unsigned* err) {
  double H;
  bg_eval(F, y[3], nullptr, &H);
  const double k0 = y[4];
  const double k1 = y[5], k2 = y[6], k3 = y[7];
  T phi = (T)0, g[3] = {(T)0, (T)0, (T)0}, pe = (T)0;
  if (grav) {
    int l;
    if (!sample_field<T, IP>(F, y, y[3], &phi, g, &pe, &l, err)) return false;
    if (lf) *lf = l;
  } else if (lf) {
    double u[3];
    if (!coarse_coords<T>(F, y, u)) return false;
    *lf = locate_level(F, u, err);
  }
  dy[0] = k1;
  dy[1] = k2;
  dy[2] = k3;
  dy[3] = k0;
  const double bgk = -2.0 * H * k0;
  if (sizeof(T) == 8) {
    const double dphidl = (double)g[0] * k1 + (double)g[1] * k2 + (double)g[2] * k3 + (double)pe * k0;
    dy[4] = bgk * k0 - 2.0 * dphidl * k0 + 2.0 * (double)pe * k0 * k0;
    dy[5] = bgk * k1 + 2.0 * dphidl * k1 - 2.0 * (double)g[0] * k0 * k0;
    dy[6] = bgk * k2 + 2.0 * dphidl * k2 - 2.0 * (double)g[1] * k0 * k0;
    dy[7] = bgk * k3 + 2.0 * dphidl * k3 - 2.0 * (double)g[2] * k0 * k0;
    dy[8] = -(double)pe * k0;
    dy[9] = sqrt(k1 * k1 + k2 * k2 + k3 * k3);
  } else {
    const float fk0 = (float)k0, fk1 = (float)k1, fk2 = (float)k2, fk3 = (float)k3;
    const float dphidl = (float)g[0] * fk1 + (float)g[1] * fk2 + (float)g[2] * fk3 + (float)pe * fk0;
    const float k00 = fk0 * fk0;
    dy[4] = bgk * k0 + (double)(-2.0f * dphidl * fk0 + 2.0f * (float)pe * k00);
    dy[5] = bgk * k1 + (double)(2.0f * dphidl * fk1 - 2.0f * (float)g[0] * k00);
    dy[6] = bgk * k2 + (double)(2.0f * dphidl * fk2 - 2.0f * (float)g[1] * k00);
    dy[7] = bgk * k3 + (double)(2.0f * dphidl * fk3 - 2.0f * (float)g[2] * k00);
    dy[8] = (double)(-(float)pe * fk0);
    dy[9] = (double)sqrtf(fk1 * fk1 + fk2 * fk2 + fk3 * fk3);
  }
  return true;
}

struct RayState {
  double y[10];
  double lambda;
  double phi_o;
  double eta_stop;
  double xo[3];
  int n_steps;
  int status;
};

// Initial state of a ray leaving observer xo at eta_o along the unit direction nd (Sect. 2.2):
// k0 = -1 and k^i = n sqrt((1 + 2 phi_o)/(1 - 2 phi_o)) (null condition of Eq. 1).
template <class T>
__device__ __noinline__ RayState ray_start_dir(const DevField& F, const double* xo, double eta_stop, const double* nd,
                                               bool grav, unsigned* err) {
  RayState r;
  r.xo[0] = xo[0];
  r.xo[1] = xo[1];
  r.xo[2] = xo[2];
  r.eta_stop = eta_stop;
  double phi_o = 0.0;
  if (grav) {
    T p, g[3], pe;
    int l;
    if (sample_field<T, kInterpRuntime>(F, r.xo, F.eta_o, &p, g, &pe, &l, err)) phi_o = (double)p;
  }
  const double kn = sqrt((1.0 + 2.0 * phi_o) / (1.0 - 2.0 * phi_o));
  r.y[0] = r.xo[0];
  r.y[1] = r.xo[1];
  r.y[2] = r.xo[2];
  r.y[3] = F.eta_o;
  r.y[4] = -1.0;
  r.y[5] = nd[0] * kn;
  r.y[6] = nd[1] * kn;
  r.y[7] = nd[2] * kn;
  r.y[8] = 0.0;
  r.y[9] = 0.0;
  r.lambda = 0.0;
  r.phi_o = phi_o;
  r.n_steps = 0;
  r.status = MT_RAY_OK;
  return r;
}

// The same along dirs[:, ray] ([3][n], structure of arrays).
template <class T>
__device__ __noinline__ RayState ray_start(const DevField& F, const double* xo, double eta_stop,
                                              const double* __restrict__ dirs, long long n, long long ray, bool grav,
                                              unsigned* err) {
  const double nd[3] = {__ldg(&dirs[ray]), __ldg(&dirs[n + ray]), __ldg(&dirs[2 * n + ray])};
  return ray_start_dir<T>(F, xo, eta_stop, nd, grav, err);
}

// One RK4 step (Sect. 2.2).  Returns true when the ray is finished.
// One RK4 step in FP64 arithmetic with T-precision field records.  Returns true when the ray
// is finished.
template <class T, int IP = MT_INTERP_CIC>
__device__ __forceinline__ bool ray_step_fp64(const DevField& F, const TraceArgs& A, RayState& r, unsigned* err) {
  // a ray that starts on or past its stop surface takes no step; afterwards only the
  // shortened last step ends the ray (a full step that overshoots eta_stop is followed by
  // a short step back onto the surface)
  if (r.n_steps == 0 && !(r.y[3] > r.eta_stop)) return true;
  if (r.n_steps >= A.max_steps) {
    r.status = MT_RAY_MAX_STEPS;
    return true;
  }
  const bool grav = A.gravity_on != 0;
  double k[10], acc[10], t[10];
  int lf = 0;
  if (!geodesic_rhs<T, IP>(F, grav, r.y, k, &lf, err)) {
    r.status = MT_RAY_LEFT_DOMAIN;
    return true;
  }
  const double k0 = r.y[4];
  const double dxl = F.dx0 / (double)(1u << lf);
  double h = dxl / ((double)A.steps_per_cell * fabs(k0));
  bool last = false;
  if (r.y[3] + k0 * h <= r.eta_stop) {
    h = (r.eta_stop - r.y[3]) / k0;
    last = true;
  }
  // classical RK4, y + (h/6) (k1 + 2 k2 + 2 k3 + k4), the weighted sum formed left to right
  const double h2 = 0.5 * h;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    acc[i] = k[i];
    t[i] = r.y[i] + h2 * k[i];
  }
  if (!geodesic_rhs<T, IP>(F, grav, t, k, nullptr, err)) {
    r.status = MT_RAY_LEFT_DOMAIN;
    return true;
  }
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    acc[i] = acc[i] + 2.0 * k[i];
    t[i] = r.y[i] + h2 * k[i];
  }
  if (!geodesic_rhs<T, IP>(F, grav, t, k, nullptr, err)) {
    r.status = MT_RAY_LEFT_DOMAIN;
    return true;
  }
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    acc[i] = acc[i] + 2.0 * k[i];
    t[i] = r.y[i] + h * k[i];
  }
  if (!geodesic_rhs<T, IP>(F, grav, t, k, nullptr, err)) {
    r.status = MT_RAY_LEFT_DOMAIN;
    return true;
  }
  const double h6 = h / 6.0;
  bool finite = true;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    r.y[i] = r.y[i] + h6 * (acc[i] + k[i]);
    finite = finite && isfinite(r.y[i]);
  }
  r.lambda += h;
  r.n_steps += 1;
  if (!finite) {
    r.status = MT_RAY_NONFINITE;
    return true;
  }
  return last;
}

// One RK4 step of the trace kernels: FP64 fields integrate in FP64; FP32 fields use the
// mixed-precision step (mt_mixed.cuh).
template <class T, int IP = MT_INTERP_CIC>
__device__ __forceinline__ bool ray_step(const DevField& F, const TraceArgs& A, RayState& r, unsigned* err,
                                         const LaneCache* lc = nullptr) {
  if constexpr (sizeof(T) == 4) {
    return ray_step_mixed<IP>(F, A, r, err, lc);
  } else {
    return ray_step_fp64<T, IP>(F, A, r, err);
  }
}

template <class T>
__device__ __noinline__ void ray_finish(const DevField& F, const TraceArgs& A, const RayState r, long long ray, long long n,
                           const OutPtrs& O, unsigned* err) {
  const double* y = r.y;
  double a_s;
  bg_eval(F, y[3], &a_s, nullptr);
  double phi_s = 0.0;
  int lev = -1;
  double u[3];
  if (r.status != MT_RAY_NONFINITE && coarse_coords<T>(F, y, u)) lev = locate_level(F, u, err);
  if (A.gravity_on && r.status != MT_RAY_NONFINITE) {
    T p, g[3], pe;
    int l;
    if (sample_field<T, kInterpRuntime>(F, y, y[3], &p, g, &pe, &l, err)) phi_s = (double)p;
  }
  const double dx = y[0] - r.xo[0], dy = y[1] - r.xo[1], dz = y[2] - r.xo[2];
  const double chi = sqrt(dx * dx + dy * dy + dz * dz);
  const double z0 = 1.0 / a_s - 1.0;                                        // Eq. (23)
  const double z1 = z0 + (r.phi_o - phi_s) / a_s;                           // Eq. (24)
  const double z4 = z1 - 2.0 * y[8] / a_s;                                  // Eq. (27), v = 0
  const double z5 = (a_s * fabs(y[4]) * (1.0 + phi_s)) / (1.0 + r.phi_o) - 1.0;  // Eq. (28), v = 0
  if (O.x) {
    O.x[ray] = y[0];
    O.x[n + ray] = y[1];
    O.x[2 * n + ray] = y[2];
  }
  if (O.k) {
    O.k[ray] = y[4];
    O.k[n + ray] = y[5];
    O.k[2 * n + ray] = y[6];
    O.k[3 * n + ray] = y[7];
  }
  if (O.eta) O.eta[ray] = y[3];
  if (O.lambda) O.lambda[ray] = r.lambda;
  if (O.chi) O.chi[ray] = chi;
  if (O.path) O.path[ray] = y[9];
  if (O.z0) O.z0[ray] = z0;
  if (O.z1) O.z1[ray] = z1;
  if (O.z4) O.z4[ray] = z4;
  if (O.z5) O.z5[ray] = z5;
  if (O.d_a) O.d_a[ray] = a_s * chi;
  if (O.d_l) O.d_l[ray] = (1.0 + z5) * (1.0 + z5) * a_s * chi;
  if (O.phi_o) O.phi_o[ray] = r.phi_o;
  if (O.phi_s) O.phi_s[ray] = phi_s;
  if (O.isw) O.isw[ray] = y[8];
  if (O.n_steps) O.n_steps[ray] = r.n_steps;
  if (O.level) O.level[ray] = lev;
  if (O.status) O.status[ray] = r.status;
  if (O.xi) {
    const double de = y[3] - r.eta_stop;
    O.xi[ray] = y[0] - (y[5] / y[4]) * de;
    O.xi[n + ray] = y[1] - (y[6] / y[4]) * de;
    O.xi[2 * n + ray] = y[2] - (y[7] / y[4]) * de;
  }
}

// Screen basis of Sect. 2.3.2 for the direction v (any length): e1 = e_phi = (-sin p, cos p, 0),
// e2 = -e_theta = (-cos p cos t, -sin p cos t, sin t) with p = atan2(v_y, v_x), t = acos(v_z / |v|).
__device__ __forceinline__ void screen_vectors(const double* v, double* e1, double* e2) {
  const double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  const double t1 = atan2(v[1], v[0]);
  const double t2 = acos(fmin(1.0, fmax(-1.0, v[2] / n)));
  double s1, c1, s2, c2;
  sincos(t1, &s1, &c1);
  sincos(t2, &s2, &c2);
  e1[0] = -s1;
  e1[1] = c1;
  e1[2] = 0.0;
  e2[0] = -c1 * c2;
  e2[1] = -s1 * c2;
  e2[2] = s2;
}

// Distortion matrix outputs: jac [4][n] = A11, A12, A21, A22 and lens [5][n] = kappa, gamma1,
// gamma2, omega and 1/mu = det A from the decomposition of Eq. (11),
// A = R(omega) [[1 - kappa - gamma1, -gamma2], [-gamma2, 1 - kappa + gamma1]].
__device__ __forceinline__ void write_distortion(double A11, double A12, double A21, double A22, long long ray,
                                                 long long n, double* jac, double* lens) {
  if (jac) {
    jac[ray] = A11;
    jac[n + ray] = A12;
    jac[2 * n + ray] = A21;
    jac[3 * n + ray] = A22;
  }
  if (lens) {
    const double tr = A11 + A22, an = A21 - A12;
    const double om = atan2(an, tr);
    const double one_k = 0.5 * sqrt(tr * tr + an * an);
    double so, co;
    sincos(om, &so, &co);
    const double S11 = co * A11 + so * A21, S12 = co * A12 + so * A22;
    const double S21 = -so * A11 + co * A21, S22 = -so * A12 + co * A22;
    lens[ray] = 1.0 - one_k;
    lens[n + ray] = 0.5 * (S22 - S11);
    lens[2 * n + ray] = -0.5 * (S12 + S21);
    lens[3 * n + ray] = om;
    lens[4 * n + ray] = A11 * A22 - A12 * A21;
  }
}

// Launches of the FP64-field kernels, defined in the translation units compiled without FMA
// contraction (MT_TU_FP64), so each FP64 operation there is one IEEE-754 operation.
void launch_trace_fp64(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O,
                       const TraceArgs& A, cudaStream_t stream);
void launch_tangent_fp64(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O, double* jac,
                         double* lens, const TraceArgs& A, cudaStream_t stream);
void launch_lensing_fp64(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O, double* jac,
                         double* lens, const TraceArgs& A, cudaStream_t stream);
void launch_beams_fp64(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O, double* jac,
                       double* lens, const TraceArgs& A, double tan_eps, int screen, cudaStream_t stream);

mt_status check_trace_params(const mt_trace_params* p, int64_t n_rays);
void fill_cones(const mt_octree* tree, const mt_trace_params* params, DevCones* C);
cudaError_t launch_tangent(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O, double* jac,
                           double* lens, const TraceArgs& A, cudaStream_t stream);
mt_status run_adjoint_mixed(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O,
                            const double* dL_dxi, double* const* dL_drec, int checkpoint_every, const TraceArgs& A,
                            cudaStream_t stream);
cudaError_t adjoint_checkpoint_layout(const int* d_steps, long long n, int seg_len, long long** d_off, double** d_ck,
                                      cudaStream_t stream);
mt_status run_adjoint(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O,
                      const double* dL_dxi, double* const* dL_drec, int checkpoint_every, const TraceArgs& A,
                      cudaStream_t stream);

}  // namespace mt
