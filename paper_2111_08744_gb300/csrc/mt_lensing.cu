// build: precision-split
// Infinitesimal-beam distortion matrix along the traced rays (Sect. 2.3.1, Eq. 12):
//   A_ab = delta_ab - 2 int_0^chi_s dchi (chi_s - chi) chi / chi_s  d_a d_b phi,
// with the Cartesian Hessian of phi from central differences of the interpolated force (Eq. 13,
// step h = size of the most refined cell containing the photon, d_i d_j taken equal to d_j d_i)
// and its screen components at the photon's angular position seen from the observer
// (Eqs. 14-16, written on the screen basis e_1 = e_phi, e_2 = -e_theta of the finite beams).
// The integral runs over the step points of each ray by the trapezoidal rule, split as
// int chi f - (1/chi_s) int chi^2 f so that chi_s, known at the end, factors out.  With
// gravity off the rays follow FLRW trajectories: the Born approximation.
//
// The rays advance exactly as in mt_trace_rays (same step, same shared-memory neighbourhood
// for FP32 fields); after every step the Hessian is sampled at 6 points around the new position
// in FP64 coordinates.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mt_trace_device.cuh"

namespace mt {
namespace {

constexpr int kLensBlock = 128;

struct InfBeam {
  double I1[3], I2[3];  // int chi f dchi and int chi^2 f dchi for f = (d1d1, d2d2, d1d2) phi
  double prev_chi, prev_f[3];
};

// Screen components of the Hessian at x (Eqs. 13-16).  False when a sample point is outside a
// non-periodic domain.
template <class T, int IP>
__device__ __noinline__ bool screen_hessian(const DevField& F, const double* x, double eta, const double* xo,
                                            double* fo, unsigned* err) {
  double u[3];
  if (!coarse_coords<T>(F, x, u)) return false;
  const int lf = locate_level(F, u, err);
  const double h = F.dx0 / (double)(1ll << lf);
  double H[3][3];
  for (int i = 0; i < 3; ++i) {
    double xp[3] = {x[0], x[1], x[2]}, xm[3] = {x[0], x[1], x[2]};
    xp[i] += h;
    xm[i] -= h;
    T phi, gp[3], gm[3], pe;
    int l;
    if (!sample_field<T, IP>(F, xp, eta, &phi, gp, &pe, &l, err)) return false;
    if (!sample_field<T, IP>(F, xm, eta, &phi, gm, &pe, &l, err)) return false;
    for (int j = i; j < 3; ++j) H[i][j] = ((double)gp[j] - (double)gm[j]) / (2.0 * h);
  }
  const double v[3] = {x[0] - xo[0], x[1] - xo[1], x[2] - xo[2]};
  const double rr = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  double sp, cp, st, ct;
  sincos(atan2(v[1], v[0]), &sp, &cp);
  sincos(acos(fmin(1.0, fmax(-1.0, v[2] / rr))), &st, &ct);
  const double Hxx = H[0][0], Hyy = H[1][1], Hzz = H[2][2], Hxy = H[0][1], Hxz = H[0][2], Hyz = H[1][2];
  fo[0] = sp * sp * Hxx + cp * cp * Hyy - 2.0 * sp * cp * Hxy;
  fo[1] = cp * cp * ct * ct * Hxx + sp * sp * ct * ct * Hyy + st * st * Hzz + 2.0 * sp * cp * ct * ct * Hxy -
          2.0 * sp * st * ct * Hyz - 2.0 * cp * st * ct * Hxz;
  fo[2] = -(ct * cp * sp * (Hyy - Hxx) + (cp * cp - sp * sp) * ct * Hxy + sp * st * Hxz - cp * st * Hyz);
  return true;
}

// Trapezoidal update of the two integrals with the integrand at the ray's new step point.
template <class T, int IP>
__device__ __noinline__ void inf_beam_add(const DevField& F, const RayState& r, InfBeam& ib, unsigned* err) {
  double f[3] = {0.0, 0.0, 0.0};
  const double d[3] = {r.y[0] - r.xo[0], r.y[1] - r.xo[1], r.y[2] - r.xo[2]};
  const double chi = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  if (!screen_hessian<T, IP>(F, r.y, r.y[3], r.xo, f, err)) f[0] = f[1] = f[2] = 0.0;
  const double dchi = chi - ib.prev_chi;
  for (int c = 0; c < 3; ++c) {
    ib.I1[c] += 0.5 * (ib.prev_chi * ib.prev_f[c] + chi * f[c]) * dchi;
    ib.I2[c] += 0.5 * (ib.prev_chi * ib.prev_chi * ib.prev_f[c] + chi * chi * f[c]) * dchi;
    ib.prev_f[c] = f[c];
  }
  ib.prev_chi = chi;
}

__device__ __noinline__ void inf_beam_finish(const InfBeam& ib, long long ray, long long n, double* jac,
                                             double* lens) {
  double m[3];
  for (int c = 0; c < 3; ++c) m[c] = ib.prev_chi > 0.0 ? ib.I1[c] - ib.I2[c] / ib.prev_chi : 0.0;
  write_distortion(1.0 - 2.0 * m[0], -2.0 * m[2], -2.0 * m[2], 1.0 - 2.0 * m[1], ray, n, jac, lens);
}

template <class T, int IP>
__global__ void __launch_bounds__(kLensBlock) lensing_kernel(DevField F, DevCones C, const double* __restrict__ dirs,
                                                             OutPtrs O, double* jac, double* lens, TraceArgs A,
                                                             unsigned long long* ws) {
  unsigned* err = (unsigned*)(ws + 1);
  const unsigned lane = threadIdx.x & 31u;
  const long long n = A.n_rays;
  const bool grav = A.gravity_on != 0;
  extern __shared__ float4 smem[];
  LaneCache lc;
  lc.rec = smem + threadIdx.x;
  lc.key = (int4*)(smem + 16 * kLensBlock) + threadIdx.x;
  lc.stride = kLensBlock;
  lc.loc = (int4*)(smem + 16 * kLensBlock) + kLensBlock + threadIdx.x;
  lc.neg = (int4*)(smem + 16 * kLensBlock) + 2 * kLensBlock + threadIdx.x;
  if (sizeof(T) == 4) {
    *lc.loc = make_int4(0, 0, 0, -1);
    lc.neg[0] = lc.neg[kLensBlock] = make_int4(-1, 0, 0, 0);
  }
  const LaneCache* lcp = sizeof(T) == 4 ? &lc : nullptr;
  RayState r;
  InfBeam ib;
  long long ray = -1;
  bool exhausted = false;
  for (;;) {
    const bool need = (ray < 0) && !exhausted;
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(ws, (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const long long id = (long long)base + __popc(m & ((1u << lane) - 1u));
        if (id < n) {
          ray = id;
          int c = 0;
          while (c + 1 < C.n && C.begin[c + 1] <= ray) ++c;
          r = ray_start<T>(F, C.obs[c], C.eta_stop[c], dirs, n, ray, grav, err);
          for (int q = 0; q < 3; ++q) ib.I1[q] = ib.I2[q] = ib.prev_f[q] = 0.0;
          ib.prev_chi = 0.0;
          if (lcp) *lc.key = make_int4(-1, 0, 0, 0);
        } else {
          exhausted = true;
        }
      }
    }
    const bool alive = ray >= 0;
    if (!__any_sync(0xffffffffu, alive)) break;
    if (alive) {
      const int before = r.n_steps;
      const bool done = ray_step<T, IP>(F, A, r, err, lcp);
      if (r.n_steps > before && r.status == MT_RAY_OK) inf_beam_add<T, IP>(F, r, ib, err);
      if (done) {
        ray_finish<T>(F, A, r, ray, n, O, err);
        inf_beam_finish(ib, ray, n, jac, lens);
        ray = -1;
      }
    }
  }
}

constexpr size_t kLensSmem = (size_t)kLensBlock * (16 * sizeof(float4) + 4 * sizeof(int4));

template <class T, int IP>
void launch_lensing(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O, double* jac,
                    double* lens, const TraceArgs& A, cudaStream_t stream) {
  static int bps = -1;
  const size_t sm = sizeof(T) == 4 ? kLensSmem : 0;
  if (bps < 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, lensing_kernel<T, IP>, kLensBlock, sm) != cudaSuccess ||
        b < 1)
      b = 1;
    bps = b;
  }
  lensing_kernel<T, IP><<<tree->num_sms * bps, kLensBlock, sm, stream>>>(launch_field(tree, A), C, dirs, O, jac,
                                                                          lens, A, tree->ws);
}

template <class T>
void launch_lensing_scheme(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O,
                           double* jac, double* lens, const TraceArgs& A, cudaStream_t stream) {
  switch (A.interp) {
    case MT_INTERP_NGP: launch_lensing<T, MT_INTERP_NGP>(tree, C, dirs, O, jac, lens, A, stream); break;
    case MT_INTERP_TSC: launch_lensing<T, MT_INTERP_TSC>(tree, C, dirs, O, jac, lens, A, stream); break;
    default: launch_lensing<T, MT_INTERP_CIC>(tree, C, dirs, O, jac, lens, A, stream); break;
  }
}

}  // namespace

#ifdef MT_TU_FP64
// FP64-field instantiations (this translation unit is compiled without FMA contraction).
void launch_lensing_fp64(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O, double* jac,
                         double* lens, const TraceArgs& A, cudaStream_t stream) {
  launch_lensing_scheme<double>(tree, C, dirs, O, jac, lens, A, stream);
}
#endif

}  // namespace mt

#ifndef MT_TU_FP64
using namespace mt;

extern "C" mt_status mt_trace_rays_lensing(const mt_octree* tree, const mt_trace_params* params, const double* dirs,
                                           int64_t n_rays, const mt_ray_out* out, double* jac, double* lens,
                                           void* stream_) {
  if (!tree || !out) return MT_ERR_INVALID_ARG;
  mt_status st = check_trace_params(params, n_rays);
  if (st != MT_OK) return st;
  if (!jac && !lens) return MT_ERR_INVALID_ARG;
  if (n_rays > 0 && !dirs) return MT_ERR_INVALID_ARG;
  if (n_rays == 0) return MT_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != tree->device && cudaSetDevice(tree->device) != cudaSuccess) return MT_ERR_CUDA;
  cudaStream_t stream = (cudaStream_t)stream_;
  DevCones C;
  fill_cones(tree, params, &C);
  OutPtrs O = {out->x, out->k, out->eta, out->lambda, out->chi, out->path, out->z0, out->z1, out->z4, out->z5,
               out->d_a, out->d_l, out->phi_o, out->phi_s, out->isw, out->n_steps, out->level, out->status, out->xi};
  TraceArgs A;
  A.steps_per_cell = params->steps_per_cell;
  A.interp = params->interp;
  A.ray_chunk = 32;
  A.gravity_on = params->gravity_on ? 1 : 0;
  A.max_steps = params->max_steps;
  A.n_rays = n_rays;
  cudaError_t e = cudaMemsetAsync(tree->ws, 0, sizeof(unsigned long long), stream);
  if (e == cudaSuccess) {
    if (tree->precision == MT_FIELD_FP64) {
      launch_lensing_fp64(tree, C, dirs, O, jac, lens, A, stream);
    } else {
      launch_lensing_scheme<float>(tree, C, dirs, O, jac, lens, A, stream);
    }
    e = cudaGetLastError();
  }
  if (prev >= 0 && prev != tree->device) cudaSetDevice(prev);
  return e == cudaSuccess ? MT_OK : MT_ERR_CUDA;
}
#endif  // MT_TU_FP64
