// Distortion matrix by forward-mode tangents of the discrete ray map (Sect. 2.3).
//
// For each ray two tangent vectors dY_b = (dx[3], deta, dk0, dk[3]) are carried alongside
// the FP64 RK4 integration of mt_trace_rays: the initial direction is perturbed along the
// screen vectors e_1, e_2 of Sect. 2.3.2 (dk = |k| e_b), every stage applies the exact
// derivative of the right-hand side of Eqs. (2)-(4) -- including the derivative of the
// trilinear (CIC) interpolant of grad phi and of phi_eta, and of H(eta) -- and the step
// size's dependence on the state (h ~ 1/|k0| and the shortened last step) is
// differentiated too.  At the end the end points are moved onto the iso-eta surface,
//   xi = x - (k/k0)(eta - eta_stop),  dxi = dx - (dk/k0 - k dk0/k0^2)(eta - eta_stop) - (k/k0) deta,
// and A_ab = dxi_b . e~_a / chi on the beta-screen e~ of Sect. 2.3.2 (Eq. 21 in the limit of a
// vanishing beam, without neighbouring rays).  The decomposition of Eq. (11) gives
// kappa, gamma_1, gamma_2, omega and 1/mu = det A.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mt_deriv.cuh"

namespace mt {
namespace {

constexpr int kTanBlock = 128;

// Right-hand side K = f(y) (as geodesic_rhs) and its tangents dK_b = J(y) dY_b, b = 0, 1.
// Tangent layout: dx[3], deta, dk0, dk[3].
template <class T>
__device__ bool rhs_tangent(const DevField& F, bool grav, const double* y, const double (*dY)[8], double* K,
                            double (*dK)[8], int* lf, unsigned* err) {
  double H, dH;
  bg_eval_d(F, y[3], &H, &dH);
  const double k0 = y[4], k[3] = {y[5], y[6], y[7]};
  FieldD fd = {};
  if (grav) {
    int l;
    if (!sample_field_d<T>(F, y, y[3], &fd, &l, err)) return false;
    if (lf) *lf = l;
  } else if (lf) {
    double u[3];
    if (!coarse_coords<T>(F, y, u)) return false;
    *lf = locate_level(F, u, err);
  }
  const double* g = fd.g;
  const double pe = fd.pe;
  const double D = g[0] * k[0] + g[1] * k[1] + g[2] * k[2] + pe * k0;
  K[0] = k[0];
  K[1] = k[1];
  K[2] = k[2];
  K[3] = k0;
  const double bgk = -2.0 * H * k0;
  K[4] = bgk * k0 - 2.0 * D * k0 + 2.0 * pe * k0 * k0;
  for (int i = 0; i < 3; ++i) K[5 + i] = bgk * k[i] + 2.0 * D * k[i] - 2.0 * g[i] * k0 * k0;
  K[8] = -pe * k0;
  K[9] = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const double* t = dY[b];
    double dg[3];
    for (int i = 0; i < 3; ++i) dg[i] = fd.G[i][0] * t[0] + fd.G[i][1] * t[1] + fd.G[i][2] * t[2] + fd.ge[i] * t[3];
    const double dpe = fd.dpe[0] * t[0] + fd.dpe[1] * t[1] + fd.dpe[2] * t[2];
    const double dHb = dH * t[3];
    const double dk0 = t[4];
    const double dD = dg[0] * k[0] + dg[1] * k[1] + dg[2] * k[2] + g[0] * t[5] + g[1] * t[6] + g[2] * t[7] +
                      dpe * k0 + pe * dk0;
    dK[b][0] = t[5];
    dK[b][1] = t[6];
    dK[b][2] = t[7];
    dK[b][3] = dk0;
    dK[b][4] = -2.0 * dHb * k0 * k0 - 4.0 * H * k0 * dk0 - 2.0 * dD * k0 - 2.0 * D * dk0 + 2.0 * dpe * k0 * k0 +
               4.0 * pe * k0 * dk0;
    for (int i = 0; i < 3; ++i)
      dK[b][5 + i] = -2.0 * dHb * k0 * k[i] - 2.0 * H * dk0 * k[i] - 2.0 * H * k0 * t[5 + i] + 2.0 * dD * k[i] +
                     2.0 * D * t[5 + i] - 2.0 * dg[i] * k0 * k0 - 4.0 * g[i] * k0 * dk0;
  }
  return true;
}

struct TanState {
  double d[2][8];
};

// One RK4 step of the state and its two tangents.  Returns true when the ray is finished.
template <class T>
__device__ bool tangent_step(const DevField& F, const TraceArgs& A, RayState& r, TanState& ts, unsigned* err) {
  if (r.n_steps == 0 && !(r.y[3] > r.eta_stop)) return true;
  if (r.n_steps >= A.max_steps) {
    r.status = MT_RAY_MAX_STEPS;
    return true;
  }
  const bool grav = A.gravity_on != 0;
  double K[10], acc[10], t[10];
  double dK[2][8], dacc[2][8], dt[2][8];
  int lf = 0;
  if (!rhs_tangent<T>(F, grav, r.y, ts.d, K, dK, &lf, err)) {
    r.status = MT_RAY_LEFT_DOMAIN;
    return true;
  }
  const double k0 = r.y[4];
  const double dxl = F.dx0 / (double)(1u << lf);
  double h = dxl / ((double)A.steps_per_cell * fabs(k0));
  bool last = false;
  double dh[2];
  if (r.y[3] + k0 * h <= r.eta_stop) {
    h = (r.eta_stop - r.y[3]) / k0;
    last = true;
    for (int b = 0; b < 2; ++b) dh[b] = -(ts.d[b][3] + h * ts.d[b][4]) / k0;
  } else {
    for (int b = 0; b < 2; ++b) dh[b] = -h * ts.d[b][4] / k0;
  }
  const double h2 = 0.5 * h, h3 = h / 3.0, h6 = h / 6.0;
  // stage 1 -> 2
  for (int i = 0; i < 10; ++i) {
    acc[i] = r.y[i] + h6 * K[i];
    t[i] = r.y[i] + h2 * K[i];
  }
  for (int b = 0; b < 2; ++b)
    for (int i = 0; i < 8; ++i) {
      dacc[b][i] = ts.d[b][i] + (dh[b] / 6.0) * K[i] + h6 * dK[b][i];
      dt[b][i] = ts.d[b][i] + (0.5 * dh[b]) * K[i] + h2 * dK[b][i];
    }
  if (!rhs_tangent<T>(F, grav, t, dt, K, dK, nullptr, err)) {
    r.status = MT_RAY_LEFT_DOMAIN;
    return true;
  }
  for (int i = 0; i < 10; ++i) {
    acc[i] += h3 * K[i];
    t[i] = r.y[i] + h2 * K[i];
  }
  for (int b = 0; b < 2; ++b)
    for (int i = 0; i < 8; ++i) {
      dacc[b][i] += (dh[b] / 3.0) * K[i] + h3 * dK[b][i];
      dt[b][i] = ts.d[b][i] + (0.5 * dh[b]) * K[i] + h2 * dK[b][i];
    }
  if (!rhs_tangent<T>(F, grav, t, dt, K, dK, nullptr, err)) {
    r.status = MT_RAY_LEFT_DOMAIN;
    return true;
  }
  for (int i = 0; i < 10; ++i) {
    acc[i] += h3 * K[i];
    t[i] = r.y[i] + h * K[i];
  }
  for (int b = 0; b < 2; ++b)
    for (int i = 0; i < 8; ++i) {
      dacc[b][i] += (dh[b] / 3.0) * K[i] + h3 * dK[b][i];
      dt[b][i] = ts.d[b][i] + dh[b] * K[i] + h * dK[b][i];
    }
  if (!rhs_tangent<T>(F, grav, t, dt, K, dK, nullptr, err)) {
    r.status = MT_RAY_LEFT_DOMAIN;
    return true;
  }
  bool finite = true;
  for (int i = 0; i < 10; ++i) {
    r.y[i] = acc[i] + h6 * K[i];
    finite = finite && isfinite(r.y[i]);
  }
  for (int b = 0; b < 2; ++b)
    for (int i = 0; i < 8; ++i) ts.d[b][i] = dacc[b][i] + (dh[b] / 6.0) * K[i] + h6 * dK[b][i];
  r.lambda += h;
  r.n_steps += 1;
  if (!finite) {
    r.status = MT_RAY_NONFINITE;
    return true;
  }
  return last;
}

__device__ void screen_vectors(const double* v, double* e1, double* e2) {
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

__device__ __noinline__ void tangent_finish(const RayState r, const TanState ts, long long ray, long long n,
                                            double* jac, double* lens) {
  const double* y = r.y;
  const double k0 = y[4];
  const double de = y[3] - r.eta_stop;
  double xi[3], dxi[2][3];
  for (int d = 0; d < 3; ++d) xi[d] = y[d] - (y[5 + d] / k0) * de;
  for (int b = 0; b < 2; ++b)
    for (int d = 0; d < 3; ++d)
      dxi[b][d] = ts.d[b][d] - (ts.d[b][5 + d] / k0 - y[5 + d] * ts.d[b][4] / (k0 * k0)) * de -
                  (y[5 + d] / k0) * ts.d[b][3];
  const double v[3] = {xi[0] - r.xo[0], xi[1] - r.xo[1], xi[2] - r.xo[2]};
  const double chi = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  double s1[3], s2[3];
  screen_vectors(v, s1, s2);
  const double A11 = (dxi[0][0] * s1[0] + dxi[0][1] * s1[1] + dxi[0][2] * s1[2]) / chi;
  const double A12 = (dxi[1][0] * s1[0] + dxi[1][1] * s1[1] + dxi[1][2] * s1[2]) / chi;
  const double A21 = (dxi[0][0] * s2[0] + dxi[0][1] * s2[1] + dxi[0][2] * s2[2]) / chi;
  const double A22 = (dxi[1][0] * s2[0] + dxi[1][1] * s2[1] + dxi[1][2] * s2[2]) / chi;
  if (jac) {
    jac[ray] = A11;
    jac[n + ray] = A12;
    jac[2 * n + ray] = A21;
    jac[3 * n + ray] = A22;
  }
  if (lens) {
    // Eq. (11): A = R(omega) [[1 - kappa - gamma1, -gamma2], [-gamma2, 1 - kappa + gamma1]]
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

template <class T>
__global__ void __launch_bounds__(kTanBlock) tangent_kernel(DevField F, DevCones C, const double* __restrict__ dirs,
                                                            OutPtrs O, double* jac, double* lens, TraceArgs A,
                                                            unsigned long long* ws) {
  unsigned* err = (unsigned*)(ws + 1);
  const unsigned lane = threadIdx.x & 31u;
  const long long n = A.n_rays;
  const bool grav = A.gravity_on != 0;
  RayState r;
  TanState ts;
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
          // initial tangents: direction perturbed along the observer's screen vectors e_1, e_2
          const double nd[3] = {__ldg(&dirs[ray]), __ldg(&dirs[n + ray]), __ldg(&dirs[2 * n + ray])};
          double e1[3], e2[3];
          screen_vectors(nd, e1, e2);
          const double kn = sqrt(r.y[5] * r.y[5] + r.y[6] * r.y[6] + r.y[7] * r.y[7]) /
                            sqrt(nd[0] * nd[0] + nd[1] * nd[1] + nd[2] * nd[2]);
          for (int b = 0; b < 2; ++b) {
            const double* e = b == 0 ? e1 : e2;
            for (int i = 0; i < 5; ++i) ts.d[b][i] = 0.0;
            for (int d = 0; d < 3; ++d) ts.d[b][5 + d] = kn * e[d];
          }
        } else {
          exhausted = true;
        }
      }
    }
    const bool alive = ray >= 0;
    if (!__any_sync(0xffffffffu, alive)) break;
    if (alive) {
      if (tangent_step<T>(F, A, r, ts, err)) {
        ray_finish<T>(F, A, r, ray, n, O, err);
        tangent_finish(r, ts, ray, n, jac, lens);
        ray = -1;
      }
    }
  }
}

template <class T>
int tangent_blocks_per_sm() {
  static int cached = -1;
  if (cached < 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tangent_kernel<T>, kTanBlock, 0) != cudaSuccess || b < 1)
      b = 1;
    cached = b;
  }
  return cached;
}

}  // namespace

// Enqueue the tangent kernel (called by mt_trace_rays_adjoint).
cudaError_t launch_tangent(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O, double* jac,
                           double* lens, const TraceArgs& A, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(tree->ws, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  if (tree->precision == MT_FIELD_FP64) {
    tangent_kernel<double><<<tree->num_sms * tangent_blocks_per_sm<double>(), kTanBlock, 0, stream>>>(
        tree->f, C, dirs, O, jac, lens, A, tree->ws);
  } else {
    tangent_kernel<float><<<tree->num_sms * tangent_blocks_per_sm<float>(), kTanBlock, 0, stream>>>(
        tree->f, C, dirs, O, jac, lens, A, tree->ws);
  }
  return cudaGetLastError();
}

}  // namespace mt
