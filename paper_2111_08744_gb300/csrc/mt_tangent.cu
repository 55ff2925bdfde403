// build: precision-split
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
template <class T, int IP>
__device__ bool rhs_tangent(const DevField& F, bool grav, const double* y, const double (*dY)[8], double* K,
                            double (*dK)[8], int* lf, unsigned* err) {
  double H, dH;
  bg_eval_d(F, y[3], &H, &dH);
  const double k0 = y[4], k[3] = {y[5], y[6], y[7]};
  FieldD fd = {};
  if (grav) {
    int l;
    if (!sample_field_d<T, IP>(F, y, y[3], &fd, &l, err)) return false;
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
template <class T, int IP>
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
  if (!rhs_tangent<T, IP>(F, grav, r.y, ts.d, K, dK, &lf, err)) {
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
  // stage 1 -> 2 (the state as ray_step_fp64: y + (h/6) (K1 + 2 K2 + 2 K3 + K4), summed left to right)
  for (int i = 0; i < 10; ++i) {
    acc[i] = K[i];
    t[i] = r.y[i] + h2 * K[i];
  }
  for (int b = 0; b < 2; ++b)
    for (int i = 0; i < 8; ++i) {
      dacc[b][i] = ts.d[b][i] + (dh[b] / 6.0) * K[i] + h6 * dK[b][i];
      dt[b][i] = ts.d[b][i] + (0.5 * dh[b]) * K[i] + h2 * dK[b][i];
    }
  if (!rhs_tangent<T, IP>(F, grav, t, dt, K, dK, nullptr, err)) {
    r.status = MT_RAY_LEFT_DOMAIN;
    return true;
  }
  for (int i = 0; i < 10; ++i) {
    acc[i] = acc[i] + 2.0 * K[i];
    t[i] = r.y[i] + h2 * K[i];
  }
  for (int b = 0; b < 2; ++b)
    for (int i = 0; i < 8; ++i) {
      dacc[b][i] += (dh[b] / 3.0) * K[i] + h3 * dK[b][i];
      dt[b][i] = ts.d[b][i] + (0.5 * dh[b]) * K[i] + h2 * dK[b][i];
    }
  if (!rhs_tangent<T, IP>(F, grav, t, dt, K, dK, nullptr, err)) {
    r.status = MT_RAY_LEFT_DOMAIN;
    return true;
  }
  for (int i = 0; i < 10; ++i) {
    acc[i] = acc[i] + 2.0 * K[i];
    t[i] = r.y[i] + h * K[i];
  }
  for (int b = 0; b < 2; ++b)
    for (int i = 0; i < 8; ++i) {
      dacc[b][i] += (dh[b] / 3.0) * K[i] + h3 * dK[b][i];
      dt[b][i] = ts.d[b][i] + dh[b] * K[i] + h * dK[b][i];
    }
  if (!rhs_tangent<T, IP>(F, grav, t, dt, K, dK, nullptr, err)) {
    r.status = MT_RAY_LEFT_DOMAIN;
    return true;
  }
  bool finite = true;
  for (int i = 0; i < 10; ++i) {
    r.y[i] = r.y[i] + h6 * (acc[i] + K[i]);
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

// Mixed-precision form for FP32 fields, arranged as ray_step_mixed: the ray advances exactly as
// in the mixed trace (FP32 stages, FP64 state); the tangents' stage derivatives are FP32 and the
// tangent state FP64.  Stage j of tangent b is dY_b + doff_b with doff_b = c_j (dh K + h dK) of
// the previous stage, and the step adds sum_j b_j (dh K_j + h dK_j), as in tangent_step; the
// parts linear in the step-start state (dh k + h dk for the position-like components) are
// applied in FP64, the stage corrections in FP32.
template <int IP>
__device__ bool tangent_step_mixed(const DevField& F, const TraceArgs& A, RayState& r, TanState& ts, unsigned* err,
                                   const LaneCache* lc) {
  if (r.n_steps == 0 && !(r.y[3] > r.eta_stop)) return true;
  if (r.n_steps >= A.max_steps) {
    r.status = MT_RAY_MAX_STEPS;
    return true;
  }
  const bool grav = A.gravity_on != 0;
  MixedStep B;
  if (!mixed_begin(F, r.y, B)) {
    r.status = MT_RAY_LEFT_DOMAIN;
    return true;
  }
  const double eta = r.y[3];
  const float k0s = (float)r.y[4];
  const float ks[3] = {(float)r.y[5], (float)r.y[6], (float)r.y[7]};
  float dst[2][8];
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int i = 0; i < 8; ++i) dst[b][i] = (float)ts.d[b][i];
  float offx[3] = {0.0f, 0.0f, 0.0f}, offe = 0.0f, offk0 = 0.0f, offk[3] = {0.0f, 0.0f, 0.0f};
  float sx[3] = {0.0f, 0.0f, 0.0f}, se = 0.0f, sk0 = 0.0f, sk[3] = {0.0f, 0.0f, 0.0f}, sI = 0.0f, ss = 0.0f;
  float doff[2][8], sdo[2][4], sdK[2][4];
#pragma unroll
  for (int b = 0; b < 2; ++b) {
#pragma unroll
    for (int i = 0; i < 8; ++i) doff[b][i] = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) sdo[b][i] = sdK[b][i] = 0.0f;
  }
  float h = 0.0f, dh[2] = {0.0f, 0.0f};
  bool last = false;
#pragma unroll 1
  for (int st = 0; st < 4; ++st) {
    const float kst0 = k0s + offk0;
    const float kst[3] = {ks[0] + offk[0], ks[1] + offk[1], ks[2] + offk[2]};
    float Kk0, Kk[3], KI, Ks;
    StageF sf;
    int lf = 0;
    if (!rhs_mixed<true, IP>(F, grav, B, eta, offx, offe, kst0, kst, &Kk0, Kk, &KI, &Ks, st == 0 ? &lf : nullptr, err,
                         lc, &sf)) {
      r.status = MT_RAY_LEFT_DOMAIN;
      return true;
    }
    if (st == 0) {
      const float dxl = F.dx0_f / (float)(1 << lf);
      h = dxl / ((float)A.steps_per_cell * fabsf(k0s));
      const float d = (float)(r.eta_stop - eta);
      if (k0s * h <= d) {
        h = d / k0s;
        last = true;
      }
#pragma unroll
      for (int b = 0; b < 2; ++b) dh[b] = last ? -(dst[b][3] + h * dst[b][4]) / k0s : -h * dst[b][4] / k0s;
    }
    const float bw = (st == 0 || st == 3) ? (1.0f / 6.0f) : (1.0f / 3.0f);
    const float a = st == 2 ? 1.0f : 0.5f;  // next stage at y + a h K, dY + a (dh K + h dK)
    const float c = a * h;
    const float k00 = kst0 * kst0;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      float t[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) t[i] = dst[b][i] + doff[b][i];
      float dg[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) dg[i] = sf.G[i][0] * t[0] + sf.G[i][1] * t[1] + sf.G[i][2] * t[2] + sf.ge[i] * t[3];
      const float dpe = sf.dpe[0] * t[0] + sf.dpe[1] * t[1] + sf.dpe[2] * t[2];
      const float dHb = sf.dH * t[3];
      const float dD = dg[0] * kst[0] + dg[1] * kst[1] + dg[2] * kst[2] + sf.g[0] * t[5] + sf.g[1] * t[6] +
                       sf.g[2] * t[7] + dpe * kst0 + sf.pe * t[4];
      float dK[4];
      dK[0] = -2.0f * dHb * k00 - 4.0f * sf.H * kst0 * t[4] - 2.0f * dD * kst0 - 2.0f * sf.D * t[4] +
              2.0f * dpe * k00 + 4.0f * sf.pe * kst0 * t[4];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        dK[1 + i] = -2.0f * dHb * kst0 * kst[i] - 2.0f * sf.H * t[4] * kst[i] - 2.0f * sf.H * kst0 * t[5 + i] +
                    2.0f * dD * kst[i] + 2.0f * sf.D * t[5 + i] - 2.0f * dg[i] * k00 - 4.0f * sf.g[i] * kst0 * t[4];
      sdo[b][0] += bw * doff[b][5];
      sdo[b][1] += bw * doff[b][6];
      sdo[b][2] += bw * doff[b][7];
      sdo[b][3] += bw * doff[b][4];
#pragma unroll
      for (int i = 0; i < 4; ++i) sdK[b][i] += bw * dK[i];
#pragma unroll
      for (int i = 0; i < 3; ++i) doff[b][i] = a * (dh[b] * kst[i] + h * t[5 + i]);
      doff[b][3] = a * (dh[b] * kst0 + h * t[4]);
      doff[b][4] = a * (dh[b] * Kk0 + h * dK[0]);
#pragma unroll
      for (int i = 0; i < 3; ++i) doff[b][5 + i] = a * (dh[b] * Kk[i] + h * dK[1 + i]);
    }
    sk0 += bw * Kk0;
    sk[0] += bw * Kk[0];
    sk[1] += bw * Kk[1];
    sk[2] += bw * Kk[2];
    sI += bw * KI;
    ss += bw * Ks;
    se += bw * offk0;
    sx[0] += bw * offk[0];
    sx[1] += bw * offk[1];
    sx[2] += bw * offk[2];
    offx[0] = c * kst[0];
    offx[1] = c * kst[1];
    offx[2] = c * kst[2];
    offe = c * kst0;
    offk0 = c * Kk0;
    offk[0] = c * Kk[0];
    offk[1] = c * Kk[1];
    offk[2] = c * Kk[2];
  }
  const double hd = (double)h;
  // tangents first: their position-like parts use the step-start k and dk
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const double dhb = (double)dh[b];
    double* d = ts.d[b];
#pragma unroll
    for (int i = 0; i < 3; ++i) d[i] += dhb * r.y[5 + i] + hd * d[5 + i] + (double)(dh[b] * sx[i] + h * sdo[b][i]);
    d[3] += dhb * r.y[4] + hd * d[4] + (double)(dh[b] * se + h * sdo[b][3]);
    d[4] += (double)(dh[b] * sk0 + h * sdK[b][0]);
#pragma unroll
    for (int i = 0; i < 3; ++i) d[5 + i] += (double)(dh[b] * sk[i] + h * sdK[b][1 + i]);
  }
  bool finite = true;
  r.y[0] += hd * r.y[5] + (double)(h * sx[0]);
  r.y[1] += hd * r.y[6] + (double)(h * sx[1]);
  r.y[2] += hd * r.y[7] + (double)(h * sx[2]);
  r.y[3] += hd * r.y[4] + (double)(h * se);
  r.y[4] += (double)(h * sk0);
  r.y[5] += (double)(h * sk[0]);
  r.y[6] += (double)(h * sk[1]);
  r.y[7] += (double)(h * sk[2]);
  r.y[8] += (double)(h * sI);
  r.y[9] += (double)(h * ss);
#pragma unroll
  for (int i = 0; i < 10; ++i) finite = finite && isfinite(r.y[i]);
  r.lambda += hd;
  r.n_steps += 1;
  if (!finite) {
    r.status = MT_RAY_NONFINITE;
    return true;
  }
  return last;
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
  write_distortion(A11, A12, A21, A22, ray, n, jac, lens);
}

// Initial tangents: the direction perturbed along the observer's screen vectors e_1, e_2.
__device__ __noinline__ void tangent_init_dir(const double* nd, const RayState& r, TanState& ts) {
  double e1[3], e2[3];
  screen_vectors(nd, e1, e2);
  const double kn = sqrt(r.y[5] * r.y[5] + r.y[6] * r.y[6] + r.y[7] * r.y[7]) /
                    sqrt(nd[0] * nd[0] + nd[1] * nd[1] + nd[2] * nd[2]);
  for (int b = 0; b < 2; ++b) {
    const double* e = b == 0 ? e1 : e2;
    for (int i = 0; i < 5; ++i) ts.d[b][i] = 0.0;
    for (int d = 0; d < 3; ++d) ts.d[b][5 + d] = kn * e[d];
  }
}

__device__ __forceinline__ void tangent_init(const double* __restrict__ dirs, long long n, long long ray,
                                             const RayState& r, TanState& ts) {
  const double nd[3] = {__ldg(&dirs[ray]), __ldg(&dirs[n + ray]), __ldg(&dirs[2 * n + ray])};
  tangent_init_dir(nd, r, ts);
}

template <class T, int IP>
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
          tangent_init(dirs, n, ray, r, ts);
        } else {
          exhausted = true;
        }
      }
    }
    const bool alive = ray >= 0;
    if (!__any_sync(0xffffffffu, alive)) break;
    if (alive) {
      if (tangent_step<T, IP>(F, A, r, ts, err)) {
        ray_finish<T>(F, A, r, ray, n, O, err);
        tangent_finish(r, ts, ray, n, jac, lens);
        ray = -1;
      }
    }
  }
}

// Ray ids a warp of the mixed tangent kernel claims at a time (sky neighbours share cache lines,
// as in trace_kernel).
constexpr int kTanChunk = 32;

// FP32 fields: the mixed tangent step, with each ray's CIC neighbourhood staged in shared
// memory as in trace_kernel.
template <int IP>
__global__ void __launch_bounds__(kTanBlock) tangent_kernel_mixed(DevField F, DevCones C,
                                                                  const double* __restrict__ dirs, OutPtrs O,
                                                                  double* jac, double* lens, TraceArgs A,
                                                                  unsigned long long* ws) {
  unsigned* err = (unsigned*)(ws + 1);
  const unsigned lane = threadIdx.x & 31u;
  const long long n = A.n_rays;
  const bool grav = A.gravity_on != 0;
  extern __shared__ float4 smem[];
  LaneCache lc;
  lc.rec = smem + threadIdx.x;
  lc.key = (int4*)(smem + 16 * kTanBlock) + threadIdx.x;
  lc.stride = kTanBlock;
  lc.loc = (int4*)(smem + 16 * kTanBlock) + kTanBlock + threadIdx.x;
  lc.neg = (int4*)(smem + 16 * kTanBlock) + 2 * kTanBlock + threadIdx.x;
  *lc.loc = make_int4(0, 0, 0, -1);
  lc.neg[0] = lc.neg[kTanBlock] = make_int4(-1, 0, 0, 0);
  RayState r;
  TanState ts;
  long long ray = -1;
  bool exhausted = false;
  unsigned long long pool = 0;  // next id of this warp's chunk of kTanChunk consecutive ids (warp-uniform)
  int pool_left = 0;
  for (;;) {
    const bool need = (ray < 0) && !exhausted;
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (m) {
      const int leader = __ffs(m) - 1;
      const int k = __popc(m);
      const int from_pool = k < pool_left ? k : pool_left;
      unsigned long long fresh = 0;
      if (k > from_pool) {
        if ((int)lane == leader) fresh = atomicAdd(ws, (unsigned long long)kTanChunk);
        fresh = __shfl_sync(0xffffffffu, fresh, leader);
      }
      const int rank = __popc(m & ((1u << lane) - 1u));
      const unsigned long long pick = rank < from_pool ? pool + rank : fresh + (rank - from_pool);
      if (k > from_pool) {
        pool = fresh + (k - from_pool);
        pool_left = kTanChunk - (k - from_pool);
      } else {
        pool += k;
        pool_left -= k;
      }
      if (need) {
        const long long id = (long long)pick;
        if (id < n) {
          ray = id;
          int c = 0;
          while (c + 1 < C.n && C.begin[c + 1] <= ray) ++c;
          r = ray_start<float>(F, C.obs[c], C.eta_stop[c], dirs, n, ray, grav, err);
          tangent_init(dirs, n, ray, r, ts);
          *lc.key = make_int4(-1, 0, 0, 0);
        } else {
          exhausted = true;
        }
      }
    }
    const bool alive = ray >= 0;
    if (!__any_sync(0xffffffffu, alive)) break;
    if (alive) {
      if (tangent_step_mixed<IP>(F, A, r, ts, err, &lc)) {
        ray_finish<float>(F, A, r, ray, n, O, err);
        tangent_finish(r, ts, ray, n, jac, lens);
        ray = -1;
      }
    }
  }
}

constexpr size_t kTanMixedSmem = (size_t)kTanBlock * (16 * sizeof(float4) + 4 * sizeof(int4));

template <int IP>
int tangent_mixed_blocks_per_sm() {
  static int cached = -1;
  if (cached < 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tangent_kernel_mixed<IP>, kTanBlock, kTanMixedSmem) !=
            cudaSuccess ||
        b < 1)
      b = 1;
    cached = b;
  }
  return cached;
}

template <int IP>
int tangent_blocks_per_sm() {
  static int cached = -1;
  if (cached < 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tangent_kernel<double, IP>, kTanBlock, 0) != cudaSuccess ||
        b < 1)
      b = 1;
    cached = b;
  }
  return cached;
}

// FP64 field: FP64 tangent step (FP64 translation unit); FP32 field: the mixed tangent step.
template <int IP>
void launch_tangent_scheme(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O,
                           double* jac, double* lens, const TraceArgs& A, cudaStream_t stream) {
#ifdef MT_TU_FP64
  tangent_kernel<double, IP><<<tree->num_sms * tangent_blocks_per_sm<IP>(), kTanBlock, 0, stream>>>(
      launch_field(tree, A), C, dirs, O, jac, lens, A, tree->ws);
#else
  tangent_kernel_mixed<IP><<<tree->num_sms * tangent_mixed_blocks_per_sm<IP>(), kTanBlock, kTanMixedSmem, stream>>>(
      launch_field(tree, A), C, dirs, O, jac, lens, A, tree->ws);
#endif
}

// ----------------------------------------------------------------------------- geodesic finder

// Geodesic finder (Sect. 2.5, Eq. 22): the observed direction theta whose ray, stopped on the sphere
// |x - x_o| = chi_s of the source, is seen from the observer in the source's direction beta.
// Newton on the screen (e_1, e_2) of theta_i:  theta_{i+1} = theta_i - A^{-1} (beta_i - beta), with
// A = d beta / d theta the exact derivative of the discrete map (the forward tangents, projected
// onto the sphere along k) from the first iteration; after max_newton iterations a shrinking 5 x 5
// grid of directions around the best one.  Status: 0 Newton converged, 1 grid converged, 2 not
// converged, 3 the ray failed (left the domain, step cap, or the background table ended first).
}  // namespace

// (outside the unnamed namespace: the FP64 translation unit's launch takes it too)
struct FinderPtrs {
  const double* src;
  double* theta;
  double* jac;
  double* resid;
  int32_t* iters;
  int32_t* status;
};

namespace {

struct SphereHit {
  double xp[3];       // end point on the sphere
  double dxp[2][3];   // its derivatives along the screen of theta
};

// Trace from x_o along th with tangents until |x - x_o| >= chi_s, then move the end point back along
// k onto the sphere: xp = x - t k, t the smaller root of |x - t k - x_o| = chi_s; its tangents
// dxp = dx - t dk - dt k with dt from the constraint (xp - x_o) . dxp = 0.  r ends at (xp, eta - t k0).
template <class T, int IP, bool MIXED>
__device__ bool trace_to_sphere(const DevField& F, const TraceArgs& A, const double* xo, double eta_lo,
                                const double* th, double chi_s, RayState& r, TanState& ts, SphereHit& hit,
                                unsigned* err, const LaneCache* lc) {
  r = ray_start_dir<T>(F, xo, eta_lo, th, A.gravity_on != 0, err);
  tangent_init_dir(th, r, ts);
  if (lc) *lc->key = make_int4(-1, 0, 0, 0);
  for (;;) {
    bool done;
    if constexpr (MIXED) {
      done = tangent_step_mixed<IP>(F, A, r, ts, err, lc);
    } else {
      done = tangent_step<T, IP>(F, A, r, ts, err);
    }
    if (r.status != MT_RAY_OK) return false;
    const double d[3] = {r.y[0] - xo[0], r.y[1] - xo[1], r.y[2] - xo[2]};
    const double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (dd >= chi_s * chi_s) {
      const double* k = r.y + 5;
      const double kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
      const double b = d[0] * k[0] + d[1] * k[1] + d[2] * k[2];
      const double t = (b - sqrt(fmax(0.0, b * b - kk * (dd - chi_s * chi_s)))) / kk;
      for (int q = 0; q < 3; ++q) hit.xp[q] = r.y[q] - t * k[q];
      const double rp[3] = {hit.xp[0] - xo[0], hit.xp[1] - xo[1], hit.xp[2] - xo[2]};
      const double rk = rp[0] * k[0] + rp[1] * k[1] + rp[2] * k[2];
      for (int bb = 0; bb < 2; ++bb) {
        double u[3];
        for (int q = 0; q < 3; ++q) u[q] = ts.d[bb][q] - t * ts.d[bb][5 + q];
        const double dt = (rp[0] * u[0] + rp[1] * u[1] + rp[2] * u[2]) / rk;
        for (int q = 0; q < 3; ++q) hit.dxp[bb][q] = u[q] - dt * k[q];
      }
      for (int q = 0; q < 3; ++q) r.y[q] = hit.xp[q];
      r.y[3] -= t * r.y[4];
      r.eta_stop = r.y[3];
      return true;
    }
    if (done) return false;  // the background table ended before the sphere
  }
}

// beta_i - beta on the screen of th, and its length.
__device__ __forceinline__ double finder_residual(const double* xp, const double* xo, double chi_s, const double* beta,
                                                  const double* e1, const double* e2, double* D) {
  double v[3];
  for (int q = 0; q < 3; ++q) v[q] = (xp[q] - xo[q]) / chi_s - beta[q];
  D[0] = v[0] * e1[0] + v[1] * e1[1] + v[2] * e1[2];
  D[1] = v[0] * e2[0] + v[1] * e2[1] + v[2] * e2[2];
  return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
}

__device__ __forceinline__ void unit_step(const double* th, const double* e1, const double* e2, double a, double b,
                                          double* out) {
  double nn = 0.0;
  for (int q = 0; q < 3; ++q) {
    out[q] = th[q] + a * e1[q] + b * e2[q];
    nn += out[q] * out[q];
  }
  nn = sqrt(nn);
  for (int q = 0; q < 3; ++q) out[q] /= nn;
}

template <class T, int IP, bool MIXED>
__global__ void __launch_bounds__(kTanBlock) finder_kernel(DevField F, DevCones C, OutPtrs O, FinderPtrs P,
                                                           TraceArgs A, double tol, int max_newton, int max_grid,
                                                           unsigned long long* ws) {
  unsigned* err = (unsigned*)(ws + 1);
  const unsigned lane = threadIdx.x & 31u;
  const long long n = A.n_rays;
  extern __shared__ float4 smem[];
  LaneCache lc;
  lc.rec = smem + threadIdx.x;
  lc.key = (int4*)(smem + 16 * kTanBlock) + threadIdx.x;
  lc.stride = kTanBlock;
  lc.loc = (int4*)(smem + 16 * kTanBlock) + kTanBlock + threadIdx.x;
  lc.neg = (int4*)(smem + 16 * kTanBlock) + 2 * kTanBlock + threadIdx.x;
  if (MIXED) {
    *lc.loc = make_int4(0, 0, 0, -1);
    lc.neg[0] = lc.neg[kTanBlock] = make_int4(-1, 0, 0, 0);
  }
  const LaneCache* lcp = MIXED ? &lc : nullptr;
  long long src = -1;
  bool exhausted = false;
  for (;;) {
    const bool need = (src < 0) && !exhausted;
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(ws, (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const long long id = (long long)base + __popc(m & ((1u << lane) - 1u));
        if (id < n) src = id; else exhausted = true;
      }
    }
    if (!__any_sync(0xffffffffu, src >= 0)) break;
    if (src < 0) continue;
    int c = 0;
    while (c + 1 < C.n && C.begin[c + 1] <= src) ++c;
    const double* xo = C.obs[c];
    double beta[3] = {P.src[src] - xo[0], P.src[n + src] - xo[1], P.src[2 * n + src] - xo[2]};
    const double chi_s = sqrt(beta[0] * beta[0] + beta[1] * beta[1] + beta[2] * beta[2]);
    for (int q = 0; q < 3; ++q) beta[q] /= chi_s;
    double th[3] = {beta[0], beta[1], beta[2]};
    RayState r;
    TanState ts;
    SphereHit hit;
    double e1[3], e2[3], D[2];
    double res = 1e300;
    int status = 2, it = 0;
    bool have = false;  // r, ts, hit hold the trace of th
    for (; it < max_newton; ++it) {
      if (!trace_to_sphere<T, IP, MIXED>(F, A, xo, C.eta_stop[c], th, chi_s, r, ts, hit, err, lcp)) {
        status = 3;
        break;
      }
      have = true;
      screen_vectors(th, e1, e2);
      res = finder_residual(hit.xp, xo, chi_s, beta, e1, e2, D);
      if (res < tol) {
        status = 0;
        break;
      }
      // A_ab = e_a . dxp_b / chi_s; theta <- theta - A^{-1} D on the screen of theta
      double a11 = 0, a12 = 0, a21 = 0, a22 = 0;
      for (int q = 0; q < 3; ++q) {
        a11 += e1[q] * hit.dxp[0][q];
        a12 += e1[q] * hit.dxp[1][q];
        a21 += e2[q] * hit.dxp[0][q];
        a22 += e2[q] * hit.dxp[1][q];
      }
      a11 /= chi_s; a12 /= chi_s; a21 /= chi_s; a22 /= chi_s;
      const double det = a11 * a22 - a12 * a21;
      if (!(fabs(det) > 1e-12)) break;  // singular (a caustic): leave it to the grid
      const double d1 = (a22 * D[0] - a12 * D[1]) / det, d2 = (-a21 * D[0] + a11 * D[1]) / det;
      double nt[3];
      unit_step(th, e1, e2, -d1, -d2, nt);
      for (int q = 0; q < 3; ++q) th[q] = nt[q];
      have = false;
    }
    if (status == 2 && it >= max_newton) it = max_newton;
    if (status == 2 && res < 1e299) {
      // shrinking grid around the best direction so far
      if (!have) {
        if (trace_to_sphere<T, IP, MIXED>(F, A, xo, C.eta_stop[c], th, chi_s, r, ts, hit, err, lcp)) {
          screen_vectors(th, e1, e2);
          res = finder_residual(hit.xp, xo, chi_s, beta, e1, e2, D);
        }
      }
      double sp = 2.0 * res;
      for (int g = 0; g < max_grid && status == 2; ++g) {
        screen_vectors(th, e1, e2);
        double best[3] = {th[0], th[1], th[2]};
        double bres = res;
        for (int gi = -2; gi <= 2; ++gi)
          for (int gj = -2; gj <= 2; ++gj) {
            if (gi == 0 && gj == 0) continue;
            double cand[3];
            unit_step(th, e1, e2, gi * sp, gj * sp, cand);
            if (!trace_to_sphere<T, IP, MIXED>(F, A, xo, C.eta_stop[c], cand, chi_s, r, ts, hit, err, lcp)) continue;
            double ce1[3], ce2[3], cD[2];
            screen_vectors(cand, ce1, ce2);
            const double cr = finder_residual(hit.xp, xo, chi_s, beta, ce1, ce2, cD);
            if (cr < bres) {
              bres = cr;
              for (int q = 0; q < 3; ++q) best[q] = cand[q];
            }
          }
        for (int q = 0; q < 3; ++q) th[q] = best[q];
        res = bres;
        sp *= 0.5;
        ++it;
        if (res < tol) status = 1;
      }
      have = false;
    }
    if (status != 3 && !have) {
      if (trace_to_sphere<T, IP, MIXED>(F, A, xo, C.eta_stop[c], th, chi_s, r, ts, hit, err, lcp)) {
        screen_vectors(th, e1, e2);
        res = finder_residual(hit.xp, xo, chi_s, beta, e1, e2, D);
        have = true;
      } else {
        status = 3;
      }
    }
    if (have) {
      ray_finish<T>(F, A, r, src, n, O, err);
      if (P.jac) {
        double a[4] = {0, 0, 0, 0};
        for (int q = 0; q < 3; ++q) {
          a[0] += e1[q] * hit.dxp[0][q];
          a[1] += e1[q] * hit.dxp[1][q];
          a[2] += e2[q] * hit.dxp[0][q];
          a[3] += e2[q] * hit.dxp[1][q];
        }
        for (int q = 0; q < 4; ++q) P.jac[q * n + src] = a[q] / chi_s;
      }
    }
    for (int q = 0; q < 3; ++q) P.theta[q * n + src] = th[q];
    if (P.resid) P.resid[src] = res;
    if (P.iters) P.iters[src] = it + 1;
    P.status[src] = status;
    src = -1;
  }
}

template <class T, int IP, bool MIXED>
void launch_finder_t(const mt_octree* tree, const DevCones& C, const OutPtrs& O, const FinderPtrs& P,
                     const TraceArgs& A, double tol, int max_newton, int max_grid, cudaStream_t stream) {
  static int bps = -1;
  const size_t sm = MIXED ? kTanMixedSmem : 0;
  if (bps < 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, finder_kernel<T, IP, MIXED>, kTanBlock, sm) !=
            cudaSuccess ||
        b < 1)
      b = 1;
    bps = b;
  }
  finder_kernel<T, IP, MIXED><<<tree->num_sms * bps, kTanBlock, sm, stream>>>(launch_field(tree, A), C, O, P, A, tol,
                                                                              max_newton, max_grid, tree->ws);
}

template <int IP>
void launch_finder_scheme(const mt_octree* tree, const DevCones& C, const OutPtrs& O, const FinderPtrs& P,
                          const TraceArgs& A, double tol, int max_newton, int max_grid, cudaStream_t stream) {
#ifdef MT_TU_FP64
  launch_finder_t<double, IP, false>(tree, C, O, P, A, tol, max_newton, max_grid, stream);
#else
  launch_finder_t<float, IP, true>(tree, C, O, P, A, tol, max_newton, max_grid, stream);
#endif
}

}  // namespace

// The tangent and finder kernels of this translation unit's field precision: FP64 fields in the
// unit compiled with MT_TU_FP64 (no FMA contraction), FP32 fields in the other.
#ifdef MT_TU_FP64
void launch_tangent_fp64(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O, double* jac,
                         double* lens, const TraceArgs& A, cudaStream_t stream) {
#else
static void launch_tangent_fp32(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O,
                                double* jac, double* lens, const TraceArgs& A, cudaStream_t stream) {
#endif
  switch (A.interp) {
    case MT_INTERP_NGP: launch_tangent_scheme<MT_INTERP_NGP>(tree, C, dirs, O, jac, lens, A, stream); break;
    case MT_INTERP_TSC: launch_tangent_scheme<MT_INTERP_TSC>(tree, C, dirs, O, jac, lens, A, stream); break;
    default: launch_tangent_scheme<MT_INTERP_CIC>(tree, C, dirs, O, jac, lens, A, stream); break;
  }
}

#ifdef MT_TU_FP64
void launch_finder_fp64(const mt_octree* tree, const DevCones& C, const OutPtrs& O, const FinderPtrs& P,
                        const TraceArgs& A, double tol, int max_newton, int max_grid, cudaStream_t stream) {
#else
static void launch_finder_fp32(const mt_octree* tree, const DevCones& C, const OutPtrs& O, const FinderPtrs& P,
                               const TraceArgs& A, double tol, int max_newton, int max_grid, cudaStream_t stream) {
#endif
  switch (A.interp) {
    case MT_INTERP_NGP: launch_finder_scheme<MT_INTERP_NGP>(tree, C, O, P, A, tol, max_newton, max_grid, stream); break;
    case MT_INTERP_TSC: launch_finder_scheme<MT_INTERP_TSC>(tree, C, O, P, A, tol, max_newton, max_grid, stream); break;
    default: launch_finder_scheme<MT_INTERP_CIC>(tree, C, O, P, A, tol, max_newton, max_grid, stream); break;
  }
}

#ifndef MT_TU_FP64
void launch_finder_fp64(const mt_octree* tree, const DevCones& C, const OutPtrs& O, const FinderPtrs& P,
                        const TraceArgs& A, double tol, int max_newton, int max_grid, cudaStream_t stream);

// Enqueue the tangent kernel (called by mt_trace_rays_adjoint).
cudaError_t launch_tangent(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O, double* jac,
                           double* lens, const TraceArgs& A, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(tree->ws, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  if (tree->precision == MT_FIELD_FP64) {
    launch_tangent_fp64(tree, C, dirs, O, jac, lens, A, stream);
  } else {
    launch_tangent_fp32(tree, C, dirs, O, jac, lens, A, stream);
  }
  return cudaGetLastError();
}

// Enqueue the geodesic finder (called by mt_find_geodesics).
void launch_finder(const mt_octree* tree, const DevCones& C, const OutPtrs& O, const FinderPtrs& P, const TraceArgs& A,
                   double tol, int max_newton, int max_grid, cudaStream_t stream) {
  if (tree->precision == MT_FIELD_FP64) {
    launch_finder_fp64(tree, C, O, P, A, tol, max_newton, max_grid, stream);
  } else {
    launch_finder_fp32(tree, C, O, P, A, tol, max_newton, max_grid, stream);
  }
}
#endif

}  // namespace mt

#ifndef MT_TU_FP64
using namespace mt;

extern "C" mt_status mt_find_geodesics(const mt_octree* tree, const mt_trace_params* params, const double* src,
                                       int64_t n_src, double tol, int32_t max_newton, int32_t max_grid,
                                       const mt_ray_out* out, double* theta, double* jac, double* resid,
                                       int32_t* iters, int32_t* status, void* stream_) {
  if (!tree || !out) return MT_ERR_INVALID_ARG;
  mt_status st = check_trace_params(params, n_src);
  if (st != MT_OK) return st;
  if (!(tol > 0.0) || max_newton < 1 || max_newton > 100 || max_grid < 0 || max_grid > 64) return MT_ERR_INVALID_ARG;
  if (n_src > 0 && (!src || !theta || !status)) return MT_ERR_INVALID_ARG;
  if (n_src == 0) return MT_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != tree->device && cudaSetDevice(tree->device) != cudaSuccess) return MT_ERR_CUDA;
  cudaStream_t stream = (cudaStream_t)stream_;
  DevCones C;
  fill_cones(tree, params, &C);
  for (int c = 0; c < C.n; ++c) C.eta_stop[c] = tree->bg_host[0];  // the sphere stops the rays, not eta
  OutPtrs O = {out->x, out->k, out->eta, out->lambda, out->chi, out->path, out->z0, out->z1, out->z4, out->z5,
               out->d_a, out->d_l, out->phi_o, out->phi_s, out->isw, out->n_steps, out->level, out->status, out->xi};
  TraceArgs A;
  A.steps_per_cell = params->steps_per_cell;
  A.interp = params->interp;
  A.ray_chunk = 32;
  A.gravity_on = params->gravity_on ? 1 : 0;
  A.max_steps = params->max_steps;
  A.n_rays = n_src;
  FinderPtrs P = {src, theta, jac, resid, iters, status};
  cudaError_t e = cudaMemsetAsync(tree->ws, 0, sizeof(unsigned long long), stream);
  if (e == cudaSuccess) {
    launch_finder(tree, C, O, P, A, tol, max_newton, max_grid, stream);
    e = cudaGetLastError();
  }
  if (prev >= 0 && prev != tree->device) cudaSetDevice(prev);
  return e == cudaSuccess ? MT_OK : MT_ERR_CUDA;
}
#endif  // MT_TU_FP64
