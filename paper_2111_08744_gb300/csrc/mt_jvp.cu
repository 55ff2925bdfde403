// build: fp64
// Forward-mode derivative of the rays' end points with respect to the gridded potential records:
// the Jacobian-vector product dxi = J v of the map records -> xi (xi = x - (k/k0)(eta - eta_stop),
// the end point on the iso-eta surface), the forward counterpart of the reverse mode of
// mt_trace_rays_adjoint (which gives J^T w).
//
// Per ray (one thread, FP64 arithmetic, records of the octree's precision) one tangent
// dY = (dx[3], deta, dk0, dk[3]) is carried along the RK4 integration of Eqs. (2)-(4):
//   * start: k = n sqrt((1 + 2 phi_o)/(1 - 2 phi_o)) depends on phi at the observer, so
//     dk = n 2 / (kn (1 - 2 phi_o)^2) dphi_o with dphi_o the interpolated perturbation there;
//   * every stage: the derivative of the right-hand side with respect to the state (the trilinear
//     interpolant's spatial derivatives, the slices' eta dependence, H(eta)) applied to the stage
//     tangent, plus its derivative with respect to (grad phi, phi_eta) applied to the perturbation
//     v interpolated with the same CIC weights, level and slices (Eqs. 8 and the slice rule);
//   * the step size h = dx_l / (N |k0|) and the shortened last step are differentiated;
//   * end: dxi = dx - (dk / k0 - k dk0 / k0^2)(eta - eta_stop) - (k / k0) deta.
// The level and cell decisions of the trajectory are those of the forward trace (the derivative of
// the discrete map where it is differentiable).  CIC only, as the reverse mode.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mt_deriv.cuh"

namespace mt {
namespace {

constexpr int kJvpBlock = 128;

struct RecDir {
  const double* lv[kMaxLevels + 1];  // perturbation [count][S][4] per level (NULL: zero on that level)
};

// The perturbation v interpolated as sample_field interpolates the records at (x, eta): CIC at the
// same level (the most refined level holding all 8 neighbours), the same weights and slices.
// vphi, vg[3], vpe: the interpolated d phi, d grad phi and d phi_eta.
template <class T>
__device__ bool interp_dir(const DevField& F, const RecDir& V, const double* x, double eta, double* vphi, double* vg,
                           double* vpe, unsigned* err) {
  double u[3];
  if (!coarse_coords<T>(F, x, u)) return false;
  const int lfin = locate_level(F, u, err);
  int s = 0;
  while (s < F.S - 2 && F.seta[s + 1] <= eta) ++s;
  const int s1 = F.S > 1 ? s + 1 : s;
  for (int l = lfin; l >= 0; --l) {
    const double sc = (double)(1ll << l);
    long long i0[3];
    double f[3];
    for (int d = 0; d < 3; ++d) {
      const double U = u[d] * sc - 0.5;
      const double fl = floor(U);
      i0[d] = (long long)fl;
      f[d] = U - fl;
    }
    unsigned rows[8];
    if (!cic_rows(F, l, i0, rows, err)) continue;
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const double* base = V.lv[l];
    if (base) {
      for (int c = 0; c < 8; ++c) {
        const double wx = (c & 1) ? f[0] : 1.0 - f[0];
        const double wy = (c & 2) ? f[1] : 1.0 - f[1];
        const double wz = (c & 4) ? f[2] : 1.0 - f[2];
        const double w = wx * wy * wz;
        const double* r0 = base + ((size_t)rows[c] * F.S + s) * 4;
        const double* r1 = base + ((size_t)rows[c] * F.S + s1) * 4;
        for (int q = 0; q < 4; ++q) {
          v[q] += w * r0[q];
          v[4 + q] += w * r1[q];
        }
      }
    }
    if (F.S == 1) {
      *vphi = v[0];
      for (int i = 0; i < 3; ++i) vg[i] = v[1 + i];
      *vpe = 0.0;
    } else {
      const double de = F.seta[s + 1] - F.seta[s];
      const double wt = (eta - F.seta[s]) / de;
      *vphi = v[0] + wt * (v[4] - v[0]);
      for (int i = 0; i < 3; ++i) vg[i] = v[1 + i] + wt * (v[5 + i] - v[1 + i]);
      *vpe = (v[4] - v[0]) / de;
    }
    return true;
  }
  return false;
}

// K = f(y) (as geodesic_rhs) and dK = J(y) dY + (d f / d(g, phi_eta)) (vg, vpe).
template <class T>
__device__ bool rhs_jvp(const DevField& F, const RecDir& V, bool grav, const double* y, const double* t, double* K,
                        double* dK, int* lf, unsigned* err) {
  double H, dH;
  bg_eval_d(F, y[3], &H, &dH);
  const double k0 = y[4], k[3] = {y[5], y[6], y[7]};
  FieldD fd = {};
  double vphi = 0.0, vg[3] = {0.0, 0.0, 0.0}, vpe = 0.0;
  if (grav) {
    int l;
    if (!sample_field_d<T>(F, y, y[3], &fd, &l, err)) return false;
    if (lf) *lf = l;
    if (!interp_dir<T>(F, V, y, y[3], &vphi, vg, &vpe, err)) return false;
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
  double dg[3];
  for (int i = 0; i < 3; ++i)
    dg[i] = fd.G[i][0] * t[0] + fd.G[i][1] * t[1] + fd.G[i][2] * t[2] + fd.ge[i] * t[3] + vg[i];
  const double dpe = fd.dpe[0] * t[0] + fd.dpe[1] * t[1] + fd.dpe[2] * t[2] + vpe;
  const double dHb = dH * t[3];
  const double dk0 = t[4];
  const double dD =
      dg[0] * k[0] + dg[1] * k[1] + dg[2] * k[2] + g[0] * t[5] + g[1] * t[6] + g[2] * t[7] + dpe * k0 + pe * dk0;
  dK[0] = t[5];
  dK[1] = t[6];
  dK[2] = t[7];
  dK[3] = dk0;
  dK[4] = -2.0 * dHb * k0 * k0 - 4.0 * H * k0 * dk0 - 2.0 * dD * k0 - 2.0 * D * dk0 + 2.0 * dpe * k0 * k0 +
          4.0 * pe * k0 * dk0;
  for (int i = 0; i < 3; ++i)
    dK[5 + i] = -2.0 * dHb * k0 * k[i] - 2.0 * H * dk0 * k[i] - 2.0 * H * k0 * t[5 + i] + 2.0 * dD * k[i] +
                2.0 * D * t[5 + i] - 2.0 * dg[i] * k0 * k0 - 4.0 * g[i] * k0 * dk0;
  return true;
}

// One RK4 step of the state (as ray_step_fp64) and its tangent.  Returns true when the ray ends.
template <class T>
__device__ bool jvp_step(const DevField& F, const RecDir& V, const TraceArgs& A, RayState& r, double* dy,
                         unsigned* err) {
  if (r.n_steps == 0 && !(r.y[3] > r.eta_stop)) return true;
  if (r.n_steps >= A.max_steps) {
    r.status = MT_RAY_MAX_STEPS;
    return true;
  }
  const bool grav = A.gravity_on != 0;
  double K[10], acc[10], t[10], dK[8], dacc[8], dt[8];
  int lf = 0;
  if (!rhs_jvp<T>(F, V, grav, r.y, dy, K, dK, &lf, err)) {
    r.status = MT_RAY_LEFT_DOMAIN;
    return true;
  }
  const double k0 = r.y[4];
  const double dxl = F.dx0 / (double)(1u << lf);
  double h = dxl / ((double)A.steps_per_cell * fabs(k0));
  bool last = false;
  double dh;
  if (r.y[3] + k0 * h <= r.eta_stop) {
    h = (r.eta_stop - r.y[3]) / k0;
    last = true;
    dh = -(dy[3] + h * dy[4]) / k0;
  } else {
    dh = -h * dy[4] / k0;
  }
  const double h2 = 0.5 * h;
  // stage weights c_j of the next stage and b_j of the combination
  const double cnext[3] = {h2, h2, h};
  const double dcnext[3] = {0.5 * dh, 0.5 * dh, dh};
  for (int i = 0; i < 10; ++i) acc[i] = K[i];
  for (int i = 0; i < 8; ++i) dacc[i] = (dh / 6.0) * K[i] + (h / 6.0) * dK[i];
  for (int st = 0; st < 3; ++st) {
    for (int i = 0; i < 10; ++i) t[i] = r.y[i] + cnext[st] * K[i];
    for (int i = 0; i < 8; ++i) dt[i] = dy[i] + dcnext[st] * K[i] + cnext[st] * dK[i];
    if (!rhs_jvp<T>(F, V, grav, t, dt, K, dK, nullptr, err)) {
      r.status = MT_RAY_LEFT_DOMAIN;
      return true;
    }
    const double b = st < 2 ? 2.0 : 1.0;  // weights of stages 2, 3 (2/6) and 4 (1/6)
    if (st < 2) {
      for (int i = 0; i < 10; ++i) acc[i] = acc[i] + 2.0 * K[i];
    }
    for (int i = 0; i < 8; ++i) dacc[i] += (b * dh / 6.0) * K[i] + (b * h / 6.0) * dK[i];
  }
  const double h6 = h / 6.0;
  bool finite = true;
  for (int i = 0; i < 10; ++i) {
    r.y[i] = r.y[i] + h6 * (acc[i] + K[i]);
    finite = finite && isfinite(r.y[i]);
  }
  for (int i = 0; i < 8; ++i) dy[i] += dacc[i];
  r.lambda += h;
  r.n_steps += 1;
  if (!finite) {
    r.status = MT_RAY_NONFINITE;
    return true;
  }
  return last;
}

template <class T>
__global__ void __launch_bounds__(kJvpBlock) jvp_kernel(DevField F, DevCones C, const double* __restrict__ dirs,
                                                        OutPtrs O, TraceArgs A, RecDir V, double* dxi,
                                                        unsigned long long* ws) {
  unsigned* err = (unsigned*)(ws + 1);
  const unsigned lane = threadIdx.x & 31u;
  const long long n = A.n_rays;
  const bool grav = A.gravity_on != 0;
  RayState r;
  double dy[8];
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
          for (int i = 0; i < 8; ++i) dy[i] = 0.0;
          if (grav) {
            double vphi = 0.0, vg[3], vpe;
            if (interp_dir<T>(F, V, r.xo, F.eta_o, &vphi, vg, &vpe, err)) {
              const double nd[3] = {__ldg(&dirs[ray]), __ldg(&dirs[n + ray]), __ldg(&dirs[2 * n + ray])};
              const double po = r.phi_o;
              const double kn = sqrt((1.0 + 2.0 * po) / (1.0 - 2.0 * po));
              const double dkn = 2.0 / (kn * (1.0 - 2.0 * po) * (1.0 - 2.0 * po)) * vphi;
              for (int d = 0; d < 3; ++d) dy[5 + d] = nd[d] * dkn;
            }
          }
        } else {
          exhausted = true;
        }
      }
    }
    const bool alive = ray >= 0;
    if (!__any_sync(0xffffffffu, alive)) break;
    if (alive) {
      if (jvp_step<T>(F, V, A, r, dy, err)) {
        ray_finish<T>(F, A, r, ray, n, O, err);
        const double* y = r.y;
        const double k0 = y[4], de = y[3] - r.eta_stop;
        for (int d = 0; d < 3; ++d) {
          double v = 0.0;
          if (r.status == MT_RAY_OK)
            v = dy[d] - (dy[5 + d] / k0 - y[5 + d] * dy[4] / (k0 * k0)) * de - (y[5 + d] / k0) * dy[3];
          dxi[d * n + ray] = v;
        }
        ray = -1;
      }
    }
  }
}

template <class T>
void launch_jvp(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O, const TraceArgs& A,
                const RecDir& V, double* dxi, cudaStream_t stream) {
  static int bps = -1;
  if (bps < 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, jvp_kernel<T>, kJvpBlock, 0) != cudaSuccess || b < 1) b = 1;
    bps = b;
  }
  jvp_kernel<T><<<tree->num_sms * bps, kJvpBlock, 0, stream>>>(launch_field(tree, A), C, dirs, O, A, V, dxi,
                                                              tree->ws);
}

}  // namespace
}  // namespace mt

using namespace mt;

extern "C" mt_status mt_trace_rays_jvp(const mt_octree* tree, const mt_trace_params* params, const double* dirs,
                                       int64_t n_rays, const mt_ray_out* out, const double* const* d_rec,
                                       double* dxi, void* stream_) {
  if (!tree || !out || !d_rec) return MT_ERR_INVALID_ARG;
  mt_status st = check_trace_params(params, n_rays);
  if (st != MT_OK) return st;
  if (params->interp != MT_INTERP_CIC) return MT_ERR_UNSUPPORTED;
  if (n_rays > 0 && (!dirs || !dxi)) return MT_ERR_INVALID_ARG;
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
  RecDir V;
  for (int l = 0; l <= kMaxLevels; ++l) V.lv[l] = (l <= tree->n_levels) ? d_rec[l] : nullptr;
  cudaError_t e = cudaMemsetAsync(tree->ws, 0, sizeof(unsigned long long), stream);
  if (e == cudaSuccess) {
    if (tree->precision == MT_FIELD_FP64) {
      launch_jvp<double>(tree, C, dirs, O, A, V, dxi, stream);
    } else {
      launch_jvp<float>(tree, C, dirs, O, A, V, dxi, stream);
    }
    e = cudaGetLastError();
  }
  if (prev >= 0 && prev != tree->device) cudaSetDevice(prev);
  return e == cudaSuccess ? MT_OK : MT_ERR_CUDA;
}
