// build: precision-split
// Finite-beam distortion matrix (Sect. 2.3.2, Eqs. 17-21) on the GPU.
//
// A beam is a central ray plus four rays at semi-aperture eps around it: directions
// n +- tan(eps) e_1 (rays A, B) and n -+ tan(eps) e_2 (rays C, D), normalised, with (e_1, e_2) the
// screen basis of the central direction.  Every ray stops on the cone's iso-eta surface, and its end
// point is moved along k onto that surface (xi).  With v = xi_central - x_o (beta-screen) or the
// central ray's end wave vector (Sachs screen) and its screen basis (e~_1, e~_2),
//   A_a1 = (xi_A - xi_B) . e~_a / (2 chi tan eps),   A_a2 = (xi_D - xi_C) . e~_a / (2 chi tan eps),
// chi = |xi_central - x_o|; the second column takes xi_D - xi_C so that A is the identity without
// gravity.  Eq. (11) then gives kappa, gamma_1, gamma_2, omega and det A.
//
// One lane owns one beam and integrates its five rays one after the other with the trace step (the
// FP32-field mixed step with its shared-memory neighbourhood, or the FP64 step), so the kernel needs
// no memory beyond its outputs; lanes refill from the beam queue as in trace_kernel.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mt_trace_device.cuh"

namespace mt {
namespace {

constexpr int kBeamBlock = 128;

struct Beam {
  double n[3];       // central direction
  double xi[5][3];   // end points on the iso-eta surface: central, A, B, C, D
  double kend[3];    // central ray's end wave vector (Sachs screen)
  int sub;           // ray of the beam being integrated (0: central, 1..4: A..D)
};

__device__ __forceinline__ void beam_direction(const Beam& b, double tan_eps, int sub, double* d) {
  double e1[3], e2[3];
  screen_vectors(b.n, e1, e2);
  const double* e = sub <= 2 ? e1 : e2;
  const double sg = (sub == 1 || sub == 4) ? 1.0 : -1.0;
  double nn = 0.0;
  for (int q = 0; q < 3; ++q) {
    d[q] = b.n[q] + sg * tan_eps * e[q];
    nn += d[q] * d[q];
  }
  nn = sqrt(nn);
  for (int q = 0; q < 3; ++q) d[q] /= nn;
}

__device__ __noinline__ void beam_finish(const Beam& b, const double* xo, double tan_eps, int screen, long long beam,
                                         long long n, double* jac, double* lens) {
  const double* xr = b.xi[0];
  double v[3];
  for (int q = 0; q < 3; ++q) v[q] = screen == 0 ? xr[q] - xo[q] : b.kend[q];
  double s1[3], s2[3];
  screen_vectors(v, s1, s2);
  const double dx[3] = {xr[0] - xo[0], xr[1] - xo[1], xr[2] - xo[2]};
  const double chi = sqrt(dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]);
  double dAB[3], dDC[3];
  for (int q = 0; q < 3; ++q) {
    dAB[q] = b.xi[1][q] - b.xi[2][q];
    dDC[q] = b.xi[4][q] - b.xi[3][q];
  }
  const double den = 2.0 * chi * tan_eps;
  write_distortion((dAB[0] * s1[0] + dAB[1] * s1[1] + dAB[2] * s1[2]) / den,
                   (dDC[0] * s1[0] + dDC[1] * s1[1] + dDC[2] * s1[2]) / den,
                   (dAB[0] * s2[0] + dAB[1] * s2[1] + dAB[2] * s2[2]) / den,
                   (dDC[0] * s2[0] + dDC[1] * s2[1] + dDC[2] * s2[2]) / den, beam, n, jac, lens);
}

template <class T, int IP>
__global__ void __launch_bounds__(kBeamBlock) beam_kernel(DevField F, DevCones C, const double* __restrict__ dirs,
                                                          OutPtrs O, double* jac, double* lens, TraceArgs A,
                                                          double tan_eps, int screen, unsigned long long* ws) {
  unsigned* err = (unsigned*)(ws + 1);
  const unsigned lane = threadIdx.x & 31u;
  const long long n = A.n_rays;
  const bool grav = A.gravity_on != 0;
  extern __shared__ float4 smem[];
  LaneCache lc;
  lc.rec = smem + threadIdx.x;
  lc.key = (int4*)(smem + 16 * kBeamBlock) + threadIdx.x;
  lc.stride = kBeamBlock;
  lc.loc = (int4*)(smem + 16 * kBeamBlock) + kBeamBlock + threadIdx.x;
  lc.neg = (int4*)(smem + 16 * kBeamBlock) + 2 * kBeamBlock + threadIdx.x;
  if (sizeof(T) == 4) {
    *lc.loc = make_int4(0, 0, 0, -1);
    lc.neg[0] = lc.neg[kBeamBlock] = make_int4(-1, 0, 0, 0);
  }
  const LaneCache* lcp = sizeof(T) == 4 ? &lc : nullptr;
  RayState r;
  Beam b;
  int cone = 0;
  long long beam = -1;
  bool exhausted = false;
  for (;;) {
    const bool need = (beam < 0) && !exhausted;
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(ws, (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const long long id = (long long)base + __popc(m & ((1u << lane) - 1u));
        if (id < n) {
          beam = id;
          cone = 0;
          while (cone + 1 < C.n && C.begin[cone + 1] <= beam) ++cone;
          b.n[0] = __ldg(&dirs[beam]);
          b.n[1] = __ldg(&dirs[n + beam]);
          b.n[2] = __ldg(&dirs[2 * n + beam]);
          b.sub = 0;
          r = ray_start_dir<T>(F, C.obs[cone], C.eta_stop[cone], b.n, grav, err);
          if (lcp) *lc.key = make_int4(-1, 0, 0, 0);
        } else {
          exhausted = true;
        }
      }
    }
    const bool alive = beam >= 0;
    if (!__any_sync(0xffffffffu, alive)) break;
    if (alive) {
      if (ray_step<T, IP>(F, A, r, err, lcp)) {
        const double de = r.y[3] - r.eta_stop;
        for (int q = 0; q < 3; ++q) b.xi[b.sub][q] = r.y[q] - (r.y[5 + q] / r.y[4]) * de;
        if (b.sub == 0) {
          ray_finish<T>(F, A, r, beam, n, O, err);
          b.kend[0] = r.y[5];
          b.kend[1] = r.y[6];
          b.kend[2] = r.y[7];
        }
        if (b.sub == 4) {
          beam_finish(b, C.obs[cone], tan_eps, screen, beam, n, jac, lens);
          beam = -1;
        } else {
          b.sub += 1;
          double d[3];
          beam_direction(b, tan_eps, b.sub, d);
          r = ray_start_dir<T>(F, C.obs[cone], C.eta_stop[cone], d, grav, err);
          if (lcp) *lc.key = make_int4(-1, 0, 0, 0);
        }
      }
    }
  }
}

constexpr size_t kBeamSmem = (size_t)kBeamBlock * (16 * sizeof(float4) + 4 * sizeof(int4));

template <class T, int IP>
void launch_beams(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O, double* jac,
                  double* lens, const TraceArgs& A, double tan_eps, int screen, cudaStream_t stream) {
  static int bps = -1;
  const size_t sm = sizeof(T) == 4 ? kBeamSmem : 0;
  if (bps < 0) {
    int q = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, beam_kernel<T, IP>, kBeamBlock, sm) != cudaSuccess || q < 1)
      q = 1;
    bps = q;
  }
  beam_kernel<T, IP><<<tree->num_sms * bps, kBeamBlock, sm, stream>>>(launch_field(tree, A), C, dirs, O, jac, lens, A,
                                                                       tan_eps, screen, tree->ws);
}

template <class T>
void launch_beams_scheme(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O,
                         double* jac, double* lens, const TraceArgs& A, double tan_eps, int screen,
                         cudaStream_t stream) {
  switch (A.interp) {
    case MT_INTERP_NGP: launch_beams<T, MT_INTERP_NGP>(tree, C, dirs, O, jac, lens, A, tan_eps, screen, stream); break;
    case MT_INTERP_TSC: launch_beams<T, MT_INTERP_TSC>(tree, C, dirs, O, jac, lens, A, tan_eps, screen, stream); break;
    default: launch_beams<T, MT_INTERP_CIC>(tree, C, dirs, O, jac, lens, A, tan_eps, screen, stream); break;
  }
}

}  // namespace

#ifdef MT_TU_FP64
// FP64-field instantiations (this translation unit is compiled without FMA contraction).
void launch_beams_fp64(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O, double* jac,
                       double* lens, const TraceArgs& A, double tan_eps, int screen, cudaStream_t stream) {
  launch_beams_scheme<double>(tree, C, dirs, O, jac, lens, A, tan_eps, screen, stream);
}
#endif

}  // namespace mt

#ifndef MT_TU_FP64
using namespace mt;

extern "C" mt_status mt_trace_beams(const mt_octree* tree, const mt_trace_params* params, const double* dirs,
                                    int64_t n_beams, double eps, int32_t screen, const mt_ray_out* out, double* jac,
                                    double* lens, void* stream_) {
  if (!tree || !out) return MT_ERR_INVALID_ARG;
  mt_status st = check_trace_params(params, n_beams);
  if (st != MT_OK) return st;
  if (!jac && !lens) return MT_ERR_INVALID_ARG;
  if (!(eps > 0.0) || !(eps < 0.5) || (screen != 0 && screen != 1)) return MT_ERR_INVALID_ARG;
  if (n_beams > 0 && !dirs) return MT_ERR_INVALID_ARG;
  if (n_beams == 0) return MT_OK;
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
  A.n_rays = n_beams;
  const double tan_eps = std::tan(eps);
  cudaError_t e = cudaMemsetAsync(tree->ws, 0, sizeof(unsigned long long), stream);
  if (e == cudaSuccess) {
    if (tree->precision == MT_FIELD_FP64) {
      launch_beams_fp64(tree, C, dirs, O, jac, lens, A, tan_eps, screen, stream);
    } else {
      launch_beams_scheme<float>(tree, C, dirs, O, jac, lens, A, tan_eps, screen, stream);
    }
    e = cudaGetLastError();
  }
  if (prev >= 0 && prev != tree->device) cudaSetDevice(prev);
  return e == cudaSuccess ? MT_OK : MT_ERR_CUDA;
}
#endif  // MT_TU_FP64
