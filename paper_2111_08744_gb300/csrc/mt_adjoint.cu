// build: fp64
// Reverse mode: gradient of a loss on the rays' end points with respect to the gridded
// potential records (every level, slice and component), by the exact adjoint of the
// discrete ray map (RK4 of Eqs. 2-4 with CIC interpolation and level fallback, Sect. 2.2).
//
// FP64 octrees (FP32 octrees: mt_adjoint_mixed.cu, the adjoint of the mixed-precision step).
// Per ray (one thread):
//   1. integrate forward (FP64 arithmetic), keeping the state every
//      `checkpoint_every` steps in a global checkpoint buffer;
//   2. from the cotangent dL/dxi of the end point on the iso-eta surface,
//      xi = x - (k/k0)(eta - eta_stop), form the cotangent of the final state;
//   3. for each segment, last to first (a warp's 32 rays in lockstep, aligned on their last
//      segments): recompute its steps from the checkpoint into a per-thread buffer, then run each
//      step backward: recompute the 4 RK4 stages, and apply
//      the transposed stage Jacobians (including the dependence of the step size on the state
//      and of the shortened last step), scattering the cotangents of grad phi and phi_eta at
//      every stage onto the 8 CIC records of both bracketing slices with FP64 atomics;
//   4. propagate the cotangent of the initial wave vector to phi at the observer.
// Rays that did not reach their stop surface (status != MT_RAY_OK) contribute nothing.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <vector>

#include "mt_deriv.cuh"

namespace mt {
namespace {

constexpr int kAdjBlock = 64;
constexpr int kMaxSegment = 64;

struct RecBar {
  double* lv[kMaxLevels + 1];  // [count][S][4] cotangent buffers per level (NULL: skip the level)
};

// Per-lane accumulator of record cotangents in shared memory: the 8 CIC records of both
// bracketing slices of the last neighbourhood a stage scattered to (acc[(8 c + 4 slice + q) *
// stride]), their rows and key (level << 8 | slice, i0).  Consecutive stages of a ray mostly land
// in the same neighbourhood, so the FP64 atomics into the record gradients are issued only when it
// changes (and at the end of the ray) instead of at every stage.
struct ScatterCache {
  double* acc;
  unsigned* rows;
  int4* key;   // x = -1: empty
  int stride;
};

// Add the accumulated cotangents into the record gradients and empty the accumulator.
__device__ __noinline__ void scatter_flush(const DevField& F, const RecBar& R, const ScatterCache& sc) {
  const int4 k = *sc.key;
  if (k.x < 0) return;
  const int l = k.x >> 8, s = k.x & 255;
  double* base = R.lv[l];
  const int ns = F.S > 1 ? 2 : 1;
  for (int c = 0; c < 8; ++c) {
    const unsigned row = sc.rows[c * sc.stride];
    for (int sl = 0; sl < ns; ++sl) {
      double* r = base + ((size_t)row * F.S + s + sl) * 4;
      for (int q = 0; q < 4; ++q) {
        double* a = sc.acc + (8 * c + 4 * sl + q) * sc.stride;
        if (*a != 0.0) atomicAdd(r + q, *a);
        *a = 0.0;
      }
    }
  }
  *sc.key = make_int4(-1, 0, 0, 0);
}

// Scatter cotangents of (grad phi, phi_eta, phi) at (x, eta) onto the CIC records used there
// (through the lane's accumulator when sc is non-null).
template <class T>
__device__ void scatter_cotangent(const DevField& F, const double* x, double eta, const double* gbar, double pebar,
                                  double phibar, const RecBar& R, unsigned* err, const ScatterCache* cache = nullptr) {
  double u[3];
  if (!coarse_coords<T>(F, x, u)) return;
  const int lfin = locate_level(F, u, err);
  int s = 0;
  while (s < F.S - 2 && F.seta[s + 1] <= eta) ++s;
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
    const int4 key = make_int4((l << 8) | s, (int)i0[0], (int)i0[1], (int)i0[2]);
    const bool hit = cache && cache->key->x == key.x && cache->key->y == key.y && cache->key->z == key.z &&
                     cache->key->w == key.w;
    unsigned rows[8];
    if (!hit && !cic_rows(F, l, i0, rows, err)) continue;
    double* base = R.lv[l];
    if (!base) return;
    if (cache && !hit) {
      scatter_flush(F, R, *cache);
      for (int c = 0; c < 8; ++c) cache->rows[c * cache->stride] = rows[c];
      *cache->key = key;
    }
    double a0[4], a1[4];  // per-slice cotangent of (phi, g0, g1, g2) before the CIC weight
    if (F.S == 1) {
      a0[0] = phibar;
      for (int i = 0; i < 3; ++i) a0[1 + i] = gbar[i];
    } else {
      const double de = F.seta[s + 1] - F.seta[s];
      const double wt = (eta - F.seta[s]) / de;
      a0[0] = (1.0 - wt) * phibar - pebar / de;
      a1[0] = wt * phibar + pebar / de;
      for (int i = 0; i < 3; ++i) {
        a0[1 + i] = (1.0 - wt) * gbar[i];
        a1[1 + i] = wt * gbar[i];
      }
    }
    for (int c = 0; c < 8; ++c) {
      const double wx = (c & 1) ? f[0] : 1.0 - f[0];
      const double wy = (c & 2) ? f[1] : 1.0 - f[1];
      const double wz = (c & 4) ? f[2] : 1.0 - f[2];
      const double w = wx * wy * wz;
      if (w == 0.0) continue;
      if (cache) {
        for (int q = 0; q < 4; ++q) cache->acc[(8 * c + q) * cache->stride] += w * a0[q];
        if (F.S > 1)
          for (int q = 0; q < 4; ++q) cache->acc[(8 * c + 4 + q) * cache->stride] += w * a1[q];
        continue;
      }
      double* r0 = base + ((size_t)rows[c] * F.S + s) * 4;
      for (int q = 0; q < 4; ++q)
        if (a0[q] != 0.0) atomicAdd(r0 + q, w * a0[q]);
      if (F.S > 1) {
        double* r1 = r0 + 4;
        for (int q = 0; q < 4; ++q)
          if (a1[q] != 0.0) atomicAdd(r1 + q, w * a1[q]);
      }
    }
    return;
  }
}

// Transposed stage Jacobian: ybar += J(y)^T w (8 components: x[3], eta, k0, k[3]); scatters the
// cotangents of the interpolated field at y onto the records.
template <class T>
__device__ bool stage_adjoint(const DevField& F, bool grav, const double* y, const double* w, double* ybar,
                              const RecBar& R, unsigned* err, const ScatterCache* sc) {
  double H, dH;
  bg_eval_d(F, y[3], &H, &dH);
  const double k0 = y[4], k[3] = {y[5], y[6], y[7]};
  FieldD fd = {};
  if (grav) {
    int l;
    if (!sample_field_d<T>(F, y, y[3], &fd, &l, err)) return false;
  }
  const double* g = fd.g;
  const double pe = fd.pe;
  const double D = g[0] * k[0] + g[1] * k[1] + g[2] * k[2] + pe * k0;
  const double wk0 = w[4];
  const double* wk = w + 5;
  // outputs x and eta are k and k0
  double tb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  tb[5] += w[0];
  tb[6] += w[1];
  tb[7] += w[2];
  tb[4] += w[3];
  double dHbar = -2.0 * k0 * k0 * wk0;
  tb[4] += (-4.0 * H * k0 - 2.0 * D + 4.0 * pe * k0) * wk0;
  double dDbar = -2.0 * k0 * wk0;
  double dpebar = 2.0 * k0 * k0 * wk0;
  double dgbar[3];
  for (int j = 0; j < 3; ++j) {
    dHbar += -2.0 * k0 * k[j] * wk[j];
    tb[4] += (-2.0 * H * k[j] - 4.0 * g[j] * k0) * wk[j];
    tb[5 + j] += (-2.0 * H * k0 + 2.0 * D) * wk[j];
    dDbar += 2.0 * k[j] * wk[j];
    dgbar[j] = -2.0 * k0 * k0 * wk[j];
  }
  for (int i = 0; i < 3; ++i) {
    dgbar[i] += k[i] * dDbar;
    tb[5 + i] += g[i] * dDbar;
  }
  dpebar += k0 * dDbar;
  tb[4] += pe * dDbar;
  tb[3] += dH * dHbar;
  for (int d = 0; d < 3; ++d) {
    tb[d] += fd.dpe[d] * dpebar;
    for (int i = 0; i < 3; ++i) tb[d] += fd.G[i][d] * dgbar[i];
  }
  for (int i = 0; i < 3; ++i) tb[3] += fd.ge[i] * dgbar[i];
  for (int i = 0; i < 8; ++i) ybar[i] += tb[i];
  if (grav) scatter_cotangent<T>(F, y, y[3], dgbar, dpebar, 0.0, R, err, sc);
  return true;
}

// Step size of the step starting at y (as ray_step_fp64): returns h, sets *last.
template <class T>
__device__ bool step_size(const DevField& F, const TraceArgs& A, const double* y, double eta_stop, bool force_last,
                          double* K1, double* h_out, unsigned* err) {
  int lf = 0;
  if (!geodesic_rhs<T>(F, A.gravity_on != 0, y, K1, &lf, err)) return false;
  const double k0 = y[4];
  const double dxl = F.dx0 / (double)(1u << lf);
  double h = dxl / ((double)A.steps_per_cell * fabs(k0));
  if (force_last) h = (eta_stop - y[3]) / k0;
  *h_out = h;
  return true;
}

// Reverse of one FP64 step from the step-start state y (x[3], eta, k0, k[3]): yb holds the cotangent
// of the step's end state on entry and of its start state on return; last: the ray's final
// (shortened) step.  False if a stage left a non-periodic domain.
template <class T>
__device__ bool reverse_step_fp64(const DevField& F, const TraceArgs& A, bool grav, const double* y, bool last,
                                  double eta_stop, double* yb, const RecBar& R, unsigned* err, const ScatterCache* sc) {
  double y10[10];
  for (int i = 0; i < 8; ++i) y10[i] = y[i];
  y10[8] = y10[9] = 0.0;
  double K1[10], K2[10], K3[10], K4[10], Y2[10], Y3[10], Y4[10], h;
  if (!step_size<T>(F, A, y10, eta_stop, last, K1, &h, err)) return false;
  const double h2 = 0.5 * h;
  for (int i = 0; i < 10; ++i) Y2[i] = y10[i] + h2 * K1[i];
  geodesic_rhs<T>(F, grav, Y2, K2, nullptr, err);
  for (int i = 0; i < 10; ++i) Y3[i] = y10[i] + h2 * K2[i];
  geodesic_rhs<T>(F, grav, Y3, K3, nullptr, err);
  for (int i = 0; i < 10; ++i) Y4[i] = y10[i] + h * K3[i];
  geodesic_rhs<T>(F, grav, Y4, K4, nullptr, err);
  // reverse of y' = y + h/6 (K1 + 2 K2 + 2 K3 + K4)
  double hbar = 0.0, kb1[8], kb2[8], kb3[8], kb4[8], nyb[8];
  for (int i = 0; i < 8; ++i) {
    hbar += yb[i] * (K1[i] + 2.0 * K2[i] + 2.0 * K3[i] + K4[i]) / 6.0;
    kb1[i] = yb[i] * (h / 6.0);
    kb2[i] = yb[i] * (h / 3.0);
    kb3[i] = yb[i] * (h / 3.0);
    kb4[i] = yb[i] * (h / 6.0);
    nyb[i] = yb[i];
  }
  double Yb[8];
  // stage 4 at Y4 = y + h K3
  for (int i = 0; i < 8; ++i) Yb[i] = 0.0;
  stage_adjoint<T>(F, grav, Y4, kb4, Yb, R, err, sc);
  for (int i = 0; i < 8; ++i) {
    nyb[i] += Yb[i];
    kb3[i] += h * Yb[i];
    hbar += Yb[i] * K3[i];
  }
  // stage 3 at Y3 = y + h/2 K2
  for (int i = 0; i < 8; ++i) Yb[i] = 0.0;
  stage_adjoint<T>(F, grav, Y3, kb3, Yb, R, err, sc);
  for (int i = 0; i < 8; ++i) {
    nyb[i] += Yb[i];
    kb2[i] += h2 * Yb[i];
    hbar += 0.5 * Yb[i] * K2[i];
  }
  // stage 2 at Y2 = y + h/2 K1
  for (int i = 0; i < 8; ++i) Yb[i] = 0.0;
  stage_adjoint<T>(F, grav, Y2, kb2, Yb, R, err, sc);
  for (int i = 0; i < 8; ++i) {
    nyb[i] += Yb[i];
    kb1[i] += h2 * Yb[i];
    hbar += 0.5 * Yb[i] * K1[i];
  }
  // stage 1 at y
  for (int i = 0; i < 8; ++i) Yb[i] = 0.0;
  stage_adjoint<T>(F, grav, y10, kb1, Yb, R, err, sc);
  for (int i = 0; i < 8; ++i) nyb[i] += Yb[i];
  // step size: h = dx_l / (N |k0|), or (eta_stop - eta) / k0 on the last step
  const double k0 = y[4];
  if (last) nyb[3] += -hbar / k0;
  nyb[4] += -hbar * h / k0;
  for (int i = 0; i < 8; ++i) yb[i] = nyb[i];
  return true;
}

// Warp-synchronous sweep (as the mixed-precision one): a warp takes 32 consecutive rays per turn,
// integrates them forward together, then reverses them segment by segment aligned on each ray's last
// segment, with warp-uniform loop bounds.
template <class T>
__global__ void __launch_bounds__(kAdjBlock) adjoint_kernel(DevField F, DevCones C, const double* __restrict__ dirs,
                                                            OutPtrs O, TraceArgs A, const double* __restrict__ dL_dxi,
                                                            RecBar R, double* ckpt, const long long* ck_off,
                                                            int seg_len, unsigned long long* ws) {
  unsigned* err = (unsigned*)(ws + 1);
  const unsigned lane = threadIdx.x & 31u;
  const long long n = A.n_rays;
  const bool grav = A.gravity_on != 0;
  double ys[kMaxSegment][8];
  extern __shared__ double adj_smem[];
  ScatterCache sc;
  sc.stride = kAdjBlock;
  sc.acc = adj_smem + threadIdx.x;
  sc.rows = (unsigned*)(adj_smem + 64 * kAdjBlock) + threadIdx.x;
  sc.key = (int4*)((unsigned*)(adj_smem + 64 * kAdjBlock) + 8 * kAdjBlock) + threadIdx.x;
  for (int j = 0; j < 64; ++j) sc.acc[j * sc.stride] = 0.0;
  *sc.key = make_int4(-1, 0, 0, 0);
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(ws, 32ull);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= (unsigned long long)n) break;
    const long long ray = (long long)base + lane;
    const bool have = ray < n;
    RayState r;
    long long off = 0, n_ck = 0;
    bool ok = have;
    double k_init_scale = 0.0;
    if (have) {
      int c = 0;
      while (c + 1 < C.n && C.begin[c + 1] <= ray) ++c;
      r = ray_start<T>(F, C.obs[c], C.eta_stop[c], dirs, n, ray, grav, err);
      k_init_scale = sqrt(r.y[5] * r.y[5] + r.y[6] * r.y[6] + r.y[7] * r.y[7]);
      off = ck_off[ray];
      n_ck = ck_off[ray + 1] - off;
    }
    // 1. forward with checkpoints, the warp's rays in lockstep
    bool fwd = have;
    while (__any_sync(0xffffffffu, fwd)) {
      if (fwd) {
        if (r.n_steps % seg_len == 0) {
          const long long j = r.n_steps / seg_len;
          if (j >= n_ck) {
            atomicOr(err, kErrOOB);  // more steps than the first pass counted
            ok = false;
            fwd = false;
          } else {
            double* cp = ckpt + (off + j) * 8;
            for (int i = 0; i < 8; ++i) cp[i] = r.y[i];
          }
        }
        if (fwd && ray_step_fp64<T>(F, A, r, err)) fwd = false;
      }
    }
    if (have) ray_finish<T>(F, A, r, ray, n, O, err);
    const bool active = ok && have && r.status == MT_RAY_OK && r.n_steps > 0;
    const int n_steps = active ? r.n_steps : 0;
    const int n_seg = (n_steps + seg_len - 1) / seg_len;
    const int max_seg = (int)__reduce_max_sync(0xffffffffu, (unsigned)n_seg);
    // 2. cotangent of the end state from dL/dxi
    double yb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (active) {
      const double* y = r.y;
      const double k0 = y[4], de = y[3] - r.eta_stop;
      const double xb[3] = {dL_dxi[ray], dL_dxi[n + ray], dL_dxi[2 * n + ray]};
      const double xk = xb[0] * y[5] + xb[1] * y[6] + xb[2] * y[7];
      for (int d = 0; d < 3; ++d) {
        yb[d] = xb[d];
        yb[5 + d] = -xb[d] * de / k0;
      }
      yb[3] = -xk / k0;
      yb[4] = xk * de / (k0 * k0);
    }
    // 3. segments from the last, aligned on each ray's last segment
    bool alive = active;
    for (int j = max_seg - 1; j >= 0; --j) {
      const int sgi = j - (max_seg - n_seg);
      const bool on = alive && sgi >= 0;
      const int s0 = on ? sgi * seg_len : 0;
      const int len = on ? min(n_steps, s0 + seg_len) - s0 : 0;
      RayState q = r;
      if (on) {
        const double* cp = ckpt + (off + sgi) * 8;
        for (int i = 0; i < 8; ++i) q.y[i] = cp[i];
        q.n_steps = s0;
      }
      for (int st = 0; st < seg_len; ++st) {
        if (st < len) {
          for (int i = 0; i < 8; ++i) ys[st][i] = q.y[i];
          if (st + 1 < len) ray_step_fp64<T>(F, A, q, err);
        }
      }
      for (int st = seg_len - 1; st >= 0; --st) {
        if (st < len && alive) {
          if (!reverse_step_fp64<T>(F, A, grav, ys[st], s0 + st == n_steps - 1, r.eta_stop, yb, R, err, &sc))
            alive = false;
        }
      }
    }
    // 4. initial wave vector k = n sqrt((1 + 2 phi_o)/(1 - 2 phi_o)) depends on phi_o
    if (alive && grav) {
      const double nd[3] = {__ldg(&dirs[ray]), __ldg(&dirs[n + ray]), __ldg(&dirs[2 * n + ray])};
      const double po = r.phi_o;
      const double dkn = 2.0 / (k_init_scale / sqrt(nd[0] * nd[0] + nd[1] * nd[1] + nd[2] * nd[2]) *
                                (1.0 - 2.0 * po) * (1.0 - 2.0 * po));
      const double phib = (yb[5] * nd[0] + yb[6] * nd[1] + yb[7] * nd[2]) * dkn;
      const double zero[3] = {0.0, 0.0, 0.0};
      scatter_cotangent<T>(F, r.xo, F.eta_o, zero, 0.0, phib, R, err, &sc);
    }
    scatter_flush(F, R, sc);
  }
}

template <class T>
__global__ void __launch_bounds__(128) count_steps_kernel(DevField F, DevCones C, const double* __restrict__ dirs,
                                                          TraceArgs A, int* n_steps, unsigned long long* ws) {
  unsigned* err = (unsigned*)(ws + 1);
  const long long n = A.n_rays;
  for (long long ray = blockIdx.x * (long long)blockDim.x + threadIdx.x; ray < n;
       ray += (long long)gridDim.x * blockDim.x) {
    int c = 0;
    while (c + 1 < C.n && C.begin[c + 1] <= ray) ++c;
    RayState r = ray_start<T>(F, C.obs[c], C.eta_stop[c], dirs, n, ray, A.gravity_on != 0, err);
    while (!ray_step_fp64<T>(F, A, r, err)) {
    }
    n_steps[ray] = r.n_steps;
  }
}

template <class T>
cudaError_t launch_adjoint(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O,
                           const TraceArgs& A, const double* dL_dxi, const RecBar& R, int seg_len, int* d_steps,
                           long long** d_off_out, double** d_ck_out, cudaStream_t stream) {
  const long long n = A.n_rays;
  count_steps_kernel<T><<<(int)std::min<long long>((n + 127) / 128, 65535), 128, 0, stream>>>(launch_field(tree, A), C, dirs, A,
                                                                                            d_steps, tree->ws);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = adjoint_checkpoint_layout(d_steps, n, seg_len, d_off_out, d_ck_out, stream);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(tree->ws, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)kAdjBlock * (64 * sizeof(double) + 8 * sizeof(unsigned) + sizeof(int4));
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, adjoint_kernel<T>, kAdjBlock, smem);
  if (bps < 1) bps = 1;
  adjoint_kernel<T><<<tree->num_sms * bps, kAdjBlock, smem, stream>>>(launch_field(tree, A), C, dirs, O, A, dL_dxi, R, *d_ck_out,
                                                                    *d_off_out, seg_len, tree->ws);
  return cudaGetLastError();
}

}  // namespace

// Checkpoint layout of a reverse sweep from the per-ray step counts d_steps [n] (device): ray i
// gets ceil(steps_i / seg_len) + 1 slots of 8 doubles at slot offset (*d_off)[i].  Waits for
// `stream`; allocates *d_off ([n + 1] offsets) and *d_ck (the checkpoints), which the caller frees.
cudaError_t adjoint_checkpoint_layout(const int* d_steps, long long n, int seg_len, long long** d_off, double** d_ck,
                                      cudaStream_t stream) {
  std::vector<int> hs(n);
  cudaError_t e = cudaMemcpyAsync(hs.data(), d_steps, sizeof(int) * n, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return e;
  std::vector<long long> off(n + 1);
  off[0] = 0;
  for (long long i = 0; i < n; ++i) off[i + 1] = off[i] + std::max(1, (hs[i] + seg_len - 1) / seg_len) + 1;
  e = cudaMalloc(d_off, sizeof(long long) * (n + 1));
  if (e != cudaSuccess) return e;
  e = cudaMalloc(d_ck, sizeof(double) * 8 * (size_t)off[n]);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*d_off, off.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice);
}

mt_status run_adjoint(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O,
                      const double* dL_dxi, double* const* dL_drec, int checkpoint_every, const TraceArgs& A,
                      cudaStream_t stream) {
  if (checkpoint_every < 1 || checkpoint_every > kMaxSegment) return MT_ERR_INVALID_ARG;
  // FP32 octrees: the adjoint of the mixed-precision step the trace integrates there
  if (tree->precision != MT_FIELD_FP64)
    return run_adjoint_mixed(tree, C, dirs, O, dL_dxi, dL_drec, checkpoint_every, A, stream);
  RecBar R;
  for (int l = 0; l <= kMaxLevels; ++l) R.lv[l] = (l <= tree->n_levels) ? dL_drec[l] : nullptr;
  int* d_steps = nullptr;
  long long* d_off = nullptr;
  double* d_ck = nullptr;
  cudaError_t e = cudaMalloc(&d_steps, sizeof(int) * std::max<long long>(1, A.n_rays));
  if (e == cudaSuccess) {
    e = launch_adjoint<double>(tree, C, dirs, O, A, dL_dxi, R, checkpoint_every, d_steps, &d_off, &d_ck, stream);
  }
  cudaError_t e2 = cudaStreamSynchronize(stream);
  if (d_steps) cudaFree(d_steps);
  if (d_off) cudaFree(d_off);
  if (d_ck) cudaFree(d_ck);
  if (e == cudaErrorMemoryAllocation) return MT_ERR_OOM;
  return (e == cudaSuccess && e2 == cudaSuccess) ? MT_OK : MT_ERR_CUDA;
}

}  // namespace mt

using namespace mt;

extern "C" mt_status mt_trace_rays_adjoint(const mt_octree* tree, const mt_trace_params* params, const double* dirs,
                                           int64_t n_rays, const mt_ray_out* out, double* jac, double* lens,
                                           const double* dL_dxi, double* const* dL_drec, int32_t checkpoint_every,
                                           void* stream_) {
  if (!tree || !out) return MT_ERR_INVALID_ARG;
  mt_status st = check_trace_params(params, n_rays);
  if (st != MT_OK) return st;
  const bool fwd = jac || lens;
  const bool rev = dL_dxi || dL_drec;
  if (!fwd && !rev) return MT_ERR_INVALID_ARG;
  if (rev && (!dL_dxi || !dL_drec)) return MT_ERR_INVALID_ARG;
  if (rev && (checkpoint_every < 1 || checkpoint_every > 64)) return MT_ERR_INVALID_ARG;
  if (rev && params->interp != MT_INTERP_CIC) return MT_ERR_UNSUPPORTED;
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
  mt_status res = MT_OK;
  if (fwd) {
    cudaError_t e = launch_tangent(tree, C, dirs, O, jac, lens, A, stream);
    if (e != cudaSuccess) res = MT_ERR_CUDA;
  }
  if (res == MT_OK && rev) {
    // the tangent pass (if any) already wrote the ray outputs; the reverse pass writes them again
    res = run_adjoint(tree, C, dirs, O, dL_dxi, dL_drec, checkpoint_every, A, stream);
  }
  if (prev >= 0 && prev != tree->device) cudaSetDevice(prev);
  return res;
}
