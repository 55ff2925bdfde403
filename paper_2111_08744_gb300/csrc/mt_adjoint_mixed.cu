// Reverse mode on FP32 octrees: the exact adjoint of the mixed-precision ray map that mt_trace_rays
// integrates there (FP32 stage arithmetic, FP64 ray state; mt_mixed.cuh), giving the gradient of a
// loss on the end points with respect to the records (Sect. 2.2: RK4 of Eqs. 2-4, CIC with level
// fallback, slices linear in eta).
//
// Per ray:
//   1. integrate forward with the mixed step (checkpoint_mixed_kernel, scheduled as trace_kernel:
//      a lane whose ray ends takes the next id of its warp's chunk), keeping the FP64 state every
//      `checkpoint_every` steps, and write the ray's outputs;
//   2. form the cotangent of the final state from dL/dxi, xi = x - (k/k0)(eta - eta_stop);
//   3. (adjoint_mixed_kernel: a warp takes 32 consecutive ray ids at a time and runs their phases
//      in lockstep) for each segment, last to first: recompute its steps from the checkpoint,
//      keeping each step's start state and stage data (the stage wave-vector offsets, right-hand
//      sides and step size), then reverse each step: the stages from the last to the first are
//      interpolated again (FP32) and their transposed Jacobians applied in FP32 to the stage
//      cotangents, while the state's cotangent accumulates in FP64.  The parts of the step that are
//      linear in the step-start state (x += h k, eta += h k0, and the step size's dependence on k0
//      and eta) are applied in FP64, as in the forward step;
//   4. the cotangents of grad phi and phi_eta at each stage go to the stage's 8 CIC records of both
//      bracketing slices through a per-lane FP32 accumulator in shared memory, flushed with FP64
//      atomics when the neighbourhood changes; the same pass over the 8 corners pulls them back to
//      the stage position through the derivative of the CIC weights; phi at the observer (the
//      initial wave vector) scatters once per ray.
// Rays that do not end with MT_RAY_OK contribute nothing.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mt_deriv.cuh"

namespace mt {
namespace {

constexpr int kAdjMBlock = 128;
constexpr int kAdjMChunk = 32;
constexpr int kMaxSegmentM = 64;

struct RecBarM {
  double* lv[kMaxLevels + 1];  // record cotangents [count][S][4] per level (NULL: skip the level)
};

// Per-lane FP32 accumulator of record cotangents: the 8 corners x 2 slices x 4 components of the
// last CIC neighbourhood a stage scattered to, the corners' rows and the neighbourhood's key.
struct ScatterAcc {
  float* acc;      // acc[(8 c + 4 slice + q) * stride]
  unsigned* rows;  // rows[c * stride]
  int4* key;       // (level << 8 | slice, i0); x = -1: empty
  int stride;
};

__device__ __noinline__ void acc_flush(const DevField& F, const RecBarM& R, const ScatterAcc& sc) {
  const int4 k = *sc.key;
  if (k.x < 0) return;
  const int l = k.x >> 8, s = k.x & 255;
  double* base = R.lv[l];
  const int ns = F.S > 1 ? 2 : 1;
  for (int c = 0; c < 8; ++c) {
    const unsigned row = sc.rows[c * sc.stride];
    for (int sl = 0; sl < 2; ++sl) {
      for (int q = 0; q < 4; ++q) {
        float* a = sc.acc + (8 * c + 4 * sl + q) * sc.stride;
        if (base && sl < ns && *a != 0.0f) atomicAdd(base + ((size_t)row * F.S + s + sl) * 4 + q, (double)*a);
        *a = 0.0f;
      }
    }
  }
  *sc.key = make_int4(-1, 0, 0, 0);
}

// Add the cotangents (gbar, pebar) of the stage's interpolated grad phi and phi_eta to its CIC
// records: g = v_s + wt (v_{s+1} - v_s), phi_eta = (phi_{s+1} - phi_s) ids, each corner with weight
// prod (f or 1 - f); and, in the same pass over the corners, their pull-back to the stage position,
// tb[d] += sum_c (d weight_c / dx_d) (a0 . r_c,s + a1 . r_c,s+1) with the stage's records r from the
// lane cache (which holds the neighbourhood the stage interpolated from) and a0, a1 the cotangents
// of the two slices' records.
__device__ void acc_add(const DevField& F, const RecBarM& R, const ScatterAcc& sc, const LaneCache& lc,
                        const StageF& sf, const float* gbar, float pebar, float* tb, unsigned* err) {
  const int4 key = make_int4((sf.lev << 8) | sf.sl, sf.i0[0], sf.i0[1], sf.i0[2]);
  const int4 old = *sc.key;
  bool scatter = true;
  if (!(old.x == key.x && old.y == key.y && old.z == key.z && old.w == key.w)) {
    acc_flush(F, R, sc);
    if (sf.rows_ok) {  // the stage staged this neighbourhood and looked its rows up already
#pragma unroll
      for (int c = 0; c < 8; ++c) sc.rows[c * sc.stride] = sf.rows[c];
      *sc.key = key;
    } else {
      const long long i0l[3] = {sf.i0[0], sf.i0[1], sf.i0[2]};
      unsigned rows[8];
      // the stage interpolated from these 8 cells, so they exist; should the lookup fail all the same,
      // the record cotangents are dropped (the accumulator stays empty) and the position part kept
      scatter = cic_rows_compact(F, sf.lev, i0l, rows, err);
      if (scatter) {
#pragma unroll
        for (int c = 0; c < 8; ++c) sc.rows[c * sc.stride] = rows[c];
        *sc.key = key;
      }
    }
  }
  float a0[4], a1[4];
  if (F.S == 1) {
    a0[0] = 0.0f;
    a1[0] = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      a0[1 + i] = gbar[i];
      a1[1 + i] = 0.0f;
    }
  } else {
    a0[0] = -sf.ids * pebar;
    a1[0] = sf.ids * pebar;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      a0[1 + i] = (1.0f - sf.wt) * gbar[i];
      a1[1 + i] = sf.wt * gbar[i];
    }
  }
  float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f;
#pragma unroll 1
  for (int c = 0; c < 8; ++c) {
    const float wx = (c & 1) ? sf.f[0] : 1.0f - sf.f[0];
    const float wy = (c & 2) ? sf.f[1] : 1.0f - sf.f[1];
    const float wz = (c & 4) ? sf.f[2] : 1.0f - sf.f[2];
    const float w = wx * wy * wz;
    const float4 r0 = lc.rec[(2 * c) * lc.stride];
    const float4 r1 = lc.rec[(2 * c + 1) * lc.stride];
    const float ar = a0[0] * r0.x + a0[1] * r0.y + a0[2] * r0.z + a0[3] * r0.w + a1[0] * r1.x + a1[1] * r1.y +
                     a1[2] * r1.z + a1[3] * r1.w;
    p0 += ((c & 1) ? 1.0f : -1.0f) * wy * wz * ar;
    p1 += ((c & 2) ? 1.0f : -1.0f) * wx * wz * ar;
    p2 += ((c & 4) ? 1.0f : -1.0f) * wx * wy * ar;
    if (scatter) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        sc.acc[(8 * c + q) * sc.stride] += w * a0[q];
        sc.acc[(8 * c + 4 + q) * sc.stride] += w * a1[q];
      }
    }
  }
  const float inv = F.inv_dxf_f / (float)(1 << (F.L - sf.lev));  // d (level cell coordinate) / d x
  tb[0] += p0 * inv;
  tb[1] += p1 * inv;
  tb[2] += p2 * inv;
}

// Transposed Jacobian of the FP32 right-hand side at a stage (Eqs. 2-4 with Eq. 4's D = grad phi . k
// + phi_eta k0): tb = J^T w for the stage state (x[3], eta, k0, k[3]) and the cotangents of the
// interpolated grad phi and phi_eta.  w: cotangents of K = (k[3], k0, dk0/dlambda, dk/dlambda).
// The terms of tb[0..2] that go through the interpolant's spatial derivative are left to acc_add.
__device__ __forceinline__ void stage_adjoint_mixed(const StageF& sf, float k0, const float* k, const float* w,
                                                    float* tb, float* gbar, float* pebar) {
  const float H = sf.H, pe = sf.pe, D = sf.D;
  const float wk0 = w[4];
  const float* wk = w + 5;
  tb[0] = tb[1] = tb[2] = tb[3] = 0.0f;
  tb[5] = w[0];
  tb[6] = w[1];
  tb[7] = w[2];
  tb[4] = w[3];
  float dHbar = -2.0f * k0 * k0 * wk0;
  tb[4] += (-4.0f * H * k0 - 2.0f * D + 4.0f * pe * k0) * wk0;
  float dDbar = -2.0f * k0 * wk0;
  float dpebar = 2.0f * k0 * k0 * wk0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    dHbar += -2.0f * k0 * k[j] * wk[j];
    tb[4] += (-2.0f * H * k[j] - 4.0f * sf.g[j] * k0) * wk[j];
    tb[5 + j] += (-2.0f * H * k0 + 2.0f * D) * wk[j];
    dDbar += 2.0f * k[j] * wk[j];
    gbar[j] = -2.0f * k0 * k0 * wk[j];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    gbar[i] += k[i] * dDbar;
    tb[5 + i] += sf.g[i] * dDbar;
  }
  dpebar += k0 * dDbar;
  tb[4] += pe * dDbar;
  tb[3] += sf.dH * dHbar;
#pragma unroll
  for (int i = 0; i < 3; ++i) tb[3] += sf.ge[i] * gbar[i];
  *pebar = dpebar;
  // the position part, sum_i gbar_i d g_i / dx_d + pebar d phi_eta / dx_d, is added by acc_add from the
  // stage's records (the derivative of the interpolant applied to the cotangents directly)
}

// Reverse of one mixed step from the step-start state y (FP64 x[3], eta, k0, k[3]) and the step's
// stage data `rec` (recorded by ray_step_mixed when the segment was recomputed): yb holds the
// cotangent of the step's end state on entry and of its start state on return.  False if a stage
// left a non-periodic domain (cannot happen on a ray that ended with MT_RAY_OK).
template <bool Grav>
__device__ bool reverse_step_mixed(const DevField& F, const TraceArgs& A, const double* y, const float* rec,
                                   double* yb, const LaneCache* lc, const ScatterAcc& sc, const RecBarM& R,
                                   unsigned* err) {
  MixedStep B;
  if (!mixed_begin(F, y, B)) return false;
  const double eta = y[3];
  const float k0s = (float)y[4];
  const float ks[3] = {(float)y[5], (float)y[6], (float)y[7]};
  // the stages' wave-vector offsets (k0, k) from the step start (stage st's wave vector is the step
  // start's plus okk(st, .)) and their right-hand sides Kk(st, .) = (dk0, dk)/dlambda
  const auto okk = [rec](int st, int i) { return rec[4 * st + i]; };
  const auto Kk = [rec](int st, int i) { return rec[16 + 4 * st + i]; };
  const float h = rec[32];
  const bool last = rec[33] != 0.0f;
  // y' = y + h sum_j b_j K_j, K_j = (k + dk_j, k0 + dk0_j, Kk0_j, Kk_j) with the FP64 step-start k, k0
  // (x and eta advance by h k in FP64 and h sum_j b_j dk_j in FP32, as in ray_step_mixed): the
  // cotangents of the stage right-hand sides, and of h, whose step-start part is formed in FP64 (it
  // cancels against the eta part on the last step).
  const double hd = (double)h;
  double hbar = yb[0] * y[5] + yb[1] * y[6] + yb[2] * y[7] + yb[3] * y[4];
  float hbar_f = 0.0f;
  float ybf[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) ybf[i] = (float)yb[i];
#pragma unroll 1
  for (int st = 0; st < 4; ++st) {
    const float b = (st == 0 || st == 3) ? (1.0f / 6.0f) : (1.0f / 3.0f);
    hbar_f += b * (ybf[0] * okk(st, 1) + ybf[1] * okk(st, 2) + ybf[2] * okk(st, 3) + ybf[3] * okk(st, 0) +
                   ybf[4] * Kk(st, 0) + ybf[5] * Kk(st, 1) + ybf[6] * Kk(st, 2) + ybf[7] * Kk(st, 3));
  }
  // stages from the last to the first.  Stage j sits at y + a_{j-1} h K_{j-1}, so the cotangent of
  // K_j is b_j h yb' (the step's sum) plus a_j h times the cotangent of stage j + 1's state.
  float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // sum of the stage-state cotangents (added to yb in FP64)
  float tbn[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // cotangent of the state of the stage after this one
#pragma unroll 1
  for (int st = 3; st >= 0; --st) {
    float offx[3] = {0.0f, 0.0f, 0.0f}, offe = 0.0f;
    const float a = st == 3 ? 1.0f : 0.5f;  // stage st sits at y + a h K_{st-1}
    float kp0 = 0.0f, kp[3] = {0.0f, 0.0f, 0.0f};  // wave vector of stage st - 1
    if (st > 0) {
      kp0 = k0s + okk(st - 1, 0);
      kp[0] = ks[0] + okk(st - 1, 1);
      kp[1] = ks[1] + okk(st - 1, 2);
      kp[2] = ks[2] + okk(st - 1, 3);
      const float c = a * h;
      offx[0] = c * kp[0];
      offx[1] = c * kp[1];
      offx[2] = c * kp[2];
      offe = c * kp0;
    }
    const float b = (st == 0 || st == 3) ? (1.0f / 6.0f) : (1.0f / 3.0f);
    const float an = st == 2 ? 1.0f : 0.5f;  // stage st + 1 sits at y + an h K_st
    float Kb[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) Kb[i] = b * h * ybf[i] + (st < 3 ? an * h * tbn[i] : 0.0f);
    const float k0v = k0s + okk(st, 0);
    const float kv[3] = {ks[0] + okk(st, 1), ks[1] + okk(st, 2), ks[2] + okk(st, 3)};
    float Kk0, Kkv[3], KI, Ks;
    StageF sf;
    if (!rhs_mixed<true, MT_INTERP_CIC, true>(F, Grav, B, eta, offx, offe, k0v, kv, &Kk0, Kkv, &KI, &Ks, nullptr, err,
                                        lc, &sf))
      return false;
    float gbar[3], pebar;
    stage_adjoint_mixed(sf, k0v, kv, Kb, tbn, gbar, &pebar);
    if (Grav) acc_add(F, R, sc, *lc, sf, gbar, pebar, tbn, err);
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] += tbn[i];
    if (st > 0) {
      // Y_st = y + a h K_{st-1}, K_{st-1} = (k, k0, Kk0, Kk) of stage st - 1
      const float Kprev[8] = {kp[0],         kp[1],         kp[2],         kp0,
                              Kk(st - 1, 0), Kk(st - 1, 1), Kk(st - 1, 2), Kk(st - 1, 3)};
      float dot = 0.0f;
#pragma unroll
      for (int i = 0; i < 8; ++i) dot += tbn[i] * Kprev[i];
      hbar_f += a * dot;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) yb[i] += (double)acc[i];
  hbar += (double)hbar_f;
  // h = dx_l / (N |k0|), or (eta_stop - eta) / k0 on the last step
  const double k0 = y[4];
  if (last) yb[3] += -hbar / k0;
  yb[4] += -hbar * hd / k0;
  return true;
}

// Ray id of a warp lane: warps claim chunks of consecutive ids (as trace_kernel).
struct WarpQueue {
  unsigned long long pool = 0;
  int pool_left = 0;
  __device__ long long next(bool need, unsigned lane, unsigned long long* counter) {
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (!m) return -1;
    const int leader = __ffs(m) - 1;
    const int k = __popc(m);
    const int from_pool = k < pool_left ? k : pool_left;
    unsigned long long fresh = 0;
    if (k > from_pool) {
      if ((int)lane == leader) fresh = atomicAdd(counter, (unsigned long long)kAdjMChunk);
      fresh = __shfl_sync(0xffffffffu, fresh, leader);
    }
    const int rank = __popc(m & ((1u << lane) - 1u));
    const unsigned long long pick = rank < from_pool ? pool + rank : fresh + (rank - from_pool);
    if (k > from_pool) {
      pool = fresh + (k - from_pool);
      pool_left = kAdjMChunk - (k - from_pool);
    } else {
      pool += k;
      pool_left -= k;
    }
    return need ? (long long)pick : -1;
  }
};

__device__ void lane_cache_init(LaneCache& lc, float4* smem) {
  lc.rec = smem + threadIdx.x;
  lc.key = (int4*)(smem + 16 * kAdjMBlock) + threadIdx.x;
  lc.stride = kAdjMBlock;
  lc.loc = (int4*)(smem + 16 * kAdjMBlock) + kAdjMBlock + threadIdx.x;
  *lc.loc = make_int4(0, 0, 0, -1);
  *lc.key = make_int4(-1, 0, 0, 0);
}

// The same with the keys of the lane's last two incomplete CIC neighbourhoods (the level fallback
// passes over them without probing, as in trace_kernel), for the forward kernels.
__device__ void lane_cache_init_neg(LaneCache& lc, float4* smem) {
  lane_cache_init(lc, smem);
  lc.neg = (int4*)(smem + 16 * kAdjMBlock) + 2 * kAdjMBlock + threadIdx.x;
  lc.neg[0] = lc.neg[kAdjMBlock] = make_int4(-1, 0, 0, 0);
}

constexpr size_t kLaneCacheBytes = (size_t)kAdjMBlock * (16 * sizeof(float4) + 2 * sizeof(int4));
constexpr size_t kLaneCacheNegBytes = kLaneCacheBytes + (size_t)kAdjMBlock * 2 * sizeof(int4);
constexpr size_t kAccBytes = (size_t)kAdjMBlock * (64 * sizeof(float) + 8 * sizeof(unsigned) + sizeof(int4));

// Step counts of the mixed trace (the checkpoint layout).
__global__ void __launch_bounds__(kAdjMBlock) count_mixed_kernel(DevField F, DevCones C, const double* __restrict__ dirs,
                                                                 TraceArgs A, int* n_steps, unsigned long long* ws) {
  unsigned* err = (unsigned*)(ws + 1);
  extern __shared__ float4 smem_c[];
  LaneCache lc;
  lane_cache_init_neg(lc, smem_c);
  const unsigned lane = threadIdx.x & 31u;
  const long long n = A.n_rays;
  const bool grav = A.gravity_on != 0;
  WarpQueue q;
  long long ray = -1;
  bool exhausted = false;
  RayState r;
  for (;;) {
    const bool need = ray < 0 && !exhausted;
    const long long id = q.next(need, lane, ws);
    if (need) {
      if (id >= 0 && id < n) {
        ray = id;
        int c = 0;
        while (c + 1 < C.n && C.begin[c + 1] <= ray) ++c;
        r = ray_start<float>(F, C.obs[c], C.eta_stop[c], dirs, n, ray, grav, err);
        *lc.key = make_int4(-1, 0, 0, 0);
      } else {
        exhausted = true;
      }
    }
    if (!__any_sync(0xffffffffu, ray >= 0)) break;
    if (ray >= 0 && ray_step_mixed<MT_INTERP_CIC>(F, A, r, err, &lc)) {
      n_steps[ray] = r.n_steps;
      ray = -1;
    }
  }
}

// Forward pass of the reverse mode, with the scheduling of trace_kernel (a lane whose ray ends takes
// the next id of its warp's chunk): the mixed trace of every ray, writing its FP64 state every seg_len
// steps into its checkpoint slots (ck_off), its outputs, and what the sweep starts from: the cotangent
// of the end state from dL/dxi (xi = x - (k/k0)(eta - eta_stop)) in yb0[0..7][n], phi at the observer
// in yb0[8][n], and the number of steps to reverse in n_rev (0 for a ray that did not end with
// MT_RAY_OK).
__global__ void __launch_bounds__(kAdjMBlock, 4) checkpoint_mixed_kernel(DevField F, DevCones C,
                                                                      const double* __restrict__ dirs, OutPtrs O,
                                                                      TraceArgs A, const double* __restrict__ dL_dxi,
                                                                      double* ckpt, const long long* ck_off, int seg_len,
                                                                      double* yb0, int* n_rev, unsigned long long* ws) {
  unsigned* err = (unsigned*)(ws + 1);
  extern __shared__ float4 smem_k[];
  LaneCache lc;
  lane_cache_init_neg(lc, smem_k);
  const unsigned lane = threadIdx.x & 31u;
  const long long n = A.n_rays;
  const bool grav = A.gravity_on != 0;
  WarpQueue q;
  long long ray = -1;
  bool exhausted = false;
  RayState r;
  long long off = 0, n_ck = 0;
  bool ok = false;
  for (;;) {
    const bool need = ray < 0 && !exhausted;
    const long long id = q.next(need, lane, ws);
    if (need) {
      if (id >= 0 && id < n) {
        ray = id;
        int c = 0;
        while (c + 1 < C.n && C.begin[c + 1] <= ray) ++c;
        r = ray_start<float>(F, C.obs[c], C.eta_stop[c], dirs, n, ray, grav, err);
        off = ck_off[ray];
        n_ck = ck_off[ray + 1] - off;
        ok = true;
        *lc.key = make_int4(-1, 0, 0, 0);
      } else {
        exhausted = true;
      }
    }
    if (!__any_sync(0xffffffffu, ray >= 0)) break;
    if (ray < 0) continue;
    bool done = false;
    if (r.n_steps % seg_len == 0) {
      const long long j = r.n_steps / seg_len;
      if (j >= n_ck) {
        atomicOr(err, kErrOOB);  // more steps than the counting pass found
        ok = false;
        done = true;
      } else {
        double* cp = ckpt + (off + j) * 8;
        for (int i = 0; i < 8; ++i) cp[i] = r.y[i];
      }
    }
    if (!done) done = ray_step_mixed<MT_INTERP_CIC>(F, A, r, err, &lc);
    if (done) {
      ray_finish<float>(F, A, r, ray, n, O, err);
      const bool active = ok && r.status == MT_RAY_OK && r.n_steps > 0;
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
      for (int i = 0; i < 8; ++i) yb0[i * n + ray] = yb[i];
      yb0[8 * n + ray] = r.phi_o;
      n_rev[ray] = active ? r.n_steps : 0;
      ray = -1;
    }
  }
}

// The mixed step of the segment recompute: its CIC in the compact form (the sweep's code must fit
// the instruction cache beside the reverse step), recording the step's stage data for the reverse
// step in rec.
__device__ __forceinline__ bool segment_step(const DevField& F, const TraceArgs& A, RayState& r, unsigned* err,
                                          const LaneCache* lc, float* rec) {
  return ray_step_mixed<MT_INTERP_CIC, true, true>(F, A, r, err, lc, rec);
}

// Scatter the cotangent phib of phi at the observer (the initial wave vector depends on it) onto the
// CIC records ray_start sampled there (FP64 coordinates, FP32 weights, the slice bracket of eta_o).
__device__ void scatter_observer(const DevField& F, const RecBarM& R, const double* xo, double phib, unsigned* err) {
  double u[3];
  if (!coarse_coords<float>(F, xo, u)) return;
  const int lfin = locate_level(F, u, err);
  int s = 0;
  while (s < F.S - 2 && F.seta[s + 1] <= F.eta_o) ++s;
  for (int l = lfin; l >= 0; --l) {
    const double scl = (double)(1ll << l);
    long long i0[3];
    float f[3];
    for (int d = 0; d < 3; ++d) {
      const double U = u[d] * scl - 0.5;
      const double fl = floor(U);
      i0[d] = (long long)fl;
      f[d] = (float)(U - fl);
    }
    unsigned rows[8];
    if (!cic_rows(F, l, i0, rows, err)) continue;
    double* base = R.lv[l];
    if (!base) return;
    const float wt = F.S > 1 ? (float)((F.eta_o - F.seta[s]) / (F.seta[s + 1] - F.seta[s])) : 0.0f;
    for (int c = 0; c < 8; ++c) {
      const float wx = (c & 1) ? f[0] : 1.0f - f[0];
      const float wy = (c & 2) ? f[1] : 1.0f - f[1];
      const float wz = (c & 4) ? f[2] : 1.0f - f[2];
      const double w = (double)(wx * wy * wz);
      double* r0 = base + ((size_t)rows[c] * F.S + s) * 4;
      if (F.S == 1) {
        atomicAdd(r0, w * phib);
      } else {
        atomicAdd(r0, w * (double)(1.0f - wt) * phib);
        atomicAdd(r0 + 4, w * (double)wt * phib);
      }
    }
    return;
  }
}

// Warp-synchronous sweep: a warp takes 32 consecutive rays per turn (sky neighbours), starts from
// what checkpoint_mixed_kernel left (step counts, checkpoints, end cotangents, phi at the observer)
// and reverses them segment by segment, aligned on each ray's last segment, with warp-uniform loop
// bounds, so that the lanes run the same phase (recompute or reverse) at the same time; only the
// rays' different step counts leave lanes idle.  The segment recompute evaluates the forward pass's
// arithmetic (the mixed step, its CIC in the compact form, which changes no result), so it retraces
// the forward pass bit for bit.
template <bool Grav>
__global__ void __launch_bounds__(kAdjMBlock, 3) adjoint_mixed_kernel(DevField F, DevCones C,
                                                                   const double* __restrict__ dirs, TraceArgs A,
                                                                   RecBarM R, const double* ckpt,
                                                                   const long long* ck_off, int seg_len,
                                                                   const double* yb0, const int* n_rev,
                                                                   unsigned long long* ws) {
  unsigned* err = (unsigned*)(ws + 1);
  extern __shared__ float4 smem_a[];
  LaneCache lc;
  lane_cache_init(lc, smem_a);
  ScatterAcc sc;
  sc.stride = kAdjMBlock;
  float* accbase = (float*)((char*)smem_a + kLaneCacheBytes);
  sc.acc = accbase + threadIdx.x;
  sc.rows = (unsigned*)(accbase + 64 * kAdjMBlock) + threadIdx.x;
  sc.key = (int4*)((unsigned*)(accbase + 64 * kAdjMBlock) + 8 * kAdjMBlock) + threadIdx.x;
  for (int j = 0; j < 64; ++j) sc.acc[j * sc.stride] = 0.0f;
  *sc.key = make_int4(-1, 0, 0, 0);
  double ys[kMaxSegmentM][8];
  float rs[kMaxSegmentM][kStepRecordFloats];
  const unsigned lane = threadIdx.x & 31u;
  const long long n = A.n_rays;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(ws, (unsigned long long)kAdjMChunk);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= (unsigned long long)n) break;
    const long long ray = (long long)base + lane;
    const bool have = ray < n;
    // the ray's forward pass (checkpoint_mixed_kernel): its step count, checkpoints and end cotangent
    RayState r;
    long long off = 0;
    int n_steps = 0;
    double yb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (have) {
      int c = 0;
      while (c + 1 < C.n && C.begin[c + 1] <= ray) ++c;
      r.xo[0] = C.obs[c][0];
      r.xo[1] = C.obs[c][1];
      r.xo[2] = C.obs[c][2];
      r.eta_stop = C.eta_stop[c];
      r.y[8] = r.y[9] = 0.0;
      r.lambda = 0.0;
      r.phi_o = yb0[8 * n + ray];
      r.status = MT_RAY_OK;
      n_steps = n_rev[ray];
      off = ck_off[ray];
      for (int i = 0; i < 8; ++i) yb[i] = yb0[i * n + ray];
    }
    *lc.key = make_int4(-1, 0, 0, 0);
    const bool active = n_steps > 0;
    const int n_seg = (n_steps + seg_len - 1) / seg_len;
    const int max_seg = (int)__reduce_max_sync(0xffffffffu, (unsigned)n_seg);
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
      // every lane runs these loops with the same bounds, so all 32 reach each __syncwarp: the warp
      // reconverges after every step instead of letting its lanes drift apart in the branches
      for (int st = 0; st < seg_len; ++st) {
        if (st < len) {
          for (int i = 0; i < 8; ++i) ys[st][i] = q.y[i];
          segment_step(F, A, q, err, &lc, rs[st]);  // the last step's end state is not kept
        }
        __syncwarp();
      }
      for (int st = seg_len - 1; st >= 0; --st) {
        if (st < len && alive) {
          if (!reverse_step_mixed<Grav>(F, A, ys[st], rs[st], yb, &lc, sc, R, err)) alive = false;
        }
        __syncwarp();
      }
    }
    // 4. the initial wave vector k = n sqrt((1 + 2 phi_o)/(1 - 2 phi_o)) depends on phi_o
    if (alive && Grav) {
      const double nd[3] = {__ldg(&dirs[ray]), __ldg(&dirs[n + ray]), __ldg(&dirs[2 * n + ray])};
      const double po = r.phi_o;
      const double kn = sqrt((1.0 + 2.0 * po) / (1.0 - 2.0 * po));
      const double phib =
          (yb[5] * nd[0] + yb[6] * nd[1] + yb[7] * nd[2]) * 2.0 / (kn * (1.0 - 2.0 * po) * (1.0 - 2.0 * po));
      scatter_observer(F, R, r.xo, phib, err);
    }
    acc_flush(F, R, sc);
  }
}

}  // namespace

// Reverse mode on an FP32 octree (called by run_adjoint): counts the mixed steps per ray, lays out
// the checkpoints and runs the sweep.
mt_status run_adjoint_mixed(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O,
                            const double* dL_dxi, double* const* dL_drec, int checkpoint_every, const TraceArgs& A,
                            cudaStream_t stream) {
  if (checkpoint_every < 1 || checkpoint_every > kMaxSegmentM) return MT_ERR_INVALID_ARG;
  RecBarM R;
  for (int l = 0; l <= kMaxLevels; ++l) R.lv[l] = (l <= tree->n_levels) ? dL_drec[l] : nullptr;
  const long long n = A.n_rays;
  int* d_steps = nullptr;
  long long* d_off = nullptr;
  double* d_ck = nullptr;
  double* d_yb0 = nullptr;
  cudaError_t e = cudaMalloc(&d_steps, sizeof(int) * std::max<long long>(1, n));
  if (e == cudaSuccess) e = cudaMemsetAsync(tree->ws, 0, sizeof(unsigned long long), stream);
  if (e == cudaSuccess) {
    static int bps_c = -1;
    if (bps_c < 0) {
      int b = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, count_mixed_kernel, kAdjMBlock, kLaneCacheNegBytes) !=
              cudaSuccess ||
          b < 1)
        b = 1;
      bps_c = b;
    }
    count_mixed_kernel<<<tree->num_sms * bps_c, kAdjMBlock, kLaneCacheNegBytes, stream>>>(launch_field(tree, A), C,
                                                                                            dirs, A, d_steps, tree->ws);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = adjoint_checkpoint_layout(d_steps, n, checkpoint_every, &d_off, &d_ck, stream);
  // forward pass: checkpoints, outputs and the end cotangents
  if (e == cudaSuccess) e = cudaMalloc(&d_yb0, sizeof(double) * 9 * (size_t)std::max<long long>(1, n));
  if (e == cudaSuccess) e = cudaMemsetAsync(tree->ws, 0, sizeof(unsigned long long), stream);
  if (e == cudaSuccess) {
    static int bps_k = -1;
    if (bps_k < 0) {
      int b = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, checkpoint_mixed_kernel, kAdjMBlock, kLaneCacheNegBytes) !=
              cudaSuccess ||
          b < 1)
        b = 1;
      bps_k = b;
    }
    checkpoint_mixed_kernel<<<tree->num_sms * bps_k, kAdjMBlock, kLaneCacheNegBytes, stream>>>(
        launch_field(tree, A), C, dirs, O, A, dL_dxi, d_ck, d_off, checkpoint_every, d_yb0, d_steps, tree->ws);
    e = cudaGetLastError();
  }
  // reverse sweep
  if (e == cudaSuccess) e = cudaMemsetAsync(tree->ws, 0, sizeof(unsigned long long), stream);
  if (e == cudaSuccess) {
    const size_t smem = kLaneCacheBytes + kAccBytes;
    static int bps[2] = {-1, -1};
    const int g = A.gravity_on ? 1 : 0;
    if (bps[g] < 0) {
      const void* fn = g ? (const void*)adjoint_mixed_kernel<true> : (const void*)adjoint_mixed_kernel<false>;
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      int b = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kAdjMBlock, smem) != cudaSuccess || b < 1) b = 1;
      bps[g] = b;
    }
    const int grid = tree->num_sms * bps[g];
    if (g) {
      adjoint_mixed_kernel<true><<<grid, kAdjMBlock, smem, stream>>>(launch_field(tree, A), C, dirs, A, R, d_ck, d_off,
                                                                     checkpoint_every, d_yb0, d_steps, tree->ws);
    } else {
      adjoint_mixed_kernel<false><<<grid, kAdjMBlock, smem, stream>>>(launch_field(tree, A), C, dirs, A, R, d_ck, d_off,
                                                                      checkpoint_every, d_yb0, d_steps, tree->ws);
    }
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaStreamSynchronize(stream);
  if (d_steps) cudaFree(d_steps);
  if (d_off) cudaFree(d_off);
  if (d_ck) cudaFree(d_ck);
  if (d_yb0) cudaFree(d_yb0);
  if (e == cudaErrorMemoryAllocation) return MT_ERR_OOM;
  return (e == cudaSuccess && e2 == cudaSuccess) ? MT_OK : MT_ERR_CUDA;
}

}  // namespace mt
