// Mixed-precision RK4 step (FP32 field and arithmetic inside a step, FP64 ray state).
//
// Same method as the FP64 step (Sect. 2.2: RK4 in lambda, N steps per AMR cell, CIC with
// level fallback, Eqs. 2-4), arranged so that double precision is spent only where it
// carries accuracy:
//   * at the step start the FP64 position is split once into an integer cell index on the
//     finest level plus an FP32 in-cell fraction; stage positions are FP32 offsets from it,
//     so locate and CIC run on integers and floats only;
//   * the background H(eta) is a single-precision Hermite interpolant around the step's
//     table node; the time slices are bracketed by FP32 offsets from the step start;
//   * the right-hand side of Eqs. (2)-(4) is evaluated in FP32 at FP32 stage states
//     (its rounding enters the state only through h * derivative);
//   * the state update y += h sum_i b_i K_i stays FP64: x and eta advance by h k(step
//     start) in FP64 plus an FP32 correction from the stage offsets of k.
#pragma once

#include "mt_internal.cuh"

namespace mt {

// Finest-level integer index and FP32 fraction of an FP64 position (once per step).  The
// periodic wrap is an integer mask: shifting by whole periods leaves the fraction unchanged.
__device__ __forceinline__ bool finest_base(const DevField& F, const double* x, int* ib, float* fb) {
  bool inside = true;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double v = x[d] * F.inv_dxf;
    const double fl = floor(v);
    const long long il = (long long)fl;
    if (F.periodic) {
      ib[d] = (int)(il & (long long)(F.nf - 1));
    } else {
      inside = inside && (il >= 0) && (il < (long long)F.nf);
      ib[d] = (int)il;
    }
    fb[d] = (float)(v - fl);
  }
  return inside;
}

// Stage position: base index + (fraction + offset) in finest cells.
__device__ __forceinline__ bool stage_coords(const DevField& F, const int* ib, const float* fb, const float* offx,
                                             int* ic, float* fc) {
  bool inside = true;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float U = fb[d] + offx[d] * F.inv_dxf_f;
    const float c = floorf(U);
    int i = ib[d] + (int)c;
    fc[d] = U - c;
    if (F.periodic) {
      i &= (F.nf - 1);
    } else {
      inside = inside && (i >= 0) && (i < F.nf);
    }
    ic[d] = i;
  }
  return inside;
}

// Per-ray staging of the last CIC neighbourhood in shared memory: the 8 corner records of
// both bracketing slices (16 float4) and their key (level, slice, lower corner).  Consecutive
// RK4 stages of a ray stay in one neighbourhood most of the time (a step moves 1/N of a cell), so
// most stages read their records from shared memory instead of L1/L2, and skip the index work.
struct LaneCache {
  float4* rec;   // rec[j * stride] for j = 0..15 (corner-major, lanes interleaved: no bank conflicts);
                 // the TSC instances keep the 27 neighbour rows here instead (tsc_gather_cached)
  int4* key;     // (level << 8 | slice, i0x, i0y, i0z) (TSC: the cell, not the lower corner); level -1: empty
  int stride;
  int4* loc;     // last locate answer: the cell (x, y, z) of level w that contains the point, w the
                 // finest level there (w = -1: empty); a property of the field, valid across rays;
                 // may be null
  int4* neg = nullptr;  // neg[0], neg[stride]: keys (as `key`) of the lane's two last CIC (TSC)
                        // neighbourhoods found incomplete at their level (level -1: empty); a property
                        // of the field, valid across rays; may be null
};

__device__ __forceinline__ bool same_key(const int4& a, const int4& b) {
  return a.x == b.x && a.y == b.y && a.z == b.z && a.w == b.w;
}

// Lower corner and in-cell fractions of the level-l CIC neighbourhood of the point with
// finest-level integer coordinates ic and fractions fc (Eq. 8: the 8 cells whose centres surround
// it), and its key (level << 8 | slice, i0).
__device__ __forceinline__ int4 cic_key(const DevField& F, int l, const int* ic, const float* fc, int s, int* i0,
                                        float* f) {
  const int sh = F.L - l;
  const float inv = 1.0f / (float)(1 << sh);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int ilev = ic[d] >> sh;
    const float fl = ((float)(ic[d] & ((1 << sh) - 1)) + fc[d]) * inv;
    if (fl >= 0.5f) {
      i0[d] = ilev;
      f[d] = fl - 0.5f;
    } else {
      i0[d] = ilev - 1;
      f[d] = fl + 0.5f;
    }
  }
  return make_int4((l << 8) | s, i0[0], i0[1], i0[2]);
}

// First level of the CIC fallback (Sect. 2.2, Fig. 1) for a point whose finest level is l: levels
// whose neighbourhood of the point is one the lane found incomplete before are passed over
// without probing (a neighbourhood's completeness is a property of the field), so a ray that
// stays near the edge of a refined region does not re-probe the missing cells at every stage.
__device__ __forceinline__ int cic_first_level(const DevField& F, int l, const int* ic, const float* fc, int s,
                                               const LaneCache& lc) {
  while (l > 0) {
    int i0[3];
    float f[3];
    const int4 key = cic_key(F, l, ic, fc, s, i0, f);
    if (!same_key(key, lc.neg[0]) && !same_key(key, lc.neg[lc.stride])) break;
    --l;
  }
  return l;
}

// The same for TSC (Eq. 9): the neighbourhood of level l is the 27 cells around the point's
// level-l cell, keyed by that cell (as tsc_gather_cached keys its rows).
__device__ __forceinline__ int tsc_first_level(const DevField& F, int l, const int* ic, int s, const LaneCache& lc) {
  while (l > 0) {
    const int sh = F.L - l;
    const int4 key = make_int4((l << 8) | s, ic[0] >> sh, ic[1] >> sh, ic[2] >> sh);
    if (!same_key(key, lc.neg[0]) && !same_key(key, lc.neg[lc.stride])) break;
    --l;
  }
  return l;
}

// CIC at level l (FP32) from finest-level integer coordinates; v as in cic_gather.  With
// WithD, dv[d][q] also receives the derivative of the interpolant of component q with respect
// to the level-l cell coordinate d (the weights' derivatives, +-1 times the other two weights).
// i0_out, f_out (if non-null) receive the lower corner and the in-cell fractions of the neighbourhood.
// A neighbourhood found incomplete (false) is remembered in lc.neg when the lane has one.
// rows_out, rows_ok (if non-null): when this call staged the neighbourhood, the rows of its 8 cells
// and true (a call that reuses the staged neighbourhood leaves them as they were).
// Compact: the miss path looks the rows up out of line and the corner loop stays rolled (the same
// arithmetic in fewer instructions, for kernels whose hot loop outgrows the instruction cache).
template <bool WithD = false, bool Compact = false>
__device__ __forceinline__ bool cic_int_cached(const DevField& F, int l, const int* ic, const float* fc, int s,
                                               float* v, unsigned* err, const LaneCache& lc,
                                               float (*dv)[8] = nullptr, int* i0_out = nullptr,
                                               float* f_out = nullptr, unsigned* rows_out = nullptr,
                                               bool* rows_ok = nullptr) {
  int i0[3];
  float f[3];
  const int4 key = cic_key(F, l, ic, fc, s, i0, f);
  if (i0_out) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      i0_out[d] = i0[d];
      f_out[d] = f[d];
    }
  }
  const int4 old = *lc.key;
  const bool hit = same_key(old, key);
  // the miss path rejoins before the gather (no early exit from inside it): the lanes that staged a
  // new neighbourhood and those that reuse theirs then run the weights and the gather together
  bool ok = true;
  if (!hit) {
    const long long i0l[3] = {i0[0], i0[1], i0[2]};
    unsigned rows[8];
    if constexpr (Compact) {
      ok = cic_rows_compact(F, l, i0l, rows, err);
    } else {
      ok = cic_rows(F, l, i0l, rows, err);
    }
    if (ok) {
      const float4* rec = (const float4*)F.rec[l];
      const int S = F.S;
      const int s1 = (S > 1) ? s + 1 : s;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float4* rc = rec + (size_t)rows[c] * (size_t)S;
        lc.rec[(2 * c) * lc.stride] = __ldg(rc + s);
        lc.rec[(2 * c + 1) * lc.stride] = __ldg(rc + s1);
      }
      *lc.key = key;
      if (rows_out) {
#pragma unroll
        for (int c = 0; c < 8; ++c) rows_out[c] = rows[c];
        *rows_ok = true;
      }
    } else if (lc.neg) {
      lc.neg[lc.stride] = lc.neg[0];
      lc.neg[0] = key;
    }
  }
  if (!ok) return false;
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = 0.0f;
  if constexpr (WithD) {
#pragma unroll
    for (int q = 0; q < 8; ++q) dv[0][q] = dv[1][q] = dv[2][q] = 0.0f;
  }
#pragma unroll(Compact ? 1 : 8)
  for (int c = 0; c < 8; ++c) {
    const float wx = (c & 1) ? f[0] : 1.0f - f[0];
    const float wy = (c & 2) ? f[1] : 1.0f - f[1];
    const float wz = (c & 4) ? f[2] : 1.0f - f[2];
    const float w = wx * wy * wz;
    const float4 r0 = lc.rec[(2 * c) * lc.stride];
    const float4 r1 = lc.rec[(2 * c + 1) * lc.stride];
    v[0] += w * r0.x;
    v[1] += w * r0.y;
    v[2] += w * r0.z;
    v[3] += w * r0.w;
    v[4] += w * r1.x;
    v[5] += w * r1.y;
    v[6] += w * r1.z;
    v[7] += w * r1.w;
    if constexpr (WithD) {
      const float dw[3] = {((c & 1) ? 1.0f : -1.0f) * wy * wz, ((c & 2) ? 1.0f : -1.0f) * wx * wz,
                           ((c & 4) ? 1.0f : -1.0f) * wx * wy};
      const float rr[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int q = 0; q < 8; ++q) dv[d][q] += dw[d] * rr[q];
    }
  }
  return true;
}

// CIC at level l (FP32) from finest-level integer coordinates; v as in cic_gather.
__device__ __forceinline__ bool cic_int(const DevField& F, int l, const int* ic, const float* fc, int s, float* v,
                                        unsigned* err) {
  const int sh = F.L - l;
  const float inv = 1.0f / (float)(1 << sh);
  long long i0[3];
  float f[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int ilev = ic[d] >> sh;
    const float fl = ((float)(ic[d] & ((1 << sh) - 1)) + fc[d]) * inv;  // fraction in the level-l cell
    if (fl >= 0.5f) {
      i0[d] = ilev;
      f[d] = fl - 0.5f;
    } else {
      i0[d] = (long long)ilev - 1;
      f[d] = fl + 0.5f;
    }
  }
  const float w[3][2] = {{1.0f - f[0], f[0]}, {1.0f - f[1], f[1]}, {1.0f - f[2], f[2]}};
  return cic_gather<float>(F, l, i0, w, s, v, err);
}

// TSC (Eq. 9) at level l around cell c with the lane's neighbour cache: the rows of the 27 cells
// around c (the same for every position inside c) are kept in the lane cache's record area, keyed by
// (level, slice bracket, c), and reused while the photon stays in that cell, so the octet probes and
// the Morton arithmetic run only when it enters another cell (the neighbour caching of the paper's
// TSC mode, Sect. 2.2); the 27 x 2 records are read at every stage.  v, dout as tsc_gather.
template <bool WithD>
__device__ __forceinline__ bool tsc_gather_cached(const DevField& F, int l, const long long* c, const float* t, int s,
                                                  float* out, unsigned* err, const LaneCache& lc,
                                                  float (*dout)[8] = nullptr) {
  // the lane's 27 rows, interleaved with the other lanes' at 4-byte granularity over the record
  // area (every kernel sets lc.rec = block base + threadIdx.x float4s, stride = threads per block):
  // rows[m * stride], m = mx + 3 my + 9 mz, within the area's 64 x stride words
  unsigned* rows = reinterpret_cast<unsigned*>(lc.rec - threadIdx.x) + threadIdx.x;
  const int4 key = make_int4((l << 8) | s, (int)c[0], (int)c[1], (int)c[2]);
  const int4 old = *lc.key;
  if (!(old.x == key.x && old.y == key.y && old.z == key.z && old.w == key.w)) {
    unsigned a[3][3], plo[3], oct[8];
    if (!tsc_octets(F, l, c, a, plo, oct, err)) {
      if (lc.neg) {
        lc.neg[lc.stride] = lc.neg[0];
        lc.neg[0] = key;
      }
      return false;
    }
#pragma unroll 1
    for (int mz = 0; mz < 3; ++mz)
#pragma unroll 1
      for (int my = 0; my < 3; ++my)
#pragma unroll
        for (int mx = 0; mx < 3; ++mx) rows[(mx + 3 * my + 9 * mz) * lc.stride] = tsc_row(l, a, plo, oct, mx, my, mz);
    *lc.key = key;
  }
  float w[3][3], dw[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d) tsc_weights<float>(t[d], w[d], WithD ? dw[d] : nullptr);
  const float4* rec = (const float4*)F.rec[l];
  const int S = F.S;
  const int s1 = (S > 1) ? s + 1 : s;
#pragma unroll
  for (int q = 0; q < 8; ++q) out[q] = 0.0f;
  if constexpr (WithD) {
#pragma unroll
    for (int q = 0; q < 8; ++q) dout[0][q] = dout[1][q] = dout[2][q] = 0.0f;
  }
#pragma unroll 1
  for (int mz = 0; mz < 3; ++mz) {
#pragma unroll 1
    for (int my = 0; my < 3; ++my) {
#pragma unroll
      for (int mx = 0; mx < 3; ++mx) {
        const float4* rc = rec + (size_t)rows[(mx + 3 * my + 9 * mz) * lc.stride] * (size_t)S;
        const float4 r0 = __ldg(rc + s), r1 = __ldg(rc + s1);
        const float rr[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
        const float wgt = w[0][mx] * w[1][my] * w[2][mz];
#pragma unroll
        for (int q = 0; q < 8; ++q) out[q] += wgt * rr[q];
        if constexpr (WithD) {
          const float wyz = w[1][my] * w[2][mz];
          const float d0 = dw[0][mx] * wyz, d1 = w[0][mx] * dw[1][my] * w[2][mz], d2 = w[0][mx] * w[1][my] * dw[2][mz];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            dout[0][q] += d0 * rr[q];
            dout[1][q] += d1 * rr[q];
            dout[2][q] += d2 * rr[q];
          }
        }
      }
    }
  }
  return true;
}

// NGP or TSC (Eqs. 7, 9) at level l (FP32) from finest-level integer coordinates: the level-l
// cell is ic >> (L - l) and t the position in it relative to its centre; v (and dv with WithD)
// as in cic_int_cached.  TSC with a lane cache keeps the cell's 27 neighbour rows
// (tsc_gather_cached).
template <bool WithD, int IP>
__device__ __forceinline__ bool interp_int(const DevField& F, int l, const int* ic, const float* fc, int s, float* v,
                                           unsigned* err, float (*dv)[8] = nullptr, const LaneCache* lc = nullptr) {
  const int sh = F.L - l;
  const float inv = 1.0f / (float)(1 << sh);
  long long c[3];
  float t[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    c[d] = ic[d] >> sh;
    t[d] = ((float)(ic[d] & ((1 << sh) - 1)) + fc[d]) * inv - 0.5f;
  }
  if constexpr (IP == MT_INTERP_NGP) {
    if constexpr (WithD) {
#pragma unroll
      for (int q = 0; q < 8; ++q) dv[0][q] = dv[1][q] = dv[2][q] = 0.0f;
    }
    return ngp_gather<float>(F, l, c, s, v, err);
  }
  if (lc) return tsc_gather_cached<WithD>(F, l, c, t, s, v, err, *lc, WithD ? dv : nullptr);
  return tsc_gather<float>(F, l, c, t, s, v, err, WithD ? dv : nullptr);
}

// Most refined level containing the finest cell ic: the coarse refinement bitmap answers
// level 1 (a 4-byte load from a small, cache-resident array), hash probes the deeper levels.
__device__ __forceinline__ int locate_level_int(const DevField& F, const int* ic, unsigned* err,
                                                const LaneCache* lc = nullptr) {
  if (F.L == 0) return 0;
  if (lc && lc->loc) {
    // the answer depends only on the cell of the level found (it exists and, refined levels holding
    // whole octets, has no children): reuse it while the point stays in that cell
    const int4 c = *lc->loc;
    if (c.w >= 0) {
      const int sh = F.L - c.w;
      if ((ic[0] >> sh) == c.x && (ic[1] >> sh) == c.y && (ic[2] >> sh) == c.z) return c.w;
    }
  }
  const unsigned sh0 = (unsigned)F.L;
  const unsigned long long crow = morton((unsigned)ic[0] >> sh0, (unsigned)ic[1] >> sh0, (unsigned)ic[2] >> sh0);
  int lf = 0;
  if ((__ldg(&F.refbits[crow >> 5]) >> (crow & 31ull)) & 1u) {
    lf = 1;
    for (int l = 2; l <= F.L; ++l) {
      const int sh = F.L - l + 1;
      const unsigned long long pk = morton((unsigned)ic[0] >> sh, (unsigned)ic[1] >> sh, (unsigned)ic[2] >> sh);
      if (hash_find(F.hash[l], pk, err) < 0) break;
      lf = l;
    }
  }
  if (lc && lc->loc) {
    const int sh = F.L - lf;
    *lc->loc = make_int4(ic[0] >> sh, ic[1] >> sh, ic[2] >> sh, lf);
  }
  return lf;
}

struct MixedStep {
  int ib[3];
  float fb[3];
  int jb;        // background node of the step start
  float tb;      // fractional node coordinate of the step start
  int sb;        // slice bracket at the step start
  float e_lo;    // eta_step - eta_{sb}
  float e_hi;    // eta_step - eta_{sb+1}
};

// What the tangent of the right-hand side needs at a stage (FP32): the interpolated force and
// phi_eta, D = d phi / d lambda of Eq. (4), H, and their derivatives.
struct StageF {
  float g[3], pe, D, H, dH;
  float G[3][3];  // G[i][d] = d g_i / d x_d (derivative of the trilinear interpolant)
  float ge[3];    // d g_i / d eta (slope between the bracketing slices)
  float dpe[3];   // d phi_eta / d x_d
  // the CIC neighbourhood the stage interpolated from (CIC only): level, slice bracket, lower
  // corner, in-cell fractions, slice weight and 1 / (eta_{s+1} - eta_s) (0 with one slice)
  int lev, sl;
  int i0[3];
  float f[3];
  float wt, ids;
  // the rows of the 8 cells, when the stage staged the neighbourhood (rows_ok; CIC only)
  unsigned rows[8];
  bool rows_ok;
};

// FP32 right-hand side of Eqs. (2)-(4) at the stage with offsets (offx, offe) from the step
// start and wave vector (k0, k).  *lf (if non-null) receives the most refined level.  With
// WithD (which needs the lane cache) *sf receives the stage's field values and derivatives.
template <bool WithD = false, int IP = MT_INTERP_CIC, bool Compact = false>
__device__ __forceinline__ bool rhs_mixed(const DevField& F, bool grav, const MixedStep& B, double eta_step,
                                          const float* offx, float offe, float k0, const float* k, float* Kk0,
                                          float* Kk, float* KI, float* Ks, int* lf, unsigned* err,
                                          const LaneCache* lc, StageF* sf = nullptr) {
  // background H(eta_step + offe)
  const float t = B.tb + offe * F.bg_inv_deta_f;
  const float ct = floorf(t);
  int j = B.jb + (int)ct;
  float ft = t - ct;
  if (j < 0) {
    ft += (float)j;
    j = 0;
  } else if (j > F.bg_n - 2) {
    ft += (float)(j - (F.bg_n - 2));
    j = F.bg_n - 2;
  }
  const float4 p = __ldg(&F.bgf[j]);
  const float t2 = ft * ft, t3 = t2 * ft;
  const float H = (2.0f * t3 - 3.0f * t2 + 1.0f) * p.x + (t3 - 2.0f * t2 + ft) * p.y + (-2.0f * t3 + 3.0f * t2) * p.z +
                  (t3 - t2) * p.w;
  float phi = 0.0f, g0 = 0.0f, g1 = 0.0f, g2 = 0.0f, pe = 0.0f;
  if constexpr (WithD) {
    sf->H = H;
    sf->dH = ((6.0f * t2 - 6.0f * ft) * p.x + (3.0f * t2 - 4.0f * ft + 1.0f) * p.y + (6.0f * ft - 6.0f * t2) * p.z +
              (3.0f * t2 - 2.0f * ft) * p.w) *
             F.bg_inv_deta_f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      sf->ge[i] = sf->dpe[i] = 0.0f;
#pragma unroll
      for (int d = 0; d < 3; ++d) sf->G[i][d] = 0.0f;
    }
  }
  if (grav || lf) {
    int ic[3];
    float fc[3];
    if (!stage_coords(F, B.ib, B.fb, offx, ic, fc)) return false;
    const int lfin = locate_level_int(F, ic, err, lc);
    if (lf) *lf = lfin;
    if (grav) {
      int s = B.sb;
      float es = B.e_lo;  // eta_stage - eta_s = es + offe
      if (F.S > 1) {
        const bool below = (s > 0) && (B.e_lo + offe < 0.0f);
        const bool above = (s < F.S - 2) && (B.e_hi + offe >= 0.0f);
        if (below || above) {  // the stage left the step's slice bracket (rare): re-bracket in FP64
          const double e = eta_step + (double)offe;
          s = 0;
          while (s < F.S - 2 && F.seta[s + 1] <= e) ++s;
          es = (float)(eta_step - F.seta[s]);
        }
      }
      float v[8];
      float dv[WithD ? 3 : 1][8];
      int l = lfin;
      if constexpr (IP != MT_INTERP_CIC) {
        if constexpr (IP == MT_INTERP_TSC) {
          if (lc && lc->neg) l = tsc_first_level(F, l, ic, s, *lc);
        }
        for (; l >= 0; --l)
          if (interp_int<WithD, IP>(F, l, ic, fc, s, v, err, WithD ? dv : nullptr, lc)) break;
      } else if constexpr (WithD) {
        if (lc->neg) l = cic_first_level(F, l, ic, fc, s, *lc);
        sf->rows_ok = false;
        for (; l >= 0; --l)
          if (cic_int_cached<true, Compact>(F, l, ic, fc, s, v, err, *lc, dv, sf->i0, sf->f, sf->rows,
                                            &sf->rows_ok))
            break;
      } else if (lc) {
        if (lc->neg) l = cic_first_level(F, l, ic, fc, s, *lc);
        for (; l >= 0; --l)
          if (cic_int_cached<false, Compact>(F, l, ic, fc, s, v, err, *lc)) break;
      } else {
        for (; l >= 0; --l)
          if (cic_int(F, l, ic, fc, s, v, err)) break;
      }
      if (l < 0) return false;
      if (F.S == 1) {
        phi = v[0];
        g0 = v[1];
        g1 = v[2];
        g2 = v[3];
      } else {
        const float ids = F.inv_dseta[s];
        const float w = (es + offe) * ids;
        phi = v[0] + w * (v[4] - v[0]);
        g0 = v[1] + w * (v[5] - v[1]);
        g1 = v[2] + w * (v[6] - v[2]);
        g2 = v[3] + w * (v[7] - v[3]);
        pe = (v[4] - v[0]) * ids;
      }
      if constexpr (WithD) {
        sf->lev = l;
        sf->sl = s;
        sf->wt = F.S > 1 ? (es + offe) * F.inv_dseta[s] : 0.0f;
        sf->ids = F.S > 1 ? F.inv_dseta[s] : 0.0f;
        const float inv = F.inv_dxf_f / (float)(1 << (F.L - l));  // d (level-l cell coordinate) / d x
        if (F.S == 1) {
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int d = 0; d < 3; ++d) sf->G[i][d] = dv[d][1 + i] * inv;
        } else {
          const float ids = F.inv_dseta[s];
          const float w = (es + offe) * ids;
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            sf->ge[i] = (v[5 + i] - v[1 + i]) * ids;
#pragma unroll
            for (int d = 0; d < 3; ++d) sf->G[i][d] = (dv[d][1 + i] + w * (dv[d][5 + i] - dv[d][1 + i])) * inv;
            sf->dpe[i] = (dv[i][4] - dv[i][0]) * ids * inv;
          }
        }
      }
    }
  }
  (void)phi;
  const float dphidl = g0 * k[0] + g1 * k[1] + g2 * k[2] + pe * k0;
  if constexpr (WithD) {
    sf->g[0] = g0;
    sf->g[1] = g1;
    sf->g[2] = g2;
    sf->pe = pe;
    sf->D = dphidl;
  }
  const float k00 = k0 * k0;
  const float bg = -2.0f * H * k0;
  *Kk0 = bg * k0 - 2.0f * dphidl * k0 + 2.0f * pe * k00;
  Kk[0] = bg * k[0] + 2.0f * dphidl * k[0] - 2.0f * g0 * k00;
  Kk[1] = bg * k[1] + 2.0f * dphidl * k[1] - 2.0f * g1 * k00;
  Kk[2] = bg * k[2] + 2.0f * dphidl * k[2] - 2.0f * g2 * k00;
  *KI = -pe * k0;
  *Ks = sqrtf(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
  return true;
}

// Step-start quantities of a mixed step: finest-level base cell and fraction, background node
// and slice bracket of eta.  The node and bracket come from the FP32 offset e = eta - eta_0 of the
// table start (one FP64 subtraction): its rounding (~1e-7 e) moves H(eta) and the slice weight
// by far less than the FP32 interpolation itself.  False when the position is outside a
// non-periodic domain.
__device__ __forceinline__ bool mixed_begin(const DevField& F, const double* y, MixedStep& B) {
  if (!finest_base(F, y, B.ib, B.fb)) return false;
  const float e = (float)(y[3] - F.bg_eta0);
  const float t0 = e * F.bg_inv_deta_f;
  const float jf = floorf(t0);
  B.jb = (int)jf;
  B.tb = t0 - jf;
  int s = 0;
  while (s < F.S - 2 && F.seta_rel_f[s + 1] <= e) ++s;
  B.sb = s;
  B.e_lo = e - F.seta_rel_f[s];
  B.e_hi = F.S > 1 ? e - F.seta_rel_f[s + 1] : 0.0f;
  return true;
}

// Stage data of one mixed step that its reverse needs (Record instances of ray_step_mixed): the
// wave-vector offsets (k0, k) of the 4 stages from the step start, their right-hand sides
// (dk0, dk)/dlambda, the step size and whether the step was the last.
constexpr int kStepRecordFloats = 34;  // [0, 16) offsets, [16, 32) right-hand sides, 32: h, 33: last

// One mixed-precision RK4 step; state and status conventions as ray_step.  Record: if rec is not
// null it receives the step's stage data (kStepRecordFloats floats).  Compact: the CIC in the
// compact form of cic_int_cached (same results).
template <int IP = MT_INTERP_CIC, bool Record = false, bool Compact = false, class RayStateT, class TraceArgsT>
__device__ bool ray_step_mixed(const DevField& F, const TraceArgsT& A, RayStateT& r, unsigned* err,
                               const LaneCache* lc = nullptr, float* rec = nullptr) {
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
  // stage offsets (from the step start) and weighted sums of the stage derivatives
  float offx[3] = {0.0f, 0.0f, 0.0f}, offe = 0.0f, offk0 = 0.0f, offk[3] = {0.0f, 0.0f, 0.0f};
  float sx[3] = {0.0f, 0.0f, 0.0f}, se = 0.0f, sk0 = 0.0f, sk[3] = {0.0f, 0.0f, 0.0f}, sI = 0.0f, ss = 0.0f;
  float h = 0.0f;
  bool last = false;
#pragma unroll 1
  for (int st = 0; st < 4; ++st) {
    const float kst0 = k0s + offk0;
    const float kst[3] = {ks[0] + offk[0], ks[1] + offk[1], ks[2] + offk[2]};
    float Kk0, Kk[3], KI, Ks;
    int lf = 0;
    if (!rhs_mixed<false, IP, Compact>(F, grav, B, eta, offx, offe, kst0, kst, &Kk0, Kk, &KI, &Ks,
                                       st == 0 ? &lf : nullptr, err, lc)) {
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
    }
    if constexpr (Record) {
      if (rec) {
        rec[4 * st] = offk0;
        rec[4 * st + 1] = offk[0];
        rec[4 * st + 2] = offk[1];
        rec[4 * st + 3] = offk[2];
        rec[16 + 4 * st] = Kk0;
        rec[16 + 4 * st + 1] = Kk[0];
        rec[16 + 4 * st + 2] = Kk[1];
        rec[16 + 4 * st + 3] = Kk[2];
      }
    }
    const float b = (st == 0 || st == 3) ? (1.0f / 6.0f) : (1.0f / 3.0f);
    sk0 += b * Kk0;
    sk[0] += b * Kk[0];
    sk[1] += b * Kk[1];
    sk[2] += b * Kk[2];
    sI += b * KI;
    ss += b * Ks;
    se += b * offk0;
    sx[0] += b * offk[0];
    sx[1] += b * offk[1];
    sx[2] += b * offk[2];
    const float c = (st == 2 ? 1.0f : 0.5f) * h;  // next stage at y + c K
    offx[0] = c * kst[0];
    offx[1] = c * kst[1];
    offx[2] = c * kst[2];
    offe = c * kst0;
    offk0 = c * Kk0;
    offk[0] = c * Kk[0];
    offk[1] = c * Kk[1];
    offk[2] = c * Kk[2];
  }
  if constexpr (Record) {
    if (rec) {
      rec[32] = h;
      rec[33] = last ? 1.0f : 0.0f;
    }
  }
  const double hd = (double)h;
  bool finite = true;
  // positions and eta: h k(step start) in FP64 plus the FP32 stage corrections
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
  // the state stays finite while every FP32 increment does (the FP64 sums cannot overflow at
  // these magnitudes): one FP32 test instead of ten FP64 ones
  finite = isfinite(h + sx[0] + sx[1] + sx[2] + se + sk0 + sk[0] + sk[1] + sk[2] + sI + ss);
  r.lambda += hd;
  r.n_steps += 1;
  if (!finite) {
    r.status = MT_RAY_NONFINITE;
    return true;
  }
  return last;
}

}  // namespace mt
