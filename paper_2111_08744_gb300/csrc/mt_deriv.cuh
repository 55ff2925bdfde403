// Derivatives of the interpolated field and of the background, shared by the tangent and
// adjoint kernels (Sect. 2.3 distortion matrix, gradients with respect to the gridded phi).
#pragma once

#include "mt_trace_device.cuh"

namespace mt {

// Hermite H(eta) and its derivative dH/deta (the interpolant of bg_eval).
__device__ __forceinline__ void bg_eval_d(const DevField& F, double eta, double* H, double* dH) {
  dvec4 p, q;
  bg_interval(F, eta, &p, &q);
  const double d = q.x - p.x;
  const double t = (eta - p.x) / d;
  const double t2 = t * t, t3 = t2 * t;
  *H = (2.0 * t3 - 3.0 * t2 + 1.0) * p.z + (t3 - 2.0 * t2 + t) * d * p.w + (-2.0 * t3 + 3.0 * t2) * q.z +
       (t3 - t2) * d * q.w;
  *dH = ((6.0 * t2 - 6.0 * t) * p.z + (3.0 * t2 - 4.0 * t + 1.0) * d * p.w + (-6.0 * t2 + 6.0 * t) * q.z +
         (3.0 * t2 - 2.0 * t) * d * q.w) /
        d;
}

struct FieldD {
  double g[3];      // grad phi
  double pe;        // d phi / d eta
  double G[3][3];   // G[i][d] = d g_i / d x_d (derivative of the trilinear interpolant)
  double ge[3];     // d g_i / d eta (slope between slices)
  double dpe[3];    // d pe / d x_d
};

// CIC with level fallback (as sample_field) that also returns the spatial derivatives of the
// trilinear interpolant.
template <class T, int IP = MT_INTERP_CIC>
__device__ __forceinline__ bool sample_field_d(const DevField& F, const double* x, double eta, FieldD* fd, int* lf, unsigned* err) {
  using V = typename Vec4<T>::type;
  double u[3];
  if (!coarse_coords<T>(F, x, u)) return false;
  const int lfin = locate_level(F, u, err);
  *lf = lfin;
  int s = 0;
  while (s < F.S - 2 && F.seta[s + 1] <= eta) ++s;
  const int s1 = F.S > 1 ? s + 1 : s;
  double v[8], dv[3][8];
  int l = lfin;
  const int ip = IP >= 0 ? IP : F.interp;
  for (; l >= 0; --l) {
    const double sc = (double)(1ll << l);
    if (ip != MT_INTERP_CIC) {  // NGP (piecewise constant: zero spatial derivative) or TSC
      long long c[3];
      double t[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double U = u[d] * sc;
        const double fl = floor(U);
        c[d] = (long long)fl;
        t[d] = U - fl - 0.5;
      }
      if (ip == MT_INTERP_NGP) {
        if (!ngp_gather<T, double>(F, l, c, s, v, err)) continue;
#pragma unroll
        for (int q = 0; q < 8; ++q) dv[0][q] = dv[1][q] = dv[2][q] = 0.0;
      } else if (!tsc_gather<T, double>(F, l, c, t, s, v, err, dv)) {
        continue;
      }
      break;
    }
    long long i0[3];
    double f[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double U = u[d] * sc - 0.5;
      const double fl = floor(U);
      i0[d] = (long long)fl;
      f[d] = U - fl;
    }
    unsigned rows[8];
    if (!cic_rows(F, l, i0, rows, err)) continue;
    const V* rec = (const V*)F.rec[l];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      v[q] = 0.0;
      dv[0][q] = dv[1][q] = dv[2][q] = 0.0;
    }
    for (int c = 0; c < 8; ++c) {
      const double wx = (c & 1) ? f[0] : 1.0 - f[0], sx = (c & 1) ? 1.0 : -1.0;
      const double wy = (c & 2) ? f[1] : 1.0 - f[1], sy = (c & 2) ? 1.0 : -1.0;
      const double wz = (c & 4) ? f[2] : 1.0 - f[2], sz = (c & 4) ? 1.0 : -1.0;
      const double w = wx * wy * wz;
      const double dw[3] = {sx * wy * wz, wx * sy * wz, wx * wy * sz};
      const V* rc = rec + (size_t)rows[c] * (size_t)F.S;
      const V r0 = ldg4(rc + s), r1 = ldg4(rc + s1);
      const double rr[8] = {(double)r0.x, (double)r0.y, (double)r0.z, (double)r0.w,
                            (double)r1.x, (double)r1.y, (double)r1.z, (double)r1.w};
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        v[q] += w * rr[q];
        dv[0][q] += dw[0] * rr[q];
        dv[1][q] += dw[1] * rr[q];
        dv[2][q] += dw[2] * rr[q];
      }
    }
    break;
  }
  if (l < 0) return false;
  const double inv_dx = (double)(1ll << l) / F.dx0;  // d f / d x
  if (F.S == 1) {
    for (int i = 0; i < 3; ++i) {
      fd->g[i] = v[1 + i];
      fd->ge[i] = 0.0;
      fd->dpe[i] = 0.0;
      for (int d = 0; d < 3; ++d) fd->G[i][d] = dv[d][1 + i] * inv_dx;
    }
    fd->pe = 0.0;
    return true;
  }
  const double de = F.seta[s + 1] - F.seta[s];
  const double wt = (eta - F.seta[s]) / de;
  for (int i = 0; i < 3; ++i) {
    fd->g[i] = v[1 + i] + wt * (v[5 + i] - v[1 + i]);
    fd->ge[i] = (v[5 + i] - v[1 + i]) / de;
    for (int d = 0; d < 3; ++d) fd->G[i][d] = (dv[d][1 + i] + wt * (dv[d][5 + i] - dv[d][1 + i])) * inv_dx;
    fd->dpe[i] = (dv[i][4] - dv[i][0]) / de * inv_dx;
  }
  fd->pe = (v[4] - v[0]) / de;
  return true;
}

}  // namespace mt
