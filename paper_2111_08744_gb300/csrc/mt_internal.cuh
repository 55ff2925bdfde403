// Device-side data layout and helpers of the GB300 ray tracer (sm_103a).
//
// Octree (Sect. 2.1, flattened AMR with a binary cell index):
//   * level 0: dense N_0^3 record array in Morton order, indexed directly by key;
//   * level l >= 1: whole octets, records in key order (octet o holds rows 8o..8o+7,
//     child c = key & 7), plus an open-addressing hash  parent key -> octet index.
//     A CIC neighbourhood at level l spans 1, 2, 4 or 8 octets, so one hash probe
//     serves up to 8 corner cells.
// Records: [count][S] of dvec4 (FP64 field) or float4 (FP32 field) holding
//   phi, dphi/dx, dphi/dy, dphi/dz per slice; the two bracketing slices of a cell
//   are adjacent in memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mt.h"

namespace mt {

constexpr int kMaxLevels = MT_MAX_LEVELS;
constexpr int kMaxSlices = MT_MAX_SLICES;
constexpr int kMaxCones = MT_MAX_CONES;
constexpr unsigned long long kEmptyKey = ~0ull;
constexpr unsigned long long kHashMul = 0x9E3779B97F4A7C15ull;  // Fibonacci hashing (Knuth)

enum : unsigned { kErrOOB = 1u, kErrTimeout = 2u, kErrTree = 4u };

// 4 doubles, 16-byte aligned (records and background nodes)
struct alignas(16) dvec4 {
  double x, y, z, w;
};

struct HashTable {
  const ulonglong2* slots;  // {key, octet index}; empty slots hold kEmptyKey
  unsigned long long mask;  // capacity - 1 (capacity a power of two)
  int shift;                // 64 - log2(capacity)
  int pad;
};

struct DevField {
  const void* rec[kMaxLevels + 1];
  HashTable hash[kMaxLevels + 1];  // [0] unused
  double box;
  double dx0;       // box / N_0
  double inv_dx0;   // N_0 / box (mixed path only)
  int nc;           // N_0
  int L;            // refined levels
  int periodic;
  int S;            // slices
  double seta[kMaxSlices];
  const dvec4* bg;  // (eta, a, H, dH/deta) nodes, uniform in eta
  int bg_n;
  int interp;       // MT_INTERP_CIC / NGP / TSC (set per launch from the trace parameters)
  double bg_eta0, bg_deta, bg_inv_deta;
  double eta_o;     // observer time = last background node
  // mixed-precision path: finest-level integer coordinates and single-precision tables
  const float4* bgf;  // per node j: H_j, deta H'_j, H_{j+1}, deta H'_{j+1}
  double inv_dxf;     // N_L / box (finest level cells per unit length)
  int nf;             // N_L = N_0 2^L
  float inv_dxf_f;    // N_L / box
  float dx0_f;        // dx_0
  float bg_inv_deta_f;
  float inv_dseta[kMaxSlices];  // 1 / (eta_{s+1} - eta_s)
  float seta_rel_f[kMaxSlices]; // eta_s - bg_eta0 (the mixed step's slice bracket)
  const unsigned* refbits;      // one bit per coarse cell (Morton order): has children on level 1
};

struct DevCones {
  int n;
  int pad;
  long long begin[kMaxCones + 1];
  double obs[kMaxCones][3];
  double eta_stop[kMaxCones];
};

// ----------------------------------------------------------------- Morton keys

__host__ __device__ __forceinline__ unsigned long long spread_bits3(unsigned long long v) {
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

__host__ __device__ __forceinline__ unsigned long long morton(unsigned i, unsigned j, unsigned k) {
  return spread_bits3(i) | (spread_bits3(j) << 1) | (spread_bits3(k) << 2);
}

// ----------------------------------------------------------------- hash

__device__ __forceinline__ long long hash_find(const HashTable& t, unsigned long long key, unsigned* err) {
  unsigned long long h = (key * kHashMul) >> t.shift;
  for (unsigned long long probe = 0; probe <= t.mask; ++probe) {
    ulonglong2 s = __ldg(&t.slots[h]);
    if (s.x == key) return (long long)s.y;
    if (s.x == kEmptyKey) return -1;
    h = (h + 1) & t.mask;
  }
  atomicOr(err, kErrOOB);  // a table with no empty slot: cannot happen at load <= 1/2
  return -1;
}

// ----------------------------------------------------------------- read-only vector loads

__device__ __forceinline__ dvec4 ldg4(const dvec4* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  const double2 a = __ldg(q), b = __ldg(q + 1);
  return dvec4{a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }

// ----------------------------------------------------------------- background (Sect. 2.2 tables)

// Node interval of the background table holding eta: eta_j <= eta < eta_{j+1}, clamped to the
// table's first and last intervals.  The uniform spacing gives the guess; a guess one node off (eta
// within rounding of a node) is corrected against the nodes themselves.  *p, *q: nodes j, j + 1.
__device__ __forceinline__ int bg_interval(const DevField& F, double eta, dvec4* p, dvec4* q) {
  double jf = floor((eta - F.bg_eta0) * F.bg_inv_deta);
  jf = fmin(fmax(jf, 0.0), (double)(F.bg_n - 2));
  int j = (int)jf;
  *p = ldg4(&F.bg[j]);
  *q = ldg4(&F.bg[j + 1]);
  if (j > 0 && eta < p->x) {
    --j;
    *q = *p;
    *p = ldg4(&F.bg[j]);
  } else if (j < F.bg_n - 2 && !(eta < q->x)) {
    ++j;
    *p = *q;
    *q = ldg4(&F.bg[j + 1]);
  }
  return j;
}

// Cubic Hermite interpolation of a(eta) (slopes a H) and H(eta) (slopes dH/deta) on the node
// interval holding eta, t = (eta - eta_j) / (eta_{j+1} - eta_j).
__device__ __forceinline__ void bg_eval(const DevField& F, double eta, double* a, double* H) {
  dvec4 p, q;
  bg_interval(F, eta, &p, &q);
  const double d = q.x - p.x;
  const double t = (eta - p.x) / d;
  const double t2 = t * t, t3 = t2 * t;
  const double h00 = 2.0 * t3 - 3.0 * t2 + 1.0;
  const double h10 = t3 - 2.0 * t2 + t;
  const double h01 = -2.0 * t3 + 3.0 * t2;
  const double h11 = t3 - t2;
  if (a) *a = h00 * p.y + h10 * d * (p.y * p.z) + h01 * q.y + h11 * d * (q.y * q.z);
  if (H) *H = h00 * p.z + h10 * d * p.w + h01 * q.z + h11 * d * q.w;
}

// ----------------------------------------------------------------- field sampling

template <class T>
struct Vec4;
template <>
struct Vec4<double> {
  using type = dvec4;
};
template <>
struct Vec4<float> {
  using type = float4;
};

// Coarse-cell coordinates u = x / dx_0 (IEEE division in the FP64 path, a reciprocal
// multiply in the mixed path), wrapped into [0, N_0) when periodic.  Returns false when
// the point is outside a non-periodic box.
template <class T>
__device__ __forceinline__ bool coarse_coords(const DevField& F, const double* x, double* u) {
  const double nc = (double)F.nc;
  bool inside = true;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double v = (sizeof(T) == 8) ? x[d] / F.dx0 : x[d] * F.inv_dx0;
    if (F.periodic) {
      v = v - nc * floor(v * (1.0 / nc));
    } else {
      inside = inside && (v >= 0.0) && (v < nc);
    }
    u[d] = v;
  }
  return inside;
}

// Most refined level whose cell contains the point (Sect. 2.2 step 1): level l + 1
// exists there iff the level-l cell containing it has children (one hash probe).
__device__ __forceinline__ int locate_level(const DevField& F, const double* u, unsigned* err) {
  int lf = 0;
  const unsigned nc = (unsigned)F.nc;
  for (int l = 1; l <= F.L; ++l) {
    const double s = (double)(1u << (l - 1));
    const unsigned m = (nc << (l - 1)) - 1u;
    unsigned c0 = (unsigned)(long long)floor(u[0] * s) & m;
    unsigned c1 = (unsigned)(long long)floor(u[1] * s) & m;
    unsigned c2 = (unsigned)(long long)floor(u[2] * s) & m;
    if (hash_find(F.hash[l], morton(c0, c1, c2), err) < 0) break;
    lf = l;
  }
  return lf;
}

// Rows of the 8 CIC neighbours at level l around lower corner i0 (unwrapped level-l indices),
// corner c = (c & 1, (c >> 1) & 1, (c >> 2) & 1).  Returns false if a neighbour is absent.
// Row indices fit 32 bits (level-0 rows < 2^31, octets < 2^28); addresses are formed in 64 bits.
__device__ __forceinline__ bool cic_rows(const DevField& F, int l, const long long* i0, unsigned* rows,
                                         unsigned* err) {
  const long long Nl = (long long)F.nc << l;
  // wrapped corner coordinates a[d][c] for c = 0, 1
  unsigned a[3][2];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      long long v = i0[d] + c;
      if (F.periodic) {
        v &= (Nl - 1);
      } else if (v < 0 || v >= Nl) {
        return false;
      }
      a[d][c] = (unsigned)v;
    }
  }
  if (l == 0) {
#pragma unroll
    for (int c = 0; c < 8; ++c) rows[c] = (unsigned)morton(a[0][c & 1], a[1][(c >> 1) & 1], a[2][(c >> 2) & 1]);
    return true;
  }
  // parents of the two corners per axis coincide iff the lower corner index is even
  const int ox = (int)(i0[0] & 1), oy = (int)(i0[1] & 1), oz = (int)(i0[2] & 1);
  unsigned oct[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int qx = q & 1, qy = (q >> 1) & 1, qz = (q >> 2) & 1;
    if ((qx && !ox) || (qy && !oy) || (qz && !oz)) {
      oct[q] = 0u;
      continue;
    }
    const unsigned long long pk = morton(a[0][qx] >> 1, a[1][qy] >> 1, a[2][qz] >> 1);
    const long long o = hash_find(F.hash[l], pk, err);
    if (o < 0) return false;
    oct[q] = (unsigned)o;
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
    const int q = (ox ? cx : 0) | ((oy ? cy : 0) << 1) | ((oz ? cz : 0) << 2);
    const unsigned child = (a[0][cx] & 1u) | ((a[1][cy] & 1u) << 1) | ((a[2][cz] & 1u) << 2);
    rows[c] = oct[q] * 8u + child;
  }
  return true;
}

// The rows of cic_rows with the corner and octet loops kept rolled: the same lookups in about a
// tenth of the instructions, out of line, for kernels whose hot loop outgrows the instruction
// cache (one Morton key and one probe loop in the code instead of eight of each).
static __device__ __noinline__ bool cic_rows_compact(const DevField& F, int l, const long long* i0, unsigned* rows,
                                                     unsigned* err) {
  const long long Nl = (long long)F.nc << l;
  unsigned a0[3], a1[3];  // wrapped coordinates of the lower and upper corners per axis
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    long long v0 = i0[d], v1 = i0[d] + 1;
    if (F.periodic) {
      v0 &= (Nl - 1);
      v1 &= (Nl - 1);
    } else if (v0 < 0 || v1 >= Nl) {
      return false;
    }
    a0[d] = (unsigned)v0;
    a1[d] = (unsigned)v1;
  }
  if (l == 0) {
#pragma unroll 1
    for (int c = 0; c < 8; ++c)
      rows[c] = (unsigned)morton((c & 1) ? a1[0] : a0[0], (c & 2) ? a1[1] : a0[1], (c & 4) ? a1[2] : a0[2]);
    return true;
  }
  // parents of the two corners per axis coincide iff the lower corner index is even
  const int ox = (int)(i0[0] & 1), oy = (int)(i0[1] & 1), oz = (int)(i0[2] & 1);
  unsigned oct[8];
#pragma unroll 1
  for (int q = 0; q < 8; ++q) {
    const int qx = q & 1, qy = (q >> 1) & 1, qz = (q >> 2) & 1;
    if ((qx && !ox) || (qy && !oy) || (qz && !oz)) continue;
    const unsigned long long pk = morton((qx ? a1[0] : a0[0]) >> 1, (qy ? a1[1] : a0[1]) >> 1, (qz ? a1[2] : a0[2]) >> 1);
    const long long o = hash_find(F.hash[l], pk, err);
    if (o < 0) return false;
    oct[q] = (unsigned)o;
  }
#pragma unroll 1
  for (int c = 0; c < 8; ++c) {
    const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
    const int q = (ox ? cx : 0) | ((oy ? cy : 0) << 1) | ((oz ? cz : 0) << 2);
    const unsigned child = ((cx ? a1[0] : a0[0]) & 1u) | (((cy ? a1[1] : a0[1]) & 1u) << 1) |
                           (((cz ? a1[2] : a0[2]) & 1u) << 2);
    rows[c] = oct[q] * 8u + child;
  }
  return true;
}

// CIC (Eq. 8) gather at level l around lower corner i0, for the two bracketing slices s, s+1 (or
// slice 0 when S = 1): out[0..3] at slice s, out[4..7] at slice s+1.  w[d][b]: the weight along axis
// d of the corner i0_d + b; corner c weighs w[0][c & 1] w[1][c >> 1 & 1] w[2][c >> 2 & 1].  Returns
// false if a neighbour is absent.
template <class T>
__device__ __forceinline__ bool cic_gather(const DevField& F, int l, const long long* i0, const T (*w)[2], int s,
                                          T* out, unsigned* err) {
  using V = typename Vec4<T>::type;
  unsigned rows[8];
  if (!cic_rows(F, l, i0, rows, err)) return false;
  const V* rec = (const V*)F.rec[l];
  const int S = F.S;
  const int s1 = (S > 1) ? s + 1 : s;
#pragma unroll
  for (int q = 0; q < 8; ++q) out[q] = (T)0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const T wc = w[0][c & 1] * w[1][(c >> 1) & 1] * w[2][(c >> 2) & 1];
    const V* rc = rec + (size_t)rows[c] * (size_t)S;
    const V r0 = ldg4(rc + s);
    const V r1 = ldg4(rc + s1);
    out[0] += wc * r0.x;
    out[1] += wc * r0.y;
    out[2] += wc * r0.z;
    out[3] += wc * r0.w;
    out[4] += wc * r1.x;
    out[5] += wc * r1.y;
    out[6] += wc * r1.z;
    out[7] += wc * r1.w;
  }
  return true;
}

// CIC at level l from coarse-cell coordinates u: U = u 2^l, lower corner i0 = floor(U - 1/2), and
// the weights of Eq. (8) as defined, W = 1 - |r| with r = U - (centre of the corner cell).
template <class T>
__device__ __forceinline__ bool cic_level(const DevField& F, int l, const double* u, int s, T* out, unsigned* err) {
  const double sc = (double)(1ll << l);
  long long i0[3];
  T w[3][2];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double U = u[d] * sc;
    const double fl = floor(U - 0.5);
    i0[d] = (long long)fl;
    w[d][0] = (T)(1.0 - fabs(U - (fl + 0.5)));
    w[d][1] = (T)(1.0 - fabs(U - (fl + 1.5)));
  }
  return cic_gather<T>(F, l, i0, (const T(*)[2])w, s, out, err);
}

// ----------------------------------------------------------------- NGP and TSC (Eqs. 7, 9)

// The parent octets of the 3 x 3 x 3 cells around cell c of level l >= 1: along each axis
// the three cells c-1, c, c+1 have exactly two distinct parents, so 8 probes cover the 27
// cells.  a[d][m] receives the wrapped coordinate of cell c + m - 1, oct[q] the octet of
// parent (q & 1, q >> 1 & 1, q >> 2) (lower or upper parent per axis).  False when one of the
// cells is outside a non-periodic domain or its octet is absent.
__device__ __forceinline__ bool tsc_octets(const DevField& F, int l, const long long* c, unsigned (*a)[3],
                                           unsigned* plo, unsigned* oct, unsigned* err) {
  const long long Nl = (long long)F.nc << l;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      long long v = c[d] + m - 1;
      if (F.periodic) {
        v &= (Nl - 1);
      } else if (v < 0 || v >= Nl) {
        return false;
      }
      a[d][m] = (unsigned)v;
    }
    plo[d] = a[d][0] >> 1;
  }
  if (l == 0) return true;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const unsigned px = (q & 1) ? a[0][2] >> 1 : plo[0];
    const unsigned py = (q & 2) ? a[1][2] >> 1 : plo[1];
    const unsigned pz = (q & 4) ? a[2][2] >> 1 : plo[2];
    const long long o = hash_find(F.hash[l], morton(px, py, pz), err);
    if (o < 0) return false;
    oct[q] = (unsigned)o;
  }
  return true;
}

// Row of cell (mx, my, mz) in {0,1,2}^3 of the neighbourhood described by tsc_octets.
__device__ __forceinline__ unsigned tsc_row(int l, const unsigned (*a)[3], const unsigned* plo, const unsigned* oct,
                                            int mx, int my, int mz) {
  const unsigned x = a[0][mx], y = a[1][my], z = a[2][mz];
  if (l == 0) return (unsigned)morton(x, y, z);
  const int q = ((x >> 1) != plo[0] ? 1 : 0) | ((y >> 1) != plo[1] ? 2 : 0) | ((z >> 1) != plo[2] ? 4 : 0);
  return oct[q] * 8u + ((x & 1u) | ((y & 1u) << 1) | ((z & 1u) << 2));
}

// TSC weights of Eq. (9) for the cells c-1, c, c+1 along one axis, t = U - c - 1/2 in [-1/2, 1/2)
// (distances 1 + t, t, 1 - t from their centres); dw: derivatives with respect to U.
template <class T>
__device__ __forceinline__ void tsc_weights(T t, T* w, T* dw) {
  const T lo = (T)0.5 - t, hi = (T)0.5 + t;
  w[0] = (T)0.5 * lo * lo;
  w[1] = (T)0.75 - t * t;
  w[2] = (T)0.5 * hi * hi;
  if (dw) {
    dw[0] = -lo;
    dw[1] = (T)-2 * t;
    dw[2] = hi;
  }
}

// TSC gather at level l around cell c (t as in tsc_weights), slices s, s+1 as cic_gather; with
// dout, dout[d][q] receives the derivative with respect to the level-l coordinate d.  R: record
// precision, T: arithmetic.
// wdef (if non-null): the weights along each axis, given (then t is not used and dout must be null).
template <class R, class T = R>
__device__ __forceinline__ bool tsc_gather(const DevField& F, int l, const long long* c, const T* t, int s, T* out,
                                          unsigned* err, T (*dout)[8] = nullptr, const T (*wdef)[3] = nullptr) {
  using V = typename Vec4<R>::type;
  unsigned a[3][3], plo[3], oct[8];
  if (!tsc_octets(F, l, c, a, plo, oct, err)) return false;
  T w[3][3], dw[3][3];
  if (wdef) {
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int m = 0; m < 3; ++m) w[d][m] = wdef[d][m];
  } else {
#pragma unroll
    for (int d = 0; d < 3; ++d) tsc_weights<T>(t[d], w[d], dout ? dw[d] : nullptr);
  }
  const V* rec = (const V*)F.rec[l];
  const int S = F.S;
  const int s1 = (S > 1) ? s + 1 : s;
#pragma unroll
  for (int q = 0; q < 8; ++q) out[q] = (T)0;
  if (dout) {
#pragma unroll
    for (int q = 0; q < 8; ++q) dout[0][q] = dout[1][q] = dout[2][q] = (T)0;
  }
#pragma unroll 1
  for (int mz = 0; mz < 3; ++mz) {
#pragma unroll 1
    for (int my = 0; my < 3; ++my) {
#pragma unroll
      for (int mx = 0; mx < 3; ++mx) {
        const V* rc = rec + (size_t)tsc_row(l, a, plo, oct, mx, my, mz) * (size_t)S;
        const V r0 = ldg4(rc + s), r1 = ldg4(rc + s1);
        const T rr[8] = {(T)r0.x, (T)r0.y, (T)r0.z, (T)r0.w, (T)r1.x, (T)r1.y, (T)r1.z, (T)r1.w};
        const T wgt = w[0][mx] * w[1][my] * w[2][mz];
#pragma unroll
        for (int q = 0; q < 8; ++q) out[q] += wgt * rr[q];
        if (dout) {
          const T wyz = w[1][my] * w[2][mz];
          const T d0 = dw[0][mx] * wyz, d1 = w[0][mx] * dw[1][my] * w[2][mz], d2 = w[0][mx] * w[1][my] * dw[2][mz];
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

// NGP (Eq. 7): the records of cell c of level l (slices s, s+1 as cic_gather).
template <class R, class T = R>
__device__ __forceinline__ bool ngp_gather(const DevField& F, int l, const long long* c, int s, T* out, unsigned* err) {
  using V = typename Vec4<R>::type;
  const long long Nl = (long long)F.nc << l;
  unsigned v[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    long long x = c[d];
    if (F.periodic) {
      x &= (Nl - 1);
    } else if (x < 0 || x >= Nl) {
      return false;
    }
    v[d] = (unsigned)x;
  }
  unsigned long long row;
  if (l == 0) {
    row = morton(v[0], v[1], v[2]);
  } else {
    const long long o = hash_find(F.hash[l], morton(v[0] >> 1, v[1] >> 1, v[2] >> 1), err);
    if (o < 0) return false;
    row = (unsigned long long)o * 8ull + ((v[0] & 1u) | ((v[1] & 1u) << 1) | ((v[2] & 1u) << 2));
  }
  const V* rc = (const V*)F.rec[l] + (size_t)row * (size_t)F.S;
  const V r0 = ldg4(rc + s), r1 = ldg4(rc + ((F.S > 1) ? s + 1 : s));
  out[0] = (T)r0.x;
  out[1] = (T)r0.y;
  out[2] = (T)r0.z;
  out[3] = (T)r0.w;
  out[4] = (T)r1.x;
  out[5] = (T)r1.y;
  out[6] = (T)r1.z;
  out[7] = (T)r1.w;
  return true;
}

// Interpolation scheme of a code path: MT_INTERP_* fixed at compile time (the per-step code of
// the kernels is instantiated per scheme, so CIC carries no TSC registers), or kInterpRuntime to
// read DevField::interp (the once-per-ray observer and end-point samples).
constexpr int kInterpRuntime = -1;

// The interpolation scheme at level l from coarse-cell coordinates u.
template <class T, int IP = MT_INTERP_CIC>
__device__ __forceinline__ bool interp_level(const DevField& F, int l, const double* u, int s, T* out, unsigned* err) {
  const int ip = IP >= 0 ? IP : F.interp;
  if (ip == MT_INTERP_CIC) return cic_level<T>(F, l, u, s, out, err);
  const double sc = (double)(1ll << l);
  long long c[3];
  T t[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double U = u[d] * sc;
    const double fl = floor(U);
    c[d] = (long long)fl;
    t[d] = (T)(U - fl - 0.5);
  }
  if (ip == MT_INTERP_NGP) return ngp_gather<T>(F, l, c, s, out, err);
  // the weights of Eq. (9) as defined, W(r) with r = U - (centre of the cell c + m - 1)
  T wdef[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double U = u[d] * sc;
    const double fl = (double)c[d];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const double r = U - ((fl + (double)(m - 1)) + 0.5);
      const double a = fabs(r);
      wdef[d][m] = (T)(a < 0.5 ? 0.75 - r * r : (a < 1.5 ? 0.5 * (1.5 - a) * (1.5 - a) : 0.0));
    }
  }
  return tsc_gather<T, T>(F, l, c, t, s, out, err, nullptr, (const T(*)[3])wdef);
}

// Field at (x, eta): phi, grad phi and d phi/d eta, with the level fallback of Sect. 2.2
// (start at the most refined level containing the photon; while one of the cells the scheme
// needs -- 8 for CIC, 27 for TSC -- is missing, retry one level coarser; NGP takes the
// containing cell).  Time: linear in eta between the
// bracketing slices, extended linearly outside them.  *lf receives the most refined
// level.  Returns false when the point is outside a non-periodic domain.
template <class T, int IP = MT_INTERP_CIC>
__device__ __forceinline__ bool sample_field(const DevField& F, const double* x, double eta, T* phi, T* g, T* pe,
                                             int* lf, unsigned* err) {
  double u[3];
  if (!coarse_coords<T>(F, x, u)) return false;
  const int lfin = locate_level(F, u, err);
  *lf = lfin;
  int s = 0;
  while (s < F.S - 2 && F.seta[s + 1] <= eta) ++s;
  T v[8];
  int l = lfin;
  for (; l >= 0; --l)
    if (interp_level<T, IP>(F, l, u, s, v, err)) break;
  if (l < 0) return false;
  if (F.S == 1) {
    *phi = v[0];
    g[0] = v[1];
    g[1] = v[2];
    g[2] = v[3];
    *pe = (T)0;
    return true;
  }
  const double de = F.seta[s + 1] - F.seta[s];
  const T w = (T)((eta - F.seta[s]) / de);
  *phi = v[0] + w * (v[4] - v[0]);
  g[0] = v[1] + w * (v[5] - v[1]);
  g[1] = v[2] + w * (v[6] - v[2]);
  g[2] = v[3] + w * (v[7] - v[3]);
  *pe = (v[4] - v[0]) / (T)de;
  return true;
}

}  // namespace mt

// Library handle (host side).
struct mt_octree {
  int device;
  int precision;
  int n_levels;
  int n_slices;
  mt::DevField f;
  void* rec_alloc[mt::kMaxLevels + 1];
  ulonglong2* hash_alloc[mt::kMaxLevels + 1];
  unsigned long long* octkey[mt::kMaxLevels + 1];  // parent key of every octet of a refined level
  unsigned* refbits;                               // coarse-cell refinement bitmap
  int64_t count[mt::kMaxLevels + 1];
  double* bg_dev;
  float4* bgf_dev;
  double* bg_host;
  int bg_n;
  unsigned long long* ws;  // [0] ray queue counter, [1] error flags
  int64_t device_bytes;
  int num_sms;
  int launch_block;  // trace kernel threads per block (0: default 128)
  int launch_bps;    // trace kernel blocks per SM (0: as many as fit)
  int ray_chunk;     // trace kernel: ray ids a warp claims per refill (0: default 32)
  int staging;       // trace kernel, FP32 field, CIC: 0/1 per-lane shared-memory neighbourhood, 2 direct loads
};

namespace mt {
double host_eta_stop(const mt_octree* t, double z);
void host_bg_eval(const double* tab, int n, double eta, double* a, double* H);
}  // namespace mt
