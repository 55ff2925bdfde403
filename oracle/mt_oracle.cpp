// FP64 CPU oracle of the null-geodesic ray tracer (arXiv 2111.08744, Sect. 2.2-2.5).
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
// benchmark's CPU-baseline leg may load this library; the product path (the
// CUDA library and its Python binding) never does and shares no code with it.
//
// Plain, slow, obviously correct: every stage of every RK4 step re-derives the
// cell indices from the position, looks each cell up by binary search in the
// level's sorted key vector (the paper's sorted-vector octree, Sect. 3.1), and
// evaluates the weights of Eq. (8) (CIC; or Eq. 7, NGP, or Eq. 9, TSC) cell by cell.  Compiled with
// -ffp-contract=off so every operation is a single IEEE-754 double operation.
//
// Conventions (c = 1, lengths and eta in h^-1 Mpc, phi = Phi/c^2):
//   * state y = (x[3], eta, k0, k[3], I, s), affine parameter lambda;
//   * rays start at the observer with k0 = -1 (past-directed, so eta decreases
//     while lambda increases; Eqs. (2)-(3) are invariant under k -> -k) and
//     k^i = n sqrt((1 + 2 phi_o)/(1 - 2 phi_o)) (null condition of Eq. (1));
//   * coarse cell coordinates u = x / dx_0 (IEEE division), wrapped into
//     [0, N_c) by u - N_c floor(u / N_c) when periodic; level-l coordinates are
//     u 2^l (exact);
//   * a step uses h = dx_l / (N |k0|) with l the most refined level whose cell
//     contains the photon at the step start (Sect. 2.2, "N steps per AMR cell");
//   * the last step is shortened so that eta lands on eta_stop (iso-eta stop).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

extern "C" {

struct orc_grid {
  double box;
  int32_t n_coarse;
  int32_t n_levels;      // refined levels; level indices 0..n_levels
  int32_t periodic;
  int32_t n_slices;
  const double* slice_eta;  // [n_slices], ascending
};

struct orc_level {
  const uint64_t* keys;     // [count], ascending Morton keys (x bit 0, y bit 1, z bit 2)
  const double* records;    // [count][n_slices][4]: phi, dphi/dx, dphi/dy, dphi/dz
  int64_t count;
};

struct orc_params {
  int32_t n_cones;
  int32_t steps_per_cell;
  int32_t gravity_on;
  int32_t interp;           // 0: CIC, 1: NGP, 2: TSC (Sect. 2.2 weighting functions)
  const double* observer;   // [n_cones][3]
  const double* z_max;      // [n_cones]
  const int64_t* ray_begin; // [n_cones + 1]
  int64_t max_steps;
};

struct orc_out {
  double* x;        // [3][N] end position (unwrapped)
  double* k;        // [4][N] end k0, k1, k2, k3
  double* eta;      // [N]
  double* lambda;   // [N]
  double* chi;      // [N] |x_s - x_o|
  double* path;     // [N] integral of |k| d lambda
  double* z0;       // [N] Eq. (23)
  double* z1;       // [N] Eq. (24)
  double* z4;       // [N] Eq. (27) with v = 0
  double* z5;       // [N] Eq. (28) with v = 0
  double* d_a;      // [N] a_s chi
  double* d_l;      // [N] (1 + z5)^2 d_a
  double* phi_o;    // [N]
  double* phi_s;    // [N]
  double* isw;      // [N] int phi_eta d eta from eta_s to eta_o
  int32_t* n_steps; // [N]
  int32_t* level;   // [N] most refined level containing the end point
  int32_t* status;  // [N] 0 ok, 1 left domain, 2 max steps, 3 non-finite
  double* tie;      // [N] smallest margin of any index decision along the ray (cell units for
                    //     locate/CIC floors, relative for the stop test); NULL to skip
};

}  // extern "C"

namespace {

enum { ST_OK = 0, ST_LEFT = 1, ST_MAXSTEPS = 2, ST_NONFINITE = 3 };

uint64_t morton_key(int64_t i, int64_t j, int64_t k) {
  uint64_t key = 0;
  for (int b = 0; b < 21; ++b) {
    key |= ((uint64_t)((i >> b) & 1)) << (3 * b);
    key |= ((uint64_t)((j >> b) & 1)) << (3 * b + 1);
    key |= ((uint64_t)((k >> b) & 1)) << (3 * b + 2);
  }
  return key;
}

// Background a(eta) and H(eta) = a'/a from the tabulated nodes (eta, a, H, dH/deta):
// cubic Hermite interpolation with slopes a' = a H and H' (Sect. 2.2, "external
// pre-computed tables").
struct Background {
  const double* tab;
  int n;
  int bracket(double eta) const {
    // j with eta_j <= eta < eta_{j+1}, clamped to [0, n-2]
    int lo = 0, hi = n - 1;
    if (eta <= tab[0]) return 0;
    if (eta >= tab[4 * (n - 1)]) return n - 2;
    while (hi - lo > 1) {
      int mid = (lo + hi) / 2;
      if (tab[4 * mid] <= eta) lo = mid; else hi = mid;
    }
    return lo;
  }
  void eval(double eta, double* a, double* H) const {
    int j = bracket(eta);
    const double* p = tab + 4 * j;
    const double* q = p + 4;
    double d = q[0] - p[0];
    double t = (eta - p[0]) / d;
    double t2 = t * t, t3 = t2 * t;
    double h00 = 2.0 * t3 - 3.0 * t2 + 1.0;
    double h10 = t3 - 2.0 * t2 + t;
    double h01 = -2.0 * t3 + 3.0 * t2;
    double h11 = t3 - t2;
    if (a) *a = h00 * p[1] + h10 * d * (p[1] * p[2]) + h01 * q[1] + h11 * d * (q[1] * q[2]);
    if (H) *H = h00 * p[2] + h10 * d * p[3] + h01 * q[2] + h11 * d * q[3];
  }
  double a_of(double eta) const { double a; eval(eta, &a, nullptr); return a; }
  // eta at which a(eta) = 1/(1+z), by bisection on the interpolant (monotone in eta)
  double eta_stop(double z) const {
    double target = 1.0 / (1.0 + z);
    double lo = tab[0], hi = tab[4 * (n - 1)];
    if (target >= a_of(hi)) return hi;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (lo + hi);
      if (mid == lo || mid == hi) break;
      if (a_of(mid) < target) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
  }
};

enum { INTERP_CIC = 0, INTERP_NGP = 1, INTERP_TSC = 2 };

struct Field {
  double box;
  int nc, L, S;
  int interp = INTERP_CIC;
  bool periodic;
  const double* seta;
  const orc_level* lv;
  // analytic potential phi = A sin(k . x), static (test mode: (A, k_x, k_y, k_z), k a multiple of
  // 2 pi / box per axis so that it is periodic); NULL: the octree's records
  const double* analytic = nullptr;

  int64_t n_at(int l) const { return (int64_t)nc << l; }
  double dx(int l) const { return box / (double)n_at(l); }

  // coarse-unit coordinates of x (wrapped when periodic)
  void coarse_coords(const double* x, double* u) const {
    for (int d = 0; d < 3; ++d) {
      double v = x[d] / dx(0);
      if (periodic) v = v - (double)nc * std::floor(v / (double)nc);
      u[d] = v;
    }
  }
  // row of cell (i, j, k) at level l, or -1 when absent (binary search, Sect. 3.1)
  int64_t find(int l, int64_t i, int64_t j, int64_t k) const {
    int64_t n = n_at(l);
    if (periodic) {
      i = ((i % n) + n) % n; j = ((j % n) + n) % n; k = ((k % n) + n) % n;
    } else if (i < 0 || j < 0 || k < 0 || i >= n || j >= n || k >= n) {
      return -1;
    }
    uint64_t key = morton_key(i, j, k);
    const uint64_t* b = lv[l].keys;
    const uint64_t* e = b + lv[l].count;
    const uint64_t* p = std::lower_bound(b, e, key);
    if (p == e || *p != key) return -1;
    return (int64_t)(p - b);
  }
  // distance of v to the nearest integer: how close a floor() decision came to a tie
  static void note_tie(double v, double* tie) {
    if (!tie) return;
    double r = std::fabs(v - std::nearbyint(v));
    if (r < *tie) *tie = r;
  }
  // most refined level whose cell contains the point (-1: outside the domain)
  int finest(const double* u, double* tie = nullptr) const {
    int best = -1;
    for (int l = 0; l <= L; ++l) {
      double s = std::ldexp(1.0, l);
      int64_t c[3];
      for (int d = 0; d < 3; ++d) { c[d] = (int64_t)std::floor(u[d] * s); note_tie(u[d] * s, tie); }
      if (find(l, c[0], c[1], c[2]) < 0) break;
      best = l;
    }
    return best;
  }
  // CIC (Eq. 8) of the 4 record components at slice s, level l; false when a neighbour is absent.
  bool cic_level(int l, const double* u, double (*vals)[4], double* tie = nullptr) const {
    double s = std::ldexp(1.0, l);
    double U[3];
    int64_t i0[3];
    for (int d = 0; d < 3; ++d) {
      U[d] = u[d] * s;
      i0[d] = (int64_t)std::floor(U[d] - 0.5);
      note_tie(U[d] - 0.5, tie);
    }
    int64_t rows[8];
    for (int c = 0; c < 8; ++c) {
      rows[c] = find(l, i0[0] + (c & 1), i0[1] + ((c >> 1) & 1), i0[2] + ((c >> 2) & 1));
      if (rows[c] < 0) return false;
    }
    for (int sl = 0; sl < S; ++sl)
      for (int q = 0; q < 4; ++q) vals[sl][q] = 0.0;
    for (int c = 0; c < 8; ++c) {
      double w = 1.0;
      for (int d = 0; d < 3; ++d) {
        double centre = (double)(i0[d] + ((c >> d) & 1)) + 0.5;
        double r = U[d] - centre;
        w = w * (1.0 - std::fabs(r));   // W_CIC(r) = 1 - |r| for |r| < 1
      }
      const double* rec = lv[l].records + (size_t)rows[c] * (size_t)S * 4;
      for (int sl = 0; sl < S; ++sl)
        for (int q = 0; q < 4; ++q) vals[sl][q] += w * rec[sl * 4 + q];
    }
    return true;
  }
  // NGP (Eq. 7, Sect. 2.2): the records of the level-l cell containing the point.
  bool ngp_level(int l, const double* u, double (*vals)[4]) const {
    double s = std::ldexp(1.0, l);
    int64_t c[3];
    for (int d = 0; d < 3; ++d) c[d] = (int64_t)std::floor(u[d] * s);
    int64_t row = find(l, c[0], c[1], c[2]);
    if (row < 0) return false;
    const double* rec = lv[l].records + (size_t)row * (size_t)S * 4;
    for (int sl = 0; sl < S; ++sl)
      for (int q = 0; q < 4; ++q) vals[sl][q] = rec[sl * 4 + q];
    return true;
  }
  // W_TSC, Eq. (9): 3/4 - r^2 for |r| < 1/2, (3/2 - |r|)^2 / 2 for 1/2 <= |r| < 3/2, else 0
  static double w_tsc(double r) {
    double a = std::fabs(r);
    if (a < 0.5) return 0.75 - r * r;
    if (a < 1.5) return 0.5 * (1.5 - a) * (1.5 - a);
    return 0.0;
  }
  // TSC at level l: the cell containing the point and its 26 neighbours (27 cells, the same
  // for every position inside that cell); false when one of them is absent.
  bool tsc_level(int l, const double* u, double (*vals)[4], double* tie = nullptr) const {
    double s = std::ldexp(1.0, l);
    double U[3];
    int64_t c[3];
    for (int d = 0; d < 3; ++d) {
      U[d] = u[d] * s;
      c[d] = (int64_t)std::floor(U[d]);
      note_tie(U[d], tie);
    }
    int64_t rows[27];
    for (int m = 0; m < 27; ++m) {
      int o[3] = {m % 3 - 1, (m / 3) % 3 - 1, m / 9 - 1};
      rows[m] = find(l, c[0] + o[0], c[1] + o[1], c[2] + o[2]);
      if (rows[m] < 0) return false;
    }
    for (int sl = 0; sl < S; ++sl)
      for (int q = 0; q < 4; ++q) vals[sl][q] = 0.0;
    for (int m = 0; m < 27; ++m) {
      int o[3] = {m % 3 - 1, (m / 3) % 3 - 1, m / 9 - 1};
      double w = 1.0;
      for (int d = 0; d < 3; ++d) {
        double centre = (double)(c[d] + o[d]) + 0.5;
        w = w * w_tsc(U[d] - centre);
      }
      const double* rec = lv[l].records + (size_t)rows[m] * (size_t)S * 4;
      for (int sl = 0; sl < S; ++sl)
        for (int q = 0; q < 4; ++q) vals[sl][q] += w * rec[sl * 4 + q];
    }
    return true;
  }
  // Interpolated phi, grad phi and d phi/d eta at (u, eta), with the level fallback of
  // Sect. 2.2 (start at the most refined level containing the photon, go coarser while a
  // neighbour is missing; NGP takes the containing cell itself).  Time: linear in eta
  // between the bracketing slices.  Returns false when even level 0 lacks neighbours (edge
  // of a non-periodic domain).
  bool sample(const double* u, double eta, double* phi, double* grad, double* phi_eta, int* lev_used,
              double* tie = nullptr) const {
    int lf = finest(u, tie);
    if (lf < 0) return false;
    if (analytic) {
      // exact phi and grad phi at x = u dx_0 (the wrapped position; the field is periodic in the box)
      double arg = 0.0;
      for (int d = 0; d < 3; ++d) arg += analytic[1 + d] * (u[d] * dx(0));
      *phi = analytic[0] * std::sin(arg);
      for (int d = 0; d < 3; ++d) grad[d] = analytic[0] * analytic[1 + d] * std::cos(arg);
      *phi_eta = 0.0;
      if (lev_used) *lev_used = lf;
      return true;
    }
    double vals[64][4];
    int l = lf;
    for (; l >= 0; --l) {
      bool ok = interp == INTERP_NGP ? ngp_level(l, u, vals)
                : interp == INTERP_TSC ? tsc_level(l, u, vals, tie)
                                       : cic_level(l, u, vals, tie);
      if (ok) break;
    }
    if (l < 0) return false;
    if (lev_used) *lev_used = l;
    if (S == 1) {
      *phi = vals[0][0];
      for (int d = 0; d < 3; ++d) grad[d] = vals[0][1 + d];
      *phi_eta = 0.0;
      return true;
    }
    int s = 0;
    while (s < S - 2 && seta[s + 1] <= eta) ++s;
    double de = seta[s + 1] - seta[s];
    double w = (eta - seta[s]) / de;   // linear in eta; outside the slices: extended linearly
    *phi = vals[s][0] + w * (vals[s + 1][0] - vals[s][0]);
    for (int d = 0; d < 3; ++d) grad[d] = vals[s][1 + d] + w * (vals[s + 1][1 + d] - vals[s][1 + d]);
    *phi_eta = (vals[s + 1][0] - vals[s][0]) / de;
    return true;
  }
};

struct Tracer {
  Field f;
  Background bg;
  int N;          // steps per cell
  bool gravity;
  int64_t max_steps;

  // Right-hand side of Eqs. (2)-(3) with d phi/d lambda from the chain rule, Eq. (4).
  bool rhs(const double* y, double* dy, double* tie) const {
    const double* x = y;
    double eta = y[3], k0 = y[4];
    const double* k = y + 5;
    double a, H;
    bg.eval(eta, &a, &H);
    double phi = 0.0, g[3] = {0.0, 0.0, 0.0}, pe = 0.0;
    if (gravity) {
      double u[3];
      f.coarse_coords(x, u);
      if (!f.sample(u, eta, &phi, g, &pe, nullptr, tie)) return false;
    }
    double dphidl = g[0] * k[0] + g[1] * k[1] + g[2] * k[2] + pe * k0;
    dy[0] = k[0];
    dy[1] = k[1];
    dy[2] = k[2];
    dy[3] = k0;
    dy[4] = -2.0 * H * k0 * k0 - 2.0 * dphidl * k0 + 2.0 * pe * k0 * k0;
    for (int i = 0; i < 3; ++i)
      dy[5 + i] = -2.0 * H * k0 * k[i] + 2.0 * dphidl * k[i] - 2.0 * g[i] * k0 * k0;
    dy[8] = -pe * k0;
    dy[9] = std::sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
    return true;
  }

  // Infinitesimal-beam integrand at a point of the ray (Sect. 2.3.1): the Cartesian Hessian of
  // phi by Eq. (13), central differences of the interpolated grad phi with the step h = size of
  // the most refined cell containing the point (only i <= j is computed, d_i d_j = d_j d_i), then
  // its components on the screen of the photon's angular position (phi_a, theta_a) seen from the
  // observer, Eqs. (14)-(16), written for e_1 = e_phi and e_2 = -e_theta (the screen basis of the
  // finite beams, Eq. 21).  fo[0] = d1 d1 phi, fo[1] = d2 d2 phi, fo[2] = d1 d2 phi.  False if a
  // sample point lies outside a non-periodic domain.
  bool screen_hessian(const double* x, double eta, const double* xo, double* fo) const {
    double u[3];
    f.coarse_coords(x, u);
    int lf = f.finest(u);
    if (lf < 0) return false;
    double h = f.dx(lf);
    double H[3][3];
    for (int i = 0; i < 3; ++i) {
      double gp[3], gm[3], up[3], um[3], phi, pe;
      double xp[3] = {x[0], x[1], x[2]}, xm[3] = {x[0], x[1], x[2]};
      xp[i] += h;
      xm[i] -= h;
      f.coarse_coords(xp, up);
      f.coarse_coords(xm, um);
      if (!f.sample(up, eta, &phi, gp, &pe, nullptr)) return false;
      if (!f.sample(um, eta, &phi, gm, &pe, nullptr)) return false;
      for (int j = i; j < 3; ++j) H[i][j] = (gp[j] - gm[j]) / (2.0 * h);
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < i; ++j) H[i][j] = H[j][i];
    double v[3] = {x[0] - xo[0], x[1] - xo[1], x[2] - xo[2]};
    double rr = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double ph = std::atan2(v[1], v[0]);
    double th = std::acos(std::max(-1.0, std::min(1.0, v[2] / rr)));
    double sp = std::sin(ph), cp = std::cos(ph), st = std::sin(th), ct = std::cos(th);
    double Hxx = H[0][0], Hyy = H[1][1], Hzz = H[2][2], Hxy = H[0][1], Hxz = H[0][2], Hyz = H[1][2];
    fo[0] = sp * sp * Hxx + cp * cp * Hyy - 2.0 * sp * cp * Hxy;                                  // Eq. (14)
    fo[1] = cp * cp * ct * ct * Hxx + sp * sp * ct * ct * Hyy + st * st * Hzz + 2.0 * sp * cp * ct * ct * Hxy -
           2.0 * sp * st * ct * Hyz - 2.0 * cp * st * ct * Hxz;                                  // Eq. (15)
    fo[2] = -(ct * cp * sp * (Hyy - Hxx) + (cp * cp - sp * sp) * ct * Hxy + sp * st * Hxz - cp * st * Hyz);  // -Eq. (16)
    return true;
  }

  struct Result {
    double y[10];
    double lambda, phi_o, phi_s;
    int n_steps, level, status;
    double tie;
    double A[4];   // infinitesimal-beam distortion matrix (when requested): A11, A12, A21, A22
  };

  // Eq. (12) along the traced ray by the trapezoidal rule over its step points, split as
  // int chi f dchi - (1/chi_s) int chi^2 f dchi so that chi_s (known at the end) factors out.
  struct InfBeam {
    double I1[3] = {0, 0, 0}, I2[3] = {0, 0, 0};
    double prev_chi = 0.0, prev_f[3] = {0, 0, 0};
    void add(double chi, const double* f) {
      double dchi = chi - prev_chi;
      for (int c = 0; c < 3; ++c) {
        I1[c] += 0.5 * (prev_chi * prev_f[c] + chi * f[c]) * dchi;
        I2[c] += 0.5 * (prev_chi * prev_chi * prev_f[c] + chi * chi * f[c]) * dchi;
        prev_f[c] = f[c];
      }
      prev_chi = chi;
    }
    void matrix(double* A) const {
      double m[3];
      for (int c = 0; c < 3; ++c) m[c] = prev_chi > 0.0 ? I1[c] - I2[c] / prev_chi : 0.0;
      A[0] = 1.0 - 2.0 * m[0];
      A[1] = -2.0 * m[2];
      A[2] = -2.0 * m[2];
      A[3] = 1.0 - 2.0 * m[1];
    }
  };

  // chi_stop > 0: the iso-chi stop of the geodesic finder (Sect. 2.5): the ray steps as usual
  // until its comoving distance |x - x_o| reaches chi_stop, and the end point is then moved back
  // along k onto that sphere: x - t k with the smaller root t of |x - t k - x_o| = chi_stop (and
  // eta - t k0).  eta_stop then only bounds the integration.
  Result trace(const double* xo, const double* n, double eta_stop, bool inf_beam = false,
               double chi_stop = -1.0) const {
    Result r;
    InfBeam ib;
    double* y = r.y;
    double eta_o = bg.tab[4 * (bg.n - 1)];
    double phi_o = 0.0;
    if (gravity) {
      double u[3], g[3], pe;
      f.coarse_coords(xo, u);
      if (!f.sample(u, eta_o, &phi_o, g, &pe, nullptr)) phi_o = 0.0;
    }
    double kn = std::sqrt((1.0 + 2.0 * phi_o) / (1.0 - 2.0 * phi_o));
    for (int d = 0; d < 3; ++d) y[d] = xo[d];
    y[3] = eta_o;
    y[4] = -1.0;
    for (int d = 0; d < 3; ++d) y[5 + d] = n[d] * kn;
    y[8] = 0.0;
    y[9] = 0.0;
    r.lambda = 0.0;
    r.phi_o = phi_o;
    r.n_steps = 0;
    r.status = ST_OK;
    r.tie = 1.0;
    if (!(y[3] > eta_stop)) goto done;
    for (;;) {
      if (r.n_steps >= max_steps) { r.status = ST_MAXSTEPS; break; }
      double u[3];
      f.coarse_coords(y, u);
      // decisions at the observer itself are exact on any implementation: not tracked
      double* tie0 = r.n_steps > 0 ? &r.tie : nullptr;
      int lf = f.finest(u, tie0);
      if (lf < 0) { r.status = ST_LEFT; break; }
      double k0 = y[4];
      double h = f.dx(lf) / ((double)N * std::fabs(k0));
      bool last = false;
      {
        double m = std::fabs((y[3] + k0 * h) - eta_stop) / std::fabs(k0 * h);
        if (m < r.tie) r.tie = m;
      }
      if (y[3] + k0 * h <= eta_stop) { h = (eta_stop - y[3]) / k0; last = true; }
      // classical RK4
      double k1[10], k2[10], k3[10], k4[10], t[10];
      if (!rhs(y, k1, tie0)) { r.status = ST_LEFT; break; }
      for (int i = 0; i < 10; ++i) t[i] = y[i] + 0.5 * h * k1[i];
      if (!rhs(t, k2, &r.tie)) { r.status = ST_LEFT; break; }
      for (int i = 0; i < 10; ++i) t[i] = y[i] + 0.5 * h * k2[i];
      if (!rhs(t, k3, &r.tie)) { r.status = ST_LEFT; break; }
      for (int i = 0; i < 10; ++i) t[i] = y[i] + h * k3[i];
      if (!rhs(t, k4, &r.tie)) { r.status = ST_LEFT; break; }
      for (int i = 0; i < 10; ++i) y[i] = y[i] + (h / 6.0) * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
      r.lambda += h;
      r.n_steps += 1;
      bool finite = true;
      for (int i = 0; i < 10; ++i) finite = finite && std::isfinite(y[i]);
      if (!finite) { r.status = ST_NONFINITE; break; }
      if (inf_beam) {
        double fv[3] = {0.0, 0.0, 0.0};
        double d[3] = {y[0] - xo[0], y[1] - xo[1], y[2] - xo[2]};
        double chi = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (!screen_hessian(y, y[3], xo, fv)) fv[0] = fv[1] = fv[2] = 0.0;
        ib.add(chi, fv);
      }
      if (chi_stop > 0.0) {
        double d[3] = {y[0] - xo[0], y[1] - xo[1], y[2] - xo[2]};
        double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (dd >= chi_stop * chi_stop) {
          double kk = y[5] * y[5] + y[6] * y[6] + y[7] * y[7];
          double b = d[0] * y[5] + d[1] * y[6] + d[2] * y[7];
          double c = dd - chi_stop * chi_stop;
          double t = (b - std::sqrt(std::max(0.0, b * b - kk * c))) / kk;
          for (int q = 0; q < 3; ++q) y[q] -= t * y[5 + q];
          y[3] -= t * y[4];
          break;
        }
      }
      if (last) break;
    }
  done:
    ib.matrix(r.A);
    r.phi_s = 0.0;
    r.level = -1;
    {
      double u[3];
      f.coarse_coords(y, u);
      r.level = r.status == ST_NONFINITE ? -1 : f.finest(u, &r.tie);
      if (gravity && r.status != ST_NONFINITE) {
        double g[3], pe;
        if (!f.sample(u, y[3], &r.phi_s, g, &pe, nullptr)) r.phi_s = 0.0;
      }
    }
    return r;
  }
};

Tracer make_tracer(const orc_grid* g, const orc_level* lv, const double* bg, int bg_n, const orc_params* p) {
  Tracer t;
  t.f.box = g->box;
  t.f.nc = g->n_coarse;
  t.f.L = g->n_levels;
  t.f.S = g->n_slices;
  t.f.periodic = g->periodic != 0;
  t.f.seta = g->slice_eta;
  t.f.lv = lv;
  t.f.interp = p->interp;
  t.bg.tab = bg;
  t.bg.n = bg_n;
  t.N = p->steps_per_cell;
  t.gravity = p->gravity_on != 0;
  t.max_steps = p->max_steps;
  return t;
}

int cone_of(const orc_params* p, int64_t i) {
  int c = 0;
  while (c + 1 < p->n_cones && p->ray_begin[c + 1] <= i) ++c;
  return c;
}

template <class F>
void parallel_for(int64_t n, int n_threads, F fn) {
  if (n_threads <= 1) { for (int64_t i = 0; i < n; ++i) fn(i); return; }
  std::atomic<int64_t> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < n_threads; ++t)
    th.emplace_back([&]() {
      for (;;) {
        int64_t i = next.fetch_add(1);
        if (i >= n) break;
        fn(i);
      }
    });
  for (auto& x : th) x.join();
}

bool keys_sorted(const orc_grid* g, const orc_level* lv) {
  for (int l = 0; l <= g->n_levels; ++l)
    for (int64_t i = 1; i < lv[l].count; ++i)
      if (!(lv[l].keys[i - 1] < lv[l].keys[i])) return false;
  return true;
}

void xi_of(const double* y, double eta_stop, double* xi) {
  // end point moved along the ray onto the iso-eta surface eta = eta_stop
  for (int d = 0; d < 3; ++d) xi[d] = y[d] - (y[5 + d] / y[4]) * (y[3] - eta_stop);
}

}  // namespace

extern "C" {

double orc_eta_stop(const double* bg, int bg_n, double z) {
  Background b{bg, bg_n};
  return b.eta_stop(z);
}

void orc_background(const double* bg, int bg_n, const double* eta, int64_t n, double* a, double* H) {
  Background b{bg, bg_n};
  for (int64_t i = 0; i < n; ++i) b.eval(eta[i], a ? a + i : nullptr, H ? H + i : nullptr);
}

// Interpolated field at arbitrary points (tests of the lookup and of Eq. 8).
int orc_sample(const orc_grid* g, const orc_level* lv, const double* pts /*[3][n]*/, const double* eta, int64_t n,
               double* phi, double* grad /*[3][n]*/, double* phi_eta, int32_t* level_finest, int32_t* level_cic,
               int interp) {
  if (!keys_sorted(g, lv)) return 4;
  if (interp < INTERP_CIC || interp > INTERP_TSC) return 5;
  Field f;
  f.box = g->box; f.nc = g->n_coarse; f.L = g->n_levels; f.S = g->n_slices;
  f.periodic = g->periodic != 0; f.seta = g->slice_eta; f.lv = lv; f.interp = interp;
  for (int64_t i = 0; i < n; ++i) {
    double x[3] = {pts[i], pts[n + i], pts[2 * n + i]}, u[3], gr[3] = {0, 0, 0}, p = 0, pe = 0;
    f.coarse_coords(x, u);
    int lu = -1;
    level_finest[i] = f.finest(u);
    bool ok = f.sample(u, eta[i], &p, gr, &pe, &lu);
    level_cic[i] = ok ? lu : -1;
    phi[i] = p; phi_eta[i] = pe;
    for (int d = 0; d < 3; ++d) grad[d * n + i] = gr[d];
  }
  return 0;
}

static int trace_rays_impl(const orc_grid* g, const orc_level* lv, const double* bg, int bg_n, const orc_params* p,
                    const double* dirs /*[3][N]*/, int64_t n_rays, const double* chi_stop, orc_out* o,
                    int n_threads, const double* analytic = nullptr) {
  if (!keys_sorted(g, lv)) return 4;
  if (p->interp < INTERP_CIC || p->interp > INTERP_TSC) return 5;
  Tracer t = make_tracer(g, lv, bg, bg_n, p);
  t.f.analytic = analytic;
  std::vector<double> es(p->n_cones);
  for (int c = 0; c < p->n_cones; ++c) es[c] = chi_stop ? bg[0] : t.bg.eta_stop(p->z_max[c]);
  parallel_for(n_rays, n_threads, [&](int64_t i) {
    int c = cone_of(p, i);
    const double* xo = p->observer + 3 * c;
    double n[3] = {dirs[i], dirs[n_rays + i], dirs[2 * n_rays + i]};
    Tracer::Result r = t.trace(xo, n, es[c], false, chi_stop ? chi_stop[i] : -1.0);
    const double* y = r.y;
    double a_s = t.bg.a_of(y[3]);
    double dxo[3] = {y[0] - xo[0], y[1] - xo[1], y[2] - xo[2]};
    double chi = std::sqrt(dxo[0] * dxo[0] + dxo[1] * dxo[1] + dxo[2] * dxo[2]);
    for (int d = 0; d < 3; ++d) o->x[d * n_rays + i] = y[d];
    o->k[i] = y[4];
    for (int d = 0; d < 3; ++d) o->k[(1 + d) * n_rays + i] = y[5 + d];
    o->eta[i] = y[3];
    o->lambda[i] = r.lambda;
    o->chi[i] = chi;
    o->path[i] = y[9];
    double z0 = 1.0 / a_s - 1.0;                         // Eq. (23), a_0 = 1
    double z1 = z0 + (r.phi_o - r.phi_s) / a_s;          // Eq. (24)
    double z4 = z1 - 2.0 * y[8] / a_s;                   // Eq. (27), v = 0 so z3 = z2 = z1
    // Eq. (28) with g_{mu nu} k^mu u^nu = -a k0 (1 + phi), v = 0, a_o = 1, k0_o = -1
    double z5 = (a_s * std::fabs(y[4]) * (1.0 + r.phi_s)) / (1.0 * (1.0 + r.phi_o)) - 1.0;
    o->z0[i] = z0; o->z1[i] = z1; o->z4[i] = z4; o->z5[i] = z5;
    o->d_a[i] = a_s * chi;
    o->d_l[i] = (1.0 + z5) * (1.0 + z5) * a_s * chi;
    o->phi_o[i] = r.phi_o;
    o->phi_s[i] = r.phi_s;
    o->isw[i] = y[8];
    o->n_steps[i] = r.n_steps;
    o->level[i] = r.level;
    o->status[i] = r.status;
    if (o->tie) o->tie[i] = r.tie;
  });
  return 0;
}

// HEALPix pixel of direction v (Gorski et al. 2005, the sky pixelisation of Sect. 2.4), written
// through the HEALPix projection of the sphere onto the plane (Calabretta & Roukema 2007), in which
// every pixel boundary is a straight line at 45 degrees.  In units of pi/4:
//   equatorial zone |z| <= 2/3:  X = phi / (pi/4),  Y = 3 z / 2;
//   polar caps |z| > 2/3:        s = sqrt(3 (1 - |z|)),  X = X_c + (phi / (pi/4) - X_c) s,
//                                Y = sign(z) (2 - s),  X_c = 2 q + 1 the centre of the quarter q of phi.
// In the rotated coordinates p = X + Y, m = X - Y the 12 base pixels are the squares
// [2P - 1, 2P + 1) x [2M - 1, 2M + 1): P = M is an equatorial face (4 + P mod 4), P = M + 1 a
// northern one (M mod 4), M = P + 1 a southern one (8 + P mod 4).  Inside a face, the pixel
// coordinates run along p (ix, from the south corner towards the east one) and along -m (iy,
// towards the west one) in N steps.  Rings are horizontal lines of Y (ring i through the pixel
// centres at Y = 2 - i / N), so the ring of (ix, iy) is j_f N - ix - iy - 1 with j_f = 3 - Y_c
// (Y_c the face centre), and its place along the ring follows from X.
static int64_t healpix_pixel(int64_t N, const double* v, bool nest) {
  const double pi = 3.14159265358979323846;
  const double r = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  const double z = v[2] / r;
  double ph = std::atan2(v[1], v[0]);
  if (ph < 0.0) ph += 2.0 * pi;
  double X = ph / (0.25 * pi);
  if (X >= 8.0) X -= 8.0;
  double Y;
  if (std::fabs(z) <= 2.0 / 3.0) {
    Y = 1.5 * z;
  } else {
    const double s = std::sqrt(3.0 * (1.0 - std::fabs(z)));
    double q = std::floor(0.5 * X);
    if (q > 3.0) q = 3.0;
    const double xc = 2.0 * q + 1.0;
    X = xc + (X - xc) * s;
    Y = z > 0 ? 2.0 - s : s - 2.0;
  }
  const double p = X + Y, m = X - Y;
  const int64_t P = (int64_t)std::floor(0.5 * (p + 1.0));
  const int64_t M = (int64_t)std::floor(0.5 * (m + 1.0));
  int64_t face, yc;  // yc: the face centre's Y
  if (P == M) {
    face = 4 + ((P % 4) + 4) % 4;
    yc = 0;
  } else if (P == M + 1) {
    face = ((M % 4) + 4) % 4;
    yc = 1;
  } else {
    face = 8 + ((P % 4) + 4) % 4;
    yc = -1;
  }
  // position in the face: a along p, b along -m, both in [0, 1]
  const double a = 0.5 * (p - (double)(2 * P - 1));
  const double b = 0.5 * ((double)(2 * M + 1) - m);
  int64_t ix = (int64_t)std::floor(a * (double)N), iy = (int64_t)std::floor(b * (double)N);
  ix = std::min<int64_t>(std::max<int64_t>(ix, 0), N - 1);
  iy = std::min<int64_t>(std::max<int64_t>(iy, 0), N - 1);
  if (nest) {
    int64_t pix = 0;
    for (int bit = 0; bit < 31; ++bit)
      pix |= (((ix >> bit) & 1) << (2 * bit)) | (((iy >> bit) & 1) << (2 * bit + 1));
    return face * N * N + pix;
  }
  // RING: ring i (1 .. 4N - 1 from the north pole) and the place j (1 .. pixels in the ring) of the
  // pixel centre X = X_f + (ix - iy) / N along it; X_f = the face centre's X
  const int64_t xf = face < 4 ? 2 * face + 1 : face < 8 ? 2 * (face - 4) : 2 * (face - 8) + 1;
  const int64_t i = (3 - yc) * N - ix - iy - 1;
  int64_t nr, before, shift;
  if (i < N) {                 // northern cap: 4 i pixels, centres at X = (2 j - 1) / i
    nr = i;
    before = 2 * i * (i - 1);
    shift = 0;
  } else if (i > 3 * N) {      // southern cap
    nr = 4 * N - i;
    before = 12 * N * N - 2 * nr * (nr + 1);
    shift = 0;
  } else {                     // equatorial rings: 4 N pixels, every other ring offset by half a pixel
    nr = N;
    before = 2 * N * (N - 1) + (i - N) * 4 * N;
    shift = (i - N) & 1;
  }
  int64_t j = (xf * nr + ix - iy + 1 + shift) / 2;
  if (j > 4 * nr) j -= 4 * nr;
  if (j < 1) j += 4 * nr;
  return before + j - 1;
}

// HEALPix pixels of n directions ([3][n]); nest: 1 NESTED, 0 RING.
void orc_healpix_pixels(const double* v, int64_t n, int64_t nside, int nest, int64_t* pix) {
  for (int64_t i = 0; i < n; ++i) {
    double d[3] = {v[i], v[n + i], v[2 * n + i]};
    pix[i] = healpix_pixel(nside, d, nest != 0);
  }
}

// Infinitesimal-beam distortion matrix, Eq. (12) with Eqs. (13)-(16), integrated along each
// traced ray (trapezoidal rule over the step points); with gravity off the rays are FLRW
// trajectories: the Born approximation of Sect. 2.3.1.  A: [4][N] = A11, A12, A21, A22.
int orc_infinitesimal(const orc_grid* g, const orc_level* lv, const double* bg, int bg_n, const orc_params* p,
                      const double* dirs, int64_t n_rays, double* A, int n_threads) {
  if (!keys_sorted(g, lv)) return 4;
  if (p->interp < INTERP_CIC || p->interp > INTERP_TSC) return 5;
  Tracer t = make_tracer(g, lv, bg, bg_n, p);
  std::vector<double> es(p->n_cones);
  for (int c = 0; c < p->n_cones; ++c) es[c] = t.bg.eta_stop(p->z_max[c]);
  parallel_for(n_rays, n_threads, [&](int64_t i) {
    int c = cone_of(p, i);
    double n[3] = {dirs[i], dirs[n_rays + i], dirs[2 * n_rays + i]};
    Tracer::Result r = t.trace(p->observer + 3 * c, n, es[c], true);
    for (int q = 0; q < 4; ++q) A[q * n_rays + i] = r.A[q];
  });
  return 0;
}

int orc_trace(const orc_grid* g, const orc_level* lv, const double* bg, int bg_n, const orc_params* p,
              const double* dirs /*[3][N]*/, int64_t n_rays, orc_out* o, int n_threads) {
  return trace_rays_impl(g, lv, bg, bg_n, p, dirs, n_rays, nullptr, o, n_threads);
}

// Rays through the analytic potential phi = A sin(k . x) (analytic = (A, k_x, k_y, k_z)) instead of the
// records: the same integrator with an exactly smooth field (a test of the integration order with the
// gravitational terms); the octree still sets the levels and so the step size.
int orc_trace_analytic(const orc_grid* g, const orc_level* lv, const double* bg, int bg_n, const orc_params* p,
                       const double* dirs, int64_t n_rays, const double* analytic, orc_out* o, int n_threads) {
  return trace_rays_impl(g, lv, bg, bg_n, p, dirs, n_rays, nullptr, o, n_threads, analytic);
}

// Rays stopped at the comoving distances chi_stop[i] (the geodesic finder's iso-chi surface, Sect. 2.5).
int orc_trace_to_chi(const orc_grid* g, const orc_level* lv, const double* bg, int bg_n, const orc_params* p,
                     const double* dirs, int64_t n_rays, const double* chi_stop, orc_out* o, int n_threads) {
  return trace_rays_impl(g, lv, bg, bg_n, p, dirs, n_rays, chi_stop, o, n_threads);
}

// Finite-beam distortion matrix, Eqs. (17)-(21): four rays at semi-aperture eps around
// each central direction, all stopped on the iso-eta surface of the cone, end points
// projected onto that surface, differences projected onto the screen (screen = 0:
// the beta-screen orthogonal to the central ray's source direction; 1: the Sachs screen
// orthogonal to the central ray's wave vector at the end).  Column 2 is taken as
// (xi_D - xi_C) so that A reduces to the identity when phi = 0.
int orc_bundle(const orc_grid* g, const orc_level* lv, const double* bg, int bg_n, const orc_params* p,
               const double* dirs, int64_t n_rays, double eps, int screen, double* A /*[4][N]*/, int n_threads) {
  if (!keys_sorted(g, lv)) return 4;
  if (p->interp < INTERP_CIC || p->interp > INTERP_TSC) return 5;
  Tracer t = make_tracer(g, lv, bg, bg_n, p);
  std::vector<double> es(p->n_cones);
  for (int c = 0; c < p->n_cones; ++c) es[c] = t.bg.eta_stop(p->z_max[c]);
  parallel_for(n_rays, n_threads, [&](int64_t i) {
    int c = cone_of(p, i);
    const double* xo = p->observer + 3 * c;
    double r[3] = {dirs[i], dirs[n_rays + i], dirs[2 * n_rays + i]};
    double th1 = std::atan2(r[1], r[0]);
    double th2 = std::acos(std::max(-1.0, std::min(1.0, r[2])));
    double e1[3] = {-std::sin(th1), std::cos(th1), 0.0};
    double e2[3] = {-std::cos(th1) * std::cos(th2), -std::sin(th1) * std::cos(th2), std::sin(th2)};
    double te = std::tan(eps);
    double dir[4][3];
    double sgn[4] = {+1.0, -1.0, -1.0, +1.0};  // A, B, C, D
    for (int b = 0; b < 4; ++b) {
      const double* e = b < 2 ? e1 : e2;
      double nn = 0.0;
      for (int d = 0; d < 3; ++d) { dir[b][d] = r[d] + sgn[b] * te * e[d]; nn += dir[b][d] * dir[b][d]; }
      nn = std::sqrt(nn);
      for (int d = 0; d < 3; ++d) dir[b][d] /= nn;
    }
    Tracer::Result ref = t.trace(xo, r, es[c]);
    double xr[3];
    xi_of(ref.y, es[c], xr);
    double xi[4][3];
    for (int b = 0; b < 4; ++b) {
      Tracer::Result rb = t.trace(xo, dir[b], es[c]);
      xi_of(rb.y, es[c], xi[b]);
    }
    double v[3];
    if (screen == 0) {
      for (int d = 0; d < 3; ++d) v[d] = xr[d] - xo[d];
    } else {
      for (int d = 0; d < 3; ++d) v[d] = ref.y[5 + d];
    }
    double vn = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double b1 = std::atan2(v[1], v[0]);
    double b2 = std::acos(std::max(-1.0, std::min(1.0, v[2] / vn)));
    double s1[3] = {-std::sin(b1), std::cos(b1), 0.0};
    double s2[3] = {-std::cos(b1) * std::cos(b2), -std::sin(b1) * std::cos(b2), std::sin(b2)};
    double chi0 = std::sqrt((xr[0] - xo[0]) * (xr[0] - xo[0]) + (xr[1] - xo[1]) * (xr[1] - xo[1]) +
                            (xr[2] - xo[2]) * (xr[2] - xo[2]));
    double dAB[3], dDC[3];
    for (int d = 0; d < 3; ++d) { dAB[d] = xi[0][d] - xi[1][d]; dDC[d] = xi[3][d] - xi[2][d]; }
    double den = 2.0 * chi0 * te;
    A[0 * n_rays + i] = (dAB[0] * s1[0] + dAB[1] * s1[1] + dAB[2] * s1[2]) / den;  // A11
    A[1 * n_rays + i] = (dDC[0] * s1[0] + dDC[1] * s1[1] + dDC[2] * s1[2]) / den;  // A12
    A[2 * n_rays + i] = (dAB[0] * s2[0] + dAB[1] * s2[1] + dAB[2] * s2[2]) / den;  // A21
    A[3 * n_rays + i] = (dDC[0] * s2[0] + dDC[1] * s2[1] + dDC[2] * s2[2]) / den;  // A22
  });
  return 0;
}

}  // extern "C"
