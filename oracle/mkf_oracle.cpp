// mkf_oracle.cpp -- TEST INFRASTRUCTURE ONLY.
//
// Plain, slow, scalar FP64 reference for combinatorial Kalman-filter track
// building and the fixed-assignment Kalman fit (the method of the paper: Sec. 1
// defines the two KF steps -- propagate layer N-1 -> N, then update with the
// hit -- and the two uses, building and fitting; Sec. 2 the lightweight
// geometry, the per-seed cap on best-ranking candidates; Sec. 3 the hole count
// and the score; the abstract the short-track stash and the duplicate removal).
// The paper prints no formulas, so the arithmetic below is textbook Kalman
// filtering (Fruhwirth 1987, the paper's ref. [1]), helix motion in a uniform
// solenoid field and the PDG Highland multiple-scattering width.
//
// Only the tests, the package smoke check and the benchmark's CPU-baseline leg
// may load this library.  It shares no code with the CUDA library.
//
// Design choices that keep it obviously correct:
//  * every routine is a template on the scalar type, so that
//      - the propagation Jacobian is the forward-mode derivative of the
//        propagator itself (a dual-number pass per input direction, which
//        includes the dependence of the path length on the start state);
//      - the reference gradient of the fit is the same code run on dual
//        numbers (one pass per input direction);
//  * the hit search is brute force: chi2 against every hit of the layer;
//  * the cylinder crossing is the circle-circle intersection, polished by
//    Newton steps on the exact helix.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>

namespace orc {

using std::atan2;
using std::cos;
using std::fabs;
using std::log;
using std::sin;
using std::sqrt;

static const double kAlpha = 0.00299792458;   // GeV/(T cm)
static const double kPionMass = 0.13957;      // GeV
static const double kNavEps = 1e-6;           // cm
static const double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// forward-mode dual numbers (nestable)
template <class T>
struct Dual {
  T v, d;
  Dual() : v(0.0), d(0.0) {}
  Dual(double x) : v(x), d(0.0) {}
  Dual(const T& a, const T& b) : v(a), d(b) {}
};
inline double val(double x) { return x; }
template <class T> double val(const Dual<T>& x) { return val(x.v); }

template <class T> Dual<T> operator+(const Dual<T>& a, const Dual<T>& b) { return Dual<T>(a.v + b.v, a.d + b.d); }
template <class T> Dual<T> operator-(const Dual<T>& a, const Dual<T>& b) { return Dual<T>(a.v - b.v, a.d - b.d); }
template <class T> Dual<T> operator*(const Dual<T>& a, const Dual<T>& b) { return Dual<T>(a.v * b.v, a.d * b.v + a.v * b.d); }
template <class T> Dual<T> operator/(const Dual<T>& a, const Dual<T>& b) {
  T q = a.v / b.v;
  return Dual<T>(q, (a.d - q * b.d) / b.v);
}
template <class T> Dual<T> operator-(const Dual<T>& a) { return Dual<T>(-a.v, -a.d); }
template <class T> Dual<T> operator+(const Dual<T>& a, double b) { return Dual<T>(a.v + b, a.d); }
template <class T> Dual<T> operator+(double b, const Dual<T>& a) { return Dual<T>(a.v + b, a.d); }
template <class T> Dual<T> operator-(const Dual<T>& a, double b) { return Dual<T>(a.v - b, a.d); }
template <class T> Dual<T> operator-(double b, const Dual<T>& a) { return Dual<T>(b - a.v, -a.d); }
template <class T> Dual<T> operator*(const Dual<T>& a, double b) { return Dual<T>(a.v * b, a.d * b); }
template <class T> Dual<T> operator*(double b, const Dual<T>& a) { return Dual<T>(a.v * b, a.d * b); }
template <class T> Dual<T> operator/(const Dual<T>& a, double b) { return Dual<T>(a.v / b, a.d / b); }
template <class T> Dual<T> operator/(double b, const Dual<T>& a) { return Dual<T>(b) / a; }
template <class T> Dual<T>& operator+=(Dual<T>& a, const Dual<T>& b) { a = a + b; return a; }
template <class T> Dual<T>& operator-=(Dual<T>& a, const Dual<T>& b) { a = a - b; return a; }
template <class T> Dual<T>& operator*=(Dual<T>& a, const Dual<T>& b) { a = a * b; return a; }
template <class T> Dual<T> sin(const Dual<T>& a) { return Dual<T>(sin(a.v), cos(a.v) * a.d); }
template <class T> Dual<T> cos(const Dual<T>& a) { return Dual<T>(cos(a.v), -(sin(a.v) * a.d)); }
template <class T> Dual<T> sqrt(const Dual<T>& a) { T r = sqrt(a.v); return Dual<T>(r, a.d / (2.0 * r)); }
template <class T> Dual<T> log(const Dual<T>& a) { return Dual<T>(log(a.v), a.d / a.v); }
template <class T> Dual<T> fabs(const Dual<T>& a) { return val(a) < 0 ? -a : a; }
template <class T> Dual<T> atan2(const Dual<T>& y, const Dual<T>& x) {
  T den = x.v * x.v + y.v * y.v;
  return Dual<T>(atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / den);
}

// ---------------------------------------------------------------------------
// geometry
struct Layer {
  int kind;      // 0 barrel cylinder r = pos, z in [lo, hi]; 1 disk z = pos, r in [lo, hi]
  double pos, lo, hi, x0;
};
struct Geom {
  std::vector<Layer> layers;
  double bz;
  double r_max;   // outer radius of the tracking volume
};
static Geom make_geom(const double* tab, int L, double bz) {
  Geom g;
  g.bz = bz;
  g.r_max = 0;
  for (int l = 0; l < L; ++l) {
    const double* t = tab + 5 * l;
    g.layers.push_back(Layer{(int)t[0], t[1], t[2], t[3], t[4]});
    g.r_max = std::max(g.r_max, (int)t[0] == 0 ? t[1] : t[3]);
  }
  return g;
}

// A surface as seen by one propagation: its position and its material may be
// perturbed (alignment, thickness), hence scalar-typed.
template <class T>
struct Surf {
  int kind;
  T pos;
  double lo, hi;
  T x0;
};

inline int ci(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

template <class T> T wrap_phi(const T& a) {
  double v = val(a);
  double k = std::floor((v + kPi) / (2 * kPi));
  T r = a - 2 * kPi * k;               // (-pi, pi]
  if (val(r) <= -kPi) r = r + 2 * kPi;
  return r;
}

// sin(u)/u, Taylor series near 0 so that the derivatives stay exact.
template <class T> T sinc(const T& u) {
  if (fabs(val(u)) < 0.05) {
    T u2 = u * u;
    return 1.0 - u2 / 6.0 + u2 * u2 / 120.0 - u2 * u2 * u2 / 5040.0 + u2 * u2 * u2 * u2 / 362880.0;
  }
  return sin(u) / u;
}

// Helix in a uniform field Bz: transverse path s, signed curvature
// omega = -alpha*Bz*kappa, u = omega*s/2.
//   x = x0 + s cos(phi0+u) sinc(u),  y = y0 + s sin(phi0+u) sinc(u),
//   z = z0 + s cot(theta),           phi = phi0 + omega s.
template <class T> void helix_at(const T p[6], const T& s, double bz, T q[6]) {
  T omega = -kAlpha * bz * p[3];
  T u = 0.5 * omega * s;
  T f = s * sinc(u);
  q[0] = p[0] + f * cos(p[4] + u);
  q[1] = p[1] + f * sin(p[4] + u);
  q[2] = p[2] + s * cos(p[5]) / sin(p[5]);
  q[3] = p[3];
  q[4] = p[4] + 2.0 * u;
  q[5] = p[5];
}

// Bookkeeping of how close each discrete decision came to flipping (relative).
struct Margin {
  double m = 1e300;
  void add(double v) { if (v < m) m = v; }
};

// Transverse path to the cylinder r = R: the root of x(s)^2 + y(s)^2 = R^2
// closest to the start in direction dir (+1: s > 0, -1: s < 0).  The start
// value comes from the circle-circle intersection (or the line when the field
// is negligible) and is polished by Newton steps on the exact helix, which in
// dual arithmetic also yields ds/d(inputs).
template <class T> bool cyl_path(const T p[6], const T& R, double bz, int dir, T& s_out, Margin* mg) {
  const double x = val(p[0]), y = val(p[1]), ph = val(p[4]);
  const double om = -kAlpha * bz * val(p[3]);
  const double r = val(R);
  double best = 0;
  bool found = false;
  if (fabs(om) < 1e-13) {
    double a = x * cos(ph) + y * sin(ph);
    double c = x * x + y * y - r * r;
    double disc = a * a - c;
    if (mg) mg->add(fabs(disc) / (r * r));
    if (disc < 0) return false;
    double sq = sqrt(disc);
    double roots[2] = {-a - sq, -a + sq};
    for (double s : roots) {
      if (dir * s > 0 && (!found || fabs(s) < fabs(best))) { best = s; found = true; }
    }
  } else {
    const double Rc = 1.0 / fabs(om);
    const double cx = x - sin(ph) / om, cy = y + cos(ph) / om;
    const double d = std::hypot(cx, cy);
    if (mg) {
      mg->add(fabs(r + Rc - d) / r);
      mg->add(fabs(d - fabs(r - Rc)) / r);
    }
    if (d > r + Rc || d < fabs(r - Rc) || d == 0) return false;
    const double a = (r * r - Rc * Rc + d * d) / (2 * d);
    const double h = sqrt(std::max(r * r - a * a, 0.0));
    const double ux = cx / d, uy = cy / d;
    for (int sg = -1; sg <= 1; sg += 2) {
      double qx = a * ux - sg * h * uy, qy = a * uy + sg * h * ux;
      double v0x = x - cx, v0y = y - cy, v1x = qx - cx, v1y = qy - cy;
      double ang = atan2(v0x * v1y - v0y * v1x, v0x * v1x + v0y * v1y) * (om > 0 ? 1.0 : -1.0);
      if (dir > 0 && ang <= 1e-14) ang += 2 * kPi;
      if (dir < 0 && ang >= -1e-14) ang -= 2 * kPi;
      double s = ang * Rc;
      if (!found || fabs(s) < fabs(best)) { best = s; found = true; }
    }
  }
  if (!found) return false;
  T s = T(best);
  for (int it = 0; it < 3; ++it) {
    T q[6];
    helix_at(p, s, bz, q);
    T g = q[0] * q[0] + q[1] * q[1] - R * R;
    T gp = 2.0 * (q[0] * cos(q[4]) + q[1] * sin(q[4]));
    s = s - g / gp;
  }
  s_out = s;
  return true;
}

// Transverse path to the plane z = Z.
template <class T> bool plane_path(const T p[6], const T& Z, int dir, T& s_out) {
  double ct = cos(val(p[5]));
  if (ct == 0.0) return false;
  T s = (Z - p[2]) * sin(p[5]) / cos(p[5]);
  if (!(dir * val(s) > 0)) return false;
  s_out = s;
  return true;
}

template <class T> bool surf_path(const T p[6], const Surf<T>& sf, double bz, int dir, T& s, Margin* mg) {
  return sf.kind == 0 ? cyl_path(p, sf.pos, bz, dir, s, mg) : plane_path(p, sf.pos, dir, s);
}

// Transport (p, C) to a surface: p' = helix(p, s*(p)), C' = J C J^T with
// J = d p' / d p (forward-mode, includes d s*/d p).  The path root is chosen on
// the values and kept by continuity in every derivative pass.
template <class T> bool transport(const T p[6], const T C[21], const Surf<T>& sf, double bz, int dir,
                                  T pout[6], T Cout[21], T* Jout) {
  typedef Dual<T> D;
  T s;
  if (!surf_path(p, sf, bz, dir, s, nullptr)) return false;
  T J[6][6];
  Surf<D> sd{sf.kind, D(sf.pos, T(0.0)), sf.lo, sf.hi, D(sf.x0, T(0.0))};
  for (int j = 0; j < 6; ++j) {
    D pd[6], qd[6], sdv;
    for (int k = 0; k < 6; ++k) pd[k] = D(p[k], T(k == j ? 1.0 : 0.0));
    if (!surf_path(pd, sd, bz, dir, sdv, nullptr)) return false;
    helix_at(pd, sdv, bz, qd);
    for (int i = 0; i < 6; ++i) J[i][j] = qd[i].d;
    if (j == 0) for (int i = 0; i < 6; ++i) pout[i] = qd[i].v;
  }
  pout[4] = wrap_phi(pout[4]);
  T CJt[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      T acc = T(0.0);
      for (int k = 0; k < 6; ++k) acc = acc + C[ci(i, k)] * J[j][k];
      CJt[i][j] = acc;
    }
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j <= i; ++j) {
      T acc = T(0.0);
      for (int k = 0; k < 6; ++k) acc = acc + J[i][k] * CJt[k][j];
      Cout[ci(i, j)] = acc;
    }
  if (Jout)
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) Jout[6 * i + j] = J[i][j];
  return true;
}

// Multiple scattering at a crossed surface (PDG Highland, pion mass, no energy
// loss): effective thickness t = x0/|n.u|; theta0 = 0.0136/(beta p) sqrt(t)
// (1 + 0.038 ln t); C_phiphi += theta0^2/sin^2(theta), C_thetatheta += theta0^2.
template <class T> void add_material(const T p[6], const Surf<T>& sf, T C[21]) {
  if (!(val(sf.x0) > 0)) return;
  T cosinc;
  if (sf.kind == 0) {
    T r = sqrt(p[0] * p[0] + p[1] * p[1]);
    cosinc = sin(p[5]) * (p[0] * cos(p[4]) + p[1] * sin(p[4])) / r;
  } else {
    cosinc = cos(p[5]);
  }
  T t = sf.x0 / fabs(cosinc);
  T mom = 1.0 / (fabs(p[3]) * sin(p[5]));
  T beta_p = mom * mom / sqrt(mom * mom + kPionMass * kPionMass);
  T th0 = 0.0136 / beta_p * sqrt(t) * (1.0 + 0.038 * log(t));
  T st = sin(p[5]);
  C[ci(4, 4)] = C[ci(4, 4)] + th0 * th0 / (st * st);
  C[ci(5, 5)] = C[ci(5, 5)] + th0 * th0;
}

// Two-dimensional measurement in the hit's local frame (hit azimuth phi_h):
// row a = (-sin phi_h, cos phi_h, 0, 0, 0, 0)  with m_a = 0       (r*phi),
// row b = barrel (0, 0, 1, 0, 0, 0) with m_b = z_h;
//         disk   (cos phi_h, sin phi_h, 0, 0, 0, 0) with m_b = r_h.
template <class T>
struct Meas {
  int kind;
  T c, s, w;
  double v00, v01, v11;
};

template <class T>
Meas<T> make_meas(int kind, const T& hx, const T& hy, const T& hz, const double* lcov, const T& dr,
                  const T& dphi, const T& dz) {
  Meas<T> m;
  m.kind = kind;
  T ph = atan2(hy, hx) + dphi;
  m.c = cos(ph);
  m.s = sin(ph);
  m.w = kind == 0 ? hz + dz : sqrt(hx * hx + hy * hy) + dr;
  m.v00 = lcov[0];
  m.v11 = lcov[1];
  m.v01 = lcov[2];
  return m;
}

// Is the state in the hit's half plane (the r*phi coordinate is only single
// valued there)?
template <class T> bool same_side(const T p[6], const Meas<T>& m) {
  return val(m.c) * val(p[0]) + val(m.s) * val(p[1]) > 0;
}

// Predicted chi2 with R = V + H C H^T; when apply: K = C H^T R^-1, p += K r,
// and the updated covariance C' = C - K R K^T written in Joseph form,
// C' = (I - K H) C (I - K H)^T + K V K^T.  The two are the same matrix (expand
// the Joseph form with K R = C H^T); the Joseph form is a sum of two positive
// semi-definite terms, so rounding cannot make C' indefinite, which the
// difference C - K R K^T can on ill-conditioned measurements (a strip disk
// with sigma_r / sigma_rphi = 333).
template <class T> T kf_update(T p[6], T C[21], const Meas<T>& m, bool apply) {
  T H[2][6];
  for (int k = 0; k < 6; ++k) H[0][k] = H[1][k] = T(0.0);
  H[0][0] = -m.s;
  H[0][1] = m.c;
  if (m.kind == 0) {
    H[1][2] = T(1.0);
  } else {
    H[1][0] = m.c;
    H[1][1] = m.s;
  }
  T res[2];
  for (int a = 0; a < 2; ++a) {
    T hp = T(0.0);
    for (int k = 0; k < 6; ++k) hp = hp + H[a][k] * p[k];
    res[a] = (a == 0 ? T(0.0) : m.w) - hp;
  }
  T B[6][2];
  for (int i = 0; i < 6; ++i)
    for (int a = 0; a < 2; ++a) {
      T acc = T(0.0);
      for (int k = 0; k < 6; ++k) acc = acc + C[ci(i, k)] * H[a][k];
      B[i][a] = acc;
    }
  T R[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      T acc = T(0.0);
      for (int k = 0; k < 6; ++k) acc = acc + H[a][k] * B[k][b];
      R[a][b] = acc;
    }
  R[0][0] = R[0][0] + m.v00;
  R[1][1] = R[1][1] + m.v11;
  R[0][1] = R[0][1] + m.v01;
  R[1][0] = R[1][0] + m.v01;
  T det = R[0][0] * R[1][1] - R[0][1] * R[1][0];
  T W[2][2] = {{R[1][1] / det, -R[0][1] / det}, {-R[1][0] / det, R[0][0] / det}};
  T chi2 = T(0.0);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) chi2 = chi2 + res[a] * W[a][b] * res[b];
  if (!apply) return chi2;
  T K[6][2];
  for (int i = 0; i < 6; ++i)
    for (int a = 0; a < 2; ++a) K[i][a] = B[i][0] * W[0][a] + B[i][1] * W[1][a];
  for (int i = 0; i < 6; ++i) p[i] = p[i] + K[i][0] * res[0] + K[i][1] * res[1];
  p[4] = wrap_phi(p[4]);
  // A = I - K H
  T A[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) A[i][j] = T(i == j ? 1.0 : 0.0) - (K[i][0] * H[0][j] + K[i][1] * H[1][j]);
  // AC = A C, then C' = AC A^T + K V K^T
  T AC[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      T acc = T(0.0);
      for (int k = 0; k < 6; ++k) acc = acc + A[i][k] * C[ci(k, j)];
      AC[i][j] = acc;
    }
  const double V[2][2] = {{m.v00, m.v01}, {m.v01, m.v11}};
  T Cn[21];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j <= i; ++j) {
      T acc = T(0.0);
      for (int k = 0; k < 6; ++k) acc = acc + AC[i][k] * A[j][k];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) acc = acc + K[i][a] * V[a][b] * K[j][b];
      Cn[ci(i, j)] = acc;
    }
  for (int k = 0; k < 21; ++k) C[k] = Cn[k];
  return chi2;
}

// ---------------------------------------------------------------------------
// navigation: the next surface outward
struct NavResult {
  int layer = -1;
  double s = 0;
};

static Surf<double> plain_surf(const Layer& ly) { return Surf<double>{ly.kind, ly.pos, ly.lo, ly.hi, ly.x0}; }

// Candidates: barrels with r_L > rho_ref + eps; disks on the side of motion with
// |z_L| > zeta_ref + eps that are crossed before the particle leaves the
// tracking volume (r > r_max).  For each, the first crossing s > 0; keep those
// inside acceptance; the next surface is the one with the smallest s.
static NavResult next_surface(const Geom& g, const double p[6], double rho_ref, double zeta_ref, Margin* mg) {
  NavResult best;
  std::vector<std::pair<double, int>> acc;
  std::vector<std::pair<double, double>> rejected;   // (s, margin) of crossings outside acceptance
  const double cot = cos(p[5]) / sin(p[5]);
  bool exit_known = false;
  double s_exit = 1e300;
  for (int l = 0; l < (int)g.layers.size(); ++l) {
    const Layer& ly = g.layers[l];
    // (a reference equal to a nominal surface position is exact: no margin)
    if (ly.kind == 0) {
      if (mg && ly.pos != rho_ref) mg->add(fabs(ly.pos - rho_ref - kNavEps) / ly.pos);
      if (!(ly.pos > rho_ref + kNavEps)) continue;
    } else {
      if (mg && fabs(ly.pos) != zeta_ref) mg->add(fabs(fabs(ly.pos) - zeta_ref - kNavEps) / fabs(ly.pos));
      if (!(fabs(ly.pos) > zeta_ref + kNavEps)) continue;
      if (!((ly.pos > 0) == (cot > 0)) || cot == 0) continue;
    }
    Surf<double> sf = plain_surf(ly);
    double s;
    if (!surf_path(p, sf, g.bz, +1, s, mg)) continue;
    if (ly.kind == 1) {
      // a particle leaving the tracking volume (r > r_max) is lost: the disk
      // counts only when it is crossed before that exit
      if (!exit_known) {
        double se;
        s_exit = cyl_path(p, g.r_max, g.bz, +1, se, nullptr) ? se : 1e300;
        exit_known = true;
      }
      if (mg) mg->add(fabs(s - s_exit) / std::max(s, 1.0));
      if (!(s < s_exit)) continue;
    }
    double q[6];
    helix_at(p, s, g.bz, q);
    double coord = ly.kind == 0 ? q[2] : std::hypot(q[0], q[1]);
    double edge_m = std::min(fabs(coord - ly.lo) / std::max(1.0, fabs(ly.lo)),
                             fabs(coord - ly.hi) / std::max(1.0, fabs(ly.hi)));
    if (coord >= ly.lo && coord <= ly.hi) {
      acc.push_back({s, l});
      rejected.push_back({s, edge_m});
    } else {
      rejected.push_back({s, edge_m});
    }
  }
  if (!acc.empty()) {
    std::sort(acc.begin(), acc.end());
    best.layer = acc[0].second;
    best.s = acc[0].first;
    if (mg && acc.size() > 1) mg->add((acc[1].first - acc[0].first) / acc[0].first);
  }
  if (mg) {
    // acceptance decisions that could change the choice: crossings not beyond the chosen one
    for (auto& r : rejected)
      if (best.layer < 0 || r.first <= best.s * (1 + 1e-9)) mg->add(r.second);
  }
  return best;
}

// ---------------------------------------------------------------------------
// combinatorial building for one seed
struct Cand {
  double p[6], C[21];
  double score = 0;
  int nh = 0, nholes = 0;
  double rho = 0, zeta = 0;
  std::vector<int> hits, layers;   // per step: hit id (-1 hole), surface id
};

struct Child {
  double score;
  int parent;
  int hit;        // global hit id, -1 for the hole child
  double chi2;
};

static bool child_before(const Child& a, const Child& b) {
  if (a.score != b.score) return a.score > b.score;
  if (a.parent != b.parent) return a.parent < b.parent;
  bool ha = a.hit < 0, hb = b.hit < 0;
  if (ha != hb) return hb;             // hole last
  return a.hit < b.hit;
}

struct HitSet {
  const double* xyz;     // [H][3]
  const double* lcov;    // [H][3]
  const int* layer;      // [H]
  int n;
  long base;             // global id of local hit 0
  std::vector<std::vector<int>> by_layer;
};

struct BuildParams {
  double chi2_cut;
  int max_cands, max_holes, min_hits;
  double dup_frac;
  double tol;
};

struct Track {
  Cand c;
  bool valid = false;
};

static inline double rel_gap(double a, double b) { return fabs(a - b) / std::max(1.0, std::max(fabs(a), fabs(b))); }

static Track build_seed(const Geom& g, const HitSet& hs, const double* sp, const double* sc, const BuildParams& bp,
                        Margin* mg, long long* stats) {
  std::vector<Cand> cands(1);
  Cand& c0 = cands[0];
  for (int k = 0; k < 6; ++k) c0.p[k] = sp[k];
  for (int k = 0; k < 21; ++k) c0.C[k] = sc[k];
  c0.rho = std::hypot(sp[0], sp[1]);
  c0.zeta = fabs(sp[2]);
  std::vector<Cand> finished;
  const int L = (int)g.layers.size();
  for (int step = 0; step <= L && !cands.empty(); ++step) {
    struct Prop {
      double p[6], C[21];
      int layer;
      double rho, zeta;
    };
    std::vector<Prop> props(cands.size());
    std::vector<Child> kids;
    for (int slot = 0; slot < (int)cands.size(); ++slot) {
      Cand& c = cands[slot];
      NavResult nv = next_surface(g, c.p, c.rho, c.zeta, mg);
      if (nv.layer < 0) {
        finished.push_back(c);
        continue;
      }
      const Layer& ly = g.layers[nv.layer];
      Surf<double> sf = plain_surf(ly);
      Prop& pr = props[slot];
      pr.layer = nv.layer;
      if (!transport(c.p, c.C, sf, g.bz, +1, pr.p, pr.C, (double*)nullptr)) {
        finished.push_back(c);
        continue;
      }
      if (stats) stats[0] += 1;   // candidate step
      add_material(pr.p, sf, pr.C);
      double rc = std::hypot(pr.p[0], pr.p[1]);
      if (ly.kind == 0) {
        pr.rho = ly.pos;
        pr.zeta = std::max(c.zeta, fabs(pr.p[2]));
      } else {
        pr.zeta = fabs(ly.pos);
        pr.rho = std::max(c.rho, rc);
      }
      int nk = 0;
      for (int h : hs.by_layer[nv.layer]) {
        const double* x = hs.xyz + 3 * h;
        Meas<double> m = make_meas<double>(ly.kind, x[0], x[1], x[2], hs.lcov + 3 * h, 0.0, 0.0, 0.0);
        if (!same_side(pr.p, m)) continue;
        double pp[6], CC[21];
        std::memcpy(pp, pr.p, sizeof pp);
        std::memcpy(CC, pr.C, sizeof CC);
        double chi2 = kf_update(pp, CC, m, false);
        if (stats) stats[1] += 1;
        if (mg) mg->add(fabs(chi2 - bp.chi2_cut) / bp.chi2_cut);
        if (chi2 < bp.chi2_cut) {
          kids.push_back(Child{c.score + 10.0 - chi2, slot, (int)(hs.base + h), chi2});
          ++nk;
        }
      }
      if (c.nholes + 1 <= bp.max_holes) {
        kids.push_back(Child{c.score - 10.0, slot, -1, 0.0});
        ++nk;
      }
      if (nk == 0) finished.push_back(c);
    }
    std::sort(kids.begin(), kids.end(), child_before);
    const int nsel = std::min((int)kids.size(), bp.max_cands);
    if (mg && (int)kids.size() > bp.max_cands)
      mg->add(rel_gap(kids[bp.max_cands - 1].score, kids[bp.max_cands].score));
    std::vector<Cand> next;
    for (int k = 0; k < nsel; ++k) {
      const Child& ch = kids[k];
      const Cand& par = cands[ch.parent];
      const Prop& pr = props[ch.parent];
      Cand nc;
      std::memcpy(nc.p, pr.p, sizeof nc.p);
      std::memcpy(nc.C, pr.C, sizeof nc.C);
      nc.rho = pr.rho;
      nc.zeta = pr.zeta;
      nc.hits = par.hits;
      nc.layers = par.layers;
      nc.layers.push_back(pr.layer);
      nc.hits.push_back(ch.hit);
      nc.nh = par.nh;
      nc.nholes = par.nholes;
      if (ch.hit >= 0) {
        long h = ch.hit - hs.base;
        const double* x = hs.xyz + 3 * h;
        Meas<double> m = make_meas<double>(g.layers[pr.layer].kind, x[0], x[1], x[2], hs.lcov + 3 * h, 0.0, 0.0, 0.0);
        kf_update(nc.p, nc.C, m, true);
        nc.nh += 1;
        if (stats) stats[2] += 1;
      } else {
        nc.nholes += 1;
      }
      nc.score = ch.score;
      next.push_back(nc);
    }
    cands.swap(next);
  }
  for (auto& c : cands) finished.push_back(c);
  Track t;
  int bi = -1;
  for (int i = 0; i < (int)finished.size(); ++i)
    if (bi < 0 || finished[i].score > finished[bi].score) bi = i;
  if (bi >= 0) {
    if (mg)
      for (int i = 0; i < (int)finished.size(); ++i)
        if (i != bi) mg->add(rel_gap(finished[i].score, finished[bi].score));
    t.c = finished[bi];
    t.valid = true;
  }
  return t;
}

// Greedy duplicate removal: tracks in order of score (desc), seed id (asc); a
// track is dropped when it shares more than dup_frac of min(n_a, n_b) hits with
// an already kept track.  flags: 0 short/none, 1 kept, 2 duplicate.
static void dedup(int S, const double* score, const int* nh, const int* hits, int L, int min_hits, double dup_frac,
                  int* flags, double tol, int* fragile) {
  std::vector<int> order;
  for (int s = 0; s < S; ++s) {
    flags[s] = 0;
    if (nh[s] >= min_hits) order.push_back(s);
  }
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    if (score[a] != score[b]) return score[a] > score[b];
    return a < b;
  });
  std::map<int, std::vector<int>> users;   // hit id -> kept tracks using it
  for (int a : order) {
    std::map<int, int> shared;              // kept track -> hits shared with a
    for (int i = 0; i < L; ++i) {
      int ha = hits[(size_t)a * L + i];
      if (ha < 0) continue;
      auto it = users.find(ha);
      if (it == users.end()) continue;
      for (int b : it->second) shared[b] += 1;
    }
    bool dup = false;
    for (auto& kv : shared) {
      int b = kv.first;
      if (kv.second > dup_frac * std::min(nh[a], nh[b])) {
        dup = true;
        if (fragile && rel_gap(score[a], score[b]) < tol) { fragile[a] = 1; fragile[b] = 1; }
      }
    }
    if (dup) {
      flags[a] = 2;
    } else {
      flags[a] = 1;
      for (int i = 0; i < L; ++i) {
        int ha = hits[(size_t)a * L + i];
        if (ha >= 0) users[ha].push_back(a);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// fixed-assignment fit (forward or backward), templated for the dual gradient
template <class T>
struct FitInputs {
  const Geom* g;
  const T* hxyz;          // [H][3]
  const double* lcov;     // [H][3]
  const int* hlayer;      // [H]
  const T* align;         // [L][3] (dr, dphi, dz) or null
  const T* x0;            // [L] or null
};

template <class T> Surf<T> fit_surf(const FitInputs<T>& in, int l) {
  const Layer& ly = in.g->layers[l];
  Surf<T> sf;
  sf.kind = ly.kind;
  sf.lo = ly.lo;
  sf.hi = ly.hi;
  T shift = in.align ? (ly.kind == 0 ? in.align[3 * l + 0] : in.align[3 * l + 2]) : T(0.0);
  sf.pos = T(ly.pos) + shift;
  sf.x0 = in.x0 ? in.x0[l] : T(ly.x0);
  return sf;
}

template <class T> Meas<T> fit_meas(const FitInputs<T>& in, int h) {
  int l = in.hlayer[h];
  T dr(0.0), dphi(0.0), dz(0.0);
  if (in.align) {
    dr = in.align[3 * l + 0];
    dphi = in.align[3 * l + 1];
    dz = in.align[3 * l + 2];
  }
  return make_meas<T>(in.g->layers[l].kind, in.hxyz[3 * h], in.hxyz[3 * h + 1], in.hxyz[3 * h + 2], in.lcov + 3 * h,
                      dr, dphi, dz);
}

// Forward: propagate outward to each listed hit's surface, add its material,
// update.  Returns false when a surface is not reached.
template <class T> bool fit_forward(const FitInputs<T>& in, const int* ids, int K, T p[6], T C[21], T& chi2) {
  chi2 = T(0.0);
  for (int k = 0; k < K; ++k) {
    int h = ids[k];
    if (h < 0) continue;
    int l = in.hlayer[h];
    Surf<T> sf = fit_surf(in, l);
    T pp[6], CC[21];
    if (!transport(p, C, sf, in.g->bz, +1, pp, CC, (T*)nullptr)) return false;
    add_material(pp, sf, CC);
    Meas<T> m = fit_meas(in, h);
    chi2 = chi2 + kf_update(pp, CC, m, true);
    for (int i = 0; i < 6; ++i) p[i] = pp[i];
    for (int i = 0; i < 21; ++i) C[i] = CC[i];
  }
  return true;
}

// Backward: from the forward result at the outermost hit, covariance reset to
// 100 x the seed-style diagonal; update with the outermost hit in place, then
// propagate inward (s < 0) to each earlier hit, add material, update.  A row
// with no listed hit keeps the starting state with that reset covariance (the
// caller's covariance is never an input of the backward fit).
template <class T> bool fit_backward(const FitInputs<T>& in, const int* ids, int K, T p[6], T C[21], T& chi2) {
  chi2 = T(0.0);
  for (int i = 0; i < 21; ++i) C[i] = T(0.0);
  const double d[6] = {0.01, 0.01, 0.01, -1.0, 0.0025, 0.0025};
  for (int i = 0; i < 6; ++i) C[ci(i, i)] = T(100.0 * d[i]);
  C[ci(3, 3)] = 100.0 * (0.05 * p[3]) * (0.05 * p[3]);
  int last = -1;
  for (int k = K - 1; k >= 0; --k)
    if (ids[k] >= 0) { last = k; break; }
  if (last < 0) return true;
  {
    Meas<T> m = fit_meas(in, ids[last]);
    chi2 = chi2 + kf_update(p, C, m, true);
  }
  for (int k = last - 1; k >= 0; --k) {
    int h = ids[k];
    if (h < 0) continue;
    int l = in.hlayer[h];
    Surf<T> sf = fit_surf(in, l);
    T pp[6], CC[21];
    if (!transport(p, C, sf, in.g->bz, -1, pp, CC, (T*)nullptr)) return false;
    add_material(pp, sf, CC);
    Meas<T> m = fit_meas(in, h);
    chi2 = chi2 + kf_update(pp, CC, m, true);
    for (int i = 0; i < 6; ++i) p[i] = pp[i];
    for (int i = 0; i < 21; ++i) C[i] = CC[i];
  }
  return true;
}

}  // namespace orc

using namespace orc;

// ===========================================================================
// C ABI for ctypes (all arrays row-major, float64 unless stated)
extern "C" {

// Path length and intersection point of one helix with one layer surface.
// Returns 1 when the surface is crossed (acceptance is NOT applied), else 0.
int orc_path(const double* layers, int L, double bz, const double* p, int layer, int dir, double* s_out,
             double* q_out) {
  Geom g = make_geom(layers, L, bz);
  Surf<double> sf = plain_surf(g.layers[layer]);
  double s;
  if (!surf_path(p, sf, bz, dir, s, nullptr)) return 0;
  *s_out = s;
  if (q_out) helix_at(p, s, bz, q_out);
  return 1;
}

// Helix position after a given transverse path s (no surface).
void orc_helix(double bz, const double* p, double s, double* q) { helix_at(p, s, bz, q); }

// Transport (p, C) to a layer surface, optionally adding its material.
// J_out (36, row-major d p'_i / d p_j) may be null.  Returns 1 on success.
int orc_transport(const double* layers, int L, double bz, const double* p, const double* C, int layer, int dir,
                  int material, double* p_out, double* C_out, double* J_out) {
  Geom g = make_geom(layers, L, bz);
  Surf<double> sf = plain_surf(g.layers[layer]);
  if (!transport(p, C, sf, bz, dir, p_out, C_out, J_out)) return 0;
  if (material) add_material(p_out, sf, C_out);
  return 1;
}

// Kalman update of (p, C) with one hit of a layer of the given kind.
// Returns the predicted chi2; p_out/C_out receive the updated state.
double orc_update(int kind, const double* p, const double* C, const double* hit_xyz, const double* hit_lcov,
                  double* p_out, double* C_out) {
  for (int i = 0; i < 6; ++i) p_out[i] = p[i];
  for (int i = 0; i < 21; ++i) C_out[i] = C[i];
  Meas<double> m = make_meas<double>(kind, hit_xyz[0], hit_xyz[1], hit_xyz[2], hit_lcov, 0.0, 0.0, 0.0);
  return kf_update(p_out, C_out, m, true);
}

// Navigation: next surface outward from a state with reference radius/|z|.
int orc_next_surface(const double* layers, int L, double bz, const double* p, double rho_ref, double zeta_ref,
                     double* s_out) {
  Geom g = make_geom(layers, L, bz);
  NavResult nv = next_surface(g, p, rho_ref, zeta_ref, nullptr);
  if (s_out) *s_out = nv.s;
  return nv.layer;
}

// Combinatorial building of one event (hits of that event only; hit ids in
// outputs are hit_base + local index).  Per seed outputs:
//   out_hits/out_layers [S][L] step-ordered hit id (-1 hole) / surface id (-1 past the end)
//   out_par [S][6], out_cov [S][21], out_score, out_chi2 [S] (doubles)
//   out_nhits, out_nholes, out_nsteps, out_flags (0 short/none, 1 kept, 2 duplicate), out_fragile [S] (ints)
//   out_margin [S]: smallest relative margin of any discrete decision on the seed's path
// stats[0] candidate steps, [1] chi2 evaluations, [2] hit updates of kept children.
int orc_build(const double* layers, int L, double bz, const double* hit_xyz, const double* hit_lcov,
              const int* hit_layer, int H, long hit_base, const double* seed_par, const double* seed_cov, int S,
              double chi2_cut, int max_cands, int max_holes, int min_hits, double dup_frac, double tol,
              int* out_hits, int* out_layers, double* out_par, double* out_cov, double* out_score, double* out_chi2,
              int* out_nhits, int* out_nholes, int* out_nsteps, int* out_flags, int* out_fragile,
              double* out_margin, long long* stats, int do_dedup) {
  Geom g = make_geom(layers, L, bz);
  HitSet hs{hit_xyz, hit_lcov, hit_layer, H, hit_base, {}};
  hs.by_layer.resize(L);
  for (int h = 0; h < H; ++h)
    if (hit_layer[h] >= 0 && hit_layer[h] < L) hs.by_layer[hit_layer[h]].push_back(h);
  BuildParams bp{chi2_cut, max_cands, max_holes, min_hits, dup_frac, tol};
  std::vector<double> sc(S);
  std::vector<int> nh(S), hl((size_t)S * L, -1);
  for (int s = 0; s < S; ++s) {
    Margin mg;
    Track t = build_seed(g, hs, seed_par + 6 * s, seed_cov + 21 * s, bp, &mg, stats);
    for (int k = 0; k < L; ++k) {
      out_hits[(size_t)s * L + k] = -1;
      out_layers[(size_t)s * L + k] = -1;
    }
    const Cand& c = t.c;
    int n = (int)c.hits.size();
    for (int k = 0; k < n && k < L; ++k) {
      out_hits[(size_t)s * L + k] = c.hits[k];
      out_layers[(size_t)s * L + k] = c.layers[k];
      hl[(size_t)s * L + k] = c.hits[k];
    }
    for (int k = 0; k < 6; ++k) out_par[6 * s + k] = c.p[k];
    for (int k = 0; k < 21; ++k) out_cov[21 * s + k] = c.C[k];
    out_score[s] = c.score;
    out_chi2[s] = 10.0 * c.nh - 10.0 * c.nholes - c.score;
    out_nhits[s] = c.nh;
    out_nholes[s] = c.nholes;
    out_nsteps[s] = n;
    out_margin[s] = mg.m;
    out_fragile[s] = mg.m < tol ? 1 : 0;
    sc[s] = c.score;
    nh[s] = c.nh;
  }
  if (do_dedup) {
    dedup(S, sc.data(), nh.data(), hl.data(), L, min_hits, dup_frac, out_flags, tol, out_fragile);
  } else {
    for (int s = 0; s < S; ++s) out_flags[s] = nh[s] >= min_hits ? 1 : 0;
  }
  return 0;
}

// Duplicate removal alone on given tracks: hits [S][L] (-1 none), score [S], nhits [S].
int orc_dedup(int S, int L, const int* hits, const double* score, const int* nhits, int min_hits, double dup_frac,
              int* out_flags) {
  dedup(S, score, nhits, hits, L, min_hits, dup_frac, out_flags, 0.0, nullptr);
  return 0;
}

// Fixed-assignment fit of T tracks.  hits [T][K] hit ids in crossing order (-1
// skipped).  dir +1 forward from init_par/init_cov; dir -1 backward (init_par is
// the forward result at the outermost hit, init_cov ignored).  align [L][3],
// x0 [L] may be null.  out_ok[t] = 1 when every surface was reached.
int orc_fit(const double* layers, int L, double bz, const double* hit_xyz, const double* hit_lcov,
            const int* hit_layer, int H, const int* hits, int K, const double* init_par, const double* init_cov,
            int T, const double* align, const double* x0, int dir, double* out_par, double* out_cov,
            double* out_chi2, int* out_ok) {
  Geom g = make_geom(layers, L, bz);
  FitInputs<double> in{&g, hit_xyz, hit_lcov, hit_layer, align, x0};
  for (int t = 0; t < T; ++t) {
    double p[6], C[21], chi2 = 0;
    for (int k = 0; k < 6; ++k) p[k] = init_par[6 * t + k];
    for (int k = 0; k < 21; ++k) C[k] = init_cov[21 * t + k];
    bool ok = dir > 0 ? fit_forward(in, hits + (size_t)t * K, K, p, C, chi2)
                      : fit_backward(in, hits + (size_t)t * K, K, p, C, chi2);
    out_ok[t] = ok ? 1 : 0;
    for (int k = 0; k < 6; ++k) out_par[6 * t + k] = p[k];
    for (int k = 0; k < 21; ++k) out_cov[21 * t + k] = C[k];
    out_chi2[t] = chi2;
  }
  return 0;
}

// Overlap-hit recovery (Sec. 3: hits in overlapping detector modules, more
// than one hit per layer assigned to a track; the paper plans the feature and
// fixes no rule, so this is a reading): run the forward fit of each track;
// after the update with its hit h on layer l, every other hit of the same
// event on layer l in the state's half plane that lies in the adjacent-module
// box around h (|R sin(phi_2 - phi_h)| <= max_drphi with cos > 0, R the layer
// radius on a barrel or h's radius on a disk, and |w_2 - w_h| <= max_dw, w = z
// on a barrel, r on a disk) is a candidate, with the
// predicted chi2 of that hit against the updated state (the state is not
// updated with it); the overlap hit is the candidate of smallest chi2 below
// chi2_cut (ties: smaller id).  Outputs per (track, slot): out_hit (-1:
// none), out_chi2, and for comparisons out_gap = the relative chi2 gap from
// the best candidate to the next one (inf if none) and out_best = the best
// candidate's chi2 whether or not it passes the cut (inf if none).
int orc_overlaps(const double* layers, int L, double bz, const double* hit_xyz, const double* hit_lcov,
                 const int* hit_layer, int H, const long long* ev_hit_off, int n_events, const int* hits, int K,
                 const double* init_par, const double* init_cov, int T, double chi2_cut, double max_drphi,
                 double max_dw, int* out_hit, double* out_chi2, double* out_gap, double* out_best) {
  Geom g = make_geom(layers, L, bz);
  FitInputs<double> in{&g, hit_xyz, hit_lcov, hit_layer, nullptr, nullptr};
  for (int t = 0; t < T; ++t) {
    const int* ids = hits + (size_t)t * K;
    for (int k = 0; k < K; ++k) {
      out_hit[(size_t)t * K + k] = -1;
      out_chi2[(size_t)t * K + k] = 0.0;
      out_gap[(size_t)t * K + k] = INFINITY;
      out_best[(size_t)t * K + k] = INFINITY;
    }
    int first = -1;
    for (int k = 0; k < K && first < 0; ++k) first = ids[k];
    if (first < 0) continue;
    int e = 0;   // the track's event: the one holding its first hit
    while (e + 1 < n_events && ev_hit_off[e + 1] <= first) ++e;
    double p[6], C[21];
    for (int k = 0; k < 6; ++k) p[k] = init_par[6 * t + k];
    for (int k = 0; k < 21; ++k) C[k] = init_cov[21 * t + k];
    for (int k = 0; k < K; ++k) {
      const int h = ids[k];
      if (h < 0) continue;
      const int l = hit_layer[h];
      Surf<double> sf = fit_surf(in, l);
      double pp[6], CC[21];
      if (!transport(p, C, sf, g.bz, +1, pp, CC, (double*)nullptr)) break;
      add_material(pp, sf, CC);
      kf_update(pp, CC, fit_meas(in, h), true);
      for (int i = 0; i < 6; ++i) p[i] = pp[i];
      for (int i = 0; i < 21; ++i) C[i] = CC[i];
      double best = INFINITY, second = INFINITY;
      int best_id = -1;
      const Meas<double> mh = fit_meas(in, h);
      const double Rh = g.layers[l].kind == 0 ? g.layers[l].pos : mh.w;
      for (long long h2 = ev_hit_off[e]; h2 < ev_hit_off[e + 1]; ++h2) {
        if (h2 == h || hit_layer[h2] != l) continue;
        const Meas<double> m2 = fit_meas(in, (int)h2);
        const double cd = mh.c * m2.c + mh.s * m2.s, sd = mh.c * m2.s - mh.s * m2.c;
        if (!(cd > 0.0) || std::fabs(Rh * sd) > max_drphi || std::fabs(m2.w - mh.w) > max_dw) continue;
        if (!same_side(p, m2)) continue;
        double q[6], Q[21];
        for (int i = 0; i < 6; ++i) q[i] = p[i];
        for (int i = 0; i < 21; ++i) Q[i] = C[i];
        const double c2 = kf_update(q, Q, m2, false);
        if (c2 < best) {
          second = best;
          best = c2;
          best_id = (int)h2;
        } else if (c2 < second) {
          second = c2;
        }
      }
      const size_t o = (size_t)t * K + k;
      out_best[o] = best;
      out_gap[o] = best_id >= 0 ? (second - best) / std::max(1.0, best) : INFINITY;
      if (best_id >= 0 && best < chi2_cut) {
        out_hit[o] = best_id;
        out_chi2[o] = best;
      }
    }
  }
  return 0;
}

// Reference gradient of the forward fit, by forward-mode dual numbers (one
// pass per input direction):  loss = sum_t g_chi2[t] chi2_t + g_par[t].p_t +
// g_cov[t].C_t (packed entries); returns d loss / d hit xyz [H][3],
// d/d align [L][3] (dr, dphi, dz), d/d x0 [L].  g_par/g_cov may be null.
int orc_fit_grad(const double* layers, int L, double bz, const double* hit_xyz, const double* hit_lcov,
                 const int* hit_layer, int H, const int* hits, int K, const double* init_par, const double* init_cov,
                 int T, const double* align, const double* x0, const double* g_chi2, const double* g_par,
                 const double* g_cov, double* out_g_hit, double* out_g_align, double* out_g_x0) {
  typedef Dual<double> D;
  Geom g = make_geom(layers, L, bz);
  std::vector<D> hx((size_t)3 * H), al((size_t)3 * L), xx(L);
  for (int i = 0; i < 3 * H; ++i) hx[i] = D(hit_xyz[i]);
  for (int l = 0; l < L; ++l) {
    for (int c = 0; c < 3; ++c) al[3 * l + c] = D(align ? align[3 * l + c] : 0.0);
    xx[l] = D(x0 ? x0[l] : g.layers[l].x0);
  }
  FitInputs<D> in{&g, hx.data(), hit_lcov, hit_layer, al.data(), xx.data()};
  auto track_loss = [&](int t) -> double {
    D p[6], C[21], chi2;
    for (int k = 0; k < 6; ++k) p[k] = D(init_par[6 * t + k]);
    for (int k = 0; k < 21; ++k) C[k] = D(init_cov[21 * t + k]);
    fit_forward(in, hits + (size_t)t * K, K, p, C, chi2);
    double d = g_chi2 ? g_chi2[t] * chi2.d : 0.0;
    if (g_par)
      for (int k = 0; k < 6; ++k) d += g_par[6 * t + k] * p[k].d;
    if (g_cov)
      for (int k = 0; k < 21; ++k) d += g_cov[21 * t + k] * C[k].d;
    return d;
  };
  for (int i = 0; i < 3 * H; ++i) out_g_hit[i] = 0.0;
  for (int t = 0; t < T; ++t) {
    for (int k = 0; k < K; ++k) {
      int h = hits[(size_t)t * K + k];
      if (h < 0) continue;
      for (int c = 0; c < 3; ++c) {
        hx[3 * h + c].d = 1.0;
        out_g_hit[3 * h + c] += track_loss(t);
        hx[3 * h + c].d = 0.0;
      }
    }
  }
  for (int l = 0; l < L; ++l) {
    for (int c = 0; c < 4; ++c) {
      D& v = c < 3 ? al[3 * l + c] : xx[l];
      v.d = 1.0;
      double acc = 0.0;
      for (int t = 0; t < T; ++t) acc += track_loss(t);
      v.d = 0.0;
      if (c < 3)
        out_g_align[3 * l + c] = acc;
      else
        out_g_x0[l] = acc;
    }
  }
  return 0;
}

}  // extern "C"
