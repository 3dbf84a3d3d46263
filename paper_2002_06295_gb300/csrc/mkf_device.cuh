// mkf_device.cuh -- per-candidate Kalman-filter arithmetic in registers.
//
// Kalman filter steps of the paper (Sec. 1): propagate the state and its
// covariance from one layer to the next, then update with the hit.  The
// paper gives no formulas; these are textbook KF equations (Fruhwirth 1987,
// the paper's ref. [1]) for a helix in a uniform field Bz, with Highland
// multiple scattering at each crossed layer (Sec. 2: material description).
//
// State p = (x, y, z, kappa = q/pT, phi, theta); covariance C packed lower
// triangle, index(i, j) = i*(i+1)/2 + j.  Everything is written with
// compile-time indices so that p and C stay in registers.  The routines are
// templates on the scalar type: float for building and the outward fit,
// double for the inward fit, and a forward-mode dual number for the second
// derivatives that the fit adjoint needs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mkf {

constexpr float kAlpha = 0.00299792458f;   // GeV / (T cm)
constexpr float kPionMass2 = 0.13957f * 0.13957f;
constexpr float kNavEps = 1e-6f;           // cm
constexpr float kPi = 3.14159265358979f;
constexpr float kTwoPi = 6.28318530717959f;
constexpr double kPiD = 3.14159265358979323846;

__host__ __device__ constexpr int ci(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

// ---- scalar-type dispatch (float / double; the dual type adds its own) ----
__device__ __forceinline__ float vv(float x) { return x; }
__device__ __forceinline__ double vv(double x) { return x; }
__device__ __forceinline__ float mfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double mfma(double a, double b, double c) { return fma(a, b, c); }
// FP32 sincos and atan are called from several places of the building
// kernel; one out-of-line copy each (with their rarely taken large-argument
// paths) keeps the kernel's code small enough for the instruction caches.
static __device__ __noinline__ float2 msincos_f(float x) {
  float2 r;
  sincosf(x, &r.x, &r.y);
  return r;
}
__device__ __forceinline__ void msincos(float x, float* s, float* c) {
  const float2 r = msincos_f(x);
  *s = r.x;
  *c = r.y;
}
__device__ __forceinline__ void msincos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ float msqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double msqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float mrsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double mrsqrt(double x) { return rsqrt(x); }
static __device__ __noinline__ float matan_f(float x) { return atanf(x); }
__device__ __forceinline__ float matan(float x) { return matan_f(x); }
__device__ __forceinline__ double matan(double x) { return atan(x); }
__device__ __forceinline__ float mlog(float x) { return logf(x); }
__device__ __forceinline__ double mlog(double x) { return log(x); }
__device__ __forceinline__ float mabs(float x) { return fabsf(x); }
__device__ __forceinline__ double mabs(double x) { return fabs(x); }
__device__ __forceinline__ float mrint(float x) { return rintf(x); }
__device__ __forceinline__ double mrint(double x) { return rint(x); }
__device__ __forceinline__ float mcopysign(float a, float b) { return copysignf(a, b); }
__device__ __forceinline__ double mcopysign(double a, double b) { return copysign(a, b); }

template <class T> __device__ __forceinline__ T wrap_phi(T a) {
  return a - T(2.0 * kPiD) * mrint(a * T(1.0 / (2.0 * kPiD)));
}

// Convert a root sigma = tan(omega s / 2) / omega of the crossing equation
// into the transverse path s in the requested direction (dir > 0: s > 0,
// smallest; dir < 0: s < 0, smallest |s|).  atan(t)/t -> 1 keeps omega -> 0
// exact.  s has the sign of sigma and grows with it; a root on the wrong side
// is moved one turn on, beyond every root on the right side.
template <class T> __device__ __forceinline__ T sigma_to_path(T sig, T omega, int dir) {
  T t = omega * sig;
  T s;
  if (mabs(vv(t)) < 1e-3f) {
    s = T(2.0) * sig * (T(1.0) - t * t * T(1.0 / 3.0));
  } else {
    s = T(2.0) * matan(t) / omega;
  }
  using S = decltype(vv(omega));
  const S turn = S(2.0 * kPiD) / mabs(vv(omega));
  if (dir > 0) {
    if (!(vv(s) > 0)) s = s + T(turn);
  } else {
    if (!(vv(s) < 0)) s = s - T(turn);
  }
  return s;
}

// Transverse path to the cylinder x^2 + y^2 = R^2.  With a = P.T, b = P.N
// (T, N: unit tangent and left normal at the start), D = |P|^2 - R^2 and
// sigma = tan(omega s/2)/omega the crossing condition is the quadratic
//   (1 + b omega + D omega^2 / 4) sigma^2 + a sigma + D/4 = 0,
// regular at omega = 0 (straight line: s = 2 sigma).  Returns +inf (dir > 0)
// or -inf (dir < 0) when the circle never reaches R.  The root is chosen on
// the values, so that a dual-number evaluation differentiates that root.
template <class T>
__device__ __forceinline__ T cylinder_path(T x0, T y0, T cph, T sph, T omega, T R, int dir) {
  T D = mfma(x0, x0, mfma(y0, y0, -R * R));
  T a = mfma(x0, cph, y0 * sph);
  T b = mfma(y0, cph, -x0 * sph);
  T A = mfma(T(0.25) * D * omega, omega, mfma(b, omega, T(1.0)));
  T disc = mfma(a, a, -A * D);
  if (!(vv(disc) >= 0)) return T(dir > 0 ? INFINITY : -INFINITY);
  T q = T(-0.5) * (a + mcopysign(msqrt(disc), a));
  const T g1 = q / A, g2 = T(0.25) * D / q;
  // The root giving the shortest path in the requested direction, chosen on
  // sigma and then converted alone: s grows with sigma and has its sign, and a
  // root on the wrong side is moved by one turn, which keeps the order among
  // roots on the same side.  So, both on the same side: dir > 0 takes the
  // smaller sigma, dir < 0 the larger; otherwise the root on the requested side.
  const auto v1 = vv(g1), v2 = vv(g2);
  bool take2;
  if (dir > 0) {
    const bool p1 = v1 > 0, p2 = v2 > 0;
    take2 = p1 == p2 ? v2 < v1 : p2;
  } else {
    const bool n1 = v1 < 0, n2 = v2 < 0;
    take2 = n1 == n2 ? v2 > v1 : n2;
  }
  return sigma_to_path(take2 ? g2 : g1, omega, dir);
}

// Transverse path to the plane z = Z (+-inf when parallel or behind).
template <class T> __device__ __forceinline__ T plane_path(T z0, T cot_t, T Z, int dir) {
  T s = (Z - z0) / cot_t;
  if (dir > 0) return vv(s) > 0 ? s : T(INFINITY);
  return vv(s) < 0 ? s : T(-INFINITY);
}

// Helix point after transverse path s plus the partial derivatives needed by
// the Jacobian.
template <class T> struct HelixPt {
  T x, y, z, phi;   // position and momentum azimuth at s
  T cphi, sphi;     // cos/sin of phi
  T dx_dom, dy_dom; // d x / d omega, d y / d omega at fixed s
};

// (cphi0, sphi0) = cos/sin of phi0, which every caller needs anyway; the
// azimuth at the chord, phi0 + u, is then obtained by angle addition.  For
// |u| < 0.1 sin u, cos u, sinc u = sin(u)/u and its derivative come from their
// series (first omitted terms below 3e-14 relative), else from sincos.
template <class T>
__device__ __forceinline__ HelixPt<T> helix_at(T x0, T y0, T z0, T phi0, T cphi0, T sphi0, T cot_t, T omega, T s) {
  HelixPt<T> h;
  T u = T(0.5) * omega * s;
  T su, cu, sc, dsc;
  if (mabs(vv(u)) < 0.1f) {
    const T u2 = u * u;
    sc = T(1.0) - u2 * T(1.0 / 6.0) * (T(1.0) - u2 * T(1.0 / 20.0) * (T(1.0) - u2 * T(1.0 / 42.0)));
    dsc = -u * T(1.0 / 3.0) * (T(1.0) - u2 * T(1.0 / 10.0) * (T(1.0) - u2 * T(1.0 / 28.0)));
    su = u * sc;
    cu = T(1.0) - T(0.5) * u2 * (T(1.0) - u2 * T(1.0 / 12.0) * (T(1.0) - u2 * T(1.0 / 30.0) *
                                                                       (T(1.0) - u2 * T(1.0 / 56.0))));
  } else {
    msincos(u, &su, &cu);
    const T iu = T(1.0) / u;
    sc = su * iu;
    dsc = (cu - sc) * iu;
  }
  const T cp = cphi0 * cu - sphi0 * su;   // cos(phi0 + u)
  const T sp = sphi0 * cu + cphi0 * su;   // sin(phi0 + u)
  T f = s * sc;
  h.x = mfma(f, cp, x0);
  h.y = mfma(f, sp, y0);
  h.z = mfma(s, cot_t, z0);
  h.phi = phi0 + T(2.0) * u;
  h.cphi = cp * cu - sp * su;   // cos(phi0 + 2u)
  h.sphi = sp * cu + cp * su;   // sin(phi0 + 2u)
  T df = T(0.5) * s * s * dsc;
  T hs = T(0.5) * s;
  h.dx_dom = df * cp - f * sp * hs;
  h.dy_dom = df * sp + f * cp * hs;
  return h;
}

// Jacobian rows for (x, y, z, phi) of the transport p0 -> p(s*(p0)) onto a
// surface: J = A + v w^T with A = dp/dp0 at fixed s, v = dp/ds and
// w = ds*/dp0 = -(dg/dp0)/(dg/ds), g = x^2 + y^2 - R^2 (cylinder) or z - Z
// (plane).  Rows for kappa and theta are the identity.
template <class T> struct Jac4 {
  T r[4][6];
};

template <class T>
__device__ __forceinline__ Jac4<T> transport_jacobian(int kind, const T p0[6], const HelixPt<T>& h, T s, T omega,
                                                      T c_kappa, T cot_t, T sin_t) {
  Jac4<T> J;
  const T zero(0.0), one(1.0);
  T inv_s2 = one / (sin_t * sin_t);
  // A: dp/dp0 at fixed s
  T A[4][6] = {{one, zero, zero, c_kappa * h.dx_dom, -(h.y - p0[1]), zero},
               {zero, one, zero, c_kappa * h.dy_dom, h.x - p0[0], zero},
               {zero, zero, one, zero, zero, -s * inv_s2},
               {zero, zero, zero, c_kappa * s, one, zero}};
  T v[4] = {h.cphi, h.sphi, cot_t, omega};
  T w[6];
  if (kind == 0) {
    T inv_ds = -one / mfma(h.x, h.cphi, h.y * h.sphi);
#pragma unroll
    for (int j = 0; j < 6; ++j) w[j] = inv_ds * mfma(h.x, A[0][j], h.y * A[1][j]);
  } else {
    T inv_ct = -one / cot_t;
#pragma unroll
    for (int j = 0; j < 6; ++j) w[j] = inv_ct * A[2][j];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) J.r[i][j] = mfma(v[i], w[j], A[i][j]);
  return J;
}

// C <- J C J^T using the identity rows of kappa (3) and theta (5).
template <class T> __device__ __forceinline__ void similarity(const Jac4<T>& J, T C[21]) {
  constexpr int R[4] = {0, 1, 2, 4};
  T T4[4][6];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      T acc(0.0);
#pragma unroll
      for (int k = 0; k < 6; ++k) acc = mfma(J.r[i][k], C[ci(k, j)], acc);
      T4[i][j] = acc;
    }
  T out[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      T acc(0.0);
#pragma unroll
      for (int k = 0; k < 6; ++k) acc = mfma(T4[i][k], J.r[j][k], acc);
      out[i][j] = acc;
    }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    C[ci(3, R[i])] = T4[i][3];
    C[ci(5, R[i])] = T4[i][5];
#pragma unroll
    for (int j = 0; j <= i; ++j) C[ci(R[i], R[j])] = out[i][j];
  }
}

// Highland multiple scattering at a crossed surface (pion mass, no energy
// loss): t = x0/|n.u|, theta0 = 0.0136/(beta p) sqrt(t) (1 + 0.038 ln t).
// Returns theta0^2; the covariance gets C_phiphi += theta0^2/sin^2(theta),
// C_thetatheta += theta0^2.
template <class T>
__device__ __forceinline__ T highland_theta0_sq(int kind, T x0, T x, T y, T cphi, T sphi, T kappa, T sin_t, T cos_t) {
  T cosinc;
  if (kind == 0) {
    cosinc = sin_t * mfma(x, cphi, y * sphi) * mrsqrt(mfma(x, x, y * y));
  } else {
    cosinc = cos_t;
  }
  T t = x0 / mabs(cosinc);
  T inv_p = mabs(kappa) * sin_t;            // 1/p
  // 1/(beta p) = sqrt(p^2 + m^2)/p^2 = inv_p * sqrt(1 + m^2 inv_p^2)
  T inv_bp = inv_p * msqrt(mfma(T(kPionMass2) * inv_p, inv_p, T(1.0)));
  T th0 = T(0.0136) * inv_bp * msqrt(t) * mfma(T(0.038), mlog(t), T(1.0));
  return th0 * th0;
}

template <class T>
__device__ __forceinline__ void add_material(int kind, T x0, T x, T y, T cphi, T sphi, T kappa, T sin_t, T cos_t,
                                             T C[21]) {
  if (!(vv(x0) > 0)) return;
  T th2 = highland_theta0_sq(kind, x0, x, y, cphi, sphi, kappa, sin_t, cos_t);
  C[ci(4, 4)] += th2 / (sin_t * sin_t);
  C[ci(5, 5)] += th2;
}

// A hit in its local measurement frame (phi_h = hit azimuth):
//   row a = (-sin phi_h, cos phi_h, 0...), m_a = 0            (r*phi)
//   row b = barrel (0, 0, 1, 0...), m_b = z_h; disk (cos, sin, 0...), m_b = r_h
struct HitRec {
  float c, s, w, v00;     // cos phi_h, sin phi_h, z_h or r_h, var_a
  float v01, v11;         // cov_ab, var_b
  int orig;               // caller's hit index
  int bin;                // bin index inside the event's bin block
};

template <class T> struct Meas {
  T c, s, w, v00, v01, v11;
};

// Position part of a propagated state: what the chi2 of a hit needs.
struct PosState {
  float x, y, z;
  float cxx, cxy, cyy, cxz, cyz, czz;
};

// Predicted chi2 (2 dof) of a hit against a propagated state; returns +inf
// when the state is not in the hit's half plane, and also for every hit that
// is not below `cut`: chi2 = num/det < cut is decided as num < cut det
// without a division (det > 0), so the divisions run only for accepted hits
// and use the fast reciprocal (2 ulp; chi2 values feed scores whose ties are
// resolved at 1e-4 relative, far above that).
__device__ __forceinline__ float hit_chi2(int kind, const PosState& q, const HitRec& h, float cut) {
  if (!(fmaf(h.c, q.x, h.s * q.y) > 0.0f)) return INFINITY;
  float ra = fmaf(h.s, q.x, -h.c * q.y);
  float hab, hbb, rb;
  float haa = fmaf(h.s * h.s, q.cxx, fmaf(-2.0f * h.s * h.c, q.cxy, h.c * h.c * q.cyy));
  if (kind == 0) {
    rb = h.w - q.z;
    hab = fmaf(-h.s, q.cxz, h.c * q.cyz);
    hbb = q.czz;
  } else {
    rb = h.w - fmaf(h.c, q.x, h.s * q.y);
    hab = fmaf(h.s * h.c, q.cyy - q.cxx, (h.c * h.c - h.s * h.s) * q.cxy);
    hbb = fmaf(h.c * h.c, q.cxx, fmaf(2.0f * h.s * h.c, q.cxy, h.s * h.s * q.cyy));
  }
  float Raa = haa + h.v00, Rab = hab + h.v01, Rbb = hbb + h.v11;
  float det = fmaf(Raa, Rbb, -Rab * Rab);
  float num = fmaf(Rbb * ra, ra, fmaf(-2.0f * Rab * ra, rb, Raa * rb * rb));
  if (!(det > 0.0f) || !(num < cut * det)) return INFINITY;
  // For positive-definite R, chi2 >= r_a^2/R_aa and chi2 >= r_b^2/R_bb exactly
  // (Cauchy-Schwarz); when R is so ill-conditioned that FP32 rounding breaks
  // those bounds (elongated position uncertainty seen from a rotated hit
  // frame), the bound is the trustworthy value.  It keeps every accepted hit
  // inside the search window, which is built on the same bound with a 5 %
  // margin (far above the reciprocal's 2 ulp).
  const float chi2 = __fdividef(num, det);
  return fmaxf(chi2, fmaxf(__fdividef(ra * ra, Raa), __fdividef(rb * rb, Rbb)));
}

// Box test ahead of the chi2: the residuals of hit_chi2 against the
// half-widths (ha, hb) of the candidate's search window.  Every hit that
// hit_chi2 accepts passes it: its bound gives r_a^2 < cut R_aa and
// r_b^2 < cut R_bb, and the window's half-widths bound sqrt(cut R_aa) and
// sqrt(cut R_bb) from above with a 5% margin.
__device__ __forceinline__ bool hit_in_box(int kind, float x, float y, float z, const HitRec& h, float ha,
                                           float hb) {
  const float along = fmaf(h.c, x, h.s * y);
  const float ra = fmaf(h.s, x, -h.c * y);
  const float rb = kind == 0 ? h.w - z : h.w - along;
  return along > 0.0f && fabsf(ra) < ha && fabsf(rb) < hb;
}

__device__ __forceinline__ PosState pos_state(const float p[6], const float C[21]) {
  return PosState{p[0], p[1], p[2], C[ci(0, 0)], C[ci(1, 0)], C[ci(1, 1)], C[ci(2, 0)], C[ci(2, 1)], C[ci(2, 2)]};
}

// Kalman update with the hit: B = C H^T, R = V + H B, K = B R^-1,
// p += K r, C -= B R^-1 B^T.  Returns the predicted chi2.  JOSEPH selects the
// Joseph form of the covariance update (needed in FP32, see below); the plain
// form C - B W B^T is used in FP64, where it keeps full precision at less than
// half the operations.
template <class T, bool JOSEPH = true>
__device__ __forceinline__ T kf_update(int kind, T p[6], T C[21], const Meas<T>& h) {
  T B[6][2];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    B[i][0] = mfma(-h.s, C[ci(i, 0)], h.c * C[ci(i, 1)]);
    B[i][1] = kind == 0 ? C[ci(i, 2)] : mfma(h.c, C[ci(i, 0)], h.s * C[ci(i, 1)]);
  }
  T ra = mfma(h.s, p[0], -h.c * p[1]);
  T rb = kind == 0 ? h.w - p[2] : h.w - mfma(h.c, p[0], h.s * p[1]);
  T Raa = mfma(-h.s, B[0][0], h.c * B[1][0]) + h.v00;
  T Rab = mfma(-h.s, B[0][1], h.c * B[1][1]) + h.v01;
  T Rbb = (kind == 0 ? B[2][1] : mfma(h.c, B[0][1], h.s * B[1][1])) + h.v11;
  T idet = T(1.0) / mfma(Raa, Rbb, -Rab * Rab);
  T Waa = Rbb * idet, Wab = -Rab * idet, Wbb = Raa * idet;
  T chi2 = mfma(Waa * ra, ra, mfma(T(2.0) * Wab * ra, rb, Wbb * rb * rb));
  T K[6][2];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    K[i][0] = mfma(B[i][0], Waa, B[i][1] * Wab);
    K[i][1] = mfma(B[i][0], Wab, B[i][1] * Wbb);
    p[i] = mfma(K[i][0], ra, mfma(K[i][1], rb, p[i]));
  }
  p[4] = wrap_phi(p[4]);
  if (!JOSEPH) {
    // C' = C - B W B^T = C - K B^T
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) C[ci(i, j)] = mfma(-K[i][0], B[j][0], mfma(-K[i][1], B[j][1], C[ci(i, j)]));
    return chi2;
  }
  // Covariance in Joseph form, C' = (I - K H) C (I - K H)^T + K V K^T: a sum of
  // positive terms whose rounding does not grow when the hit shrinks a variance
  // by orders of magnitude (the plain C - B W B^T loses those digits in FP32).
  // K H only has position columns (0..2).
  const T Ha[3] = {-h.s, h.c, T(0.0)};
  const T Hb[3] = {kind == 0 ? T(0.0) : h.c, kind == 0 ? T(0.0) : h.s, kind == 0 ? T(1.0) : T(0.0)};
  T KH[6][3];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) KH[i][k] = mfma(K[i][0], Ha[k], K[i][1] * Hb[k]);
  T AC[6][6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      T acc = C[ci(i, j)];
#pragma unroll
      for (int k = 0; k < 3; ++k) acc = mfma(-KH[i][k], C[ci(k, j)], acc);
      AC[i][j] = acc;
    }
  T KV[6][2];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    KV[i][0] = mfma(K[i][0], h.v00, K[i][1] * h.v01);
    KV[i][1] = mfma(K[i][0], h.v01, K[i][1] * h.v11);
  }
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      T acc = mfma(KV[i][0], K[j][0], KV[i][1] * K[j][1]);
      acc = acc + AC[i][j];
#pragma unroll
      for (int k = 0; k < 3; ++k) acc = mfma(-AC[i][k], KH[j][k], acc);
      C[ci(i, j)] = acc;
    }
  return chi2;
}

__device__ __forceinline__ float kf_update(int kind, float p[6], float C[21], const HitRec& h) {
  Meas<float> m{h.c, h.s, h.w, h.v00, h.v01, h.v11};
  return kf_update(kind, p, C, m);
}

}  // namespace mkf
