// fit.cu -- Kalman fit over a fixed hit assignment (Sec. 1: fitting applies
// the KF procedure to all hits found in building), outward and inward.
// One thread per track; the state stays in registers for all its hits.
//
// The outward fit runs in FP32.  The inward fit starts from a prior 100 times
// wider than the seed's, so its first updates shrink variances by factors up
// to 1e5, and on mixed barrel/disk tracks the state keeps correlations close
// to 1 for many hits: FP32 cannot carry its covariance to 1e-4, so the inward
// fit runs in FP64.
#include "mkf_device.cuh"
#include "mkf_fit_common.cuh"
#include "mkf_internal.h"

namespace mkf {

namespace {

template <class T>
__global__ void k_fit(const GeomDev* __restrict__ g, const float* __restrict__ xyz,
                      const float* __restrict__ lcov, const int* __restrict__ layer, int64_t H,
                      const int* __restrict__ hits, int K, const float* __restrict__ init_par,
                      const float* __restrict__ init_cov, int64_t NT, const float* __restrict__ align,
                      const float* __restrict__ x0, float* __restrict__ out_par, float* __restrict__ out_cov,
                      float* __restrict__ out_chi2, int* __restrict__ out_ok, float* __restrict__ ckpt) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NT) return;
  const T ck = T(g->c_kappa);
  T p[6], C[21];
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = T(init_par[k * NT + t]);
  T chi2(0.0);
  int ok = 1;
  const int* row = hits + t * K;
#pragma unroll
  for (int k = 0; k < 21; ++k) C[k] = T(init_cov[k * NT + t]);
  for (int k = 0; k < K; ++k) {
    if (ckpt) {
      float* c = ckpt + (size_t)k * 27 * NT + t;
#pragma unroll
      for (int i = 0; i < 6; ++i) c[i * NT] = float(p[i]);
#pragma unroll
      for (int i = 0; i < 21; ++i) c[(6 + i) * NT] = float(C[i]);
    }
    FitHit<T> f;
    if (!load_fit_hit(g, xyz, lcov, layer, H, row[k], align, x0, f)) continue;
    if (!step_to(f, p, C, ck, +1)) {
      ok = 0;
      // mark the steps that did not happen (x = NaN) for the adjoint
      if (ckpt)
        for (int k2 = k; k2 < K; ++k2) ckpt[(size_t)k2 * 27 * NT + t] = __int_as_float(0x7fc00000);
      break;
    }
    chi2 += kf_update(f.kind, p, C, f.m);
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) out_par[k * NT + t] = float(p[k]);
#pragma unroll
  for (int k = 0; k < 21; ++k) out_cov[k * NT + t] = float(C[k]);
  out_chi2[t] = float(chi2);
  if (out_ok) out_ok[t] = ok;
}

// The listed slot before slot k of a track's hit row (-1 when there is none).
__device__ __forceinline__ int prev_listed(const int* __restrict__ row, int k) {
  do {
    --k;
  } while (k >= 0 && row[k] < 0);
  return k;
}

// ---- the inward fit's FP64 step
//
// The same transport and update as step_to / kf_update in FP64, arranged so
// that fewer FP64 instructions sit on each hit's dependent chain (one warp per
// SM sub-partition runs at the rate of its FP64 unit there):
//  * cos/sin of phi and theta are carried with the state: the transport turns
//    phi by the helix angle (angle addition, already in helix_at) and the update
//    turns both by its small increments, so no sincos is evaluated per hit;
//  * one reciprocal serves several quotients (1/sin theta for cot theta, the
//    Jacobian and the material term; 1/(q A) for both roots of the crossing
//    quadratic);
//  * atan(t)/t comes from its Taylor series for |t| < 0.1 (the usual step);
//  * the covariance algebra runs in double-float on the FP32 pipes (below).

struct InwardHit {
  int kind;
  double pos;     // surface r (barrel) or z (disk), aligned
  float x0;       // thickness
  Meas<double> m;
  float v00, v01, v11;   // the hit's covariance as stored (FP32)
};

// load_fit_hit in FP64 with the hit's unit vector from one rsqrt.
__device__ __forceinline__ bool load_inward_hit(const GeomDev* __restrict__ g, const float* __restrict__ xyz,
                                                const float* __restrict__ lcov, const int* __restrict__ layer,
                                                int64_t H, int h, const float* __restrict__ align,
                                                const float* __restrict__ x0, InwardHit& f) {
  if (h < 0 || h >= H) return false;
  const int l = layer[h];
  if (l < 0 || l >= g->n_layers) return false;
  const LayerDev ly = g->L[l];
  double dr = 0.0, dphi = 0.0, dz = 0.0;
  if (align) {
    dr = double(align[3 * l]);
    dphi = double(align[3 * l + 1]);
    dz = double(align[3 * l + 2]);
  }
  const double x = double(xyz[h]), y = double(xyz[H + h]), z = double(xyz[2 * H + h]);
  const double r2 = fma(x, x, y * y);
  const double ir = rsqrt(r2);
  double sd = 0.0, cd = 1.0;
  if (align) sincos(dphi, &sd, &cd);
  f.kind = ly.kind;
  f.pos = ly.kind == 0 ? double(ly.pos) + dr : double(ly.pos) + dz;
  f.x0 = x0 ? x0[l] : ly.x0;
  f.m.c = (x * cd - y * sd) * ir;
  f.m.s = (x * sd + y * cd) * ir;
  f.m.w = ly.kind == 0 ? z + dz : r2 * ir + dr;
  f.v00 = lcov[h];
  f.v11 = lcov[H + h];
  f.v01 = lcov[2 * H + h];
  f.m.v00 = double(f.v00);
  f.m.v11 = double(f.v11);
  f.m.v01 = double(f.v01);
  return true;
}

// (c, s) = cos/sin of an angle that moved by d to a_new: a rotation by d with
// sin d and cos d from their Taylor series (first omitted terms below 3e-19
// for |d| < 0.1), else a fresh sincos of a_new.
__device__ __forceinline__ void turn_by(double d, double a_new, double& c, double& s) {
  if (fabs(d) < 0.1) {
    const double d2 = d * d;
    const double sd =
        d * fma(fma(fma(fma(d2, 1.0 / 362880.0, -1.0 / 5040.0), d2, 1.0 / 120.0), d2, -1.0 / 6.0), d2, 1.0);
    const double cd = fma(
        fma(fma(fma(fma(d2, -1.0 / 3628800.0, 1.0 / 40320.0), d2, -1.0 / 720.0), d2, 1.0 / 24.0), d2, -0.5), d2,
        1.0);
    const double c2 = fma(c, cd, -s * sd);
    s = fma(s, cd, c * sd);
    c = c2;
  } else {
    sincos(a_new, &s, &c);
  }
}

// Transverse path (s < 0, smallest |s|) to the cylinder r = R: cylinder_path
// with dir < 0, one reciprocal for both roots, and 2 atan(t)/omega written as
// 2 sigma atan(t)/t with the Taylor series of atan(t)/t for |t| < 0.1 (first
// omitted term t^16/17 < 1e-17).
__device__ __forceinline__ double cylinder_path_inward(double x0, double y0, double cph, double sph, double omega,
                                                       double R) {
  const double D = fma(x0, x0, fma(y0, y0, -R * R));
  const double a = fma(x0, cph, y0 * sph);
  const double b = fma(y0, cph, -x0 * sph);
  const double A = fma(0.25 * D * omega, omega, fma(b, omega, 1.0));
  const double disc = fma(a, a, -A * D);
  if (!(disc >= 0.0)) return -INFINITY;
  const double q = -0.5 * (a + copysign(sqrt(disc), a));
  const double rqa = 1.0 / (q * A);
  const double g1 = q * q * rqa, g2 = 0.25 * D * A * rqa;   // q / A and D / (4 q)
  const bool n1 = g1 < 0.0, n2 = g2 < 0.0;
  const double sig = (n1 == n2 ? g2 > g1 : n2) ? g2 : g1;
  const double t = omega * sig;
  double s;
  if (fabs(t) < 0.1) {
    const double t2 = t * t;
    const double at = fma(fma(fma(fma(fma(fma(fma(t2, -1.0 / 15.0, 1.0 / 13.0), t2, -1.0 / 11.0), t2, 1.0 / 9.0), t2,
                                      -1.0 / 7.0), t2, 1.0 / 5.0), t2, -1.0 / 3.0), t2, 1.0);
    s = 2.0 * sig * at;
  } else {
    s = 2.0 * atan(t) / omega;
  }
  if (!(s < 0.0)) s -= 2.0 * kPiD / fabs(omega);
  return s;
}

// ---- double-float arithmetic for the inward fit's covariance
//
// A value is held as the unevaluated sum h + l of two floats (about 48
// significant bits), built from error-free transformations: TwoSum (Knuth),
// FastTwoSum (Dekker) and the exact product error fma(a, b, -a b).  The
// __f*_rn intrinsics keep the compiler from contracting their adds and
// multiplies into FMAs, which would break the transformations.  The
// covariance needs far more than FP32 (the first updates shrink variances by
// up to 1e5, and mixed barrel/disk tracks keep correlations close to 1) but far
// less than FP64's 53 bits, and the FP32 pipes are idle in this kernel while
// its FP64 unit is the bottleneck.
struct f2 {
  float h, l;
};

__device__ __forceinline__ f2 f2_fast_two_sum(float a, float b) {   // needs |a| >= |b| (or a = 0)
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ f2 f2_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ f2 f2_of(double x) {
  const float h = float(x);
  return {h, float(x - double(h))};
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  const f2 s = f2_two_sum(a.h, b.h);
  return f2_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  const float p = __fmul_rn(a.h, b.h);
  return f2_fast_two_sum(p, fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p))));
}
__device__ __forceinline__ f2 f2_mulf(f2 a, float b) {
  const float p = __fmul_rn(a.h, b);
  return f2_fast_two_sum(p, fmaf(a.l, b, fmaf(a.h, b, -p)));
}
// 1/d: the float reciprocal refined by one Newton step, e = 1 - d y exactly to
// double-float precision (1 - (d y)_h is exact near 1).
__device__ __forceinline__ f2 f2_recip(f2 d) {
  const float y = __frcp_rn(d.h);
  const f2 t = f2_mulf(d, y);
  const float e = __fsub_rn(__fsub_rn(1.0f, t.h), t.l);
  return f2_fast_two_sum(y, __fmul_rn(y, e));
}

// A running sum of products: s collects the leading parts by TwoSum, c the
// rounding errors and low-order terms (float), normalised once at the end.
struct f2acc {
  float s, c;
};
__device__ __forceinline__ f2acc f2acc_of(f2 x) { return {x.h, x.l}; }
__device__ __forceinline__ void f2acc_add_mulf(f2acc& a, f2 x, float y) {   // a += x y
  const float p = __fmul_rn(x.h, y);
  const float e = fmaf(x.l, y, fmaf(x.h, y, -p));
  const f2 t = f2_two_sum(a.s, p);
  a.s = t.h;
  a.c = __fadd_rn(a.c, __fadd_rn(t.l, e));
}
__device__ __forceinline__ void f2acc_add_mul(f2acc& a, f2 x, f2 y) {   // a += x y
  const float p = __fmul_rn(x.h, y.h);
  const float e = fmaf(x.h, y.l, fmaf(x.l, y.h, fmaf(x.h, y.h, -p)));
  const f2 t = f2_two_sum(a.s, p);
  a.s = t.h;
  a.c = __fadd_rn(a.c, __fadd_rn(t.l, e));
}
__device__ __forceinline__ f2 f2acc_get(const f2acc& a) { return f2_two_sum(a.s, a.c); }

// C <- J C J^T for J = A + v w^T on the rows (x, y, z, phi), kappa and theta
// rows the identity, C in double-float and J's factors in FP32 (a Jacobian
// off by ~1e-7 relative transports C by a slightly different map, which keeps
// it a covariance; the rounding of C itself is what needs the precision).
// With u = C w: J C = A C + v u^T and J C J^T = (J C) A^T + z v^T with
// z = J C w = A u + (w.u) v; A's fixed ones and zeros leave 139 products
// instead of the dense 204.
__device__ __forceinline__ void similarity_rank1_f2(float a03, float a04, float a13, float a14, float a25, float a33,
                                                    const float v[4], const float w[6], f2 C[21]) {
  f2 u[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    f2acc acc{0.0f, 0.0f};
#pragma unroll
    for (int j = 0; j < 6; ++j) f2acc_add_mulf(acc, C[ci(k, j)], w[j]);
    u[k] = f2acc_get(acc);
  }
  f2 JC[4][6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    f2acc r0 = f2acc_of(C[ci(0, j)]);
    f2acc_add_mulf(r0, C[ci(3, j)], a03);
    f2acc_add_mulf(r0, C[ci(4, j)], a04);
    f2acc_add_mulf(r0, u[j], v[0]);
    JC[0][j] = f2acc_get(r0);
    f2acc r1 = f2acc_of(C[ci(1, j)]);
    f2acc_add_mulf(r1, C[ci(3, j)], a13);
    f2acc_add_mulf(r1, C[ci(4, j)], a14);
    f2acc_add_mulf(r1, u[j], v[1]);
    JC[1][j] = f2acc_get(r1);
    f2acc r2 = f2acc_of(C[ci(2, j)]);
    f2acc_add_mulf(r2, C[ci(5, j)], a25);
    f2acc_add_mulf(r2, u[j], v[2]);
    JC[2][j] = f2acc_get(r2);
    f2acc r3 = f2acc_of(C[ci(4, j)]);
    f2acc_add_mulf(r3, C[ci(3, j)], a33);
    f2acc_add_mulf(r3, u[j], v[3]);
    JC[3][j] = f2acc_get(r3);
  }
  f2acc wa{0.0f, 0.0f};
#pragma unroll
  for (int j = 0; j < 6; ++j) f2acc_add_mulf(wa, u[j], w[j]);
  const f2 wu = f2acc_get(wa);
  f2 zz[4];
  {
    f2acc z0 = f2acc_of(u[0]);
    f2acc_add_mulf(z0, u[3], a03);
    f2acc_add_mulf(z0, u[4], a04);
    f2acc_add_mulf(z0, wu, v[0]);
    zz[0] = f2acc_get(z0);
    f2acc z1 = f2acc_of(u[1]);
    f2acc_add_mulf(z1, u[3], a13);
    f2acc_add_mulf(z1, u[4], a14);
    f2acc_add_mulf(z1, wu, v[1]);
    zz[1] = f2acc_get(z1);
    f2acc z2 = f2acc_of(u[2]);
    f2acc_add_mulf(z2, u[5], a25);
    f2acc_add_mulf(z2, wu, v[2]);
    zz[2] = f2acc_get(z2);
    f2acc z3 = f2acc_of(u[4]);
    f2acc_add_mulf(z3, u[3], a33);
    f2acc_add_mulf(z3, wu, v[3]);
    zz[3] = f2acc_get(z3);
  }
  constexpr int R[4] = {0, 1, 2, 4};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    // (J C A^T)[i][l] + z_i v_l for the rows l <= i
#pragma unroll
    for (int l = 0; l <= i; ++l) {
      f2acc o;
      if (l == 0) {
        o = f2acc_of(JC[i][0]);
        f2acc_add_mulf(o, JC[i][3], a03);
        f2acc_add_mulf(o, JC[i][4], a04);
      } else if (l == 1) {
        o = f2acc_of(JC[i][1]);
        f2acc_add_mulf(o, JC[i][3], a13);
        f2acc_add_mulf(o, JC[i][4], a14);
      } else if (l == 2) {
        o = f2acc_of(JC[i][2]);
        f2acc_add_mulf(o, JC[i][5], a25);
      } else {
        o = f2acc_of(JC[i][4]);
        f2acc_add_mulf(o, JC[i][3], a33);
      }
      f2acc_add_mulf(o, zz[i], v[l]);
      C[ci(R[i], R[l])] = f2acc_get(o);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    C[ci(3, R[i])] = JC[i][3];
    C[ci(5, R[i])] = JC[i][5];
  }
}

// The cached trigonometry of the state: cos/sin of phi (p[4]) and theta (p[5]).
struct InwardTrig {
  double cph, sph, cth, sth;
};

// step_to (dir < 0) with the state and path in FP64, the Jacobian's factors in
// FP32 from the FP64 crossing, and C in double-float; updates tr to the
// crossing.  Returns false when the surface is not reached.
__device__ __forceinline__ bool step_inward(const InwardHit& f, double p[6], f2 C[21], double ck, InwardTrig& tr) {
  const double rs = 1.0 / tr.sth;
  const double cot_t = tr.cth * rs;
  const double omega = ck * p[3];
  double s;
  if (f.kind == 0) {
    s = cylinder_path_inward(p[0], p[1], tr.cph, tr.sph, omega, f.pos);
  } else {
    s = (f.pos - p[2]) / cot_t;
    if (!(s < 0.0)) s = -INFINITY;
  }
  if (!(fabs(s) < INFINITY)) return false;
  const HelixPt<double> h = helix_at(p[0], p[1], p[2], p[4], tr.cph, tr.sph, cot_t, omega, s);
  // Jacobian factors (transport_jacobian) in FP32: A's free entries, v = dp/ds,
  // w = ds*/dp0; displacements are formed in FP64 before rounding
  const float fck = float(ck), fs = float(s), rsf = float(rs);
  const float inv_s2f = rsf * rsf;
  const float hx = float(h.x), hy = float(h.y), cph = float(h.cphi), sph = float(h.sphi);
  const float cotf = float(cot_t), omf = float(omega);
  const float a03 = fck * float(h.dx_dom), a04 = -float(h.y - p[1]);
  const float a13 = fck * float(h.dy_dom), a14 = float(h.x - p[0]);
  const float a25 = -fs * inv_s2f, a33 = fck * fs;
  const float v[4] = {cph, sph, cotf, omf};
  float w[6];
  if (f.kind == 0) {
    const float inv_ds = -1.0f / fmaf(hx, cph, hy * sph);
    w[0] = inv_ds * hx;
    w[1] = inv_ds * hy;
    w[2] = 0.0f;
    w[3] = inv_ds * fmaf(hx, a03, hy * a13);
    w[4] = inv_ds * fmaf(hx, a04, hy * a14);
    w[5] = 0.0f;
  } else {
    const float inv_ct = -1.0f / cotf;
    w[0] = w[1] = w[3] = w[4] = 0.0f;
    w[2] = inv_ct;
    w[5] = inv_ct * a25;
  }
  similarity_rank1_f2(a03, a04, a13, a14, a25, a33, v, w, C);
  p[0] = h.x;
  p[1] = h.y;
  p[2] = h.z;
  p[4] = wrap_phi(h.phi);
  tr.cph = h.cphi;
  tr.sph = h.sphi;
  if (f.x0 > 0.0f) {
    const float th2 = highland_theta0_sq(f.kind, f.x0, hx, hy, cph, sph, float(p[3]), float(tr.sth),
                                         float(tr.cth));
    const float pr = __fmul_rn(th2, inv_s2f);
    C[ci(4, 4)] = f2_add(C[ci(4, 4)], f2{pr, fmaf(th2, inv_s2f, -pr)});
    C[ci(5, 5)] = f2_add(C[ci(5, 5)], f2{th2, 0.0f});
  }
  return true;
}

// kf_update (plain form C - K B^T) with the covariance algebra in
// double-float and the residuals and the state in FP64.  The measurement rows
// are rounded to FP32 for the covariance (a frame turned by ~1e-8 rad, used
// consistently there); the residuals use the FP64 rows.  The state increment
// K r is formed in double-float and then added in FP64: in the early, weakly
// constrained updates its terms are large and nearly cancel, and an FP32
// increment put the curvature of short-lever-arm tracks 2e-4 off.  The chi2
// needs no more than FP32.  Returns the predicted chi2.
__device__ __forceinline__ double update_inward(const InwardHit& f, double p[6], f2 C[21]) {
  const int kind = f.kind;
  const Meas<double>& m = f.m;
  const float c = float(m.c), sn = float(m.s);
  f2 B[6][2];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    f2acc b0{0.0f, 0.0f};
    f2acc_add_mulf(b0, C[ci(i, 0)], -sn);
    f2acc_add_mulf(b0, C[ci(i, 1)], c);
    B[i][0] = f2acc_get(b0);
    if (kind == 0) {
      B[i][1] = C[ci(i, 2)];
    } else {
      f2acc b1{0.0f, 0.0f};
      f2acc_add_mulf(b1, C[ci(i, 0)], c);
      f2acc_add_mulf(b1, C[ci(i, 1)], sn);
      B[i][1] = f2acc_get(b1);
    }
  }
  f2acc raa{f.v00, 0.0f}, rab{f.v01, 0.0f}, rbb{f.v11, 0.0f};
  f2acc_add_mulf(raa, B[0][0], -sn);
  f2acc_add_mulf(raa, B[1][0], c);
  f2acc_add_mulf(rab, B[0][1], -sn);
  f2acc_add_mulf(rab, B[1][1], c);
  if (kind == 0) {
    const f2 b = B[2][1];
    f2acc_add_mulf(rbb, b, 1.0f);
  } else {
    f2acc_add_mulf(rbb, B[0][1], c);
    f2acc_add_mulf(rbb, B[1][1], sn);
  }
  const f2 Raa = f2acc_get(raa), Rab = f2acc_get(rab), Rbb = f2acc_get(rbb);
  f2acc dt{0.0f, 0.0f};
  f2acc_add_mul(dt, Raa, Rbb);
  f2acc_add_mul(dt, Rab, f2{-Rab.h, -Rab.l});
  const f2 idet = f2_recip(f2acc_get(dt));
  const f2 Waa = f2_mul(Rbb, idet), Wab = f2_mul(f2{-Rab.h, -Rab.l}, idet), Wbb = f2_mul(Raa, idet);
  // residuals in FP64
  const double ra = fma(m.s, p[0], -m.c * p[1]);
  const double rb = kind == 0 ? m.w - p[2] : m.w - fma(m.c, p[0], m.s * p[1]);
  const f2 ra2 = f2_of(ra), rb2 = f2_of(rb);
  const float raf = ra2.h, rbf = rb2.h;
  const float chi2 = fmaf(Waa.h * raf, raf, fmaf(2.0f * Wab.h * raf, rbf, Wbb.h * rbf * rbf));
  f2 Kg[6][2];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    f2acc k0{0.0f, 0.0f}, k1{0.0f, 0.0f};
    f2acc_add_mul(k0, B[i][0], Waa);
    f2acc_add_mul(k0, B[i][1], Wab);
    f2acc_add_mul(k1, B[i][0], Wab);
    f2acc_add_mul(k1, B[i][1], Wbb);
    Kg[i][0] = f2acc_get(k0);
    Kg[i][1] = f2acc_get(k1);
    // the two terms can be large and nearly cancel (early, weakly constrained
    // updates): the increment is formed in double-float, then widened
    f2acc dp{0.0f, 0.0f};
    f2acc_add_mul(dp, Kg[i][0], ra2);
    f2acc_add_mul(dp, Kg[i][1], rb2);
    const f2 d = f2acc_get(dp);
    p[i] += double(d.h) + double(d.l);
  }
  p[4] = wrap_phi(p[4]);
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      f2acc a = f2acc_of(C[ci(i, j)]);
      f2acc_add_mul(a, Kg[i][0], f2{-B[j][0].h, -B[j][0].l});
      f2acc_add_mul(a, Kg[i][1], f2{-B[j][1].h, -B[j][1].l});
      C[ci(i, j)] = f2acc_get(a);
    }
  return double(chi2);
}

// Inward fit: covariance reset to 100 x the seed-style diagonal, update with
// the outermost hit in place, then propagate inward hit by hit (state and
// transport in FP64, covariance in double-float, plain covariance update).
__global__ void k_fit_inward(const GeomDev* __restrict__ g, const float* __restrict__ xyz,
                             const float* __restrict__ lcov, const int* __restrict__ layer, int64_t H,
                             const int* __restrict__ hits, int K, const float* __restrict__ init_par, int64_t NT,
                             const float* __restrict__ align, const float* __restrict__ x0,
                             float* __restrict__ out_par, float* __restrict__ out_cov, float* __restrict__ out_chi2,
                             int* __restrict__ out_ok) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NT) return;
  const int* row = hits + t * K;
  double p[6];
  f2 C[21];
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = double(init_par[k * NT + t]);
#pragma unroll
  for (int k = 0; k < 21; ++k) C[k] = f2{0.0f, 0.0f};
  C[ci(0, 0)] = C[ci(1, 1)] = C[ci(2, 2)] = f2{1.0f, 0.0f};
  C[ci(3, 3)] = f2_of(100.0 * (0.05 * p[3]) * (0.05 * p[3]));
  C[ci(4, 4)] = C[ci(5, 5)] = f2{0.25f, 0.0f};
  const int last = prev_listed(row, K);
  double chi2 = 0.0;
  int ok = 1;
  const double ck = double(g->c_kappa);
  InwardTrig tr;
  sincos(p[4], &tr.sph, &tr.cph);
  sincos(p[5], &tr.sth, &tr.cth);
  InwardHit f;
  // each lane walks its own listed hits (prev_listed skips empty slots)
  for (int k = last; k >= 0; k = prev_listed(row, k)) {
    if (!load_inward_hit(g, xyz, lcov, layer, H, row[k], align, x0, f)) continue;
    if (k != last && !step_inward(f, p, C, ck, tr)) {
      ok = 0;
      break;
    }
    const double phi0 = p[4], theta0 = p[5];
    chi2 += update_inward(f, p, C);
    turn_by(wrap_phi(p[4] - phi0), p[4], tr.cph, tr.sph);
    turn_by(p[5] - theta0, p[5], tr.cth, tr.sth);
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) out_par[i * NT + t] = float(p[i]);
#pragma unroll
  for (int i = 0; i < 21; ++i) out_cov[i * NT + t] = __fadd_rn(C[i].h, C[i].l);
  out_chi2[t] = float(chi2);
  if (out_ok) out_ok[t] = ok;
}

}  // namespace

cudaError_t launch_fit(mkf_ctx* ctx, int direction, const float* xyz, const float* lcov, const int* layer,
                       int64_t n_hits, const int* hits, int K, const float* init_par, const float* init_cov,
                       int64_t n_tracks, const float* align, const float* x0, float* out_par, float* out_cov,
                       float* out_chi2, int* out_ok, float* ckpt, cudaStream_t st) {
  if (n_tracks == 0) return cudaSuccess;
  // one thread per track; small blocks when there are few tracks so that the
  // work spreads over every SM
  const int T = n_tracks >= (int64_t)ctx->n_sm * 128 ? 128 : (n_tracks >= (int64_t)ctx->n_sm * 64 ? 64 : 32);
  const int tid = direction > 0 ? kTFit : kTBackward;
  const unsigned grid = (unsigned)((n_tracks + T - 1) / T);
  ctx->tick(tid, st);
  if (direction > 0)
    k_fit<float><<<grid, T, 0, st>>>(ctx->geom_dev.as<GeomDev>(), xyz, lcov, layer, n_hits, hits, K, init_par,
                                     init_cov, n_tracks, align, x0, out_par, out_cov, out_chi2, out_ok, ckpt);
  else
    k_fit_inward<<<grid, T, 0, st>>>(ctx->geom_dev.as<GeomDev>(), xyz, lcov, layer, n_hits, hits, K, init_par,
                                     n_tracks, align, x0, out_par, out_cov, out_chi2, out_ok);
  ctx->tock(tid, st);
  return cudaGetLastError();
}

}  // namespace mkf
