// fit.cu -- Kalman fit over a fixed hit assignment (Sec. 1: fitting applies
// the KF procedure to all hits found in building), outward and inward.
// One thread per track; the state stays in registers for all its hits.
//
// The outward fit runs in FP32 with the covariance in U-D factorised form
// (mkf_ud.cuh), which keeps the small conditional variances that pixel hits
// and strip disks leave.  The inward fit starts from a prior 100 times wider
// than the seed's, so its first updates shrink variances by factors up to 1e5
// and, on built tracks that carry wrong picks, move the state by hundreds of
// standard deviations: an FP32 state (with U-D factors) then ends up to 0.3 of
// its curvature away from FP64, so the inward fit runs in FP64.
#include "mkf_device.cuh"
#include "mkf_fit_common.cuh"
#include "mkf_ud.cuh"
#include "mkf_internal.h"

namespace mkf {

namespace {

__global__ void k_fit(const GeomDev* __restrict__ g, const float* __restrict__ xyz, const float* __restrict__ lcov,
                      const int* __restrict__ layer, int64_t H, const int* __restrict__ hits, int K,
                      const float* __restrict__ init_par, const float* __restrict__ init_cov, int64_t NT,
                      const float* __restrict__ align, const float* __restrict__ x0, float* __restrict__ out_par,
                      float* __restrict__ out_cov, float* __restrict__ out_chi2, int* __restrict__ out_ok,
                      float* __restrict__ ckpt) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NT) return;
  const float ck = g->c_kappa;
  float p[6], C[21];
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = init_par[k * NT + t];
#pragma unroll
  for (int k = 0; k < 21; ++k) C[k] = init_cov[k * NT + t];
  UD6 u;
  ud_from_cov(C, u);
  float chi2 = 0.0f;
  int ok = 1;
  const int* row = hits + t * K;
  for (int k = 0; k < K; ++k) {
    if (ckpt) {
      // the adjoint recomputes each step from the state before it, in the
      // plain covariance form: checkpoint k holds p and C = U D U^T
      float* c = ckpt + (size_t)k * 27 * NT + t;
#pragma unroll
      for (int i = 0; i < 6; ++i) c[i * NT] = p[i];
      if (k == 0) {
#pragma unroll
        for (int i = 0; i < 21; ++i) c[(6 + i) * NT] = init_cov[i * NT + t];
      } else {
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
          for (int j = 0; j <= i; ++j) c[(6 + ci(i, j)) * NT] = ud_cov_entry(u, i, j);
      }
    }
    FitHit<float> f;
    if (!load_fit_hit(g, xyz, lcov, layer, H, row[k], align, x0, f)) continue;
    if (ok == 1 && disk_multi_turn(f, p, ck)) ok = 2;
    if (!step_to_ud(f, p, u, ck, +1)) {
      ok = 0;
      // mark the steps that did not happen (x = NaN) for the adjoint
      if (ckpt)
        for (int k2 = k; k2 < K; ++k2) ckpt[(size_t)k2 * 27 * NT + t] = __int_as_float(0x7fc00000);
      break;
    }
    chi2 += ud_update(f.kind, p, u, f.m);
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) out_par[k * NT + t] = p[k];
  ud_to_cov(u, C);
#pragma unroll
  for (int k = 0; k < 21; ++k) out_cov[k * NT + t] = C[k];
  out_chi2[t] = chi2;
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
//  * J C J^T uses the rank-one form of the Jacobian (similarity_rank1).

struct InwardHit {
  int kind;
  double pos;     // surface r (barrel) or z (disk), aligned
  float x0;       // thickness
  Meas<double> m;
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
  f.m.v00 = double(lcov[h]);
  f.m.v11 = double(lcov[H + h]);
  f.m.v01 = double(lcov[2 * H + h]);
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

// C <- J C J^T for J = A + v w^T on the rows (x, y, z, phi), kappa and theta
// rows the identity.  With u = C w: J C = A C + v u^T and
// J C J^T = (J C) A^T + z v^T with z = J C w = A u + (w.u) v.  A's fixed ones
// and zeros (transport_jacobian) leave 139 FMAs instead of the dense 204.
__device__ __forceinline__ void similarity_rank1(double a03, double a04, double a13, double a14, double a25,
                                                 double a33, const double v[4], const double w[6], double C[21]) {
  double u[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double acc = C[ci(k, 0)] * w[0];
#pragma unroll
    for (int j = 1; j < 6; ++j) acc = fma(C[ci(k, j)], w[j], acc);
    u[k] = acc;
  }
  double JC[4][6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    JC[0][j] = fma(v[0], u[j], fma(a04, C[ci(4, j)], fma(a03, C[ci(3, j)], C[ci(0, j)])));
    JC[1][j] = fma(v[1], u[j], fma(a14, C[ci(4, j)], fma(a13, C[ci(3, j)], C[ci(1, j)])));
    JC[2][j] = fma(v[2], u[j], fma(a25, C[ci(5, j)], C[ci(2, j)]));
    JC[3][j] = fma(v[3], u[j], fma(a33, C[ci(3, j)], C[ci(4, j)]));
  }
  double wu = u[0] * w[0];
#pragma unroll
  for (int j = 1; j < 6; ++j) wu = fma(u[j], w[j], wu);
  double zz[4];
  zz[0] = fma(wu, v[0], fma(a04, u[4], fma(a03, u[3], u[0])));
  zz[1] = fma(wu, v[1], fma(a14, u[4], fma(a13, u[3], u[1])));
  zz[2] = fma(wu, v[2], fma(a25, u[5], u[2]));
  zz[3] = fma(wu, v[3], fma(a33, u[3], u[4]));
  constexpr int R[4] = {0, 1, 2, 4};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    // (J C A^T)[i][l] for the rows l <= i, plus z_i v_l
    const double o0 = fma(zz[i], v[0], fma(a04, JC[i][4], fma(a03, JC[i][3], JC[i][0])));
    const double o1 = fma(zz[i], v[1], fma(a14, JC[i][4], fma(a13, JC[i][3], JC[i][1])));
    const double o2 = fma(zz[i], v[2], fma(a25, JC[i][5], JC[i][2]));
    const double o3 = fma(zz[i], v[3], fma(a33, JC[i][3], JC[i][4]));
    const double o[4] = {o0, o1, o2, o3};
#pragma unroll
    for (int l = 0; l <= i; ++l) C[ci(R[i], R[l])] = o[l];
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

// step_to (dir < 0) in FP64 with the cached trigonometry; updates tr to the
// crossing.  Returns false when the surface is not reached.
__device__ __forceinline__ bool step_inward(const InwardHit& f, double p[6], double C[21], double ck, InwardTrig& tr) {
  const double rs = 1.0 / tr.sth;
  const double cot_t = tr.cth * rs, inv_s2 = rs * rs;
  const double omega = ck * p[3];
  double s, ict = 0.0;
  if (f.kind == 0) {
    s = cylinder_path_inward(p[0], p[1], tr.cph, tr.sph, omega, f.pos);
  } else {
    ict = 1.0 / cot_t;
    s = (f.pos - p[2]) * ict;
    if (!(s < 0.0)) s = -INFINITY;
  }
  if (!(fabs(s) < INFINITY)) return false;
  const HelixPt<double> h = helix_at(p[0], p[1], p[2], p[4], tr.cph, tr.sph, cot_t, omega, s);
  // Jacobian factors (transport_jacobian): A's free entries, v = dp/ds, w = ds*/dp0
  const double a03 = ck * h.dx_dom, a04 = -(h.y - p[1]);
  const double a13 = ck * h.dy_dom, a14 = h.x - p[0];
  const double a25 = -s * inv_s2, a33 = ck * s;
  const double v[4] = {h.cphi, h.sphi, cot_t, omega};
  double w[6];
  if (f.kind == 0) {
    const double inv_ds = -1.0 / fma(h.x, h.cphi, h.y * h.sphi);
    w[0] = inv_ds * h.x;
    w[1] = inv_ds * h.y;
    w[2] = 0.0;
    w[3] = inv_ds * fma(h.x, a03, h.y * a13);
    w[4] = inv_ds * fma(h.x, a04, h.y * a14);
    w[5] = 0.0;
  } else {
    w[0] = w[1] = w[3] = w[4] = 0.0;
    w[2] = -ict;
    w[5] = -ict * a25;
  }
  similarity_rank1(a03, a04, a13, a14, a25, a33, v, w, C);
  p[0] = h.x;
  p[1] = h.y;
  p[2] = h.z;
  p[4] = wrap_phi(h.phi);
  tr.cph = h.cphi;
  tr.sph = h.sphi;
  if (f.x0 > 0.0f) {
    const float th2 = highland_theta0_sq(f.kind, f.x0, float(h.x), float(h.y), float(h.cphi), float(h.sphi),
                                         float(p[3]), float(tr.sth), float(tr.cth));
    C[ci(4, 4)] = fma(double(th2), inv_s2, C[ci(4, 4)]);
    C[ci(5, 5)] += double(th2);
  }
  return true;
}

// Inward fit of track t: covariance reset to 100 x the seed-style diagonal,
// update with the outermost hit in place, then propagate inward hit by hit
// (FP64, plain covariance update).
__device__ __forceinline__ void fit_inward_track(const GeomDev* __restrict__ g, const float* __restrict__ xyz,
                                                 const float* __restrict__ lcov, const int* __restrict__ layer,
                                                 int64_t H, const int* __restrict__ hits, int K,
                                                 const float* __restrict__ init_par, int64_t NT,
                                                 const float* __restrict__ align, const float* __restrict__ x0,
                                                 float* __restrict__ out_par, float* __restrict__ out_cov,
                                                 float* __restrict__ out_chi2, int* __restrict__ out_ok, int64_t t) {
  const int* row = hits + t * K;
  double p[6], C[21];
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = double(init_par[k * NT + t]);
#pragma unroll
  for (int k = 0; k < 21; ++k) C[k] = 0.0;
  C[ci(0, 0)] = C[ci(1, 1)] = C[ci(2, 2)] = 1.0;
  C[ci(3, 3)] = 100.0 * (0.05 * p[3]) * (0.05 * p[3]);
  C[ci(4, 4)] = C[ci(5, 5)] = 0.25;
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
    chi2 += kf_update<double, false>(f.kind, p, C, f.m);
    turn_by(wrap_phi(p[4] - phi0), p[4], tr.cph, tr.sph);
    turn_by(p[5] - theta0, p[5], tr.cth, tr.sth);
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) out_par[i * NT + t] = float(p[i]);
#pragma unroll
  for (int i = 0; i < 21; ++i) out_cov[i * NT + t] = float(C[i]);
  out_chi2[t] = float(chi2);
  if (out_ok) out_ok[t] = ok;
}

// Inward fit of the tracks t, t + (threads of the grid), ... (the launch caps
// the grid at two blocks per SM when there are many tracks).  Bounded to 128
// registers (no spills), so two blocks leave room for two of the adjoint's.
__global__ void __launch_bounds__(128, 4)
    k_fit_inward(const GeomDev* __restrict__ g, const float* __restrict__ xyz, const float* __restrict__ lcov,
                 const int* __restrict__ layer, int64_t H, const int* __restrict__ hits, int K,
                 const float* __restrict__ init_par, int64_t NT, const float* __restrict__ align,
                 const float* __restrict__ x0, float* __restrict__ out_par, float* __restrict__ out_cov,
                 float* __restrict__ out_chi2, int* __restrict__ out_ok) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < NT; t += (int64_t)gridDim.x * blockDim.x)
    fit_inward_track(g, xyz, lcov, layer, H, hits, K, init_par, NT, align, x0, out_par, out_cov, out_chi2, out_ok, t);
}

}  // namespace

constexpr unsigned kInwardBlocksPerSm = 2;

cudaError_t launch_fit(mkf_ctx* ctx, int direction, const float* xyz, const float* lcov, const int* layer,
                       int64_t n_hits, const int* hits, int K, const float* init_par, const float* init_cov,
                       int64_t n_tracks, const float* align, const float* x0, float* out_par, float* out_cov,
                       float* out_chi2, int* out_ok, float* ckpt, cudaStream_t st) {
  if (n_tracks == 0) return cudaSuccess;
  // one thread per track; small blocks when there are few tracks so that the
  // work spreads over every SM
  const int T = n_tracks >= (int64_t)ctx->n_sm * 128 ? 128 : (n_tracks >= (int64_t)ctx->n_sm * 64 ? 64 : 32);
  const int tid = direction > 0 ? kTFit : kTBackward;
  unsigned grid = (unsigned)((n_tracks + T - 1) / T);
  // The inward fit is bound by the FP64 unit of each SM sub-partition (a
  // warp-wide FP64 instruction holds it for ~67 cycles).  With many tracks,
  // two 128-thread blocks per SM loop over them: one warp per sub-partition
  // leaves the unit idle while it waits on loads (the inward fit took twice as
  // long on a 256-event batch), while one thread per track fills every SM's
  // registers (three blocks of the former 140-register kernel, four now) and
  // leaves little room for the adjoint that runs beside it on another stream;
  // two leave room for two of its blocks (whole step on that batch -2 %, on 64
  // events of 10000 tracks -2 %).
  if (direction < 0 && T == 128) {
    const unsigned cap = (unsigned)ctx->n_sm * kInwardBlocksPerSm;
    if (grid > cap) grid = cap;
  }
  ctx->tick(tid, st);
  if (direction > 0)
    k_fit<<<grid, T, 0, st>>>(ctx->geom_dev.as<GeomDev>(), xyz, lcov, layer, n_hits, hits, K, init_par,
                                     init_cov, n_tracks, align, x0, out_par, out_cov, out_chi2, out_ok, ckpt);
  else
    k_fit_inward<<<grid, T, 0, st>>>(ctx->geom_dev.as<GeomDev>(), xyz, lcov, layer, n_hits, hits, K, init_par,
                                     n_tracks, align, x0, out_par, out_cov, out_chi2, out_ok);
  ctx->tock(tid, st);
  return cudaGetLastError();
}

}  // namespace mkf
