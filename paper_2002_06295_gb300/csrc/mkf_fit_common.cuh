// mkf_fit_common.cuh -- pieces shared by the fit and its adjoint: a listed
// hit in its aligned local frame, and one outward/inward step onto its surface.
#pragma once
#include "mkf_device.cuh"
#include "mkf_internal.h"

namespace mkf {

// A listed hit plus the surface it sits on, after alignment:
// barrel: surface r_L + dr, hit azimuth + dphi, hit z + dz;
// disk:   surface z_L + dz, hit azimuth + dphi, hit r + dr.
template <class T> struct FitHit {
  int kind;
  int layer;
  T pos;      // surface r (barrel) or z (disk)
  T x0;       // thickness
  Meas<T> m;  // (cos phi_h, sin phi_h, z_h or r_h, V)
};

template <class T>
__device__ __forceinline__ bool load_fit_hit(const GeomDev* __restrict__ g, const float* __restrict__ xyz,
                                             const float* __restrict__ lcov, const int* __restrict__ layer,
                                             int64_t H, int h, const float* __restrict__ align,
                                             const float* __restrict__ x0, FitHit<T>& f) {
  if (h < 0 || h >= H) return false;
  const int l = layer[h];
  if (l < 0 || l >= g->n_layers) return false;
  const LayerDev ly = g->L[l];
  T dr(0.0), dphi(0.0), dz(0.0);
  if (align) {
    dr = T(align[3 * l]);
    dphi = T(align[3 * l + 1]);
    dz = T(align[3 * l + 2]);
  }
  const T x = T(xyz[h]), y = T(xyz[H + h]), z = T(xyz[2 * H + h]);
  const T r = msqrt(mfma(x, x, y * y));
  const T ir = T(1.0) / r;
  T sd(0.0), cd(1.0);
  if (align) msincos(dphi, &sd, &cd);
  f.kind = ly.kind;
  f.layer = l;
  f.pos = ly.kind == 0 ? T(ly.pos) + dr : T(ly.pos) + dz;
  f.x0 = x0 ? T(x0[l]) : T(ly.x0);
  f.m.c = (x * cd - y * sd) * ir;
  f.m.s = (x * sd + y * cd) * ir;
  f.m.w = ly.kind == 0 ? z + dz : r + dr;
  f.m.v00 = T(lcov[h]);
  f.m.v11 = T(lcov[H + h]);
  f.m.v01 = T(lcov[2 * H + h]);
  return true;
}

// Multiple scattering added to the transported covariance.  The term only adds
// to two diagonal entries, so its FP32 value (relative error ~1e-7) is as good
// as an FP64 one for an FP64 covariance, at a fraction of the FP64 work.
__device__ __forceinline__ void add_material_step(int kind, float x0, float x, float y, float cphi, float sphi,
                                                  float kappa, float sin_t, float cos_t, float C[21]) {
  add_material(kind, x0, x, y, cphi, sphi, kappa, sin_t, cos_t, C);
}
__device__ __forceinline__ void add_material_step(int kind, double x0, double x, double y, double cphi, double sphi,
                                                  double kappa, double sin_t, double cos_t, double C[21]) {
  if (!(x0 > 0.0)) return;
  const float st = float(sin_t);
  const float th2 = highland_theta0_sq(kind, float(x0), float(x), float(y), float(cphi), float(sphi), float(kappa), st,
                                       float(cos_t));
  C[ci(4, 4)] += double(th2) / (sin_t * sin_t);
  C[ci(5, 5)] += double(th2);
}

// Propagate (p, C) onto the hit's surface in direction dir and add its
// material.  Returns false when the surface is not reached.
template <class T> __device__ __forceinline__ bool step_to(const FitHit<T>& f, T p[6], T C[21], T ck, int dir) {
  T sin_t, cos_t;
  msincos(p[5], &sin_t, &cos_t);
  const T cot_t = cos_t / sin_t;
  const T omega = ck * p[3];
  T sph, cph;
  msincos(p[4], &sph, &cph);
  T s;
  if (f.kind == 0) {
    s = cylinder_path(p[0], p[1], cph, sph, omega, f.pos, dir);
  } else {
    s = plane_path(p[2], cot_t, f.pos, dir);
  }
  if (!(mabs(vv(s)) < INFINITY)) return false;
  const auto h = helix_at(p[0], p[1], p[2], p[4], cph, sph, cot_t, omega, s);
  const auto J = transport_jacobian(f.kind, p, h, s, omega, ck, cot_t, sin_t);
  similarity(J, C);
  p[0] = h.x;
  p[1] = h.y;
  p[2] = h.z;
  p[4] = wrap_phi(h.phi);
  add_material_step(f.kind, f.x0, h.x, h.y, h.cphi, h.sphi, p[3], sin_t, cos_t, C);
  return true;
}

}  // namespace mkf
