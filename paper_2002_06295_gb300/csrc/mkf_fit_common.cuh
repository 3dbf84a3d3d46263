// mkf_fit_common.cuh -- pieces shared by the fits, the overlap search and the
// fit adjoint: a listed hit in its aligned local frame, and one outward or
// inward step onto its surface with the covariance in U-D form.
#pragma once
#include "mkf_device.cuh"
#include "mkf_internal.h"
#include "mkf_ud.cuh"

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

// True when the outward transport from state p onto disk surface f spans a
// full turn of the helix or more (|s omega| >= 2 pi): a slow particle near
// theta = pi/2 that drifts from one endcap disk to the next over several
// turns.  Such a transport's Jacobian has entries that grow with the path
// (ds/dtheta ~ dz / cos^2 theta), and the fit's reverse sweep, which
// multiplies the covariance adjoint by J^T ... J at every step, loses all
// accuracy on it in FP32 (measured against the FP64 oracle on the tracks
// built on the CMS-like event: hit gradients wrong by up to 1e29 of the
// track's largest, four of them overflowing, while tracks below one turn
// agree within 1e-3).  The forward fit reports these tracks and the adjoint
// leaves them out; both evaluate this same expression on the same state.
// A barrel crossing is always the first one within a turn, so only disks can
// qualify.
__device__ __forceinline__ bool disk_multi_turn(const FitHit<float>& f, const float p[6], float ck) {
  if (f.kind != 1) return false;
  float sin_t, cos_t;
  msincos(p[5], &sin_t, &cos_t);
  const float cot_t = cos_t / sin_t;
  const float omega = ck * p[3];
  const float s = plane_path(p[2], cot_t, f.pos, +1);
  return s < INFINITY && fabsf(s * omega) >= kTwoPi;
}

// Propagate the state onto the hit's surface in direction dir, transporting
// the U-D factors of its covariance and adding the surface's multiple
// scattering (Highland, on phi and theta).  Returns false when the surface is
// not reached.
__device__ __forceinline__ bool step_to_ud(const FitHit<float>& f, float p[6], UD6& u, float ck, int dir) {
  float sin_t, cos_t;
  msincos(p[5], &sin_t, &cos_t);
  const float cot_t = cos_t / sin_t;
  const float omega = ck * p[3];
  float sph, cph;
  msincos(p[4], &sph, &cph);
  const float s = f.kind == 0 ? cylinder_path(p[0], p[1], cph, sph, omega, f.pos, dir)
                              : plane_path(p[2], cot_t, f.pos, dir);
  if (!(fabsf(s) < INFINITY)) return false;
  const auto h = helix_at(p[0], p[1], p[2], p[4], cph, sph, cot_t, omega, s);
  const auto J = transport_jacobian(f.kind, p, h, s, omega, ck, cot_t, sin_t);
  float q_phi = 0.0f, q_theta = 0.0f;
  if (f.x0 > 0.0f) {
    q_theta = highland_theta0_sq(f.kind, f.x0, h.x, h.y, h.cphi, h.sphi, p[3], sin_t, cos_t);
    q_phi = q_theta / (sin_t * sin_t);
  }
  ud_transport(J, u, q_phi, q_theta);
  p[0] = h.x;
  p[1] = h.y;
  p[2] = h.z;
  p[4] = wrap_phi(h.phi);
  return true;
}

}  // namespace mkf
