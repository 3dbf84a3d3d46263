// seed_oracle.cpp -- TEST INFRASTRUCTURE ONLY: plain FP64 reference of the
// hit-based seeding of prompt tracks from the four innermost barrel (pixel)
// layers (Sec. 3).  The paper names the layers and the prompt-track target
// only; the rules below are this project's reading, taken by the CUDA kernel
// too:
//  * radii R0 < R1 < R2 < R3 are the four innermost barrel layers; a hit is
//    its measured direction (x, y) / |(x, y)| on its layer's radius, and z;
//  * a pair (a on layer 0, b on layer 1) defines the circle through the
//    origin, a and b (signed curvature omega = 2 (A x B) / (|A| |B| |A - B|),
//    positive counter-clockwise), the transverse path s(r) = 2 asin(omega r /
//    2) / omega from the origin, and the line z = z0 + cot s through a and b;
//    it passes if |omega| <= omega_max = alpha Bz / pt_min and |z0| <= z_max;
//  * a hit c on layer 2 passes if, against that helix's point at R2, its
//    transverse residual R2 sin(phi_c - phi_pred) and z residual are within
//    rphi_tol and z_tol;
//  * the circle through the origin, a and c and the line through a and c
//    predict layer 3 the same way for a hit d;
//  * every hit after a must lie on the predicted side: b within 90 degrees of
//    a in azimuth, c and d within 90 degrees of their predictions (the sine
//    residual alone cannot tell a hit from its mirror image through the beam
//    line, and a pair on opposite sides of it defines a circle that does not
//    pass outward through both);
//  * the seed state is at the beam line (0, 0, z0): curvature and direction
//    from the circle through the origin, b and d, cot theta and z0 from the
//    line through a and d; kappa = -omega / (alpha Bz);
//  * a circle that does not reach R3 (|omega R3 / 2| >= 1) predicts nothing
//    (with |omega| <= omega_max and omega_max R3 / 2 < 1 this only happens
//    to circles through a far-off layer-2 or layer-3 hit).
// Every cut is reported as a margin 1 - |value| / limit (>= 0: passes), so a
// caller can tell quadruplets near a cut from the others.  All pairs are tried
// (no binning).  Shares no code with the CUDA library.
#include <cmath>
#include <cstdint>
#include <vector>

namespace {

constexpr double kAlpha = 0.00299792458;   // GeV / (T cm)

struct Hit {
  double c, s, z;
  int id;
};

double arc_s(double omega, double r) {
  const double x = 0.5 * omega * r;
  return std::fabs(x) < 1e-12 ? r : 2.0 * std::asin(x) / omega;
}

// signed curvature of the circle through the origin, A = ra (ca, sa) and B = rb (cb, sb)
double circle_origin(double ra, const Hit& a, double rb, const Hit& b) {
  const double cross = ra * rb * (a.c * b.s - a.s * b.c);
  const double dx = rb * b.c - ra * a.c, dy = rb * b.s - ra * a.s;
  return 2.0 * cross / (ra * rb * std::sqrt(dx * dx + dy * dy));
}

// Helix through the origin, a (on ra) and b (on rb): direction of its point at
// radius r (cos, sin) and its z there.
struct Pred {
  double c, s, z;
};
Pred predict(double omega, double ra, const Hit& a, double rb, const Hit& b, double r, double* z0_out) {
  const double sa = arc_s(omega, ra), sb = arc_s(omega, rb);
  const double cot = (b.z - a.z) / (sb - sa);
  const double z0 = a.z - cot * sa;
  if (z0_out) *z0_out = z0;
  const double d = std::asin(0.5 * omega * r) - std::asin(0.5 * omega * ra);
  const double cd = std::cos(d), sd = std::sin(d);
  return Pred{a.c * cd - a.s * sd, a.s * cd + a.c * sd, z0 + cot * arc_s(omega, r)};
}

double margin(double v, double limit) { return 1.0 - std::fabs(v) / limit; }

}  // namespace

// layers: the four seeding layer ids (innermost barrel first) and their radii.
// Outputs, up to max_out quadruplets whose smallest margin is >= -eps (the
// count returned may be larger): hits [n][4] caller ids, margin [n], par
// [n][6] (x, y, z, kappa, phi, theta).
extern "C" int64_t orc_seed_quads(const double* xyz, const int* layer, int64_t n_hits, const int64_t* ev_hit_off,
                                  int n_events, const int* seed_layers, const double* radii, double bz,
                                  double pt_min, double z_max, double rphi_tol, double z_tol, double eps,
                                  int64_t max_out, int* out_hits, double* out_margin, double* out_par,
                                  int* out_event) {
  const double omega_max = kAlpha * bz / pt_min;
  const double R0 = radii[0], R1 = radii[1], R2 = radii[2], R3 = radii[3];
  int64_t n_out = 0;
  for (int e = 0; e < n_events; ++e) {
    std::vector<Hit> on[4];
    for (int64_t h = ev_hit_off[e]; h < ev_hit_off[e + 1]; ++h)
      for (int k = 0; k < 4; ++k)
        if (layer[h] == seed_layers[k]) {
          const double x = xyz[3 * h], y = xyz[3 * h + 1], r = std::hypot(x, y);
          on[k].push_back(Hit{x / r, y / r, xyz[3 * h + 2], (int)(h - ev_hit_off[e])});
        }
    for (const Hit& a : on[0])
      for (const Hit& b : on[1]) {
        if (a.c * b.c + a.s * b.s <= 0.0) continue;   // opposite sides of the beam line
        const double omega = circle_origin(R0, a, R1, b);
        const double m1 = margin(omega, omega_max);
        if (m1 < -eps) continue;
        double z0;
        const Pred p2 = predict(omega, R0, a, R1, b, R2, &z0);
        const double m2 = margin(z0, z_max);
        if (m2 < -eps) continue;
        for (const Hit& c : on[2]) {
          if (c.c * p2.c + c.s * p2.s <= 0.0) continue;
          const double m3 = margin(R2 * (c.s * p2.c - c.c * p2.s), rphi_tol);
          const double m4 = margin(c.z - p2.z, z_tol);
          if (m3 < -eps || m4 < -eps) continue;
          const double omega2 = circle_origin(R0, a, R2, c);
          if (std::fabs(0.5 * omega2 * R3) >= 1.0) continue;   // that circle never reaches layer 3
          const Pred p3 = predict(omega2, R0, a, R2, c, R3, nullptr);
          for (const Hit& d : on[3]) {
            if (d.c * p3.c + d.s * p3.s <= 0.0) continue;
            const double m5 = margin(R3 * (d.s * p3.c - d.c * p3.s), rphi_tol);
            const double m6 = margin(d.z - p3.z, z_tol);
            const double m = std::fmin(std::fmin(std::fmin(m1, m2), std::fmin(m3, m4)), std::fmin(m5, m6));
            if (m < -eps) continue;
            const double w3 = circle_origin(R1, b, R3, d);
            if (std::fabs(0.5 * w3 * R3) >= 1.0) continue;
            if (n_out < max_out) {
              // seed state: circle through the origin, b and d; line through a and d
              const double pb = std::atan2(b.s, b.c);
              const double phi = std::remainder(pb - std::asin(0.5 * w3 * R1), 2.0 * M_PI);
              const double sa = arc_s(w3, R0), sd = arc_s(w3, R3);
              const double cot = (d.z - a.z) / (sd - sa);
              const double z0s = a.z - cot * sa;
              const int hs[4] = {a.id, b.id, c.id, d.id};
              for (int k = 0; k < 4; ++k) out_hits[4 * n_out + k] = (int)ev_hit_off[e] + hs[k];
              out_margin[n_out] = m;
              double* q = out_par + 6 * n_out;
              q[0] = 0.0;
              q[1] = 0.0;
              q[2] = z0s;
              q[3] = -w3 / (kAlpha * bz);
              q[4] = phi;
              q[5] = std::atan2(1.0, cot);
              out_event[n_out] = e;
            }
            ++n_out;
          }
        }
      }
  }
  return n_out;
}
