// fit_adjoint.cu -- reverse-mode derivative of the outward Kalman fit (not in
// the paper).  Gradient of
//   loss = sum_t g_chi2[t] chi2_t + g_par[.][t] . p_t + g_cov[.][t] . C_t
// with respect to hit positions, per-layer alignment (dr, dphi, dz) and
// per-layer thickness.
//
// One thread per track, or a group of 8 lanes per track when there are few
// tracks (lane e then runs dual pass e of steps (2) and (4) below and the
// lanes exchange the results by shuffles; everything else is computed by every
// lane of the group, so each track's contribution is the same bit for bit),
// sweeps the track's steps backwards.  Each step is recomputed
// from the checkpoint written by the forward fit (state before the step),
// then the adjoint is pushed back through
//   (1) the Kalman update  p_k = p + K r, C_k = C - B W B^T, chi2 = r^T W r
//       with B = C H^T, W = (V + H B)^-1, K = B W  (hand-written matrix calculus);
//   (2) the material term  C += diag(theta0^2 / sin^2 theta, theta0^2) on
//       (phi, theta), differentiated by forward-mode dual numbers;
//   (3) the covariance transport C_1 = J C_0 J^T:  G_0 = J^T G_1 J and
//       J_bar = 2 G_1 J C_0;
//   (4) the propagation p = P(p_0, surface), whose Jacobian J itself depends
//       on p_0 and on the surface position: dual-number passes give
//       dP/d(p_0, surface) and dJ/d(p_0, surface) for the contraction with J_bar;
//   (5) the hit's local frame (azimuth, z or r) and the surface position,
//       back to hit x, y, z and the layer's alignment.
// Covariance adjoints use the full symmetric-matrix convention
// dL = sum_ij G_ij dC_ij, stored as the packed lower triangle.
#include "mkf_device.cuh"
#include "mkf_dual.cuh"
#include "mkf_fit_common.cuh"
#include "mkf_internal.h"

namespace mkf {

namespace {

constexpr int kAdjThreads = 128;

__device__ __forceinline__ float Gf(const float G[21], int i, int j) { return G[ci(i, j)]; }

// derivative of g44 C_phiphi + g55 C_thetatheta (material term) along input w_
// of theta0^2: pp x (0), y (1), kappa (3), phi (4), theta (5), thickness (6)
__device__ __forceinline__ float material_pass(int w_, const float pp[6], const FitHit<float>& f, float g44,
                                               float g55) {
  DF X(pp[0], w_ == 0 ? 1.f : 0.f), Y(pp[1], w_ == 1 ? 1.f : 0.f), KA(pp[3], w_ == 3 ? 1.f : 0.f);
  DF PH(pp[4], w_ == 4 ? 1.f : 0.f), TH(pp[5], w_ == 5 ? 1.f : 0.f), X0(f.x0, w_ == 6 ? 1.f : 0.f);
  DF sp, cph, st, ct;
  msincos(PH, &sp, &cph);
  msincos(TH, &st, &ct);
  const DF th2 = highland_theta0_sq(f.kind, X0, X, Y, cph, sp, KA, st, ct);
  const DF q44 = th2 / (st * st);
  return fmaf(g44, q44.d, g55 * th2.d);
}

// p0bar_e = sum_i ppbar_i dpp_i/de + sum Jbar . dJ/de along input e of the
// propagation: p0[0..5] (e < 6) or the surface position (e = 6)
__device__ __forceinline__ float prop_pass(int e, const float p0[6], const FitHit<float>& f, float ck,
                                           const float ppb[6], const float Jb[4][6]) {
  DF q[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) q[i] = DF(p0[i], e == i ? 1.f : 0.f);
  const DF posd(f.pos, e == 6 ? 1.f : 0.f);
  DF st, ct;
  msincos(q[5], &st, &ct);
  const DF cot = ct / st;
  const DF om = DF(ck) * q[3];
  DF sph, cph;
  msincos(q[4], &sph, &cph);
  DF sd;
  if (f.kind == 0) {
    sd = cylinder_path(q[0], q[1], cph, sph, om, posd, +1);
  } else {
    sd = plane_path(q[2], cot, posd, +1);
  }
  const auto hd = helix_at(q[0], q[1], q[2], q[4], cph, sph, cot, om, sd);
  const auto Jd = transport_jacobian(f.kind, q, hd, sd, om, DF(ck), cot, st);
  float acc_e = fmaf(ppb[0], hd.x.d, fmaf(ppb[1], hd.y.d, fmaf(ppb[2], hd.z.d, ppb[4] * hd.phi.d)));
  if (e == 3) acc_e += ppb[3];
  if (e == 5) acc_e += ppb[5];
#pragma unroll
  for (int qq = 0; qq < 4; ++qq)
#pragma unroll
    for (int j = 0; j < 6; ++j) acc_e = fmaf(Jb[qq][j], Jd.r[qq][j].d, acc_e);
  return acc_e;
}

// The listed slot before slot k of a track's hit row (-1 when there is none).
__device__ __forceinline__ int prev_listed(const int* __restrict__ row, int k) {
  do {
    --k;
  } while (k >= 0 && row[k] < 0);
  return k;
}

// Four 128-thread blocks per SM (128 registers a thread, a few spilled): the
// extra warps hide more latency than the spills cost (C3 adjoint -11 %).
template <int LPT>
__global__ void __launch_bounds__(kAdjThreads, 4)
    k_fit_adjoint(const GeomDev* __restrict__ g, const float* __restrict__ xyz, const float* __restrict__ lcov,
                  const int* __restrict__ layer, int64_t H, const int* __restrict__ hits, int K, int64_t NT,
                  const float* __restrict__ align, const float* __restrict__ x0, const float* __restrict__ ckpt,
                  const float* __restrict__ g_chi2, const float* __restrict__ g_par, const float* __restrict__ g_cov,
                  float* __restrict__ g_hit, float* __restrict__ g_align, float* __restrict__ g_x0) {
  __shared__ float acc[MKF_MAX_LAYERS * 4];   // per-block (dr, dphi, dz, x0) sums
  const int L = g->n_layers;
  for (int i = threadIdx.x; i < L * 4; i += blockDim.x) acc[i] = 0.0f;
  __syncthreads();
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPT;
  const int sub = threadIdx.x % LPT;                         // lane in the track's group
  const int gbase = (threadIdx.x & 31) - sub;
  const unsigned gm = LPT == 32 ? 0xffffffffu : ((1u << LPT) - 1u) << gbase;
  if (t < NT) {
    const float ck = g->c_kappa;
    float pb[6], G[21];
#pragma unroll
    for (int k = 0; k < 6; ++k) pb[k] = g_par ? g_par[k * NT + t] : 0.0f;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) {
        const float gc = g_cov ? g_cov[ci(i, j) * NT + t] : 0.0f;
        G[ci(i, j)] = i == j ? gc : 0.5f * gc;
      }
    const float chib = g_chi2 ? g_chi2[t] : 0.0f;
    const int* row = hits + t * K;
    // A track with a transport to a disk that spans a full turn of the helix
    // or more (disk_multi_turn, the forward fit's out_ok = 2) is left out:
    // the reverse sweep is not accurate there.  The test reads the same
    // checkpointed state as the forward fit did; steps that did not happen
    // (x = NaN) end the scan.
    bool multi_turn = false;
    for (int k = 0; k < K && !multi_turn; ++k) {
      const int h = row[k];
      if (h < 0 || h >= H) continue;
      const int l = layer[h];
      if (l < 0 || l >= L || g->L[l].kind != 1) continue;
      FitHit<float> f;
      if (!load_fit_hit(g, xyz, lcov, layer, H, h, align, x0, f)) continue;
      const float* cp = ckpt + (size_t)k * 27 * NT + t;
      float pk[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) pk[i] = cp[i * NT];
      if (!(pk[0] == pk[0])) break;
      multi_turn = disk_multi_turn(f, pk, ck);
    }
    if (multi_turn) row = nullptr;
    // The group walks its track's listed hits only (prev_listed skips the
    // empty slots), so a warp runs the body once per hit of its longest track
    // rather than once per slot.
    for (int k = row ? prev_listed(row, K) : -1; k >= 0; k = prev_listed(row, k)) {
      const int h = row[k];
      FitHit<float> f;
      if (!load_fit_hit(g, xyz, lcov, layer, H, h, align, x0, f)) continue;
      const float* cp = ckpt + (size_t)k * 27 * NT + t;
      float p0[6], C0[21];
#pragma unroll
      for (int i = 0; i < 6; ++i) p0[i] = cp[i * NT];
      if (!(p0[0] == p0[0])) continue;   // the forward fit stopped before this step
#pragma unroll
      for (int i = 0; i < 21; ++i) C0[i] = cp[(6 + i) * NT];

      // ---------------- forward recompute of the step
      float sin_t, cos_t;
      msincos(p0[5], &sin_t, &cos_t);
      const float cot_t = cos_t / sin_t;
      const float omega = ck * p0[3];
      float sph, cph;
      msincos(p0[4], &sph, &cph);
      float s;
      if (f.kind == 0) {
        s = cylinder_path(p0[0], p0[1], cph, sph, omega, f.pos, +1);
      } else {
        s = plane_path(p0[2], cot_t, f.pos, +1);
      }
      if (!(fabsf(s) < INFINITY)) continue;
      const auto hp = helix_at(p0[0], p0[1], p0[2], p0[4], cph, sph, cot_t, omega, s);
      const auto J4 = transport_jacobian(f.kind, p0, hp, s, omega, ck, cot_t, sin_t);
      float C2[21];
#pragma unroll
      for (int i = 0; i < 21; ++i) C2[i] = C0[i];
      similarity(J4, C2);
      const float pp[6] = {hp.x, hp.y, hp.z, p0[3], wrap_phi(hp.phi), p0[5]};
      const bool mat = f.x0 > 0.0f;
      if (mat) add_material(f.kind, f.x0, hp.x, hp.y, hp.cphi, hp.sphi, p0[3], sin_t, cos_t, C2);
      // update quantities
      const Meas<float>& m = f.m;
      float Hm[2][3] = {{-m.s, m.c, 0.f}, {f.kind == 0 ? 0.f : m.c, f.kind == 0 ? 0.f : m.s, f.kind == 0 ? 1.f : 0.f}};
      float B[6][2];
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int a = 0; a < 2; ++a) B[i][a] = fmaf(Hm[a][0], C2[ci(i, 0)], fmaf(Hm[a][1], C2[ci(i, 1)], Hm[a][2] * C2[ci(i, 2)]));
      float r[2];
      r[0] = fmaf(m.s, pp[0], -m.c * pp[1]);
      r[1] = m.w - fmaf(Hm[1][0], pp[0], fmaf(Hm[1][1], pp[1], Hm[1][2] * pp[2]));
      float R00 = fmaf(Hm[0][0], B[0][0], fmaf(Hm[0][1], B[1][0], Hm[0][2] * B[2][0])) + m.v00;
      float R01 = fmaf(Hm[0][0], B[0][1], fmaf(Hm[0][1], B[1][1], Hm[0][2] * B[2][1])) + m.v01;
      float R11 = fmaf(Hm[1][0], B[0][1], fmaf(Hm[1][1], B[1][1], Hm[1][2] * B[2][1])) + m.v11;
      const float idet = 1.0f / fmaf(R00, R11, -R01 * R01);
      const float W[2][2] = {{R11 * idet, -R01 * idet}, {-R01 * idet, R00 * idet}};
      float Kg[6][2];
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int a = 0; a < 2; ++a) Kg[i][a] = fmaf(B[i][0], W[0][a], B[i][1] * W[1][a]);
      const float Wr[2] = {fmaf(W[0][0], r[0], W[0][1] * r[1]), fmaf(W[1][0], r[0], W[1][1] * r[1])};

      // ---------------- (1) reverse of the Kalman update
      float rb[2];
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        float acc_r = 2.0f * chib * Wr[a];
#pragma unroll
        for (int i = 0; i < 6; ++i) acc_r = fmaf(Kg[i][a], pb[i], acc_r);
        rb[a] = acc_r;
      }
      float GB[6][2];   // G B with G the full symmetric adjoint of C_k
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          float s2 = 0.f;
#pragma unroll
          for (int j = 0; j < 6; ++j) s2 = fmaf(Gf(G, i, j), B[j][a], s2);
          GB[i][a] = s2;
        }
      // Bbar = -2 G B W + Kbar W,  Kbar = pb r^T
      float Bb[6][2];
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          float s2 = 0.f;
#pragma unroll
          for (int c = 0; c < 2; ++c) s2 = fmaf(fmaf(-2.0f, GB[i][c], pb[i] * r[c]), W[c][a], s2);
          Bb[i][a] = s2;
        }
      // Wbar = -B^T G B + B^T Kbar + chib r r^T, symmetrised
      float Wb[2][2];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          float s2 = chib * r[a] * r[b];
#pragma unroll
          for (int i = 0; i < 6; ++i) s2 = fmaf(B[i][a], pb[i] * r[b] - GB[i][b], s2);
          Wb[a][b] = s2;
        }
      const float ws01 = 0.5f * (Wb[0][1] + Wb[1][0]);
      const float Wbs[2][2] = {{Wb[0][0], ws01}, {ws01, Wb[1][1]}};
      // Rbar = -W Wbar W
      float T2[2][2], Rb[2][2];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) T2[a][b] = fmaf(W[a][0], Wbs[0][b], W[a][1] * Wbs[1][b]);
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) Rb[a][b] = -fmaf(T2[a][0], W[0][b], T2[a][1] * W[1][b]);
      // R = V + H B: Bbar += H^T Rbar, Hbar = Rbar B^T (position columns only)
      float Hb[2][3];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j) Hb[a][j] = fmaf(Rb[a][0], B[j][0], Rb[a][1] * B[j][1]);
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int b = 0; b < 2; ++b) Bb[j][b] = fmaf(Hm[0][j], Rb[0][b], fmaf(Hm[1][j], Rb[1][b], Bb[j][b]));
      // B = C2 H^T: G2 = G + sym(Bbar H), Hbar += Bbar^T C2
      float G2[21];
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
          float bh_ij = 0.f, bh_ji = 0.f;
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            if (j < 3) bh_ij = fmaf(Bb[i][b], Hm[b][j], bh_ij);
            if (i < 3) bh_ji = fmaf(Bb[j][b], Hm[b][i], bh_ji);
          }
          G2[ci(i, j)] = G[ci(i, j)] + 0.5f * (bh_ij + bh_ji);
        }
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          float s2 = Hb[b][j];
#pragma unroll
          for (int i = 0; i < 6; ++i) s2 = fmaf(Bb[i][b], C2[ci(i, j)], s2);
          Hb[b][j] = s2;
        }
      // r = m - H pp: ppbar = pb - H^T rbar, Hbar -= rbar pp^T, wbar = rbar_b
      float ppb[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) ppb[j] = pb[j];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        ppb[j] -= fmaf(Hm[0][j], rb[0], Hm[1][j] * rb[1]);
#pragma unroll
        for (int a = 0; a < 2; ++a) Hb[a][j] = fmaf(-rb[a], pp[j], Hb[a][j]);
      }
      const float wb = rb[1];
      float cbar = Hb[0][1], sbar = -Hb[0][0];
      if (f.kind == 1) {
        cbar += Hb[1][0];
        sbar += Hb[1][1];
      }

      // ---------------- (2) reverse of the material term (dual passes)
      float x0b = 0.f;
      if (mat) {
        const float g44 = G2[ci(4, 4)], g55 = G2[ci(5, 5)];
        constexpr int kIn[6] = {0, 1, 3, 4, 5, 6};
        if (LPT == 1) {
          // one copy of the dual pass, run six times: six inlined copies made
          // the kernel's code large enough to stall on instruction fetch
#pragma unroll 1
          for (int e = 0; e < 6; ++e) {
            const int w_ = e + (e >= 2 ? 1 : 0);   // x, y, kappa, phi, theta, thickness
            const float dF = material_pass(w_, pp, f, g44, g55);
            if (w_ == 6) x0b = dF;
#pragma unroll
            for (int j = 0; j < 6; ++j)
              if (j == w_) ppb[j] += dF;
          }
        } else {
          const float dF = material_pass(kIn[sub < 6 ? sub : 0], pp, f, g44, g55);
#pragma unroll
          for (int e = 0; e < 6; ++e) {
            const float v = __shfl_sync(gm, dF, gbase + e);
            if (kIn[e] == 6)
              x0b = v;
            else
              ppb[kIn[e]] += v;
          }
        }
      }

      // ---------------- (3) reverse of C1 = J C0 J^T
      // full J rows: 0,1,2,4 from J4; rows 3 and 5 are unit vectors
      float Jf[6][6];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        Jf[0][j] = J4.r[0][j];
        Jf[1][j] = J4.r[1][j];
        Jf[2][j] = J4.r[2][j];
        Jf[4][j] = J4.r[3][j];
        Jf[3][j] = j == 3 ? 1.f : 0.f;
        Jf[5][j] = j == 5 ? 1.f : 0.f;
      }
      float M[6][6];   // G2 J
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int l = 0; l < 6; ++l) {
          float s2 = 0.f;
#pragma unroll
          for (int j = 0; j < 6; ++j) s2 = fmaf(Gf(G2, i, j), Jf[j][l], s2);
          M[i][l] = s2;
        }
      float Gn[21];   // J^T G2 J
#pragma unroll
      for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
          float s2 = 0.f;
#pragma unroll
          for (int i = 0; i < 6; ++i) s2 = fmaf(Jf[i][a], M[i][b], s2);
          Gn[ci(a, b)] = s2;
        }
      // Jbar = 2 G2 J C0 on the rows that depend on p0 and the surface (x, y, z, phi)
      constexpr int kRow[4] = {0, 1, 2, 4};
      float Jb[4][6];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          float s2 = 0.f;
#pragma unroll
          for (int l = 0; l < 6; ++l) s2 = fmaf(M[kRow[q]][l], C0[ci(l, j)], s2);
          Jb[q][j] = 2.0f * s2;
        }

      // ---------------- (4) reverse of the propagation (dual passes)
      float p0b[6];
      float posb = 0.f;
      if (LPT == 1) {
#pragma unroll 1
        for (int e = 0; e < 7; ++e) {
          const float acc_e = prop_pass(e, p0, f, ck, ppb, Jb);
          if (e < 6)
            p0b[e] = acc_e;
          else
            posb = acc_e;
        }
      } else {
        const float acc_e = prop_pass(sub < 7 ? sub : 0, p0, f, ck, ppb, Jb);
#pragma unroll
        for (int e = 0; e < 6; ++e) p0b[e] = __shfl_sync(gm, acc_e, gbase + e);
        posb = __shfl_sync(gm, acc_e, gbase + 6);
      }

      // ---------------- (5) hit frame and surface back to hit xyz and alignment
      const float hx = xyz[h], hy = xyz[H + h];
      const float r2 = fmaf(hx, hx, hy * hy);
      const float phib = fmaf(-m.s, cbar, m.c * sbar);   // d/d(phi_h + dphi)
      float gx = phib * (-hy / r2), gy = phib * (hx / r2), gz = 0.f;
      float gdr = 0.f, gdz = 0.f;
      if (f.kind == 0) {
        gz += wb;
        gdz += wb;
        gdr += posb;
      } else {
        const float ir = rsqrtf(r2);
        gx = fmaf(wb * hx, ir, gx);
        gy = fmaf(wb * hy, ir, gy);
        gdr += wb;
        gdz += posb;
      }
      if (sub == 0) {
        atomicAdd(&g_hit[h], gx);
        atomicAdd(&g_hit[H + h], gy);
        atomicAdd(&g_hit[2 * H + h], gz);
        const int l = f.layer;
        atomicAdd(&acc[4 * l + 0], gdr);
        atomicAdd(&acc[4 * l + 1], phib);
        atomicAdd(&acc[4 * l + 2], gdz);
        atomicAdd(&acc[4 * l + 3], x0b);
      }

      // adjoints of the state before this step
#pragma unroll
      for (int i = 0; i < 6; ++i) pb[i] = p0b[i];
#pragma unroll
      for (int i = 0; i < 21; ++i) G[i] = Gn[i];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < L * 4; i += blockDim.x) {
    const float v = acc[i];
    if (v != 0.0f) {
      if ((i & 3) == 3)
        atomicAdd(&g_x0[i >> 2], v);
      else
        atomicAdd(&g_align[3 * (i >> 2) + (i & 3)], v);
    }
  }
}

}  // namespace

cudaError_t launch_fit_adjoint(mkf_ctx* ctx, const float* xyz, const float* lcov, const int* layer, int64_t n_hits,
                               const int* hits, int K, const float* init_par, const float* init_cov,
                               int64_t n_tracks, const float* align, const float* x0, const float* ckpt,
                               const float* g_chi2, const float* g_par, const float* g_cov, float* g_hit,
                               float* g_align, float* g_x0, cudaStream_t st) {
  (void)init_par;
  (void)init_cov;
  const int L = ctx->geom.n_layers;
  cudaError_t e;
  if (n_hits > 0 && (e = cudaMemsetAsync(g_hit, 0, (size_t)3 * n_hits * sizeof(float), st))) return e;
  if ((e = cudaMemsetAsync(g_align, 0, (size_t)3 * L * sizeof(float), st))) return e;
  if ((e = cudaMemsetAsync(g_x0, 0, (size_t)L * sizeof(float), st))) return e;
  if (n_tracks == 0) return cudaSuccess;
  ctx->tick(kTAdjoint, st);
  // few tracks: 8 lanes per track spread the dual passes and give the SMs
  // enough warps; many tracks: one thread per track does the least work
  int lpt = ctx->adjoint_lanes;
  if (lpt != 1 && lpt != 8) lpt = n_tracks < (int64_t)ctx->n_sm * kAdjThreads ? 8 : 1;
  if (lpt == 8) {
    const int64_t threads = n_tracks * 8;
    k_fit_adjoint<8><<<(unsigned)((threads + kAdjThreads - 1) / kAdjThreads), kAdjThreads, 0, st>>>(
        ctx->geom_dev.as<GeomDev>(), xyz, lcov, layer, n_hits, hits, K, n_tracks, align, x0, ckpt, g_chi2, g_par,
        g_cov, g_hit, g_align, g_x0);
  } else {
    const int T = n_tracks >= (int64_t)ctx->n_sm * kAdjThreads ? kAdjThreads
                : (n_tracks >= (int64_t)ctx->n_sm * 64 ? 64 : 32);
    k_fit_adjoint<1><<<(unsigned)((n_tracks + T - 1) / T), T, 0, st>>>(
        ctx->geom_dev.as<GeomDev>(), xyz, lcov, layer, n_hits, hits, K, n_tracks, align, x0, ckpt, g_chi2, g_par,
        g_cov, g_hit, g_align, g_x0);
  }
  ctx->tock(kTAdjoint, st);
  return cudaGetLastError();
}

}  // namespace mkf
