// mkf_ud.cuh -- the track covariance in U-D factorised form, FP32.
//
// The Kalman filter of the paper (Sec. 1: propagate, then update with the hit)
// is run here on the factorisation C = U D U^T, U unit upper triangular and D
// diagonal and non-negative (Bierman, "Factorization Methods for Discrete
// Sequential Estimation", 1977).  D holds conditional variances: D_j is the
// variance of parameter j given parameters j+1..5.  When hits shrink a
// variance by 1e5 and leave correlations within 1e-4 of 1 (pixel hits, strip
// disks with sigma_r / sigma_rphi = 333, the 100x prior of the inward fit),
// those small conditional variances are the numbers that matter; the plain
// covariance keeps them only as differences of nearly equal FP32 entries,
// while D stores them directly, to FP32's relative precision.
//
//  * Transport onto the next surface, C' = J C J^T + G Q G^T (multiple
//    scattering Q on phi and theta), is the modified weighted Gram-Schmidt
//    step of Thornton ("Triangular covariance factorizations for Kalman
//    filtering", 1976): the rows of W = [J U | G] are orthogonalised against
//    the weights [D, Q] from the last row to the first.  (Adding Q afterwards
//    by Agee-Turner rank-one updates needs fewer registers but was measured
//    less accurate: 9.9e-5 against 3.1e-5 of sqrt(C_ii C_jj) at worst on
//    CMS-like outward fits.)
//  * The update with a 2-D hit first decorrelates the hit covariance
//    V = L L^T, then applies Bierman's scalar update twice (an exact
//    rewriting of the 2-D update for a linear measurement; the predicted chi2
//    is the sum of the two scalar innovations' chi2).
//
// U is kept packed: U_ij (i < j) at uidx(i, j) = j (j - 1) / 2 + i, 15 floats;
// with D's 6 floats the factorisation takes the 21 floats of a packed C.
#pragma once
#include "mkf_device.cuh"

namespace mkf {

__host__ __device__ constexpr int uidx(int i, int j) { return j * (j - 1) / 2 + i; }

// A conditional variance at or below this is a direction without variance (the
// surface normal after a transport, rounded): it is set to exactly 0 with
// U_.j = 0, so that no reciprocal of a denormal (an overflow to inf) is ever
// formed.  Variances of the parameters in cm, 1/GeV and rad are above 1e-20
// for every resolution the library meets.
constexpr float kMinCondVar = 1e-30f;

struct UD6 {
  float u[15];   // U_ij, i < j, packed by column
  float d[6];    // D_j
};

// C (packed lower triangle) -> U D U^T, from the last parameter to the first:
// D_j = C_jj - sum_{k>j} U_jk^2 D_k, U_ij = (C_ij - sum_{k>j} U_ik U_jk D_k) / D_j.
// A D_j at or below kMinCondVar (a direction without variance) is set to 0
// with U_.j = 0.
__device__ __forceinline__ void ud_from_cov(const float C[21], UD6& f) {
  bool diagonal = true;
#pragma unroll
  for (int i = 1; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) diagonal = diagonal && C[ci(i, j)] == 0.0f;
  if (diagonal) {   // U = 1, D = diag(C): the usual seed
#pragma unroll
    for (int k = 0; k < 15; ++k) f.u[k] = 0.0f;
#pragma unroll
    for (int j = 0; j < 6; ++j) f.d[j] = C[ci(j, j)] > kMinCondVar ? C[ci(j, j)] : 0.0f;
    return;
  }
#pragma unroll
  for (int j = 5; j >= 0; --j) {
    float dj = C[ci(j, j)];
#pragma unroll
    for (int k = j + 1; k < 6; ++k) dj = fmaf(-f.u[uidx(j, k)] * f.u[uidx(j, k)], f.d[k], dj);
    dj = dj > kMinCondVar ? dj : 0.0f;
    f.d[j] = dj;
    const float inv = dj > 0.0f ? 1.0f / dj : 0.0f;
#pragma unroll
    for (int i = 0; i < j; ++i) {
      float a = C[ci(i, j)];
#pragma unroll
      for (int k = j + 1; k < 6; ++k) a = fmaf(-f.u[uidx(i, k)] * f.d[k], f.u[uidx(j, k)], a);
      f.u[uidx(i, j)] = a * inv;
    }
  }
}

// U_ik, with the unit diagonal and zeros below it (compile-time indices).
__device__ __forceinline__ float ud_u(const UD6& f, int i, int k) {
  return i == k ? 1.0f : (i < k ? f.u[uidx(i, k)] : 0.0f);
}

// C_ij = sum_{k >= max(i, j)} U_ik D_k U_jk
__device__ __forceinline__ float ud_cov_entry(const UD6& f, int i, int j) {
  const int m = i > j ? i : j;
  float acc = 0.0f;
#pragma unroll
  for (int k = 5; k >= m; --k) acc = fmaf(ud_u(f, i, k) * f.d[k], ud_u(f, j, k), acc);
  return acc;
}

__device__ __forceinline__ void ud_to_cov(const UD6& f, float C[21]) {
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) C[ci(i, j)] = ud_cov_entry(f, i, j);
}

// The position block (xx, yx, yy, zx, zy, zz) of C: what the chi2 of a hit
// and the search window need.
__device__ __forceinline__ void ud_pos_block(const UD6& f, float out[6]) {
  out[0] = ud_cov_entry(f, 0, 0);
  out[1] = ud_cov_entry(f, 1, 0);
  out[2] = ud_cov_entry(f, 1, 1);
  out[3] = ud_cov_entry(f, 2, 0);
  out[4] = ud_cov_entry(f, 2, 1);
  out[5] = ud_cov_entry(f, 2, 2);
}

// Thornton's transport: U' D' U'^T = W diag(D, q_phi, q_theta) W^T with
// W = [J U | e_phi | e_theta], i.e. C' = J C J^T + q_phi e_phi e_phi^T +
// q_theta e_theta e_theta^T.  J's rows for kappa and theta are the identity,
// so those rows of J U are U's own rows.  The rows of W are orthogonalised
// from the last to the first: D'_j is the weighted norm of row j, U'_ij the
// weighted projection of row i on it, which is then removed from row i.  A row
// with no weight left (D'_j <= kMinCondVar) gets D'_j = 0 and U'_.j = 0.
__device__ __forceinline__ void ud_transport(const Jac4<float>& J, UD6& f, float q_phi, float q_theta) {
  constexpr int R[4] = {0, 1, 2, 4};
  float W[6][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float acc = J.r[a][k];
#pragma unroll
      for (int m = 0; m < k; ++m) acc = fmaf(J.r[a][m], f.u[uidx(m, k)], acc);
      W[R[a]][k] = acc;
    }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    W[3][k] = ud_u(f, 3, k);
    W[5][k] = ud_u(f, 5, k);
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    W[i][6] = i == 4 ? 1.0f : 0.0f;
    W[i][7] = i == 5 ? 1.0f : 0.0f;
  }
  const float Dw[8] = {f.d[0], f.d[1], f.d[2], f.d[3], f.d[4], f.d[5], q_phi, q_theta};
  {
    // row 5 of W is e_theta + e_(theta noise): its weighted norm is
    // D_5 + q_theta, and each row i < 5 (zero in the theta-noise column)
    // projects on it with W_i5 D_5 only
    float d5 = Dw[5] + q_theta;
    d5 = d5 > kMinCondVar ? d5 : 0.0f;
    f.d[5] = d5;
    const float r5 = d5 > 0.0f ? __frcp_rn(d5) : 0.0f;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const float uij = W[i][5] * Dw[5] * r5;
      f.u[uidx(i, 5)] = uij;
      W[i][5] -= uij;
      W[i][7] = -uij;
    }
  }
#pragma unroll
  for (int j = 4; j >= 0; --j) {
    float c[8];
    float dj = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      c[k] = Dw[k] * W[j][k];
      dj = fmaf(W[j][k], c[k], dj);
    }
    dj = dj > kMinCondVar ? dj : 0.0f;
    f.d[j] = dj;
    const float inv = dj > 0.0f ? __frcp_rn(dj) : 0.0f;
#pragma unroll
    for (int i = 0; i < j; ++i) {
      float a = 0.0f;
#pragma unroll
      for (int k = 0; k < 8; ++k) a = fmaf(W[i][k], c[k], a);
      const float uij = a * inv;
      f.u[uidx(i, j)] = uij;
#pragma unroll
      for (int k = 0; k < 8; ++k) W[i][k] = fmaf(-uij, W[j][k], W[i][k]);
    }
  }
}

// Bierman's scalar update with the measurement row h (non-zero only on the
// position parameters 0..2), unit measurement variance and innovation nu.
// Returns nu^2 / alpha, alpha = h C h^T + 1; updates p, U and D.
__device__ __forceinline__ float ud_scalar_update(UD6& f, float p[6], const float h[3], float nu) {
  float fv[6], g[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    float acc = j < 3 ? h[j] : 0.0f;
#pragma unroll
    for (int i = 0; i < (j < 3 ? j : 3); ++i) acc = fmaf(f.u[uidx(i, j)], h[i], acc);
    fv[j] = acc;
    g[j] = f.d[j] * acc;
  }
  float alpha = 1.0f, ialpha = 1.0f;   // alpha_(j-1) and its reciprocal
  float b[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const float an = fmaf(fv[j], g[j], alpha);
    const float ia = __frcp_rn(an);
    const float lam = -fv[j] * ialpha;
    f.d[j] = f.d[j] * (alpha * ia);
    ialpha = ia;
#pragma unroll
    for (int i = 0; i < j; ++i) {
      const float uo = f.u[uidx(i, j)];
      f.u[uidx(i, j)] = fmaf(b[i], lam, uo);
      b[i] = fmaf(uo, g[j], b[i]);
    }
    b[j] = g[j];
    alpha = an;
  }
  const float k = nu * ialpha;
#pragma unroll
  for (int i = 0; i < 6; ++i) p[i] = fmaf(b[i], k, p[i]);
  return nu * k;
}

// Update with a hit in its local frame (rows of mkf_device.cuh's Meas):
// a = (-sin phi_h, cos phi_h, 0) with m_a = 0; b = (0, 0, 1) with m_b = z_h on
// a barrel, (cos phi_h, sin phi_h, 0) with m_b = r_h on a disk.  With
// V = L L^T (l00 = sqrt V_aa, l10 = V_ab / l00, l11 = sqrt(V_bb - l10^2)) the
// rows a' = a / l00 and b' = (b - l10 a') / l11 are independent unit-variance
// measurements.  Returns the predicted chi2 of the hit.
__device__ __forceinline__ float ud_update(int kind, float p[6], UD6& f, const Meas<float>& m) {
  const float l00 = sqrtf(m.v00);
  const float il00 = 1.0f / l00;
  const float l10 = m.v01 * il00;
  const float il11 = rsqrtf(fmaf(-l10, l10, m.v11));
  const float ha[3] = {-m.s * il00, m.c * il00, 0.0f};
  float chi2 = ud_scalar_update(f, p, ha, -fmaf(ha[0], p[0], ha[1] * p[1]));
  float hb[3];
  if (kind == 0) {
    hb[0] = -l10 * ha[0] * il11;
    hb[1] = -l10 * ha[1] * il11;
    hb[2] = il11;
  } else {
    hb[0] = fmaf(-l10, ha[0], m.c) * il11;
    hb[1] = fmaf(-l10, ha[1], m.s) * il11;
    hb[2] = 0.0f;
  }
  const float hp = fmaf(hb[0], p[0], fmaf(hb[1], p[1], hb[2] * p[2]));
  chi2 += ud_scalar_update(f, p, hb, fmaf(m.w, il11, -hp));
  p[4] = wrap_phi(p[4]);
  return chi2;
}

}  // namespace mkf
