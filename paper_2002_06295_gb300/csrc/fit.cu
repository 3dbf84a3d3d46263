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

// Inward fit: covariance reset to 100 x the seed-style diagonal, update with
// the outermost hit in place, then propagate inward hit by hit (FP64, plain
// covariance update).
__global__ void k_fit_inward(const GeomDev* __restrict__ g, const float* __restrict__ xyz,
                             const float* __restrict__ lcov, const int* __restrict__ layer, int64_t H,
                             const int* __restrict__ hits, int K, const float* __restrict__ init_par, int64_t NT,
                             const float* __restrict__ align, const float* __restrict__ x0,
                             float* __restrict__ out_par, float* __restrict__ out_cov, float* __restrict__ out_chi2,
                             int* __restrict__ out_ok) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NT) return;
  const int* row = hits + t * K;
  double p[6], C[21];
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = double(init_par[k * NT + t]);
#pragma unroll
  for (int k = 0; k < 21; ++k) C[k] = 0.0;
  C[ci(0, 0)] = C[ci(1, 1)] = C[ci(2, 2)] = 1.0;
  C[ci(3, 3)] = 100.0 * (0.05 * p[3]) * (0.05 * p[3]);
  C[ci(4, 4)] = C[ci(5, 5)] = 0.25;
  int last = -1;
  for (int k = K - 1; k >= 0; --k)
    if (row[k] >= 0) {
      last = k;
      break;
    }
  double chi2 = 0.0;
  int ok = 1;
  const double ck = double(g->c_kappa);
  FitHit<double> f;
  for (int k = last; k >= 0; --k) {
    if (!load_fit_hit(g, xyz, lcov, layer, H, row[k], align, x0, f)) continue;
    if (k != last && !step_to(f, p, C, ck, -1)) {
      ok = 0;
      break;
    }
    chi2 += kf_update<double, false>(f.kind, p, C, f.m);
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) out_par[i * NT + t] = float(p[i]);
#pragma unroll
  for (int i = 0; i < 21; ++i) out_cov[i * NT + t] = float(C[i]);
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
