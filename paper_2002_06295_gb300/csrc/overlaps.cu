// overlaps.cu -- recovery of hits in overlapping detector modules (Sec. 3:
// more than one hit per layer assigned to a track).  The paper plans the
// feature without fixing a rule; the reading here: run the forward fit of
// each track (the fit's own steps: propagate, material, update, with the
// covariance in U-D form); after the
// update with its hit h on layer l, the overlap hit is the other binned hit of
// that layer and event, inside the adjacent-module box around h (|R sin(phi_2
// - phi_h)| <= max_drphi with cos > 0, R the layer radius on a barrel or h's
// radius on a disk; |w_2 - w_h| <= max_dw, w = z on a barrel, r on a disk),
// with the smallest predicted chi2 against the updated state below the cut
// (ties: smaller id).  The state is not updated with it, so the fit result
// does not depend on the search.
//
// LPT lanes per track (1, or 8 when there are few tracks): every lane of the
// group runs the track's fit, the lanes share the hits of the search window,
// and the best candidate is reduced over the group (smallest chi2, then
// smallest id), so the result is the same for every LPT.  The search looks
// only at the bins of a conservative
// window: around the updated state, half-widths sqrt(cut (C + V_max)) + 5 % in
// r*phi and in z (barrel) or r (disk), from the state's position covariance
// and the largest hit variances of the (event, layer) -- the same bound the
// building window uses (every accepted hit has r^2 < cut R for each residual)
// -- intersected with the box around h, which bounds the work of tracks whose
// state is poorly known.
#include "mkf_device.cuh"
#include "mkf_fit_common.cuh"
#include "mkf_internal.h"

namespace mkf {

namespace {

constexpr int kOverlapThreads = 128;

__device__ __forceinline__ HitRec load_hit_rec(const float4* __restrict__ rec, int pos) {
  const float4 a = __ldg(&rec[2 * pos]);
  const float4 b = __ldg(&rec[2 * pos + 1]);
  HitRec h;
  h.c = a.x;
  h.s = a.y;
  h.w = a.z;
  h.v00 = a.w;
  h.v01 = b.x;
  h.v11 = b.y;
  h.orig = __float_as_int(b.z);
  h.bin = __float_as_int(b.w);
  return h;
}

// The work of one track (t >= NT: none), by lane `sub` of its LPT-lane group
// (group mask gm).
template <int LPT>
__device__ __forceinline__ void track_overlaps(const GeomDev* __restrict__ g, const float* __restrict__ xyz,
                                               const float* __restrict__ lcov, const int* __restrict__ layer,
                                               int64_t H, const int* __restrict__ hits, int K,
                                               const float* __restrict__ init_par, const float* __restrict__ init_cov,
                                               int64_t NT, float cut, float max_drphi, float max_dw,
                                               const float4* __restrict__ rec,
                                               const int* __restrict__ bin_off, const float* __restrict__ vmax,
                                               const int64_t* __restrict__ ev_hit_off, int n_events,
                                               int* __restrict__ out_hit, float* __restrict__ out_chi2, int64_t t,
                                               int sub, unsigned gm, int& n_fit, int& n_cand, int& n_found) {
  if (t >= NT) return;
  const int* row = hits + t * K;
  for (int k = sub; k < K; k += LPT) {
    out_hit[t * K + k] = -1;
    out_chi2[t * K + k] = 0.f;
  }
  if (LPT > 1) __syncwarp(gm);   // the slots are rewritten below by lane 0 of the group
  int first = -1;
  for (int k = 0; k < K && first < 0; ++k) first = row[k] >= 0 && row[k] < H ? row[k] : -1;
  if (first < 0) return;
  int lo = 0, hi = n_events;   // the track's event: the one holding its first hit
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(&ev_hit_off[mid]) <= first)
      lo = mid;
    else
      hi = mid;
  }
  const int e = lo, L = g->n_layers;
  const int ebase = e * g->bins_per_event;
  const float ck = g->c_kappa;
  float p[6], C[21];
#pragma unroll
  for (int i = 0; i < 6; ++i) p[i] = init_par[i * NT + t];
#pragma unroll
  for (int i = 0; i < 21; ++i) C[i] = init_cov[i * NT + t];
  UD6 u;
  ud_from_cov(C, u);
  for (int k = 0; k < K; ++k) {
    FitHit<float> f;
    const int h = row[k];
    if (!load_fit_hit(g, xyz, lcov, layer, H, h, (const float*)nullptr, (const float*)nullptr, f)) continue;
    if (!step_to_ud(f, p, u, ck, +1)) break;
    ud_update(f.kind, p, u, f.m);
    if (sub == 0) ++n_fit;
    // search window around the updated state on the same layer
    const LayerDev ly = g->L[f.layer];
    float cp[6];
    ud_pos_block(u, cp);
    const PosState q{p[0], p[1], p[2], cp[0], cp[1], cp[2], cp[3], cp[4], cp[5]};
    const float r = sqrtf(fmaf(q.x, q.x, q.y * q.y));
    if (!(r > 0.f)) continue;
    const float c = q.x / r, s = q.y / r;
    const float caa = fmaf(s * s, q.cxx, fmaf(-2.f * s * c, q.cxy, c * c * q.cyy));
    const float cbb = ly.kind == 0 ? q.czz : fmaf(c * c, q.cxx, fmaf(2.f * s * c, q.cxy, s * s * q.cyy));
    const float va = __ldg(&vmax[2 * (e * L + f.layer)]), vb = __ldg(&vmax[2 * (e * L + f.layer) + 1]);
    const float ha = 1.05f * sqrtf(cut * (fmaxf(caa, 0.f) + va)) + 1e-4f;
    const float hb = 1.05f * sqrtf(cut * (fmaxf(cbb, 0.f) + vb)) + 1e-4f;
    const float wc = ly.kind == 0 ? q.z : r;
    const float phic = atan2f(q.y, q.x);
    // the primary hit and its box; phi offsets relative to the state's azimuth
    const float rh = ly.kind == 0 ? ly.pos : f.m.w;
    const float dh = atan2f(fmaf(c, f.m.s, -s * f.m.c), fmaf(c, f.m.c, s * f.m.s));
    const float dbox = max_drphi < rh ? asinf(max_drphi / rh) + 1e-5f : kPi;
    const float dchi = ha < r ? asinf(ha / r) + 1e-5f : kPi;
    const float plo = fmaxf(-dchi, dh - dbox), phi_hi = fminf(dchi, dh + dbox);
    const float wlo = fmaxf(wc - hb, f.m.w - max_dw - 1e-4f), whi = fminf(wc + hb, f.m.w + max_dw + 1e-4f);
    if (!(plo <= phi_hi) || !(wlo <= whi)) continue;
    const int ip0 = (int)floorf((phic + plo + kPi) * ly.phi_scale);
    const int ip1 = (int)floorf((phic + phi_hi + kPi) * ly.phi_scale);
    const int nrow = min(ip1 - ip0 + 1, ly.nphi);
    const int iw0 = min(max((int)floorf((wlo - ly.lo) * ly.w_scale), 0), ly.nw - 1);
    const int iw1 = min(max((int)floorf((whi - ly.lo) * ly.w_scale), 0), ly.nw - 1);
    float best = INFINITY;
    int best_id = -1;
    for (int kr = 0; kr < nrow; ++kr) {
      int ip = (ip0 + kr) % ly.nphi;
      if (ip < 0) ip += ly.nphi;
      const int b0 = ebase + ly.bin_base + ip * ly.nw;
      const int p0 = __ldg(&bin_off[b0 + iw0]), p1 = __ldg(&bin_off[b0 + iw1 + 1]);
      for (int pos = p0 + sub; pos < p1; pos += LPT) {
        const HitRec hr = load_hit_rec(rec, pos);
        if (hr.orig == h) continue;
        const float cd = fmaf(f.m.c, hr.c, f.m.s * hr.s), sd = fmaf(f.m.c, hr.s, -f.m.s * hr.c);
        if (!(cd > 0.f) || !(fabsf(rh * sd) <= max_drphi) || !(fabsf(hr.w - f.m.w) <= max_dw)) continue;
        const float c2 = hit_chi2(ly.kind, q, hr, cut);
        ++n_cand;
        if (c2 < best || (c2 == best && hr.orig < best_id)) {
          best = c2;
          best_id = hr.orig;
        }
      }
    }
    if (LPT > 1) {
#pragma unroll
      for (int o = LPT / 2; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(gm, best, o);
        const int oi = __shfl_xor_sync(gm, best_id, o);
        if (ob < best || (ob == best && oi >= 0 && (best_id < 0 || oi < best_id))) {
          best = ob;
          best_id = oi;
        }
      }
    }
    if (sub == 0 && best_id >= 0 && best < cut) {
      out_hit[t * K + k] = best_id;
      out_chi2[t * K + k] = best;
      ++n_found;
    }
  }
}

template <int LPT>
__global__ void __launch_bounds__(kOverlapThreads)
    k_overlaps(const GeomDev* __restrict__ g, const float* __restrict__ xyz, const float* __restrict__ lcov,
               const int* __restrict__ layer, int64_t H, const int* __restrict__ hits, int K,
               const float* __restrict__ init_par, const float* __restrict__ init_cov, int64_t NT, float cut,
               float max_drphi, float max_dw, const float4* __restrict__ rec, const int* __restrict__ bin_off,
               const float* __restrict__ vmax,
               const int64_t* __restrict__ ev_hit_off, int n_events, int* __restrict__ out_hit,
               float* __restrict__ out_chi2, unsigned long long* __restrict__ stats) {
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPT;
  const int sub = threadIdx.x % LPT;
  const unsigned gm = LPT == 32 ? 0xFFFFFFFFu : ((1u << LPT) - 1u) << ((threadIdx.x & 31) - sub);
  int n_fit = 0, n_cand = 0, n_found = 0;   // work counters
  track_overlaps<LPT>(g, xyz, lcov, layer, H, hits, K, init_par, init_cov, NT, cut, max_drphi, max_dw, rec, bin_off,
                      vmax, ev_hit_off, n_events, out_hit, out_chi2, t, sub, gm, n_fit, n_cand, n_found);
  const int v[3] = {n_fit, n_cand, n_found};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    int x = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&stats[i], (unsigned long long)x);
  }
}

}  // namespace

}  // namespace mkf

extern "C" mkf_status mkf_find_overlaps(mkf_ctx* ctx, const float* xyz, const float* lcov, const int* layer,
                                        int64_t n_hits, const int* hits, int K, const float* init_par,
                                        const float* init_cov, int64_t n_tracks, float chi2_cut, float max_drphi,
                                        float max_dw, int* out_hit, float* out_chi2, void* stream) {
  using namespace mkf;
  if (!ctx) return MKF_ERR_ARG;
  if (!ctx->have_geom) return ctx->fail(MKF_ERR_STATE, "no geometry");
  if (!ctx->binned) return ctx->fail(MKF_ERR_STATE, "hits not binned");
  if (n_hits != ctx->n_hits) return ctx->fail(MKF_ERR_ARG, "hits differ from the binned hits");
  if (n_tracks < 0 || K < 0 || !(chi2_cut > 0.f) || !(max_drphi > 0.f) || !(max_dw > 0.f))
    return ctx->fail(MKF_ERR_ARG, "bad sizes or cuts");
  if (n_tracks == 0 || K == 0) return MKF_OK;
  if (!xyz || !lcov || !layer || !hits || !init_par || !init_cov || !out_hit || !out_chi2)
    return ctx->fail(MKF_ERR_ARG, "null array");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = ctx->ovl_stats.ensure(4 * sizeof(unsigned long long))) != cudaSuccess) return ctx->fail(MKF_ERR_OOM, "stats");
  if ((e = cudaMemsetAsync(ctx->ovl_stats.p, 0, 4 * sizeof(unsigned long long), st)) != cudaSuccess)
    return ctx->cuda_fail(e, "memset");
  // few tracks: eight lanes a track share its search and give the SMs enough
  // warps; many tracks: one thread a track, in small blocks when there are
  // not many, so that the work spreads over every SM
  int lpt = ctx->overlap_lanes;
  if (lpt != 1 && lpt != 8) lpt = n_tracks < (int64_t)ctx->n_sm * kOverlapThreads ? 8 : 1;
  if (lpt == 8) {
    const int64_t threads = n_tracks * 8;
    k_overlaps<8><<<(unsigned)((threads + kOverlapThreads - 1) / kOverlapThreads), kOverlapThreads, 0, st>>>(
        ctx->geom_dev.as<GeomDev>(), xyz, lcov, layer, n_hits, hits, K, init_par, init_cov, n_tracks, chi2_cut,
        max_drphi, max_dw, ctx->rec.as<float4>(), ctx->bin_off.as<int>(), ctx->vmax.as<float>(),
        ctx->ev_hit_off.as<int64_t>(), ctx->n_events, out_hit, out_chi2, ctx->ovl_stats.as<unsigned long long>());
  } else {
    const int T = n_tracks >= (int64_t)ctx->n_sm * 128 ? 128 : (n_tracks >= (int64_t)ctx->n_sm * 64 ? 64 : 32);
    const unsigned blocks = (unsigned)((n_tracks + T - 1) / T);
    k_overlaps<1><<<blocks, T, 0, st>>>(ctx->geom_dev.as<GeomDev>(), xyz, lcov, layer, n_hits, hits, K, init_par,
                                        init_cov, n_tracks, chi2_cut, max_drphi, max_dw, ctx->rec.as<float4>(),
                                        ctx->bin_off.as<int>(), ctx->vmax.as<float>(), ctx->ev_hit_off.as<int64_t>(),
                                        ctx->n_events, out_hit, out_chi2, ctx->ovl_stats.as<unsigned long long>());
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return ctx->cuda_fail(e, "overlaps");
  return MKF_OK;
}

extern "C" mkf_status mkf_set_overlap_config(mkf_ctx* ctx, int lanes_per_track) {
  if (!ctx) return MKF_ERR_ARG;
  if (lanes_per_track != 0 && lanes_per_track != 1 && lanes_per_track != 8)
    return ctx->fail(MKF_ERR_ARG, "lanes_per_track must be 0, 1 or 8");
  ctx->overlap_lanes = lanes_per_track;
  return MKF_OK;
}

extern "C" mkf_status mkf_get_overlap_stats(mkf_ctx* ctx, int64_t* out, int n, void* stream) {
  if (!ctx || !out || n < 0 || n > 3) return ctx ? ctx->fail(MKF_ERR_ARG, "overlap stats: n in 0..3") : MKF_ERR_ARG;
  unsigned long long v[4] = {};
  if (ctx->ovl_stats.p) {
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(v, ctx->ovl_stats.p, sizeof(v), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return ctx->cuda_fail(e, "overlap stats");
  }
  for (int i = 0; i < n; ++i) out[i] = (int64_t)v[i];
  return MKF_OK;
}
