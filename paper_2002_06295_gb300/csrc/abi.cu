// abi.cu -- the C ABI: context, geometry, argument checks, dispatch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "mkf_device.cuh"
#include "mkf_internal.h"

using namespace mkf;

namespace {
const char* kEmpty = "";

mkf_status check_ctx(mkf_ctx* ctx) { return ctx ? MKF_OK : MKF_ERR_ARG; }

#define MKF_CUDA(call, what)                         \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return ctx->cuda_fail(e_, what); \
  } while (0)
}  // namespace

extern "C" {

mkf_status mkf_create(mkf_ctx** out, int device) {
  if (!out) return MKF_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return MKF_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return MKF_ERR_CUDA;
  mkf_ctx* ctx = new (std::nothrow) mkf_ctx();
  if (!ctx) return MKF_ERR_OOM;
  ctx->device = device;
  cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device);
  if (ctx->status.ensure(sizeof(int)) != cudaSuccess || ctx->stats.ensure(8 * sizeof(int64_t)) != cudaSuccess ||
      ctx->seed_ctr.ensure(sizeof(unsigned long long)) != cudaSuccess) {
    delete ctx;
    return MKF_ERR_OOM;
  }
  cudaMemset(ctx->status.p, 0, sizeof(int));
  cudaMemset(ctx->stats.p, 0, 8 * sizeof(int64_t));
  *out = ctx;
  return MKF_OK;
}

void mkf_destroy(mkf_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->timers_made)
    for (int i = 0; i < kTimers; ++i) {
      cudaEventDestroy(ctx->t_beg[i]);
      cudaEventDestroy(ctx->t_end[i]);
    }
  DevBuf* bufs[] = {&ctx->geom_dev, &ctx->rec,     &ctx->rec_orig,  &ctx->perm,     &ctx->bin_off,
                    &ctx->bin_cnt,  &ctx->keys,    &ctx->ranks,     &ctx->vmax,     &ctx->ev_hit_off,
                    &ctx->scan_part, &ctx->seed_ctr, &ctx->stats,    &ctx->status,   &ctx->dd_head,
                    &ctx->dd_next,  &ctx->dd_beat, &ctx->dd_nbeat,  &ctx->dd_state, &ctx->track_hits, &ctx->build_order,
                    &ctx->strip_bits, &ctx->seed_cnt, &ctx->seed_off, &ctx->seed_part, &ctx->seed_pairs,
                    &ctx->seed_qcnt, &ctx->seed_qoff, &ctx->grid_key, &ctx->grid_rank, &ctx->grid_cnt,
                    &ctx->grid_off, &ctx->grid_rec, &ctx->seed_stats, &ctx->ovl_stats,
                    &ctx->seed_scratch, &ctx->seed_loc};
  for (DevBuf* b : bufs) b->release();
  delete ctx;
}

const char* mkf_last_error(const mkf_ctx* ctx) { return ctx ? ctx->err.c_str() : kEmpty; }

mkf_status mkf_sync(mkf_ctx* ctx, void* stream) {
  if (check_ctx(ctx)) return MKF_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int h = 0;
  MKF_CUDA(cudaMemcpyAsync(&h, ctx->status.p, sizeof(int), cudaMemcpyDeviceToHost, st), "status read");
  MKF_CUDA(cudaStreamSynchronize(st), "synchronize");
  MKF_CUDA(cudaMemsetAsync(ctx->status.p, 0, sizeof(int), st), "status clear");
  if (h & kStatCapacity) return ctx->fail(MKF_ERR_CAPACITY, "a device-side buffer overflowed");
  if (h & kStatTimeout) return ctx->fail(MKF_ERR_TIMEOUT, "a bounded device wait expired");
  if (h & kStatBadInput) return ctx->fail(MKF_ERR_ARG, "an input index was out of range");
  return MKF_OK;
}

mkf_status mkf_load_geometry(mkf_ctx* ctx, const mkf_layer* layers, int n_layers, float bz_tesla) {
  if (check_ctx(ctx)) return MKF_ERR_ARG;
  if (!layers || n_layers < 1 || n_layers > MKF_MAX_LAYERS) return ctx->fail(MKF_ERR_ARG, "n_layers out of range");
  if (!std::isfinite(bz_tesla)) return ctx->fail(MKF_ERR_ARG, "bz not finite");
  GeomDev g{};
  g.n_layers = n_layers;
  g.bz = bz_tesla;
  g.c_kappa = -kAlpha * bz_tesla;
  int base = 0;
  std::vector<std::pair<float, int>> bar, dp, dn;
  for (int l = 0; l < n_layers; ++l) {
    const mkf_layer& s = layers[l];
    if ((s.kind != 0 && s.kind != 1) || !(s.hi > s.lo) || !std::isfinite(s.pos) || !(s.x_over_x0 >= 0.0f))
      return ctx->fail(MKF_ERR_ARG, "invalid layer " + std::to_string(l));
    if (s.kind == 0 && !(s.pos > 0.0f)) return ctx->fail(MKF_ERR_ARG, "barrel radius must be positive");
    if (s.kind == 1 && s.pos == 0.0f) return ctx->fail(MKF_ERR_ARG, "disk at z = 0");
    LayerDev& d = g.L[l];
    d.kind = s.kind;
    d.pos = s.pos;
    d.lo = s.lo;
    d.hi = s.hi;
    d.x0 = s.x_over_x0;
    d.nphi = s.n_phi_bins > 0 ? s.n_phi_bins : 64;
    d.nw = s.n_w_bins > 0 ? s.n_w_bins : 16;
    if (d.nphi > 4096 || d.nw > 4096) return ctx->fail(MKF_ERR_ARG, "too many bins");
    d.bin_base = base;
    base += d.nphi * d.nw;
    d.phi_scale = (float)d.nphi / kTwoPi;
    d.w_scale = (float)d.nw / (s.hi - s.lo);
    g.r_max = std::max(g.r_max, s.kind == 0 ? s.pos : s.hi);
    if (s.kind == 0)
      bar.push_back({s.pos, l});
    else if (s.pos > 0)
      dp.push_back({s.pos, l});
    else
      dn.push_back({-s.pos, l});
  }
  std::sort(bar.begin(), bar.end());
  std::sort(dp.begin(), dp.end());
  std::sort(dn.begin(), dn.end());
  g.n_barrel = (int)bar.size();
  g.n_dpos = (int)dp.size();
  g.n_dneg = (int)dn.size();
  for (size_t i = 0; i < bar.size(); ++i) {
    g.barrel_order[i] = (int8_t)bar[i].second;
    g.barrel_r[i] = bar[i].first;
  }
  for (size_t i = 0; i < dp.size(); ++i) {
    g.dpos_order[i] = (int8_t)dp[i].second;
    g.dpos_z[i] = dp[i].first;
  }
  for (size_t i = 0; i < dn.size(); ++i) {
    g.dneg_order[i] = (int8_t)dn[i].second;
    g.dneg_z[i] = dn[i].first;
  }
  g.bins_per_event = base;
  if (ctx->geom_dev.ensure(sizeof(GeomDev)) != cudaSuccess) return ctx->fail(MKF_ERR_OOM, "geometry buffer");
  MKF_CUDA(cudaMemcpy(ctx->geom_dev.p, &g, sizeof(GeomDev), cudaMemcpyHostToDevice), "geometry upload");
  ctx->geom = g;
  ctx->have_geom = true;
  ctx->binned = false;
  return MKF_OK;
}

mkf_status mkf_bin_hits(mkf_ctx* ctx, const float* xyz, const float* lcov, const int* layer, int64_t n_hits,
                        const int64_t* ev_hit_off, int n_events, void* stream) {
  return mkf_bin_hits_masked(ctx, xyz, lcov, layer, n_hits, ev_hit_off, n_events, nullptr, stream);
}

mkf_status mkf_used_hits(mkf_ctx* ctx, const int* hits, int L, const int* flags, int64_t n_tracks, int64_t n_hits,
                         uint8_t* mask, void* stream) {
  if (check_ctx(ctx)) return MKF_ERR_ARG;
  if (L < 1 || L > MKF_MAX_LAYERS || n_tracks < 0 || n_hits < 0 || n_tracks > (int64_t)INT32_MAX / MKF_MAX_LAYERS)
    return ctx->fail(MKF_ERR_ARG, "bad sizes");
  if (n_tracks > 0 && (!hits || !flags || !mask)) return ctx->fail(MKF_ERR_ARG, "null array");
  if ((ctx->status.ensure(sizeof(int))) != cudaSuccess) return ctx->fail(MKF_ERR_OOM, "status word");
  cudaError_t e = launch_used_hits(ctx, hits, flags, n_tracks, L, n_hits, mask, (cudaStream_t)stream);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "used_hits");
  return MKF_OK;
}

mkf_status mkf_bin_hits_masked(mkf_ctx* ctx, const float* xyz, const float* lcov, const int* layer, int64_t n_hits,
                               const int64_t* ev_hit_off, int n_events, const uint8_t* mask, void* stream) {
  if (check_ctx(ctx)) return MKF_ERR_ARG;
  if (!ctx->have_geom) return ctx->fail(MKF_ERR_STATE, "no geometry loaded");
  if (n_hits < 0 || n_hits > (int64_t)INT32_MAX - 1 || n_events < 1 || !ev_hit_off)
    return ctx->fail(MKF_ERR_ARG, "bad sizes");
  if (n_hits > 0 && (!xyz || !lcov || !layer)) return ctx->fail(MKF_ERR_ARG, "null hit array");
  if ((int64_t)n_events * ctx->geom.bins_per_event >= (int64_t)INT32_MAX)
    return ctx->fail(MKF_ERR_ARG, "too many bins for int32 offsets");
  cudaError_t e = launch_bin_hits(ctx, xyz, lcov, layer, n_hits, ev_hit_off, n_events, mask, (cudaStream_t)stream);
  if (e == cudaErrorMemoryAllocation) return ctx->fail(MKF_ERR_OOM, "binning workspace");
  if (e != cudaSuccess) return ctx->cuda_fail(e, "bin_hits");
  ctx->binned = true;
  return MKF_OK;
}

mkf_status mkf_get_binning(mkf_ctx* ctx, int* perm, int* bin_off, int64_t* n_bins, void* stream) {
  if (check_ctx(ctx)) return MKF_ERR_ARG;
  if (!ctx->binned) return ctx->fail(MKF_ERR_STATE, "hits not binned");
  cudaStream_t st = (cudaStream_t)stream;
  if (n_bins) *n_bins = ctx->n_bins_total;
  MKF_CUDA(launch_bin_order(ctx, st), "bin order");
  if (perm && ctx->n_hits)
    MKF_CUDA(cudaMemcpyAsync(perm, ctx->perm.p, ctx->n_hits * sizeof(int), cudaMemcpyDeviceToDevice, st), "perm");
  if (bin_off)
    MKF_CUDA(cudaMemcpyAsync(bin_off, ctx->bin_off.p, (ctx->n_bins_total + 1) * sizeof(int),
                             cudaMemcpyDeviceToDevice, st),
             "bin_off");
  return MKF_OK;
}

mkf_status mkf_build_tracks(mkf_ctx* ctx, const float* seed_par, const float* seed_cov, const int64_t* ev_seed_off,
                            int64_t n_seeds, float chi2_cut, int max_cands, int max_holes, int min_hits,
                            float dup_frac, int* out_hits, int* out_layers, float* out_par, float* out_cov,
                            float* out_score, float* out_chi2, int* out_counts, int* out_flags, void* stream) {
  if (check_ctx(ctx)) return MKF_ERR_ARG;
  if (!ctx->binned) return ctx->fail(MKF_ERR_STATE, "hits not binned");
  if (n_seeds < 0 || n_seeds > (int64_t)INT32_MAX / MKF_MAX_LAYERS) return ctx->fail(MKF_ERR_ARG, "n_seeds");
  if (max_cands < 1 || max_cands > MKF_MAX_CANDS) return ctx->fail(MKF_ERR_ARG, "max_cands out of range");
  if (max_holes < 0 || min_hits < 0 || !(dup_frac >= 0.0f && dup_frac <= 1.0f) || !(chi2_cut > 0.0f))
    return ctx->fail(MKF_ERR_ARG, "bad build parameters");
  if (!ev_seed_off) return ctx->fail(MKF_ERR_ARG, "null ev_seed_off");
  if (n_seeds > 0 && (!seed_par || !seed_cov || !out_hits || !out_par || !out_cov || !out_score || !out_chi2 ||
                      !out_flags))
    return ctx->fail(MKF_ERR_ARG, "null array");
  BuildArgs a{seed_par, seed_cov, ev_seed_off, n_seeds, chi2_cut, max_cands, max_holes, min_hits, dup_frac,
              out_hits, out_layers, out_par, out_cov, out_score, out_chi2, out_counts, out_flags};
  cudaError_t e = launch_build(ctx, a, (cudaStream_t)stream);
  if (e == cudaErrorMemoryAllocation) return ctx->fail(MKF_ERR_OOM, "build workspace");
  if (e != cudaSuccess) return ctx->cuda_fail(e, "build_tracks");
  return MKF_OK;
}

mkf_status mkf_set_build_config(mkf_ctx* ctx, int warps_per_block, int lanes_per_seed) {
  if (check_ctx(ctx)) return MKF_ERR_ARG;
  if (warps_per_block != 1 && warps_per_block != 2 && warps_per_block != 4 && warps_per_block != 8)
    return ctx->fail(MKF_ERR_ARG, "warps_per_block must be 1, 2, 4 or 8");
  if (lanes_per_seed != 0 && lanes_per_seed != 1 && lanes_per_seed != 2 && lanes_per_seed != 4 &&
      lanes_per_seed != 8 && lanes_per_seed != 16 && lanes_per_seed != 32)
    return ctx->fail(MKF_ERR_ARG, "lanes_per_seed must be 0 or a power of two up to 32");
  ctx->build_warps = warps_per_block;
  ctx->build_group = lanes_per_seed;
  return MKF_OK;
}

mkf_status mkf_set_build_dedup(mkf_ctx* ctx, int enabled) {
  if (check_ctx(ctx)) return MKF_ERR_ARG;
  if (enabled != 0 && enabled != 1) return ctx->fail(MKF_ERR_ARG, "enabled must be 0 or 1");
  ctx->build_dedup = enabled;
  return MKF_OK;
}

mkf_status mkf_set_adjoint_config(mkf_ctx* ctx, int lanes_per_track) {
  if (check_ctx(ctx)) return MKF_ERR_ARG;
  if (lanes_per_track != 0 && lanes_per_track != 1 && lanes_per_track != 8)
    return ctx->fail(MKF_ERR_ARG, "lanes_per_track must be 0, 1 or 8");
  ctx->adjoint_lanes = lanes_per_track;
  return MKF_OK;
}

mkf_status mkf_set_debug(mkf_ctx* ctx, int brute_force_window_check) {
  if (check_ctx(ctx)) return MKF_ERR_ARG;
  ctx->debug_window = brute_force_window_check ? 1 : 0;
  return MKF_OK;
}

mkf_status mkf_set_timing(mkf_ctx* ctx, int on) {
  if (check_ctx(ctx)) return MKF_ERR_ARG;
  if (on && !ctx->timers_made) {
    for (int i = 0; i < kTimers; ++i) {
      MKF_CUDA(cudaEventCreate(&ctx->t_beg[i]), "event create");
      MKF_CUDA(cudaEventCreate(&ctx->t_end[i]), "event create");
    }
    ctx->timers_made = true;
  }
  ctx->timing = on ? 1 : 0;
  for (int i = 0; i < kTimers; ++i) ctx->timer_used[i] = false;
  return MKF_OK;
}

mkf_status mkf_get_timings(mkf_ctx* ctx, float* ms, int n, void* stream) {
  if (check_ctx(ctx)) return MKF_ERR_ARG;
  if (!ms || n < 0 || n > kTimers) return ctx->fail(MKF_ERR_ARG, "timings size");
  MKF_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "synchronize");
  for (int i = 0; i < n; ++i) {
    ms[i] = -1.0f;
    if (ctx->timers_made && ctx->timer_used[i]) MKF_CUDA(cudaEventElapsedTime(&ms[i], ctx->t_beg[i], ctx->t_end[i]), "elapsed");
  }
  return MKF_OK;
}

mkf_status mkf_get_stats(mkf_ctx* ctx, int64_t* out, int n, void* stream) {
  if (check_ctx(ctx)) return MKF_ERR_ARG;
  if (!out || n < 0 || n > 8) return ctx->fail(MKF_ERR_ARG, "stats size");
  cudaStream_t st = (cudaStream_t)stream;
  MKF_CUDA(cudaMemcpyAsync(out, ctx->stats.p, n * sizeof(int64_t), cudaMemcpyDeviceToHost, st), "stats read");
  MKF_CUDA(cudaStreamSynchronize(st), "synchronize");
  return MKF_OK;
}

mkf_status mkf_dedup_tracks(mkf_ctx* ctx, const int* hits, int L, const float* score, const int* nhits,
                            const int64_t* ev_seed_off, int n_events, int64_t n_seeds, int64_t n_hits_total,
                            int min_hits, float dup_frac, int* out_flags, void* stream) {
  if (check_ctx(ctx)) return MKF_ERR_ARG;
  if (L < 1 || L > MKF_MAX_LAYERS || n_events < 1 || n_seeds < 0 || n_hits_total < 0 ||
      n_hits_total > (int64_t)INT32_MAX - 1 || n_seeds > (int64_t)INT32_MAX / MKF_MAX_LAYERS)
    return ctx->fail(MKF_ERR_ARG, "bad sizes");
  if (min_hits < 0 || !(dup_frac >= 0.0f && dup_frac <= 1.0f)) return ctx->fail(MKF_ERR_ARG, "bad parameters");
  if (!ev_seed_off || (n_seeds > 0 && (!hits || !score || !nhits || !out_flags)))
    return ctx->fail(MKF_ERR_ARG, "null array");
  cudaError_t e = launch_dedup(ctx, hits, L, score, nhits, ev_seed_off, n_events, n_seeds, n_hits_total, min_hits,
                               dup_frac, out_flags, (cudaStream_t)stream);
  if (e == cudaErrorMemoryAllocation) return ctx->fail(MKF_ERR_OOM, "dedup workspace");
  if (e != cudaSuccess) return ctx->cuda_fail(e, "dedup");
  return MKF_OK;
}

static mkf_status fit_checks(mkf_ctx* ctx, const float* xyz, const float* lcov, const int* layer, int64_t n_hits,
                             const int* hits, int K, const float* init_par, int64_t n_tracks, const float* out_par,
                             const float* out_cov, const float* out_chi2) {
  if (check_ctx(ctx)) return MKF_ERR_ARG;
  if (!ctx->have_geom) return ctx->fail(MKF_ERR_STATE, "no geometry loaded");
  if (n_hits < 0 || n_hits > (int64_t)INT32_MAX - 1 || K < 1 || K > 4 * MKF_MAX_LAYERS || n_tracks < 0 ||
      n_tracks > (int64_t)INT32_MAX)
    return ctx->fail(MKF_ERR_ARG, "bad sizes");
  if (n_tracks > 0 && (!xyz || !lcov || !layer || !hits || !init_par || !out_par || !out_cov || !out_chi2))
    return ctx->fail(MKF_ERR_ARG, "null array");
  return MKF_OK;
}

mkf_status mkf_fit_tracks(mkf_ctx* ctx, const float* xyz, const float* lcov, const int* layer, int64_t n_hits,
                          const int* hits, int K, const float* init_par, const float* init_cov, int64_t n_tracks,
                          const float* align, const float* x0, float* out_par, float* out_cov, float* out_chi2,
                          int* out_ok, float* ckpt, void* stream) {
  mkf_status s = fit_checks(ctx, xyz, lcov, layer, n_hits, hits, K, init_par, n_tracks, out_par, out_cov, out_chi2);
  if (s) return s;
  if (n_tracks > 0 && !init_cov) return ctx->fail(MKF_ERR_ARG, "null init_cov");
  cudaError_t e = launch_fit(ctx, +1, xyz, lcov, layer, n_hits, hits, K, init_par, init_cov, n_tracks, align, x0,
                             out_par, out_cov, out_chi2, out_ok, ckpt, (cudaStream_t)stream);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "fit_tracks");
  return MKF_OK;
}

mkf_status mkf_fit_backward(mkf_ctx* ctx, const float* xyz, const float* lcov, const int* layer, int64_t n_hits,
                            const int* hits, int K, const float* init_par, int64_t n_tracks, const float* align,
                            const float* x0, float* out_par, float* out_cov, float* out_chi2, int* out_ok,
                            void* stream) {
  mkf_status s = fit_checks(ctx, xyz, lcov, layer, n_hits, hits, K, init_par, n_tracks, out_par, out_cov, out_chi2);
  if (s) return s;
  cudaError_t e = launch_fit(ctx, -1, xyz, lcov, layer, n_hits, hits, K, init_par, nullptr, n_tracks, align, x0,
                             out_par, out_cov, out_chi2, out_ok, nullptr, (cudaStream_t)stream);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "fit_backward");
  return MKF_OK;
}

mkf_status mkf_fit_tracks_adjoint(mkf_ctx* ctx, const float* xyz, const float* lcov, const int* layer,
                                  int64_t n_hits, const int* hits, int K, const float* init_par,
                                  const float* init_cov, int64_t n_tracks, const float* align, const float* x0,
                                  const float* ckpt, const float* g_chi2, const float* g_par, const float* g_cov,
                                  float* g_hit_xyz, float* g_align, float* g_x0, void* stream) {
  if (check_ctx(ctx)) return MKF_ERR_ARG;
  if (!ctx->have_geom) return ctx->fail(MKF_ERR_STATE, "no geometry loaded");
  if (n_hits < 0 || n_hits > (int64_t)INT32_MAX - 1 || K < 1 || K > 4 * MKF_MAX_LAYERS || n_tracks < 0 ||
      n_tracks > (int64_t)INT32_MAX)
    return ctx->fail(MKF_ERR_ARG, "bad sizes");
  if (n_tracks > 0 && (!xyz || !lcov || !layer || !hits || !init_par || !init_cov || !ckpt))
    return ctx->fail(MKF_ERR_ARG, "null array");
  if (!g_hit_xyz || !g_align || !g_x0) return ctx->fail(MKF_ERR_ARG, "null gradient output");
  cudaError_t e = launch_fit_adjoint(ctx, xyz, lcov, layer, n_hits, hits, K, init_par, init_cov, n_tracks, align,
                                     x0, ckpt, g_chi2, g_par, g_cov, g_hit_xyz, g_align, g_x0, (cudaStream_t)stream);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "fit_tracks_adjoint");
  return MKF_OK;
}

}  // extern "C"
