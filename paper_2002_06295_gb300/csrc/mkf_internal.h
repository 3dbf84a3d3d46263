// mkf_internal.h -- context, device geometry table and launch declarations
// shared by the translation units of the library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "mkf.h"
#include "mkf_geom.h"

namespace mkf {

// Grow-only device buffer owned by the context.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t want = bytes < 256 ? 256 : bytes;
    cudaError_t e = cudaMalloc(&p, want);
    if (e == cudaSuccess) cap = want;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <class T> T* as() const { return static_cast<T*>(p); }
};

struct BuildArgs {
  const float* seed_par;
  const float* seed_cov;
  const int64_t* ev_seed_off;
  int64_t n_seeds;
  float chi2_cut;
  int max_cands, max_holes, min_hits;
  float dup_frac;
  int* out_hits;
  int* out_layers;
  float* out_par;
  float* out_cov;
  float* out_score;
  float* out_chi2;
  int* out_counts;
  int* out_flags;
};

}  // namespace mkf

namespace mkf {
enum TimerId { kTBuild = 0, kTBin = 1, kTDedup = 2, kTFit = 3, kTAdjoint = 4, kTBackward = 5, kTimers = 8 };
}

struct mkf_ctx {
  int device = 0;
  int n_sm = 0;
  std::string err;
  bool have_geom = false;
  mkf::GeomDev geom{};
  mkf::DevBuf geom_dev;
  int debug_window = 0;
  int build_warps = 4;   // warps per block of the building kernel
  int build_group = 0;   // lanes per seed (0: max_cands rounded up to a power of two)
  int build_dedup = 1;   // mkf_build_tracks ends with duplicate removal
  int adjoint_lanes = 0; // lanes per track of the fit adjoint (0: by track count)
  int overlap_lanes = 0; // lanes per track of the overlap-hit search (0: by track count)
  int strip_chunk = 0;   // strips per staged chunk of the clustering kernel (0: default)
  int strip_events = 0;  // events per clustering work item (0: default)
  int strip_stages = 0;  // pipeline stages per warp of the clustering kernel (0: default)

  // binning
  bool binned = false;
  bool bins_ordered = false;   // each bin sorted by the caller's hit index
  int64_t n_hits = 0;
  int n_events = 0;
  int64_t n_bins_total = 0;
  mkf::DevBuf rec, rec_orig, perm, bin_off, bin_cnt, keys, ranks, vmax, ev_hit_off, scan_part;

  // build / dedup
  mkf::DevBuf seed_ctr, stats, status, dd_head, dd_next, dd_beat, dd_nbeat, dd_state, track_hits;
  mkf::DevBuf build_order;  // seeds in building order (per event, expected cost descending)
  mkf::DevBuf strip_bits;  // bad-strip flags packed to bits for the clustering kernel
  mkf::DevBuf seed_cnt, seed_off, seed_part, seed_pairs, seed_qcnt, seed_qoff;   // hit-based seeding
  mkf::DevBuf grid_key, grid_rank, grid_cnt, grid_off, grid_rec;                // its search grid
  mkf::DevBuf seed_stats;                                                       // its work counters
  mkf::DevBuf seed_scratch, seed_loc;   // per-warp triplet lists of the counting pass, their places
  int64_t seed_trip_hint = 0;           // triplets of the last seeding call (sizes the scratch)
  int64_t seed_trip_cap = 0;            // fixed triplet capacity of seeding (0: sized by a read-back)
  mkf::DevBuf ovl_stats;                                                        // overlap-hit search counters

  // optional stage timing (CUDA events on the launch stream)
  int timing = 0;
  bool timers_made = false;
  bool timer_used[mkf::kTimers] = {};
  cudaEvent_t t_beg[mkf::kTimers] = {}, t_end[mkf::kTimers] = {};
  void tick(int i, cudaStream_t st) {
    if (timing && timers_made) cudaEventRecord(t_beg[i], st);
  }
  void tock(int i, cudaStream_t st) {
    if (timing && timers_made) {
      cudaEventRecord(t_end[i], st);
      timer_used[i] = true;
    }
  }

  mkf_status fail(mkf_status code, const std::string& msg) {
    err = msg;
    return code;
  }
  mkf_status cuda_fail(cudaError_t e, const char* what) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return MKF_ERR_CUDA;
  }
};

namespace mkf {
// launchers (each returns the first CUDA error, or cudaSuccess)
cudaError_t launch_bin_order(mkf_ctx* ctx, cudaStream_t st);
// out[i] = in[0] + ... + in[i-1] for i <= n (out has n + 1 entries); part is scratch
cudaError_t launch_excl_scan(const int* in, int64_t n, int* out, DevBuf& part, cudaStream_t st);
cudaError_t launch_bin_hits(mkf_ctx* ctx, const float* xyz, const float* lcov, const int* layer, int64_t n_hits,
                            const int64_t* ev_hit_off, int n_events, const uint8_t* mask, cudaStream_t st);
cudaError_t launch_used_hits(mkf_ctx* ctx, const int* hits, const int* flags, int64_t n_tracks, int L,
                             int64_t n_hits, uint8_t* mask, cudaStream_t st);
cudaError_t launch_build(mkf_ctx* ctx, const BuildArgs& a, cudaStream_t st);
cudaError_t launch_dedup(mkf_ctx* ctx, const int* hits, int L, const float* score, const int* nhits,
                         const int64_t* ev_seed_off, int n_events, int64_t n_seeds, int64_t n_hits_total,
                         int min_hits, float dup_frac, int* out_flags, cudaStream_t st);
cudaError_t launch_fit(mkf_ctx* ctx, int direction, const float* xyz, const float* lcov, const int* layer,
                       int64_t n_hits, const int* hits, int K, const float* init_par, const float* init_cov,
                       int64_t n_tracks, const float* align, const float* x0, float* out_par, float* out_cov,
                       float* out_chi2, int* out_ok, float* ckpt, cudaStream_t st);
cudaError_t launch_fit_adjoint(mkf_ctx* ctx, const float* xyz, const float* lcov, const int* layer, int64_t n_hits,
                               const int* hits, int K, const float* init_par, const float* init_cov,
                               int64_t n_tracks, const float* align, const float* x0, const float* ckpt,
                               const float* g_chi2, const float* g_par, const float* g_cov, float* g_hit,
                               float* g_align, float* g_x0, cudaStream_t st);
}  // namespace mkf
