// dedup.cu -- duplicate removal (abstract: the excess of duplicate tracks is
// removed in an additional processing step).
//
// Rule: visit tracks by score (descending, ties by seed index) and drop a track
// that shares more than dup_frac * min(n_a, n_b) hits with an already kept one.
// That greedy result is the lexicographically first independent set of the
// "conflict" graph in rank order, and it is reached in parallel: a track is
// kept once every conflicting better-ranked track is decided and none is kept,
// dropped as soon as one of them is kept.  Each round decides at least the
// best undecided track, so the loop ends; the result does not depend on the
// order in which threads see the decisions.
//
// Hit ids are unique across events, so tracks of different events never
// conflict; one block resolves one event.
#include "mkf_internal.h"

namespace mkf {

namespace {

constexpr int kMaxNeighbours = 64;   // distinct tracks sharing a hit with one track
constexpr int kMaxBeaters = 32;      // conflicting better-ranked tracks kept per track

__global__ void k_dd_link(const int* __restrict__ hits, int L, const int* __restrict__ nhits, int64_t n_seeds,
                          int64_t n_hits, int min_hits, int* __restrict__ head, int* __restrict__ next,
                          int* __restrict__ status) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_seeds) return;
  if (nhits[a] < min_hits) return;
  for (int k = 0; k < L; ++k) {
    const int h = hits[a * L + k];
    if (h < 0) continue;
    if (h >= n_hits) {
      atomicOr(status, kStatBadInput);
      continue;
    }
    const int pair = (int)(a * L + k);
    next[pair] = atomicExch(&head[h], pair);
  }
}

__device__ __forceinline__ bool beats(float sb, int b, float sa, int a) { return sb > sa || (sb == sa && b < a); }

__global__ void k_dd_conflicts(const int* __restrict__ hits, int L, const float* __restrict__ score,
                               const int* __restrict__ nhits, int64_t n_seeds, int64_t n_hits, int min_hits,
                               float dup_frac, const int* __restrict__ head, const int* __restrict__ next,
                               int* __restrict__ beat, int* __restrict__ nbeat, int* __restrict__ status) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_seeds) return;
  nbeat[a] = 0;
  const int na = nhits[a];
  if (na < min_hits) return;
  int nb_id[kMaxNeighbours];
  int nb_ct[kMaxNeighbours];
  int n = 0;
  bool overflow = false;
  for (int k = 0; k < L; ++k) {
    const int h = hits[a * L + k];
    if (h < 0 || h >= n_hits) continue;
    for (int pr = head[h]; pr >= 0; pr = next[pr]) {
      const int b = pr / L;
      if (b == a) continue;
      int j = 0;
      while (j < n && nb_id[j] != b) ++j;
      if (j < n) {
        ++nb_ct[j];
      } else if (n < kMaxNeighbours) {
        nb_id[n] = b;
        nb_ct[n] = 1;
        ++n;
      } else {
        overflow = true;
      }
    }
  }
  const float sa = score[a];
  int m = 0;
  for (int j = 0; j < n; ++j) {
    const int b = nb_id[j];
    const int nmin = min(na, nhits[b]);
    if ((float)nb_ct[j] > dup_frac * (float)nmin && beats(score[b], b, sa, (int)a)) {
      if (m < kMaxBeaters)
        beat[a * kMaxBeaters + m] = b;
      else
        overflow = true;
      ++m;
    }
  }
  nbeat[a] = min(m, kMaxBeaters);
  if (overflow) atomicOr(status, kStatCapacity);
}

// state: 0 undecided, 1 kept, 2 duplicate, 3 short
__global__ void k_dd_resolve(const int64_t* __restrict__ ev_seed_off, const int* __restrict__ nhits, int min_hits,
                             const int* __restrict__ beat, const int* __restrict__ nbeat, int* state,
                             int* __restrict__ out_flags, unsigned long long* __restrict__ stats,
                             int* __restrict__ status) {
  const int64_t s0 = ev_seed_off[blockIdx.x], s1 = ev_seed_off[blockIdx.x + 1];
  for (int64_t a = s0 + threadIdx.x; a < s1; a += blockDim.x) state[a] = nhits[a] >= min_hits ? 0 : 3;
  __syncthreads();
  volatile int* vs = state;
  const int64_t rounds = s1 - s0 + 1;
  bool pending = true;
  for (int64_t r = 0; r < rounds && pending; ++r) {
    int changed = 0, undecided = 0;
    for (int64_t a = s0 + threadIdx.x; a < s1; a += blockDim.x) {
      if (vs[a] != 0) continue;
      bool any_kept = false, all_done = true;
      const int nb = nbeat[a];
      for (int j = 0; j < nb; ++j) {
        const int sb = vs[beat[a * kMaxBeaters + j]];
        if (sb == 1) {
          any_kept = true;
          break;
        }
        if (sb == 0) all_done = false;
      }
      if (any_kept) {
        vs[a] = 2;
        changed = 1;
      } else if (all_done) {
        vs[a] = 1;
        changed = 1;
      } else {
        undecided = 1;
      }
    }
    pending = __syncthreads_or(undecided) != 0;
    if (!__syncthreads_or(changed) && pending) {
      if (threadIdx.x == 0) atomicOr(status, kStatTimeout);
      break;
    }
  }
  __syncthreads();
  unsigned long long kept = 0;
  for (int64_t a = s0 + threadIdx.x; a < s1; a += blockDim.x) {
    const int st = vs[a];
    out_flags[a] = st == 1 ? MKF_TRK_KEPT : (st == 2 ? MKF_TRK_DUP : MKF_TRK_SHORT);
    kept += st == 1;
    if (st == 0) atomicOr(status, kStatTimeout);
  }
  for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
  if ((threadIdx.x & 31) == 0 && kept) atomicAdd(&stats[3], kept);
}

}  // namespace

cudaError_t launch_dedup(mkf_ctx* ctx, const int* hits, int L, const float* score, const int* nhits,
                         const int64_t* ev_seed_off, int n_events, int64_t n_seeds, int64_t n_hits_total,
                         int min_hits, float dup_frac, int* out_flags, cudaStream_t st) {
  cudaError_t e;
  const int64_t S = n_seeds > 0 ? n_seeds : 1;
  const int64_t H = n_hits_total > 0 ? n_hits_total : 1;
  if ((e = ctx->dd_head.ensure((size_t)H * 4)) != cudaSuccess) return e;
  if ((e = ctx->dd_next.ensure((size_t)S * L * 4)) != cudaSuccess) return e;
  if ((e = ctx->dd_beat.ensure((size_t)S * kMaxBeaters * 4)) != cudaSuccess) return e;
  if ((e = ctx->dd_nbeat.ensure((size_t)S * 4)) != cudaSuccess) return e;
  if ((e = ctx->dd_state.ensure((size_t)S * 4)) != cudaSuccess) return e;
  if (n_seeds == 0) return cudaSuccess;
  int* status = ctx->status.as<int>();
  if ((e = cudaMemsetAsync(ctx->dd_head.p, 0xFF, (size_t)H * 4, st))) return e;
  const int T = 256;
  ctx->tick(kTDedup, st);
  const unsigned gs = (unsigned)((n_seeds + T - 1) / T);
  k_dd_link<<<gs, T, 0, st>>>(hits, L, nhits, n_seeds, n_hits_total, min_hits, ctx->dd_head.as<int>(),
                              ctx->dd_next.as<int>(), status);
  k_dd_conflicts<<<gs, T, 0, st>>>(hits, L, score, nhits, n_seeds, n_hits_total, min_hits, dup_frac,
                                   ctx->dd_head.as<int>(), ctx->dd_next.as<int>(), ctx->dd_beat.as<int>(),
                                   ctx->dd_nbeat.as<int>(), status);
  k_dd_resolve<<<(unsigned)n_events, 1024, 0, st>>>(ev_seed_off, nhits, min_hits, ctx->dd_beat.as<int>(),
                                                    ctx->dd_nbeat.as<int>(), ctx->dd_state.as<int>(), out_flags,
                                                    ctx->stats.as<unsigned long long>(), status);
  ctx->tock(kTDedup, st);
  return cudaGetLastError();
}

}  // namespace mkf
