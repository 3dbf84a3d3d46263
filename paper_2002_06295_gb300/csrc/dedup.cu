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

constexpr int kMaxNeighbours = 64;   // distinct tracks sharing a hit with one track, listed
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

// Calls f(b) for every beater b of track a: a track that shares more than
// dup_frac * min(n_a, n_b) hits with a and ranks higher.  Every track b that
// shares a hit with a is met through the hit -> track lists; the pair is
// taken once, at a's first hit that b also holds, where the shared hits are
// counted directly from both rows (L^2 compares).  Nothing is stored per
// neighbour, so any number of tracks may share a's hits.  f returns false to
// stop early.
template <class F>
__device__ __forceinline__ void for_each_beater(int64_t a, const int* __restrict__ hits, int L,
                                                const float* __restrict__ score, const int* __restrict__ nhits,
                                                int64_t n_hits, float dup_frac, const int* __restrict__ head,
                                                const int* __restrict__ next, F f) {
  const int* ra = hits + a * L;
  const int na = nhits[a];
  const float sa = score[a];
  for (int k = 0; k < L; ++k) {
    const int h = ra[k];
    if (h < 0 || h >= n_hits) continue;
    for (int pr = head[h]; pr >= 0; pr = next[pr]) {
      const int b = pr / L;
      if (b == a) continue;
      const int* rb = hits + (int64_t)b * L;
      int shared = 0, first = L;
      for (int j = 0; j < L; ++j) {
        const int hj = ra[j];
        if (hj < 0 || hj >= n_hits) continue;
        bool in_b = false;
        for (int q = 0; q < L && !in_b; ++q) in_b = rb[q] == hj;
        if (in_b) {
          ++shared;
          first = j < first ? j : first;
        }
      }
      if (first != k) continue;   // taken at an earlier hit of a
      const int nmin = min(na, nhits[b]);
      if ((float)shared > dup_frac * (float)nmin && beats(score[b], b, sa, (int)a))
        if (!f(b)) return;
    }
  }
}

// Beaters of each track from its neighbours: every track sharing a hit with
// it is met through the hit -> track lists and its shared hits counted in a
// short list.  A track with more than kMaxNeighbours neighbours or
// kMaxBeaters beaters is marked (nbeat = -1): the resolution then derives its
// beaters again with for_each_beater, which stores nothing per neighbour, each
// time it looks at it.  So no input overflows; the marked tracks (tens of the
// 1.4 M of a hit-seeded batch) only cost more.
__global__ void k_dd_conflicts(const int* __restrict__ hits, int L, const float* __restrict__ score,
                               const int* __restrict__ nhits, int64_t n_seeds, int64_t n_hits, int min_hits,
                               float dup_frac, const int* __restrict__ head, const int* __restrict__ next,
                               int* __restrict__ beat, int* __restrict__ nbeat) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_seeds) return;
  nbeat[a] = 0;
  const int na = nhits[a];
  if (na < min_hits) return;
  int nb_id[kMaxNeighbours];
  int nb_ct[kMaxNeighbours];
  int n = 0;
  bool overflow = false;
  for (int k = 0; k < L && !overflow; ++k) {
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
        break;
      }
    }
  }
  const float sa = score[a];
  int m = 0;
  for (int j = 0; j < n && !overflow; ++j) {
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
  nbeat[a] = overflow ? -1 : m;
}

// state: 0 undecided, 1 kept, 2 duplicate, 3 short.  The event offsets come
// from the caller's device memory: they are clamped to [0, n_seeds] (and the
// end to no less than the start) so that a wrong offset can never index past
// the track arrays; clamping sets the bad-input status bit.  stats may be NULL.
__global__ void k_dd_resolve(const int64_t* __restrict__ ev_seed_off, int64_t n_seeds, const int* __restrict__ nhits,
                             int min_hits, const int* __restrict__ beat, const int* __restrict__ nbeat, int* state,
                             int* __restrict__ out_flags, unsigned long long* __restrict__ stats,
                             int* __restrict__ status, const int* __restrict__ hits, int L,
                             const float* __restrict__ score, int64_t n_hits, float dup_frac,
                             const int* __restrict__ head, const int* __restrict__ next) {
  const int64_t r0 = ev_seed_off[blockIdx.x], r1 = ev_seed_off[blockIdx.x + 1];
  const int64_t s0 = r0 < 0 ? 0 : (r0 > n_seeds ? n_seeds : r0);
  const int64_t s1 = r1 < s0 ? s0 : (r1 > n_seeds ? n_seeds : r1);
  if ((s0 != r0 || s1 != r1) && threadIdx.x == 0) atomicOr(status, kStatBadInput);
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
      if (nb >= 0) {
        for (int j = 0; j < nb; ++j) {
          const int sb = vs[beat[a * kMaxBeaters + j]];
          if (sb == 1) {
            any_kept = true;
            break;
          }
          if (sb == 0) all_done = false;
        }
      } else {
        for_each_beater(a, hits, L, score, nhits, n_hits, dup_frac, head, next, [&](int b) {
          const int sb = vs[b];
          if (sb == 1) any_kept = true;
          if (sb == 0) all_done = false;
          return !any_kept;
        });
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
  if (stats && (threadIdx.x & 31) == 0 && kept) atomicAdd(&stats[3], kept);
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
                                   ctx->dd_nbeat.as<int>());
  k_dd_resolve<<<(unsigned)n_events, 1024, 0, st>>>(ev_seed_off, n_seeds, nhits, min_hits, ctx->dd_beat.as<int>(),
                                                    ctx->dd_nbeat.as<int>(), ctx->dd_state.as<int>(), out_flags,
                                                    ctx->stats.as<unsigned long long>(), status, hits, L, score,
                                                    n_hits_total, dup_frac, ctx->dd_head.as<int>(),
                                                    ctx->dd_next.as<int>());
  ctx->tock(kTDedup, st);
  return cudaGetLastError();
}

}  // namespace mkf

// ---------------------------------------------------------------------------
// Allocation-free duplicate removal.
//
// Some callers cannot allocate device memory once they are running: a trigger
// or online-reconstruction process that reserves its whole memory budget at
// start-up, or a host thread that must not take cudaMalloc's implicit device
// synchronisation while other streams are busy.  For them this variant keeps
// its working memory in one fixed array in the library's device image (held
// by every GPU that loads the library until the process exits) and never calls
// cudaMalloc, cudaFree or any allocating routine.  Sizes beyond the array's
// limits are rejected with MKF_ERR_CAPACITY before anything is enqueued.
// Every call uses the same array: calls whose work overlaps on the GPU (other
// streams, other host threads) race with each other and must be serialised by
// the caller.
#include <mutex>

namespace mkf {
namespace {

constexpr int64_t kNaMaxSeeds = 16384;
constexpr int64_t kNaMaxHits = 524288;
constexpr size_t kNaHead = (size_t)kNaMaxHits;                        // head[hit]
constexpr size_t kNaNext = (size_t)kNaMaxSeeds * MKF_MAX_LAYERS;      // next[seed * L + k]
constexpr size_t kNaBeat = (size_t)kNaMaxSeeds * kMaxBeaters;         // beat[seed * 32 + j]
constexpr size_t kNaWords = kNaHead + kNaNext + kNaBeat + 2 * (size_t)kNaMaxSeeds + 64;

// 8.5 MB of working memory, 256-byte aligned, in the device image.
static __device__ __align__(256) int g_dedup_scratch[kNaWords];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
int* g_na_ptr[kNaMaxDevices] = {};

// Device address of g_dedup_scratch on the current device, looked up once per
// device (the host-side symbol is only a stand-in and must not be passed to a
// kernel).  The address is cached for the life of the process: it assumes the
// device's primary context stays alive.  After cudaDeviceReset (or anything
// else that destroys and recreates the primary context) the cached address is
// stale, so this entry point must not be called again in that process.
cudaError_t noalloc_scratch(int** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_dedup_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = static_cast<int*>(p);
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace mkf

extern "C" mkf_status mkf_dedup_tracks_noalloc(const int* hits, int L, const float* score, const int* nhits,
                                               const int64_t* ev_seed_off, int n_events, int64_t n_seeds,
                                               int64_t n_hits_total, int min_hits, float dup_frac, int* out_flags,
                                               int* out_status, void* stream) {
  using namespace mkf;
  if (L < 1 || L > MKF_MAX_LAYERS || n_events < 1 || n_seeds < 0 || n_hits_total < 0) return MKF_ERR_ARG;
  if (min_hits < 0 || !(dup_frac >= 0.0f && dup_frac <= 1.0f)) return MKF_ERR_ARG;
  if (!ev_seed_off || (n_seeds > 0 && (!hits || !score || !nhits || !out_flags))) return MKF_ERR_ARG;
  if (n_seeds > kNaMaxSeeds || n_hits_total > kNaMaxHits) return MKF_ERR_CAPACITY;
  cudaStream_t st = (cudaStream_t)stream;
  int* base = nullptr;
  if (noalloc_scratch(&base) != cudaSuccess) return MKF_ERR_CUDA;
  int* head = base;
  int* next = head + kNaHead;
  int* beat = next + kNaNext;
  int* nbeat = beat + kNaBeat;
  int* state = nbeat + kNaMaxSeeds;
  // status word used when the caller passes none (the kept-track counter of the
  // context path is not kept here: no shared counter grows across calls)
  int* status = out_status ? out_status : state + kNaMaxSeeds;
  // the array keeps the previous call's contents: reset what must start fresh
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return MKF_ERR_CUDA;
  if (n_seeds == 0) return MKF_OK;
  const int64_t H = n_hits_total > 0 ? n_hits_total : 1;
  if (cudaMemsetAsync(head, 0xFF, (size_t)H * sizeof(int), st) != cudaSuccess) return MKF_ERR_CUDA;
  const int T = 256;
  const unsigned gs = (unsigned)((n_seeds + T - 1) / T);
  k_dd_link<<<gs, T, 0, st>>>(hits, L, nhits, n_seeds, n_hits_total, min_hits, head, next, status);
  k_dd_conflicts<<<gs, T, 0, st>>>(hits, L, score, nhits, n_seeds, n_hits_total, min_hits, dup_frac, head, next, beat,
                                   nbeat);
  k_dd_resolve<<<(unsigned)n_events, 1024, 0, st>>>(ev_seed_off, n_seeds, nhits, min_hits, beat, nbeat, state,
                                                    out_flags, nullptr, status, hits, L, score, n_hits_total,
                                                    dup_frac, head, next);
  return cudaGetLastError() == cudaSuccess ? MKF_OK : MKF_ERR_CUDA;
}
