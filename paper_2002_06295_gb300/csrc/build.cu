// build.cu -- combinatorial Kalman-filter track building, persistent kernel.
//
// Method (paper Sec. 1-3 and abstract): every candidate of every seed is,
// step by step, propagated outward to its next reachable surface with its
// covariance transported and inflated for material; compatible hits are found
// from the (event, layer, phi, z|r) bins; chi2 is computed for each; children
// (hits with chi2 < cut, plus a hole child within the hole budget) are ranked
// by score = 10 n_hits - 10 n_holes - sum chi2 and only the best max_cands per
// seed are kept (the per-seed cap of Sec. 2); a candidate with no next surface
// or no child is finished and kept (short candidates, abstract); the best
// finished candidate is the seed's track.
//
// GB300 mapping:
//  * a seed is owned by a group of GS consecutive lanes of a warp (GS a power
//    of two >= N = max_cands, chosen per workload); lane k < N of the group
//    holds candidate slot k (6 parameters and the 21 floats of its covariance's
//    U-D factors, mkf_ud.cuh, in registers) for navigation, propagation,
//    the factors' transport with material; the propagated state, its position
//    covariance and the search window go to shared memory, the pre-step state
//    stays in registers;
//  * the whole warp scans the windows of all its candidates together: the phi
//    rows of the windows, then the hits of those rows, are dealt to the 32
//    lanes, and each lane's next hit record is copied to shared memory
//    (cp.async) while it works on the current one; a box test on the residuals
//    comes before the chi2;
//  * an accepted child (64-bit key: score, parent slot, hit index) goes into
//    its seed's top-N slots in shared memory by an atomicMin cascade, which
//    leaves the N best in order whatever the interleaving; lane k takes slot k;
//  * only the selected children are Kalman-updated (the score needs only the
//    predicted chi2), reading the parent's propagated state from shared memory;
//  * groups take seeds from a global queue (atomic counter) and refill as soon
//    as their seed is done, so one launch covers many events of uneven size;
//    the queue holds each event's seeds most expensive first (by 1/p), and
//    its first places are dealt so that those seeds spread one to a warp over
//    all blocks;
//    a warp without seeds helps the other warps of its block scan their wide
//    windows (shared-memory jobs claimed by CAS, every wait bounded);
//  * the parent pointers and hits of every step stay in shared memory and are
//    walked back once per seed.
#include "mkf_device.cuh"
#include "mkf_internal.h"
#include "mkf_ud.cuh"

namespace mkf {

namespace {

constexpr int kMaxWarps = 8;
// per-lane shared slot: p[6], U-D factors[21] (u[15], d[6]), score, nh,
// nholes|layer, rho, zeta, position covariance (xx, yx, yy, zx, zy, zz) (+1
// pad: an odd stride puts the same word of different lanes in different banks)
constexpr int kSlotWords = 39;
constexpr int kSlotPos = 32;   // first word of the position covariance
// per-lane window: kind, base bin, nphi, nw, b0, nb, iw0, iw1, ha, hb, hit base (+2 pad, odd stride)
constexpr int kWinWords = 13;
constexpr uint32_t kHoleKey = 0x0FFFFFFFu;
// block-level sharing of wide scans (see the kernel): a job has fewer than 2^16
// hit rounds (the round count shares a word with the job's epoch); every wait
// is bounded
constexpr int kJobMaxRounds = 1 << 16;
constexpr int kJobClaimTries = 256;
constexpr int kOwnerWaitLimit = 1 << 22;
constexpr int kHelperPollLimit = 1 << 24;
constexpr uint32_t kHistHole = 0x3FFFFFu;  // 22-bit local hit index field

struct BuildDev {
  const GeomDev* geom;
  const float4* rec;
  const float4* rec_orig;
  const int* bin_off;
  const float* vmax;
  const int64_t* ev_hit_off;
  const float* seed_par;
  const float* seed_cov;
  const int64_t* ev_seed_off;
  const int* order;   // building order of the seed rows (k_seed_order)
  int64_t n_seeds;
  int n_events;
  float chi2_cut;
  int ncand;
  int gsize;          // lanes per seed: a power of two >= ncand, <= 32
  int max_holes;
  int debug;
  int* out_hits;
  int* out_layers;
  float* out_par;
  float* out_cov;
  float* out_score;
  float* out_chi2;
  int* out_counts;
  int* out_flags;
  int* track_nh;
  unsigned long long* seed_ctr;
  unsigned long long* stats;
  int* status;
};

__device__ __forceinline__ uint32_t ordered(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unordered(uint32_t o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o);
}
// smaller key = better child: score descending, parent slot, hit (the caller's
// index of the hit relative to the event's first hit; kHoleKey for a hole)
__device__ __forceinline__ uint64_t child_key(float score, int slot, uint32_t hitkey) {
  return ((uint64_t)(~ordered(score)) << 32) | ((uint64_t)slot << 28) | hitkey;
}

// Plain (volatile) read of the NMAX slots of a seed's top-N array; the array
// starts on a 16-byte boundary when NMAX >= 2.
template <int NMAX>
__device__ __forceinline__ void top_read(const unsigned long long* ts, unsigned long long (&v)[NMAX]) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(ts);
  if constexpr (NMAX == 1) {
    asm volatile("ld.volatile.shared.u64 %0, [%1];\n" : "=l"(v[0]) : "r"(a) : "memory");
  } else {
#pragma unroll
    for (int j = 0; j < NMAX; j += 2)
      asm volatile("ld.volatile.shared.v2.u64 {%0, %1}, [%2];\n" : "=l"(v[j]), "=l"(v[j + 1]) : "r"(a + 8 * j) : "memory");
  }
}

// Insert key k into the ascending array ts[0..n) that holds the n smallest
// keys inserted so far (~0 = empty).  Any number of lanes may insert
// concurrently: every key reaching slot j leaves the smaller of it and the
// slot's value there and carries the larger on, so slot j ends up holding the
// j-th smallest key whatever the interleaving.  Slot values only decrease, so
// a slot read at or below the carried key stays there, and its atomicMin
// would change nothing: such slots are skipped on the strength of one plain
// read of the array, and the cascade of atomics starts at the first slot read
// above the key (a key not below the last slot can never enter and is
// dropped at once).  The result is the same as with an atomic on every slot.
template <int NMAX>
__device__ __forceinline__ void top_insert(unsigned long long* ts, int n, unsigned long long k) {
  unsigned long long v[NMAX];
  top_read<NMAX>(ts, v);
  unsigned long long last = v[0];
#pragma unroll
  for (int j = 1; j < NMAX; ++j)
    if (j == n - 1) last = v[j];
  if (!(k < last)) return;
#pragma unroll
  for (int j = 0; j < NMAX; ++j) {
    if (j >= n) break;
    if (v[j] <= k) continue;
    const unsigned long long old = atomicMin(&ts[j], k);
    if (old == ~0ull) return;
    k = old > k ? old : k;
  }
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory");
}

__device__ __forceinline__ HitRec unpack_rec(const float4 a, const float4 b) {
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
__device__ __forceinline__ HitRec load_rec(const float4* __restrict__ rec, int pos) {
  return unpack_rec(__ldg(&rec[2 * pos]), __ldg(&rec[2 * pos + 1]));
}

// first index of the ascending array v[0..n) whose value is above x (n if none,
// also for x = NaN)
__device__ __forceinline__ int first_above(const float* v, int n, float x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (v[mid] > x)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ int event_of(const int64_t* off, int n_events, int64_t i) {
  int lo = 0, hi = n_events;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= i)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// max of a 64-bit key over the lanes of a group (gm = the group's lane mask):
// a 32-bit reduction of the high words, then of the low words of the lanes
// that hold the largest high word
__device__ __forceinline__ uint64_t group_max(uint64_t v, unsigned gm) {
  const unsigned hi = (unsigned)(v >> 32), lo = (unsigned)v;
  const unsigned mh = __reduce_max_sync(gm, hi);
  const unsigned ml = __reduce_max_sync(gm, hi == mh ? lo : 0u);
  return ((uint64_t)mh << 32) | ml;
}

// MINB = 2 caps the registers at 128 per thread so that two 8-warp blocks fit
// an SM (the batched workloads, whose shared footprint allows two); MINB = 1
// lets the compiler keep the whole per-step working set in registers (no
// spills) where shared memory admits only one block per SM anyway.
template <int NMAX, bool DEBUG, int MINB>
__global__ void __launch_bounds__(kMaxWarps * 32, MINB) k_build(const BuildDev a) {
  extern __shared__ __align__(16) unsigned char smem[];
  GeomDev& G = *reinterpret_cast<GeomDev*>(smem);
  // shared scan jobs, one per warp: next = epoch << 16 | rounds claimed
  __shared__ int job_next[kMaxWarps], job_total[kMaxWarps], job_hw[kMaxWarps], job_done[kMaxWarps];
  __shared__ int n_idle, n_alive;
  if (threadIdx.x < kMaxWarps) {
    job_next[threadIdx.x] = 0;
    job_total[threadIdx.x] = 0;
    job_hw[threadIdx.x] = 0;
    job_done[threadIdx.x] = 0;
  }
  if (threadIdx.x == 0) {
    n_idle = 0;
    n_alive = blockDim.x >> 5;
  }
  {
    const int4* src = reinterpret_cast<const int4*>(a.geom);
    int4* dst = reinterpret_cast<int4*>(smem);
    for (int i = threadIdx.x; i < (int)(sizeof(GeomDev) / 16); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int W = blockDim.x >> 5;
  const int L = G.n_layers;
  const int N = a.ncand;
  const int GS = a.gsize;                     // lanes per seed (candidates on lanes 0..N-1)
  const int NG = 32 / GS;                     // groups per warp
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int gi = lane / GS;
  const int li = lane - gi * GS;
  const int gbase = gi * GS;
  const unsigned gfull = GS == 32 ? 0xffffffffu : ((1u << GS) - 1u);
  const unsigned gmask = gfull << gbase;

  float4* stage = reinterpret_cast<float4*>(smem + sizeof(GeomDev));               // [W][4 slots][32]
  float* prop = reinterpret_cast<float*>(stage + W * 32 * 4);                       // [W][32][kSlotWords]
  int* win = reinterpret_cast<int*>(prop + W * 32 * kSlotWords);                   // [W][32][kWinWords]
  int* cnt = win + W * 32 * kWinWords;                                              // [W][32] has a child
  int* rowp = cnt + W * 32;                                                         // [W][32]
  int* rpre = rowp + W * 32;                                                        // [W][32]
  int2* rbc = reinterpret_cast<int2*>(rpre + W * 32);                               // [W][32]
  unsigned long long* top = reinterpret_cast<unsigned long long*>(rbc + W * 32);    // [W][NG][NMAX]
  float* bests = reinterpret_cast<float*>(top + W * NG * NMAX);                     // [W][NG][32]
  uint32_t* hist = reinterpret_cast<uint32_t*>(bests + W * NG * 32);                // [W][NG][L][NMAX]
  float* myprop = prop + (warp * 32 + lane) * kSlotWords;
  // staging slot k of this lane: slot-major, so that the lanes' 16-byte
  // accesses to one slot are consecutive (no bank conflicts)
  float4* mystage = stage + warp * 32 * 4 + lane;
  float* gprop = prop + (warp * 32 + gbase) * kSlotWords;
  int* mywin = win + (warp * 32 + lane) * kWinWords;
  int* gwin = win + (warp * 32 + gbase) * kWinWords;
  const int* wrowp = rowp + warp * 32;
  const int* wpre = rpre + warp * 32;
  const int2* wbc = rbc + warp * 32;
  const int* wwin = win + warp * 32 * kWinWords;
  float* best = bests + (warp * NG + gi) * 32;
  unsigned long long* wtop = top + warp * NG * NMAX;
  unsigned long long* gtop = wtop + gi * NMAX;
  uint32_t* ghist = hist + (size_t)(warp * NG + gi) * L * NMAX;

  const float cut = a.chi2_cut;
  const float ck = G.c_kappa;
  // seeds whose count is known only on the device (hit-based seeding with a
  // fixed capacity): build the first ev_seed_off[E] of the n_seeds rows and
  // write the rest as empty tracks
  int64_t n_run = a.ev_seed_off[a.n_events];
  n_run = n_run < 0 ? 0 : (n_run < a.n_seeds ? n_run : a.n_seeds);
  for (int64_t r = n_run + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.n_seeds;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t S = a.n_seeds;
    for (int k = 0; k < 6; ++k) a.out_par[k * S + r] = 0.0f;
    for (int k = 0; k < 21; ++k) a.out_cov[k * S + r] = 0.0f;
    a.out_score[r] = 0.0f;
    a.out_chi2[r] = 0.0f;
    a.track_nh[r] = 0;
    if (a.out_counts) a.out_counts[r] = a.out_counts[S + r] = a.out_counts[2 * S + r] = 0;
    for (int k = 0; k < L; ++k) {
      a.out_hits[r * L + k] = -1;
      if (a.out_layers) a.out_layers[r * L + k] = -1;
    }
    a.out_flags[r] = MKF_TRK_SHORT;
  }
  unsigned long long n_steps = 0, n_chi2 = 0, n_full = 0, n_upd = 0, n_nav = 0, n_viol = 0;

  // per-group seed state (replicated over the group's lanes)
  int64_t seed = -1;
  int ev = 0, step = 0;
  int hit_base = 0, ebin = 0;
  // per-lane candidate
  bool active = false;
  float p[6];
  UD6 u;
  float score = 0.f, rho = 0.f, zeta = 0.f;
  int nh = 0, nholes = 0;

  // Take the next seed for every group with want == true.  Called by all lanes
  // of the warp together (it shuffles).
  // The first seeds are dealt, not queued: group g of warp w in block b takes
  // place (g W + w) gridDim + b of the building order, so the most expensive
  // seeds of an event (the order puts them first) go one to a warp and spread
  // over all blocks, instead of landing wherever the queue's first atomics
  // happen to come from; every later seed comes from the queue.
  const int64_t n_dealt = (int64_t)gridDim.x * W * NG;
  bool first = true;
  auto fetch = [&](bool want) {
    unsigned long long s = 0;
    if (want && li == 0) {
      if (first)
        s = ((unsigned long long)gi * W + warp) * gridDim.x + blockIdx.x;
      else
        s = (unsigned long long)n_dealt + atomicAdd(a.seed_ctr, 1ull);
    }
    first = false;
    s = __shfl_sync(0xffffffffu, s, gbase);
    if (!want) return;
    if ((int64_t)s < n_run) {
      // order[] holds every row below n_run once when the event offsets are
      // consistent; anything else read there is replaced by the plain row
      const int o = a.order[s];
      seed = o >= 0 && (int64_t)o < n_run ? (int64_t)o : (int64_t)s;
    } else {
      seed = -1;
    }
    active = false;
    step = 0;
    if (seed >= 0) {
      ev = event_of(a.ev_seed_off, a.n_events, seed);
      hit_base = (int)a.ev_hit_off[ev];
      ebin = ev * G.bins_per_event;
      if (li == 0) {
        active = true;
        const int64_t S = a.n_seeds;
#pragma unroll
        for (int k = 0; k < 6; ++k) p[k] = a.seed_par[k * S + seed];
        float C[21];
#pragma unroll
        for (int k = 0; k < 21; ++k) C[k] = a.seed_cov[k * S + seed];
        ud_from_cov(C, u);
        score = 0.f;
        nh = nholes = 0;
        rho = sqrtf(fmaf(p[0], p[0], p[1] * p[1]));
        zeta = fabsf(p[2]);
        best[30] = __int_as_float(-2);   // no finished candidate yet
        atomicAdd(&a.stats[6], 1ull);
      }
    }
  };
  fetch(true);

  // One candidate-hit pair of warp ow's scan: box test, chi2, and an accepted
  // child into the seed's top-N slots (any warp of the block may run it).
  auto scan_pair = [&](int ow, int cc, const HitRec& hr) {
    const int* wd = win + (ow * 32 + cc) * kWinWords;
    const float* ps = prop + (ow * 32 + cc) * kSlotWords;
    const int kind = wd[0];
    ++n_chi2;
    if (hit_in_box(kind, ps[0], ps[1], ps[2], hr, __int_as_float(wd[8]), __int_as_float(wd[9]))) {
      ++n_full;
      const PosState q{ps[0], ps[1], ps[2], ps[kSlotPos], ps[kSlotPos + 1], ps[kSlotPos + 2],
                       ps[kSlotPos + 3], ps[kSlotPos + 4], ps[kSlotPos + 5]};
      const float chi2 = hit_chi2(kind, q, hr, cut);
      if (chi2 < cut) {
        cnt[ow * 32 + cc] = 1;   // the candidate has a child (only "none" is tested)
        const uint32_t hloc = (uint32_t)(hr.orig - wd[10]);
        top_insert<NMAX>(top + (ow * NG + cc / GS) * NMAX, N,
                   child_key(ps[27] + 10.0f - chi2, cc & (GS - 1), hloc < kHoleKey ? hloc : kHoleKey - 1));
      }
    }
  };
  // Claim hit rounds of warp ow's published job and scan them until none is
  // left; the rounds done are then added to the job's count.  A claim is a CAS
  // on (epoch, rounds claimed): a stale read of a finished job fails the CAS.
  auto work_job = [&](int ow) {
    int processed = 0;
    for (int it = 0; it < kJobMaxRounds; ++it) {
      int r = -1, hw = 0;
      if (lane == 0) {
        for (int tries = 0; tries < kJobClaimTries; ++tries) {
          const int v = *reinterpret_cast<volatile int*>(&job_next[ow]);
          __threadfence_block();
          const int tot = *reinterpret_cast<volatile int*>(&job_total[ow]);
          if ((v & 0xFFFF) >= tot) break;
          hw = *reinterpret_cast<volatile int*>(&job_hw[ow]);
          if (atomicCAS(&job_next[ow], v, v + 1) == v) {
            r = v & 0xFFFF;
            break;
          }
        }
      }
      r = __shfl_sync(0xffffffffu, r, 0);
      hw = __shfl_sync(0xffffffffu, hw, 0);
      if (r < 0) break;
      const int h = r * 32 + lane;
      if (h < hw) {
        const int* opre = rpre + ow * 32;
        int j = 0;
#pragma unroll
        for (int st = 16; st > 0; st >>= 1)
          if (opre[j + st] <= h) j += st;
        const int2 bc = rbc[ow * 32 + j];
        scan_pair(ow, bc.y, load_rec(a.rec, bc.x + (h - opre[j])));
      }
      ++processed;
    }
    __syncwarp();
    if (lane == 0 && processed > 0) {
      __threadfence_block();
      atomicAdd(&job_done[ow], processed);
    }
  };

  for (;;) {
    if (__all_sync(0xffffffffu, seed < 0)) break;
    // ---- (1) navigation: next reachable surface outward
    int nl = -1;
    float ns = INFINITY;
    HelixPt<float> hn;        // the helix at a disk crossing found by the navigation
    bool have_hn = false;
    float sin_t = 1.f, cos_t = 0.f, cot_t = 0.f, omega = 0.f, sph = 0.f, cph = 1.f;
    if (active && step < L) {
      msincos(p[5], &sin_t, &cos_t);
      cot_t = cos_t / sin_t;
      omega = ck * p[3];
      msincos(p[4], &sph, &cph);
      // The transverse path to radius R is at least R - r0 (an arc is no
      // shorter than its chord), and z moves monotonically along it, so a
      // barrel whose z range lies behind z0 + (R - r0) cot(theta) on the side
      // of motion cannot be crossed inside its acceptance.  The path bound is
      // shrunk by a margin far above FP32 rounding, so this test rejects only
      // barrels that the exact crossing would reject too; it is armed once a
      // crossing has fallen outside a barrel's z range (forward tracks), so
      // that tracks accepted by their first barrel pay nothing for it.
      bool zcut = false;
      float r0 = 0.f;
      // surfaces already passed form a prefix of each sorted list
      for (int i = first_above(G.barrel_r, G.n_barrel, rho + kNavEps); i < G.n_barrel; ++i) {
        const int l = G.barrel_order[i];
        const LayerDev& ly = G.L[l];
        if (zcut) {
          const float smin = fmaf(ly.pos - r0, 0.999f, -1e-3f);
          if (smin > 0.0f) {
            const float zb = fmaf(smin, cot_t, p[2]);
            if (cot_t > 0.0f ? zb > ly.hi : zb < ly.lo) continue;
          }
        }
        ++n_nav;
        const float s = cylinder_path(p[0], p[1], cph, sph, omega, ly.pos, +1);
        if (!(s < INFINITY)) break;    // the particle's circle stays inside: larger radii too
        const float z = fmaf(s, cot_t, p[2]);
        if (z >= ly.lo && z <= ly.hi) {
          nl = l;
          ns = s;
          break;
        }
        if (!zcut) {
          zcut = true;
          r0 = sqrtf(fmaf(p[0], p[0], p[1] * p[1]));
        }
      }
      if (cot_t != 0.0f) {
        const int nd = cot_t > 0.f ? G.n_dpos : G.n_dneg;
        const int8_t* ord = cot_t > 0.f ? G.dpos_order : G.dneg_order;
        const float* dz = cot_t > 0.f ? G.dpos_z : G.dneg_z;
        // a particle leaving the tracking volume is lost: disks count only
        // when crossed before r = r_max
        float s_lim = ns;
        bool exit_known = false;
        for (int i = first_above(dz, nd, zeta + kNavEps); i < nd; ++i) {
          const int l = ord[i];
          const LayerDev& ly = G.L[l];
          ++n_nav;
          const float s = plane_path(p[2], cot_t, ly.pos, +1);
          if (!(s < s_lim)) break;     // |z| ordered: later disks are farther
          if (!exit_known) {
            s_lim = fminf(ns, cylinder_path(p[0], p[1], cph, sph, omega, G.r_max, +1));
            exit_known = true;
            if (!(s < s_lim)) break;
          }
          const auto h = helix_at(p[0], p[1], p[2], p[4], cph, sph, cot_t, omega, s);
          const float r = sqrtf(fmaf(h.x, h.x, h.y * h.y));
          if (r >= ly.lo && r <= ly.hi) {
            nl = l;
            ns = s;
            hn = h;
            have_hn = true;
            break;
          }
        }
      }
    }
    // ---- (2) propagate, transport the covariance, add material, build the
    // window, and publish the propagated state and window for the group
    bool hole_ok = false;
    mywin[5] = 0;
    if (nl >= 0) {
      ++n_steps;
      const LayerDev ly = G.L[nl];
      const int kind = ly.kind;
      const auto h = have_hn ? hn : helix_at(p[0], p[1], p[2], p[4], cph, sph, cot_t, omega, ns);
      const auto J = transport_jacobian(kind, p, h, ns, omega, ck, cot_t, sin_t);
      float ms_phi = 0.0f, ms_theta = 0.0f;
      if (ly.x0 > 0.0f) {
        ms_theta = highland_theta0_sq(kind, ly.x0, h.x, h.y, h.cphi, h.sphi, p[3], sin_t, cos_t);
        ms_phi = ms_theta / (sin_t * sin_t);
      }
      // The transported factors go to shared memory and the candidate keeps its
      // pre-step factors in registers (the state a candidate that finishes
      // here is stored with).  To free registers during the transport, the
      // pre-step factors wait in the slot, the transport runs in place, and
      // the two are then swapped word by word.
#pragma unroll
      for (int k = 0; k < 15; ++k) myprop[6 + k] = u.u[k];
#pragma unroll
      for (int k = 0; k < 6; ++k) myprop[21 + k] = u.d[k];
      ud_transport(J, u, ms_phi, ms_theta);
      float cp6[6];
      ud_pos_block(u, cp6);
#pragma unroll
      for (int k = 0; k < 15; ++k) {
        const float t = myprop[6 + k];
        myprop[6 + k] = u.u[k];
        u.u[k] = t;
      }
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const float t = myprop[21 + k];
        myprop[21 + k] = u.d[k];
        u.d[k] = t;
      }
#pragma unroll
      for (int k = 0; k < 6; ++k) myprop[kSlotPos + k] = cp6[k];
      const float cpos[4] = {cp6[0], cp6[1], cp6[2], cp6[5]};
      const float rc = sqrtf(fmaf(h.x, h.x, h.y * h.y));
      // conservative window: |r_i| < sqrt(cut R_ii) (Cauchy-Schwarz), R_ii bounded
      // by the largest eigenvalue of C_xy (or C_zz) plus the layer's largest hit variance
      const float va = __ldg(&a.vmax[2 * (ev * L + nl)]);
      const float vb = __ldg(&a.vmax[2 * (ev * L + nl) + 1]);
      const float cxx = cpos[0], cyy = cpos[2], cxy = cpos[1];
      const float hd = 0.5f * (cxx - cyy);
      const float lam = 0.5f * (cxx + cyy) + sqrtf(fmaf(hd, hd, cxy * cxy));
      const float ha = sqrtf(cut * (lam + va)) * 1.05f + 1e-4f;
      const float hb = sqrtf(cut * ((kind == 0 ? cpos[3] : lam) + vb)) * 1.05f + 1e-4f;
      const float phic = atan2f(h.y, h.x);
      float dphi = ha >= rc ? 0.5f * kPi : asinf(ha / rc);
      dphi = dphi * 1.001f + 1e-5f;
      const float lo_f = floorf((phic - dphi + kPi) * ly.phi_scale);
      const float hi_f = floorf((phic + dphi + kPi) * ly.phi_scale);
      float wlo, whi;
      if (kind == 0) {
        wlo = h.z - hb;
        whi = h.z + hb;
      } else {
        wlo = fmaf(rc, cosf(fminf(dphi, 0.5f * kPi)), -hb);
        whi = rc + hb;
      }
      mywin[0] = kind;
      mywin[1] = ebin + ly.bin_base;
      mywin[2] = ly.nphi;
      mywin[3] = ly.nw;
      mywin[4] = (int)lo_f;
      mywin[5] = max(min((int)(hi_f - lo_f) + 1, ly.nphi), 1);
      mywin[6] = min(max((int)floorf((wlo - ly.lo) * ly.w_scale), 0), ly.nw - 1);
      mywin[7] = min(max((int)floorf((whi - ly.lo) * ly.w_scale), 0), ly.nw - 1);
      mywin[8] = __float_as_int(ha);
      mywin[9] = __float_as_int(hb);
      mywin[10] = hit_base;
      myprop[0] = h.x;
      myprop[1] = h.y;
      myprop[2] = h.z;
      myprop[3] = p[3];
      myprop[4] = wrap_phi(h.phi);
      myprop[5] = p[5];
      myprop[27] = score;
      myprop[28] = __int_as_float(nh);
      myprop[29] = __int_as_float(nholes | (nl << 16));
      myprop[30] = kind == 0 ? ly.pos : fmaxf(rho, rc);
      myprop[31] = kind == 0 ? fmaxf(zeta, fabsf(h.z)) : fabsf(ly.pos);
      hole_ok = nholes + 1 <= a.max_holes;
    }
    cnt[warp * 32 + lane] = 0;
    __syncwarp();
    // ---- (3) the warp scans the windows of all its candidates together.
    // A window is nb phi rows, each a contiguous range of hits (w bins
    // iw0..iw1).  The rows of all the warp's candidates are dealt to the 32
    // lanes, then the hits of those rows, so every lane's loads are
    // independent and a seed with a wide window does not hold up the warp;
    // each lane's next hit record is copied to shared memory (cp.async) while
    // it works on the current one.  Each hit gets the box test, then its chi2 if
    // it passes; an accepted child goes straight into its seed's top-N slots.
    if (li < N) gtop[li] = ~0ull;
    __syncwarp();
    {
      const int nbl = mywin[5];
      int incl = nbl;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += o;
      }
      const int Mw = __shfl_sync(0xffffffffu, incl, 31);
      rowp[warp * 32 + lane] = incl - nbl;
      __syncwarp();
      for (int r0 = 0; r0 < Mw; r0 += 32) {
        const int t = r0 + lane;
        int beg = 0, len = 0, cl = 0;
        if (t < Mw) {
          // candidate lane owning row t: last lane whose row prefix is <= t
#pragma unroll
          for (int st = 16; st > 0; st >>= 1)
            if (wrowp[cl + st] <= t) cl += st;
          const int* wd = wwin + cl * kWinWords;
          int b = (wd[4] + (t - wrowp[cl])) % wd[2];
          if (b < 0) b += wd[2];
          const int row = wd[1] + b * wd[3];
          beg = __ldg(&a.bin_off[row + wd[6]]);
          len = __ldg(&a.bin_off[row + wd[7] + 1]) - beg;
        }
        int hin = len;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const int o = __shfl_up_sync(0xffffffffu, hin, off);
          if (lane >= off) hin += o;
        }
        const int Hw = __shfl_sync(0xffffffffu, hin, 31);
        rpre[warp * 32 + lane] = hin - len;
        rbc[warp * 32 + lane] = make_int2(beg, cl);
        __syncwarp();
        const int R = (Hw + 31) >> 5;
        int idle = 0;
        if (lane == 0 && R >= 2 && R < kJobMaxRounds) idle = *reinterpret_cast<volatile int*>(&n_idle);
        idle = __shfl_sync(0xffffffffu, idle, 0);
        if (idle > 0) {
          // warps of this block whose seeds are all done share these hit rounds
          if (lane == 0) {
            // close the job word first (round field 0xFFFF: no claim passes and
            // every stale CAS fails), then write the job, then open it
            const int ep = ((job_next[warp] >> 16) + 1) & 0x7FFF;
            atomicExch(&job_next[warp], (ep << 16) | 0xFFFF);
            __threadfence_block();
            job_total[warp] = R;
            job_hw[warp] = Hw;
            job_done[warp] = 0;
            __threadfence_block();
            atomicExch(&job_next[warp], ep << 16);
          }
          __syncwarp();
          int fin = 0;
          for (int it = 0; it < kOwnerWaitLimit; ++it) {
            work_job(warp);
            if (lane == 0) fin = *reinterpret_cast<volatile int*>(&job_done[warp]) >= R;
            fin = __shfl_sync(0xffffffffu, fin, 0);
            if (fin) break;
            __nanosleep(32);
          }
          if (!fin && lane == 0) atomicOr(a.status, kStatTimeout);
          __threadfence_block();
          __syncwarp();
          continue;
        }
        // the row holding flattened hit h: last lane whose hit prefix is <= h
        auto locate = [&](int h, int& cc, int& pos) {
          int j = 0;
#pragma unroll
          for (int st = 16; st > 0; st >>= 1)
            if (wpre[j + st] <= h) j += st;
          const int2 bc = wbc[j];
          cc = bc.y;
          pos = bc.x + (h - wpre[j]);
        };
        // a lane's next record is copied to shared memory while it works on the current one
        int cc_n = -1, pos_n = 0;
        if (lane < Hw) {
          locate(lane, cc_n, pos_n);
          cp_async16(mystage, a.rec + 2 * pos_n);
          cp_async16(mystage + 32, a.rec + 2 * pos_n + 1);
        }
        cp_async_commit();
        for (int h0 = 0, buf = 0; h0 < Hw; h0 += 32, buf ^= 2) {
          const int cc = cc_n;
          cc_n = -1;
          if (h0 + 32 + lane < Hw) {
            locate(h0 + 32 + lane, cc_n, pos_n);
            cp_async16(mystage + 32 * (buf ^ 2), a.rec + 2 * pos_n);
            cp_async16(mystage + 32 * ((buf ^ 2) + 1), a.rec + 2 * pos_n + 1);
          }
          cp_async_commit();
          cp_async_wait<1>();
          if (cc >= 0) scan_pair(warp, cc, unpack_rec(mystage[32 * buf], mystage[32 * (buf + 1)]));
        }
        cp_async_wait<0>();
        __syncwarp();
      }
    }
    if (DEBUG) {
      // brute force over each candidate's whole layer: every accepted hit must
      // pass the box test and lie in the window's bins
      for (int c = 0; c < N; ++c) {
        const int* wd = gwin + c * kWinWords;
        const int nb = wd[5];
        if (nb <= 0) continue;
        const int kind = wd[0], base = wd[1], nphi = wd[2], nw = wd[3], b0 = wd[4], iw0 = wd[6], iw1 = wd[7];
        const float* ps = gprop + c * kSlotWords;
        const PosState q{ps[0], ps[1], ps[2], ps[kSlotPos], ps[kSlotPos + 1], ps[kSlotPos + 2],
                         ps[kSlotPos + 3], ps[kSlotPos + 4], ps[kSlotPos + 5]};
        const int lbase = base - ebin;
        const int beg = __ldg(&a.bin_off[base]);
        const int end = __ldg(&a.bin_off[base + nphi * nw]);
        for (int qh = beg + li; qh < end; qh += GS) {
          const HitRec hr = load_rec(a.rec, qh);
          if (hit_chi2(kind, q, hr, cut) < cut) {
            const int lb = hr.bin - lbase;
            const int ip = lb / nw, iw = lb - ip * nw;
            int d = (ip - b0) % nphi;
            if (d < 0) d += nphi;
            const bool in_box = hit_in_box(kind, q.x, q.y, q.z, hr, __int_as_float(wd[8]), __int_as_float(wd[9]));
            if (!(iw >= iw0 && iw <= iw1 && d < nb && in_box)) ++n_viol;
          }
        }
      }
    }
    if (hole_ok) top_insert<NMAX>(gtop, N, child_key(score - 10.0f, li, kHoleKey));
    __syncwarp();
    const int nk = nl >= 0 ? cnt[warp * 32 + lane] + (hole_ok ? 1 : 0) : 0;
    const bool finishing = active && (nl < 0 || nk == 0);
    // ---- (4) per-seed selection: the slots hold the seed's best N children in
    // order; lane li of the group takes the li-th
    const uint64_t my_child = li < N ? gtop[li] : ~0ull;
    // ---- (5) finished candidates: keep the group's best (score, then earlier step, lower slot)
    {
      const uint64_t fk = finishing ? (((uint64_t)ordered(score) << 32) | (uint32_t)(NMAX - li)) : 0ull;
      const uint64_t fb = group_max(fk, gmask);
      if (finishing && fk == fb) {
        const int last = __float_as_int(best[30]);
        if (last == -2 || score > best[27]) {
#pragma unroll
          for (int k = 0; k < 6; ++k) best[k] = p[k];
#pragma unroll
          for (int k = 0; k < 15; ++k) best[6 + k] = u.u[k];
#pragma unroll
          for (int k = 0; k < 6; ++k) best[21 + k] = u.d[k];
          best[27] = score;
          best[28] = __int_as_float(nh);
          best[29] = __int_as_float(nholes);
          best[30] = __int_as_float(step - 1);
          best[31] = __int_as_float(li);
        }
      }
    }
    __syncwarp();
    // ---- (6) Kalman update of the selected children
    active = false;
    if (my_child != ~0ull) {
      const int parent = (int)((my_child >> 28) & 0xFu);
      const uint32_t hk = (uint32_t)(my_child & 0x0FFFFFFFu);
      const float* ps = gprop + parent * kSlotWords;
#pragma unroll
      for (int k = 0; k < 6; ++k) p[k] = ps[k];
#pragma unroll
      for (int k = 0; k < 15; ++k) u.u[k] = ps[6 + k];
#pragma unroll
      for (int k = 0; k < 6; ++k) u.d[k] = ps[21 + k];
      nh = __float_as_int(ps[28]);
      const int packed = __float_as_int(ps[29]);
      nholes = packed & 0xFFFF;
      const int lay = packed >> 16;
      rho = ps[30];
      zeta = ps[31];
      score = unordered(~(uint32_t)(my_child >> 32));
      uint32_t hloc = kHistHole;
      if (hk != kHoleKey) {
        const HitRec hr = load_rec(a.rec_orig, hit_base + (int)hk);
        const Meas<float> m{hr.c, hr.s, hr.w, hr.v00, hr.v01, hr.v11};
        ud_update(G.L[lay].kind, p, u, m);
        ++nh;
        ++n_upd;
        hloc = hk;
        if (hloc >= kHistHole) atomicOr(a.status, kStatCapacity);
      } else {
        ++nholes;
      }
      ghist[step * NMAX + li] = (hloc & kHistHole) | ((uint32_t)lay << 22) | ((uint32_t)parent << 28);
      active = true;
    }
    __syncwarp();
    // ---- (7) seed done: write the track, take the next seed
    const bool any = (__ballot_sync(0xffffffffu, active) & gmask) != 0;
    const bool done = seed >= 0 && !any;
    if (done) {
      const int64_t S = a.n_seeds;
      const int last = __float_as_int(best[30]);
      const int bslot = __float_as_int(best[31]);
      for (int k = li; k < 6; k += GS) a.out_par[k * S + seed] = best[k];
      if (li == 0) {
        UD6 fb;
#pragma unroll
        for (int k = 0; k < 15; ++k) fb.u[k] = best[6 + k];
#pragma unroll
        for (int k = 0; k < 6; ++k) fb.d[k] = best[21 + k];
        float Cb[21];
        ud_to_cov(fb, Cb);
#pragma unroll
        for (int k = 0; k < 21; ++k) a.out_cov[k * S + seed] = Cb[k];
      }
      if (li == 0) {
        const int bnh = __float_as_int(best[28]);
        const int bho = __float_as_int(best[29]);
        const float bsc = best[27];
        a.out_score[seed] = bsc;
        a.out_chi2[seed] = 10.0f * (float)(bnh - bho) - bsc;
        a.track_nh[seed] = bnh;
        if (a.out_counts) {
          a.out_counts[seed] = bnh;
          a.out_counts[S + seed] = bho;
          a.out_counts[2 * S + seed] = last + 1;
        }
        int* oh = a.out_hits + seed * L;
        int* ol = a.out_layers ? a.out_layers + seed * L : nullptr;
        for (int k = last + 1; k < L; ++k) {
          oh[k] = -1;
          if (ol) ol[k] = -1;
        }
        int slot = bslot;
        for (int k = last; k >= 0; --k) {
          const uint32_t e = ghist[k * NMAX + slot];
          const uint32_t hl = e & kHistHole;
          oh[k] = hl == kHistHole ? -1 : hit_base + (int)hl;
          if (ol) ol[k] = (int)((e >> 22) & 0x3Fu);
          slot = (int)(e >> 28);
        }
      }
    } else if (seed >= 0) {
      ++step;
    }
    __syncwarp();
    fetch(done);
  }
  // ---- no seed left for this warp: help the block's other warps with their
  // wide scans until every warp of the block is done
  if (lane == 0) {
    atomicAdd(&n_idle, 1);
    atomicSub(&n_alive, 1);
  }
  for (int it = 0; it < kHelperPollLimit; ++it) {
    int alive = 0, pending = 0;
    if (lane == 0) {
      alive = *reinterpret_cast<volatile int*>(&n_alive);
      for (int ow = 0; ow < W; ++ow) {
        const int v = *reinterpret_cast<volatile int*>(&job_next[ow]);
        const int tot = *reinterpret_cast<volatile int*>(&job_total[ow]);
        if ((v & 0xFFFF) < tot) pending |= 1 << ow;
      }
    }
    alive = __shfl_sync(0xffffffffu, alive, 0);
    pending = __shfl_sync(0xffffffffu, pending, 0);
    if (pending) {
      for (int ow = 0; ow < W; ++ow)
        if (pending & (1 << ow)) work_job(ow);
    } else {
      if (alive == 0) break;
      __nanosleep(64);
    }
    if (it == kHelperPollLimit - 1 && lane == 0) atomicOr(a.status, kStatTimeout);
  }
  // ---- counters
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n_steps += __shfl_xor_sync(0xffffffffu, n_steps, o);
    n_chi2 += __shfl_xor_sync(0xffffffffu, n_chi2, o);
    n_full += __shfl_xor_sync(0xffffffffu, n_full, o);
    n_upd += __shfl_xor_sync(0xffffffffu, n_upd, o);
    n_nav += __shfl_xor_sync(0xffffffffu, n_nav, o);
    n_viol += __shfl_xor_sync(0xffffffffu, n_viol, o);
  }
  if (lane == 0) {
    atomicAdd(&a.stats[0], n_steps);
    atomicAdd(&a.stats[1], n_chi2);
    atomicAdd(&a.stats[2], n_upd);
    atomicAdd(&a.stats[4], n_viol);
    atomicAdd(&a.stats[5], n_nav);
    atomicAdd(&a.stats[7], n_full);
  }
}

// Building order of the seed rows: within each event (whose rows stay in
// their range, events in order) the seeds by descending expected cost, taken
// as sin(theta) |kappa| = 1/p of the seed: slow particles curl and scatter,
// so their windows are wide and their chains of steps long.  The order only
// decides when a seed is built; the tracks do not depend on it.  One block per
// event: a 64-bucket counting sort on log2(1/p) (quarter octaves), rows of one
// bucket in any order.
constexpr int kOrderBuckets = 64;
constexpr int kOrderThreads = 1024;
__device__ __forceinline__ int order_bucket(const float* __restrict__ seed_par, int64_t n_seeds, int64_t r) {
  const float ip = fabsf(seed_par[3 * n_seeds + r]) * fabsf(__sinf(seed_par[5 * n_seeds + r]));
  // 1/p from 2^-4 to 2^12 /GeV in quarter octaves; heavy (large 1/p) first
  const float q = 4.0f * (__log2f(fmaxf(ip, 1e-30f)) + 4.0f);
  const int b = (int)fminf(fmaxf(q, 0.0f), (float)(kOrderBuckets - 1));
  return kOrderBuckets - 1 - b;
}
// Rows before the first offset count with event 0 (as in the building kernel's
// event lookup); offsets are clamped to the rows that are built.  The lanes of
// a warp that fall in one bucket are counted and placed with one atomic
// (__match_any_sync), so that heavy traffic on a few buckets does not
// serialise the block.
__global__ void __launch_bounds__(kOrderThreads) k_seed_order(const float* __restrict__ seed_par,
                                                              const int64_t* __restrict__ ev_seed_off, int n_events,
                                                              int64_t n_seeds, int* __restrict__ order) {
  __shared__ int cnt[kOrderBuckets];
  int64_t n_run = ev_seed_off[n_events];
  n_run = n_run < 0 ? 0 : (n_run < n_seeds ? n_run : n_seeds);
  const int e = blockIdx.x;
  int64_t s0 = e == 0 ? 0 : ev_seed_off[e];
  int64_t s1 = ev_seed_off[e + 1];
  s0 = s0 < 0 ? 0 : (s0 < n_run ? s0 : n_run);
  s1 = s1 < s0 ? s0 : (s1 < n_run ? s1 : n_run);
  if (threadIdx.x < kOrderBuckets) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  // the loops run a whole number of warp rounds, so every lane reaches the
  // warp-wide calls; lanes past the range take part with bucket -1
  const int64_t n = s1 - s0;
  const int64_t rounds = (n + blockDim.x - 1) / blockDim.x;
  for (int64_t it = 0; it < rounds; ++it) {
    const int64_t r = s0 + it * blockDim.x + threadIdx.x;
    const int b = r < s1 ? order_bucket(seed_par, n_seeds, r) : -1;
    const unsigned m = __match_any_sync(0xffffffffu, b);
    if (b >= 0 && (m & lt) == 0) atomicAdd(&cnt[b], __popc(m));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int b = 0; b < kOrderBuckets; ++b) {
      const int c = cnt[b];
      cnt[b] = acc;
      acc += c;
    }
  }
  __syncthreads();
  for (int64_t it = 0; it < rounds; ++it) {
    const int64_t r = s0 + it * blockDim.x + threadIdx.x;
    const int b = r < s1 ? order_bucket(seed_par, n_seeds, r) : -1;
    const unsigned m = __match_any_sync(0xffffffffu, b);
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (b >= 0 && lane == leader) base = atomicAdd(&cnt[b], __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (b >= 0) order[s0 + base + __popc(m & lt)] = (int)r;
  }
}

template <int NMAX>
size_t build_smem(int L, int W, int GS) {
  const int NG = 32 / GS;
  return sizeof(GeomDev) + (size_t)W * 32 * 64 + (size_t)W * 32 * (kSlotWords + kWinWords + 1 + 4) * 4 +
         (size_t)W * NG * NMAX * 8 +
         (size_t)W * NG * 32 * 4 +
         (size_t)W * NG * L * NMAX * 4;
}

template <int NMAX, bool DEBUG, int MINB>
cudaError_t launch_build_kernel(mkf_ctx* ctx, const BuildDev& d, int W, size_t sm, int per_sm, cudaStream_t st) {
  const int GS = d.gsize;
  const int64_t groups_needed = (d.n_seeds + (32 / GS) - 1) / (32 / GS);
  const int64_t blocks = (groups_needed + W - 1) / W;
  int64_t grid = (int64_t)ctx->n_sm * per_sm;
  if (blocks < grid) grid = blocks;
  if (grid < 1) grid = 1;
  ctx->tick(kTBuild, st);
  k_build<NMAX, DEBUG, MINB><<<(unsigned)grid, W * 32, sm, st>>>(d);
  ctx->tock(kTBuild, st);
  return cudaGetLastError();
}

// Blocks of the kernel instance that fit one SM with this launch's shared memory.
template <int NMAX, bool DEBUG, int MINB>
cudaError_t build_occupancy(int W, size_t sm, int* per_sm) {
  cudaError_t e =
      cudaFuncSetAttribute(k_build<NMAX, DEBUG, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  *per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_build<NMAX, DEBUG, MINB>, W * 32, sm);
  if (*per_sm < 1) *per_sm = 1;
  return e;
}

// The register-unbounded instance (MINB = 1) is launched when it keeps as many
// blocks per SM as the 128-register one; otherwise the 128-register instance.
template <int NMAX, bool DEBUG>
cudaError_t run_build(mkf_ctx* ctx, const BuildDev& d, cudaStream_t st) {
  int W = ctx->build_warps;
  if (W < 1 || W > kMaxWarps) W = 4;
  const size_t sm = build_smem<NMAX>(ctx->geom.n_layers, W, d.gsize);
  int per2 = 0, per1 = 0;
  cudaError_t e = build_occupancy<NMAX, DEBUG, 2>(W, sm, &per2);
  if (e != cudaSuccess) return e;
  if constexpr (!DEBUG) {
    if ((e = build_occupancy<NMAX, DEBUG, 1>(W, sm, &per1)) != cudaSuccess) return e;
    if (per1 >= per2) return launch_build_kernel<NMAX, DEBUG, 1>(ctx, d, W, sm, per1, st);
  }
  return launch_build_kernel<NMAX, DEBUG, 2>(ctx, d, W, sm, per2, st);
}

}  // namespace

cudaError_t launch_build(mkf_ctx* ctx, const BuildArgs& a, cudaStream_t st) {
  cudaError_t e;
  const int64_t S = a.n_seeds;
  if ((e = ctx->track_hits.ensure((size_t)(S > 0 ? S : 1) * 4)) != cudaSuccess) return e;
  if ((e = ctx->build_order.ensure((size_t)(S > 0 ? S : 1) * 4)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(ctx->seed_ctr.p, 0, sizeof(unsigned long long), st))) return e;
  if ((e = cudaMemsetAsync(ctx->stats.p, 0, 8 * sizeof(int64_t), st))) return e;
  if (S > 0) {
    BuildDev d;
    d.geom = ctx->geom_dev.as<GeomDev>();
    d.rec = ctx->rec.as<float4>();
    d.rec_orig = ctx->rec_orig.as<float4>();
    d.bin_off = ctx->bin_off.as<int>();
    d.vmax = ctx->vmax.as<float>();
    d.ev_hit_off = ctx->ev_hit_off.as<int64_t>();
    d.seed_par = a.seed_par;
    d.seed_cov = a.seed_cov;
    d.ev_seed_off = a.ev_seed_off;
    d.order = ctx->build_order.as<int>();
    d.n_seeds = S;
    d.n_events = ctx->n_events;
    d.chi2_cut = a.chi2_cut;
    d.ncand = a.max_cands;
    {
      int gs = 1;
      while (gs < a.max_cands) gs <<= 1;
      d.gsize = ctx->build_group > gs ? ctx->build_group : gs;
    }
    d.max_holes = a.max_holes;
    d.debug = ctx->debug_window;
    d.out_hits = a.out_hits;
    d.out_layers = a.out_layers;
    d.out_par = a.out_par;
    d.out_cov = a.out_cov;
    d.out_score = a.out_score;
    d.out_chi2 = a.out_chi2;
    d.out_counts = a.out_counts;
    d.out_flags = a.out_flags;
    d.track_nh = ctx->track_hits.as<int>();
    d.seed_ctr = ctx->seed_ctr.as<unsigned long long>();
    d.stats = ctx->stats.as<unsigned long long>();
    d.status = ctx->status.as<int>();
    if (ctx->n_events > 0)
      k_seed_order<<<(unsigned)ctx->n_events, kOrderThreads, 0, st>>>(a.seed_par, a.ev_seed_off, ctx->n_events, S,
                                                            ctx->build_order.as<int>());
    // the brute-force window check has a kernel of its own (any N <= 8), so
    // the production kernels carry none of its code
    if (d.debug)
      e = run_build<8, true>(ctx, d, st);
    else if (a.max_cands <= 1)
      e = run_build<1, false>(ctx, d, st);
    else if (a.max_cands <= 2)
      e = run_build<2, false>(ctx, d, st);
    else if (a.max_cands <= 4)
      e = run_build<4, false>(ctx, d, st);
    else
      e = run_build<8, false>(ctx, d, st);
    if (e != cudaSuccess) return e;
  }
  if (!ctx->build_dedup) return cudaSuccess;   // the caller runs mkf_dedup_tracks
  return launch_dedup(ctx, a.out_hits, ctx->geom.n_layers, a.out_score, ctx->track_hits.as<int>(), a.ev_seed_off,
                      ctx->n_events, S, ctx->n_hits, a.min_hits, a.dup_frac, a.out_flags, st);
}

}  // namespace mkf
