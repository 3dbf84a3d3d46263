// seeds.cu -- hit-based seeding of prompt tracks from the four innermost
// barrel (pixel) layers (Sec. 3).  The paper names the layers and the target
// (prompt tracks) only; the rules are this library's reading:
//  * a pair (a on layer 0, b on layer 1) gives the circle through the beam
//    line (origin), a and b -- signed curvature omega = 2 (A x B) / (|A| |B|
//    |A - B|) -- and the line z = z0 + cot s in the transverse path s(r) =
//    2 asin(omega r / 2) / omega; it passes if |omega| <= alpha Bz / pt_min
//    and |z0| <= z_max;
//  * a hit c on layer 2 passes if its transverse residual R2 sin(phi_c -
//    phi_pred) and its z residual against that helix are within rphi_tol and
//    z_tol; the helix through the origin, a and c predicts layer 3 the same
//    way for a hit d;
//  * b lies within 90 degrees of a in azimuth, c and d within 90 degrees of
//    their predictions (a sine residual alone would also pass a hit's mirror
//    image through the beam line);
//  * the seed state sits on the beam line (0, 0, z0): curvature and direction
//    from the circle through the origin, b and d, cot theta and z0 from the
//    line through a and d.
// Hits are their measured direction on the layer radius (cos phi, sin phi, z
// from the building records).  Windows come from a seeding grid of fine
// (phi, z) cells over the four layers, built here by a counting sort: each
// pair looks only at the layer-1 cells its cuts allow (a conservative phi and
// z range), each triplet at the cells around its predictions.
// Two stages, each a counting pass, an exclusive scan and a writing pass, so
// the seeds come in a fixed order (event, layer-0 bin, hit, then the window
// order, bins sorted by hit id) and ev_seed_off is a plain CSR:
//  1. one warp per layer-0 hit: the rows of its layer-1 window are fetched
//     together and the lanes test the window's hits 32 at a time; a lane whose
//     pair passes searches that pair's layer-2 window -> triplet list.  The
//     counting pass also keeps each hit's triplets (in order) in a per-warp
//     scratch segment, so the writing pass is a copy to the scanned places
//     (or, if a segment overflowed, the search again);
//  2. one thread per triplet: its layer-3 window -> seeds.
// The triplet total is read back once (one stream synchronisation) to size
// the triplet list; so the call returns when stage 1 is done, and it cannot be
// captured in a CUDA graph.
#include <algorithm>

#include "mkf_device.cuh"
#include "mkf_internal.h"

namespace mkf {

namespace {

constexpr float kAlphaF = 0.00299792458f;   // GeV / (T cm)
constexpr int kSeedThreads = 128;
constexpr float kWinPhiPad = 2e-5f;   // rad, rounding pad of the phi windows
constexpr float kWinZPad = 1e-3f;     // cm, rounding pad of the z windows

// Seeding grid: each seeding layer of each event is cut into kGridPhi x kGridZ
// cells (much finer than the building bins, whose size suits the building
// windows), so a layer-2 or layer-3 window holds one or two cells.
constexpr int kGridPhi = 256;
constexpr int kGridZ = 32;
constexpr int kGridCells = kGridPhi * kGridZ;

struct SeedArgs {
  LayerDev L[4];          // the seeding grid of each seeding layer (lo, nphi, nw, bin_base, scales)
  int mb0[4], mb1[4];     // local bin range of each seeding layer in the building bins
  float R[4];
  float omega_max, z_max, rphi_tol, z_tol;
  float dphi1;            // half-width of the layer-1 phi window
  float rho_lo, rho_hi;   // range of s(R1) / s(R0) over |omega| <= omega_max
  float dphi2, dphi3;     // half-widths of the layer-2 and layer-3 phi windows
  float bz;
  int n_events, bins_per_event;
  int64_t max_seeds;
};

struct SHit {
  float c, s, z;
  int orig;
};

// seeding-grid record: cos phi, sin phi, z, caller hit id
__device__ __forceinline__ SHit load_shit(const float4* __restrict__ rec, int pos) {
  const float4 a = __ldg(&rec[pos]);
  return SHit{a.x, a.y, a.z, __float_as_int(a.w)};
}

// transverse path from the origin to radius r on a circle of curvature omega
__device__ __forceinline__ float arc_sf(float omega, float r) {
  const float x = 0.5f * omega * r;
  return fabsf(x) < 1e-4f ? r * fmaf(x * x, 1.0f / 6.0f, 1.0f) : 2.0f * asinf(x) / omega;
}

// signed curvature of the circle through the origin, ra (a.c, a.s) and rb (b.c, b.s)
__device__ __forceinline__ float circle_origin(float ra, const SHit& a, float rb, const SHit& b) {
  const float cross = ra * rb * fmaf(a.c, b.s, -a.s * b.c);
  const float dx = fmaf(rb, b.c, -ra * a.c), dy = fmaf(rb, b.s, -ra * a.s);
  return 2.0f * cross / (ra * rb * sqrtf(fmaf(dx, dx, dy * dy)));
}

// direction of the point at radius r of the circle through the origin and ra (a.c, a.s)
__device__ __forceinline__ void circle_dir(float omega, float ra, const SHit& a, float r, float* c, float* s) {
  const float d = asinf(0.5f * omega * r) - asinf(0.5f * omega * ra);
  float sd, cd;
  sincosf(d, &sd, &cd);
  *c = fmaf(a.c, cd, -a.s * sd);
  *s = fmaf(a.s, cd, a.c * sd);
}

// Window of one layer of one event: phi rows from the low edge (wrapping),
// z bins [iw0, iw1] of each row (contiguous hits).
struct Window {
  int ip0, nrow, iw0, iw1;
};

__device__ __forceinline__ Window make_window(const LayerDev& ly, float phi_c, float dphi, float z_lo, float z_hi) {
  Window w;
  w.ip0 = (int)floorf((phi_c - dphi + kPi) * ly.phi_scale);
  const int ip1 = (int)floorf((phi_c + dphi + kPi) * ly.phi_scale);
  w.nrow = min(ip1 - w.ip0 + 1, ly.nphi);
  w.iw0 = min(max((int)floorf((z_lo - ly.lo) * ly.w_scale), 0), ly.nw - 1);
  w.iw1 = min(max((int)floorf((z_hi - ly.lo) * ly.w_scale), 0), ly.nw - 1);
  return w;
}

// hit range [p0, p1) of row k of a window
__device__ __forceinline__ int2 window_row(const LayerDev& ly, int ebase, const Window& w, int k,
                                           const int* __restrict__ bin_off) {
  int ip = (w.ip0 + k) % ly.nphi;
  if (ip < 0) ip += ly.nphi;
  const int b0 = ebase + ly.bin_base + ip * ly.nw;
  return make_int2(__ldg(&bin_off[b0 + w.iw0]), __ldg(&bin_off[b0 + w.iw1 + 1]));
}

// One thread visits the hits of a window in order (rows, z bins, bin order).
template <class F>
__device__ __forceinline__ void for_window(const LayerDev& ly, int ebase, const Window& w,
                                           const int* __restrict__ bin_off, const float4* __restrict__ rec, F&& f) {
  for (int k = 0; k < w.nrow; ++k) {
    const int2 r = window_row(ly, ebase, w, k, bin_off);
    for (int p = r.x; p < r.y; ++p) f(load_shit(rec, p), p);
  }
}

// asin(x) / x, exact to FP32 rounding also near x = 0
__device__ __forceinline__ float asin_over(float x) {
  return fabsf(x) < 1e-4f ? fmaf(x * x, 1.0f / 6.0f, 1.0f) : asinf(x) / x;
}

// Pair cuts for the layer-0 hit a and a layer-1 hit b.  A passing pair keeps
// what its layer-2 prediction needs: curvature w, g0 = asin(u0) / u0 (u0 = w
// R0 / 2; s(R0) = R0 g0) and cot theta.
struct PairCut {
  bool ok;
  float w, g0, cot;
};
__device__ __forceinline__ PairCut pair_cut(const SeedArgs& A, const SHit& a, const SHit& b) {
  PairCut p{false, 0.f, 0.f, 0.f};
  if (!(fmaf(a.c, b.c, a.s * b.s) > 0.f)) return p;   // opposite sides of the beam line
  p.w = circle_origin(A.R[0], a, A.R[1], b);
  if (!(fabsf(p.w) <= A.omega_max)) return p;
  p.g0 = asin_over(0.5f * p.w * A.R[0]);
  const float s0 = A.R[0] * p.g0;
  p.cot = (b.z - a.z) / (A.R[1] * asin_over(0.5f * p.w * A.R[1]) - s0);
  p.ok = fabsf(fmaf(-p.cot, s0, a.z)) <= A.z_max;
  return p;
}

// Prediction on layer 2 of a passing pair (azimuth, direction, z): one more
// arcsine serves both the path s(R2) = R2 asin(u2) / u2 and the turning angle.
struct PairPred {
  bool ok;
  float phip, cp, sp, zp;
};
__device__ __forceinline__ PairPred pair_predict(const SeedArgs& A, const SHit& a, float phia, const PairCut& p) {
  PairPred q{true, 0.f, 0.f, 0.f, 0.f};
  const float u0 = 0.5f * p.w * A.R[0], u2 = 0.5f * p.w * A.R[2];
  const float g2 = asin_over(u2);
  const float z0 = fmaf(-p.cot, A.R[0] * p.g0, a.z);
  const float d = fmaf(u2, g2, -u0 * p.g0);   // asin(u2) - asin(u0)
  float sd, cd;
  sincosf(d, &sd, &cd);
  q.cp = fmaf(a.c, cd, -a.s * sd);
  q.sp = fmaf(a.s, cd, a.c * sd);
  q.phip = phia + d;
  q.zp = fmaf(p.cot, A.R[2] * g2, z0);
  return q;
}

// Layer-2 hits that continue a passing pair: f(c, position) for each, in window order.
template <class F>
__device__ __forceinline__ void for_layer2(const SeedArgs& A, int ebase, const PairPred& q,
                                           const int* __restrict__ bin_off, const float4* __restrict__ rec,
                                           int& examined, F&& f) {
  const Window w2 = make_window(A.L[2], q.phip, A.dphi2, q.zp - A.z_tol - kWinZPad, q.zp + A.z_tol + kWinZPad);
  for_window(A.L[2], ebase, w2, bin_off, rec, [&](const SHit& c, int p) {
    ++examined;
    if (fmaf(c.c, q.cp, c.s * q.sp) > 0.f && fabsf(A.R[2] * fmaf(c.s, q.cp, -c.c * q.sp)) <= A.rphi_tol &&
        fabsf(c.z - q.zp) <= A.z_tol)
      f(c, p);
  });
}

// Work counters (layer-1 hits examined, pairs passed, layer-2 hits examined,
// triplets; layer-3 hits examined, seeds): one atomic per warp and counter.
__device__ __forceinline__ void warp_add_stats(unsigned long long* stats, int v0, int v1, int v2, int v3, int k0) {
  int v[4] = {v0, v1, v2, v3};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    int x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&stats[k0 + k], (unsigned long long)x);
  }
}

// Stage 1: one warp per layer-0 hit (items over all events; l0_cum is the CSR
// of the events' layer-0 hit counts), persistent grid.  The rows of its
// layer-1 window are fetched together (one per lane) and the lanes take the
// window's hits 32 at a time in order; passing pairs go to a per-warp queue
// (in order) and are taken 32 at a time, one per lane, to search their
// layer-2 windows.  Count pass: tcnt[item] = triplets; write pass:
// triplets[toff[item] + k] = (layer-0, layer-1, layer-2 positions, event's
// first cell), in order (pair, then layer-2 hit).
template <bool WRITE>
__global__ void __launch_bounds__(kSeedThreads)
    k_seed_triplets(const SeedArgs A, const float4* __restrict__ rec, const int* __restrict__ bin_off,
                    const int* __restrict__ l0_cum, int64_t n_slots, int* __restrict__ tcnt,
                    const int* __restrict__ toff, int4* __restrict__ trip, unsigned long long* __restrict__ stats,
                    int4* __restrict__ scratch, int64_t seg_cap, int64_t* __restrict__ item_loc,
                    int* __restrict__ overflow, int64_t trip_cap = -1) {
  const int lane = threadIdx.x & 31;
  // write pass launched without a host decision (fixed triplet capacity): it
  // runs only if a scratch segment overflowed, and only if the list fits
  if (WRITE && trip_cap >= 0 && (!*(volatile int*)overflow || __ldg(&toff[n_slots]) > trip_cap)) return;
  // count pass with a scratch list: the warp keeps each item's triplets, in
  // order and contiguous, in its own segment of `scratch`
  const bool keep = !WRITE && scratch != nullptr;
  const int64_t seg_base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * seg_cap;
  int64_t cursor = 0;      // used part of the warp's segment (uniform)
  bool full = false;       // the segment overflowed (uniform)
  int st_l1 = 0, st_pairs = 0, st_l2 = 0, st_trip = 0;   // work counters (count pass; per lane)
  __shared__ int4 queue_all[kSeedThreads / 32][64];   // per warp: passing pairs in order (layer-1 position, w, g0, cot)
  int4* queue = queue_all[threadIdx.x >> 5];
  const int64_t B = A.bins_per_event;
  const int n_items = __ldg(&l0_cum[A.n_events]);
  const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); item < n_items;
       item += n_warps) {
    int lo = 0, hi = A.n_events;   // event: l0_cum[e] <= item < l0_cum[e + 1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(&l0_cum[mid]) <= item)
        lo = mid;
      else
        hi = mid;
    }
    const int ebase = (int)(lo * B);
    const int pos = __ldg(&bin_off[ebase + A.L[0].bin_base]) + (int)(item - __ldg(&l0_cum[lo]));
    const SHit a = load_shit(rec, pos);
    // layer-1 z range: z_b = z_a rho - z0 (rho - 1), rho = s1 / s0 in [rho_lo, rho_hi], |z0| <= z_max
    const float zc0 = fmaf(a.z, A.rho_lo, -A.z_max * (A.rho_lo - 1.f));
    const float zc1 = fmaf(a.z, A.rho_lo, A.z_max * (A.rho_lo - 1.f));
    const float zc2 = fmaf(a.z, A.rho_hi, -A.z_max * (A.rho_hi - 1.f));
    const float zc3 = fmaf(a.z, A.rho_hi, A.z_max * (A.rho_hi - 1.f));
    const Window w1 = make_window(A.L[1], atan2f(a.s, a.c), A.dphi1,
                                  fminf(fminf(zc0, zc1), fminf(zc2, zc3)) - kWinZPad,
                                  fmaxf(fmaxf(zc0, zc1), fmaxf(zc2, zc3)) + kWinZPad);
    int n = 0;   // triplets of this layer-0 hit so far (uniform)
    const int64_t base = WRITE ? (int64_t)__ldg(&toff[item]) : 0;
    const float phia = atan2f(a.s, a.c);
    int queued = 0;   // passing pairs waiting in the warp's queue (uniform)
    // the first `cnt` queued pairs, one per lane, search their layer-2 windows
    auto drain = [&](int cnt) {
      const bool have = lane < cnt;
      const int pb = have ? queue[lane].x : -1;
      const PairCut pc{have, have ? __int_as_float(queue[lane].y) : 0.f, have ? __int_as_float(queue[lane].z) : 0.f,
                       have ? __int_as_float(queue[lane].w) : 0.f};
      __syncwarp();
      for (int j = lane; j + 32 < queued; j += 32) queue[j] = queue[j + 32];   // keep the rest in order
      __syncwarp();
      int mine = 0;
      PairPred q{false, 0.f, 0.f, 0.f, 0.f};
      if (have) {
        q = pair_predict(A, a, phia, pc);
        for_layer2(A, ebase, q, bin_off, rec, st_l2, [&](const SHit&, int) { ++mine; });
      }
      int ex = mine;   // prefix of the lanes' triplet counts
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xFFFFFFFFu, ex, o);
        if (lane >= o) ex += v;
      }
      const int group = __shfl_sync(0xFFFFFFFFu, ex, 31);
      ex -= mine;
      if (WRITE && mine > 0) {
        int64_t i = base + n + ex;
        int unused = 0;
        for_layer2(A, ebase, q, bin_off, rec, unused,
                   [&](const SHit&, int pcpos) { trip[i++] = make_int4(pos, pb, pcpos, ebase); });
      }
      if (keep && !full && cursor + n + group > seg_cap) full = true;
      if (keep && !full && mine > 0) {
        int64_t i = seg_base + cursor + n + ex;
        int unused = 0;
        for_layer2(A, ebase, q, bin_off, rec, unused,
                   [&](const SHit&, int pcpos) { scratch[i++] = make_int4(pos, pb, pcpos, ebase); });
      }
      n += group;
      queued -= cnt;
    };
    for (int k0 = 0; k0 < w1.nrow; k0 += 32) {   // up to 32 rows at a time, one per lane
      const int k = k0 + lane;
      const int2 r = k < w1.nrow ? window_row(A.L[1], ebase, w1, k, bin_off) : make_int2(0, 0);
      const int len = r.y - r.x;
      int incl = len;   // inclusive prefix of the row lengths
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
      }
      const int tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
      const int nr = min(w1.nrow - k0, 32);
      for (int t0 = 0; t0 < tot; t0 += 32) {
        const int t = t0 + lane;
        int row = 0;   // row of entry t: the rows whose inclusive prefix is <= t come before it
        for (int l = 0; l < nr; ++l) row += __shfl_sync(0xFFFFFFFFu, incl, l) <= t;
        row = min(row, 31);
        const int rx = __shfl_sync(0xFFFFFFFFu, r.x, row);
        const int pre = __shfl_sync(0xFFFFFFFFu, incl - len, row);
        const int pb = t < tot ? rx + (t - pre) : -1;
        const PairCut pc = pb >= 0 ? pair_cut(A, a, load_shit(rec, pb)) : PairCut{false, 0.f, 0.f, 0.f};
        const unsigned m = __ballot_sync(0xFFFFFFFFu, pc.ok);
        st_l1 += pb >= 0;
        st_pairs += pc.ok;
        if (pc.ok)   // append in order
          queue[queued + __popc(m & ((1u << lane) - 1u))] =
              make_int4(pb, __float_as_int(pc.w), __float_as_int(pc.g0), __float_as_int(pc.cot));
        __syncwarp();
        queued += __popc(m);
        if (queued >= 32) drain(32);
      }
    }
    while (queued > 0) drain(min(queued, 32));
    st_trip += lane == 0 ? n : 0;
    if (!WRITE && lane == 0) tcnt[item] = n;
    if (keep) {
      if (lane == 0) item_loc[item] = full ? -1 : seg_base + cursor;
      if (!full) cursor += n;
    }
  }
  if (keep && full && lane == 0) atomicOr(overflow, 1);
  if (!WRITE) warp_add_stats(stats, st_l1, st_pairs, st_l2, st_trip, 0);
}

// The count pass's scratch lists to their places in the triplet list: one
// warp per layer-0 hit.
__global__ void k_seed_compact(const int* __restrict__ l0_cum, int n_events, const int* __restrict__ tcnt,
                               const int* __restrict__ toff, const int64_t* __restrict__ item_loc,
                               const int4* __restrict__ scratch, int4* __restrict__ trip,
                               const int* __restrict__ overflow = nullptr, int64_t n_slots = 0,
                               int64_t trip_cap = -1, int* __restrict__ status = nullptr) {
  const int lane = threadIdx.x & 31;
  // launched without a host decision (fixed triplet capacity): nothing to do
  // if a segment overflowed (the write pass searches again), and nothing is
  // written if the list does not fit (capacity bit)
  if (trip_cap >= 0) {
    if (*(volatile const int*)overflow) return;
    if (__ldg(&toff[n_slots]) > trip_cap) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kStatCapacity);
      return;
    }
  }
  const int n_items = __ldg(&l0_cum[n_events]);
  const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); item < n_items;
       item += n_warps) {
    const int cnt = __ldg(&tcnt[item]);
    const int64_t src = __ldg(&item_loc[item]), dst = __ldg(&toff[item]);
    for (int j = lane; j < cnt; j += 32) trip[dst + j] = __ldg(&scratch[src + j]);
  }
}

// Stage 2: one thread per triplet, its layer-3 window.  Count pass: qcnt[j] =
// seeds; write pass: seeds at qoff[j] ...
template <bool WRITE>
__global__ void __launch_bounds__(kSeedThreads)
    k_seed_quads(const SeedArgs A, const float4* __restrict__ rec, const int* __restrict__ bin_off,
                 const int4* __restrict__ trip, int n_trip, int* __restrict__ qcnt, const int* __restrict__ qoff,
                 float* __restrict__ par, float* __restrict__ cov, int* __restrict__ hits, int* __restrict__ status,
                 unsigned long long* __restrict__ stats, const int* __restrict__ n_trip_dev = nullptr,
                 int64_t stride = 0) {
  int st_l3 = 0, st_seeds = 0;   // work counters (count pass; per thread)
  // with a fixed triplet capacity n_trip is that capacity and the list's
  // length is read here (a list that did not fit is not searched)
  if (n_trip_dev) {
    const int64_t nt = __ldg(n_trip_dev);
    if (nt > n_trip) return;
    n_trip = (int)nt;
  }
  const int64_t total = WRITE ? (int64_t)__ldg(&qoff[n_trip]) : 0;
  if (WRITE && total > A.max_seeds) {   // nothing is written; the caller sees the count
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kStatCapacity);
    return;
  }
  const int64_t cs = stride > 0 ? stride : total;   // column stride of par and cov
  const float R0 = A.R[0], R1 = A.R[1], R2 = A.R[2], R3 = A.R[3];
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_trip;
       j += (int64_t)gridDim.x * blockDim.x) {
    if (WRITE && __ldg(&qoff[j + 1]) == __ldg(&qoff[j])) continue;   // most triplets make no seed
    const int4 tr = __ldg(&trip[j]);
    const SHit a = load_shit(rec, tr.x), b = load_shit(rec, tr.y), c = load_shit(rec, tr.z);
    int n = 0;
    const int64_t base = WRITE ? (int64_t)__ldg(&qoff[j]) : 0;
    const float w2c = circle_origin(R0, a, R2, c);
    if (fabsf(0.5f * w2c * R3) < 1.0f) {   // else that circle never reaches layer 3
      const float s0c = arc_sf(w2c, R0);
      const float cot2 = (c.z - a.z) / (arc_sf(w2c, R2) - s0c);
      const float z02 = fmaf(-cot2, s0c, a.z);
      float cq, sq;
      circle_dir(w2c, R0, a, R3, &cq, &sq);
      const float zq = fmaf(cot2, arc_sf(w2c, R3), z02);
      const Window w3 = make_window(A.L[3], atan2f(sq, cq), A.dphi3, zq - A.z_tol - kWinZPad, zq + A.z_tol + kWinZPad);
      for_window(A.L[3], tr.w, w3, bin_off, rec, [&](const SHit& d, int) {
        ++st_l3;
        if (!(fmaf(d.c, cq, d.s * sq) > 0.f) || !(fabsf(R3 * fmaf(d.s, cq, -d.c * sq)) <= A.rphi_tol) ||
            !(fabsf(d.z - zq) <= A.z_tol))
          return;
        const float w3c = circle_origin(R1, b, R3, d);
        if (!(fabsf(0.5f * w3c * R3) < 1.0f)) return;
        if (WRITE) {
          const int64_t i = base + n;
          float phi = atan2f(b.s, b.c) - asinf(0.5f * w3c * R1);
          if (phi > kPi) phi -= kTwoPi;
          if (phi < -kPi) phi += kTwoPi;
          const float sa = arc_sf(w3c, R0);
          const float cot3 = (d.z - a.z) / (arc_sf(w3c, R3) - sa);
          const float kappa = -w3c / (kAlphaF * A.bz);
          const float p6[6] = {0.f, 0.f, fmaf(-cot3, sa, a.z), kappa, phi, atan2f(1.f, cot3)};
          // fixed diagonal covariance: beam spot, z0, 5 % in kappa (+ 0.01 /GeV), 5 mrad
          const float var[6] = {1e-4f, 1e-4f, 2.5e-3f, fmaf(2.5e-3f * kappa, kappa, 1e-4f), 2.5e-5f, 2.5e-5f};
#pragma unroll
          for (int k = 0; k < 6; ++k) par[k * cs + i] = p6[k];
#pragma unroll
          for (int k = 0; k < 21; ++k) cov[k * cs + i] = 0.f;
#pragma unroll
          for (int k = 0; k < 6; ++k) cov[ci(k, k) * cs + i] = var[k];
          hits[4 * i] = a.orig;
          hits[4 * i + 1] = b.orig;
          hits[4 * i + 2] = c.orig;
          hits[4 * i + 3] = d.orig;
        }
        ++n;
      });
    }
    if (!WRITE) qcnt[j] = n;
    st_seeds += n;
  }
  if (!WRITE) warp_add_stats(stats, st_l3, st_seeds, 0, 0, 4);
}

// Stage 0, the seeding grid (a counting sort of the seeding layers' hits):
// cell of every binned hit on a seeding layer, from its building record.
__global__ void k_grid_keys(const SeedArgs A, const float4* __restrict__ rec_orig, const int* __restrict__ keys,
                            int64_t n_hits, int main_bins_per_event, int* __restrict__ gkey,
                            int* __restrict__ grank, int* __restrict__ gcnt) {
  const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= n_hits) return;
  const int key = keys[h];
  int k = -1;
  if (key >= 0) {   // binned (not masked)
    const int lb = __float_as_int(rec_orig[2 * h + 1].w);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (lb >= A.mb0[j] && lb < A.mb1[j]) k = j;
  }
  if (k < 0) {
    gkey[h] = -1;
    return;
  }
  const float4 r = rec_orig[2 * h];
  const LayerDev& ly = A.L[k];
  const int ip = min(max((int)floorf((atan2f(r.y, r.x) + kPi) * ly.phi_scale), 0), ly.nphi - 1);
  const int iw = min(max((int)floorf((r.z - ly.lo) * ly.w_scale), 0), ly.nw - 1);
  const int g = (key / main_bins_per_event) * A.bins_per_event + ly.bin_base + ip * ly.nw + iw;
  gkey[h] = g;
  grank[h] = atomicAdd(&gcnt[g], 1);
}

__global__ void k_grid_scatter(const float4* __restrict__ rec_orig, int64_t n_hits, const int* __restrict__ gkey,
                               const int* __restrict__ grank, const int* __restrict__ goff,
                               float4* __restrict__ grec) {
  const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= n_hits) return;
  const int g = gkey[h];
  if (g < 0) return;
  const float4 r = rec_orig[2 * h];
  grec[goff[g] + grank[h]] = make_float4(r.x, r.y, r.z, __int_as_float((int)h));
}

// each cell in ascending hit id (cells hold a few hits), so the search order is fixed
__global__ void k_grid_order(const int* __restrict__ goff, int64_t n_cells, float4* __restrict__ grec) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const int b = goff[c], e = goff[c + 1];
  for (int i = b + 1; i < e; ++i) {
    const float4 v = grec[i];
    int j = i - 1;
    while (j >= b && __float_as_int(grec[j].w) > __float_as_int(v.w)) {
      grec[j + 1] = grec[j];
      --j;
    }
    grec[j + 1] = v;
  }
}

// layer-0 hits of each event: n0[e] = positions of its layer-0 cells
__global__ void k_seed_l0_counts(const int* __restrict__ bin_off, int64_t bins_per_event, int base0, int nb0,
                                 int n_events, int* __restrict__ n0) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_events) return;
  const int64_t b = (int64_t)e * bins_per_event + base0;
  n0[e] = bin_off[b + nb0] - bin_off[b];
}

// ev_seed_off[e] = qoff[poff[l0_cum[e]]], e = 0..E (all seeds of event e
// come from its layer-0 hits, whose pairs come first in the pair list)
__global__ void k_seed_event_off(const int* __restrict__ l0_cum, int n_events, const int* __restrict__ poff,
                                 const int* __restrict__ qoff, int64_t q_len, int64_t* __restrict__ ev_seed_off) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e > n_events) return;
  // a triplet list longer than a fixed capacity was not searched (capacity bit
  // set): its offsets are clamped to the scanned range
  const int64_t j = poff[l0_cum[e]];
  ev_seed_off[e] = qoff[j < q_len ? j : q_len];
}

}  // namespace

}  // namespace mkf

extern "C" mkf_status mkf_seed_tracks(mkf_ctx* ctx, float pt_min, float z_max, float rphi_tol, float z_tol,
                                      int64_t max_seeds, float* seed_par, float* seed_cov, int* seed_hits,
                                      int64_t* ev_seed_off, void* stream) {
  using namespace mkf;
  if (!ctx) return MKF_ERR_ARG;
  if (!ctx->have_geom) return ctx->fail(MKF_ERR_STATE, "no geometry");
  if (!ctx->binned) return ctx->fail(MKF_ERR_STATE, "hits not binned");
  const GeomDev& g = ctx->geom;
  if (g.n_barrel < 4) return ctx->fail(MKF_ERR_ARG, "seeding needs four barrel layers");
  if (!(pt_min > 0.f) || !(z_max > 0.f) || !(rphi_tol > 0.f) || !(z_tol > 0.f) || max_seeds < 0)
    return ctx->fail(MKF_ERR_ARG, "bad seeding cuts");
  if (!ev_seed_off || (max_seeds > 0 && (!seed_par || !seed_cov || !seed_hits)))
    return ctx->fail(MKF_ERR_ARG, "null array");
  SeedArgs A{};
  for (int k = 0; k < 4; ++k) {
    const LayerDev& m = g.L[g.barrel_order[k]];
    A.mb0[k] = m.bin_base;
    A.mb1[k] = m.bin_base + m.nphi * m.nw;
    LayerDev q = m;
    q.nphi = kGridPhi;
    q.nw = kGridZ;
    q.bin_base = k * kGridCells;
    q.phi_scale = (float)kGridPhi / kTwoPi;
    q.w_scale = (float)kGridZ / (m.hi - m.lo);
    A.L[k] = q;
    A.R[k] = g.barrel_r[k];
  }
  const double alpha = 0.00299792458, wmax = alpha * (double)g.bz / (double)pt_min;
  const double R0 = A.R[0], R1 = A.R[1], R2 = A.R[2], R3 = A.R[3];
  if (!(0.5 * wmax * R3 <= 0.9)) return ctx->fail(MKF_ERR_ARG, "pt_min too low for the seeding layers");
  if (!(rphi_tol < 0.5 * R2)) return ctx->fail(MKF_ERR_ARG, "rphi_tol too large");
  A.omega_max = (float)wmax;
  A.z_max = z_max;
  A.rphi_tol = rphi_tol;
  A.z_tol = z_tol;
  A.dphi1 = (float)(std::asin(0.5 * wmax * R1) - std::asin(0.5 * wmax * R0)) + kWinPhiPad;
  A.rho_lo = (float)(R1 / R0) * (1.f - 1e-6f);
  A.rho_hi = (float)(std::asin(0.5 * wmax * R1) / std::asin(0.5 * wmax * R0)) * (1.f + 1e-6f);
  A.dphi2 = (float)std::asin(rphi_tol / R2) + kWinPhiPad;
  A.dphi3 = (float)std::asin(rphi_tol / R3) + kWinPhiPad;
  A.bz = g.bz;
  A.n_events = ctx->n_events;
  A.bins_per_event = 4 * kGridCells;
  if ((int64_t)ctx->n_events * A.bins_per_event >= (int64_t)INT32_MAX)
    return ctx->fail(MKF_ERR_ARG, "too many events for the seeding grid");
  A.max_seeds = max_seeds;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t H = ctx->n_hits;
  const int E = ctx->n_events;
  cudaError_t e;
  // seed_cnt: pcnt [H] | n0 [E + 1]; seed_off: poff [H + 1] | l0_cum [E + 1];
  // seed_pairs, seed_qcnt, seed_qoff: pair list, its seed counts and their scan; seed_part: scan scratch
  if ((e = ctx->seed_cnt.ensure((size_t)(H + E + 2) * 4)) != cudaSuccess) return ctx->fail(MKF_ERR_OOM, "seed counts");
  if ((e = ctx->seed_off.ensure((size_t)(H + 2 * E + 4) * 4)) != cudaSuccess)
    return ctx->fail(MKF_ERR_OOM, "seed offsets");
  int* status = ctx->status.as<int>();
  const int T = 128;
  // stage 0: the seeding grid
  const int64_t n_cells = (int64_t)E * A.bins_per_event;
  if ((e = ctx->grid_key.ensure((size_t)(H + 1) * 4)) != cudaSuccess ||
      (e = ctx->grid_rank.ensure((size_t)(H + 1) * 4)) != cudaSuccess ||
      (e = ctx->grid_cnt.ensure((size_t)(n_cells + 1) * 4)) != cudaSuccess ||
      (e = ctx->grid_off.ensure((size_t)(n_cells + 1) * 4)) != cudaSuccess ||
      (e = ctx->grid_rec.ensure((size_t)(H + 1) * 16)) != cudaSuccess)
    return ctx->fail(MKF_ERR_OOM, "seeding grid");
  if (n_cells > 0 && (e = cudaMemsetAsync(ctx->grid_cnt.p, 0, (size_t)n_cells * 4, st)) != cudaSuccess)
    return ctx->cuda_fail(e, "memset");
  const float4* rec_orig = ctx->rec_orig.as<float4>();
  if (H > 0)
    k_grid_keys<<<(unsigned)((H + 255) / 256), 256, 0, st>>>(A, rec_orig, ctx->keys.as<int>(), H, g.bins_per_event,
                                                           ctx->grid_key.as<int>(), ctx->grid_rank.as<int>(),
                                                           ctx->grid_cnt.as<int>());
  if ((e = launch_excl_scan(ctx->grid_cnt.as<int>(), n_cells, ctx->grid_off.as<int>(), ctx->seed_part, st)) !=
      cudaSuccess)
    return ctx->cuda_fail(e, "grid scan");
  if (H > 0)
    k_grid_scatter<<<(unsigned)((H + 255) / 256), 256, 0, st>>>(rec_orig, H, ctx->grid_key.as<int>(),
                                                              ctx->grid_rank.as<int>(), ctx->grid_off.as<int>(),
                                                              ctx->grid_rec.as<float4>());
  if (n_cells > 0)
    k_grid_order<<<(unsigned)((n_cells + 255) / 256), 256, 0, st>>>(ctx->grid_off.as<int>(), n_cells,
                                                                  ctx->grid_rec.as<float4>());
  if ((e = cudaGetLastError()) != cudaSuccess) return ctx->cuda_fail(e, "seeding grid");
  int* pcnt = ctx->seed_cnt.as<int>();
  int* n0 = pcnt + H;
  int* poff = ctx->seed_off.as<int>();
  int* l0_cum = poff + H + 1;
  if (E > 0)
    k_seed_l0_counts<<<(unsigned)((E + T - 1) / T), T, 0, st>>>(ctx->grid_off.as<int>(), A.bins_per_event,
                                                                 A.L[0].bin_base, kGridCells, E, n0);
  if ((e = launch_excl_scan(n0, E, l0_cum, ctx->seed_part, st)) != cudaSuccess) return ctx->cuda_fail(e, "scan");
  if (H > 0 && (e = cudaMemsetAsync(pcnt, 0, (size_t)H * 4, st)) != cudaSuccess) return ctx->cuda_fail(e, "memset");
  const unsigned blocks = (unsigned)(ctx->n_sm * 8);   // persistent: 32 warps per SM
  const float4* rec = ctx->grid_rec.as<float4>();
  const int* bin_off = ctx->grid_off.as<int>();
  // stage 1: triplet counts, their scan, and the triplet total read back to size what follows
  if ((e = ctx->seed_stats.ensure(8 * sizeof(unsigned long long))) != cudaSuccess) return ctx->fail(MKF_ERR_OOM, "stats");
  if ((e = cudaMemsetAsync(ctx->seed_stats.p, 0, 8 * sizeof(unsigned long long), st)) != cudaSuccess)
    return ctx->cuda_fail(e, "memset");
  unsigned long long* stats = ctx->seed_stats.as<unsigned long long>();
  // the count pass also keeps each layer-0 hit's triplets in a per-warp
  // scratch segment, sized from the last call's triplet total (or the hits)
  const int64_t n_warps = (int64_t)blocks * (kSeedThreads / 32);
  const int64_t hint = ctx->seed_trip_hint > 0 ? ctx->seed_trip_hint : H;
  const int64_t seg_cap = std::max<int64_t>(2048, 2 * hint / n_warps + 256);
  if ((e = ctx->seed_scratch.ensure((size_t)(n_warps * seg_cap) * sizeof(int4))) != cudaSuccess ||
      (e = ctx->seed_loc.ensure((size_t)(H + 1) * sizeof(int64_t) + 16)) != cudaSuccess)
    return ctx->fail(MKF_ERR_OOM, "seed scratch");
  int* overflow = reinterpret_cast<int*>(ctx->seed_loc.as<char>() + (size_t)(H + 1) * sizeof(int64_t));
  if ((e = cudaMemsetAsync(overflow, 0, sizeof(int), st)) != cudaSuccess) return ctx->cuda_fail(e, "memset");
  if (H > 0)
    k_seed_triplets<false><<<blocks, kSeedThreads, 0, st>>>(A, rec, bin_off, l0_cum, H, pcnt, nullptr, nullptr, stats,
                                                             ctx->seed_scratch.as<int4>(), seg_cap,
                                                             ctx->seed_loc.as<int64_t>(), overflow);
  if ((e = launch_excl_scan(pcnt, H, poff, ctx->seed_part, st)) != cudaSuccess) return ctx->cuda_fail(e, "triplet scan");
  const int64_t cap = ctx->seed_trip_cap;   // 0: size the triplet list from its count (one read-back)
  int n_trip = 0, over = 0;
  if (cap == 0) {
    if ((e = cudaMemcpyAsync(&n_trip, poff + H, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&over, overflow, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return ctx->cuda_fail(e, "triplet count");
    ctx->seed_trip_hint = n_trip;
  }
  const int64_t P = cap == 0 ? n_trip : cap;
  if ((e = ctx->seed_pairs.ensure((size_t)(P + 1) * sizeof(int4))) != cudaSuccess ||
      (e = ctx->seed_qcnt.ensure((size_t)(P + 1) * 4)) != cudaSuccess ||
      (e = ctx->seed_qoff.ensure((size_t)(P + 1) * 4)) != cudaSuccess)
    return ctx->fail(MKF_ERR_OOM, "seed triplets");
  int4* trip = ctx->seed_pairs.as<int4>();
  int* qcnt = ctx->seed_qcnt.as<int>();
  int* qoff = ctx->seed_qoff.as<int>();
  if (cap == 0) {
    if (H > 0 && !over)   // scratch lists in place: move them
      k_seed_compact<<<blocks, kSeedThreads, 0, st>>>(l0_cum, E, pcnt, poff, ctx->seed_loc.as<int64_t>(),
                                                      ctx->seed_scratch.as<int4>(), trip);
    else if (H > 0)        // a segment overflowed: search again and write
      k_seed_triplets<true><<<blocks, kSeedThreads, 0, st>>>(A, rec, bin_off, l0_cum, H, nullptr, poff, trip, stats,
                                                              nullptr, 0, nullptr, nullptr);
  } else if (H > 0) {
    // both launched; each decides on the device (overflow flag, triplet count)
    k_seed_compact<<<blocks, kSeedThreads, 0, st>>>(l0_cum, E, pcnt, poff, ctx->seed_loc.as<int64_t>(),
                                                    ctx->seed_scratch.as<int4>(), trip, overflow, H, cap, status);
    k_seed_triplets<true><<<blocks, kSeedThreads, 0, st>>>(A, rec, bin_off, l0_cum, H, nullptr, poff, trip, stats,
                                                            nullptr, 0, nullptr, overflow, cap);
  }
  // stage 2 over the triplet list
  const int* n_trip_dev = cap == 0 ? nullptr : poff + H;
  const int64_t stride = cap == 0 ? 0 : max_seeds;
  if (cap > 0 && (e = cudaMemsetAsync(qcnt, 0, (size_t)(P + 1) * 4, st)) != cudaSuccess)
    return ctx->cuda_fail(e, "memset");
  if (P > 0)
    k_seed_quads<false><<<blocks, kSeedThreads, 0, st>>>(A, rec, bin_off, trip, (int)P, qcnt, nullptr, nullptr,
                                                          nullptr, nullptr, status, stats, n_trip_dev);
  if ((e = launch_excl_scan(qcnt, P, qoff, ctx->seed_part, st)) != cudaSuccess) return ctx->cuda_fail(e, "seed scan");
  if (P > 0)
    k_seed_quads<true><<<blocks, kSeedThreads, 0, st>>>(A, rec, bin_off, trip, (int)P, nullptr, qoff, seed_par,
                                                         seed_cov, seed_hits, status, stats, n_trip_dev, stride);
  k_seed_event_off<<<(unsigned)((E + 1 + T - 1) / T), T, 0, st>>>(l0_cum, E, poff, qoff, P, ev_seed_off);
  if ((e = cudaGetLastError()) != cudaSuccess) return ctx->cuda_fail(e, "seeding");
  return MKF_OK;
}

extern "C" mkf_status mkf_set_seed_config(mkf_ctx* ctx, int64_t max_triplets) {
  if (!ctx) return MKF_ERR_ARG;
  if (max_triplets < 0 || max_triplets >= (int64_t)INT32_MAX)
    return ctx->fail(MKF_ERR_ARG, "max_triplets must be in 0..2^31-2");
  ctx->seed_trip_cap = max_triplets;
  return MKF_OK;
}

extern "C" mkf_status mkf_get_seed_stats(mkf_ctx* ctx, int64_t* out, int n, void* stream) {
  if (!ctx || !out || n < 0 || n > 6) return ctx ? ctx->fail(MKF_ERR_ARG, "seed stats: n in 0..6") : MKF_ERR_ARG;
  unsigned long long v[8] = {};
  if (ctx->seed_stats.p) {
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(v, ctx->seed_stats.p, sizeof(v), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return ctx->cuda_fail(e, "seed stats");
  }
  for (int i = 0; i < n; ++i) out[i] = (int64_t)v[i];
  return MKF_OK;
}
