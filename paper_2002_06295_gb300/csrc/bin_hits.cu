// bin_hits.cu -- position-based hit lookup structure (Sec. 2: the geometry has
// no modules, the search relies on the 3-D hit positions).
//
// key = event * B + layer_base + phi_bin * n_w + w_bin   (w = z on a barrel, r on a disk)
// A counting sort: per-key counts (atomics) -> exclusive scan -> scatter.  The
// order inside a bin is made ascending in the caller's hit index only when the
// binning is read back (the search does not depend on it).  Each sorted hit is stored as a 32-byte
// measurement record (cos phi_h, sin phi_h, w, V) ready for the chi2 kernel.
#include "mkf_device.cuh"
#include "mkf_internal.h"

namespace mkf {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int event_of(const int64_t* off, int n_events, int64_t i) {
  int lo = 0, hi = n_events;   // off[lo] <= i < off[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= i)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Bin key and rank of every hit, and the largest hit variances per (event,
// layer).  The variance maxima are first reduced in shared memory over the
// block's hits (a block's consecutive hits lie in one or two events), so the
// global atomics per (event, layer) are one per block instead of one per hit.
__global__ void k_bin_keys(const GeomDev* __restrict__ gdev, const float* __restrict__ xyz,
                           const float* __restrict__ lcov, const int* __restrict__ layer, int64_t n_hits,
                           const int64_t* __restrict__ ev_off, int n_events, int* __restrict__ keys,
                           int* __restrict__ ranks, int* __restrict__ counts, float* __restrict__ vmax,
                           const uint8_t* __restrict__ mask, int* __restrict__ status) {
  __shared__ int sv[2][MKF_MAX_LAYERS][2];   // float bits; variances are >= 0, so int order = float order
  __shared__ int e_first;
  const int L = gdev->n_layers;
  for (int i = threadIdx.x; i < 2 * MKF_MAX_LAYERS * 2; i += blockDim.x) (&sv[0][0][0])[i] = 0;
  const int64_t h0 = (int64_t)blockIdx.x * blockDim.x;
  if (threadIdx.x == 0) e_first = event_of(ev_off, n_events, h0 < n_hits ? h0 : n_hits - 1);
  __syncthreads();
  const int64_t h = h0 + threadIdx.x;
  if (h < n_hits) {
    const int l = layer[h];
    if (l < 0 || l >= L) {
      keys[h] = -1;
      atomicOr(status, kStatBadInput);
    } else if (mask && mask[h]) {
      keys[h] = -1;   // masked: left out of every bin, so no search can return it
    } else {
      const LayerDev ly = gdev->L[l];
      const float x = xyz[h], y = xyz[n_hits + h], z = xyz[2 * n_hits + h];
      const float phi = atan2f(y, x);
      const float w = ly.kind == 0 ? z : sqrtf(fmaf(x, x, y * y));
      int ip = (int)floorf((phi + kPi) * ly.phi_scale);
      ip = min(max(ip, 0), ly.nphi - 1);
      int iw = (int)floorf((w - ly.lo) * ly.w_scale);
      iw = min(max(iw, 0), ly.nw - 1);
      int e = e_first;
      if (e + 1 < n_events && h >= ev_off[e + 1]) {
        ++e;
        if (e + 1 < n_events && h >= ev_off[e + 1]) e = event_of(ev_off, n_events, h);
      }
      const int key = e * gdev->bins_per_event + ly.bin_base + ip * ly.nw + iw;
      keys[h] = key;
      ranks[h] = atomicAdd(&counts[key], 1);
      // largest hit variances of the (event, layer): they bound the search window
      const int va = __float_as_int(fmaxf(lcov[h], 0.0f)), vb = __float_as_int(fmaxf(lcov[n_hits + h], 0.0f));
      const int de = e - e_first;
      if (de < 2) {
        atomicMax(&sv[de][l][0], va);
        atomicMax(&sv[de][l][1], vb);
      } else {
        atomicMax(reinterpret_cast<int*>(&vmax[2 * (e * L + l)]), va);
        atomicMax(reinterpret_cast<int*>(&vmax[2 * (e * L + l) + 1]), vb);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * L * 2; i += blockDim.x) {
    const int de = i / (2 * L), l = (i / 2) % L, c = i & 1;
    const int v = sv[de][l][c];
    if (v > 0 && e_first + de < n_events)
      atomicMax(reinterpret_cast<int*>(&vmax[2 * ((e_first + de) * L + l) + c]), v);
  }
}

// inclusive warp scan
__device__ __forceinline__ int warp_incl(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// exclusive block scan of one value per thread; returns the block total in *total
__device__ __forceinline__ int block_excl(int v, int* sh, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int inc = warp_incl(v);
  if (lane == 31) sh[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int s = lane < nw ? sh[lane] : 0;
    int si = warp_incl(s);
    if (lane < nw) sh[lane] = si - s;
    if (lane == nw - 1) sh[32] = si;
  }
  __syncthreads();
  int r = inc - v + sh[wid];
  *total = sh[32];
  __syncthreads();
  return r;
}

__global__ void k_scan_reduce(const int* __restrict__ in, int64_t n, int* __restrict__ part) {
  __shared__ int sh[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
  int total;
  block_excl(s, sh, &total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void k_scan_partials(int* __restrict__ part, int n_parts) {
  __shared__ int sh[33];
  int carry = 0;
  for (int base = 0; base < n_parts; base += blockDim.x) {
    int i = base + threadIdx.x;
    int v = i < n_parts ? part[i] : 0;
    int total;
    int ex = block_excl(v, sh, &total);
    if (i < n_parts) part[i] = carry + ex;
    carry += total;
  }
}

// out[i] = exclusive prefix of in; out[n] = total.
__global__ void k_scan_apply(const int* __restrict__ in, int64_t n, const int* __restrict__ part,
                             int* __restrict__ out) {
  __shared__ int sh[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int v[kScanItems];
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    v[k] = i < n ? in[i] : 0;
    s += v[k];
  }
  int total;
  int ex = block_excl(s, sh, &total) + part[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    if (i < n) out[i] = ex;
    if (i == n - 1) out[n] = ex + v[k];
    ex += v[k];
  }
}

__global__ void k_bin_scatter(const GeomDev* __restrict__ gdev, const float* __restrict__ xyz,
                              const float* __restrict__ lcov, const int* __restrict__ layer, int64_t n_hits,
                              const int* __restrict__ keys, const int* __restrict__ ranks,
                              const int* __restrict__ bin_off, float4* __restrict__ rec,
                              float4* __restrict__ rec_orig, int* __restrict__ perm) {
  const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= n_hits) return;
  const int key = keys[h];
  if (key < 0) return;
  const int pos = bin_off[key] + ranks[h];
  const LayerDev ly = gdev->L[layer[h]];
  const float x = xyz[h], y = xyz[n_hits + h], z = xyz[2 * n_hits + h];
  const float r = sqrtf(fmaf(x, x, y * y));
  const float ir = 1.0f / r;
  const float w = ly.kind == 0 ? z : r;
  const int local_bin = key % gdev->bins_per_event;
  const float4 r0 = make_float4(x * ir, y * ir, w, lcov[h]);
  const float4 r1 = make_float4(lcov[2 * n_hits + h], lcov[n_hits + h], __int_as_float((int)h),
                                __int_as_float(local_bin));
  rec[2 * pos] = r0;
  rec[2 * pos + 1] = r1;
  rec_orig[2 * h] = r0;
  rec_orig[2 * h + 1] = r1;
  perm[pos] = (int)h;
}

// Make the order inside each bin ascending in the caller's hit index.
__global__ void k_bin_order(const int* __restrict__ bin_off, int64_t n_bins, float4* __restrict__ rec,
                            int* __restrict__ perm) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_bins) return;
  const int lo = bin_off[b], hi = bin_off[b + 1];
  if (hi - lo < 2) return;
  for (int i = lo + 1; i < hi; ++i) {
    const int key = perm[i];
    const float4 r0 = rec[2 * i], r1 = rec[2 * i + 1];
    int j = i - 1;
    while (j >= lo && perm[j] > key) {
      perm[j + 1] = perm[j];
      rec[2 * (j + 1)] = rec[2 * j];
      rec[2 * (j + 1) + 1] = rec[2 * j + 1];
      --j;
    }
    perm[j + 1] = key;
    rec[2 * (j + 1)] = r0;
    rec[2 * (j + 1) + 1] = r1;
  }
}

// mask[h] = 1 for every hit of a track whose flag is MKF_TRK_KEPT
__global__ void k_used_hits(const int* __restrict__ hits, const int* __restrict__ flags, int64_t n_tracks, int L,
                            int64_t n_hits, uint8_t* __restrict__ mask, int* __restrict__ status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_tracks * L) return;
  const int64_t t = i / L;
  if (flags[t] != MKF_TRK_KEPT) return;
  const int h = hits[i];
  if (h < 0) return;
  if (h >= n_hits) {
    atomicOr(status, kStatBadInput);
    return;
  }
  mask[h] = 1;
}

}  // namespace

cudaError_t launch_used_hits(mkf_ctx* ctx, const int* hits, const int* flags, int64_t n_tracks, int L,
                             int64_t n_hits, uint8_t* mask, cudaStream_t st) {
  const int64_t n = n_tracks * L;
  if (n == 0) return cudaSuccess;
  const int T = 256;
  k_used_hits<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(hits, flags, n_tracks, L, n_hits, mask,
                                                         ctx->status.as<int>());
  return cudaGetLastError();
}

cudaError_t launch_excl_scan(const int* in, int64_t n, int* out, DevBuf& part, cudaStream_t st) {
  cudaError_t e;
  if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(int), st);
  const int64_t n_parts = (n + kScanTile - 1) / kScanTile;
  if ((e = part.ensure((size_t)n_parts * 4)) != cudaSuccess) return e;
  k_scan_reduce<<<(unsigned)n_parts, kScanThreads, 0, st>>>(in, n, part.as<int>());
  k_scan_partials<<<1, 1024, 0, st>>>(part.as<int>(), (int)n_parts);
  k_scan_apply<<<(unsigned)n_parts, kScanThreads, 0, st>>>(in, n, part.as<int>(), out);
  return cudaGetLastError();
}

cudaError_t launch_bin_hits(mkf_ctx* ctx, const float* xyz, const float* lcov, const int* layer, int64_t n_hits,
                            const int64_t* ev_hit_off, int n_events, const uint8_t* mask, cudaStream_t st) {
  const GeomDev& g = ctx->geom;
  const int64_t n_bins = (int64_t)n_events * g.bins_per_event;
  const int64_t n_parts = (n_bins + kScanTile - 1) / kScanTile;
  const int64_t H = n_hits;
  cudaError_t e;
  if ((e = ctx->rec.ensure((size_t)(H > 0 ? H : 1) * 32)) != cudaSuccess) return e;
  if ((e = ctx->rec_orig.ensure((size_t)(H > 0 ? H : 1) * 32)) != cudaSuccess) return e;
  if ((e = ctx->perm.ensure((size_t)(H > 0 ? H : 1) * 4)) != cudaSuccess) return e;
  if ((e = ctx->keys.ensure((size_t)(H > 0 ? H : 1) * 4)) != cudaSuccess) return e;
  if ((e = ctx->ranks.ensure((size_t)(H > 0 ? H : 1) * 4)) != cudaSuccess) return e;
  if ((e = ctx->bin_cnt.ensure((size_t)n_bins * 4)) != cudaSuccess) return e;
  if ((e = ctx->bin_off.ensure((size_t)(n_bins + 1) * 4)) != cudaSuccess) return e;
  if ((e = ctx->vmax.ensure((size_t)n_events * g.n_layers * 2 * 4)) != cudaSuccess) return e;
  if ((e = ctx->ev_hit_off.ensure((size_t)(n_events + 1) * 8)) != cudaSuccess) return e;
  if ((e = ctx->scan_part.ensure((size_t)(n_parts > 0 ? n_parts : 1) * 4)) != cudaSuccess) return e;
  ctx->n_hits = n_hits;
  ctx->n_events = n_events;
  ctx->n_bins_total = n_bins;
  const GeomDev* gd = ctx->geom_dev.as<GeomDev>();
  int* status = ctx->status.as<int>();
  if ((e = cudaMemcpyAsync(ctx->ev_hit_off.p, ev_hit_off, (n_events + 1) * 8, cudaMemcpyDeviceToDevice, st)))
    return e;
  if ((e = cudaMemsetAsync(ctx->bin_cnt.p, 0, (size_t)n_bins * 4, st))) return e;
  if ((e = cudaMemsetAsync(ctx->vmax.p, 0, (size_t)n_events * g.n_layers * 2 * 4, st))) return e;
  const int T = 256;
  ctx->tick(kTBin, st);
  if (H > 0) {
    k_bin_keys<<<(unsigned)((H + T - 1) / T), T, 0, st>>>(gd, xyz, lcov, layer, H, ctx->ev_hit_off.as<int64_t>(),
                                                         n_events, ctx->keys.as<int>(), ctx->ranks.as<int>(),
                                                         ctx->bin_cnt.as<int>(), ctx->vmax.as<float>(), mask, status);
  }
  k_scan_reduce<<<(unsigned)n_parts, kScanThreads, 0, st>>>(ctx->bin_cnt.as<int>(), n_bins, ctx->scan_part.as<int>());
  k_scan_partials<<<1, 1024, 0, st>>>(ctx->scan_part.as<int>(), (int)n_parts);
  k_scan_apply<<<(unsigned)n_parts, kScanThreads, 0, st>>>(ctx->bin_cnt.as<int>(), n_bins, ctx->scan_part.as<int>(),
                                                          ctx->bin_off.as<int>());
  if (H > 0) {
    k_bin_scatter<<<(unsigned)((H + T - 1) / T), T, 0, st>>>(gd, xyz, lcov, layer, H, ctx->keys.as<int>(),
                                                            ctx->ranks.as<int>(), ctx->bin_off.as<int>(),
                                                            ctx->rec.as<float4>(), ctx->rec_orig.as<float4>(),
                                                            ctx->perm.as<int>());
  }
  ctx->bins_ordered = H == 0;
  ctx->tock(kTBin, st);
  return cudaGetLastError();
}

// The building kernel does not depend on the order of the hits inside a bin
// (candidate ranking breaks ties by the caller's hit index), so the binning
// leaves it as the count atomics made it; mkf_get_binning sorts each bin by
// the caller's hit index first, which makes the result a stable sort.
cudaError_t launch_bin_order(mkf_ctx* ctx, cudaStream_t st) {
  if (ctx->bins_ordered) return cudaSuccess;
  const int64_t n_bins = ctx->n_bins_total;
  const int T = 256;
  if (n_bins > 0)
    k_bin_order<<<(unsigned)((n_bins + T - 1) / T), T, 0, st>>>(ctx->bin_off.as<int>(), n_bins, ctx->rec.as<float4>(),
                                                               ctx->perm.as<int>());
  ctx->bins_ordered = true;
  return cudaGetLastError();
}

}  // namespace mkf
