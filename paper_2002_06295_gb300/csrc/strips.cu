// strips.cu -- silicon-strip clustering (Sec. 4, Towards an HLT implementation):
// the step before building that turns raw strip ADCs into clusters.
//  * a seed strip has ADC above 3 times its expected noise;
//  * a cluster adds to its seeds every strip above twice the noise that is
//    consecutive, or across a gap of at most max_bad_gap bad strips (bad
//    strips carry no charge and no noise);
//  * it is kept if the quadrature sum of its ADCs exceeds 5 times the
//    quadrature sum of its noises and its total charge reaches q_min.
// Noise comes in eighths of an ADC count, so each test is an exact integer
// comparison: candidate 4 a > nq, seed 8 a > 3 nq, kept 64 sum a^2 > 25 sum nq^2.
//
// The work is a stream over the ADC array (HBM-bound).  Each lane owns one row
// (event x module).  A warp takes items of 32 consecutive modules x E events
// and runs its own pipeline of S stages: per chunk of CH strips one lane issues
// three TMA box loads (ADC [E][32][CH] and noise [32][CH] into swizzled shared
// memory, bad-strip bits [CH/32][32 modules]) completed on an mbarrier, so the
// calibration of a chunk is staged once for E events.  The bad flags are first
// packed to one bit a strip by a small kernel.  Per 32 strips each lane forms
// its candidate mask with two strips per instruction (an unsigned 16x2 min and
// a subtract whose sign bits answer 4 a > nq), restores strip order with a
// perfect shuffle, and visits only the candidate strips: whether a candidate
// continues the open cluster (nothing but at most max_bad_gap bad strips since
// the last one) is answered by bit arithmetic on the break mask.  Kept clusters
// go to a small per-warp ring in shared memory flushed with one global atomic
// per batch.  Rows whose width or pointers break the TMA alignment rules take a
// plain one-strip-at-a-time kernel with the same results.
#include <type_traits>

#include <cuda.h>   // CUtensorMap and its enums (the encoder is fetched from the driver at run time)

#include "mkf_internal.h"

namespace mkf {

namespace {

constexpr int kTmaWarps = 4;               // warps per block of the TMA kernel
constexpr int kRingCap = 64;               // clusters a warp buffers before a flush
constexpr int kWaitLimit = 1 << 22;        // bounded mbarrier wait: try_wait polls ...
constexpr uint64_t kWaitNs = 100000000;    // ... and wall time (100 ms)
constexpr int kFallbackThreads = 256;

struct Cluster {
  int row, first, last, charge;
  float center;
};

__device__ __forceinline__ void put_cluster(const Cluster& c, unsigned long long slot, int* __restrict__ out_row,
                                            int* __restrict__ out_first, int* __restrict__ out_last,
                                            int* __restrict__ out_charge, float* __restrict__ out_center,
                                            int64_t max_out, int* __restrict__ status) {
  if ((int64_t)slot < max_out) {
    out_row[slot] = c.row;
    out_first[slot] = c.first;
    out_last[slot] = c.last;
    out_charge[slot] = c.charge;
    out_center[slot] = c.center;
  } else {
    atomicOr(status, kStatCapacity);
  }
}

// Cluster being grown along one row (plain kernel).  d = sum (64 a^2 -
// 25 nq^2), so the quadrature test is d > 0; qi = sum (i - first) a, the first
// moment about the first strip; pend = bad strips since the last candidate.
struct Run {
  int first, last, pend;
  bool open, seeded;
  long long q, d, qi;
};

__device__ __forceinline__ bool run_kept(const Run& s, int q_min) {
  return s.open && s.seeded && s.d > 0 && s.q >= q_min;
}

__device__ __forceinline__ Cluster run_cluster(const Run& s, int row) {
  return Cluster{row, s.first, s.last, (int)s.q, (float)s.first + (float)s.qi / (float)s.q};
}

// The same for the TMA kernel (rows of at most 65536 strips, so q < 2^32):
// sums of squares kept apart so that each strip costs 32 x 32 -> 64-bit
// multiply-adds only.
struct RunU {
  int first, last;
  bool open, seeded;
  uint32_t q;
  unsigned long long q2, n2, qi;
};

__device__ __forceinline__ bool runu_kept(const RunU& s, int q_min) {
  if (!s.open || !s.seeded || (long long)s.q < q_min) return false;
  return 64 * s.q2 > 25 * s.n2;
}

__device__ __forceinline__ Cluster runu_cluster(const RunU& s, int row) {
  const float qi = fmaf((float)(uint32_t)(s.qi >> 32), 4294967296.0f, (float)(uint32_t)s.qi);
  return Cluster{row, s.first, s.last, (int)s.q, (float)s.first + qi / (float)s.q};
}

// ---------------------------------------------------------------------------
// TMA path
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait (polls and wall time); false, with the timeout bit set, if the
// phase did not complete.  The answer is the same on every lane of the warp.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* status) {
  bool ok = mbar_try_wait(bar, parity);
  if (!ok) {
    const uint64_t t0 = global_ns();
    for (int i = 0; i < kWaitLimit && !ok; ++i) {
      ok = mbar_try_wait(bar, parity);
      if ((i & 255) == 255 && global_ns() - t0 > kWaitNs) break;
    }
  }
  ok = __all_sync(0xFFFFFFFFu, ok);
  if (!ok && (threadIdx.x & 31) == 0) atomicOr(status, kStatTimeout);
  return ok;
}

__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int x, int y, uint32_t bar,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, "
      "%3}], [%4], %5;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(bar), "l"(policy)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, int x, int y, int z, uint32_t bar,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, "
      "%3, %4}], [%5], %6;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(bar), "l"(policy)
      : "memory");
}

// Per 16-bit half: min(a, b), unsigned.
__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// Outer perfect shuffle: bit i of the low half goes to bit 2i, bit i of the
// high half to bit 2i + 1 (a byte swap, then three delta swaps).
__device__ __forceinline__ uint32_t perfect_shuffle(uint32_t x) {
  x = __byte_perm(x, 0, 0x3120);
  uint32_t t = ((x >> 4) ^ x) & 0x00F000F0u;
  x ^= t ^ (t << 4);
  t = ((x >> 2) ^ x) & 0x0C0C0C0Cu;
  x ^= t ^ (t << 2);
  t = ((x >> 1) ^ x) & 0x22222222u;
  x ^= t ^ (t << 1);
  return x;
}

// Byte offset inside a 1024-byte-aligned box written by TMA with the swizzle
// whose span is the row size RB (32, 64 or 128 bytes): the 16-byte chunk index
// is XORed with the address bits just above the 128-byte line.
template <int RB>
__device__ __forceinline__ int swz(int off) {
  return off ^ (((off >> 7) & (RB / 16 - 1)) << 4);
}

__device__ __forceinline__ uint4 lds128(const unsigned char* base, int off) {
  return *reinterpret_cast<const uint4*>(base + off);
}

template <int CH, int E, int S>
struct TmaShape {
  static constexpr int RB = CH * 2;                     // bytes per ADC / noise row in shared memory
  static constexpr int A_BYTES = E * 32 * RB;           // ADC box [E][32][CH], swizzled
  static constexpr int N_BYTES = 32 * RB;               // noise box [32][CH], swizzled
  static constexpr int SW_STAGE = A_BYTES + N_BYTES;
  static constexpr int BAD_BYTES = (CH / 32) * 128;     // bad-bit box [CH/32][32 modules] of 32-bit words
  static constexpr int STAGE_TX = SW_STAGE + BAD_BYTES; // bytes one stage's loads deliver
  static constexpr int RING_BYTES = 5 * kRingCap * 4;
  static constexpr int WARP_TAIL = (S * BAD_BYTES + S * 8 + RING_BYTES + 16 + 127) / 128 * 128;
  static constexpr int SMEM = 1024 + kTmaWarps * (S * SW_STAGE + WARP_TAIL);
  static_assert(A_BYTES % 1024 == 0 && N_BYTES % 1024 == 0, "swizzled boxes keep 1024-byte alignment");
};

template <int CH, int E, int S>
__global__ void __launch_bounds__(kTmaWarps * 32)
    k_strip_cluster_tma(const __grid_constant__ CUtensorMap tm_adc, const __grid_constant__ CUtensorMap tm_noise,
                        const __grid_constant__ CUtensorMap tm_bad, int n_events, int n_modules, int n_strips,
                        int max_bad_gap, int q_min, int* __restrict__ out_row, int* __restrict__ out_first,
                        int* __restrict__ out_last, int* __restrict__ out_charge, float* __restrict__ out_center,
                        int64_t max_out, unsigned long long* __restrict__ count, int* __restrict__ status) {
  using T = TmaShape<CH, E, S>;
  using Mask = typename std::conditional<CH == 64, unsigned long long, uint32_t>::type;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024 - (smem_addr(smem_raw) & 1023)) & 1023);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned char* stages = smem + w * S * T::SW_STAGE;
  unsigned char* tail = smem + kTmaWarps * S * T::SW_STAGE + w * T::WARP_TAIL;
  unsigned char* bad_boxes = tail;                                       // [S][BAD_BYTES]
  uint64_t* bars = reinterpret_cast<uint64_t*>(tail + S * T::BAD_BYTES); // [S]
  int* ring = reinterpret_cast<int*>(tail + S * T::BAD_BYTES + S * 8);   // [5][kRingCap]: row, first, last, charge, center
  int* fill = ring + 5 * kRingCap;

  const int n_g = (n_modules + 31) / 32, nc = (n_strips + CH - 1) / CH;
  const int64_t n_items = (int64_t)n_g * ((n_events + E - 1) / E);
  const int64_t GW = (int64_t)gridDim.x * kTmaWarps;

  if (lane == 0) {
    for (int s = 0; s < S; ++s) mbar_init(smem_addr(&bars[s]));
    *fill = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncwarp();
  const uint64_t pol_stream = l2_policy_evict_first(), pol_keep = l2_policy_evict_last();

  // A cursor walks this warp's chunks in order: items gw, gw + GW, ..., chunks
  // 0..nc-1 of each, stages 0..S-1 round and round (phase flips per round).
  struct Cursor {
    int64_t it;
    int c, g, h, st;
    uint32_t ph;
  };
  auto start_item = [&](Cursor& k, int64_t it) {
    k.it = it;
    k.c = 0;
    k.g = (int)(it % n_g);
    k.h = (int)(it / n_g);
  };
  auto advance = [&](Cursor& k) {
    if (++k.st == S) {
      k.st = 0;
      k.ph ^= 1u;
    }
    if (++k.c == nc) start_item(k, k.it + GW);
  };
  Cursor cons, prod;
  cons.st = prod.st = 0;
  cons.ph = prod.ph = 0;
  start_item(cons, (int64_t)blockIdx.x * kTmaWarps + w);
  prod = cons;
  uint32_t pend = 0, pend_ph = 0;   // stages with a load in flight, and its phase
  auto issue = [&]() {              // next chunk of the producer cursor
    const uint32_t bar = smem_addr(&bars[prod.st]);
    unsigned char* sb = stages + prod.st * T::SW_STAGE;
    if (lane == 0) {
      mbar_expect_tx(bar, T::STAGE_TX);
      tma_load_3d(smem_addr(sb), &tm_adc, prod.c * CH, prod.g * 32, prod.h * E, bar, pol_stream);
      tma_load_2d(smem_addr(sb + T::A_BYTES), &tm_noise, prod.c * CH, prod.g * 32, bar, pol_keep);
      tma_load_2d(smem_addr(bad_boxes + prod.st * T::BAD_BYTES), &tm_bad, prod.g * 32, prod.c * (CH / 32), bar,
                  pol_keep);
    }
    pend |= 1u << prod.st;
    pend_ph = (pend_ph & ~(1u << prod.st)) | (prod.ph << prod.st);
    advance(prod);
  };
  for (int s = 0; s < S && prod.it < n_items; ++s) issue();

  auto flush = [&]() {   // whole warp, converged
    __syncwarp();
    const int n = min(*(volatile int*)fill, kRingCap);
    if (n > 0) {
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(count, (unsigned long long)n);
      base = __shfl_sync(0xFFFFFFFFu, base, 0);
      for (int j = lane; j < n; j += 32)
        put_cluster(Cluster{ring[j], ring[kRingCap + j], ring[2 * kRingCap + j], ring[3 * kRingCap + j],
                            __int_as_float(ring[4 * kRingCap + j])},
                    base + j, out_row, out_first, out_last, out_charge, out_center, max_out, status);
    }
    __syncwarp();
    if (lane == 0) *fill = 0;
    __syncwarp();
  };
  auto close = [&](RunU& s, bool valid, int row) {   // divergent
    if (valid && runu_kept(s, q_min)) {
      const Cluster c = runu_cluster(s, row);
      const int idx = atomicAdd(fill, 1);
      if (idx < kRingCap) {
        ring[idx] = c.row;
        ring[kRingCap + idx] = c.first;
        ring[2 * kRingCap + idx] = c.last;
        ring[3 * kRingCap + idx] = c.charge;
        ring[4 * kRingCap + idx] = __float_as_int(c.center);
      } else {
        put_cluster(c, atomicAdd(count, 1ull), out_row, out_first, out_last, out_charge, out_center, max_out,
                    status);
      }
    }
    s.open = false;
  };

  RunU run[E];
  bool timed_out = false;
  while (cons.it < n_items) {
    const int c = cons.c, h = cons.h, st = cons.st;
    const int m = cons.g * 32 + lane;
    if (!mbar_wait(smem_addr(&bars[st]), cons.ph, status)) {
      timed_out = true;
      break;
    }
    pend &= ~(1u << st);
    const unsigned char* sa = stages + st * T::SW_STAGE;
    const unsigned char* sn = sa + T::A_BYTES;
    const uint32_t* sbad = reinterpret_cast<const uint32_t*>(bad_boxes + st * T::BAD_BYTES);
    if (c == 0) {
#pragma unroll
      for (int k = 0; k < E; ++k) run[k].open = false;
    }
    // masks of the chunk: candidates and breaks (good strips below threshold)
    Mask cmk[E], brkk[E];
#pragma unroll
    for (int k = 0; k < E; ++k) cmk[k] = brkk[k] = 0;
#pragma unroll
    for (int sb = 0; sb < CH / 32; ++sb) {   // 32-strip blocks of the chunk
      // calibration: 0x8000 | floor(nq / 4) per half (4 a > nq <=> a > floor(nq / 4) for integers)
      uint32_t tq[16];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint4 v = lds128(sn, swz<T::RB>(lane * T::RB + sb * 64 + j * 16));
        tq[4 * j] = ((v.x >> 2) & 0x3FFF3FFFu) | 0x80008000u;
        tq[4 * j + 1] = ((v.y >> 2) & 0x3FFF3FFFu) | 0x80008000u;
        tq[4 * j + 2] = ((v.z >> 2) & 0x3FFF3FFFu) | 0x80008000u;
        tq[4 * j + 3] = ((v.w >> 2) & 0x3FFF3FFFu) | 0x80008000u;
      }
      const uint32_t bm = sbad[sb * 32 + lane];
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const int r = k * 32 + lane;
        // candidate bits: with a' = min(a, 0x7FFF) (> floor(nq / 4) exactly when a is), the
        // half (0x8000 | floor(nq / 4)) - a' keeps its top bit unless the strip is a candidate
        uint32_t v = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint4 av = lds128(sa, swz<T::RB>(r * T::RB + sb * 64 + j * 16));
          const uint32_t aw[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int kk = 4 * j + i;   // word kk holds strips 2kk (low half) and 2kk + 1 (high half)
            const uint32_t x = tq[kk] - min_u16x2(aw[i], 0x7FFF7FFFu);
            v |= (~x & 0x80008000u) >> (15 - kk);
          }
        }
        const uint32_t cm = perfect_shuffle(v) & ~bm;
        cmk[k] |= (Mask)cm << (32 * sb);
        brkk[k] |= (Mask)(~(cm | bm)) << (32 * sb);
      }
    }
    const int c0 = c * CH;
    // shared-memory offset of strip p of row r: the swizzle XOR depends on the row only
    const int nrow = lane * T::RB, nx = swz<T::RB>(nrow) - nrow;
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int e = h * E + k, r = k * 32 + lane;
      const bool valid = e < n_events && m < n_modules;
      const int row = e * n_modules + m;
      const int arow = r * T::RB, ax = swz<T::RB>(arow) - arow;
      const Mask brk = brkk[k];
      RunU& s = run[k];
      Mask todo = cmk[k];
      while (todo) {
        const int p = (CH == 64) ? __ffsll((long long)todo) - 1 : __ffs((int)todo) - 1;
        todo &= todo - 1;
        const int gi = c0 + p;
        if (s.open) {   // only bad strips, at most max_bad_gap of them, since the last candidate?
          const int lo = max(s.last + 1 - c0, 0);
          const Mask between = brk & (((Mask)1 << p) - 1) & (~(Mask)0 << lo);
          if (between != 0 || gi - s.last - 1 > max_bad_gap) close(s, valid, row);
        }
        const uint32_t a = *reinterpret_cast<const uint16_t*>(sa + arow + ((2 * p) ^ ax));
        const uint32_t nq = *reinterpret_cast<const uint16_t*>(sn + nrow + ((2 * p) ^ nx));
        const bool fresh = !s.open;
        s.first = fresh ? gi : s.first;
        s.q = (fresh ? 0u : s.q) + a;
        s.q2 = (unsigned long long)a * a + (fresh ? 0ull : s.q2);
        s.n2 = (unsigned long long)nq * nq + (fresh ? 0ull : s.n2);
        s.qi = (unsigned long long)(uint32_t)(gi - s.first) * a + (fresh ? 0ull : s.qi);
        s.seeded = (s.seeded && !fresh) || 8 * a > 3 * nq;
        s.open = true;
        s.last = gi;
      }
      if (s.open) {   // a break after the last candidate, or too many bad strips since it
        const int lo = s.last + 1 - c0;
        const Mask after = lo <= 0 ? ~(Mask)0 : lo >= CH ? (Mask)0 : ~(Mask)0 << lo;
        if ((brk & after) != 0 || c0 + CH - 1 - s.last > max_bad_gap) close(s, valid, row);
      }
      if (c == nc - 1 && s.open) close(s, valid, row);   // end of the row
    }
    __syncwarp();
    advance(cons);
    if (prod.it < n_items) {
      if (lane == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue();
    }
    if (c == nc - 1 || *(volatile int*)fill >= kRingCap / 2) flush();
  }
  if (timed_out) {   // let copies that may still be in flight land before the block exits
    for (int s = 0; s < S; ++s)
      if ((pend >> s) & 1) mbar_wait(smem_addr(&bars[s]), (pend_ph >> s) & 1, status);
  }
}

// Bad-strip flags [M][N] bytes -> bits [ceil(N/32)][Mp] words (Mp = M rounded
// up to 4, so rows are 16-byte strides for TMA; words of modules >= M are 0):
// bit i of word [w][m] is strip 32 w + i of module m.  N is a multiple of 16.
__global__ void k_pack_bad(const uint8_t* __restrict__ bad, int n_modules, int n_strips, int mp,
                           uint32_t* __restrict__ bits) {
  const int nw = (n_strips + 31) / 32;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nw * mp) return;
  const int wi = (int)(t % nw), m = (int)(t / nw);
  uint32_t word = 0;
  if (m < n_modules) {
    const uint8_t* row = bad + (int64_t)m * n_strips + wi * 32;
    const int nb = min(32, n_strips - wi * 32);   // 16 or 32
    for (int q = 0; q < nb; q += 16) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(row + q));
      const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int b = 0; b < 4; ++b) word |= (uint32_t)(((wv[i] >> (8 * b)) & 0xFFu) != 0) << (q + 4 * i + b);
    }
  }
  bits[(int64_t)wi * mp + m] = word;
}

// ---------------------------------------------------------------------------
// Plain path: any width and alignment; one lane per row, one strip at a time.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kFallbackThreads)
    k_strip_cluster_plain(const uint16_t* __restrict__ adc, const uint16_t* __restrict__ noise_q,
                          const uint8_t* __restrict__ bad, int64_t n_rows, int n_modules, int n_strips,
                          int max_bad_gap, int q_min, int* __restrict__ out_row, int* __restrict__ out_first,
                          int* __restrict__ out_last, int* __restrict__ out_charge, float* __restrict__ out_center,
                          int64_t max_out, unsigned long long* __restrict__ count, int* __restrict__ status) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n_rows) return;
  const int64_t m = row % n_modules;
  const uint16_t* a_row = adc + row * n_strips;
  const uint16_t* n_row = noise_q + m * n_strips;
  const uint8_t* b_row = bad + m * n_strips;
  Run s{0, 0, 0, false, false, 0, 0, 0};
  auto close = [&]() {
    if (run_kept(s, q_min))
      put_cluster(run_cluster(s, (int)row), atomicAdd(count, 1ull), out_row, out_first, out_last, out_charge,
                  out_center, max_out, status);
    s.open = false;
  };
  for (int i = 0; i < n_strips; ++i) {
    if (__ldg(&b_row[i])) {
      if (s.open && ++s.pend > max_bad_gap) close();
      continue;
    }
    const long long a = __ldg(&a_row[i]), nq = __ldg(&n_row[i]);
    if (4 * a > nq) {
      if (!s.open) {
        s.open = true;
        s.seeded = false;
        s.first = i;
        s.q = s.d = s.qi = 0;
      }
      s.last = i;
      s.pend = 0;
      s.q += a;
      s.d += 64 * a * a - 25 * nq * nq;
      s.qi += (i - s.first) * a;
      s.seeded |= 8 * a > 3 * nq;
    } else {
      close();
    }
  }
  close();
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static const EncodeTiled fn = []() -> EncodeTiled {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

CUtensorMapSwizzle swizzle_for(int row_bytes) {
  return row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                          : row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
}

// rank-2 or rank-3 map, dims innermost first and densely packed, element
// strides 1, zero fill outside the tensor.
bool encode(CUtensorMap* tm, CUtensorMapDataType dt, int esize, const void* base, int rank, const cuuint64_t* dims,
            const cuuint32_t* box, CUtensorMapSwizzle swizzle) {
  EncodeTiled fn = encoder();
  if (!fn) return false;
  cuuint64_t strides[2];
  strides[0] = dims[0] * esize;
  if (rank == 3) strides[1] = strides[0] * dims[1];
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(tm, dt, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int CH, int E, int S>
cudaError_t launch_tma(mkf_ctx* ctx, const uint16_t* adc, const uint16_t* noise_q, const uint8_t* bad, int n_events,
                       int n_modules, int n_strips, int max_bad_gap, int q_min, int* out_row, int* out_first,
                       int* out_last, int* out_charge, float* out_center, int64_t max_out,
                       unsigned long long* out_count, cudaStream_t st, bool* encoded) {
  using T = TmaShape<CH, E, S>;
  // bad flags -> bits [nw][mp]
  const int nw = (n_strips + 31) / 32, mp = (n_modules + 3) / 4 * 4;
  cudaError_t e = ctx->strip_bits.ensure((size_t)nw * mp * sizeof(uint32_t));
  if (e != cudaSuccess) return e;
  uint32_t* bits = ctx->strip_bits.as<uint32_t>();
  const int64_t words = (int64_t)nw * mp;
  k_pack_bad<<<(unsigned)((words + 255) / 256), 256, 0, st>>>(bad, n_modules, n_strips, mp, bits);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  CUtensorMap tm_a, tm_n, tm_b;
  const cuuint64_t da[3] = {(cuuint64_t)n_strips, (cuuint64_t)n_modules, (cuuint64_t)n_events};
  const cuuint64_t db[2] = {(cuuint64_t)mp, (cuuint64_t)nw};
  const cuuint32_t ba[3] = {CH, 32, E}, bn[2] = {CH, 32}, bb[2] = {32, CH / 32};
  *encoded = encode(&tm_a, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, adc, 3, da, ba, swizzle_for(T::RB)) &&
             encode(&tm_n, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, noise_q, 2, da, bn, swizzle_for(T::RB)) &&
             encode(&tm_b, CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, bits, 2, db, bb, CU_TENSOR_MAP_SWIZZLE_NONE);
  if (!*encoded) return cudaSuccess;
  auto kern = k_strip_cluster_tma<CH, E, S>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTmaWarps * 32, T::SMEM)) != cudaSuccess)
    return e;
  const int64_t items = (int64_t)((n_modules + 31) / 32) * ((n_events + E - 1) / E);
  const int64_t want = (items + kTmaWarps - 1) / kTmaWarps;
  const int64_t cap = (int64_t)ctx->n_sm * (per_sm > 0 ? per_sm : 1);
  const unsigned blocks = (unsigned)(want < cap ? want : cap);
  kern<<<blocks, kTmaWarps * 32, T::SMEM, st>>>(tm_a, tm_n, tm_b, n_events, n_modules, n_strips, max_bad_gap, q_min,
                                                 out_row, out_first, out_last, out_charge, out_center, max_out,
                                                 out_count, ctx->status.as<int>());
  return cudaGetLastError();
}

}  // namespace

}  // namespace mkf

namespace {
// Work splits the TMA kernel is built for: strips per chunk, events per item, stages.
constexpr int kStripSplits[][3] = {{32, 1, 1}, {32, 1, 2}, {32, 1, 3}, {32, 1, 4}, {32, 2, 2},
                                    {64, 1, 2}, {64, 1, 3}, {64, 2, 2}};
constexpr int kStripDefault[3] = {32, 1, 1};
}  // namespace

extern "C" mkf_status mkf_set_strip_config(mkf_ctx* ctx, int chunk, int events_per_item, int stages) {
  if (!ctx) return MKF_ERR_ARG;
  bool ok = chunk == 0 && events_per_item == 0 && stages == 0;
  for (const auto& k : kStripSplits) ok |= k[0] == chunk && k[1] == events_per_item && k[2] == stages;
  if (!ok) return ctx->fail(MKF_ERR_ARG, "strip config: not one of the built work splits");
  ctx->strip_chunk = chunk;
  ctx->strip_events = events_per_item;
  ctx->strip_stages = stages;
  return MKF_OK;
}

extern "C" mkf_status mkf_cluster_strips(mkf_ctx* ctx, const uint16_t* adc, const uint16_t* noise_q,
                                         const uint8_t* bad, int n_events, int n_modules, int n_strips,
                                         int max_bad_gap, int q_min, int* out_row, int* out_first, int* out_last,
                                         int* out_charge, float* out_center, int64_t max_out,
                                         unsigned long long* out_count, void* stream) {
  if (!ctx) return MKF_ERR_ARG;
  if (n_events < 0 || n_modules < 1 || n_strips < 1 || n_strips > (1 << 20) || max_bad_gap < 0 || max_out < 0 ||
      (int64_t)n_events * n_modules > (int64_t)INT32_MAX)
    return ctx->fail(MKF_ERR_ARG, "bad sizes");
  if (!noise_q || !bad || !out_count || (n_events > 0 && !adc) ||
      (max_out > 0 && (!out_row || !out_first || !out_last || !out_charge || !out_center)))
    return ctx->fail(MKF_ERR_ARG, "null array");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = ctx->status.ensure(sizeof(int));
  if (e != cudaSuccess) return ctx->fail(MKF_ERR_OOM, "status word");
  if ((e = cudaMemsetAsync(out_count, 0, sizeof(unsigned long long), st)) != cudaSuccess)
    return ctx->cuda_fail(e, "count");
  const int64_t rows = (int64_t)n_events * n_modules;
  if (rows == 0) return MKF_OK;
  // TMA needs 16-byte aligned bases and row strides (bad flags: 1 byte a strip);
  // the TMA kernel keeps a cluster's charge in 32 bits (rows of <= 65536 strips)
  const bool tma = n_strips % 16 == 0 && n_strips <= 65536 && (uintptr_t)adc % 16 == 0 && (uintptr_t)noise_q % 16 == 0 &&
                   (uintptr_t)bad % 16 == 0;
  if (tma) {
    bool encoded = false;
    // default: one event per item and one stage per warp.  A warp then holds
    // 5.8 KB of shared memory, so 9 blocks (36 warps) fit an SM, twice the
    // two-stage split's residency: the other warps' loads hide each warp's
    // load latency, and the items fill fewer, fuller rounds
    const bool dflt = ctx->strip_chunk == 0;
    const int ch = dflt ? kStripDefault[0] : ctx->strip_chunk,
              ev = dflt ? kStripDefault[1] : ctx->strip_events,
              ns = dflt ? kStripDefault[2] : ctx->strip_stages;
#define MKF_STRIP_ARGS                                                                                           \
  ctx, adc, noise_q, bad, n_events, n_modules, n_strips, max_bad_gap, q_min, out_row, out_first, out_last, \
      out_charge, out_center, max_out, out_count, st, &encoded
#define MKF_STRIP_CASE(C, E, S) \
  else if (ch == C && ev == E && ns == S) e = mkf::launch_tma<C, E, S>(MKF_STRIP_ARGS);
    if (false) {
    }
    MKF_STRIP_CASE(32, 1, 1) MKF_STRIP_CASE(32, 1, 2) MKF_STRIP_CASE(32, 1, 3) MKF_STRIP_CASE(32, 1, 4) MKF_STRIP_CASE(32, 2, 2)
    MKF_STRIP_CASE(64, 1, 2) MKF_STRIP_CASE(64, 1, 3) MKF_STRIP_CASE(64, 2, 2)
    else return ctx->fail(MKF_ERR_ARG, "strip config");
#undef MKF_STRIP_CASE
#undef MKF_STRIP_ARGS
    if (e != cudaSuccess) return ctx->cuda_fail(e, "strip clustering");
    if (!encoded) return ctx->fail(MKF_ERR_CUDA, "strip clustering: tensor map encoding failed");
    return MKF_OK;
  }
  const unsigned blocks = (unsigned)((rows + mkf::kFallbackThreads - 1) / mkf::kFallbackThreads);
  mkf::k_strip_cluster_plain<<<blocks, mkf::kFallbackThreads, 0, st>>>(
      adc, noise_q, bad, rows, n_modules, n_strips, max_bad_gap, q_min, out_row, out_first, out_last, out_charge,
      out_center, max_out, out_count, ctx->status.as<int>());
  if ((e = cudaGetLastError()) != cudaSuccess) return ctx->cuda_fail(e, "strip clustering");
  return MKF_OK;
}
