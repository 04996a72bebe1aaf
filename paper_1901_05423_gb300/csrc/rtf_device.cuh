// Device-side helpers shared by the build, sample and backward kernels.
//
// Exact integer arithmetic of the fixed-point reading of the paper's CDF
// (Sec. 1), the keys of Algorithm 1 (Sec. 3.2) in the 32-bit sample domain,
// the bounded lookback waits, and a few warp/block scan primitives.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rtf.h"

namespace rtf {

// ---------------------------------------------------------------------------
// tunables (tile shapes); the build and the workspace layout agree on them
// ---------------------------------------------------------------------------
constexpr int kTile = 2048;           // weights per scan / forest tile
constexpr int kScanThreads = 256;     // scan kernel: 8 weights per thread
constexpr int kForestThreads = 512;   // forest kernel: 4 leaves per thread
constexpr int kMaxThreads = 512;
constexpr int kTileScanChunk = 512;   // tile sums per block of the segmented tile scan
constexpr uint32_t kDeltaInf = 64;    // distance across a cell / distribution boundary
constexpr long long kSpinLimit = 1ll << 22;   // bounded waits
// Nodes of a forest tile whose range reaches past the tile (their parent needs
// distances outside it): at most 33 whose nearest larger distance on the right
// lies outside (their distances strictly decrease from left to right) plus 33
// whose nearest larger one on the left lies outside and whose right bound does
// not settle the parent (strictly increasing distances).
constexpr int kUnresCap = 72;
constexpr int kTileGroup = 64;        // forest tiles per group of the distance maxima
// Cells that no key falls into are written by whoever finishes the non-empty
// cell before them: up to kFillInline at once, longer runs listed in pieces of
// at most kFillPiece cells for the fill pass.
constexpr int kFillInline = 16;
constexpr int64_t kFillPiece = int64_t(1) << 16;

// status-word flags of the decoupled lookback (top two bits of a u64)
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagPrefix = 2ull << 62;
constexpr uint64_t kValueMask = (1ull << 62) - 1;

// ---------------------------------------------------------------------------
// workspace layout (byte offsets, 256-aligned regions)
// ---------------------------------------------------------------------------
struct WsLayout {
  size_t zero_begin;   // start of the region zero-filled by every build
  size_t counters;     // u32 tickets / done counters
  size_t dmax;         // u32 [D] max float bits per distribution / group
  size_t scan_status;  // u64 [num_tiles / kTileScanChunk + 1] status of the tile-sum scan blocks
  size_t gmax;         // u32 [num_tiles / kTileGroup] largest distance per group of tiles
  size_t zero_end;
  size_t fills;        // int4 [fill_cap] runs of empty cells: first cell, count, leaf, dist
  size_t tile_prefix;  // u64 [num_tiles]
  size_t tile_sum;     // u64 [num_tiles]
  size_t tile_first;   // u64 [num_tiles]
  size_t tile_meta;    // u32 [num_tiles]
  size_t tile_dist0;   // i32 [num_tiles]
  size_t delta;        // u8  [N] distance between leaves j and j + 1
  size_t tmax;         // u8  [num_tiles] largest distance of each forest tile
  size_t unres;        // i32 [num_tiles * kUnresCap] nodes left to the merge pass
  size_t unres_count;  // i32 [num_tiles]
  size_t total;
};

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

__host__ __device__ inline int64_t num_tiles(int64_t n) { return (n + kTile - 1) / kTile; }

// Pieces of runs of empty cells the fill pass may receive: each run longer than
// kFillInline cells is at least kFillInline + 1 cells and splits into at most
// count / kFillPiece + 1 pieces.
__host__ __device__ inline int64_t fill_cap(int32_t D, int64_t G) {
  return G / (kFillInline + 1) + G / kFillPiece + D + 16;
}

__host__ __device__ inline WsLayout ws_layout(int64_t N, int32_t D, int64_t G) {
  WsLayout L;
  size_t o = 0;
  L.zero_begin = o;
  L.counters = o; o += 256;
  L.dmax = o; o = align256(o + sizeof(uint32_t) * (size_t)D);
  L.scan_status = o;
  o = align256(o + sizeof(uint64_t) * (size_t)(num_tiles(N) / kTileScanChunk + 1));
  L.gmax = o;
  o = align256(o + sizeof(uint32_t) * (size_t)((num_tiles(N) + kTileGroup - 1) / kTileGroup));
  L.zero_end = o;
  L.fills = o; o = align256(o + 16 * (size_t)fill_cap(D, G));
  L.tile_prefix = o; o = align256(o + sizeof(uint64_t) * (size_t)num_tiles(N));
  L.tile_sum = o; o = align256(o + sizeof(uint64_t) * (size_t)num_tiles(N));
  L.tile_first = o; o = align256(o + sizeof(uint64_t) * (size_t)num_tiles(N));
  L.tile_meta = o; o = align256(o + sizeof(uint32_t) * (size_t)num_tiles(N));
  L.tile_dist0 = o; o = align256(o + sizeof(int32_t) * (size_t)num_tiles(N));
  L.delta = o; o = align256(o + (size_t)N);
  L.tmax = o; o = align256(o + (size_t)num_tiles(N));
  L.unres = o; o = align256(o + sizeof(int32_t) * (size_t)kUnresCap * (size_t)num_tiles(N));
  L.unres_count = o; o = align256(o + sizeof(int32_t) * (size_t)num_tiles(N));
  L.total = o;
  return L;
}

// counters inside WsLayout::counters
struct Counters {
  uint32_t scan_ticket;
  uint32_t fill_count;
  uint32_t scan_done;
  uint32_t pad[61];
};

// internal rtf_dist.flags
constexpr int32_t kDistMarginal = 1;   // weights are the totals of dists [0, D-1)
constexpr int32_t kDistShared = 2;     // scale shared with every non-marginal dist

// ---------------------------------------------------------------------------
// status word
// ---------------------------------------------------------------------------
__device__ __forceinline__ void raise_status(uint32_t* status, uint32_t bits) {
  atomicOr(status, bits);
}

// ---------------------------------------------------------------------------
// float weights -> fixed point
// ---------------------------------------------------------------------------
// Bits of a weight with -0 folded to +0.
__device__ __forceinline__ uint32_t weight_bits(float x) {
  uint32_t b = __float_as_uint(x);
  return b == 0x80000000u ? 0u : b;
}

__device__ __forceinline__ bool weight_bad(uint32_t b) {
  return (b >> 31) != 0 || (b & 0x7F800000u) == 0x7F800000u;
}

// floor(log2 x) for the bits of a positive finite float (subnormals too).
__device__ __forceinline__ int floor_log2_bits(uint32_t b) {
  uint32_t E = b >> 23;
  if (E) return (int)E - 127;
  return (31 - __clz(b & 0x7FFFFFu)) - 149;
}

__host__ __device__ inline int ceil_log2_i64(int64_t n) {
  if (n <= 1) return 0;
#ifdef __CUDA_ARCH__
  return 64 - __clzll((long long)(n - 1));
#else
  return 64 - __builtin_clzll((unsigned long long)(n - 1));
#endif
}

// S = B - 1 - e_max with B = 62 - ceil(log2 n_group).
__device__ __forceinline__ int scale_from_max(uint32_t maxbits, int64_t n_group) {
  int B = 62 - ceil_log2_i64(n_group);
  return B - 1 - floor_log2_bits(maxbits);
}

// q = floor(w 2^S) from the bits of w: an exact shift of the integer
// significand.
__device__ __forceinline__ uint64_t quantize_bits(uint32_t b, int S) {
  if (b == 0) return 0;
  uint32_t E = b >> 23;
  uint64_t M;
  int e2;
  if (E) {
    M = (b & 0x7FFFFFu) | 0x800000u;
    e2 = (int)E - 150;
  } else {
    M = b & 0x7FFFFFu;
    e2 = -149;
  }
  int sh = e2 + S;
  if (sh >= 0) return M << sh;
  sh = -sh;
  return sh >= 64 ? 0ull : (M >> sh);
}

// ---------------------------------------------------------------------------
// sample-domain arithmetic
// ---------------------------------------------------------------------------
// t(u) = floor(u T / 2^32) for 0 <= u <= 2^32 (T < 2^62).
__device__ __forceinline__ uint64_t t_of(uint64_t u, uint64_t T) {
  return u >= (1ull << 32) ? T : __umul64hi(T, u << 32);
}

// floor((hi 2^64 + lo) / d) for hi < d (restoring long division; used once per
// distribution).
__device__ inline uint64_t div128_64(uint64_t hi, uint64_t lo, uint64_t d) {
  uint64_t q = 0;
  for (int i = 0; i < 64; ++i) {
    uint64_t carry = hi >> 63;
    hi = (hi << 1) | (lo >> 63);
    lo <<= 1;
    q <<= 1;
    if (carry || hi >= d) {
      hi -= d;
      q |= 1;
    }
  }
  return q;
}

// Reciprocal of the normalised total: floor((2^128 - 1) / (T << z)) - 2^64.
__device__ inline uint64_t total_recip(uint64_t T, int z) {
  uint64_t Tn = T << z;
  return div128_64(~Tn, ~0ull, Tn);
}

// Key K = ceil(C 2^32 / T): the smallest u with t(u) >= C.  With X = C << z
// and Tn = T << z, one multiply by the reciprocal gives Q' = floor(X 2^64 / Tn)
// or one less, so X 2^64 / Tn lies in [Q', Q' + 2).  Unless the low word of Q'
// is 0 or 2^32 - 1 that interval sits strictly between two multiples of 2^32
// and K = (Q' >> 32) + 1; next to a multiple, two exact checks decide.
__device__ __forceinline__ uint64_t key_of(uint64_t C, uint64_t T, uint64_t R, int z) {
  if (C >= T) return 1ull << 32;
  const uint64_t X = C << z;
  const uint64_t Q = __umul64hi(X, R) + X;
  const uint32_t lo = (uint32_t)Q;
  uint64_t v = Q >> 32;
  if (lo != 0u && lo != 0xFFFFFFFFu) return v + 1;
  if (t_of(v, T) < C) {
    ++v;
    if (t_of(v, T) < C) ++v;
  }
  return v;
}

// Cell of a key among 2^m cells; 2^m for K = 2^32.
__device__ __forceinline__ uint64_t cell_of(uint64_t K, int m) { return K >> (32 - m); }

// Distance of two neighbouring keys of one cell: bit length of their XOR
// (the XOR of two keys of one cell fits in 32 bits).
__device__ __forceinline__ uint32_t key_distance(uint64_t a, uint64_t b) {
  return 32u - (uint32_t)__clz((uint32_t)(a ^ b));
}

// Round a 64-bit unsigned integer to the nearest float32 (ties to even), the
// hardware conversion.  (A variant that normalises, folds the low bits into a
// sticky bit and converts 32 bits gives the same values; on GB300 it took more
// issue slots in the sorted sampler, 2.09 vs 1.93 ms for 2^28 samples.)
__device__ __forceinline__ float u64_to_f32(uint64_t x) { return __ull2float_rn(x); }

// ---------------------------------------------------------------------------
// memory ordering helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ---------------------------------------------------------------------------
// block-wide scans
// ---------------------------------------------------------------------------
// Segmented exclusive scan of (head, value) pairs, one pair per thread:
// (f1, s1) + (f2, s2) = (f1 | f2, f2 ? s2 : s1 + s2).  Returns the exclusive
// prefix (sum since the last head before this thread, or 0) and stores the
// block total in *total_f / *total_s.  `scratch` needs 2 * (blockDim/32)
// u64 + flags.
struct SegPair {
  uint64_t s;
  uint32_t f;
};

__device__ __forceinline__ SegPair seg_combine(SegPair a, SegPair b) {
  SegPair r;
  r.f = a.f | b.f;
  r.s = b.f ? b.s : a.s + b.s;
  return r;
}

__device__ inline SegPair block_seg_exclusive(SegPair x, SegPair* warp_tot, SegPair* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // inclusive warp scan
  SegPair inc = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    SegPair o;
    o.s = __shfl_up_sync(0xffffffffu, inc.s, d);
    o.f = __shfl_up_sync(0xffffffffu, inc.f, d);
    if (lane >= d) inc = seg_combine(o, inc);
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    SegPair v = lane < nw ? warp_tot[lane] : SegPair{0ull, 0u};
    SegPair vi = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      SegPair o;
      o.s = __shfl_up_sync(0xffffffffu, vi.s, d);
      o.f = __shfl_up_sync(0xffffffffu, vi.f, d);
      if (lane >= d) vi = seg_combine(o, vi);
    }
    if (lane < nw) warp_tot[lane] = vi;  // inclusive over warps
    if (lane == nw - 1) *total = vi;
  }
  __syncthreads();
  SegPair excl_warp = warp > 0 ? warp_tot[warp - 1] : SegPair{0ull, 0u};
  // exclusive within warp
  SegPair ex;
  ex.s = __shfl_up_sync(0xffffffffu, inc.s, 1);
  ex.f = __shfl_up_sync(0xffffffffu, inc.f, 1);
  if (lane == 0) ex = SegPair{0ull, 0u};
  SegPair r = seg_combine(excl_warp, ex);
  __syncthreads();
  return r;
}

// Plain (unsegmented) exclusive block scan of u64 values; *total receives the
// block's sum.
__device__ inline uint64_t block_exclusive_u64(uint64_t x, uint64_t* warp_tot, uint64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint64_t inc = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t o = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += o;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint64_t v = lane < nw ? warp_tot[lane] : 0ull;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t o = __shfl_up_sync(0xffffffffu, v, d);
      if (lane >= d) v += o;
    }
    if (lane < nw) warp_tot[lane] = v;
    if (lane == nw - 1) *total = v;
  }
  __syncthreads();
  const uint64_t r = (warp > 0 ? warp_tot[warp - 1] : 0ull) + inc - x;
  __syncthreads();
  return r;
}

// Plain (unsegmented) exclusive block scan of u32 values.
__device__ inline uint32_t block_exclusive_u32(uint32_t x, uint32_t* warp_tot, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t o = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += o;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = lane < nw ? warp_tot[lane] : 0u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint32_t o = __shfl_up_sync(0xffffffffu, v, d);
      if (lane >= d) v += o;
    }
    if (lane < nw) warp_tot[lane] = v;
    if (lane == nw - 1) *total = v;
  }
  __syncthreads();
  uint32_t r = (warp > 0 ? warp_tot[warp - 1] : 0u) + inc - x;
  __syncthreads();
  return r;
}

// Block-wide decoupled lookback over u64 status words (flag in the top two
// bits, value below).  Every thread of the block reads one predecessor status
// per round, so one round covers blockDim tiles.  Returns, to every thread,
// the sum of the values from tile-1 back to and including the nearest tile
// that published a prefix (`sum` = true), or that prefix's value alone
// (`sum` = false).  Waits are bounded; on expiry RTF_STATUS_TIMEOUT is raised and the
// partial result returned.
struct LookbackShared {
  int first_prefix;
  int first_invalid;
  uint64_t part[32];
  uint64_t result;
};

__device__ __forceinline__ uint64_t block_lookback(const uint64_t* st, int64_t tile, bool sum,
                                          LookbackShared* sh, uint32_t* status) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  uint64_t E = 0;
  int64_t look = tile - 1;
  long long spins = 0;
  while (look >= 0) {
    if (tid == 0) {
      sh->first_prefix = nt;
      sh->first_invalid = nt;
    }
    __syncthreads();
    const int64_t idx = look - tid;
    uint64_t s = idx >= 0 ? ld_acquire_u64(st + idx) : kFlagPrefix;
    const uint32_t flag = (uint32_t)(s >> 62);
    if (flag == 2) atomicMin(&sh->first_prefix, tid);
    if (flag == 0) atomicMin(&sh->first_invalid, tid);
    __syncthreads();
    const int p = sh->first_prefix, q = sh->first_invalid;
    if (q < p) {
      // a predecessor before the nearest prefix has not published yet
      if (++spins > kSpinLimit) {
        if (tid == 0) raise_status(status, RTF_STATUS_TIMEOUT);
        break;
      }
      __nanosleep(64);
      __syncthreads();
      continue;
    }
    uint64_t v = 0;
    if (sum) {
      v = (tid <= p && idx >= 0) ? (s & kValueMask) : 0ull;
    } else {
      v = (tid == p && idx >= 0) ? (s & kValueMask) : 0ull;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh->part[warp] = v;
    __syncthreads();
    if (tid == 0) {
      uint64_t t = 0;
      for (int w = 0; w < (nt >> 5); ++w) t += sh->part[w];
      sh->result = t;
    }
    __syncthreads();
    E += sh->result;
    if (p < nt) break;
    look -= nt;
  }
  __syncthreads();
  return E;
}

// Index of the distribution that owns element `e`: the largest d with
// dists[d].elem_off <= e (binary search over [lo, hi]).
__device__ inline int find_dist(const rtf_dist* dists, int lo, int hi, int64_t e) {
  // galloping from lo (callers pass the first distribution of a tile, and an
  // element usually lies in it or in one of the next few), then bisection
  int step = 1;
  while (lo < hi) {
    const int probe = lo + step < hi ? lo + step : hi;
    if (dists[probe].elem_off <= e) {
      lo = probe;
      step <<= 1;
    } else {
      hi = probe - 1;
      break;
    }
  }
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (dists[mid].elem_off <= e)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

}  // namespace rtf
