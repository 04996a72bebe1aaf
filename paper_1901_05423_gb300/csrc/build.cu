// Build of the radix tree forest (Binder & Keller, Sec. 3.2, Algorithm 1) and
// of the guide table (Cutpoint method, Sec. 2.5, with the encoding of
// Sec. 3.2) for one or many distributions at once (Sec. 5).
//
// Kernels, in launch order:
//   init_dists_kernel   per-distribution parameters from the plan; for a
//                       batch also the distribution of each tile's first
//                       element
//   scale_kernel        validation and max exponent (one read of w)
//   tile_sum_kernel     sums of the integer weights per tile (second read of
//                       w): for one distribution persistent blocks over
//                       ranges of tiles, the last one scanning the range
//                       totals; for a batch segmented sums, and the totals of
//                       the distributions that lie inside one tile
//   tile_scan_kernel    (batch) decoupled-lookback segmented scan of the tile
//                       sums: the prefix of every tile, the totals T (and key
//                       reciprocals) of the distributions that cross tiles; in
//                       marginal mode the last block also scans the row totals
//   forest_lean_kernel  (one distribution) and forest_kernel (batch): per
//                       2048-leaf tile C_j, keys K_j, distances, the links from
//                       the nearest larger distances, node records, the roots
//                       and guide entries of the cells that end inside the
//                       tile and of up to 16 empty cells after each (third
//                       read of w); forest_kernel sends a tile that lies
//                       inside one distribution down the same path as
//                       forest_lean_kernel
//   forest_merge_kernel the nodes whose bounding splits lie outside their tile,
//                       found in the global distance bytes with the largest
//                       distance per tile and per group of tiles
//   fill_kernel         the longer runs of cells that no key falls into
#include <algorithm>
#include <cstdint>

#include "rtf_device.cuh"

namespace rtf {

// The passes before the forest kernel read the weights with plain loads, not
// streaming ones, so that the forest kernel's third read of them (64 MB at
// n = 2^24) finds them in L2: the build 0.419 -> 0.403 ms on GB300.
__device__ __forceinline__ float4 ld_weights4(const float4* p) { return __ldg(p); }

// ---------------------------------------------------------------------------
// init
// ---------------------------------------------------------------------------
// Thread d < D fills dists[d]; thread t < ntiles also writes tile_dist0[t],
// the distribution that holds element t kTile (the last d with offsets[d] <=
// t kTile), by bisection over the offsets: the passes that follow start their
// searches there instead of at distribution 0.
__global__ void init_dists_kernel(rtf_dist* dists, int D, const int64_t* offsets,
                                  const int32_t* m_arr, const int64_t* goff, int marginal,
                                  int64_t n_single, int m_single, int32_t* tile_dist0,
                                  int64_t ntiles, uint32_t* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ntiles && offsets != nullptr) {
    const int64_t e = i * kTile;
    int lo = 0, hi = D - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (offsets[mid] <= e)
        lo = mid;
      else
        hi = mid - 1;
    }
    tile_dist0[i] = lo;
  }
  if (i >= D) return;
  const int d = (int)i;
  rtf_dist P;
  if (offsets == nullptr) {
    P.elem_off = 0;
    P.n = n_single;
    P.guide_off = 0;
    P.m = m_single;
  } else {
    P.elem_off = offsets[d];
    P.n = offsets[d + 1] - offsets[d];
    P.guide_off = goff[d];
    P.m = m_arr[d];
    bool bad = P.n < 1 || P.m < 0 || P.m > 30 ||
               goff[d + 1] - goff[d] != (int64_t(1) << (P.m < 0 || P.m > 30 ? 0 : P.m));
    if (marginal && d == D - 1 && P.n != D - 1) bad = true;
    if (bad) {
      raise_status(status, RTF_STATUS_BAD_PLAN);
      P.m = 0;
      if (P.n < 1) P.n = 1;
    }
  }
  P.total = 0;
  P.recip = 0;
  P.scale = 0;
  P.shift = 0;
  P.flags = 0;
  if (marginal) P.flags = (d == D - 1) ? kDistMarginal : kDistShared;
  P.reserved = 0;
  dists[d] = P;
}

// ---------------------------------------------------------------------------
// scale: max float bits per distribution (or per shared group) + validation
// ---------------------------------------------------------------------------
constexpr int kScaleThreads = 256;
constexpr int kScalePer = 16;
constexpr int kScaleTile = kScaleThreads * kScalePer;

template <bool SEG>
__global__ void __launch_bounds__(kScaleThreads)
    scale_kernel(const float* __restrict__ w, int64_t Nw, const rtf_dist* __restrict__ dists,
                 int Dw, const int32_t* __restrict__ tile_dist0, uint32_t* dmax,
                 uint32_t* status) {
  __shared__ uint32_t smax[SEG ? kScaleTile + 1 : 1];
  __shared__ int dfirst_s;
  __shared__ uint32_t red[kScaleThreads / 32];
  const int64_t c0 = (int64_t)blockIdx.x * kScaleTile;
  const int64_t c1 = min(c0 + (int64_t)kScaleTile, Nw);
  const int64_t e0 = c0 + (int64_t)threadIdx.x * kScalePer;
  uint32_t bad = 0;
  // one maximum for the whole block: one distribution (or one shared group),
  // or a block of a batch whose weights all belong to one distribution
  bool one = !SEG;
  uint32_t* target = dmax;
  if (SEG) {
    const int d0 = tile_dist0[c0 / kTile];
    const rtf_dist& P = dists[d0];
    if (P.elem_off <= c0 && c1 <= P.elem_off + P.n) {
      one = true;
      target = dmax + d0;
    }
  }
  if (one) {
    uint32_t mx = 0;
    if (e0 + kScalePer <= c1 && (reinterpret_cast<uintptr_t>(w) & 15) == 0) {
      const float4* p = reinterpret_cast<const float4*>(w + e0);
#pragma unroll
      for (int k = 0; k < kScalePer / 4; ++k) {
        float4 v = ld_weights4(p + k);
        uint32_t b0 = weight_bits(v.x), b1 = weight_bits(v.y), b2 = weight_bits(v.z),
                 b3 = weight_bits(v.w);
        bad |= weight_bad(b0) | weight_bad(b1) | weight_bad(b2) | weight_bad(b3);
        mx = max(mx, max(max(b0, b1), max(b2, b3)));
      }
    } else {
      for (int64_t e = e0; e < c1; ++e) {
        uint32_t b = weight_bits(w[e]);
        bad |= weight_bad(b);
        mx = max(mx, b);
      }
    }
    // invalid weights must not win the max
    if (bad) mx = 0;
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
      uint32_t v = threadIdx.x < kScaleThreads / 32 ? red[threadIdx.x] : 0u;
      v = __reduce_max_sync(0xffffffffu, v);
      if (threadIdx.x == 0 && v) atomicMax(target, v);
    }
    if (bad) raise_status(status, RTF_STATUS_BAD_WEIGHT);
    return;
  }
  // segmented: the block's elements span distributions dfirst..dlast
  if (threadIdx.x == 0) dfirst_s = tile_dist0[c0 / kTile];
  for (int k = threadIdx.x; k <= kScaleTile; k += kScaleThreads) smax[k] = 0u;
  __syncthreads();
  const int dfirst = dfirst_s;
  if (e0 < c1) {
    int hi = min(Dw - 1, dfirst + kScaleTile);
    int d = find_dist(dists, tile_dist0[e0 / kTile], hi, e0);
    int64_t next = d + 1 < Dw ? dists[d + 1].elem_off : INT64_MAX;
    uint32_t run = 0;
    const int64_t e1 = min(e0 + (int64_t)kScalePer, c1);
    // the thread's weights first, as 16-byte vectors where aligned
    float wv[kScalePer];
    if (e0 + kScalePer <= c1 && (reinterpret_cast<uintptr_t>(w) & 15) == 0) {
      const float4* p = reinterpret_cast<const float4*>(w + e0);
#pragma unroll
      for (int k = 0; k < kScalePer / 4; ++k) {
        const float4 v = ld_weights4(p + k);
        wv[4 * k] = v.x;
        wv[4 * k + 1] = v.y;
        wv[4 * k + 2] = v.z;
        wv[4 * k + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < kScalePer; ++k) wv[k] = e0 + k < c1 ? w[e0 + k] : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < kScalePer; ++k) {
      const int64_t e = e0 + k;
      if (e >= e1) break;
      if (e >= next) {
        if (run) atomicMax(&smax[d - dfirst], run);
        run = 0;
        ++d;
        next = d + 1 < Dw ? dists[d + 1].elem_off : INT64_MAX;
      }
      uint32_t b = weight_bits(wv[k]);
      if (weight_bad(b)) {
        bad = 1;
      } else {
        run = max(run, b);
      }
    }
    if (run) atomicMax(&smax[d - dfirst], run);
  }
  if (bad) raise_status(status, RTF_STATUS_BAD_WEIGHT);
  __syncthreads();
  const int dlast = (c1 > c0) ? find_dist(dists, tile_dist0[(c1 - 1) / kTile],
                                          min(Dw - 1, dfirst + kScaleTile), c1 - 1)
                              : dfirst;
  for (int d = dfirst + (int)threadIdx.x; d <= dlast; d += kScaleThreads) {
    uint32_t v = smax[d - dfirst];
    if (v) atomicMax(&dmax[d], v);
  }
}

// ---------------------------------------------------------------------------
// scan: tile sums of q with a decoupled lookback
// ---------------------------------------------------------------------------
struct DistScale {
  int S;
};

__device__ __forceinline__ int dist_scale(const rtf_dist& P, const uint32_t* dmax, int d,
                                          int64_t n_shared) {
  if (P.flags & kDistShared) return scale_from_max(dmax[0], n_shared);
  return scale_from_max(dmax[d], P.n);
}

// Finish one distribution once its total is known: T, reciprocal, scale.
__device__ inline void finish_dist(rtf_dist* dists, int d, uint64_t T, int S, uint32_t* status) {
  if (T == 0) {
    raise_status(status, RTF_STATUS_ZERO_TOTAL);
    T = 1;  // keep the key arithmetic defined; the status word says the result is void
  }
  int z = __clzll(T);
  dists[d].total = T;
  dists[d].shift = z;
  dists[d].recip = total_recip(T, z);
  dists[d].scale = S;
}

constexpr int kScanPer = kTile / kScanThreads;  // 8

// Per-tile results of tile_sum_kernel, consumed by tile_scan_kernel.
struct TileSums {
  uint64_t* sum;     // sum of q since the tile's last head (the whole tile without one)
  uint64_t* first;   // partial sum of the tile's first piece when its distribution ends here
  uint32_t* meta;    // bit0: a head lies in the tile, bit1: t0 is a head,
                     // bit2: the distribution of t0 ends inside the tile
  int32_t* dist0;    // distribution of t0
};

// Tile sums of q (second read of w, 16-byte loads).  Distributions that
// begin and end inside the tile are finished here; the tile's first piece,
// whose distribution began in an earlier tile, waits for the scan of the tile
// sums.
template <bool SEG>
__global__ void __launch_bounds__(kScanThreads)
    tile_sum_kernel(const float* __restrict__ w, int64_t Nw, rtf_dist* dists, int Dw,
                    int64_t n_shared, const uint32_t* dmax, TileSums ts, uint64_t* tile_prefix,
                    Counters* ctr, uint32_t* status) {
  __shared__ int dfirst_s;
  __shared__ SegPair wtot[kScanThreads / 32];
  __shared__ SegPair btot;
  __shared__ uint32_t meta_s;

  const int64_t tile = blockIdx.x;
  const int64_t t0 = tile * kTile, t1 = min(t0 + (int64_t)kTile, Nw);

  if (!SEG) {
    // one distribution, persistent blocks: block b sums the contiguous tiles
    // [b per, (b + 1) per) (weights straight from global memory, 16-byte
    // vectors where aligned) and writes each tile's prefix within that range
    // and the range's total; the last block to finish scans the range totals
    // into the ranges' prefixes (a tile's prefix is the two added) and
    // finishes the distribution
    __shared__ int last_s;
    __shared__ uint64_t btot_s;
    const int S = dist_scale(dists[0], dmax, 0, n_shared);
    const int64_t ntiles = (Nw + kTile - 1) / kTile;
    const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(r0 + per, ntiles);
    uint64_t local = 0;  // sum of the range's tiles so far (thread 0)
    // the next tile's weights are loaded while the current one is reduced
    auto load_tile = [&](int64_t tl, float* wv) {
      const int64_t u0 = tl * kTile, u1 = min(u0 + (int64_t)kTile, Nw);
      const int64_t e0 = u0 + (int64_t)threadIdx.x * kScanPer;
      if (e0 + kScanPer <= u1 && (reinterpret_cast<uintptr_t>(w + e0) & 15) == 0) {
#pragma unroll
        for (int h = 0; h < kScanPer / 4; ++h) {
          const float4 x = ld_weights4(reinterpret_cast<const float4*>(w + e0) + h);
          wv[4 * h] = x.x;
          wv[4 * h + 1] = x.y;
          wv[4 * h + 2] = x.z;
          wv[4 * h + 3] = x.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) wv[k] = e0 + k < u1 ? w[e0 + k] : 0.0f;
      }
    };
    float wnext[kScanPer];
    if (r0 < r1) load_tile(r0, wnext);
    for (int64_t tl = r0; tl < r1; ++tl) {
      const int64_t u0 = tl * kTile, u1 = min(u0 + (int64_t)kTile, Nw);
      const int64_t e0 = u0 + (int64_t)threadIdx.x * kScanPer;
      float wv[kScanPer];
#pragma unroll
      for (int k = 0; k < kScanPer; ++k) wv[k] = wnext[k];
      if (tl + 1 < r1) load_tile(tl + 1, wnext);
      uint64_t run = 0;
#pragma unroll
      for (int k = 0; k < kScanPer; ++k) {
        if (e0 + k < u1) {
          const uint32_t b = weight_bits(wv[k]);
          run += weight_bad(b) ? 0ull : quantize_bits(b, S);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) run += __shfl_xor_sync(0xffffffffu, run, o);
      if ((threadIdx.x & 31) == 0) wtot[threadIdx.x >> 5].s = run;
      __syncthreads();
      if (threadIdx.x == 0) {
        uint64_t sum = 0;
        for (int k = 0; k < kScanThreads / 32; ++k) sum += wtot[k].s;
        tile_prefix[tl] = local;
        local += sum;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      ts.sum[blockIdx.x] = local;  // the range's total
      __threadfence();
      last_s = atomicAdd(&ctr->scan_done, 1u) == (uint32_t)(gridDim.x - 1);
    }
    __syncthreads();
    if (!last_s) return;
    __threadfence();
    const int64_t nranges = gridDim.x;
    uint64_t carry = 0;
    for (int64_t c0 = 0; c0 < nranges; c0 += (int64_t)kScanThreads * kScanPer) {
      const int64_t b0 = c0 + (int64_t)threadIdx.x * kScanPer;
      uint64_t v[kScanPer], tsum = 0;
#pragma unroll
      for (int k = 0; k < kScanPer; ++k) {
        v[k] = b0 + k < nranges ? __ldcg(ts.sum + b0 + k) : 0ull;
        tsum += v[k];
      }
      uint64_t ex = carry + block_exclusive_u64(tsum, reinterpret_cast<uint64_t*>(wtot), &btot_s);
#pragma unroll
      for (int k = 0; k < kScanPer; ++k) {
        if (b0 + k < nranges) ts.first[b0 + k] = ex;  // prefix of range b0 + k
        ex += v[k];
      }
      carry += btot_s;
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      finish_dist(dists, 0, carry, S, status);
      ts.meta[0] = (uint32_t)per;  // tiles per range, for the forest pass
    }
    return;
  }

  // the thread's run of kScanPer consecutive weights, loaded before the
  // tile's distribution is looked up, so that the two latencies overlap
  const int64_t e0 = t0 + (int64_t)threadIdx.x * kScanPer;
  float wv[kScanPer];
  if (e0 + kScanPer <= t1 && (reinterpret_cast<uintptr_t>(w) & 15) == 0) {
#pragma unroll
    for (int h = 0; h < kScanPer / 4; ++h) {
      const float4 x = ld_weights4(reinterpret_cast<const float4*>(w + e0) + h);
      wv[4 * h] = x.x;
      wv[4 * h + 1] = x.y;
      wv[4 * h + 2] = x.z;
      wv[4 * h + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) wv[k] = e0 + k < t1 ? w[e0 + k] : 0.0f;
  }
  {
    // a tile inside one distribution (most tiles of a batch of large
    // distributions): only its total; a head can only be at t0 and an end
    // only at t1
    const int d0 = ts.dist0[tile];  // written by init_dists_kernel
    const rtf_dist& P = dists[d0];
    const int64_t pend = P.elem_off + P.n;
    if (P.elem_off <= t0 && t1 <= pend) {
      const int S = dist_scale(P, dmax, d0, n_shared);
      uint64_t run = 0;
#pragma unroll
      for (int k = 0; k < kScanPer; ++k) {
        const uint32_t b = weight_bits(wv[k]);
        if (e0 + k < t1 && !weight_bad(b)) run += quantize_bits(b, S);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) run += __shfl_xor_sync(0xffffffffu, run, o);
      if ((threadIdx.x & 31) == 0) wtot[threadIdx.x >> 5].s = run;
      __syncthreads();
      if (threadIdx.x == 0) {
        uint64_t tot = 0;
        for (int k = 0; k < kScanThreads / 32; ++k) tot += wtot[k].s;
        const bool head0 = P.elem_off == t0, ends = t1 == pend;
        ts.sum[tile] = tot;
        ts.meta[tile] = (head0 ? 3u : 0u) | (ends && !head0 ? 4u : 0u);
        if (ends && head0) finish_dist(dists, d0, tot, S, status);
        if (ends && !head0) ts.first[tile] = tot;
      }
      return;
    }
  }
  if (threadIdx.x == 0) {
    dfirst_s = ts.dist0[tile];
    meta_s = 0;
  }
  __syncthreads();
  const int dfirst = dfirst_s;

  uint64_t incl[kScanPer];
  int dk[kScanPer];
  uint32_t headmask = 0;
  uint32_t lastmask = 0;  // elements that end their distribution
  SegPair agg{0ull, 0u};
  {
    int d = dfirst;
    int64_t next = INT64_MAX;
    int64_t off = 0;
    int S = 0;
    if (e0 < t1) {
      if (SEG) {
        d = find_dist(dists, dfirst, min(Dw - 1, dfirst + kTile), e0);
        next = d + 1 < Dw ? dists[d + 1].elem_off : INT64_MAX;
      }
      const rtf_dist P = dists[d];
      off = P.elem_off;
      S = dist_scale(P, dmax, d, n_shared);
    }
    uint64_t run = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      const int64_t e = e0 + k;
      uint64_t q = 0;
      if (e < t1) {
        if (SEG && e >= next) {
          ++d;
          next = d + 1 < Dw ? dists[d + 1].elem_off : INT64_MAX;
          const rtf_dist P = dists[d];
          off = P.elem_off;
          S = dist_scale(P, dmax, d, n_shared);
        }
        if (off == e) {
          headmask |= 1u << k;
          run = 0;
        }
        const uint32_t b = weight_bits(wv[k]);
        q = weight_bad(b) ? 0ull : quantize_bits(b, S);
        if (e + 1 == min(next, Nw)) lastmask |= 1u << k;
      }
      run += q;
      incl[k] = run;
      dk[k] = d;
    }
    agg.s = run;
    agg.f = headmask ? 1u : 0u;
  }
  const SegPair ex = block_seg_exclusive(agg, wtot, &btot);
  const bool head0 = SEG ? (dists[dfirst].elem_off == t0) : (t0 == 0);

  // distributions whose last element lies in this tile
  if (lastmask) {
    const uint64_t base = ex.s;  // the tile's own partial sums (no incoming prefix)
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      const bool seen_head = (headmask & ((2u << k) - 1u)) != 0;
      const uint64_t v = seen_head ? incl[k] : base + incl[k];
      const int d = dk[k];
      if (lastmask & (1u << k)) {
        if (seen_head || ex.f) {
          const rtf_dist P = dists[d];  // began inside the tile: complete
          finish_dist(dists, d, v, dist_scale(P, dmax, d, n_shared), status);
        } else {
          ts.first[tile] = v;  // the tile's first piece: completed by the tile scan
          atomicOr(&meta_s, 4u);
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ts.sum[tile] = btot.s;
    ts.meta[tile] = meta_s | (btot.f ? 1u : 0u) | (head0 ? 2u : 0u);
  }
}

constexpr int kTileScanPer = kTileScanChunk / kScanThreads;

// Decoupled-lookback segmented scan of the tile sums (a distribution's head
// restarts the sum): the prefix of every tile's first piece, and the totals of
// the distributions that cross tiles.  In marginal mode the last block to
// finish also scans the row totals, the marginal's integer weights.
__global__ void __launch_bounds__(kScanThreads)
    tile_scan_kernel(TileSums ts, int64_t ntiles, rtf_dist* dists, int D, int Dw, int marginal,
                     int64_t n_shared, const uint32_t* dmax, uint64_t* chunk_status,
                     uint64_t* tile_prefix, Counters* ctr, uint32_t* status) {
  __shared__ uint32_t chunk_s;
  __shared__ SegPair wtot[kScanThreads / 32];
  __shared__ SegPair btot;
  __shared__ LookbackShared lb;
  __shared__ int last_s;
  if (threadIdx.x == 0) chunk_s = atomicAdd(&ctr->scan_ticket, 1u);
  __syncthreads();
  const int64_t chunk = chunk_s;
  const int64_t nchunks = (ntiles + kTileScanChunk - 1) / kTileScanChunk;
  const int64_t c0 = chunk * kTileScanChunk + (int64_t)threadIdx.x * kTileScanPer;

  uint64_t incl[kTileScanPer];
  uint32_t headmask = 0;
  uint64_t run = 0;
#pragma unroll
  for (int k = 0; k < kTileScanPer; ++k) {
    const int64_t t = c0 + k;
    incl[k] = run;  // exclusive value of tile t (since the last head before it)
    if (t < ntiles) {
      const uint64_t a = ts.sum[t];
      if (ts.meta[t] & 1u) {
        headmask |= 1u << k;  // the value passed on restarts at the tile's last head
        run = a;
      } else {
        run += a;
      }
    }
  }
  const SegPair agg{run, headmask ? 1u : 0u};
  const SegPair ex = block_seg_exclusive(agg, wtot, &btot);
  if (threadIdx.x == 0) {
    const uint64_t v = (btot.s & kValueMask) | (btot.f ? kFlagPrefix : kFlagAgg);
    st_release_u64(chunk_status + chunk, v);
  }
  // chunk 0 starts with the head at element 0, so its first tile needs no prefix
  uint64_t E = 0;
  if (chunk > 0) E = block_lookback(chunk_status, chunk, true, &lb, status);
  if (threadIdx.x == 0 && !btot.f)
    st_release_u64(chunk_status + chunk, ((E + btot.s) & kValueMask) | kFlagPrefix);
  const uint64_t base = ex.f ? ex.s : ex.s + E;
#pragma unroll
  for (int k = 0; k < kTileScanPer; ++k) {
    const int64_t t = c0 + k;
    if (t >= ntiles) break;
    // sum of the first piece's distribution before t0: the segmented
    // exclusive value of tile t (a head in tile t itself does not count)
    const bool seen_head = (headmask & ((1u << k) - 1u)) != 0;
    const uint64_t Et = seen_head ? incl[k] : base + incl[k];
    const uint32_t meta = ts.meta[t];
    const bool head0 = (meta & 2u) != 0;
    tile_prefix[t] = head0 ? 0ull : Et;
    if ((meta & 4u) && !head0) {
      const int d = ts.dist0[t];
      const rtf_dist P = dists[d];
      finish_dist(dists, d, Et + ts.first[t], dist_scale(P, dmax, d, n_shared), status);
    }
  }

  if (!marginal) return;
  // marginal mode: the last block to finish scans the row totals
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last_s = (atomicAdd(&ctr->scan_done, 1u) == (uint32_t)(nchunks - 1));
  __syncthreads();
  if (!last_s) return;
  __threadfence();
  const int H = D - 1;
  const int64_t moff = dists[D - 1].elem_off;  // == Nw
  uint64_t carry = 0;
  for (int r0 = 0; r0 < H; r0 += kScanThreads) {
    const int r = r0 + threadIdx.x;
    const uint64_t Tr = r < H ? __ldcg(&dists[r].total) : 0ull;
    const SegPair x{Tr, 0u};
    const SegPair px = block_seg_exclusive(x, wtot, &btot);
    const uint64_t excl = carry + px.s;  // sum of T over rows < r
    if (r < H) {
      const int64_t e = moff + r;
      if (e % kTile == 0) tile_prefix[e / kTile] = excl;
    }
    carry += btot.s;
    __syncthreads();
  }
  // the marginal's integers are in the units of the shared scale
  if (threadIdx.x == 0) finish_dist(dists, D - 1, carry, scale_from_max(dmax[0], n_shared), status);
}

// ---------------------------------------------------------------------------
// forest: the tree links of every node and leaf (Algorithm 1's result)
// ---------------------------------------------------------------------------
// Algorithm 1 (Sec. 3.2) grows ranges bottom-up: a range [lo, hi] becomes the
// child of the split at lo (child 1) or at hi + 1 (child 0), whichever of the
// bounding distances delta_{lo-1}, delta_hi is smaller (equal distances go to
// child 1), and the first of two siblings to arrive stops.  The tree this
// yields is fixed by the distances alone: the node of split k (between leaves
// k - 1 and k, node index k, Sec. 3.1) covers the leaves from the nearest
// split on its left with a larger distance to the nearest split on its right
// with a distance at least as large (ties go right, as the strict comparison
// sends equal distances to child 1); among those two bounding splits its
// parent is the one with the smaller distance (the right one's when the left
// is larger), and it is that parent's child 0 when the parent lies on its
// right.  A leaf is the one-leaf range between its two neighbouring splits.
// So every node and every leaf finds its parent from the two nearest larger
// distances around it, without climbing and without atomics; every child slot
// has exactly one writer.  Inside a tile the nearest larger distances are
// found with warp ballots over the bit planes of the tile's distances; a node
// whose bounding splits lie outside the tile (its range crosses a tile edge)
// is left to the merge pass, which searches the global distance array.
constexpr int kForestPer = kTile / kForestThreads;  // 4
static_assert(kForestPer == 4, "the distance write-out stores one u32 per thread");
constexpr int32_t kUnset = 0x7FFFFFFF;
constexpr int kChunks = (kTile + 1 + 31) / 32;      // 32-split chunks of positions 0..tn
constexpr uint32_t kDeltaTop = 33;                  // kDeltaInf in 6 bits (above any 0..32)

template <bool SEG>
struct ForestShared {
  alignas(16) uint64_t C[kTile + 2];  // C_{t0-1} .. C_{t1}
  alignas(16) uint64_t K[kTile + 2];  // K_{t0-1} .. K_{t1}
  alignas(16) int32_t child[kTile][2];
  int32_t dist[SEG ? kTile : 1];
  // d[p]: distance of the split at tile position p, between leaves p - 1 and
  // p (p = 0: delta_{t0-1}; p = tn: delta_{t1-1})
  uint8_t d[kChunks * 32];
  uint32_t plane[kChunks][6];  // bit b of min(d, 33) for the 32 positions of a chunk
  uint32_t valid[kChunks];     // positions <= tn
  uint32_t cmax[kChunks];      // largest min(d, 33) of the chunk's valid positions
  SegPair wtot[kForestThreads / 32];
  SegPair btot;
  uint32_t tmax;
  int dfirst;
  int dprev;
  int nunres;
  int ncells;
  float wprev;
  uint64_t prefix;
  rtf_dist P0;  // parameters of the tile's first distribution
  int32_t unres[kUnresCap];
  uint32_t cell_range[kTile];  // cells complete inside the tile: first | last << 16
};

struct ForestArgs {
  const float* w;
  int64_t N, Nw;
  const rtf_dist* dists;
  int D, Dw;
  int64_t n_shared;
  rtf_node* nodes;
  int32_t* guide;
  rtf_guide_rec* guide_recs;
  int4* fills;
  uint32_t* fill_count;
  int64_t fill_cap;
  const uint64_t* tile_prefix;
  const uint64_t* range_prefix;  // one distribution: prefix of each range of tiles
  const uint32_t* range_meta;    // [0]: tiles per range
  const uint32_t* dmax;
  uint8_t* delta;
  uint8_t* tmax;
  uint32_t* gmax;
  int32_t* unres;
  int32_t* unres_count;
  const int32_t* tile_dist0;  // distribution of each tile's first element (batches)
  uint32_t* status;
};

// Key of C_j for distribution P.
__device__ __forceinline__ uint64_t key_for(const rtf_dist& P, uint64_t C) {
  return key_of(C, P.total, P.recip, P.shift);
}

// Root of a finished cell [lo, hi] (global element indices) of distribution P
// (index d): guide entry and guide record of the cell, and of the cells after
// it that no key falls into.  K_lo / K_hi are the keys of leaves lo and hi,
// Knext that of leaf hi + 1 (2^32 after the distribution's last leaf);
// C_{lo-1} (0 when lo is the first leaf of the distribution), C_lo, C_hi and
// C_{hi+1} (T after the last leaf) their CDF bounds.  Interval hi covers every
// cell from c + 1 up to the cell of Knext (the guide entry ~hi of the Cutpoint
// method, Sec. 3.2, for a cell overlapped by one interval only); runs longer
// than kFillInline cells are listed for the fill pass.
__device__ __forceinline__ void finish_cell(const ForestArgs& a, const rtf_dist& P, int d,
                                            int64_t lo, int64_t hi, uint64_t Klo, uint64_t Khi,
                                            uint64_t Clm1, uint64_t Clo, uint64_t Chi,
                                            uint64_t Chp1, int32_t top, uint64_t Knext) {
  const uint64_t M = 1ull << P.m;
  uint64_t c = cell_of(Klo, P.m);
  if (c >= M) return;  // unreachable trailing cell of zero-width bins
  int32_t lo_l = (int32_t)(lo - P.elem_off), hi_l = (int32_t)(hi - P.elem_off);
  uint64_t start = c << (32 - P.m);
  const int64_t gi = P.guide_off + (int64_t)c;
  rtf_guide_rec rec;
  rec.hi = Chp1;
  if (Khi == start) {
    // one interval covers the whole cell (all its keys equal the cell start)
    a.guide[gi] = ~hi_l;
    rec.cdf = Chi;
    rec.child[0] = ~hi_l;
    rec.child[1] = ~hi_l;
    rec.lo = Chi;
  } else {
    a.guide[gi] = lo_l;
    rec.cdf = Clo;
    rec.child[0] = ~(lo_l > 0 ? lo_l - 1 : 0);
    rec.child[1] = top;
    rec.lo = Clm1;
  }
  a.guide_recs[gi] = rec;
  const uint64_t cn = min(cell_of(Knext, P.m), M);
  if (cn <= c + 1) return;
  const int64_t first = (int64_t)c + 1, count = (int64_t)cn - first;
  if (count <= kFillInline) {
    rtf_guide_rec cov;
    cov.cdf = Chi;
    cov.child[0] = ~hi_l;
    cov.child[1] = ~hi_l;
    cov.lo = Chi;
    cov.hi = Chp1;
    for (int64_t g = first; g < (int64_t)cn; ++g) {
      a.guide[P.guide_off + g] = ~hi_l;
      a.guide_recs[P.guide_off + g] = cov;
    }
    return;
  }
  const int64_t pieces = (count + kFillPiece - 1) / kFillPiece;
  const int64_t slot = atomicAdd(a.fill_count, (uint32_t)pieces);
  for (int64_t k = 0; k < pieces; ++k) {
    if (slot + k >= a.fill_cap) {
      raise_status(a.status, RTF_STATUS_INVARIANT);
      break;
    }
    a.fills[slot + k] = make_int4((int)(P.guide_off + first + k * kFillPiece),
                                  (int)min(kFillPiece, count - k * kFillPiece), hi_l, d);
  }
}

// Lanes of a 32-position chunk whose value (bit planes pl[0..5]) exceeds v
// (*gt) and equals it (*eq, within `valid`).
__device__ __forceinline__ void compare_planes(const uint32_t* pl, uint32_t v, uint32_t valid,
                                               uint32_t* gt, uint32_t* eq) {
  uint32_t g = 0u, e = valid;
#pragma unroll
  for (int b = 5; b >= 0; --b) {
    const uint32_t p = pl[b];
    if ((v >> b) & 1u) {
      e &= p;
    } else {
      g |= e & p;
      e &= ~p;
    }
  }
  *gt = g;
  *eq = e;
}

// Minimum resident forest blocks per SM given to the register allocator.
#ifndef RTF_FOREST_MINB
#define RTF_FOREST_MINB 3
#endif

struct LeanShared;
template <bool ONE>
__device__ __forceinline__ void lean_tile(const ForestArgs& a, LeanShared& s, const rtf_dist& P,
                                          int dd);

template <bool SEG>
__global__ void __launch_bounds__(kForestThreads, RTF_FOREST_MINB) forest_kernel(ForestArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ForestShared<SEG>& s = *reinterpret_cast<ForestShared<SEG>*>(smem_raw);
  const int64_t tile = blockIdx.x;
  const int64_t t0 = tile * kTile, t1 = min(t0 + (int64_t)kTile, a.N);
  if (SEG) {
    // a tile inside one distribution (most tiles of a batch of large
    // distributions) takes the one-distribution path
    const int df = a.tile_dist0[tile];
    const rtf_dist& P = a.dists[df];
    if ((P.flags & kDistMarginal) == 0 && P.elem_off <= t0 && t1 <= P.elem_off + P.n) {
      lean_tile<false>(a, *reinterpret_cast<LeanShared*>(smem_raw), P, df);
      return;
    }
  }
  const int tn = (int)(t1 - t0);
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;

  if (tid == 0) {
    const int df = SEG ? a.tile_dist0[tile] : 0;
    s.dfirst = df;
    s.dprev = (t0 > 0 && SEG) ? (a.dists[df].elem_off == t0 ? df - 1 : df) : df;
    s.nunres = 0;
    s.ncells = 0;
    s.tmax = 0;
    s.P0 = a.dists[df];
    s.prefix = t0 > 0 ? a.tile_prefix[tile] : 0ull;
    s.wprev = (t0 > 0 && t0 - 1 < a.Nw) ? a.w[t0 - 1] : 0.0f;
  }
  // the thread's four weights, straight from global memory (16-byte vectors
  // where aligned); the passes before this one left them in L2
  const int l0 = tid * kForestPer;  // tile-local index of the thread's first leaf
  const int64_t e0 = t0 + l0;
  float wv[kForestPer];
  if (e0 + kForestPer <= a.Nw && e0 + kForestPer <= t1 &&
      (reinterpret_cast<uintptr_t>(a.w + e0) & 15) == 0) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(a.w + e0));
    wv[0] = x.x;
    wv[1] = x.y;
    wv[2] = x.z;
    wv[3] = x.w;
  } else {
#pragma unroll
    for (int k = 0; k < kForestPer; ++k)
      wv[k] = (e0 + k < t1 && e0 + k < a.Nw) ? a.w[e0 + k] : 0.0f;
  }
  __syncthreads();
  const int dfirst = s.dfirst;

  // ---- q, C and keys of the thread's leaves ---------------------------------
  // Each thread owns kForestPer consecutive leaves; the parameters of the
  // distribution it is in stay in registers (reloaded only at a boundary).
  uint64_t q[kForestPer], incl[kForestPer];
  int dk[kForestPer];
  uint32_t headmask = 0;
  {
    int dcur = dfirst;
    int64_t next = INT64_MAX;
    int S = 0;
    int32_t flags = 0;
    int64_t off = 0;
    if (l0 < tn) {
      if (SEG) {
        dcur = find_dist(a.dists, dfirst, min(a.D - 1, dfirst + kTile), e0);
        next = dcur + 1 < a.D ? a.dists[dcur + 1].elem_off : INT64_MAX;
        const rtf_dist P = a.dists[dcur];
        flags = P.flags;
        off = P.elem_off;
        S = P.scale;
      } else {
        flags = s.P0.flags;
        off = s.P0.elem_off;
        S = s.P0.scale;
      }
    }
    uint64_t run = 0;
#pragma unroll
    for (int k = 0; k < kForestPer; ++k) {
      const int64_t e = e0 + k;
      uint64_t qq = 0;
      if (l0 + k < tn) {
        if (SEG && e >= next) {
          ++dcur;
          next = dcur + 1 < a.D ? a.dists[dcur + 1].elem_off : INT64_MAX;
          const rtf_dist P = a.dists[dcur];
          flags = P.flags;
          off = P.elem_off;
          S = P.scale;
        }
        if (off == e) {
          headmask |= 1u << k;
          run = 0;
        }
        if (SEG && (flags & kDistMarginal)) {
          qq = __ldcg(&a.dists[e - off].total);
        } else {
          const uint32_t b = weight_bits(wv[k]);
          qq = weight_bad(b) ? 0ull : quantize_bits(b, S);
        }
        if (SEG) s.dist[l0 + k] = dcur;
      }
      dk[k] = dcur;
      q[k] = qq;
      run += qq;
      incl[k] = run;
    }
    // exclusive prefix of the thread's run within the tile; one distribution
    // has its only head at element 0, where the running sum is 0 anyway, so a
    // plain scan serves
    uint64_t base;
    if (SEG) {
      const SegPair ex = block_seg_exclusive(SegPair{run, headmask ? 1u : 0u}, s.wtot, &s.btot);
      const bool head0 = a.dists[dfirst].elem_off == t0;
      const uint64_t E = head0 ? 0ull : s.prefix;
      base = ex.f ? ex.s : ex.s + E;
    } else {
      base = block_exclusive_u64(run, reinterpret_cast<uint64_t*>(s.wtot), &s.btot.s) +
             (t0 == 0 ? 0ull : s.prefix);
      headmask = 0u;
    }
    int dP = -1;
    uint64_t T = 0, R = 0;
    int z = 0;
#pragma unroll
    for (int k = 0; k < kForestPer; ++k) {
      const int l = l0 + k;
      if (l >= tn) break;
      if (dk[k] != dP) {
        dP = dk[k];
        const rtf_dist& P = SEG ? a.dists[dP] : s.P0;
        T = P.total;
        R = P.recip;
        z = P.shift;
      }
      const bool seen_head = (headmask & ((2u << k) - 1u)) != 0;
      const uint64_t inc = seen_head ? incl[k] : base + incl[k];
      const uint64_t C = inc - q[k];
      s.C[l + 1] = C;
      s.K[l + 1] = key_of(C, T, R, z);
      if (l == tn - 1) {
        s.C[tn + 1] = inc;  // C_{t1} within the distribution of t1-1
        s.K[tn + 1] = key_of(inc, T, R, z);
      }
      s.child[l][0] = kUnset;
      s.child[l][1] = kUnset;
    }
  }
  // C_{t0-1} and its key (only meaningful when t0-1 belongs to the same distribution)
  if (tid == 0) {
    s.C[0] = 0;
    s.K[0] = 0;
    if (t0 > 0 && s.dprev == dfirst) {
      const rtf_dist& P = s.P0;
      uint64_t qp;
      if (SEG && (P.flags & kDistMarginal)) {
        qp = __ldcg(&a.dists[t0 - 1 - P.elem_off].total);
      } else {
        const uint32_t b = weight_bits(s.wprev);
        qp = weight_bad(b) ? 0ull : quantize_bits(b, P.scale);
      }
      const uint64_t Cp = s.prefix - qp;  // C_{t0} is the tile prefix
      s.C[0] = Cp;
      s.K[0] = key_for(P, Cp);
    }
  }
  __syncthreads();
  // distances: delta_j for the thread's leaves j (position l + 1), delta_{t0-1}
  // (position 0) by thread 0; the tile's largest distance
  {
    int dP = -1;
    int m = 0;
    int64_t end = 0;
    uint32_t packed = 0, dmx = 0;
#pragma unroll
    for (int k = 0; k < kForestPer; ++k) {
      const int l = l0 + k;
      uint32_t dlt = kDeltaInf;
      if (l < tn) {
        if (dk[k] != dP) {
          dP = dk[k];
          const rtf_dist& P = SEG ? a.dists[dP] : s.P0;
          m = P.m;
          end = P.elem_off + P.n;
        }
        if (t0 + l + 1 < end) {
          const uint64_t Ka = s.K[l + 1], Kb = s.K[l + 2];
          if (cell_of(Ka, m) == cell_of(Kb, m)) dlt = key_distance(Ka, Kb);
        }
        s.d[l + 1] = (uint8_t)dlt;
        dmx = max(dmx, dlt);
      }
      packed |= dlt << (8 * k);
    }
    if (l0 + kForestPer <= tn) {
      *reinterpret_cast<uint32_t*>(a.delta + e0) = packed;
    } else {
      for (int k = 0; k < kForestPer && l0 + k < tn; ++k)
        a.delta[e0 + k] = (uint8_t)(packed >> (8 * k));
    }
    dmx = __reduce_max_sync(0xffffffffu, dmx);
    if (lane == 0 && dmx) atomicMax(&s.tmax, dmx);
    if (tid == 0) {
      uint32_t d0 = kDeltaInf;
      if (t0 > 0 && s.dprev == dfirst) {
        const int mm = s.P0.m;
        const uint64_t Ka = s.K[0], Kb = s.K[1];
        if (cell_of(Ka, mm) == cell_of(Kb, mm)) d0 = key_distance(Ka, Kb);
      }
      s.d[0] = (uint8_t)d0;
    }
  }
  __syncthreads();

  // ---- bit planes of the distances, per chunk of 32 positions ---------------
  const int nchunks = (tn + 1 + 31) >> 5;
  for (int c = warp; c < nchunks; c += kForestThreads / 32) {
    const int p = 32 * c + lane;
    const bool ok = p <= tn;
    const uint32_t v = ok ? min((uint32_t)s.d[p], kDeltaTop) : 0u;
    const uint32_t vm = __ballot_sync(0xffffffffu, ok);
    uint32_t mine = 0u;
#pragma unroll
    for (int b = 0; b < 6; ++b) {
      const uint32_t pb = __ballot_sync(0xffffffffu, (v >> b) & 1u);
      if (lane == b) mine = pb;
    }
    const uint32_t mx = __reduce_max_sync(0xffffffffu, v);
    if (lane < 6) s.plane[c][lane] = mine;
    if (lane == 0) {
      s.valid[c] = vm;
      s.cmax[c] = mx;
    }
  }
  if (tid == 0) {
    a.tmax[tile] = (uint8_t)s.tmax;
    if (s.tmax) atomicMax(a.gmax + tile / kTileGroup, s.tmax);
  }
  __syncthreads();

  // ---- links: node and leaf at every position p in [0, tn) -------------------
  for (int c = warp; c < nchunks; c += kForestThreads / 32) {
    const int p = 32 * c + lane;
    if (p >= tn) continue;
    const int dd = SEG ? s.dist[p] : 0;
    const rtf_dist& P = SEG ? a.dists[dd] : s.P0;
    const int32_t base_id = (int32_t)(t0 - P.elem_off);
    const uint32_t v = s.d[p];

    // leaf p, between the splits at positions p and p + 1
    {
      const uint32_t dl = v, dr = s.d[p + 1];
      const int32_t id = base_id + p;
      if (dl >= kDeltaInf) s.child[p][0] = ~(id > 0 ? id - 1 : 0);  // p starts a cell
      if (dl >= kDeltaInf && dr >= kDeltaInf) {
        // a cell of one leaf: the leaf is its root's tree
        s.child[p][1] = ~id;
        s.cell_range[atomicAdd(&s.ncells, 1)] = (uint32_t)p | ((uint32_t)p << 16);
      } else if (dl > dr) {
        if (p + 1 < tn)
          s.child[p + 1][0] = ~id;
        else
          a.nodes[t1].child[0] = ~id;
      } else {
        s.child[p][1] = ~id;
      }
    }

    // node p (the split at position p), unless p is a cell boundary
    if (v >= kDeltaInf) continue;
    uint32_t gt, eq;
    compare_planes(s.plane[c], v, s.valid[c], &gt, &eq);
    // nearest position left of p with a larger distance
    int pl = -1;
    {
      const uint32_t m = gt & ((1u << lane) - 1u);
      if (m) {
        pl = 32 * c + 31 - __clz(m);
      } else {
        for (int c2 = c - 1; c2 >= 0; --c2) {
          if (s.cmax[c2] > v) {
            uint32_t g2, e2;
            compare_planes(s.plane[c2], v, s.valid[c2], &g2, &e2);
            pl = 32 * c2 + 31 - __clz(g2);
            break;
          }
        }
      }
    }
    // nearest position right of p with a distance at least as large
    int pr = -1;
    {
      const uint32_t m = (gt | eq) & ~((2u << lane) - 1u);
      if (lane < 31 && m) {
        pr = 32 * c + __ffs(m) - 1;
      } else {
        for (int c2 = c + 1; c2 < nchunks; ++c2) {
          if (s.cmax[c2] >= v) {
            uint32_t g2, e2;
            compare_planes(s.plane[c2], v, s.valid[c2], &g2, &e2);
            pr = 32 * c2 + __ffs(g2 | e2) - 1;
            break;
          }
        }
      }
    }
    const int32_t id = base_id + p;
    if (pr < 0 || (pl < 0 && s.d[pr] > v)) {
      // the parent depends on distances outside the tile
      const int slot = atomicAdd(&s.nunres, 1);
      if (slot < kUnresCap) s.unres[slot] = p;
      continue;
    }
    const uint32_t dr = s.d[pr];
    const uint32_t dl = pl >= 0 ? s.d[pl] : kDeltaInf + 1;  // unknown, larger than v = dr
    if (dl >= kDeltaInf && dr >= kDeltaInf && pl >= 0) {
      // the top of a cell inside the tile: leaves [pl, pr - 1], root at pl
      s.child[pl][1] = id;
      s.cell_range[atomicAdd(&s.ncells, 1)] = (uint32_t)pl | ((uint32_t)(pr - 1) << 16);
    } else if (dl > dr) {
      if (pr < tn)
        s.child[pr][0] = id;
      else
        a.nodes[t1].child[0] = id;
    } else {
      s.child[pl][1] = id;
    }
  }
  __syncthreads();

  // ---- guide entries of the cells completed inside the tile -----------------
  // (by consecutive threads, after the links: done inside the links, a cell's
  // entries stalled every lane of its warp)
  for (int i = tid; i < s.ncells; i += kForestThreads) {
    const uint32_t r = s.cell_range[i];
    const int lo = (int)(r & 0xFFFFu), hi = (int)(r >> 16);
    const int dd = SEG ? s.dist[lo] : 0;
    const rtf_dist& P = SEG ? a.dists[dd] : s.P0;
    const int64_t end = P.elem_off + P.n;
    const int64_t glo = t0 + lo;
    const uint64_t Clm1 = glo > P.elem_off ? s.C[lo] : 0ull;
    const uint64_t Chp1 = t0 + hi + 1 == end ? P.total : s.C[hi + 2];
    const uint64_t Knext = t0 + hi + 1 == end ? (1ull << 32) : s.K[hi + 2];
    finish_cell(a, P, dd, glo, t0 + hi, s.K[lo + 1], s.K[hi + 1], Clm1, s.C[lo + 1], s.C[hi + 1],
                Chp1, s.child[lo][1], Knext);
  }

  // ---- node records -----------------------------------------------------------
  // Consecutive threads on consecutive records (leaf l = tid + k * blockDim); a
  // child slot written by another tile or by the merge pass is left alone.
#pragma unroll
  for (int k = 0; k < kForestPer; ++k) {
    const int l = tid + k * kForestThreads;
    if (l >= tn) break;
    const int32_t c0 = s.child[l][0], c1 = s.child[l][1];
    const uint64_t C = s.C[l + 1];
    rtf_node* rec = a.nodes + t0 + l;
    if (c0 != kUnset && c1 != kUnset) {
      rtf_node r;
      r.cdf = C;
      r.child[0] = c0;
      r.child[1] = c1;
      *rec = r;
    } else {
      rec->cdf = C;
      if (c0 != kUnset) rec->child[0] = c0;
      if (c1 != kUnset) rec->child[1] = c1;
    }
  }
  const int nu = s.nunres;
  if (tid == 0) {
    if (nu > kUnresCap) raise_status(a.status, RTF_STATUS_INVARIANT);
    a.unres_count[tile] = min(nu, kUnresCap);
  }
  if (tid < min(nu, kUnresCap)) a.unres[tile * kUnresCap + tid] = (int32_t)(t0 + s.unres[tid]);
}

// ---------------------------------------------------------------------------
// forest of a tile inside one distribution
// ---------------------------------------------------------------------------
// The same links as forest_kernel, for a tile whose leaves all belong to one
// distribution (every tile of a one-distribution build, most tiles of a
// batch).  Warp w owns the 128 consecutive leaves [128 w, 128 w + 128) of the
// tile.  The weights, the prefix sums, the keys and the distances are blocked:
// thread i holds leaves 4 i .. 4 i + 3 (one 16-byte load of weights, one warp
// scan of the thread totals and one block-wide combine, one 4-byte store of
// distances).  The masks, the links and the records are lane-strided: lane l
// holds leaves 128 w + 32 k + l (k = 0..3), so that the ballots of one k are
// the bit planes of 32 consecutive split positions and each k writes 32
// consecutive records.  Chunk c = 4 w + k holds positions 32 c + 1 .. 32 c + 32,
// the right-hand splits of the chunk's leaves; position 0 (delta_{t0-1}) lies
// in no chunk.
struct LeanShared {
  // C_{t0-1} .. C_{t1} at Cbuf[1 .. tn + 2] (the CDF of tile-local leaf l at
  // index l + 2, so that each thread's four values form two aligned 16-byte
  // stores); read through C = Cbuf + 1
  alignas(16) uint64_t Cbuf[kTile + 4];
  alignas(16) int32_t child[kTile][2];
  uint32_t cell_range[kTile];         // cells complete inside the tile: first | last << 16
  // distance at position p at dbuf[p + 3] (each thread's four distances form
  // one aligned 4-byte store); read through d = dbuf + 3
  alignas(4) uint8_t dbuf[kTile + 12];
  // per chunk: gtm[c][t] = positions with a distance > t (t = 0..31; above
  // the chunk's largest finite distance only the boundaries, infm[c])
  uint32_t gtm[kChunks][32];
  uint32_t valid[kChunks];
  uint32_t infm[kChunks];
  uint32_t cmax[kChunks];
  uint64_t wtot[kForestThreads / 32];
  uint64_t Kfirst[kForestThreads / 32 + 1];  // key of each warp's first leaf; [16]: of leaf t1
  uint64_t prefix;
  uint64_t Kprev;  // key of leaf t0 - 1
  uint32_t tmax;
  int nunres;
  int ncells;
  int32_t unres[kUnresCap];
};

static_assert(sizeof(LeanShared) <= sizeof(ForestShared<true>),
              "the batched forest kernel's shared memory holds the one-distribution tile");

// 64-bit warp shuffles
__device__ __forceinline__ uint64_t shfl_up64(uint64_t x, int d) {
  return __shfl_up_sync(0xffffffffu, (unsigned long long)x, d);
}
__device__ __forceinline__ uint64_t shfl_down64(uint64_t x, int d) {
  return __shfl_down_sync(0xffffffffu, (unsigned long long)x, d);
}
__device__ __forceinline__ uint64_t shfl_idx64(uint64_t x, int l) {
  return __shfl_sync(0xffffffffu, (unsigned long long)x, l);
}

// Positions of chunk c with a distance > v (v below kDeltaInf).
__device__ __forceinline__ uint32_t chunk_gt(const LeanShared& s, int c, uint32_t v) {
  return v < 32 ? s.gtm[c][v] : s.infm[c];
}

// ... with a distance >= v.
__device__ __forceinline__ uint32_t chunk_ge(const LeanShared& s, int c, uint32_t v) {
  return v == 0 ? s.valid[c] : chunk_gt(s, c, v - 1);
}

// Search of chunks c2 = from, from - 1, ... (dir -1, nearest position with a
// distance > v) or from, from + 1, ... below nchunks (dir +1, nearest with a
// distance >= v); -1 when no chunk holds one.
__device__ __forceinline__ int lean_walk(const LeanShared& s, int from, int nchunks, uint32_t v,
                                         int dir) {
  for (int c2 = from; c2 >= 0 && c2 < nchunks; c2 += dir) {
    if (dir < 0 ? s.cmax[c2] > v : s.cmax[c2] >= v) {
      return dir < 0 ? 32 * c2 + 1 + (31 - __clz(chunk_gt(s, c2, v)))
                     : 32 * c2 + __ffs(chunk_ge(s, c2, v));
    }
  }
  return -1;
}

// One tile inside one distribution P (index dd, not the marginal of a 2-D
// map).  ONE: the build of a single distribution (P = dists[0] over the whole
// array; the tile sums came in ranges); otherwise a tile of a batch, whose
// prefix within P is in tile_prefix.
template <bool ONE>
__device__ __forceinline__ void lean_tile(const ForestArgs& a, LeanShared& s, const rtf_dist& P,
                                          int dd) {
  uint64_t* const sC = s.Cbuf + 1;  // sC[p]: C of tile-local leaf p - 1
  uint8_t* const sd = s.dbuf + 3;   // sd[p]: distance at position p
  const int64_t tile = blockIdx.x;
  const int64_t t0 = tile * kTile, t1 = min(t0 + (int64_t)kTile, a.N);
  const int tn = (int)(t1 - t0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int S = P.scale;
  const int64_t eoff = ONE ? 0 : P.elem_off, eend = ONE ? a.N : P.elem_off + P.n;
  const int lbase = 128 * warp + lane;  // lane-strided: tile-local leaf of k = 0
  const int lb = 4 * tid;               // blocked: the thread's leaves lb .. lb + 3

  // ---- weights, quantisation, prefix sums (blocked: four consecutive leaves
  // per thread, one 16-byte load, one warp scan of the thread totals) --------
  float wv[4];
  if (lb + 4 <= tn && (reinterpret_cast<uintptr_t>(a.w) & 15) == 0) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(a.w + t0) + tid);
    wv[0] = x.x;
    wv[1] = x.y;
    wv[2] = x.z;
    wv[3] = x.w;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) wv[k] = lb + k < tn ? __ldg(a.w + t0 + lb + k) : 0.0f;
  }
  if (tid == 0) {
    s.nunres = 0;
    s.ncells = 0;
    s.tmax = 0;
    // the tile's prefix within its range of the tile sums plus the range's prefix
    s.prefix = !ONE ? a.tile_prefix[tile]
               : t0 > 0 ? a.tile_prefix[tile] + a.range_prefix[tile / a.range_meta[0]]
                        : 0ull;
  }
  uint64_t C[4];
  uint64_t tot = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t b = weight_bits(wv[k]);
    C[k] = tot;  // exclusive within the thread
    tot += (lb + k < tn && !weight_bad(b)) ? quantize_bits(b, S) : 0ull;
  }
  uint64_t incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = shfl_up64(incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s.wtot[warp] = incl;
  __syncthreads();
  // the warp's offset in the tile, the tile's prefix, C_{t0-1} and C_{t1}
  uint64_t off = lane < warp ? s.wtot[lane] : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, (unsigned long long)off, o);
  const uint64_t pre = s.prefix + off + (incl - tot);
  const uint64_t T = P.total, R = P.recip;
  const int z = P.shift, m = P.m;
  uint64_t K[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    C[k] += pre;
    K[k] = key_of(C[k], T, R, z);
  }
  if (lb + 4 <= tn) {
    ulonglong2* cv = reinterpret_cast<ulonglong2*>(sC + lb + 1);
    cv[0] = make_ulonglong2(C[0], C[1]);
    cv[1] = make_ulonglong2(C[2], C[3]);
    int4* ch = reinterpret_cast<int4*>(&s.child[lb][0]);
    ch[0] = make_int4(kUnset, kUnset, kUnset, kUnset);
    ch[1] = make_int4(kUnset, kUnset, kUnset, kUnset);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (lb + k < tn) {
        sC[lb + k + 1] = C[k];
        s.child[lb + k][0] = kUnset;
        s.child[lb + k][1] = kUnset;
      }
    }
  }
  if (ONE && lane == 0) s.Kfirst[warp] = K[0];
  if (tid == 0) {
    uint64_t tt = 0;
    for (int k = 0; k < kForestThreads / 32; ++k) tt += s.wtot[k];
    const uint64_t Ct1 = s.prefix + tt;
    sC[tn + 1] = Ct1;
    if (ONE) s.Kfirst[kForestThreads / 32] = key_of(Ct1, T, R, z);
    uint64_t Cp = 0;
    if (t0 > eoff) {
      const uint32_t b = weight_bits(a.w[t0 - 1]);
      Cp = s.prefix - (weight_bad(b) ? 0ull : quantize_bits(b, S));
    }
    sC[0] = Cp;
    s.Kprev = key_of(Cp, T, R, z);
  }
  // The key of leaf lb + 4 is the next lane's first key; for lane 31 it is the
  // next warp's first key, passed through shared memory across a barrier
  // (ONE), or, in a tile of a batch, the key of the thread's own running sum
  // past its four leaves (the C of the next warp's first leaf, C_{t1} for the
  // last warp), which saves the barrier (measured: faster for the batches,
  // whose tiles hold more cells; slower for one distribution, where the kept
  // sums spill under the three-block register cap).
  if (ONE) __syncthreads();

  // ---- distances (blocked: positions lb + 1 .. lb + 4, one 4-byte store) ----
  uint32_t dmx = 0;
  {
    uint64_t K4 = shfl_down64(K[0], 1);
    if (lane == 31) K4 = ONE ? s.Kfirst[warp + 1] : key_of(pre + tot, T, R, z);
    uint32_t packed = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int l = lb + k;
      const uint64_t Kn = k < 3 ? K[k < 3 ? k + 1 : k] : K4;
      uint32_t dlt = kDeltaInf;
      if (l < tn && t0 + l + 1 < eend && cell_of(K[k], m) == cell_of(Kn, m))
        dlt = key_distance(K[k], Kn);
      if (l < tn) {
        packed |= dlt << (8 * k);
        dmx = max(dmx, dlt);  // the boundaries included: the merge pass searches for them
      }
    }
    *reinterpret_cast<uint32_t*>(sd + lb + 1) = packed;
    if (lb + 4 <= tn) {
      *reinterpret_cast<uint32_t*>(a.delta + t0 + lb) = packed;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (lb + k < tn) a.delta[t0 + lb + k] = (uint8_t)(packed >> (8 * k));
    }
  }
  dmx = __reduce_max_sync(0xffffffffu, dmx);
  if (lane == 0 && dmx) atomicMax(&s.tmax, dmx);
  // the warp's chunks 4 warp .. 4 warp + 3 hold exactly its own 128 positions
  __syncwarp();

  // ---- threshold masks of the chunks (lane-strided: lane = position - 1 - 32 c)
  // from the six bit planes of min(d, 33): lane t compares every position
  // with t, bit plane by bit plane (t < 32, so its bit 5 is 0)
  uint32_t lt_mask[5];  // all ones where bit b of this lane's t is set
#pragma unroll
  for (int b = 0; b < 5; ++b) lt_mask[b] = ((lane >> b) & 1) ? 0xffffffffu : 0u;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int l = lbase + 32 * k;
    const int c = 4 * warp + k;
    const uint32_t dlt = l < tn ? sd[l + 1] : 0u;
    const uint32_t v = l < tn ? min(dlt, kDeltaTop) : 0u;
    const uint32_t vm = __ballot_sync(0xffffffffu, l < tn);
    const uint32_t inf = __ballot_sync(0xffffffffu, l < tn && dlt >= kDeltaInf);
    const int fm = (int)__reduce_max_sync(0xffffffffu, (l < tn && dlt < kDeltaInf) ? dlt + 1 : 0u) - 1;
    uint32_t g = inf;  // no finite distance: only the boundaries exceed any t
    if (fm >= 0) {
      uint32_t pl[6];
#pragma unroll
      for (int b = 0; b < 6; ++b) pl[b] = __ballot_sync(0xffffffffu, (v >> b) & 1u);
      uint32_t e = vm & ~pl[5];
      g = pl[5];
#pragma unroll
      for (int b = 4; b >= 0; --b) {
        g |= e & pl[b] & ~lt_mask[b];
        e &= ~(pl[b] ^ lt_mask[b]);
      }
    }
    s.gtm[c][lane] = g;
    if (lane == 0) {
      s.valid[c] = vm;
      s.infm[c] = inf;
      s.cmax[c] = inf ? kDeltaTop : (uint32_t)max(fm, 0);
    }
  }
  if (tid == 0) {
    uint32_t d0 = kDeltaInf;
    if (t0 > eoff && cell_of(s.Kprev, m) == cell_of(K[0], m)) d0 = key_distance(s.Kprev, K[0]);
    sd[0] = (uint8_t)d0;
  }
  const int nchunks = (tn + 31) >> 5;
  __syncthreads();
  if (tid == 0) {
    a.tmax[tile] = (uint8_t)s.tmax;
    if (s.tmax) atomicMax(a.gmax + tile / kTileGroup, s.tmax);
  }

  // ---- links -----------------------------------------------------------------
  // node at position 0 (delta_{t0-1}): its left bound lies outside the tile
  if (tid == 0) {
    const uint32_t v = sd[0];
    if (v < kDeltaInf) {
      const int pr = lean_walk(s, 0, nchunks, v, +1);
      if (pr >= 0 && sd[pr] == v) {
        if (pr < tn)
          s.child[pr][0] = (int32_t)(t0 - eoff);
        else
          a.nodes[t1].child[0] = (int32_t)(t0 - eoff);
      } else {
        const int slot = atomicAdd(&s.nunres, 1);
        if (slot < kUnresCap) s.unres[slot] = 0;
      }
    }
  }
  for (int k = 0; k < 4; ++k) {
    const int l = lbase + 32 * k;
    if (l >= tn) break;
    const int32_t id = (int32_t)(t0 + l - eoff);
    // leaf l, between positions l and l + 1: child 0 of node l + 1 when the
    // left distance is larger, else child 1 of node l (for a one-leaf cell,
    // node l is the cell's root and the leaf its whole tree)
    const uint32_t dl = sd[l], dr = sd[l + 1];
    if (dl >= kDeltaInf) s.child[l][0] = ~(id > 0 ? id - 1 : 0);  // l starts a cell
    const bool single = dl >= kDeltaInf && dr >= kDeltaInf;
    const bool left = dl > dr && !single;
    const int rec = left ? l + 1 : l;
    if (rec < tn)
      s.child[rec][left ? 0 : 1] = ~id;
    else
      a.nodes[t1].child[0] = ~id;
    if (single) s.cell_range[atomicAdd(&s.ncells, 1)] = (uint32_t)l | ((uint32_t)l << 16);
    // node at position p = l + 1 (the split between leaves l and l + 1)
    const int p = l + 1;
    const uint32_t v = dr;
    if (p > tn - 1 || v >= kDeltaInf) continue;
    const int c = 4 * warp + k;
    const uint32_t gt = chunk_gt(s, c, v), ge = chunk_ge(s, c, v);
    int pl;
    {
      const uint32_t msk = gt & ((1u << lane) - 1u);
      if (msk) {
        pl = 32 * c + 1 + (31 - __clz(msk));
      } else {
        pl = lean_walk(s, c - 1, nchunks, v, -1);
        if (pl < 0 && sd[0] > v) pl = 0;
      }
    }
    int pr;
    {
      const uint32_t msk = lane < 31 ? (ge & ~((2u << lane) - 1u)) : 0u;
      pr = msk ? 32 * c + __ffs(msk) : lean_walk(s, c + 1, nchunks, v, +1);
    }
    const int32_t nid = (int32_t)(t0 + p - eoff);
    if (pr < 0 || (pl < 0 && sd[pr] > v)) {
      const int slot = atomicAdd(&s.nunres, 1);
      if (slot < kUnresCap) s.unres[slot] = p;
      continue;
    }
    const uint32_t dR = sd[pr];
    const uint32_t dL = pl >= 0 ? sd[pl] : kDeltaInf + 1;
    if (dL >= kDeltaInf && dR >= kDeltaInf && pl >= 0) {
      // the top of a cell inside the tile: leaves [pl, pr - 1], root at pl
      s.child[pl][1] = nid;
      s.cell_range[atomicAdd(&s.ncells, 1)] = (uint32_t)pl | ((uint32_t)(pr - 1) << 16);
    } else if (dL > dR) {
      if (pr < tn)
        s.child[pr][0] = nid;
      else
        a.nodes[t1].child[0] = nid;
    } else {
      s.child[pl][1] = nid;
    }
  }
  __syncthreads();

  // ---- guide entries of the cells completed inside the tile -----------------
  for (int i = tid; i < s.ncells; i += kForestThreads) {
    const uint32_t r = s.cell_range[i];
    const int lo = (int)(r & 0xFFFFu), hi = (int)(r >> 16);
    const int64_t glo = t0 + lo;
    const uint64_t Clm1 = glo > eoff ? sC[lo] : 0ull;
    const uint64_t Chp1 = t0 + hi + 1 == eend ? T : sC[hi + 2];
    const uint64_t Clo = sC[lo + 1], Chi = sC[hi + 1];
    const uint64_t Knext = t0 + hi + 1 == eend ? (1ull << 32) : key_of(Chp1, T, R, z);
    // the top of the cell's tree is its root's child 1 (written in the links)
    finish_cell(a, P, dd, glo, t0 + hi, key_of(Clo, T, R, z), key_of(Chi, T, R, z), Clm1, Clo, Chi,
                Chp1, s.child[lo][1], Knext);
  }

  // ---- node records (lane-strided: each k is 32 consecutive records) ----------
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int l = lbase + 32 * k;
    if (l >= tn) break;
    const int32_t c0 = s.child[l][0], c1 = s.child[l][1];
    const uint64_t Cl = sC[l + 1];
    rtf_node* rec = a.nodes + t0 + l;
    if (c0 != kUnset && c1 != kUnset) {
      rtf_node r;
      r.cdf = Cl;
      r.child[0] = c0;
      r.child[1] = c1;
      *rec = r;
    } else {
      rec->cdf = Cl;
      if (c0 != kUnset) rec->child[0] = c0;
      if (c1 != kUnset) rec->child[1] = c1;
    }
  }
  const int nu = s.nunres;
  if (tid == 0) {
    if (nu > kUnresCap) raise_status(a.status, RTF_STATUS_INVARIANT);
    a.unres_count[tile] = min(nu, kUnresCap);
  }
  if (tid < min(nu, kUnresCap)) a.unres[tile * kUnresCap + tid] = (int32_t)(t0 + s.unres[tid]);
}

__global__ void __launch_bounds__(kForestThreads, RTF_FOREST_MINB) forest_lean_kernel(ForestArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  lean_tile<true>(a, *reinterpret_cast<LeanShared*>(smem_raw), a.dists[0], 0);
}

// Byte lanes first..last (0..3) of a 32-bit word.
__device__ __forceinline__ uint32_t byte_range(int first, int last) {
  return (0xFFFFFFFFu << (8 * first)) & (0xFFFFFFFFu >> (8 * (3 - last)));
}

// Bytes of a word that exceed v (or are at least v when GE), as 0xFF per byte;
// vv holds v in all four bytes.
template <bool GE>
__device__ __forceinline__ uint32_t bytes_above(uint32_t x, uint32_t vv) {
  return GE ? __vcmpgeu4(x, vv) : __vcmpgtu4(x, vv);
}

// Searches of one thread over a byte array (the distances per split, or the
// largest distance per tile), read as aligned 16-byte words and compared four
// bytes at a time: the nearest position in [lo, hi] to hi (scan_down) or to
// lo (scan_up) whose byte exceeds v (or is at least v when GE), or -1.  Both
// arrays are allocated in whole 256-byte units, so a word that straddles hi
// stays inside the allocation.  v < 256.
template <bool GE>
__device__ int64_t scan_down(const uint8_t* b, int64_t hi, int64_t lo, uint32_t v) {
  const uint32_t vv = v * 0x01010101u;
  for (int64_t w = hi & ~int64_t(15); w + 15 >= lo && w >= 0; w -= 16) {
    const uint4 x = __ldg(reinterpret_cast<const uint4*>(b + w));
    const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int i = 3; i >= 0; --i) {
      const int64_t base = w + 4 * i;
      if (base > hi || base + 3 < lo) continue;
      const int first = base < lo ? (int)(lo - base) : 0;
      const int last = base + 3 > hi ? (int)(hi - base) : 3;
      const uint32_t m = bytes_above<GE>(xs[i], vv) & byte_range(first, last);
      if (m) return base + (31 - __clz(m)) / 8;
    }
  }
  return -1;
}

template <bool GE>
__device__ int64_t scan_up(const uint8_t* b, int64_t lo, int64_t hi, uint32_t v) {
  const uint32_t vv = v * 0x01010101u;
  for (int64_t w = lo & ~int64_t(15); w <= hi; w += 16) {
    const uint4 x = __ldg(reinterpret_cast<const uint4*>(b + w));
    const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t base = w + 4 * i;
      if (base > hi || base + 3 < lo) continue;
      const int first = base < lo ? (int)(lo - base) : 0;
      const int last = base + 3 > hi ? (int)(hi - base) : 3;
      const uint32_t m = bytes_above<GE>(xs[i], vv) & byte_range(first, last);
      if (m) return base + (__ffs(m) - 1) / 8;
    }
  }
  return -1;
}

// The searches of the merge pass, one node per thread: the splits of j's
// tile, then the tiles of its group of kTileGroup tiles by their largest
// distance; a search that leaves the group returns -1 with *out set, and the
// warp then finds the group (group_left / group_right, 32 groups per step).
// Left: nearest split j' < j with delta_{j'} > v (the array start counts as
// infinitely far).  Right: nearest j' > j with delta_{j'} >= v (the last
// split, delta_{N-1}, is a boundary and ends every search).
__device__ int64_t left_in_group(const ForestArgs& a, int64_t j, uint32_t v, bool* out) {
  *out = false;
  const int64_t T = j / kTile;
  const int64_t r = scan_down<false>(a.delta, j - 1, T * kTile, v);
  if (r >= 0) return r;
  const int64_t G = T / kTileGroup;
  const int64_t t = scan_down<false>(a.tmax, T - 1, G * kTileGroup, v);
  if (t < 0) {
    *out = G > 0;
    return -1;
  }
  return scan_down<false>(a.delta, min(t * kTile + kTile, a.N) - 1, t * kTile, v);
}

__device__ int64_t right_in_group(const ForestArgs& a, int64_t j, uint32_t v, int64_t ntiles,
                                  bool* out) {
  *out = false;
  const int64_t T = j / kTile;
  const int64_t r = scan_up<true>(a.delta, j + 1, min(T * kTile + kTile, a.N) - 1, v);
  if (r >= 0) return r;
  const int64_t G = T / kTileGroup;
  const int64_t t = scan_up<true>(a.tmax, T + 1, min(G * kTileGroup + kTileGroup, ntiles) - 1, v);
  if (t < 0) {
    *out = true;
    return -1;
  }
  return scan_up<true>(a.delta, t * kTile, min(t * kTile + kTile, a.N) - 1, v);
}

// The nearest split in group g (known to hold one): its tiles by their
// largest distance, then that tile's splits.
__device__ int64_t left_in(const ForestArgs& a, int64_t g, uint32_t v) {
  const int64_t t = scan_down<false>(a.tmax, g * kTileGroup + kTileGroup - 1, g * kTileGroup, v);
  return t < 0 ? -1 : scan_down<false>(a.delta, min(t * kTile + kTile, a.N) - 1, t * kTile, v);
}

__device__ int64_t right_in(const ForestArgs& a, int64_t g, uint32_t v, int64_t ntiles) {
  const int64_t t =
      scan_up<true>(a.tmax, g * kTileGroup, min(g * kTileGroup + kTileGroup, ntiles) - 1, v);
  return t < 0 ? -1 : scan_up<true>(a.delta, t * kTile, min(t * kTile + kTile, a.N) - 1, v);
}

// Warp-wide: nearest group g < G with gmax > v (left) or g > G with gmax >= v
// (right), 32 groups per step; -1 when none.
__device__ int64_t group_left(const ForestArgs& a, int64_t G, uint32_t v) {
  const int lane = threadIdx.x & 31;
  for (int64_t gg = G - 1; gg >= 0; gg -= 32) {
    const int64_t x = gg - lane;
    const unsigned m = __ballot_sync(0xffffffffu, x >= 0 && a.gmax[x] > v);
    if (m) return gg - (__ffs(m) - 1);
  }
  return -1;
}

__device__ int64_t group_right(const ForestArgs& a, int64_t G, uint32_t v, int64_t ngroups) {
  const int lane = threadIdx.x & 31;
  for (int64_t gg = G + 1; gg < ngroups; gg += 32) {
    const int64_t x = gg + lane;
    const unsigned m = __ballot_sync(0xffffffffu, x < ngroups && a.gmax[x] >= v);
    if (m) return gg + (__ffs(m) - 1);
  }
  return -1;
}

// The nodes whose range crosses a tile edge: one warp per tile, one node per
// lane; the two bounding splits come from the global distances, then the link
// (or the cell's root and guide entry) is written as inside a tile.
__global__ void __launch_bounds__(128) forest_merge_kernel(ForestArgs a, int64_t ntiles) {
  const int64_t tile = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
  if (tile >= ntiles) return;  // whole warps leave together
  const int lane = threadIdx.x & 31;
  const int cnt = a.unres_count[tile];
  const int64_t ngroups = (ntiles + kTileGroup - 1) / kTileGroup;
  for (int base = 0; base < cnt; base += 32) {
    const int k = base + lane;
    const bool act = k < cnt;
    int64_t p = 0, j = 0, jl = -1, jr = -1;
    uint32_t v = 0;
    bool outl = false, outr = false;
    if (act) {
      p = a.unres[tile * kUnresCap + k];  // node p: the split between p-1 and p
      j = p - 1;
      v = a.delta[j];
      jl = left_in_group(a, j, v, &outl);
      jr = right_in_group(a, j, v, ntiles, &outr);
    }
    // searches that left their group of tiles: the groups, warp-wide, one
    // lane's search at a time
    for (unsigned m = __ballot_sync(0xffffffffu, outl); m; m &= m - 1) {
      const int src = __ffs(m) - 1;
      const int64_t G = __shfl_sync(0xffffffffu, (long long)(j / kTile / kTileGroup), src);
      const uint32_t vs = __shfl_sync(0xffffffffu, v, src);
      const int64_t g = group_left(a, G, vs);
      if (lane == src) jl = g < 0 ? -1 : left_in(a, g, v);
    }
    for (unsigned m = __ballot_sync(0xffffffffu, outr); m; m &= m - 1) {
      const int src = __ffs(m) - 1;
      const int64_t G = __shfl_sync(0xffffffffu, (long long)(j / kTile / kTileGroup), src);
      const uint32_t vs = __shfl_sync(0xffffffffu, v, src);
      const int64_t g = group_right(a, G, vs, ngroups);
      if (lane == src) jr = g < 0 ? -1 : right_in(a, g, v, ntiles);
    }
    if (!act) continue;
    if (jr < 0) {
      raise_status(a.status, RTF_STATUS_INVARIANT);
      continue;
    }
    const int d = a.D > 1 ? find_dist(a.dists, a.tile_dist0[p / kTile], a.D - 1, p) : 0;
    const rtf_dist P = a.dists[d];
    const int32_t id = (int32_t)(p - P.elem_off);
    const uint32_t dl = jl >= 0 ? (uint32_t)a.delta[jl] : kDeltaInf;
    const uint32_t dr = a.delta[jr];
    if (dl >= kDeltaInf && dr >= kDeltaInf) {
      // the top of a cell: leaves [jl + 1, jr], root at jl + 1
      const int64_t lo = jl + 1, hi = jr;
      a.nodes[lo].child[1] = id;
      const int32_t lo_l = (int32_t)(lo - P.elem_off);
      const uint64_t Clo = a.nodes[lo].cdf, Chi = a.nodes[hi].cdf;
      const uint64_t Clm1 = lo_l > 0 ? a.nodes[lo - 1].cdf : 0ull;
      const uint64_t Chp1 = hi + 1 < P.elem_off + P.n ? a.nodes[hi + 1].cdf : P.total;
      const uint64_t Knext = hi + 1 < P.elem_off + P.n ? key_for(P, Chp1) : (1ull << 32);
      finish_cell(a, P, d, lo, hi, key_for(P, Clo), key_for(P, Chi), Clm1, Clo, Chi, Chp1, id,
                  Knext);
    } else if (dl > dr) {
      a.nodes[jr + 1].child[0] = id;
    } else {
      a.nodes[jl + 1].child[1] = id;
    }
  }
}

// ---------------------------------------------------------------------------
// check of the bounded waits: a lookback on a predecessor nobody publishes
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kScanThreads) wait_probe_kernel(const uint64_t* st,
                                                                  uint32_t* status) {
  __shared__ LookbackShared lb;
  // tile 1 waits for tile 0, whose status word stays 0 (not published)
  (void)block_lookback(st, 1, true, &lb, status);
}

cudaError_t launch_wait_probe(uint32_t* status, uint64_t* scratch, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(scratch, 0, 2 * sizeof(uint64_t), st);
  if (e != cudaSuccess) return e;
  wait_probe_kernel<<<1, kScanThreads, 0, st>>>(scratch, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// fill: the long runs of empty cells listed by finish_cell
// ---------------------------------------------------------------------------
// One warp per listed piece (at most kFillPiece cells): every cell of it takes
// the interval `leaf` of its distribution, {C_i, ~i, ~i, C_i, C_{i+1}}.
__global__ void __launch_bounds__(256) fill_kernel(ForestArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t cnt = min((int64_t)*a.fill_count, a.fill_cap);
  for (int64_t i = warp; i < cnt; i += nwarps) {
    const int4 f = a.fills[i];
    const rtf_dist& P = a.dists[f.w];
    const int64_t e = P.elem_off + f.z;
    rtf_guide_rec cov;
    cov.cdf = a.nodes[e].cdf;
    cov.child[0] = ~f.z;
    cov.child[1] = ~f.z;
    cov.lo = cov.cdf;
    cov.hi = (int64_t)f.z + 1 < P.n ? a.nodes[e + 1].cdf : P.total;
    for (int64_t g = (int64_t)f.x + lane; g < (int64_t)f.x + f.y; g += 32) {
      a.guide[g] = ~f.z;
      a.guide_recs[g] = cov;
    }
  }
}

// ---------------------------------------------------------------------------
// host-side launch sequence (called from the C interface)
// ---------------------------------------------------------------------------
cudaError_t launch_build(const float* w, int64_t N, int64_t Nw, int D, int marginal,
                         const int64_t* offsets, const int32_t* m_arr, const int64_t* goff,
                         int64_t n_single, int m_single, const rtf_forest* f, void* ws,
                         cudaStream_t st) {
  const int64_t G = f->num_cells;
  WsLayout L = ws_layout(N, D, G);
  char* base = static_cast<char*>(ws);
  Counters* ctr = reinterpret_cast<Counters*>(base + L.counters);
  uint32_t* dmax = reinterpret_cast<uint32_t*>(base + L.dmax);
  uint64_t* scan_status = reinterpret_cast<uint64_t*>(base + L.scan_status);
  uint64_t* tile_prefix = reinterpret_cast<uint64_t*>(base + L.tile_prefix);
  uint8_t* delta = reinterpret_cast<uint8_t*>(base + L.delta);
  const bool seg = D > 1;
  const int Dw = marginal ? D - 1 : D;
  const int64_t n_shared = marginal ? Nw : 0;

  cudaError_t e;
  if ((e = cudaMemsetAsync(base + L.zero_begin, 0, L.zero_end - L.zero_begin, st))) return e;
  if ((e = cudaMemsetAsync(f->status, 0, sizeof(uint32_t), st))) return e;
  int32_t* tile_dist0 = reinterpret_cast<int32_t*>(base + L.tile_dist0);
  const int64_t ntiles_seg = seg ? num_tiles(N) : 0;
  init_dists_kernel<<<(unsigned)((std::max<int64_t>(D, ntiles_seg) + 255) / 256), 256, 0, st>>>(
      f->dists, D, offsets, m_arr, goff, marginal, n_single, m_single, tile_dist0, ntiles_seg,
      f->status);
  const int64_t nscale = (Nw + kScaleTile - 1) / kScaleTile;
  if (marginal || !seg) {
    // one group: a plain block max into dmax[0]
    scale_kernel<false><<<(unsigned)nscale, kScaleThreads, 0, st>>>(w, Nw, f->dists, Dw,
                                                                    tile_dist0, dmax, f->status);
  } else {
    scale_kernel<true><<<(unsigned)nscale, kScaleThreads, 0, st>>>(w, Nw, f->dists, Dw,
                                                                   tile_dist0, dmax, f->status);
  }
  const int64_t tiles_w = num_tiles(Nw);
  TileSums ts;
  ts.sum = reinterpret_cast<uint64_t*>(base + L.tile_sum);
  ts.first = reinterpret_cast<uint64_t*>(base + L.tile_first);
  ts.meta = reinterpret_cast<uint32_t*>(base + L.tile_meta);
  ts.dist0 = reinterpret_cast<int32_t*>(base + L.tile_dist0);
  if (seg) {
    tile_sum_kernel<true><<<(unsigned)tiles_w, kScanThreads, 0, st>>>(
        w, Nw, f->dists, Dw, n_shared, dmax, ts, tile_prefix, ctr, f->status);
    const int64_t chunks = (tiles_w + kTileScanChunk - 1) / kTileScanChunk;
    tile_scan_kernel<<<(unsigned)chunks, kScanThreads, 0, st>>>(ts, tiles_w, f->dists, D, Dw,
                                                               marginal, n_shared, dmax,
                                                               scan_status, tile_prefix, ctr,
                                                               f->status);
  } else {
    // one distribution: persistent blocks; the last one also scans the sums
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t grid = std::min<int64_t>(tiles_w, (int64_t)(sms > 0 ? sms : 148) * 8);
    tile_sum_kernel<false><<<(unsigned)grid, kScanThreads, 0, st>>>(
        w, Nw, f->dists, Dw, n_shared, dmax, ts, tile_prefix, ctr, f->status);
  }
  ForestArgs fa;
  fa.w = w;
  fa.N = N;
  fa.Nw = Nw;
  fa.dists = f->dists;
  fa.D = D;
  fa.Dw = Dw;
  fa.n_shared = n_shared;
  fa.nodes = f->nodes;
  fa.guide = f->guide;
  fa.guide_recs = f->guide_recs;
  fa.fills = reinterpret_cast<int4*>(base + L.fills);
  fa.fill_count = &ctr->fill_count;
  fa.fill_cap = fill_cap(D, G);
  fa.tile_prefix = tile_prefix;
  fa.dmax = dmax;
  fa.range_prefix = ts.first;
  fa.range_meta = ts.meta;
  fa.delta = delta;
  fa.tmax = reinterpret_cast<uint8_t*>(base + L.tmax);
  fa.gmax = reinterpret_cast<uint32_t*>(base + L.gmax);
  fa.unres = reinterpret_cast<int32_t*>(base + L.unres);
  fa.unres_count = reinterpret_cast<int32_t*>(base + L.unres_count);
  fa.tile_dist0 = tile_dist0;
  fa.status = f->status;
  if (seg) {
    const size_t fsmem = sizeof(ForestShared<true>);
    if ((e = cudaFuncSetAttribute(forest_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)fsmem)))
      return e;
    forest_kernel<true><<<(unsigned)num_tiles(N), kForestThreads, fsmem, st>>>(fa);
  } else {
    const size_t fsmem = sizeof(LeanShared);
    if ((e = cudaFuncSetAttribute(forest_lean_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)fsmem)))
      return e;
    forest_lean_kernel<<<(unsigned)num_tiles(N), kForestThreads, fsmem, st>>>(fa);
  }
  {
    const int64_t nt = num_tiles(N);
    forest_merge_kernel<<<(unsigned)((nt + 3) / 4), 128, 0, st>>>(fa, nt);
  }
  {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    fill_kernel<<<(unsigned)(sms > 0 ? 2 * sms : 304), 256, 0, st>>>(fa);
  }
  return cudaGetLastError();
}

}  // namespace rtf
