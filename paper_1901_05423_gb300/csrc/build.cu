// Build of the radix tree forest (Binder & Keller, Sec. 3.2, Algorithm 1) and
// of the guide table (Cutpoint method, Sec. 2.5, with the encoding of
// Sec. 3.2) for one or many distributions at once (Sec. 5).
//
// Kernels, in launch order:
//   init_dists_kernel   per-distribution parameters from the plan
//   scale_kernel        validation and max exponent (one read of w)
//   tile_sum_kernel     segmented sums of the integer weights per tile (second
//                       read of w, staged by a bulk copy); totals of the
//                       distributions that lie inside one tile
//   tile_scan_kernel    decoupled-lookback segmented scan of the tile sums:
//                       the prefix of every tile, the totals T (and key
//                       reciprocals) of the distributions that cross tiles; in
//                       marginal mode the last block also scans the row totals
//   forest_kernel       C_j, keys K_j, distances, Algorithm 1 inside each tile
//                       in shared memory; node records, roots, guide entries
//                       of non-empty cells; the tile's slice of the global
//                       otherBounds (third read of w)
//   forest_merge_kernel the hand-offs across tile edges: Algorithm 1 continued
//                       through the global otherBounds
//   guide_kernel        guide entries of cells that no key falls into: the
//                       interval of the last key before them (carry-forward
//                       scan with a decoupled lookback)
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
__global__ void init_dists_kernel(rtf_dist* dists, int D, const int64_t* offsets,
                                  const int32_t* m_arr, const int64_t* goff, int marginal,
                                  int64_t n_single, int m_single, uint32_t* status) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= D) return;
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
                 int Dw, uint32_t* dmax, uint32_t* status) {
  __shared__ uint32_t smax[SEG ? kScaleTile + 1 : 1];
  __shared__ int dfirst_s;
  __shared__ uint32_t red[kScaleThreads / 32];
  const int64_t c0 = (int64_t)blockIdx.x * kScaleTile;
  const int64_t c1 = min(c0 + (int64_t)kScaleTile, Nw);
  const int64_t e0 = c0 + (int64_t)threadIdx.x * kScalePer;
  uint32_t bad = 0;
  if (!SEG) {
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
      if (threadIdx.x == 0 && v) atomicMax(dmax, v);
    }
    if (bad) raise_status(status, RTF_STATUS_BAD_WEIGHT);
    return;
  }
  // segmented: the block's elements span distributions dfirst..dlast
  if (threadIdx.x == 0) dfirst_s = find_dist(dists, 0, Dw - 1, c0);
  for (int k = threadIdx.x; k <= kScaleTile; k += kScaleThreads) smax[k] = 0u;
  __syncthreads();
  const int dfirst = dfirst_s;
  if (e0 < c1) {
    int hi = min(Dw - 1, dfirst + kScaleTile);
    int d = find_dist(dists, dfirst, hi, e0);
    int64_t next = d + 1 < Dw ? dists[d + 1].elem_off : INT64_MAX;
    uint32_t run = 0;
    const int64_t e1 = min(e0 + (int64_t)kScalePer, c1);
    for (int64_t e = e0; e < e1; ++e) {
      if (e >= next) {
        if (run) atomicMax(&smax[d - dfirst], run);
        run = 0;
        ++d;
        next = d + 1 < Dw ? dists[d + 1].elem_off : INT64_MAX;
      }
      uint32_t b = weight_bits(w[e]);
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
  const int dlast = (c1 > c0) ? find_dist(dists, dfirst, min(Dw - 1, dfirst + kScaleTile), c1 - 1)
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

// Tile sums of q (second read of w, staged by a bulk copy).  Distributions that
// begin and end inside the tile are finished here; the tile's first piece,
// whose distribution began in an earlier tile, waits for the scan of the tile
// sums.
template <bool SEG>
__global__ void __launch_bounds__(kScanThreads)
    tile_sum_kernel(const float* __restrict__ w, int64_t Nw, rtf_dist* dists, int Dw,
                    int64_t n_shared, const uint32_t* dmax, TileSums ts, uint32_t* status) {
  __shared__ alignas(16) float wsm[kTile + 4];
  __shared__ uint64_t bar;
  __shared__ int ok_s;
  __shared__ int dfirst_s;
  __shared__ SegPair wtot[kScanThreads / 32];
  __shared__ SegPair btot;
  __shared__ uint32_t meta_s;

  const int64_t tile = blockIdx.x;
  const int64_t t0 = tile * kTile, t1 = min(t0 + (int64_t)kTile, Nw);

  if (!SEG) {
    // one distribution: the tile's sum of q (weights read straight from
    // global memory, 16-byte vectors where aligned); the last tile also
    // holds the distribution's end (finished here when the tile is also the
    // first)
    const int S = dist_scale(dists[0], dmax, 0, n_shared);
    const int64_t e0 = t0 + (int64_t)threadIdx.x * kScanPer;
    float wv[kScanPer];
    if (e0 + kScanPer <= t1 && (reinterpret_cast<uintptr_t>(w + e0) & 15) == 0) {
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
    uint64_t run = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      if (e0 + k < t1) {
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
      const bool head0 = t0 == 0;
      uint32_t meta = head0 ? 3u : 0u;
      if (t1 == Nw) {
        if (head0) {
          finish_dist(dists, 0, sum, S, status);
        } else {
          ts.first[tile] = sum;
          meta |= 4u;
        }
      }
      ts.sum[tile] = sum;
      ts.meta[tile] = meta;
      ts.dist0[tile] = 0;
    }
    return;
  }

  if (threadIdx.x == 0) {
    dfirst_s = find_dist(dists, 0, Dw - 1, t0);
    meta_s = 0;
  }
  const int wo = stage_weights(wsm, w, t0, t1, &bar, &ok_s, status);
  const int dfirst = dfirst_s;

  // per-thread run of kScanPer consecutive weights
  const int64_t e0 = t0 + (int64_t)threadIdx.x * kScanPer;
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
        const uint32_t b = weight_bits(wsm[wo + (e - t0)]);
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
    ts.dist0[tile] = dfirst;
  }
}

constexpr int kTileScanPer = 8;
constexpr int kTileScanChunk = kScanThreads * kTileScanPer;  // tiles per scan block

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
// forest: Algorithm 1 per tile in shared memory, cross-tile merges in global
// ---------------------------------------------------------------------------
constexpr int kForestPer = kTile / kForestThreads;  // 4
static_assert(kForestPer == 4, "the otherBounds write-out stores one int4 per thread");
constexpr int32_t kUnset = 0x7FFFFFFF;

template <bool SEG>
struct ForestShared {
  alignas(16) uint64_t C[kTile + 2];  // C_{t0-1} .. C_{t1}
  alignas(16) uint64_t K[kTile + 2];  // K_{t0-1} .. K_{t1}
  alignas(16) int32_t child[kTile][2];
  // the staged weights are dead once q is known; the tile's otherBounds reuse them
  union alignas(16) WO {
    float w[kTile + 4];
    int32_t other[kTile + 4];
  } wo;
  int32_t dist[SEG ? kTile : 1];
  uint8_t delta[kTile + 4];  // delta_{t0-1} .. delta_{t1-1}
  SegPair wtot[kForestThreads / 32];
  SegPair btot;
  uint64_t bar;
  int ok;
  int dfirst;
  int dprev;
  int ndefer;
  float wprev;
  uint64_t prefix;
  rtf_dist P0;  // parameters of the tile's first distribution
  int32_t defer_parent[kDeferCap];
  int32_t defer_bound[kDeferCap];
  int32_t defer_node[kDeferCap];
  int32_t defer_dist[kDeferCap];
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
  int32_t* last;
  uint64_t* last_lo;
  const uint64_t* tile_prefix;
  const uint32_t* dmax;
  uint8_t* delta;
  int32_t* other;
  uint4* items;
  int32_t* item_count;
  uint32_t* status;
};

// Key of C_j for distribution P.
__device__ __forceinline__ uint64_t key_for(const rtf_dist& P, uint64_t C) {
  return key_of(C, P.total, P.recip, P.shift);
}

// Root of a finished cell [lo, hi] (global element indices) of distribution P:
// guide entry, guide record and last-leaf entries of the cell.  K_lo / K_hi
// are the keys of leaves lo and hi; C_{lo-1} (0 when lo is the first leaf of
// the distribution), C_lo, C_hi and C_{hi+1} (T after the last leaf) their
// CDF bounds.
__device__ __forceinline__ void finish_cell(const ForestArgs& a, const rtf_dist& P, int64_t lo,
                                            int64_t hi, uint64_t Klo, uint64_t Khi,
                                            uint64_t Clm1, uint64_t Clo, uint64_t Chi,
                                            uint64_t Chp1, int32_t top) {
  uint64_t c = cell_of(Klo, P.m);
  if (c >= (1ull << P.m)) return;  // unreachable trailing cell of zero-width bins
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
  a.last[gi] = hi_l;
  a.last_lo[gi] = Chi;
}

// Continue Algorithm 1 through global memory from range [lo, hi] with node
// `node` (local reference) of distribution P.  This runs in the merge kernel,
// after every tile has written its records, distances and otherBounds slice,
// so the hand-offs are plain atomic exchanges.
__device__ void climb_global(const ForestArgs& a, const rtf_dist& P, int64_t lo, int64_t hi,
                             int32_t node) {
  for (int64_t guard = 0; guard <= a.N; ++guard) {  // each pass grows the range
    uint32_t dl = lo > 0 ? (uint32_t)a.delta[lo - 1] : kDeltaInf;
    uint32_t dr = (uint32_t)a.delta[hi];
    if (dl >= kDeltaInf && dr >= kDeltaInf) {
      rtf_node* root = a.nodes + lo;
      int32_t lo_l = (int32_t)(lo - P.elem_off);
      root->child[0] = ~(lo_l > 0 ? lo_l - 1 : 0);
      root->child[1] = node;
      const uint64_t Clo = a.nodes[lo].cdf, Chi = a.nodes[hi].cdf;
      const uint64_t Clm1 = lo_l > 0 ? a.nodes[lo - 1].cdf : 0ull;
      const uint64_t Chp1 = hi + 1 < P.elem_off + P.n ? a.nodes[hi + 1].cdf : P.total;
      finish_cell(a, P, lo, hi, key_for(P, Clo), key_for(P, Chi), Clm1, Clo, Chi, Chp1, node);
      return;
    }
    int child = dl > dr ? 0 : 1;
    int64_t parent = child ? lo : hi + 1;
    a.nodes[parent].child[child] = node;
    int ob = atomicExch(a.other + parent, (int)(child ? hi : lo));
    if (ob < 0) return;  // first of the two children
    if (child)
      lo = ob;
    else
      hi = ob;
    node = (int32_t)(parent - P.elem_off);
  }
  raise_status(a.status, RTF_STATUS_TIMEOUT);
}

// A hand-off deferred by phase A because the sibling lies in the neighbouring
// tile, packed as uint4 {parent, bound, node, dist}: the arriver's range is
// [bound, parent-1] when it is the left child (bound < parent) and
// [parent, bound] when it is the right child.
__device__ void run_deferred(const ForestArgs& a, uint4 it) {
  const int64_t parent = (int32_t)it.x, bound = (int32_t)it.y;
  const int32_t node = (int32_t)it.z;
  const int child = bound < parent ? 0 : 1;
  const rtf_dist P = a.dists[it.w];
  a.nodes[parent].child[child] = node;
  const int ob = atomicExch(a.other + parent, (int)bound);
  if (ob < 0) return;
  const int64_t lo = child ? ob : bound, hi = child ? bound : ob;
  climb_global(a, P, lo, hi, (int32_t)(parent - P.elem_off));
}

// Minimum resident forest blocks per SM given to the register allocator.
#ifndef RTF_FOREST_MINB
#define RTF_FOREST_MINB 3
#endif

template <bool SEG>
__global__ void __launch_bounds__(kForestThreads, RTF_FOREST_MINB) forest_kernel(ForestArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ForestShared<SEG>& s = *reinterpret_cast<ForestShared<SEG>*>(smem_raw);
  const int64_t tile = blockIdx.x;
  const int64_t t0 = tile * kTile, t1 = min(t0 + (int64_t)kTile, a.N);
  const int tn = (int)(t1 - t0);
  const int tid = threadIdx.x;

  if (tid == 0) {
    const int df = SEG ? find_dist(a.dists, 0, a.D - 1, t0) : 0;
    s.dfirst = df;
    s.dprev = (t0 > 0 && SEG) ? (a.dists[df].elem_off == t0 ? df - 1 : df) : df;
    s.ndefer = 0;
    // loads needed later, issued while the tile is staged
    s.P0 = a.dists[df];
    s.prefix = t0 > 0 ? a.tile_prefix[tile] : 0ull;
    s.wprev = (t0 > 0 && t0 - 1 < a.Nw) ? a.w[t0 - 1] : 0.0f;
  }
  int wo = 0;
  if (t0 < a.Nw) wo = stage_weights(s.wo.w, a.w, t0, min(t1, a.Nw), &s.bar, &s.ok, a.status);
  else __syncthreads();
  const int dfirst = s.dfirst;

  // ---- q, C and keys of the thread's leaves ---------------------------------
  // Each thread owns kForestPer consecutive leaves; the parameters of the
  // distribution it is in stay in registers (reloaded only at a boundary).
  const int l0 = tid * kForestPer;  // tile-local index of the first leaf
  const int64_t e0 = t0 + l0;
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
          const uint32_t b = weight_bits(s.wo.w[wo + l0 + k]);
          qq = weight_bad(b) ? 0ull : quantize_bits(b, S);
        }
        if (SEG) s.dist[l0 + k] = dcur;
      }
      dk[k] = dcur;
      q[k] = qq;
      run += qq;
      incl[k] = run;
    }
    // exclusive prefix of the thread's run within the tile (its barriers also
    // retire s.wo.w); one distribution has its only head at element 0, where
    // the running sum is 0 anyway, so a plain scan serves
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
      s.wo.other[l] = -1;
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
  // distances: delta_j for the thread's leaves j, and delta_{t0-1} by thread 0
  {
    int dP = -1;
    int m = 0;
    int64_t end = 0;
    uint32_t packed = 0;
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
        s.delta[l + 1] = (uint8_t)dlt;
      }
      packed |= dlt << (8 * k);
    }
    if (l0 + kForestPer <= tn) {
      *reinterpret_cast<uint32_t*>(a.delta + e0) = packed;
    } else {
      for (int k = 0; k < kForestPer && l0 + k < tn; ++k)
        a.delta[e0 + k] = (uint8_t)(packed >> (8 * k));
    }
    if (tid == 0) {
      uint32_t d0 = kDeltaInf;
      if (t0 > 0 && s.dprev == dfirst) {
        const int mm = s.P0.m;
        const uint64_t Ka = s.K[0], Kb = s.K[1];
        if (cell_of(Ka, mm) == cell_of(Kb, mm)) d0 = key_distance(Ka, Kb);
      }
      s.delta[0] = (uint8_t)d0;
      if (t0 > 0) a.delta[t0 - 1] = (uint8_t)d0;
    }
  }
  __syncthreads();

  // ---- phase A: Algorithm 1 inside the tile (tile-local indices) -----------
  // delta[l] is the distance left of leaf l, delta[l + 1] the one right of it.
#pragma unroll 1
  for (int k = 0; k < kForestPer; ++k) {
    const int l = l0 + k;
    if (l >= tn) break;
    const int d = SEG ? s.dist[l] : 0;
    const int32_t base_id = (int32_t)(t0 - (SEG ? a.dists[d].elem_off : s.P0.elem_off));
    int lo = l, hi = l;
    int32_t node = ~(base_id + l);
    while (true) {
      const uint32_t dl = s.delta[lo];
      const uint32_t dr = s.delta[hi + 1];
      if (dl >= kDeltaInf && dr >= kDeltaInf) {
        // full cell inside the tile: its root is the node of the first leaf
        const int32_t lo_id = base_id + lo;
        s.child[lo][0] = ~(lo_id > 0 ? lo_id - 1 : 0);
        s.child[lo][1] = node;
        const rtf_dist& P = SEG ? a.dists[d] : s.P0;
        // s.C[l + 1] is C of tile leaf l; s.C[0] that of t0 - 1 (same distribution)
        const uint64_t Clm1 = lo_id > 0 ? s.C[lo] : 0ull;
        const uint64_t Chp1 = t0 + hi + 1 == P.elem_off + P.n ? P.total : s.C[hi + 2];
        finish_cell(a, P, t0 + lo, t0 + hi, s.K[lo + 1], s.K[hi + 1], Clm1, s.C[lo + 1],
                    s.C[hi + 1], Chp1, node);
        break;
      }
      const int child = dl > dr ? 0 : 1;
      if ((child == 1 && lo == 0) || (child == 0 && hi == tn - 1)) {
        // the sibling lies in the neighbouring tile
        const int slot = atomicAdd(&s.ndefer, 1);
        if (slot < kDeferCap) {
          s.defer_parent[slot] = (int32_t)(t0 + (child ? lo : hi + 1));
          s.defer_bound[slot] = (int32_t)(t0 + (child ? hi : lo));
          s.defer_node[slot] = node;
          s.defer_dist[slot] = d;
        }
        break;
      }
      const int parent = child ? lo : hi + 1;
      s.child[parent][child] = node;
      const int ob = atomicExch(&s.wo.other[parent], child ? hi : lo);
      if (ob < 0) break;
      s.wo.other[parent] = -2;
      if (child)
        lo = ob;
      else
        hi = ob;
      node = base_id + parent;
    }
  }
  __syncthreads();

  // ---- node records and the tile's otherBounds slice -------------------------
  // Records go out with consecutive threads on consecutive records (leaf
  // l = tid + k * blockDim); otherBounds holds the far bound of every first
  // arrival still waiting for its sibling, -1 everywhere else.
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
  int ob4[kForestPer];
#pragma unroll
  for (int k = 0; k < kForestPer; ++k) {
    const int l = l0 + k;
    const int o = l < tn ? s.wo.other[l] : -1;
    ob4[k] = o >= 0 ? (int)(t0 + o) : -1;
  }
  if (l0 + kForestPer <= tn) {
    *reinterpret_cast<int4*>(a.other + e0) = make_int4(ob4[0], ob4[1], ob4[2], ob4[3]);
  } else {
    for (int k = 0; k < kForestPer && l0 + k < tn; ++k) a.other[e0 + k] = ob4[k];
  }

  // ---- hand-offs across tile edges -------------------------------------------
  // A first arrival that no sibling met inside the tile stays in this tile's
  // slice of the global otherBounds (written above); a range that must merge
  // with a sibling in the neighbouring tile is deferred to the merge kernel.
  const int nd = s.ndefer;
  if (tid == 0) {
    if (nd > kDeferCap) raise_status(a.status, RTF_STATUS_TIMEOUT);
    a.item_count[tile] = min(nd, kDeferCap);
  }
  if (tid < min(nd, kDeferCap)) {
    a.items[tile * kDeferCap + tid] =
        make_uint4((uint32_t)s.defer_parent[tid], (uint32_t)s.defer_bound[tid],
                   (uint32_t)s.defer_node[tid], (uint32_t)s.defer_dist[tid]);
  }
}

// Hand-offs across tile edges, after every tile finished: one thread per
// deferred range continues Algorithm 1 through the global otherBounds.
__global__ void __launch_bounds__(128) forest_merge_kernel(ForestArgs a, int64_t ntiles) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tile = i / kDeferCap;
  const int k = (int)(i % kDeferCap);
  if (tile >= ntiles || k >= a.item_count[tile]) return;
  run_deferred(a, a.items[tile * kDeferCap + k]);
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
// guide: cells without keys take the interval of the last key before them
// ---------------------------------------------------------------------------
constexpr int kGuidePer = kGuideTile / kGuideThreads;  // 4

__global__ void __launch_bounds__(kGuideThreads)
    guide_kernel(int64_t G, const int32_t* __restrict__ last, const uint64_t* __restrict__ last_lo,
                 int32_t* guide, rtf_guide_rec* guide_recs, uint64_t* gstatus, Counters* ctr,
                 uint32_t* status) {
  __shared__ uint32_t tile_s;
  __shared__ int32_t wlast[kGuideThreads / 32];
  __shared__ int32_t carry_s;
  __shared__ LookbackShared lb;
  if (threadIdx.x == 0) tile_s = atomicAdd(&ctr->guide_ticket, 1u);
  __syncthreads();
  const int64_t tile = tile_s;
  const int64_t g0 = tile * kGuideTile + (int64_t)threadIdx.x * kGuidePer;
  const int64_t gend = min(tile * kGuideTile + (int64_t)kGuideTile, G);
  // the carried value is the index of the last non-empty cell (G < 2^31)
  bool full[kGuidePer];
  int32_t tlast = -1;
#pragma unroll
  for (int k = 0; k < kGuidePer; ++k) {
    int64_t g = g0 + k;
    full[k] = g < gend && last[g] >= 0;
    if (full[k]) tlast = (int32_t)g;
  }
  // last non-empty cell of all threads before this one (warp, then block)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t inc = tlast;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int32_t o = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d && inc < 0) inc = o;
  }
  if (lane == 31) wlast[warp] = inc;
  __syncthreads();
  int32_t before_warp = -1;
  for (int w2 = 0; w2 < warp; ++w2)
    if (wlast[w2] >= 0) before_warp = wlast[w2];
  int32_t ex = __shfl_up_sync(0xffffffffu, inc, 1);
  if (lane == 0) ex = -1;
  int32_t before = ex >= 0 ? ex : before_warp;
  int32_t tile_last = -1;
  for (int w2 = 0; w2 < kGuideThreads / 32; ++w2)
    if (wlast[w2] >= 0) tile_last = wlast[w2];
  if (threadIdx.x == 0) {
    if (tile_last >= 0)
      st_release_u64(gstatus + tile, kFlagPrefix | (uint32_t)tile_last);
    else
      st_release_u64(gstatus + tile, kFlagAgg);
  }
  // the incoming carry is needed only when the tile's first cell is empty
  __shared__ int need_s;
  if (threadIdx.x == 0) {
    carry_s = -1;
    need_s = (g0 < gend && !full[0]) ? 1 : 0;
  }
  __syncthreads();
  if (need_s) {
    int32_t c = (int32_t)(uint32_t)(block_lookback(gstatus, tile, false, &lb, status) &
                                     0xffffffffull);
    if (threadIdx.x == 0) {
      carry_s = c;
      if (tile_last < 0) st_release_u64(gstatus + tile, kFlagPrefix | (uint32_t)c);
    }
  }
  __syncthreads();
  int32_t src = before >= 0 ? before : carry_s;
  rtf_guide_rec rec;
  int32_t rec_src = -1;
#pragma unroll
  for (int k = 0; k < kGuidePer; ++k) {
    int64_t g = g0 + k;
    if (g >= gend) break;
    if (full[k]) {
      src = (int32_t)g;
    } else {
      if (src < 0) {
        // cell 0 of a distribution always holds key 0, so this is unreachable;
        // the record refers to no interval (the sampler returns -1 through it)
        raise_status(status, RTF_STATUS_BAD_PLAN);
        rec = rtf_guide_rec{0ull, {INT32_MIN, INT32_MIN}, 0ull, 0ull};
        rec_src = -1;
      } else if (src != rec_src) {
        // the last interval of cell src covers this cell
        rec_src = src;
        const int32_t i = last[src];
        rec.lo = last_lo[src];
        rec.cdf = rec.lo;
        rec.child[0] = ~i;
        rec.child[1] = ~i;
        rec.hi = guide_recs[src].hi;
      }
      guide[g] = rec.child[0];
      guide_recs[g] = rec;
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
  uint64_t* guide_status = reinterpret_cast<uint64_t*>(base + L.guide_status);
  int32_t* last = reinterpret_cast<int32_t*>(base + L.last);
  uint64_t* tile_prefix = reinterpret_cast<uint64_t*>(base + L.tile_prefix);
  uint8_t* delta = reinterpret_cast<uint8_t*>(base + L.delta);
  int32_t* other = reinterpret_cast<int32_t*>(base + L.other);
  uint4* items = reinterpret_cast<uint4*>(base + L.items);
  int32_t* item_count = reinterpret_cast<int32_t*>(base + L.item_count);
  const bool seg = D > 1;
  const int Dw = marginal ? D - 1 : D;
  const int64_t n_shared = marginal ? Nw : 0;

  cudaError_t e;
  if ((e = cudaMemsetAsync(base + L.zero_begin, 0, L.zero_end - L.zero_begin, st))) return e;
  if ((e = cudaMemsetAsync(last, 0xFF, sizeof(int32_t) * (size_t)G, st))) return e;
  if ((e = cudaMemsetAsync(f->status, 0, sizeof(uint32_t), st))) return e;
  init_dists_kernel<<<(D + 255) / 256, 256, 0, st>>>(f->dists, D, offsets, m_arr, goff, marginal,
                                                      n_single, m_single, f->status);
  const int64_t nscale = (Nw + kScaleTile - 1) / kScaleTile;
  if (marginal || !seg) {
    // one group: a plain block max into dmax[0]
    scale_kernel<false><<<(unsigned)nscale, kScaleThreads, 0, st>>>(w, Nw, f->dists, Dw, dmax,
                                                                    f->status);
  } else {
    scale_kernel<true><<<(unsigned)nscale, kScaleThreads, 0, st>>>(w, Nw, f->dists, Dw, dmax,
                                                                   f->status);
  }
  const int64_t tiles_w = num_tiles(Nw);
  TileSums ts;
  ts.sum = reinterpret_cast<uint64_t*>(base + L.tile_sum);
  ts.first = reinterpret_cast<uint64_t*>(base + L.tile_first);
  ts.meta = reinterpret_cast<uint32_t*>(base + L.tile_meta);
  ts.dist0 = reinterpret_cast<int32_t*>(base + L.tile_dist0);
  if (seg)
    tile_sum_kernel<true><<<(unsigned)tiles_w, kScanThreads, 0, st>>>(w, Nw, f->dists, Dw,
                                                                     n_shared, dmax, ts, f->status);
  else
    tile_sum_kernel<false><<<(unsigned)tiles_w, kScanThreads, 0, st>>>(w, Nw, f->dists, Dw,
                                                                      n_shared, dmax, ts, f->status);
  const int64_t chunks = (tiles_w + kTileScanChunk - 1) / kTileScanChunk;
  tile_scan_kernel<<<(unsigned)chunks, kScanThreads, 0, st>>>(ts, tiles_w, f->dists, D, Dw, marginal,
                                                             n_shared, dmax, scan_status,
                                                             tile_prefix, ctr, f->status);
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
  fa.last = last;
  fa.last_lo = reinterpret_cast<uint64_t*>(base + L.last_lo);
  fa.tile_prefix = tile_prefix;
  fa.dmax = dmax;
  fa.delta = delta;
  fa.other = other;
  fa.items = items;
  fa.item_count = item_count;
  fa.status = f->status;
  if (seg) {
    const size_t fsmem = sizeof(ForestShared<true>);
    if ((e = cudaFuncSetAttribute(forest_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)fsmem)))
      return e;
    forest_kernel<true><<<(unsigned)num_tiles(N), kForestThreads, fsmem, st>>>(fa);
  } else {
    const size_t fsmem = sizeof(ForestShared<false>);
    if ((e = cudaFuncSetAttribute(forest_kernel<false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem)))
      return e;
    forest_kernel<false><<<(unsigned)num_tiles(N), kForestThreads, fsmem, st>>>(fa);
  }
  {
    const int64_t nt = num_tiles(N);
    forest_merge_kernel<<<(unsigned)((nt * kDeferCap + 127) / 128), 128, 0, st>>>(fa, nt);
  }
  const int64_t gtiles = (G + kGuideTile - 1) / kGuideTile;
  guide_kernel<<<(unsigned)gtiles, kGuideThreads, 0, st>>>(G, last, fa.last_lo, f->guide,
                                                            f->guide_recs,
                                                           guide_status, ctr, f->status);
  return cudaGetLastError();
}

}  // namespace rtf
