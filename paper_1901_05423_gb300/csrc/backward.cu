// Gradient of the in-bin sample positions with respect to the weights (not in
// the paper; the adjoint of the relaxed forward x = (xi W - C_i) / w_i with the
// bin i of each sample held fixed).
//
//   dL/dw_k = sum_{i in d} Xi_i / w_i  -  sum_{i > k, i in d} A_i / w_i  -  X_k / w_k
//   A_i = sum_{s -> i} g_s,  X_i = sum_{s -> i} g_s x_s,  Xi_i = sum_{s -> i} g_s xi_s.
//
// The sample's own xi need not be carried: the position is defined through
// the exact integer CDF, u / 2^32 = (C_i + x q_i) / T, so
// Xi_i = (A_i C_i + X_i q_i) / T with the integers of the built structure.
// Only two sums per bin are accumulated.
//
// Kernels:
//   row_sum_kernel       (2-D) real row totals R_r = sum_c w(r, c), the
//                        weights of the marginal
//   scatter kernels      one 8-byte vector atomic {g, g x} per sample into its
//                        bin, runs of equal bins inside a warp merged first
//   bin_total_kernel     G_d = sum_{i in d} Xi_i / w_i per distribution
//   suffix_kernel        reverse decoupled-lookback scan of A_i / w_i per
//                        distribution (fp32 in the tile, fp64 carry), then
//                        dL/dw_k = G_d - S_k - X_k / w_k
//   add_row_kernel       (2-D) the marginal's gradient dL/dR_r added to every
//                        weight of row r
#include <algorithm>
#include <cstdint>

#include "rtf_device.cuh"

namespace rtf {

constexpr int kBwThreads = 256;
constexpr int kBwPer = 8;
constexpr int kBwTile = kBwThreads * kBwPer;  // 2048

struct BwLayout {
  size_t acc;    // float2 [N]  {A_i, X_i}
  size_t G;      // double [D]
  size_t flags;  // u32 [tiles]
  size_t carry;  // double [tiles]   sum of a over a tile's first piece
  size_t incl;   // double [tiles]   that sum plus everything after it
  size_t ticket; // u32
  size_t zero_end;
  size_t R;      // float [D]   (2-D: row totals)
  size_t gradR;  // float [D]   (2-D: gradient of the marginal's weights)
  size_t total;
};

__host__ __device__ inline BwLayout bw_layout(int64_t N, int32_t D) {
  BwLayout L;
  size_t o = 0;
  int64_t tiles = (N + kBwTile - 1) / kBwTile;
  L.acc = o; o = align256(o + 8 * (size_t)N);
  L.G = o; o = align256(o + 8 * (size_t)D);
  L.flags = o; o = align256(o + 4 * (size_t)tiles);
  L.carry = o; o = align256(o + 8 * (size_t)tiles);
  L.incl = o; o = align256(o + 8 * (size_t)tiles);
  L.ticket = o; o = align256(o + 256);
  L.zero_end = o;
  L.R = o; o = align256(o + 4 * (size_t)D);
  L.gradR = o; o = align256(o + 4 * (size_t)D);
  L.total = o;
  return L;
}

// weight of element e: a row weight, or (2-D) the real total of marginal row e - Nw
__device__ __forceinline__ float weight_at(const float* w, const float* R, int64_t Nw, int64_t e) {
  return e < Nw ? w[e] : R[e - Nw];
}

// ---------------------------------------------------------------------------
__global__ void row_sum_kernel(const float* __restrict__ w, const rtf_dist* __restrict__ dists,
                               int H, float* R) {
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x >> 5;
  for (int r = blockIdx.x * warps + (threadIdx.x >> 5); r < H; r += gridDim.x * warps) {
    const int64_t off = dists[r].elem_off, n = dists[r].n;
    float s = 0.0f;
    for (int64_t k = lane; k < n; k += 32) s += w[off + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) R[r] = s;
  }
}

// Merge the contributions of lanes that hit the same bin (runs of equal j
// among consecutive lanes), then one vector atomic per run.
__device__ __forceinline__ void scatter_merge(float2* acc, int64_t j, float va, float vb,
                                              bool valid) {
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  const int64_t jprev = __shfl_up_sync(full, j, 1);
  const bool head = (lane == 0) || (jprev != j);
  const unsigned heads = __ballot_sync(full, head);
  if (heads != full) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const float pa = __shfl_up_sync(full, va, d);
      const float pb = __shfl_up_sync(full, vb, d);
      // lane may add lane-d's partial only if no run starts in (lane-d, lane]
      const unsigned span = (lane >= d) ? (((1u << lane) << 1) - (1u << (lane - d + 1))) : 0u;
      if (lane >= d && (heads & span) == 0) {
        va += pa;
        vb += pb;
      }
    }
  }
  const bool tail = (lane == 31) || (((heads >> (lane + 1)) & 1u) != 0);
  if (tail && valid) {
    // the per-bin sums (8 bytes per bin, about the size of L2 at 2^24 bins)
    // are added with an L2 evict-last policy while the sample stream passes
    // through with evict-first loads, so that the sums stay resident: 2^28
    // samples into 2^24 bins, backward 3.71 -> 3.14 ms on GB300 (a plain
    // vector atomic, with or without the default policy: 3.71 ms; fractions
    // 0.5-1.0 of the policy alike)
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("red.global.add.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(acc + j), "f"(va),
                 "f"(vb), "l"(pol)
                 : "memory");
  }
}

// 1-D samples (dist_id NULL -> distribution 0); bins outside [jlo, jhi) are
// left to another pass.
__global__ void __launch_bounds__(kBwThreads)
    scatter_1d_kernel(const rtf_dist* __restrict__ dists, int D, const int32_t* __restrict__ dist_id,
                      const int32_t* __restrict__ idx, const float* __restrict__ pos,
                      const float* __restrict__ gpos, int64_t count, float2* acc,
                      int64_t jlo, int64_t jhi) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t start = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t iters = (count + stride - 1) / stride;
  const int64_t off0 = dists[0].elem_off, n0 = dists[0].n;
  for (int64_t it = 0; it < iters; ++it) {
    const int64_t s = start + it * stride;
    bool valid = s < count;
    int64_t j = -1 - (int64_t)(threadIdx.x & 31);
    float va = 0.f, vb = 0.f;
    if (valid) {
      const int d = dist_id ? __ldcs(dist_id + s) : 0;
      const int32_t i = __ldcs(idx + s);
      int64_t off = off0, n = n0;
      if (dist_id) {
        valid = d >= 0 && d < D;
        if (valid) {
          off = dists[d].elem_off;
          n = dists[d].n;
        }
      }
      valid = valid && i >= 0 && (int64_t)i < n && off + i >= jlo && off + i < jhi;
      if (valid) {
        j = off + i;
        const float g = __ldcs(gpos + s);
        va = g;
        vb = g * __ldcs(pos + s);
      }
    }
    scatter_merge(acc, j, va, vb, valid);
  }
}

// 2-D samples: the row term into the marginal, the column term into the row.
__global__ void __launch_bounds__(kBwThreads)
    scatter_2d_kernel(const rtf_dist* __restrict__ dists, int D, const int2* __restrict__ idx,
                      const float2* __restrict__ pos, const float2* __restrict__ gpos,
                      int64_t count, float2* acc) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t start = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t iters = (count + stride - 1) / stride;
  const int64_t moff = dists[D - 1].elem_off;
  for (int64_t it = 0; it < iters; ++it) {
    const int64_t s = start + it * stride;
    bool valid = s < count;
    int64_t jr = -1 - (int64_t)(threadIdx.x & 31), jc = jr;
    float ra = 0.f, rb = 0.f, ca = 0.f, cb = 0.f;
    if (valid) {
      const int2 ii = __ldcs(idx + s);
      valid = ii.x >= 0 && ii.x < D - 1 && ii.y >= 0 && (int64_t)ii.y < dists[ii.x].n;
      if (valid) {
        const float2 pp = __ldcs(pos + s);
        const float2 gg = __ldcs(gpos + s);
        jr = moff + ii.x;
        ra = gg.x;
        rb = gg.x * pp.x;
        jc = dists[ii.x].elem_off + ii.y;
        ca = gg.y;
        cb = gg.y * pp.y;
      }
    }
    scatter_merge(acc, jr, ra, rb, valid);
    scatter_merge(acc, jc, ca, cb, valid);
  }
}

// G_d = sum_{i in d} Xi_i / w_i with Xi_i = (A_i C_i + X_i q_i) / T.
// Per-thread fp32 runs, then one fp64 atomic per distribution piece (a block
// inside one distribution reduces first and adds once).
__global__ void __launch_bounds__(kBwThreads)
    bin_total_kernel(const float2* __restrict__ acc, const rtf_node* __restrict__ nodes,
                     const float* __restrict__ w, const float* __restrict__ R,
                     const rtf_dist* __restrict__ dists, int D, int64_t N, int64_t Nw,
                     double* G) {
  __shared__ int dfirst_s, dlast_s;
  __shared__ float part[kBwThreads / 32];
  const int64_t t0 = (int64_t)blockIdx.x * kBwTile;
  const int64_t t1 = min(t0 + (int64_t)kBwTile, N);
  if (threadIdx.x == 0) {
    dfirst_s = find_dist(dists, 0, D - 1, t0);
    dlast_s = find_dist(dists, dfirst_s, min(D - 1, dfirst_s + kBwTile), t1 - 1);
  }
  __syncthreads();
  const int dfirst = dfirst_s, dlast = dlast_s;
  const int64_t e0 = t0 + (int64_t)threadIdx.x * kBwPer;
  int d = dfirst;
  if (e0 < t1 && dlast != dfirst) d = find_dist(dists, dfirst, dlast, e0);
  float run = 0.f;
  if (e0 < t1) {
    rtf_dist P = dists[d];
    int64_t end = P.elem_off + P.n;
    float invT = 1.0f / u64_to_f32(P.total);
    uint64_t cnext = nodes[e0].cdf;
    const int64_t e1 = min(e0 + (int64_t)kBwPer, t1);
    for (int64_t e = e0; e < e1; ++e) {
      if (e >= end) {
        if (dlast != dfirst) atomicAdd(G + d, (double)run);
        run = 0.f;
        ++d;
        P = dists[d];
        end = P.elem_off + P.n;
        invT = 1.0f / u64_to_f32(P.total);
      }
      const uint64_t c = cnext;
      cnext = (e + 1 < N) ? nodes[e + 1].cdf : 0ull;
      const uint64_t cup = (e + 1 < end) ? cnext : P.total;
      const float2 ax = acc[e];
      if (ax.x != 0.0f || ax.y != 0.0f) {
        const float cf = u64_to_f32(c) * invT;
        const float qf = u64_to_f32(cup - c) * invT;
        run += (ax.x * cf + ax.y * qf) / weight_at(w, R, Nw, e);
      }
    }
  }
  if (dlast != dfirst) {
    if (e0 < t1) atomicAdd(G + d, (double)run);
    return;
  }
  // the whole block lies in one distribution
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) run += __shfl_xor_sync(0xffffffffu, run, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = run;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kBwThreads / 32; ++k) t += (double)part[k];
    atomicAdd(G + dfirst, t);
  }
}

// Reverse segmented scan: S_k = sum_{i > k, same distribution} A_i / w_i, then
// the gradient.  Tiles are taken from the end by ticket; each tile publishes
// the sum of a over its first piece (the part of dist(t0) inside the tile)
// and, once known, that sum plus everything after it.  The lookback is
// block-wide: every thread reads one successor's flag per round.
__global__ void __launch_bounds__(kBwThreads)
    suffix_kernel(const float2* __restrict__ acc, const float* __restrict__ w,
                  const float* __restrict__ R, const rtf_dist* __restrict__ dists, int D,
                  int64_t N, int64_t Nw, const double* __restrict__ G, uint32_t* flags,
                  double* carry, double* incl, uint32_t* ticket, float* grad_w, float* gradR,
                  uint32_t* status) {
  __shared__ uint32_t tick_s;
  __shared__ int dfirst_s;
  __shared__ float ex_s[kBwThreads];
  __shared__ int exf_s[kBwThreads];
  __shared__ int first_prefix_s, first_invalid_s;
  __shared__ double part_s[kBwThreads / 32];
  __shared__ double E_s;
  if (threadIdx.x == 0) tick_s = atomicAdd(ticket, 1u);
  __syncthreads();
  const int64_t ntiles = (N + kBwTile - 1) / kBwTile;
  const int64_t tile = ntiles - 1 - (int64_t)tick_s;
  const int64_t t0 = tile * kBwTile, t1 = min(t0 + (int64_t)kBwTile, N);
  if (threadIdx.x == 0) dfirst_s = find_dist(dists, 0, D - 1, t0);
  __syncthreads();
  const int dfirst = dfirst_s;
  const int64_t e0 = t0 + (int64_t)threadIdx.x * kBwPer;

  // per-thread values; tails mark the last element of a distribution
  float a[kBwPer], b[kBwPer];
  int dk[kBwPer];
  uint32_t tailmask = 0;
  {
    int d = dfirst;
    if (e0 < t1) d = find_dist(dists, dfirst, min(D - 1, dfirst + kBwTile), e0);
#pragma unroll
    for (int k = 0; k < kBwPer; ++k) {
      const int64_t e = e0 + k;
      a[k] = 0.f;
      b[k] = 0.f;
      dk[k] = d;
      if (e < t1) {
        while (d + 1 < D && e >= dists[d + 1].elem_off) ++d;
        dk[k] = d;
        const float2 v = acc[e];
        if (v.x != 0.0f || v.y != 0.0f) {
          const float inv = 1.0f / weight_at(w, R, Nw, e);
          a[k] = v.x * inv;
          b[k] = v.y * inv;
        }
        const int64_t end = dists[d].elem_off + dists[d].n;
        if (e + 1 == end) tailmask |= 1u << k;
      }
    }
  }
  // thread aggregate continuing leftwards: sum of a from the first element up
  // to the first tail (or the whole run)
  float tot = 0.f;
#pragma unroll
  for (int k = kBwPer - 1; k >= 0; --k) {
    if (tailmask & (1u << k)) tot = 0.f;
    tot += a[k];
  }
  // segmented inclusive scan over reversed thread order: slot i holds thread
  // n-1-i, so slots run from the right end of the tile to the left
  const int myslot = kBwThreads - 1 - threadIdx.x;
  ex_s[myslot] = tot;
  exf_s[myslot] = tailmask ? 1 : 0;
  __syncthreads();
  {
    const int slot = threadIdx.x;
    float v = ex_s[slot];
    int f = exf_s[slot];
    for (int dlt = 1; dlt < kBwThreads; dlt <<= 1) {
      float pv = 0.f;
      int pf = 0;
      if (slot >= dlt) {
        pv = ex_s[slot - dlt];
        pf = exf_s[slot - dlt];
      }
      __syncthreads();
      if (slot >= dlt && !f) {
        v = pv + v;
        f = pf;
      }
      ex_s[slot] = v;
      exf_s[slot] = f;
      __syncthreads();
    }
  }
  float exv = 0.f;
  int exf = 0;
  if (myslot > 0) {
    exv = ex_s[myslot - 1];
    exf = exf_s[myslot - 1];
  }
  const float first_piece = ex_s[kBwThreads - 1];
  const bool first_piece_closed = exf_s[kBwThreads - 1] != 0;  // dist(t0) ends in this tile
  const int dlast_tile = find_dist(dists, dfirst, min(D - 1, dfirst + kBwTile), t1 - 1);
  const bool continues = (dists[dlast_tile].elem_off + dists[dlast_tile].n) > t1;
  if (threadIdx.x == 0) {
    carry[tile] = (double)first_piece;
    incl[tile] = (double)first_piece;
    __threadfence();
    atomicExch(flags + tile, first_piece_closed ? 2u : 1u);
  }
  // block-wide lookback for the incoming carry: sum of a beyond t1 in dist(t1-1)
  double E = 0.0;
  if (continues) {
    int64_t look = tile + 1;
    long long spins = 0;
    while (look < ntiles) {
      if (threadIdx.x == 0) {
        first_prefix_s = kBwThreads;
        first_invalid_s = kBwThreads;
      }
      __syncthreads();
      const int64_t idx = look + threadIdx.x;
      const uint32_t fl = idx < ntiles ? *((volatile uint32_t*)(flags + idx)) : 2u;
      if (fl == 2) atomicMin(&first_prefix_s, (int)threadIdx.x);
      if (fl == 0) atomicMin(&first_invalid_s, (int)threadIdx.x);
      __syncthreads();
      const int p = first_prefix_s, q = first_invalid_s;
      if (q < p) {
        if (++spins > kSpinLimit) {
          if (threadIdx.x == 0) raise_status(status, RTF_STATUS_TIMEOUT);
          break;
        }
        __nanosleep(64);
        __syncthreads();
        continue;
      }
      __threadfence();
      double v = 0.0;
      if ((int)threadIdx.x < p && idx < ntiles) v = *((volatile double*)(carry + idx));
      if ((int)threadIdx.x == p && idx < ntiles) v = *((volatile double*)(incl + idx));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) part_s[threadIdx.x >> 5] = v;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kBwThreads / 32; ++k) t += part_s[k];
        E_s = t;
      }
      __syncthreads();
      E += E_s;
      if (p < kBwThreads) break;
      look += kBwThreads;
    }
  }
  if (threadIdx.x == 0 && !first_piece_closed) {
    incl[tile] = (double)first_piece + E;
    __threadfence();
    atomicExch(flags + tile, 2u);
  }
  if (e0 >= t1) return;
  // element results, walking the thread's run from the right: until the first
  // tail the suffix continues past the thread (exclusive value, plus the
  // incoming carry when no tail lies to the right inside the tile)
  const double after = exf ? (double)exv : (double)exv + E;
  float inrun = 0.f;
  float base = (float)(G[dk[kBwPer - 1]] - after);
#pragma unroll
  for (int k = kBwPer - 1; k >= 0; --k) {
    const int64_t e = e0 + k;
    if (e >= t1) continue;
    if (tailmask & (1u << k)) {
      inrun = 0.f;
      base = (float)G[dk[k]];
    }
    const float gk = base - inrun - b[k];
    if (e < Nw)
      grad_w[e] = gk;
    else
      gradR[e - Nw] = gk;
    inrun += a[k];
  }
}

// One distribution (no segment ends inside the array but its last element):
// the same reverse decoupled-lookback scan and the same per-element
// arithmetic as suffix_kernel, with the tile scanned by warp shuffles instead
// of a segmented shared-memory scan and the inputs read as 16-byte vectors.
__global__ void __launch_bounds__(kBwThreads)
    suffix_single_kernel(const float2* __restrict__ acc, const float* __restrict__ w, int64_t N,
                         const double* __restrict__ G, uint32_t* flags, double* carry,
                         double* incl, uint32_t* ticket, float* grad_w, uint32_t* status) {
  __shared__ uint32_t tick_s;
  __shared__ float wtot_s[kBwThreads / 32];
  __shared__ int first_prefix_s, first_invalid_s;
  __shared__ double part_s[kBwThreads / 32];
  __shared__ double E_s;
  if (threadIdx.x == 0) tick_s = atomicAdd(ticket, 1u);
  __syncthreads();
  const int64_t ntiles = (N + kBwTile - 1) / kBwTile;
  const int64_t tile = ntiles - 1 - (int64_t)tick_s;
  const int64_t t0 = tile * kBwTile, t1 = min(t0 + (int64_t)kBwTile, N);
  const int64_t e0 = t0 + (int64_t)threadIdx.x * kBwPer;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

  float a[kBwPer], b[kBwPer];
  if (e0 + kBwPer <= t1) {
    const float4* av = reinterpret_cast<const float4*>(acc + e0);
    const float4* wv = reinterpret_cast<const float4*>(w + e0);
#pragma unroll
    for (int h = 0; h < kBwPer / 4; ++h) {
      const float4 x0 = av[2 * h], x1 = av[2 * h + 1], ww = wv[h];
      const float ax[4] = {x0.x, x0.z, x1.x, x1.z}, bx[4] = {x0.y, x0.w, x1.y, x1.w};
      const float wk[4] = {ww.x, ww.y, ww.z, ww.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        a[4 * h + k] = 0.f;
        b[4 * h + k] = 0.f;
        if (ax[k] != 0.0f || bx[k] != 0.0f) {
          const float inv = 1.0f / wk[k];
          a[4 * h + k] = ax[k] * inv;
          b[4 * h + k] = bx[k] * inv;
        }
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < kBwPer; ++k) {
      a[k] = 0.f;
      b[k] = 0.f;
      const int64_t e = e0 + k;
      if (e < t1) {
        const float2 v = acc[e];
        if (v.x != 0.0f || v.y != 0.0f) {
          const float inv = 1.0f / w[e];
          a[k] = v.x * inv;
          b[k] = v.y * inv;
        }
      }
    }
  }
  float tot = 0.f;
#pragma unroll
  for (int k = kBwPer - 1; k >= 0; --k) tot += a[k];
  // sum of the thread totals after this thread: within the warp by shuffles,
  // then over the warps after this one
  float v = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_down_sync(0xffffffffu, v, o);
    if (lane + o < 32) v += y;
  }
  if (lane == 0) wtot_s[wid] = v;
  __syncthreads();
  float exv = v - tot;
  float tile_tot = 0.f;
#pragma unroll
  for (int k = kBwThreads / 32 - 1; k >= 0; --k) {
    if (k > wid) exv += wtot_s[k];
    tile_tot += wtot_s[k];
  }
  const bool last_tile = t1 == N;  // the distribution's last element lies here
  if (threadIdx.x == 0) {
    carry[tile] = (double)tile_tot;
    incl[tile] = (double)tile_tot;
    __threadfence();
    atomicExch(flags + tile, last_tile ? 2u : 1u);
  }
  // block-wide lookback for the sum beyond t1 (as in suffix_kernel)
  double E = 0.0;
  if (!last_tile) {
    int64_t look = tile + 1;
    long long spins = 0;
    while (look < ntiles) {
      if (threadIdx.x == 0) {
        first_prefix_s = kBwThreads;
        first_invalid_s = kBwThreads;
      }
      __syncthreads();
      const int64_t idx = look + threadIdx.x;
      const uint32_t fl = idx < ntiles ? *((volatile uint32_t*)(flags + idx)) : 2u;
      if (fl == 2) atomicMin(&first_prefix_s, (int)threadIdx.x);
      if (fl == 0) atomicMin(&first_invalid_s, (int)threadIdx.x);
      __syncthreads();
      const int pfx = first_prefix_s, inv = first_invalid_s;
      if (inv < pfx) {
        if (++spins > kSpinLimit) {
          if (threadIdx.x == 0) raise_status(status, RTF_STATUS_TIMEOUT);
          break;
        }
        __nanosleep(64);
        __syncthreads();
        continue;
      }
      __threadfence();
      double x = 0.0;
      if ((int)threadIdx.x < pfx && idx < ntiles) x = *((volatile double*)(carry + idx));
      if ((int)threadIdx.x == pfx && idx < ntiles) x = *((volatile double*)(incl + idx));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) part_s[wid] = x;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kBwThreads / 32; ++k) t += part_s[k];
        E_s = t;
      }
      __syncthreads();
      E += E_s;
      if (pfx < kBwThreads) break;
      look += kBwThreads;
    }
    if (threadIdx.x == 0) {
      incl[tile] = (double)tile_tot + E;
      __threadfence();
      atomicExch(flags + tile, 2u);
    }
  }
  if (e0 >= t1) return;
  const float base = (float)(G[0] - ((double)exv + E));
  float inrun = 0.f;
  float gk[kBwPer];
#pragma unroll
  for (int k = kBwPer - 1; k >= 0; --k) {
    gk[k] = base - inrun - b[k];
    inrun += a[k];
  }
  if (e0 + kBwPer <= t1) {
    float4* gv = reinterpret_cast<float4*>(grad_w + e0);
#pragma unroll
    for (int h = 0; h < kBwPer / 4; ++h)
      gv[h] = make_float4(gk[4 * h], gk[4 * h + 1], gk[4 * h + 2], gk[4 * h + 3]);
  } else {
#pragma unroll
    for (int k = 0; k < kBwPer; ++k)
      if (e0 + k < t1) grad_w[e0 + k] = gk[k];
  }
}

__global__ void add_row_kernel(float* grad_w, const rtf_dist* __restrict__ dists, int H,
                               const float* __restrict__ gradR) {
  for (int r = blockIdx.x; r < H; r += gridDim.x) {
    const int64_t off = dists[r].elem_off, n = dists[r].n;
    const float gr = gradR[r];
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) grad_w[off + k] += gr;
  }
}

static int bw_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 148;
}

size_t backward_ws_bytes(int64_t N, int32_t D) { return bw_layout(N, D).total; }

static int64_t bw_l2_bytes() {
  int dev = 0, l2 = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  return l2 > 0 ? l2 : (int64_t(126) << 20);
}

// Passes of the 1-D scatter over the samples, each adding into one half of
// the bins.  When the per-bin sums (8 bytes per bin) exceed 3/4 of L2 the
// passing sample stream evicts them; two passes keep each half resident at the
// price of reading the samples twice, which pays with at least 4 samples per
// bin.  The whole backward of 2^28 samples on GB300 (L2 135.5 MB), one pass ->
// two passes: 2^23 bins 1.90 -> 2.33 ms (so one pass there), 2^24 bins 3.17 ->
// 2.54 ms, 2^25 bins 6.11 -> 4.01 ms; of 2^27 tagged samples into 1.19e8 bins
// (about one per bin) 6.97 -> 7.03 ms (so one pass there); three passes at
// 2^24 bins 3.48 ms.
static int scatter_passes(int64_t N, int64_t count) {
  const int64_t sums = N * (int64_t)sizeof(float2);
  return (4 * sums > 3 * bw_l2_bytes() && count >= 4 * N) ? 2 : 1;
}

// The backward in three steps: clear the per-bin sums, add the samples' terms
// (any number of times), turn the sums into the gradient.
struct BwPtrs {
  BwLayout L;
  char* base;
  float2* acc;
};

static BwPtrs bw_ptrs(const rtf_forest* f, void* ws) {
  BwPtrs p;
  p.L = bw_layout(f->num_elems, f->num_dists);
  p.base = static_cast<char*>(ws);
  p.acc = reinterpret_cast<float2*>(p.base + p.L.acc);
  return p;
}

cudaError_t launch_backward_begin(const rtf_forest* f, void* ws, cudaStream_t st) {
  const BwPtrs p = bw_ptrs(f, ws);
  return cudaMemsetAsync(p.base, 0, p.L.zero_end, st);
}

cudaError_t launch_backward_accumulate(const rtf_forest* f, const int32_t* dist_id,
                                       const int32_t* idx, const float* pos, const float* gpos,
                                       int64_t count, int mode, void* ws, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const BwPtrs p = bw_ptrs(f, ws);
  const int D = f->num_dists;
  const int sms = bw_sms();
  const int64_t blocks = std::min<int64_t>((int64_t)sms * 8, (count + kBwThreads - 1) / kBwThreads);
  if (mode == RTF_SAMPLE_2D)
    scatter_2d_kernel<<<(unsigned)blocks, kBwThreads, 0, st>>>(
        f->dists, D, reinterpret_cast<const int2*>(idx), reinterpret_cast<const float2*>(pos),
        reinterpret_cast<const float2*>(gpos), count, p.acc);
  else {
    const int64_t N = f->num_elems;
    const int passes = scatter_passes(N, count);
    for (int k = 0; k < passes; ++k)
      scatter_1d_kernel<<<(unsigned)blocks, kBwThreads, 0, st>>>(
          f->dists, D, dist_id, idx, pos, gpos, count, p.acc, N * k / passes, N * (k + 1) / passes);
  }
  return cudaGetLastError();
}

cudaError_t launch_backward_finish(const rtf_forest* f, const float* w, int mode, float* grad_w,
                                   void* ws, cudaStream_t st) {
  const BwPtrs p = bw_ptrs(f, ws);
  const BwLayout& L = p.L;
  const int64_t N = f->num_elems;
  const int D = f->num_dists;
  const bool two_d = mode == RTF_SAMPLE_2D;
  double* G = reinterpret_cast<double*>(p.base + L.G);
  uint32_t* flags = reinterpret_cast<uint32_t*>(p.base + L.flags);
  double* carry = reinterpret_cast<double*>(p.base + L.carry);
  double* incl = reinterpret_cast<double*>(p.base + L.incl);
  uint32_t* ticket = reinterpret_cast<uint32_t*>(p.base + L.ticket);
  float* R = reinterpret_cast<float*>(p.base + L.R);
  float* gradR = reinterpret_cast<float*>(p.base + L.gradR);
  const int64_t Nw = two_d ? N - (D - 1) : N;
  const int sms = bw_sms();
  if (two_d) {
    row_sum_kernel<<<(unsigned)std::min<int64_t>(sms * 4, (D + 7) / 8), 256, 0, st>>>(
        w, f->dists, D - 1, R);
  }
  const int64_t tiles = (N + kBwTile - 1) / kBwTile;
  bin_total_kernel<<<(unsigned)tiles, kBwThreads, 0, st>>>(p.acc, f->nodes, w, R, f->dists, D, N,
                                                           Nw, G);
  const bool vec_ok = (reinterpret_cast<uintptr_t>(w) & 15) == 0 &&
                      (reinterpret_cast<uintptr_t>(grad_w) & 15) == 0;
  if (D == 1 && !two_d && vec_ok)
    suffix_single_kernel<<<(unsigned)tiles, kBwThreads, 0, st>>>(p.acc, w, N, G, flags, carry,
                                                                 incl, ticket, grad_w, f->status);
  else
    suffix_kernel<<<(unsigned)tiles, kBwThreads, 0, st>>>(p.acc, w, R, f->dists, D, N, Nw, G,
                                                          flags, carry, incl, ticket, grad_w,
                                                          gradR, f->status);
  if (two_d)
    add_row_kernel<<<(unsigned)std::min<int64_t>(sms * 4, D - 1), 256, 0, st>>>(
        grad_w, f->dists, D - 1, gradR);
  return cudaGetLastError();
}

cudaError_t launch_backward(const rtf_forest* f, const float* w, const uint32_t* u,
                            const int32_t* dist_id, const int32_t* idx, const float* pos,
                            const float* gpos, int64_t count, int mode, float* grad_w, void* ws,
                            cudaStream_t st) {
  (void)u;  // xi follows exactly from the bin and the position (see the file comment)
  cudaError_t e;
  if ((e = launch_backward_begin(f, ws, st))) return e;
  if ((e = launch_backward_accumulate(f, dist_id, idx, pos, gpos, count, mode, ws, st))) return e;
  return launch_backward_finish(f, w, mode, grad_w, ws, st);
}

}  // namespace rtf
