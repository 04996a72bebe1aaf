// Gradient of the in-bin sample positions with respect to the weights (not in
// the paper).  The forward computes x = (xi T - C_i) / q_i on the quantised
// weights q_i = floor(w_i 2^S); its gradient is taken with the floor passed
// straight through and the scale S held fixed, i.e. the relaxation
// x = (xi W' - C'_i) / w'_i at the quantised weights w'_k = q_k 2^-S
// (W' = sum w', C'_i = sum_{k<i} w'_k), with the bin i of each sample fixed:
//
//   dL/dw_k = sum_{i in d} Xi_i / w'_i  -  sum_{i > k, i in d} A_i / w'_i  -  X_k / w'_k
//   A_i = sum_{s -> i} g_s,  X_i = sum_{s -> i} g_s x_s,  Xi_i = sum_{s -> i} g_s xi_s.
//
// The sample's own xi need not be carried: the position is defined through
// the exact integer CDF, u / 2^32 = (C_i + x q_i) / T, so
// Xi_i = (A_i C_i + X_i q_i) / T with the integers of the built structure.
// Only two sums per bin are accumulated.
//
// Kernels:
//   row_total_kernel     (2-D) the marginal's weights in real units,
//                        R'_r = T_r 2^-S (T_r the exact integer row total)
//   scatter kernels      one 8-byte vector atomic {g, g x} per sample into its
//                        bin, runs of equal bins inside a warp merged first
//   bin_total_kernel     G_d = sum_{i in d} Xi_i / w'_i per distribution
//   suffix_kernel        reverse decoupled-lookback scan of A_i / w'_i per
//                        distribution (double-floats in the tile and in the
//                        carries between tiles), then
//                        dL/dw_k = G_d - S_k - X_k / w'_k
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
  size_t carry;  // float2 [tiles]   sum of a over a tile's first piece (double-float)
  size_t incl;   // float2 [tiles]   that sum plus everything after it
  size_t ticket; // u32
  size_t zero_end;
  size_t R;      // float2 [D]  (2-D: row totals as double-floats)
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
  L.R = o; o = align256(o + 8 * (size_t)D);
  L.gradR = o; o = align256(o + 4 * (size_t)D);
  L.total = o;
  return L;
}

// The quantised weight in real units, w' = floor(w 2^S) 2^-S: w with the bits
// of its significand below 2^-S cleared (exact; 0 when w 2^S < 1).  w >= 0.
__device__ __forceinline__ float quantized_weight(float w, int S) {
  const uint32_t b = __float_as_uint(w) & 0x7FFFFFFFu;
  const uint32_t E = b >> 23;
  const int lsb = (E ? (int)E : 1) - 150;  // exponent of the significand's last bit
  const int sh = -S - lsb;                 // significand bits below 2^-S
  if (sh <= 0) return __uint_as_float(b);
  if (sh >= 24) return 0.0f;
  return __uint_as_float(b & ~((1u << sh) - 1u));
}

// ---------------------------------------------------------------------------
// double-float arithmetic
// ---------------------------------------------------------------------------
// A value held as the unevaluated sum hi + lo of two floats (about 48
// significant bits), built from error-free transformations: the sum of two
// floats together with its exact rounding error (Knuth's TwoSum, The Art of
// Computer Programming vol. 2, Sec. 4.2.2), and the exact residual of a
// product or a quotient by one fused multiply-add.  Every step rounds
// explicitly (__fadd_rn, __fmul_rn, __fmaf_rn) so that the compiler cannot
// contract it.  Why: the per-bin terms A_i / w'_i span many orders of
// magnitude (those of the narrowest bins reach 1e5 and more at n = 2^24); in
// float32 their rounding errors, which the suffix carries to every element
// left of them, exceed the gradient's relative error bound wherever
// G - S_k nearly cancels.  fp64 is kept to per-thread and per-tile values (its
// throughput on this part is low).
struct dflt {
  float hi, lo;
};

__device__ __forceinline__ dflt df_zero() { return dflt{0.0f, 0.0f}; }

__device__ __forceinline__ dflt df_add(dflt a, dflt b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float h = __fadd_rn(s, e);
  return dflt{h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ dflt df_sub(dflt a, dflt b) { return df_add(a, dflt{-b.hi, -b.lo}); }

__device__ __forceinline__ dflt df_mul(dflt a, dflt b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float h = __fadd_rn(p, e);
  return dflt{h, __fsub_rn(e, __fsub_rn(h, p))};
}

// x / (yh + yl) with inv ~ 1 / yh: the quotient estimate q, the residual
// x - q yh (exact) - q yl, and its correction.
__device__ __forceinline__ dflt df_div(float x, float yh, float yl, float inv) {
  const float q = __fmul_rn(x, inv);
  float r = __fmaf_rn(-q, yh, x);
  r = __fmaf_rn(-q, yl, r);
  const float c = __fmul_rn(r, inv);
  const float h = __fadd_rn(q, c);
  return dflt{h, __fsub_rn(c, __fsub_rn(h, q))};
}

__device__ __forceinline__ double df_to_double(dflt a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ dflt df_from_double(double x) {
  const float h = __double2float_rn(x);
  return dflt{h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ float df_to_float(dflt a) { return __fadd_rn(a.hi, a.lo); }

// Conversions from 64-bit integers without the fp64 unit: on this part 64-bit
// conversions run on the fp64 pipe, whose rate is a small fraction of the
// fp32 one, so one conversion per element made the backward's bin totals
// fp64-bound.  An integer below 2^23 becomes a float exactly by placing it in
// the significand of 2^23 and subtracting 2^23.
__device__ __forceinline__ float small_to_float(uint32_t x) {
  return __fsub_rn(__uint_as_float(0x4B000000u | x), 8388608.0f);
}

// q exactly, for q with at most 24 significant bits (a quantised weight of a
// float: floor(w 2^S)).  Horner over 16-bit pieces: every partial value is q
// shifted right, which keeps at most 24 significant bits, so each step is exact.
__device__ __forceinline__ float float_of_q24(uint64_t q) {
  const uint32_t hi = (uint32_t)(q >> 32), lo = (uint32_t)q;
  float f = small_to_float(hi >> 16);
  f = __fmaf_rn(f, 65536.0f, small_to_float(hi & 0xFFFFu));
  f = __fmaf_rn(f, 65536.0f, small_to_float(lo >> 16));
  return __fmaf_rn(f, 65536.0f, small_to_float(lo & 0xFFFFu));
}

// An integer below 2^63 as a double-float (relative error about 2^-47): three
// exact 21-bit pieces added with error-free sums.
__device__ __forceinline__ dflt df_from_u64(uint64_t x) {
  const float a = __fmul_rn(small_to_float((uint32_t)(x >> 42)), 4398046511104.0f);  // 2^42
  const float b = __fmul_rn(small_to_float((uint32_t)(x >> 21) & 0x1FFFFFu), 2097152.0f);  // 2^21
  const float c = small_to_float((uint32_t)x & 0x1FFFFFu);
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_add(dflt{s, e}, dflt{c, 0.0f});
}

__device__ __forceinline__ dflt df_shfl_down(dflt a, int d) {
  return dflt{__shfl_down_sync(0xffffffffu, a.hi, d), __shfl_down_sync(0xffffffffu, a.lo, d)};
}

__device__ __forceinline__ dflt df_shfl_xor(dflt a, int d) {
  return dflt{__shfl_xor_sync(0xffffffffu, a.hi, d), __shfl_xor_sync(0xffffffffu, a.lo, d)};
}

// The quantised weight q 2^-S of an integer weight q (a row weight, exact in
// the high part, or the marginal's row total) as a double-float.
__device__ __forceinline__ dflt qweight_df(uint64_t q, int S) {
  const dflt v = df_from_u64(q);
  return dflt{scalbnf(v.hi, -S), scalbnf(v.lo, -S)};
}

// 2^-S as a float, exact for S <= 126; 0 otherwise (the caller then scales
// with scalbnf).
__device__ __forceinline__ float pow2_neg(int S) {
  return (S >= -127 && S <= 126) ? __int_as_float((127 - S) << 23) : 0.0f;
}

// Reciprocal estimate (relative error below 2^-22, subnormals kept); the
// residual step of df_div makes the quotient accurate to about 2^-44.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// {a, b} = {A / w', X / w'} for the per-bin sums {A, X} and the quantised
// weight w' = wh + wl (zero for an empty bin or a zero weight).
__device__ __forceinline__ void bin_terms(float2 ax, float wh, float wl, dflt* a, dflt* b) {
  if ((ax.x != 0.0f || ax.y != 0.0f) && wh != 0.0f) {
    const float inv = rcp_approx(wh);
    *a = df_div(ax.x, wh, wl, inv);
    *b = df_div(ax.y, wh, wl, inv);
  } else {
    *a = df_zero();
    *b = df_zero();
  }
}

// ---------------------------------------------------------------------------
// R'_r = T_r 2^-S: the marginal's weights in the units of the map's weights,
// as double-floats {hi, lo}.
__global__ void row_total_kernel(const rtf_dist* __restrict__ dists, int H, float2* R) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < H; r += gridDim.x * blockDim.x) {
    const dflt v = qweight_df(dists[r].total, dists[r].scale);
    R[r] = make_float2(v.hi, v.lo);
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

// G_d = sum_{i in d} Xi_i / w'_i.  With Xi_i = (A_i C_i + X_i q_i) / T and
// q_i / w'_i = 2^S, each term is a_i c_i + X_i 2^S / T with a_i = A_i / w'_i
// and c_i = C_i / T, so G_d = sum_i a_i c_i + (2^S / T) sum_i X_i: both sums
// in double-float per thread, fp64 per distribution piece (one atomic per
// piece; a block inside one distribution reduces first and adds once).
__global__ void __launch_bounds__(kBwThreads)
    bin_total_kernel(const float2* __restrict__ acc, const rtf_node* __restrict__ nodes,
                     const float* __restrict__ w, const rtf_dist* __restrict__ dists, int D,
                     int64_t N, double* G) {
  __shared__ int dfirst_s, dlast_s;
  __shared__ double part[kBwThreads / 32];
  __shared__ dflt invT_s, K_s;
  const int64_t t0 = (int64_t)blockIdx.x * kBwTile;
  const int64_t t1 = min(t0 + (int64_t)kBwTile, N);
  if (threadIdx.x == 0) {
    const int df = find_dist(dists, 0, D - 1, t0);
    dfirst_s = df;
    dlast_s = find_dist(dists, df, min(D - 1, df + kBwTile), t1 - 1);
    // 1 / T and 2^S / T of the block's first distribution, once per block (fp64
    // divisions are slow on this part)
    const double T = (double)dists[df].total;
    invT_s = df_from_double(1.0 / T);
    K_s = df_from_double(ldexp(1.0, dists[df].scale) / T);
  }
  __syncthreads();
  const int dfirst = dfirst_s, dlast = dlast_s;
  const int64_t e0 = t0 + (int64_t)threadIdx.x * kBwPer;
  int d = dfirst;
  if (e0 < t1 && dlast != dfirst) d = find_dist(dists, dfirst, dlast, e0);
  dflt contrib = df_zero();
  if (e0 < t1) {
    rtf_dist P = dists[d];
    int64_t end = P.elem_off + P.n;
    dflt invT = invT_s, K = K_s;
    if (d != dfirst) {
      invT = df_from_double(1.0 / (double)P.total);
      K = df_from_double(ldexp(1.0, P.scale) / (double)P.total);
    }
    bool marg = (P.flags & kDistMarginal) != 0;
    float p2 = pow2_neg(P.scale);
    dflt sac = df_zero(), sx = df_zero();
    if (dlast == dfirst && e0 + kBwPer <= t1 && !marg) {
      // the usual case, a whole run inside one distribution of float
      // weights: every load of the run issued first; the quantised weights
      // w' = q 2^-S come from the weights (4 bytes each, instead of the CDF
      // differences from the 16-byte node records), C only at the run's start
      const uint64_t c0 = nodes[e0].cdf;
      float wv[kBwPer];
      if ((reinterpret_cast<uintptr_t>(w + e0) & 15) == 0) {
#pragma unroll
        for (int h = 0; h < kBwPer / 4; ++h) {
          const float4 x = reinterpret_cast<const float4*>(w + e0)[h];
          wv[4 * h] = x.x;
          wv[4 * h + 1] = x.y;
          wv[4 * h + 2] = x.z;
          wv[4 * h + 3] = x.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < kBwPer; ++k) wv[k] = w[e0 + k];
      }
      float2 ax[kBwPer];
#pragma unroll
      for (int k = 0; k < kBwPer; ++k) ax[k] = acc[e0 + k];
      const float pS = pow2_neg(-P.scale);  // 2^S, or 0 outside the float exponent range
      dflt Cd = df_from_u64(c0);
#pragma unroll
      for (int k = 0; k < kBwPer; ++k) {
        const float wq = quantized_weight(wv[k], P.scale);
        const float qf = pS != 0.0f ? wq * pS : scalbnf(wq, P.scale);  // q, exact
        if ((ax[k].x != 0.0f || ax[k].y != 0.0f) && wq != 0.0f) {
          dflt av, bv;
          bin_terms(ax[k], wq, 0.0f, &av, &bv);
          sac = df_add(sac, df_mul(av, df_mul(Cd, invT)));
          sx = df_add(sx, dflt{ax[k].y, 0.0f});
        }
        Cd = df_add(Cd, dflt{qf, 0.0f});
      }
      contrib = df_add(sac, df_mul(K, sx));
    } else {
      uint64_t cnext = nodes[e0].cdf;
      // C_e as a double-float, carried along the run (C_{e+1} = C_e + q_e; a
      // row's q_e is one exact float): one 64-bit conversion per run
      dflt Cd = df_from_u64(cnext);
      const int64_t e1 = min(e0 + (int64_t)kBwPer, t1);
      for (int64_t e = e0; e < e1; ++e) {
        if (e >= end) {
          if (dlast != dfirst) atomicAdd(G + d, df_to_double(df_add(sac, df_mul(K, sx))));
          sac = df_zero();
          sx = df_zero();
          ++d;
          P = dists[d];
          end = P.elem_off + P.n;
          invT = df_from_double(1.0 / (double)P.total);
          K = df_from_double(ldexp(1.0, P.scale) / (double)P.total);
          marg = (P.flags & kDistMarginal) != 0;
          p2 = pow2_neg(P.scale);
          Cd = df_zero();  // a new distribution starts at C = 0
        }
        const uint64_t c = cnext;
        cnext = (e + 1 < N) ? nodes[e + 1].cdf : 0ull;
        const uint64_t cup = (e + 1 < end) ? cnext : P.total;
        const float2 ax = acc[e];
        const uint64_t q = cup - c;
        // a row weight's q has at most 24 significant bits: q and w' are exact floats
        const dflt qd = marg ? df_from_u64(q) : dflt{float_of_q24(q), 0.0f};
        if ((ax.x != 0.0f || ax.y != 0.0f) && q != 0) {
          dflt wq;
          if (marg)
            wq = qweight_df(q, P.scale);
          else
            wq = dflt{p2 != 0.0f ? qd.hi * p2 : scalbnf(qd.hi, -P.scale), 0.0f};
          dflt av, bv;
          bin_terms(ax, wq.hi, wq.lo, &av, &bv);
          sac = df_add(sac, df_mul(av, df_mul(Cd, invT)));
          sx = df_add(sx, dflt{ax.y, 0.0f});
        }
        Cd = df_add(Cd, qd);
      }
      contrib = df_add(sac, df_mul(K, sx));
    }
  }
  if (dlast != dfirst) {
    if (e0 < t1) atomicAdd(G + d, df_to_double(contrib));
    return;
  }
  // the whole block lies in one distribution: the warp's sum in double-float,
  // the block's in fp64
  dflt v = contrib;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = df_to_double(v);
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kBwThreads / 32; ++k) t += part[k];
    atomicAdd(G + dfirst, t);
  }
}

// Block-wide lookback of the reverse scan: the sum of the values published by
// the tiles after `tile`, the carries (sum over a tile's first piece) of those
// before the first tile whose inclusive value (its first piece plus
// everything after it) is published, plus that inclusive value.  Every thread
// reads one successor's flag per round; the values are double-floats {hi, lo}.
// Gives up after kSpinLimit rounds without progress (RTF_STATUS_TIMEOUT).
struct SuffixLookback {
  int first_prefix, first_invalid;
  dflt part[kBwThreads / 32];
  dflt E;
};

__device__ dflt suffix_lookback(SuffixLookback& sh, int64_t tile, int64_t ntiles,
                                const uint32_t* flags, const float2* carry, const float2* incl,
                                uint32_t* status) {
  dflt E = df_zero();
  int64_t look = tile + 1;
  long long spins = 0;
  while (look < ntiles) {
    if (threadIdx.x == 0) {
      sh.first_prefix = kBwThreads;
      sh.first_invalid = kBwThreads;
    }
    __syncthreads();
    const int64_t idx = look + threadIdx.x;
    const uint32_t fl = idx < ntiles ? *((volatile uint32_t*)(flags + idx)) : 2u;
    if (fl == 2) atomicMin(&sh.first_prefix, (int)threadIdx.x);
    if (fl == 0) atomicMin(&sh.first_invalid, (int)threadIdx.x);
    __syncthreads();
    const int pfx = sh.first_prefix, inv = sh.first_invalid;
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
    dflt x = df_zero();
    if ((int)threadIdx.x <= pfx && idx < ntiles) {
      // read through L2 (not L1), where the other blocks' stores are visible
      const float2 v = __ldcg((int)threadIdx.x < pfx ? carry + idx : incl + idx);
      x = dflt{v.x, v.y};
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = df_add(x, df_shfl_xor(x, o));
    if ((threadIdx.x & 31) == 0) sh.part[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      dflt t = df_zero();
      for (int k = 0; k < kBwThreads / 32; ++k) t = df_add(t, sh.part[k]);
      sh.E = t;
    }
    __syncthreads();
    E = df_add(E, sh.E);
    if (pfx < kBwThreads) break;
    look += kBwThreads;
  }
  return E;
}

// Reverse segmented scan: S_k = sum_{i > k, same distribution} A_i / w'_i, then
// the gradient.  Tiles are taken from the end by ticket; each tile publishes
// the sum of a over its first piece (the part of dist(t0) inside the tile)
// and, once known, that sum plus everything after it.  The lookback is
// block-wide: every thread reads one successor's flag per round.  Terms and
// sums inside the tile and the carries between tiles are double-floats.
__global__ void __launch_bounds__(kBwThreads)
    suffix_kernel(const float2* __restrict__ acc, const float* __restrict__ w,
                  const float2* __restrict__ R, const rtf_dist* __restrict__ dists, int D,
                  int64_t N, int64_t Nw, const double* __restrict__ G, uint32_t* flags,
                  float2* carry, float2* incl, uint32_t* ticket, float* grad_w, float* gradR,
                  uint32_t* status) {
  __shared__ uint32_t tick_s;
  __shared__ int dfirst_s;
  __shared__ float exh_s[kBwThreads], exl_s[kBwThreads];
  __shared__ int exf_s[kBwThreads];
  __shared__ SuffixLookback lb_s;
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
  dflt a[kBwPer], b[kBwPer];
  int dk[kBwPer];
  uint32_t tailmask = 0;
  {
    int d = dfirst;
    if (e0 < t1) d = find_dist(dists, dfirst, min(D - 1, dfirst + kBwTile), e0);
#pragma unroll
    for (int k = 0; k < kBwPer; ++k) {
      const int64_t e = e0 + k;
      a[k] = df_zero();
      b[k] = df_zero();
      dk[k] = d;
      if (e < t1) {
        while (d + 1 < D && e >= dists[d + 1].elem_off) ++d;
        dk[k] = d;
        const float2 v = acc[e];
        if (v.x != 0.0f || v.y != 0.0f) {
          float wh, wl = 0.0f;
          if (e < Nw) {
            wh = quantized_weight(w[e], dists[d].scale);
          } else {
            const float2 r2 = R[e - Nw];
            wh = r2.x;
            wl = r2.y;
          }
          bin_terms(v, wh, wl, &a[k], &b[k]);
        }
        const int64_t end = dists[d].elem_off + dists[d].n;
        if (e + 1 == end) tailmask |= 1u << k;
      }
    }
  }
  // thread aggregate continuing leftwards: sum of a from the first element up
  // to the first tail (or the whole run)
  dflt tot = df_zero();
#pragma unroll
  for (int k = kBwPer - 1; k >= 0; --k) {
    if (tailmask & (1u << k)) tot = df_zero();
    tot = df_add(tot, a[k]);
  }
  // segmented inclusive scan over reversed thread order: slot i holds thread
  // n-1-i, so slots run from the right end of the tile to the left
  const int myslot = kBwThreads - 1 - threadIdx.x;
  exh_s[myslot] = tot.hi;
  exl_s[myslot] = tot.lo;
  exf_s[myslot] = tailmask ? 1 : 0;
  __syncthreads();
  {
    const int slot = threadIdx.x;
    dflt v{exh_s[slot], exl_s[slot]};
    int f = exf_s[slot];
    for (int dlt = 1; dlt < kBwThreads; dlt <<= 1) {
      dflt pv = df_zero();
      int pf = 0;
      if (slot >= dlt) {
        pv = dflt{exh_s[slot - dlt], exl_s[slot - dlt]};
        pf = exf_s[slot - dlt];
      }
      __syncthreads();
      if (slot >= dlt && !f) {
        v = df_add(pv, v);
        f = pf;
      }
      exh_s[slot] = v.hi;
      exl_s[slot] = v.lo;
      exf_s[slot] = f;
      __syncthreads();
    }
  }
  dflt exv = df_zero();
  int exf = 0;
  if (myslot > 0) {
    exv = dflt{exh_s[myslot - 1], exl_s[myslot - 1]};
    exf = exf_s[myslot - 1];
  }
  const dflt first_piece{exh_s[kBwThreads - 1], exl_s[kBwThreads - 1]};
  const bool first_piece_closed = exf_s[kBwThreads - 1] != 0;  // dist(t0) ends in this tile
  const int dlast_tile = find_dist(dists, dfirst, min(D - 1, dfirst + kBwTile), t1 - 1);
  const bool continues = (dists[dlast_tile].elem_off + dists[dlast_tile].n) > t1;
  if (threadIdx.x == 0) {
    carry[tile] = make_float2(first_piece.hi, first_piece.lo);
    incl[tile] = make_float2(first_piece.hi, first_piece.lo);
    __threadfence();
    atomicExch(flags + tile, first_piece_closed ? 2u : 1u);
  }
  // block-wide lookback for the sum beyond t1 in the distribution of t1 - 1
  const dflt E = continues ? suffix_lookback(lb_s, tile, ntiles, flags, carry, incl, status)
                           : df_zero();
  if (threadIdx.x == 0 && !first_piece_closed) {
    const dflt v = df_add(first_piece, E);
    incl[tile] = make_float2(v.hi, v.lo);
    __threadfence();
    atomicExch(flags + tile, 2u);
  }
  if (e0 >= t1) return;
  // element results, walking the thread's run from the right: until the first
  // tail the suffix continues past the thread (exclusive value, plus the
  // incoming carry when no tail lies to the right inside the tile)
  const dflt after = exf ? exv : df_add(exv, E);
  dflt inrun = df_zero();
  dflt base = df_sub(df_from_double(G[dk[kBwPer - 1]]), after);
#pragma unroll
  for (int k = kBwPer - 1; k >= 0; --k) {
    const int64_t e = e0 + k;
    if (e >= t1) continue;
    if (tailmask & (1u << k)) {
      inrun = df_zero();
      base = df_from_double(G[dk[k]]);
    }
    const float gk = df_to_float(df_sub(df_sub(base, inrun), b[k]));
    if (e < Nw)
      grad_w[e] = gk;
    else
      gradR[e - Nw] = gk;
    inrun = df_add(inrun, a[k]);
  }
}

// One distribution (no segment ends inside the array but its last element):
// the same reverse decoupled-lookback scan and the same per-element
// arithmetic as suffix_kernel, with the tile scanned by warp shuffles instead
// of a segmented shared-memory scan and the inputs read as 16-byte vectors.
__global__ void __launch_bounds__(kBwThreads)
    suffix_single_kernel(const float2* __restrict__ acc, const float* __restrict__ w,
                         const rtf_dist* __restrict__ dists, int64_t N,
                         const double* __restrict__ G, uint32_t* flags, float2* carry,
                         float2* incl, uint32_t* ticket, float* grad_w, uint32_t* status) {
  __shared__ uint32_t tick_s;
  __shared__ dflt wtot_s[kBwThreads / 32];
  __shared__ SuffixLookback lb_s;
  __shared__ dflt G_s;
  if (threadIdx.x == 0) {
    tick_s = atomicAdd(ticket, 1u);
    G_s = df_from_double(G[0]);  // once per block (fp64 is slow on this part)
  }
  __syncthreads();
  const int64_t ntiles = (N + kBwTile - 1) / kBwTile;
  const int64_t tile = ntiles - 1 - (int64_t)tick_s;
  const int64_t t0 = tile * kBwTile, t1 = min(t0 + (int64_t)kBwTile, N);
  const int64_t e0 = t0 + (int64_t)threadIdx.x * kBwPer;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int S = dists[0].scale;

  dflt a[kBwPer], b[kBwPer];
  if (e0 + kBwPer <= t1) {
    const float4* av = reinterpret_cast<const float4*>(acc + e0);
    const float4* wv = reinterpret_cast<const float4*>(w + e0);
#pragma unroll
    for (int h = 0; h < kBwPer / 4; ++h) {
      const float4 x0 = av[2 * h], x1 = av[2 * h + 1], ww = wv[h];
      const float2 ax[4] = {make_float2(x0.x, x0.y), make_float2(x0.z, x0.w),
                            make_float2(x1.x, x1.y), make_float2(x1.z, x1.w)};
      const float wk[4] = {ww.x, ww.y, ww.z, ww.w};
#pragma unroll
      for (int k = 0; k < 4; ++k)
        bin_terms(ax[k], quantized_weight(wk[k], S), 0.0f, &a[4 * h + k], &b[4 * h + k]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < kBwPer; ++k) {
      a[k] = df_zero();
      b[k] = df_zero();
      const int64_t e = e0 + k;
      if (e < t1) bin_terms(acc[e], quantized_weight(w[e], S), 0.0f, &a[k], &b[k]);
    }
  }
  dflt tot = df_zero();
#pragma unroll
  for (int k = kBwPer - 1; k >= 0; --k) tot = df_add(tot, a[k]);
  // sum of the thread totals after this thread: within the warp by shuffles
  // (inclusive from the right, then shifted by one lane), then over the warps
  // after this one
  dflt v = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const dflt y = df_shfl_down(v, o);
    if (lane + o < 32) v = df_add(v, y);
  }
  dflt exv = df_shfl_down(v, 1);
  if (lane == 31) exv = df_zero();
  if (lane == 0) wtot_s[wid] = v;
  __syncthreads();
  dflt tile_tot = df_zero();
#pragma unroll
  for (int k = kBwThreads / 32 - 1; k >= 0; --k) {
    if (k > wid) exv = df_add(exv, wtot_s[k]);
    tile_tot = df_add(tile_tot, wtot_s[k]);
  }
  const bool last_tile = t1 == N;  // the distribution's last element lies here
  if (threadIdx.x == 0) {
    carry[tile] = make_float2(tile_tot.hi, tile_tot.lo);
    incl[tile] = make_float2(tile_tot.hi, tile_tot.lo);
    __threadfence();
    atomicExch(flags + tile, last_tile ? 2u : 1u);
  }
  // block-wide lookback for the sum beyond t1 in the distribution of t1 - 1
  const dflt E = last_tile ? df_zero()
                           : suffix_lookback(lb_s, tile, ntiles, flags, carry, incl, status);
  if (!last_tile && threadIdx.x == 0) {
    const dflt v = df_add(tile_tot, E);
    incl[tile] = make_float2(v.hi, v.lo);
    __threadfence();
    atomicExch(flags + tile, 2u);
  }
  if (e0 >= t1) return;
  const dflt base = df_sub(df_sub(G_s, exv), E);
  dflt inrun = df_zero();
  float gk[kBwPer];
#pragma unroll
  for (int k = kBwPer - 1; k >= 0; --k) {
    gk[k] = df_to_float(df_sub(df_sub(base, inrun), b[k]));
    inrun = df_add(inrun, a[k]);
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
  float2* carry = reinterpret_cast<float2*>(p.base + L.carry);
  float2* incl = reinterpret_cast<float2*>(p.base + L.incl);
  uint32_t* ticket = reinterpret_cast<uint32_t*>(p.base + L.ticket);
  float2* R = reinterpret_cast<float2*>(p.base + L.R);
  float* gradR = reinterpret_cast<float*>(p.base + L.gradR);
  const int64_t Nw = two_d ? N - (D - 1) : N;
  const int sms = bw_sms();
  if (two_d) {
    row_total_kernel<<<(unsigned)std::min<int64_t>(sms * 4, (D - 1 + 255) / 256), 256, 0, st>>>(
        f->dists, D - 1, R);
  }
  const int64_t tiles = (N + kBwTile - 1) / kBwTile;
  bin_total_kernel<<<(unsigned)tiles, kBwThreads, 0, st>>>(p.acc, f->nodes, w, f->dists, D, N,
                                                          G);
  const bool vec_ok = (reinterpret_cast<uintptr_t>(w) & 15) == 0 &&
                      (reinterpret_cast<uintptr_t>(grad_w) & 15) == 0;
  if (D == 1 && !two_d && vec_ok)
    suffix_single_kernel<<<(unsigned)tiles, kBwThreads, 0, st>>>(p.acc, w, f->dists, N, G, flags,
                                                                 carry, incl, ticket, grad_w,
                                                                 f->status);
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
