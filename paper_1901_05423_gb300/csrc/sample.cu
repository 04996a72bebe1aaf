// Sampling through the guide table and the radix forest (Binder & Keller,
// Algorithm 2, Sec. 3.2) with the in-bin position of Sec. 5.
//
// Per sample u (xi = u / 2^32):
//   g = u >> (32 - m)                       guide cell (Algorithm 2, first line)
//   t = floor(u T / 2^32)                   the sample in the integer CDF domain
//   {c, j0, j1, lo, hi} = guide record g    the decision of the cell's root
//   j = t < c ? j0 : j1, then while j >= 0: j = t < C_j ? child0 : child1
//   i = ~j;  pos = (u T - C_i 2^32) / (q_i 2^32)     (Sec. 5)
//
// The node records interleave C_j with the children (16 bytes), so one load
// per visited node serves both the comparison and the next index.  C_i and
// C_{i+1} are tracked on the way down: every step to child[1] passes the lower
// bound of the final interval, every step to child[0] its upper bound, and the
// guide record holds the two bounds that lie outside the cell's tree; so the
// position needs no load after the descent.  Node loads carry an L2
// evict-last policy (the structure stays resident while the sample stream
// passes through with evict-first loads and streaming stores).  When the guide
// table of a single distribution is small it is staged in shared memory once
// per block.
#include <cstdint>

#include "rtf_device.cuh"

namespace rtf {

constexpr int kSampleThreads = 256;
constexpr int kSmemGuideMaxBits = 10;  // 32 KB of guide records in shared memory

// Tunables of the single-distribution sampler (compile-time): samples per
// thread descending in lockstep, the minimum resident blocks per SM given to
// the register allocator (0 = none), and the L2 fetch size requested with each
// node load (0 = default, 1 = 128 B, 2 = 256 B; a cell's records are
// contiguous, so a larger fetch brings the rest of its tree along).
#ifndef RTF_SAMPLE_K
#define RTF_SAMPLE_K 4
#endif
#ifndef RTF_SAMPLE_MINB
#define RTF_SAMPLE_MINB 0
#endif
#ifndef RTF_NODE_PREFETCH
#define RTF_NODE_PREFETCH 0
#endif

__device__ __forceinline__ uint64_t l2_evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ void load_node(const rtf_node* p, uint64_t pol, uint64_t& cdf,
                                          int32_t& c0, int32_t& c1) {
  uint64_t a, b;
#if RTF_NODE_PREFETCH == 2
  asm("ld.global.L2::cache_hint.L2::256B.v2.u64 {%0, %1}, [%2], %3;"
      : "=l"(a), "=l"(b)
      : "l"(p), "l"(pol));
#elif RTF_NODE_PREFETCH == 1
  asm("ld.global.L2::cache_hint.L2::128B.v2.u64 {%0, %1}, [%2], %3;"
      : "=l"(a), "=l"(b)
      : "l"(p), "l"(pol));
#else
  asm("ld.global.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
      : "=l"(a), "=l"(b)
      : "l"(p), "l"(pol));
#endif
  cdf = a;
  c0 = (int32_t)(uint32_t)(b & 0xffffffffull);
  c1 = (int32_t)(uint32_t)(b >> 32);
}

__device__ __forceinline__ void load_guide(const rtf_guide_rec* p, uint64_t pol, uint64_t& cdf,
                                           int32_t& c0, int32_t& c1, uint64_t& lo,
                                           uint64_t& hi) {
  uint64_t b;
  asm("ld.global.L2::cache_hint.v4.u64 {%0, %1, %2, %3}, [%4], %5;"
      : "=l"(cdf), "=l"(b), "=l"(lo), "=l"(hi)
      : "l"(p), "l"(pol));
  c0 = (int32_t)(uint32_t)(b & 0xffffffffull);
  c1 = (int32_t)(uint32_t)(b >> 32);
}

// t = floor(u T / 2^32) and r = (u T) mod 2^32 from two 32 x 32 -> 64 products
// (T < 2^62, so u T_hi + floor(u T_lo / 2^32) cannot overflow).
__device__ __forceinline__ void scale_sample(uint32_t u, uint64_t T, uint64_t& t, uint32_t& r) {
  const uint64_t lo = (uint64_t)(uint32_t)T * u;
  t = (uint64_t)(uint32_t)(T >> 32) * u + (lo >> 32);
  r = (uint32_t)lo;
}

// In-bin position (u T - C_i 2^32) / (q 2^32) from d = t - C_i < q, the low 32
// bits r of u T and q = C_{i+1} - C_i.  Numerator and denominator are rounded
// to float32 once each (no fp64 pipe), the quotient is the hardware
// reciprocal estimate refined by one fused residual step: within about 1.5 ulp
// of the exact value.  The result is clamped below 1.
__device__ __forceinline__ float in_bin_position(uint64_t d, uint32_t r, uint64_t q) {
  float num, den;
  if ((d >> 32) == 0) {
    num = u64_to_f32((d << 32) | r);
    den = u64_to_f32(q) * 4294967296.0f;
  } else {
    num = u64_to_f32(d);
    den = u64_to_f32(q);
  }
  float rcp;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rcp) : "f"(den));
  float p = num * rcp;
  const float e = fmaf(-den, p, num);
  p = fmaf(e, rcp, p);
  return fminf(p, 0x1.fffffep-1f);
}

struct DistView {
  const rtf_node* nodes;        // records of the distribution
  const rtf_guide_rec* guide;  // its guide records
  uint64_t T;
  int64_t n;
  int m;
};

__device__ __forceinline__ DistView dist_view(const rtf_dist* dists, int d, const rtf_node* nodes,
                                              const rtf_guide_rec* guide) {
  rtf_dist P = dists[d];
  DistView v;
  v.nodes = nodes + P.elem_off;
  v.guide = guide + P.guide_off;
  v.T = P.total;
  v.n = P.n;
  v.m = P.m;
  return v;
}

// Algorithm 2 and the position for K samples of one distribution at once: the
// K descents advance in lockstep, so each thread keeps K independent node
// loads in flight.  Every index read from the structure is checked against n
// and the descent is capped at 64 visits (a reachable path visits at most
// 2 + (32 - m) nodes), so a structure left invalid by a failed build yields
// idx = -1 instead of an out-of-bounds read.
template <int K, bool SMEM>
__device__ __forceinline__ void sample_group(const DistView& v, const rtf_guide_rec* gsm,
                                             const uint32_t (&uu)[K], uint64_t pol,
                                             int32_t (&idx)[K], float (&pos)[K]) {
  const uint32_t n32 = (uint32_t)v.n;
  int32_t j[K];
  uint64_t t[K], lo[K], hi[K];
  uint32_t r[K];
  // the guide record takes the root's decision (left neighbour interval or the
  // cell's tree); a cell that one interval i covers holds {C_i, ~i, ~i}
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t g = v.m ? (uu[k] >> (32 - v.m)) : 0u;
    scale_sample(uu[k], v.T, t[k], r[k]);
    uint64_t c, glo, ghi;
    int32_t c0, c1;
    if (SMEM) {
      const uint4* e = reinterpret_cast<const uint4*>(gsm + g);
      const uint4 a = e[0], b = e[1];
      c = ((uint64_t)a.y << 32) | a.x;
      c0 = (int32_t)a.z;
      c1 = (int32_t)a.w;
      glo = ((uint64_t)b.y << 32) | b.x;
      ghi = ((uint64_t)b.w << 32) | b.z;
    } else {
      load_guide(v.guide + g, pol, c, c0, c1, glo, ghi);
    }
    const bool left = t[k] < c;
    j[k] = left ? c0 : c1;
    lo[k] = left ? glo : c;
    hi[k] = left ? c : ghi;
  }
  bool live = false;
#pragma unroll
  for (int k = 0; k < K; ++k) live |= j[k] >= 0;
  bool bad = false;
#pragma unroll 1
  for (int step = 0; live && step < 64; ++step) {
    uint64_t c[K];
    int32_t c0[K], c1[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (j[k] >= 0) {
        if ((uint32_t)j[k] >= n32) {
          bad = true;    // invalid structure: stop this descent
          j[k] = -1;
        } else {
          load_node(v.nodes + j[k], pol, c[k], c0[k], c1[k]);
        }
      }
    }
    live = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (j[k] >= 0) {
        const bool left = t[k] < c[k];
        j[k] = left ? c0[k] : c1[k];
        if (left)
          hi[k] = c[k];
        else
          lo[k] = c[k];
        live |= j[k] >= 0;
      }
    }
  }
  bad |= live;  // a descent longer than any reachable path
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t i = (uint32_t)~j[k];
    if (!bad && i < n32 && lo[k] <= t[k] && t[k] < hi[k]) {
      idx[k] = (int32_t)i;
      pos[k] = in_bin_position(t[k] - lo[k], r[k], hi[k] - lo[k]);
    } else {
      idx[k] = -1;
      pos[k] = 0.0f;
    }
  }
}

template <bool SMEM>
__device__ __forceinline__ void sample_one(const DistView& v, const rtf_guide_rec* gsm, uint32_t u,
                                           uint64_t pol, int32_t& idx, float& pos) {
  uint32_t uu[1] = {u};
  int32_t ii[1];
  float pp[1];
  sample_group<1, SMEM>(v, gsm, uu, pol, ii, pp);
  idx = ii[0];
  pos = pp[0];
}

// 1-D, one distribution (dist 0); RTF_SAMPLE_K samples per thread per step
// (u, idx and pos move as 16-byte vectors, four samples each).
template <bool SMEM>
__global__ void __launch_bounds__(kSampleThreads, RTF_SAMPLE_MINB)
    sample_single_kernel(const rtf_node* __restrict__ nodes, const rtf_guide_rec* __restrict__ guide,
                         const rtf_dist* __restrict__ dists, const uint32_t* __restrict__ u,
                         int64_t count, int32_t* __restrict__ idx_out,
                         float* __restrict__ pos_out, int cap_bits, uint32_t* status) {
  constexpr int K = RTF_SAMPLE_K;
  static_assert(K == 1 || K == 2 || K == 4 || K == 8, "samples per thread");
  constexpr int V = K >= 4 ? K / 4 : 1;   // 16-byte vectors per step
  extern __shared__ __align__(16) int32_t gsm_words[];
  const rtf_guide_rec* gsm = reinterpret_cast<const rtf_guide_rec*>(gsm_words);
  const DistView v = dist_view(dists, 0, nodes, guide);
  if (SMEM && v.m > cap_bits) {
    // the host's max_m understated the guide size: refuse rather than overrun
    if (blockIdx.x == 0 && threadIdx.x == 0) raise_status(status, RTF_STATUS_BAD_PLAN);
    return;
  }
  if (SMEM) {
    const int vecs = 2 << v.m;
    const uint4* src = reinterpret_cast<const uint4*>(v.guide);
    uint4* dst = reinterpret_cast<uint4*>(gsm_words);
    for (int k = threadIdx.x; k < vecs; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
  }
  const uint64_t pol = l2_evict_last_policy();
  const int64_t nvec = count >> 2;
  const uint4* u4 = reinterpret_cast<const uint4*>(u);
  int4* i4 = reinterpret_cast<int4*>(idx_out);
  float4* p4 = reinterpret_cast<float4*>(pos_out);
  if (K >= 4) {
    const int64_t ngroups = nvec / V;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ngroups;
         q += (int64_t)gridDim.x * blockDim.x) {
      uint32_t uu[K];
      int32_t ii[K];
      float pp[K];
#pragma unroll
      for (int t = 0; t < V; ++t) {
        const uint4 x = __ldcs(u4 + q * V + t);
        uu[4 * t] = x.x;
        uu[4 * t + 1] = x.y;
        uu[4 * t + 2] = x.z;
        uu[4 * t + 3] = x.w;
      }
      sample_group<K, SMEM>(v, gsm, uu, pol, ii, pp);
#pragma unroll
      for (int t = 0; t < V; ++t) {
        __stcs(i4 + q * V + t, make_int4(ii[4 * t], ii[4 * t + 1], ii[4 * t + 2], ii[4 * t + 3]));
        __stcs(p4 + q * V + t, make_float4(pp[4 * t], pp[4 * t + 1], pp[4 * t + 2], pp[4 * t + 3]));
      }
    }
  } else {
    const int64_t nsub = nvec * (4 / K);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nsub;
         q += (int64_t)gridDim.x * blockDim.x) {
      uint32_t uu[K];
      int32_t ii[K];
      float pp[K];
#pragma unroll
      for (int t = 0; t < K; ++t) uu[t] = __ldcs(u + q * K + t);
      sample_group<K, SMEM>(v, gsm, uu, pol, ii, pp);
#pragma unroll
      for (int t = 0; t < K; ++t) {
        __stcs(idx_out + q * K + t, ii[t]);
        __stcs(pos_out + q * K + t, pp[t]);
      }
    }
  }
  const int64_t done = (K >= 4) ? (nvec / V) * V * 4 : nvec * 4;
  // tail
  for (int64_t s = done + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < count;
       s += (int64_t)gridDim.x * blockDim.x) {
    int32_t ii;
    float pp;
    sample_one<SMEM>(v, gsm, u[s], pol, ii, pp);
    idx_out[s] = ii;
    pos_out[s] = pp;
  }
}

// 1-D with a distribution id per sample.
__global__ void __launch_bounds__(kSampleThreads)
    sample_tagged_kernel(const rtf_node* __restrict__ nodes, const rtf_guide_rec* __restrict__ guide,
                         const rtf_dist* __restrict__ dists, int D,
                         const uint32_t* __restrict__ u, const int32_t* __restrict__ dist_id,
                         int64_t count, int32_t* __restrict__ idx_out,
                         float* __restrict__ pos_out, uint32_t* status) {
  const uint64_t pol = l2_evict_last_policy();
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < count;
       s += (int64_t)gridDim.x * blockDim.x) {
    int d = __ldcs(dist_id + s);
    uint32_t uu = __ldcs(u + s);
    int32_t ii = -1;
    float pp = 0.0f;
    if (d >= 0 && d < D) {
      const DistView v = dist_view(dists, d, nodes, guide);
      sample_one<false>(v, nullptr, uu, pol, ii, pp);
    } else {
      raise_status(status, RTF_STATUS_BAD_PLAN);
    }
    __stcs(idx_out + s, ii);
    __stcs(pos_out + s, pp);
  }
}

// 2-D: the row through the marginal (last distribution) with u1, the column
// through that row's distribution with u2 (Sec. 5).
__global__ void __launch_bounds__(kSampleThreads)
    sample_2d_kernel(const rtf_node* __restrict__ nodes, const rtf_guide_rec* __restrict__ guide,
                     const rtf_dist* __restrict__ dists, int D, const uint2* __restrict__ u,
                     int64_t count, int2* __restrict__ idx_out, float2* __restrict__ pos_out) {
  const uint64_t pol = l2_evict_last_policy();
  const DistView marg = dist_view(dists, D - 1, nodes, guide);
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < count;
       s += (int64_t)gridDim.x * blockDim.x) {
    uint2 uu = __ldcs(u + s);
    int32_t r, c;
    float pr, pc;
    sample_one<false>(marg, nullptr, uu.x, pol, r, pr);
    c = -1;
    pc = 0.0f;
    if (r >= 0 && r < D - 1) {
      const DistView row = dist_view(dists, r, nodes, guide);
      sample_one<false>(row, nullptr, uu.y, pol, c, pc);
    }
    __stcs(idx_out + s, make_int2(r, c));
    __stcs(pos_out + s, make_float2(pr, pc));
  }
}

static int g_num_sms = 0;

static int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  }
  return g_num_sms;
}

cudaError_t launch_sample(const rtf_forest* f, const uint32_t* u, const int32_t* dist_id,
                          int64_t count, int mode, int32_t* idx_out, float* pos_out,
                          cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const int sms = num_sms();
  if (mode == RTF_SAMPLE_2D) {
    int64_t blocks = min((int64_t)sms * 8, (count + kSampleThreads - 1) / kSampleThreads);
    sample_2d_kernel<<<(unsigned)blocks, kSampleThreads, 0, st>>>(
        f->nodes, f->guide_recs, f->dists, f->num_dists, reinterpret_cast<const uint2*>(u), count,
        reinterpret_cast<int2*>(idx_out), reinterpret_cast<float2*>(pos_out));
    return cudaGetLastError();
  }
  if (dist_id != nullptr) {
    int64_t blocks = min((int64_t)sms * 8, (count + kSampleThreads - 1) / kSampleThreads);
    sample_tagged_kernel<<<(unsigned)blocks, kSampleThreads, 0, st>>>(
        f->nodes, f->guide_recs, f->dists, f->num_dists, u, dist_id, count, idx_out, pos_out,
        f->status);
    return cudaGetLastError();
  }
  const int64_t per_block = (int64_t)kSampleThreads * 4;
  if (f->max_m <= kSmemGuideMaxBits && f->num_dists >= 1) {
    size_t smem = sizeof(rtf_guide_rec) << f->max_m;
    int64_t blocks = min((int64_t)sms * 8, (count + per_block - 1) / per_block);
    sample_single_kernel<true><<<(unsigned)blocks, kSampleThreads, smem, st>>>(
        f->nodes, f->guide_recs, f->dists, u, count, idx_out, pos_out, f->max_m, f->status);
  } else {
    int64_t blocks = min((int64_t)sms * 8, (count + per_block - 1) / per_block);
    sample_single_kernel<false><<<(unsigned)blocks, kSampleThreads, 0, st>>>(
        f->nodes, f->guide_recs, f->dists, u, count, idx_out, pos_out, 31, f->status);
  }
  return cudaGetLastError();
}

}  // namespace rtf
