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
#include "sample_common.cuh"

namespace rtf {

constexpr int kSmemGuideMaxBits = 10;  // 32 KB of guide records in shared memory

// Pairs per thread of the 2-D sampler (1: one pair at a time; 2 or 4: their
// descents in lockstep).  GB300, 4096 x 2048 map, 2^26 pairs: 1.54 ms with 2,
// 1.64 ms with 1, 2.36 ms with 4 (120 registers, two blocks per SM).
#ifndef RTF_2D_PAIRS
#define RTF_2D_PAIRS 2
#endif
// Samples per thread of the sampler with a distribution id per sample (their
// descents in lockstep).  GB300, 16384 ragged distributions, 2^27 samples:
// 5.83 ms with 4, 6.24 ms with 2.
// Minimum resident blocks per SM asked of the register allocator for the 2-D
// sampler (0: no bound).
#ifndef RTF_2D_MINB
#define RTF_2D_MINB 0
#endif
#ifndef RTF_TAGGED_K
#define RTF_TAGGED_K 4
#endif

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
// Grid of the single-distribution sampler, in blocks per SM (grid-stride
// loop).  When the node and guide records exceed L2, fewer resident descents
// keep more of their working set in L2: on GB300 at n = 2^24 (300 MB of
// records), 2^28 i.i.d. samples take 6.73 ms with 3 blocks per SM, 7.19 ms
// with 4 and 8.98 ms with 5 (2 starves the memory system: 7.87 ms).
#ifndef RTF_SAMPLE_BLOCKS_PER_SM
#define RTF_SAMPLE_BLOCKS_PER_SM 8
#endif
#ifndef RTF_SAMPLE_BLOCKS_PER_SM_BIG
#define RTF_SAMPLE_BLOCKS_PER_SM_BIG 3
#endif
// Algorithm 2 and the position for K samples of one distribution at once: the
// K descents advance in lockstep, so each thread keeps K independent node
// loads in flight.  Every index read from the structure is checked against n
// and the descent is capped at 64 visits (a reachable path visits at most
// 2 + (32 - m) nodes), so a structure left invalid by a failed build yields
// idx = -1 instead of an out-of-bounds read.
template <int K, bool SMEM>
__device__ __forceinline__ void sample_group(const DistView& v, const rtf_guide_rec* gsm,
                                             const uint32_t (&uu)[K], uint64_t pol,
                                             int32_t (&idx)[K], float (&pos)[K],
                                             int32_t (&nl)[K]) {
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
    nl[k] = 1;
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
          ++nl[k];
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

// The comparator of the paper (Sec. 2.5): the cutpoint method, a guide table
// that brackets the bins a cell can reach, with a binary search over the CDF
// inside the bracket.  It runs on the same structure: the first interval of
// cell g is ~child[0] of its guide record, the bracket ends at the first
// interval of cell g + 1 (n - 1 after the last cell), a covered cell needs no
// search, and lo, hi of the record are the CDF bounds of the bracket.  The
// search keeps C_a <= t < C_{b+1} for its bracket [a, b], so both bounds of
// the final interval are known when it ends.  Same bins and positions as the
// radix forest; the number of dependent loads differs.
template <int K, bool SMEM>
__device__ __forceinline__ void sample_group_bsearch(const DistView& v, const rtf_guide_rec* gsm,
                                                     const uint32_t (&uu)[K], uint64_t pol,
                                                     int32_t (&idx)[K], float (&pos)[K],
                                                     int32_t (&nl)[K]) {
  const uint32_t n32 = (uint32_t)v.n;
  const uint32_t cells = 1u << v.m;
  uint32_t a[K], b[K];
  uint64_t t[K], lo[K], hi[K];
  uint32_t r[K];
  bool bad = false;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t g = v.m ? (uu[k] >> (32 - v.m)) : 0u;
    scale_sample(uu[k], v.T, t[k], r[k]);
    uint64_t c, glo, ghi;
    int32_t c0, c1;
    if (SMEM) {
      const uint4* e = reinterpret_cast<const uint4*>(gsm + g);
      const uint4 x = e[0], y = e[1];
      c = ((uint64_t)x.y << 32) | x.x;
      c0 = (int32_t)x.z;
      c1 = (int32_t)x.w;
      glo = ((uint64_t)y.y << 32) | y.x;
      ghi = ((uint64_t)y.w << 32) | y.z;
    } else {
      load_guide(v.guide + g, pol, c, c0, c1, glo, ghi);
    }
    (void)c;
    a[k] = (uint32_t)~c0;
    b[k] = a[k];
    nl[k] = 1;
    if (c0 != c1) {  // a cell with a tree: bracket up to the next cell's first interval
      ++nl[k];
      const int32_t nxt = g + 1 < cells ? (SMEM ? gsm[g + 1].child[0] : load_child0(v.guide + g + 1, pol))
                                        : ~(int32_t)(n32 - 1);
      b[k] = (uint32_t)~nxt;
    }
    if (a[k] >= n32 || b[k] >= n32 || a[k] > b[k]) {
      bad = true;  // invalid structure
      a[k] = b[k] = 0;
    }
    lo[k] = glo;
    hi[k] = ghi;
  }
  bool live = false;
#pragma unroll
  for (int k = 0; k < K; ++k) live |= a[k] < b[k];
#pragma unroll 1
  for (int step = 0; live && step < 32; ++step) {
    uint64_t cm[K];
    uint32_t mid[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      mid[k] = a[k] + ((b[k] - a[k] + 1) >> 1);
      if (a[k] < b[k]) {
        cm[k] = load_cdf(v.nodes + mid[k], pol);
        ++nl[k];
      }
    }
    live = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (a[k] < b[k]) {
        if (cm[k] <= t[k]) {
          a[k] = mid[k];
          lo[k] = cm[k];
        } else {
          b[k] = mid[k] - 1;
          hi[k] = cm[k];
        }
        live |= a[k] < b[k];
      }
    }
  }
  bad |= live;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (!bad && lo[k] <= t[k] && t[k] < hi[k]) {
      idx[k] = (int32_t)a[k];
      pos[k] = in_bin_position(t[k] - lo[k], r[k], hi[k] - lo[k]);
    } else {
      idx[k] = -1;
      pos[k] = 0.0f;
    }
  }
}

// One of the two methods; nl receives the number of structure loads of each
// sample (guide records, node or CDF records), which only the statistics
// kernel stores.
template <int K, bool SMEM, bool BS>
__device__ __forceinline__ void sample_any(const DistView& v, const rtf_guide_rec* gsm,
                                           const uint32_t (&uu)[K], uint64_t pol,
                                           int32_t (&idx)[K], float (&pos)[K],
                                           int32_t (&nl)[K]) {
  if (BS)
    sample_group_bsearch<K, SMEM>(v, gsm, uu, pol, idx, pos, nl);
  else
    sample_group<K, SMEM>(v, gsm, uu, pol, idx, pos, nl);
}

template <int K, bool SMEM, bool BS>
__device__ __forceinline__ void sample_any(const DistView& v, const rtf_guide_rec* gsm,
                                           const uint32_t (&uu)[K], uint64_t pol,
                                           int32_t (&idx)[K], float (&pos)[K]) {
  int32_t nl[K];
  sample_any<K, SMEM, BS>(v, gsm, uu, pol, idx, pos, nl);
}

template <bool SMEM, bool BS>
__device__ __forceinline__ void sample_one(const DistView& v, const rtf_guide_rec* gsm, uint32_t u,
                                           uint64_t pol, int32_t& idx, float& pos) {
  uint32_t uu[1] = {u};
  int32_t ii[1];
  float pp[1];
  sample_any<1, SMEM, BS>(v, gsm, uu, pol, ii, pp);
  idx = ii[0];
  pos = pp[0];
}

// 1-D, one distribution (dist 0); RTF_SAMPLE_K samples per thread per step
// (u, idx and pos move as 16-byte vectors, four samples each).
template <bool SMEM, bool BS>
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
      sample_any<K, SMEM, BS>(v, gsm, uu, pol, ii, pp);
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
      sample_any<K, SMEM, BS>(v, gsm, uu, pol, ii, pp);
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
    sample_one<SMEM, BS>(v, gsm, u[s], pol, ii, pp);
    idx_out[s] = ii;
    pos_out[s] = pp;
  }
}

// Algorithm 2 for one sample from its guide record down to the leaf, the
// bounds C_i and C_{i+1} tracked on the way as in sample_group.  False when the
// structure is invalid (an index out of range, a path longer than any
// reachable one, or bounds that do not bracket t).
__device__ __forceinline__ bool descend_one(const DistView& v, uint32_t u, uint64_t t,
                                            uint64_t pol, int32_t& i, uint64_t& lo,
                                            uint64_t& hi) {
  const uint32_t n32 = (uint32_t)v.n;
  const uint32_t g = v.m ? (u >> (32 - v.m)) : 0u;
  uint64_t c, glo, ghi;
  int32_t c0, c1;
  load_guide(v.guide + g, pol, c, c0, c1, glo, ghi);
  const bool left = t < c;
  int32_t j = left ? c0 : c1;
  lo = left ? glo : c;
  hi = left ? c : ghi;
  for (int step = 0; j >= 0 && step < 64; ++step) {
    if ((uint32_t)j >= n32) return false;
    uint64_t cj;
    int32_t a, b;
    load_node(v.nodes + j, pol, cj, a, b);
    if (t < cj) {
      j = a;
      hi = cj;
    } else {
      j = b;
      lo = cj;
    }
  }
  i = ~j;
  return j < 0 && (uint32_t)i < n32 && lo <= t && t < hi;
}

constexpr int kRunSteps = 4;  // forward steps through the CDF in global memory

// Coherent samples (RTF_SAMPLE_COHERENT): samples that arrive in ascending
// order (sorted or low-discrepancy sequences, the monotone mapping of Sec. 3.2)
// mostly fall into the bin of the sample before them or into one of the next
// few.  A warp maps a contiguous stretch of the samples in batches of 32 R
// (lane l takes samples [R l, R l + R) of the batch, in order) and keeps, in
// shared memory, a window of 64 bin bounds W_j = C_{c+1+j} (T for the last bin,
// all ones past it) from bin c on, c being the bin of the last sample the warp
// mapped.  A lane places its first sample of a batch by a binary search of the
// window (a sample outside it descends from its guide record, Algorithm 2),
// then walks its run: a sample in the current bin [C_i, C_{i+1}) keeps it, one
// above steps forward through the window (past its end through the CDF in
// global memory, at most kRunSteps bins), anything else descends.  Each way
// yields the unique bin with C_i <= t < C_{i+1} and its bounds, the bits of
// Algorithm 2, whatever the input order; the order only decides the speed.
// After a batch the window restarts at the bin of the batch's last sample once
// that bin has moved 32 or more bins past c.  GB300, 2^28 sorted samples at
// n = 2^24: 0.91 ms with runs of 8 (runs of 4: 0.92 ms; of 16: 1.39 ms, the
// lanes' loads no longer coalesce); runs without the window, stepping and
// descending through global memory: 1.06 ms; a warp-wide window searched by
// shuffles for every sample: 1.34-1.44 ms; one descent per sample: 1.93 ms.
#ifndef RTF_WRUN_SAMPLES
#define RTF_WRUN_SAMPLES 8
#endif
#ifndef RTF_WRUN_MINB
#define RTF_WRUN_MINB 0
#endif
constexpr int kWinBounds = 64;

__device__ __forceinline__ void window_fill(uint64_t* win, const DistView& v, int64_t c, int lane,
                                            uint64_t pol) {
#pragma unroll
  for (int h = 0; h < kWinBounds / 32; ++h) {
    const int64_t k = c + 1 + lane + 32 * h;
    win[lane + 32 * h] = k < v.n ? load_cdf(v.nodes + k, pol) : (k == v.n ? v.T : ~0ull);
  }
  __syncwarp();
}

// The in-bin position of Sec. 5 with the bin's constants computed once per
// bin: the same operations as in_bin_position (numerator and denominator
// rounded once each, hardware reciprocal refined by one fused residual step),
// so the same bits.  q = 0 marks "no bin": no t satisfies t - lo < q.
struct BinPos {
  uint64_t lo, q;
  float den_a, rcp_a;  // t - lo < 2^32: numerator (t - lo) 2^32 + r, denominator q 2^32
  float den_b, rcp_b;  // otherwise: numerator t - lo, denominator q
  __device__ __forceinline__ void set(uint64_t l, uint64_t h) {
    lo = l;
    q = h - l;
    den_b = u64_to_f32(q);
    den_a = den_b * 4294967296.0f;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rcp_a) : "f"(den_a));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rcp_b) : "f"(den_b));
  }
  __device__ __forceinline__ float pos(uint64_t d, uint32_t r) const {
    const bool small = (d >> 32) == 0;
    const float num = u64_to_f32(small ? ((d << 32) | r) : d);
    const float den = small ? den_a : den_b;
    const float rcp = small ? rcp_a : rcp_b;
    float p = num * rcp;
    const float e = fmaf(-den, p, num);
    p = fmaf(e, rcp, p);
    return fminf(p, 0x1.fffffep-1f);
  }
};

template <int R>
__global__ void __launch_bounds__(kSampleThreads, RTF_WRUN_MINB)
    sample_wrun_kernel(const rtf_node* __restrict__ nodes, const rtf_guide_rec* __restrict__ guide,
                       const rtf_dist* __restrict__ dists, const uint32_t* __restrict__ u,
                       int64_t count, int32_t* __restrict__ idx_out,
                       float* __restrict__ pos_out) {
  static_assert(R % 4 == 0, "runs move as 16-byte vectors");
  constexpr int V = R / 4;
  __shared__ uint64_t wins[kSampleThreads / 32][kWinBounds];
  const DistView v = dist_view(dists, 0, nodes, guide);
  const uint64_t pol = l2_evict_last_policy();
  const int lane = threadIdx.x & 31;
  uint64_t* win = wins[threadIdx.x >> 5];
  const int64_t n = v.n;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t batches = count / (32 * R);
  const int64_t per = (batches + nwarps - 1) / nwarps;
  const int64_t b0 = warp * per;
  const int64_t b1 = min(b0 + per, batches);
  const uint4* u4 = reinterpret_cast<const uint4*>(u);
  int4* i4 = reinterpret_cast<int4*>(idx_out);
  float4* p4 = reinterpret_cast<float4*>(pos_out);
  int64_t c = -1;   // window start (warp-uniform); -1: no window
  uint64_t Cc = 0;  // C_c
  for (int64_t b = b0; b < b1; ++b) {
    const int64_t q0 = b * 32 + lane;  // this lane's run
    uint32_t uu[R];
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const uint4 x = __ldcs(u4 + q0 * V + k);
      uu[4 * k] = x.x;
      uu[4 * k + 1] = x.y;
      uu[4 * k + 2] = x.z;
      uu[4 * k + 3] = x.w;
    }

    if (c < 0) {
      // no window: start it at the bin of the batch's first sample
      uint64_t t0;
      uint32_t r0;
      scale_sample(uu[0], v.T, t0, r0);
      int32_t i0 = -1;
      uint64_t l0 = 0, h0 = 0;
      bool ok0 = false;
      if (lane == 0) ok0 = descend_one(v, uu[0], t0, pol, i0, l0, h0);
      const int32_t cb = __shfl_sync(0xffffffffu, ok0 ? i0 : -1, 0);
      const uint64_t cl = __shfl_sync(0xffffffffu, (unsigned long long)l0, 0);
      if (cb >= 0) {
        c = cb;
        Cc = cl;
        window_fill(win, v, c, lane, pol);
      }
    }
    // the lane's first sample: a binary search of the window
    int32_t cur = -1;
    int p = -1;  // window slot of the bin's upper bound (W_p = C_{cur+1}), -1: not from the window
    BinPos bp;
    bp.lo = 0;
    bp.q = 0;
    {
      uint64_t t0;
      uint32_t r0;
      scale_sample(uu[0], v.T, t0, r0);
      if (c >= 0 && t0 >= Cc && t0 < win[kWinBounds - 1]) {
        int cnt = 0;
#pragma unroll
        for (int step = kWinBounds / 2; step >= 1; step >>= 1)
          if (win[cnt + step - 1] <= t0) cnt += step;
        cur = (int32_t)(c + cnt);
        bp.set(cnt > 0 ? win[cnt - 1] : Cc, win[cnt]);
        p = cnt;
      }
    }
    int32_t ii[R];
    float pp[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      uint64_t t;
      uint32_t r;
      scale_sample(uu[k], v.T, t, r);
      uint64_t d = t - bp.lo;
      if (d >= bp.q) {  // not in the current bin (or no bin)
        bool ok = false;
        if (cur >= 0 && t >= bp.lo + bp.q) {
          uint64_t lo = bp.lo + bp.q;  // C_{cur+1}
          for (int st = 0; st < kWinBounds + kRunSteps && cur + 2 <= n; ++st) {
            uint64_t c2;
            if (p >= 0 && p + 1 < kWinBounds) {
              c2 = win[++p];
            } else {
              if (st >= kRunSteps) break;
              p = -1;
              c2 = cur + 2 < n ? load_cdf(v.nodes + cur + 2, pol) : v.T;
            }
            ++cur;
            if (t < c2) {
              bp.set(lo, c2);
              ok = true;
              break;
            }
            lo = c2;
          }
        }
        if (!ok) {
          uint64_t lo, hi;
          ok = descend_one(v, uu[k], t, pol, cur, lo, hi);
          p = -1;
          if (ok) {
            bp.set(lo, hi);
          } else {
            cur = -1;
            bp.lo = 0;
            bp.q = 0;
          }
        }
        d = t - bp.lo;
      }
      ii[k] = cur;
      pp[k] = cur >= 0 ? bp.pos(d, r) : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < V; ++k) {
      __stcs(i4 + q0 * V + k, make_int4(ii[4 * k], ii[4 * k + 1], ii[4 * k + 2], ii[4 * k + 3]));
      __stcs(p4 + q0 * V + k, make_float4(pp[4 * k], pp[4 * k + 1], pp[4 * k + 2], pp[4 * k + 3]));
    }
    // restart the window at the bin of the batch's last sample once it ran ahead
    const int32_t cl = __shfl_sync(0xffffffffu, cur, 31);
    const uint64_t ll = __shfl_sync(0xffffffffu, (unsigned long long)bp.lo, 31);
    __syncwarp();
    if (cl < 0) {
      c = -1;
    } else if (c < 0 || cl < c || cl - c >= kWinBounds / 2) {
      c = cl;
      Cc = ll;
      window_fill(win, v, c, lane, pol);
    }
  }
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = batches * 32 * R + gtid; s < count; s += stride) {
    int32_t ii;
    float pp;
    sample_one<false, false>(v, nullptr, u[s], pol, ii, pp);
    idx_out[s] = ii;
    pos_out[s] = pp;
  }
}

// Algorithm 2 and the position for K samples of K distributions (a distribution
// id per sample): as sample_group, with the distribution's parameters per
// slot.  A sample with an invalid id yields idx = -1 and sets bad_id.
template <int K>
__device__ __forceinline__ void sample_group_tagged(const rtf_node* __restrict__ nodes,
                                                    const rtf_guide_rec* __restrict__ guide,
                                                    const rtf_dist* __restrict__ dists, int D,
                                                    const uint32_t (&uu)[K], const int32_t (&dd)[K],
                                                    uint64_t pol, int32_t (&idx)[K],
                                                    float (&pos)[K], bool& bad_id) {
  int32_t j[K];
  uint64_t t[K], lo[K], hi[K];
  uint32_t r[K], n32[K];
  int64_t off[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    j[k] = -1;
    t[k] = 0;
    lo[k] = 1;
    hi[k] = 0;
    r[k] = 0;
    n32[k] = 0;
    off[k] = 0;
    if (dd[k] < 0 || dd[k] >= D) {
      bad_id = true;
      continue;
    }
    const rtf_dist* P = dists + dd[k];
    off[k] = __ldg(&P->elem_off);
    n32[k] = (uint32_t)__ldg(&P->n);
    const uint64_t T = __ldg(&P->total);
    const int m = __ldg(&P->m);
    const int64_t goff = __ldg(&P->guide_off);
    const uint32_t g = m ? (uu[k] >> (32 - m)) : 0u;
    scale_sample(uu[k], T, t[k], r[k]);
    uint64_t c, glo, ghi;
    int32_t c0, c1;
    load_guide(guide + goff + g, pol, c, c0, c1, glo, ghi);
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
        if ((uint32_t)j[k] >= n32[k]) {
          bad = true;  // invalid structure: stop this descent
          j[k] = -1;
        } else {
          load_node(nodes + off[k] + j[k], pol, c[k], c0[k], c1[k]);
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
  bad |= live;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t i = (uint32_t)~j[k];
    if (!bad && i < n32[k] && lo[k] <= t[k] && t[k] < hi[k]) {
      idx[k] = (int32_t)i;
      pos[k] = in_bin_position(t[k] - lo[k], r[k], hi[k] - lo[k]);
    } else {
      idx[k] = -1;
      pos[k] = 0.0f;
    }
  }
}

// 1-D with a distribution id per sample: four samples per thread in lockstep
// (u, idx and pos as 16-byte vectors) for the radix forest; one per thread
// for the binary search.
template <bool BS>
__global__ void __launch_bounds__(kSampleThreads)
    sample_tagged_kernel(const rtf_node* __restrict__ nodes, const rtf_guide_rec* __restrict__ guide,
                         const rtf_dist* __restrict__ dists, int D,
                         const uint32_t* __restrict__ u, const int32_t* __restrict__ dist_id,
                         int64_t count, int32_t* __restrict__ idx_out,
                         float* __restrict__ pos_out, uint32_t* status) {
  const uint64_t pol = l2_evict_last_policy();
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if constexpr (!BS) {
    bool bad_id = false;
    constexpr int K = RTF_TAGGED_K;
    static_assert(K == 2 || K == 4, "2 or 4 samples per thread");
    const int64_t groups = count / K;
    for (int64_t q = gtid; q < groups; q += stride) {
      uint32_t uu[K];
      int32_t dd[K], ii[K];
      float pp[K];
      if constexpr (K == 4) {
        const uint4 x = __ldcs(reinterpret_cast<const uint4*>(u) + q);
        uu[0] = x.x;
        uu[1] = x.y;
        uu[2] = x.z;
        uu[3] = x.w;
      } else {
        const uint2 x = __ldcs(reinterpret_cast<const uint2*>(u) + q);
        uu[0] = x.x;
        uu[1] = x.y;
      }
#pragma unroll
      for (int k = 0; k < K; ++k) dd[k] = __ldcs(dist_id + K * q + k);
      sample_group_tagged<K>(nodes, guide, dists, D, uu, dd, pol, ii, pp, bad_id);
      if constexpr (K == 4) {
        __stcs(reinterpret_cast<int4*>(idx_out) + q, make_int4(ii[0], ii[1], ii[2], ii[3]));
        __stcs(reinterpret_cast<float4*>(pos_out) + q, make_float4(pp[0], pp[1], pp[2], pp[3]));
      } else {
        __stcs(reinterpret_cast<int2*>(idx_out) + q, make_int2(ii[0], ii[1]));
        __stcs(reinterpret_cast<float2*>(pos_out) + q, make_float2(pp[0], pp[1]));
      }
    }
    for (int64_t s = K * groups + gtid; s < count; s += stride) {
      const uint32_t uu[1] = {__ldcs(u + s)};
      const int32_t dd[1] = {__ldcs(dist_id + s)};
      int32_t ii[1];
      float pp[1];
      sample_group_tagged<1>(nodes, guide, dists, D, uu, dd, pol, ii, pp, bad_id);
      __stcs(idx_out + s, ii[0]);
      __stcs(pos_out + s, pp[0]);
    }
    if (bad_id) raise_status(status, RTF_STATUS_BAD_PLAN);
  } else {
    for (int64_t s = gtid; s < count; s += stride) {
      int d = __ldcs(dist_id + s);
      uint32_t uu = __ldcs(u + s);
      int32_t ii = -1;
      float pp = 0.0f;
      if (d >= 0 && d < D) {
        const DistView v = dist_view(dists, d, nodes, guide);
        sample_one<false, BS>(v, nullptr, uu, pol, ii, pp);
      } else {
        raise_status(status, RTF_STATUS_BAD_PLAN);
      }
      __stcs(idx_out + s, ii);
      __stcs(pos_out + s, pp);
    }
  }
}

// Structure loads per sample (the statistics of Table 1): one thread per
// sample, guide records from global memory, 1-D modes.
template <bool BS>
__global__ void __launch_bounds__(kSampleThreads)
    sample_loads_kernel(const rtf_node* __restrict__ nodes, const rtf_guide_rec* __restrict__ guide,
                        const rtf_dist* __restrict__ dists, int D, const uint32_t* __restrict__ u,
                        const int32_t* __restrict__ dist_id, int64_t count,
                        int32_t* __restrict__ loads_out, uint32_t* status) {
  const uint64_t pol = l2_evict_last_policy();
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < count;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int d = dist_id ? dist_id[s] : 0;
    int32_t nl[1] = {0};
    if (d >= 0 && d < D) {
      const DistView v = dist_view(dists, d, nodes, guide);
      uint32_t uu[1] = {u[s]};
      int32_t ii[1];
      float pp[1];
      sample_any<1, false, BS>(v, nullptr, uu, pol, ii, pp, nl);
      if (ii[0] < 0) nl[0] = -1;
    } else {
      raise_status(status, RTF_STATUS_BAD_PLAN);
      nl[0] = -1;
    }
    loads_out[s] = nl[0];
  }
}

// 2-D: the row through the marginal (last distribution) with u1, the column
// through that row's distribution with u2 (Sec. 5).
template <bool BS>
__global__ void __launch_bounds__(kSampleThreads, RTF_2D_MINB)
    sample_2d_kernel(const rtf_node* __restrict__ nodes, const rtf_guide_rec* __restrict__ guide,
                     const rtf_dist* __restrict__ dists, int D, const uint2* __restrict__ u,
                     int64_t count, int2* __restrict__ idx_out, float2* __restrict__ pos_out) {
  const uint64_t pol = l2_evict_last_policy();
  const DistView marg = dist_view(dists, D - 1, nodes, guide);
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t done = 0;
  if constexpr (!BS && RTF_2D_PAIRS > 1) {
    // RTF_2D_PAIRS pairs per thread: their rows through the marginal in
    // lockstep, then their columns in lockstep, each through its own row (a
    // pair whose row was not found gets column -1)
    constexpr int P = RTF_2D_PAIRS;
    const int64_t groups = count / P;
    const uint4* u4 = reinterpret_cast<const uint4*>(u);
    int4* i4 = reinterpret_cast<int4*>(idx_out);
    float4* p4 = reinterpret_cast<float4*>(pos_out);
    for (int64_t q = gtid; q < groups; q += stride) {
      uint32_t u1[P], u2[P];
#pragma unroll
      for (int h = 0; h < P / 2; ++h) {
        const uint4 a = __ldcs(u4 + (P / 2) * q + h);
        u1[2 * h] = a.x;
        u2[2 * h] = a.y;
        u1[2 * h + 1] = a.z;
        u2[2 * h + 1] = a.w;
      }
      int32_t r[P], c[P], nl[P], dd[P];
      float pr[P], pc[P];
      sample_group<P, false>(marg, nullptr, u1, pol, r, pr, nl);
#pragma unroll
      for (int k = 0; k < P; ++k) dd[k] = (r[k] >= 0 && r[k] < D - 1) ? r[k] : -1;
      bool no_row = false;
      sample_group_tagged<P>(nodes, guide, dists, D, u2, dd, pol, c, pc, no_row);
#pragma unroll
      for (int h = 0; h < P / 2; ++h) {
        __stcs(i4 + (P / 2) * q + h, make_int4(r[2 * h], c[2 * h], r[2 * h + 1], c[2 * h + 1]));
        __stcs(p4 + (P / 2) * q + h, make_float4(pr[2 * h], pc[2 * h], pr[2 * h + 1], pc[2 * h + 1]));
      }
    }
    done = P * groups;
  }
  for (int64_t s = done + gtid; s < count; s += stride) {
    uint2 uu = __ldcs(u + s);
    int32_t r, c;
    float pr, pc;
    sample_one<false, BS>(marg, nullptr, uu.x, pol, r, pr);
    c = -1;
    pc = 0.0f;
    if (r >= 0 && r < D - 1) {
      const DistView row = dist_view(dists, r, nodes, guide);
      sample_one<false, BS>(row, nullptr, uu.y, pol, c, pc);
    }
    __stcs(idx_out + s, make_int2(r, c));
    __stcs(pos_out + s, make_float2(pr, pc));
  }
}


// The launch shape (rtf_set_launch_shape): blocks per SM per kind of launch,
// 0 for the built-in choice.
static std::atomic<int> g_shape[4];  // single_large, single, tagged, pairs
constexpr int kShapeBuiltin[4] = {RTF_SAMPLE_BLOCKS_PER_SM_BIG, RTF_SAMPLE_BLOCKS_PER_SM, 8, 8};

static int shape_of(int kind) {
  const int v = g_shape[kind].load(std::memory_order_relaxed);
  return v > 0 ? v : kShapeBuiltin[kind];
}

void set_launch_shape(const int32_t* v) {
  for (int k = 0; k < 4; ++k) g_shape[k].store(v ? v[k] : 0, std::memory_order_relaxed);
}

void get_launch_shape(int32_t* v) {
  for (int k = 0; k < 4; ++k) v[k] = shape_of(k);
}

template <bool BS>
static void launch_sample_t(const rtf_forest* f, const uint32_t* u, const int32_t* dist_id,
                            int64_t count, int mode, bool coherent, int32_t* idx_out,
                            float* pos_out, cudaStream_t st) {
  const int sms = num_sms();
  if (mode == RTF_SAMPLE_2D) {
    const int64_t per = BS ? 1 : RTF_2D_PAIRS;  // pairs per thread and step
    int64_t blocks = min((int64_t)sms * shape_of(3),
                         (count + kSampleThreads * per - 1) / (kSampleThreads * per));
    sample_2d_kernel<BS><<<(unsigned)blocks, kSampleThreads, 0, st>>>(
        f->nodes, f->guide_recs, f->dists, f->num_dists, reinterpret_cast<const uint2*>(u), count,
        reinterpret_cast<int2*>(idx_out), reinterpret_cast<float2*>(pos_out));
    return;
  }
  if (dist_id != nullptr) {
    const int64_t per = BS ? 1 : RTF_TAGGED_K;  // samples per thread and step
    int64_t blocks = min((int64_t)sms * shape_of(2),
                         (count + kSampleThreads * per - 1) / (kSampleThreads * per));
    sample_tagged_kernel<BS><<<(unsigned)blocks, kSampleThreads, 0, st>>>(
        f->nodes, f->guide_recs, f->dists, f->num_dists, u, dist_id, count, idx_out, pos_out,
        f->status);
    return;
  }
  if (coherent && !BS) {
    // one wave of resident blocks; each warp maps a contiguous stretch
    static std::atomic<int> resident_cache{0};  // same kernel and architecture on every device
    int resident = resident_cache.load(std::memory_order_relaxed);
    if (resident == 0) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
              &resident, sample_wrun_kernel<RTF_WRUN_SAMPLES>, kSampleThreads, 0) != cudaSuccess ||
          resident <= 0)
        resident = 4;
      resident_cache.store(resident, std::memory_order_relaxed);
    }
    const int64_t per = (int64_t)kSampleThreads * RTF_WRUN_SAMPLES;
    const int64_t blocks = min((int64_t)sms * resident, (count + per - 1) / per);
    sample_wrun_kernel<RTF_WRUN_SAMPLES><<<(unsigned)blocks, kSampleThreads, 0, st>>>(
        f->nodes, f->guide_recs, f->dists, u, count, idx_out, pos_out);
    return;
  }
  const int64_t per_block = (int64_t)kSampleThreads * 4;
  const int64_t records = (int64_t)sizeof(rtf_node) * f->num_elems +
                          (int64_t)sizeof(rtf_guide_rec) * f->num_cells;
  const int per_sm = !coherent && records > l2_bytes() ? shape_of(0) : shape_of(1);
  int64_t blocks = min((int64_t)sms * per_sm, (count + per_block - 1) / per_block);
  if (f->max_m <= kSmemGuideMaxBits) {
    size_t smem = sizeof(rtf_guide_rec) << f->max_m;
    sample_single_kernel<true, BS><<<(unsigned)blocks, kSampleThreads, smem, st>>>(
        f->nodes, f->guide_recs, f->dists, u, count, idx_out, pos_out, f->max_m, f->status);
  } else {
    sample_single_kernel<false, BS><<<(unsigned)blocks, kSampleThreads, 0, st>>>(
        f->nodes, f->guide_recs, f->dists, u, count, idx_out, pos_out, 31, f->status);
  }
}

cudaError_t launch_sample_loads(const rtf_forest* f, const uint32_t* u, const int32_t* dist_id,
                                int64_t count, int mode, int32_t* loads_out, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const int64_t blocks = min((int64_t)num_sms() * 8, (count + kSampleThreads - 1) / kSampleThreads);
  if (mode & RTF_SAMPLE_BSEARCH)
    sample_loads_kernel<true><<<(unsigned)blocks, kSampleThreads, 0, st>>>(
        f->nodes, f->guide_recs, f->dists, f->num_dists, u, dist_id, count, loads_out, f->status);
  else
    sample_loads_kernel<false><<<(unsigned)blocks, kSampleThreads, 0, st>>>(
        f->nodes, f->guide_recs, f->dists, f->num_dists, u, dist_id, count, loads_out, f->status);
  return cudaGetLastError();
}

cudaError_t launch_sample(const rtf_forest* f, const uint32_t* u, const int32_t* dist_id,
                          int64_t count, int mode, int32_t* idx_out, float* pos_out,
                          cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const int base = mode & 0xFF;
  const bool coherent = (mode & RTF_SAMPLE_COHERENT) != 0;
  if (mode & RTF_SAMPLE_BSEARCH)
    launch_sample_t<true>(f, u, dist_id, count, base, coherent, idx_out, pos_out, st);
  else
    launch_sample_t<false>(f, u, dist_id, count, base, coherent, idx_out, pos_out, st);
  return cudaGetLastError();
}

}  // namespace rtf
