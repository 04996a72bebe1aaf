// Sampling through the guide table and the radix forest (Binder & Keller,
// Algorithm 2, Sec. 3.2) with the in-bin position of Sec. 5.
//
// Per sample u (xi = u / 2^32):
//   g = u >> (32 - m)                       guide cell (Algorithm 2, first line)
//   j = guide[g]                            ~i, or the root of the cell's tree
//   t = floor(u T / 2^32)                   the sample in the integer CDF domain
//   while j >= 0: j = t < C_j ? child0 : child1     (xi < data[j], Algorithm 2)
//   i = ~j;  pos = (u T - C_i 2^32) / (q_i 2^32)     (Sec. 5)
//
// The node records interleave C_j with the children (16 bytes), so one load
// per visited node serves both the comparison and the next index.  Node loads
// carry an L2 evict-last policy (the structure stays resident while the
// sample stream passes through with evict-first loads and streaming stores).
// When the guide table of a single distribution is small it is staged in
// shared memory once per block.
#include <cstdint>

#include "rtf_device.cuh"

namespace rtf {

constexpr int kSampleThreads = 256;
constexpr int kSmemGuideMaxBits = 13;  // 32 KB of guide in shared memory

__device__ __forceinline__ uint64_t l2_evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ void load_node(const rtf_node* p, uint64_t pol, uint64_t& cdf,
                                          int32_t& c0, int32_t& c1) {
  uint64_t a, b;
  asm volatile("ld.global.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
               : "=l"(a), "=l"(b)
               : "l"(p), "l"(pol));
  cdf = a;
  c0 = (int32_t)(uint32_t)(b & 0xffffffffull);
  c1 = (int32_t)(uint32_t)(b >> 32);
}

__device__ __forceinline__ uint64_t load_cdf(const rtf_node* p, uint64_t pol) {
  uint64_t a;
  asm volatile("ld.global.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(a) : "l"(p), "l"(pol));
  return a;
}

// In-bin position (u T - C_i 2^32) / (q 2^32) from d = t - C_i, the low 32 bits
// r of u T and q = C_{i+1} - C_i: numerator and denominator are rounded to
// float32 once each, then divided (three roundings in all).
__device__ __forceinline__ float in_bin_position(uint64_t d, uint32_t r, uint64_t q) {
  float num, den;
  if ((d >> 32) == 0) {
    num = __ull2float_rn((d << 32) | r);
    den = __ull2float_rn(q) * 4294967296.0f;
  } else {
    num = __ull2float_rn(d);
    den = __ull2float_rn(q);
  }
  float p = __fdiv_rn(num, den);
  return fminf(p, 0x1.fffffep-1f);
}

struct DistView {
  const rtf_node* nodes;  // records of the distribution
  const int32_t* guide;   // its guide table
  uint64_t T;
  int64_t n;
  int m;
};

__device__ __forceinline__ DistView dist_view(const rtf_dist* dists, int d, const rtf_node* nodes,
                                              const int32_t* guide) {
  rtf_dist P = dists[d];
  DistView v;
  v.nodes = nodes + P.elem_off;
  v.guide = guide + P.guide_off;
  v.T = P.total;
  v.n = P.n;
  v.m = P.m;
  return v;
}

// Algorithm 2 and the position for one sample of one distribution.  Every
// index read from the structure is checked against n and the descent is capped
// at 64 visits (a reachable path visits at most 2 + (32 - m) nodes), so a
// structure left invalid by a failed build yields idx = -1 instead of an
// out-of-bounds read.
template <bool SMEM>
__device__ __forceinline__ void sample_one(const DistView& v, const int32_t* gsm, uint32_t u,
                                           uint64_t pol, int32_t& idx, float& pos) {
  const uint32_t g = v.m ? (u >> (32 - v.m)) : 0u;
  int32_t j = SMEM ? gsm[g] : __ldg(v.guide + g);
  const uint64_t t = __umul64hi(v.T, (uint64_t)u << 32);
  const uint32_t r = u * (uint32_t)v.T;
  uint64_t clo = 0, chi = 0;
  int known = 0;  // 1: clo known, 2: chi known
  int steps = 0;
  while (j >= 0) {
    if ((int64_t)j >= v.n || ++steps > 64) {
      idx = -1;
      pos = 0.0f;
      return;
    }
    uint64_t c;
    int32_t c0, c1;
    load_node(v.nodes + j, pol, c, c0, c1);
    if (t < c) {
      j = c0;
      chi = c;
      known = 2;
    } else {
      j = c1;
      clo = c;
      known = 1;
    }
  }
  const int32_t i = ~j;
  if ((int64_t)i >= v.n) {
    idx = -1;
    pos = 0.0f;
    return;
  }
  if (known != 1) clo = load_cdf(v.nodes + i, pol);
  if (known != 2) chi = (i + 1 < v.n) ? load_cdf(v.nodes + i + 1, pol) : v.T;
  idx = i;
  pos = in_bin_position(t - clo, r, chi - clo);
}

// 1-D, one distribution (dist 0); four samples per thread per step.
template <bool SMEM>
__global__ void __launch_bounds__(kSampleThreads)
    sample_single_kernel(const rtf_node* __restrict__ nodes, const int32_t* __restrict__ guide,
                         const rtf_dist* __restrict__ dists, const uint32_t* __restrict__ u,
                         int64_t count, int32_t* __restrict__ idx_out,
                         float* __restrict__ pos_out, int cap_bits, uint32_t* status) {
  extern __shared__ int32_t gsm[];
  const DistView v = dist_view(dists, 0, nodes, guide);
  if (SMEM && v.m > cap_bits) {
    // the host's max_m understated the guide size: refuse rather than overrun
    if (blockIdx.x == 0 && threadIdx.x == 0) raise_status(status, RTF_STATUS_BAD_PLAN);
    return;
  }
  if (SMEM) {
    const int cells = 1 << v.m;
    for (int k = threadIdx.x; k < cells; k += blockDim.x) gsm[k] = v.guide[k];
    __syncthreads();
  }
  const uint64_t pol = l2_evict_last_policy();
  const int64_t nvec = count >> 2;
  const uint4* u4 = reinterpret_cast<const uint4*>(u);
  int4* i4 = reinterpret_cast<int4*>(idx_out);
  float4* p4 = reinterpret_cast<float4*>(pos_out);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nvec;
       q += (int64_t)gridDim.x * blockDim.x) {
    uint4 uu = __ldcs(u4 + q);
    int4 ii;
    float4 pp;
    sample_one<SMEM>(v, gsm, uu.x, pol, ii.x, pp.x);
    sample_one<SMEM>(v, gsm, uu.y, pol, ii.y, pp.y);
    sample_one<SMEM>(v, gsm, uu.z, pol, ii.z, pp.z);
    sample_one<SMEM>(v, gsm, uu.w, pol, ii.w, pp.w);
    __stcs(i4 + q, ii);
    __stcs(p4 + q, pp);
  }
  // tail
  const int64_t rem0 = nvec << 2;
  for (int64_t s = rem0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < count;
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
    sample_tagged_kernel(const rtf_node* __restrict__ nodes, const int32_t* __restrict__ guide,
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
    sample_2d_kernel(const rtf_node* __restrict__ nodes, const int32_t* __restrict__ guide,
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
        f->nodes, f->guide, f->dists, f->num_dists, reinterpret_cast<const uint2*>(u), count,
        reinterpret_cast<int2*>(idx_out), reinterpret_cast<float2*>(pos_out));
    return cudaGetLastError();
  }
  if (dist_id != nullptr) {
    int64_t blocks = min((int64_t)sms * 8, (count + kSampleThreads - 1) / kSampleThreads);
    sample_tagged_kernel<<<(unsigned)blocks, kSampleThreads, 0, st>>>(
        f->nodes, f->guide, f->dists, f->num_dists, u, dist_id, count, idx_out, pos_out,
        f->status);
    return cudaGetLastError();
  }
  const int64_t per_block = (int64_t)kSampleThreads * 4;
  if (f->max_m <= kSmemGuideMaxBits && f->num_dists >= 1) {
    size_t smem = sizeof(int32_t) << f->max_m;
    int64_t blocks = min((int64_t)sms * 8, (count + per_block - 1) / per_block);
    sample_single_kernel<true><<<(unsigned)blocks, kSampleThreads, smem, st>>>(
        f->nodes, f->guide, f->dists, u, count, idx_out, pos_out, f->max_m, f->status);
  } else {
    int64_t blocks = min((int64_t)sms * 8, (count + per_block - 1) / per_block);
    sample_single_kernel<false><<<(unsigned)blocks, kSampleThreads, 0, st>>>(
        f->nodes, f->guide, f->dists, u, count, idx_out, pos_out, 31, f->status);
  }
  return cudaGetLastError();
}

}  // namespace rtf
