// 4-ary records: two levels of the radix forest collapsed into one 32-byte
// record (the section on k-ary trees: a higher branching factor results from
// collapsing levels of the binary trees, and pays where the memory transfer
// granularity exceeds what one binary decision needs; one record is one L2
// sector here).
//
// quad_kernel writes record j from node j and its two children.  The samplers
// take the guide record's decision at the cell's root (as Algorithm 2 does),
// then one record per two levels: compare t with C_j, then with the split of
// the chosen side, and move to one of four grandchildren.  Every comparison
// that sends t left lowers the upper bound of the final interval and every one
// that sends it right raises the lower bound, exactly as in the binary descent,
// so the interval and its bounds (and hence the position of Sec. 5) are the
// binary sampler's bits.
#include <cstdint>

#include "rtf_device.cuh"
#include "sample_common.cuh"

namespace rtf {

constexpr int kQuadThreads = 256;
constexpr int64_t kQuadRefMax = 16383;  // offsets stored as 2 d (+1 for a leaf) in int16

// Relative reference of x (node id, or ~bin) from node j of a distribution of
// n bins; false when it is out of range or too far for 16 bits.
__device__ __forceinline__ bool quad_ref(int32_t x, int64_t j, int64_t n, int32_t& code) {
  const bool leaf = x < 0;
  const int64_t k = leaf ? (int64_t)~x : (int64_t)x;
  if (k >= n) return false;
  const int64_t d = k - j;
  if (d < -kQuadRefMax - 1 || d > kQuadRefMax) return false;
  code = (int32_t)(2 * d + (leaf ? 1 : 0));
  return true;
}

__global__ void __launch_bounds__(kQuadThreads)
    quad_kernel(const rtf_node* __restrict__ nodes, const rtf_dist* __restrict__ dists, int D,
                int64_t N, rtf_quad_rec* __restrict__ quad) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int d = D > 1 ? find_dist(dists, 0, D - 1, e) : 0;
    const int64_t off = dists[d].elem_off;
    const int64_t n = dists[d].n;
    const int64_t j = e - off;
    const rtf_node nj = nodes[e];
    uint64_t split[2];
    int32_t code[4] = {0, 0, 0, 0};
    bool near = true;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int32_t c = nj.child[s];
      int32_t g0 = c, g1 = c;  // a leaf side names its leaf twice
      uint64_t cc = nj.cdf;    // and repeats C_j
      if (c >= 0) {
        if (c < n) {
          const rtf_node nc = nodes[off + c];
          cc = nc.cdf;
          g0 = nc.child[0];
          g1 = nc.child[1];
        } else {
          near = false;  // invalid structure: the sampler's binary step checks it
        }
      }
      split[s] = cc;
      near = quad_ref(g0, j, n, code[2 * s]) && near;
      near = quad_ref(g1, j, n, code[2 * s + 1]) && near;
    }
    const uint64_t refs = near ? ((uint64_t)(uint16_t)code[0] | ((uint64_t)(uint16_t)code[1] << 16) |
                                  ((uint64_t)(uint16_t)code[2] << 32) |
                                  ((uint64_t)(uint16_t)code[3] << 48))
                               : 0;
    ulonglong4_32a rec;
    rec.x = split[0];
    rec.y = nj.cdf | (near ? 0 : RTF_QUAD_FAR);
    rec.z = split[1];
    rec.w = refs;
    *reinterpret_cast<ulonglong4_32a*>(quad + e) = rec;
  }
}

__device__ __forceinline__ void load_quad(const rtf_quad_rec* p, uint64_t pol, uint64_t& a,
                                          uint64_t& b, uint64_t& c, uint64_t& r) {
  asm("ld.global.L2::cache_hint.v4.u64 {%0, %1, %2, %3}, [%4], %5;"
      : "=l"(a), "=l"(b), "=l"(c), "=l"(r)
      : "l"(p), "l"(pol));
}

// Decision at node j from its loaded record {a, b, c, r}: returns the next
// reference (node id >= 0 or ~bin) and narrows [lo, hi).  A far record takes
// one binary step through node j's record (one more load).
__device__ __forceinline__ int32_t quad_decide(const rtf_node* nodes, int32_t j, uint64_t a,
                                               uint64_t b, uint64_t c, uint64_t r, uint64_t t,
                                               uint64_t pol, uint64_t& lo, uint64_t& hi,
                                               int32_t& nl) {
  if (b & RTF_QUAD_FAR) {
    uint64_t cj;
    int32_t c0, c1;
    load_node(nodes + j, pol, cj, c0, c1);
    ++nl;
    if (t < cj) {
      hi = cj;
      return c0;
    }
    lo = cj;
    return c1;
  }
  const bool left = t < b;
  if (left)
    hi = b;
  else
    lo = b;
  const uint64_t s = left ? a : c;
  const bool left2 = t < s;
  if (left2)
    hi = s;
  else
    lo = s;
  const int sh = (left ? 0 : 32) + (left2 ? 0 : 16);
  const int32_t code = (int32_t)(int16_t)(uint16_t)(r >> sh);
  const int32_t k = j + (code >> 1);
  return (code & 1) ? ~k : k;
}

// K samples of one distribution in lockstep: all K record loads of a level
// pair are issued before any decision.  Indices read from the structure are
// checked against n and the descent is capped, so an invalid structure yields
// idx = -1 instead of an out-of-bounds read.
template <int K>
__device__ __forceinline__ void sample_group_quad(const DistView& v, const rtf_quad_rec* quad,
                                                  const uint32_t (&uu)[K], uint64_t pol,
                                                  int32_t (&idx)[K], float (&pos)[K],
                                                  int32_t (&nl)[K]) {
  const uint32_t n32 = (uint32_t)v.n;
  int32_t j[K];
  uint64_t t[K], lo[K], hi[K];
  uint32_t r[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t g = v.m ? (uu[k] >> (32 - v.m)) : 0u;
    scale_sample(uu[k], v.T, t[k], r[k]);
    uint64_t c, glo, ghi;
    int32_t c0, c1;
    load_guide(v.guide + g, pol, c, c0, c1, glo, ghi);
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
    uint64_t a[K], b[K], c[K], rr[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (j[k] >= 0) {
        if ((uint32_t)j[k] >= n32) {
          bad = true;
          j[k] = -1;
        } else {
          load_quad(quad + j[k], pol, a[k], b[k], c[k], rr[k]);
          ++nl[k];
        }
      }
    }
    live = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (j[k] >= 0) {
        j[k] = quad_decide(v.nodes, j[k], a[k], b[k], c[k], rr[k], t[k], pol, lo[k], hi[k], nl[k]);
        live |= j[k] >= 0;
      }
    }
  }
  bad |= live;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t i = (uint32_t)~j[k];
    if (!bad && i < n32 && lo[k] <= t[k] && t[k] < hi[k]) {
      idx[k] = (int32_t)i;
      pos[k] = in_bin_position(t[k] - lo[k], r[k], hi[k] - lo[k]);
    } else {
      idx[k] = -1;
      pos[k] = 0.0f;
      nl[k] = -1;
    }
  }
}

__device__ __forceinline__ void sample_one_quad(const DistView& v, const rtf_quad_rec* quad,
                                                uint32_t u, uint64_t pol, int32_t& idx,
                                                float& pos, int32_t& nl) {
  const uint32_t uu[1] = {u};
  int32_t ii[1], ll[1];
  float pp[1];
  sample_group_quad<1>(v, quad, uu, pol, ii, pp, ll);
  idx = ii[0];
  pos = pp[0];
  nl = ll[0];
}

// 1-D, one distribution: four samples per thread in lockstep, u, idx and pos
// as 16-byte vectors.
__global__ void __launch_bounds__(kSampleThreads)
    sample_quad_single_kernel(const rtf_node* __restrict__ nodes,
                              const rtf_guide_rec* __restrict__ guide,
                              const rtf_dist* __restrict__ dists,
                              const rtf_quad_rec* __restrict__ quad, const uint32_t* __restrict__ u,
                              int64_t count, int32_t* __restrict__ idx_out,
                              float* __restrict__ pos_out, int32_t* __restrict__ loads_out) {
  const DistView v = dist_view(dists, 0, nodes, guide);
  const uint64_t pol = l2_evict_last_policy();
  const int64_t groups = count >> 2;
  const uint4* u4 = reinterpret_cast<const uint4*>(u);
  int4* i4 = reinterpret_cast<int4*>(idx_out);
  float4* p4 = reinterpret_cast<float4*>(pos_out);
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = gtid; q < groups; q += stride) {
    const uint4 x = __ldcs(u4 + q);
    const uint32_t uu[4] = {x.x, x.y, x.z, x.w};
    int32_t ii[4], ll[4];
    float pp[4];
    sample_group_quad<4>(v, quad, uu, pol, ii, pp, ll);
    __stcs(i4 + q, make_int4(ii[0], ii[1], ii[2], ii[3]));
    __stcs(p4 + q, make_float4(pp[0], pp[1], pp[2], pp[3]));
    if (loads_out) {
#pragma unroll
      for (int k = 0; k < 4; ++k) loads_out[4 * q + k] = ll[k];
    }
  }
  for (int64_t s = 4 * groups + gtid; s < count; s += stride) {
    int32_t ii, ll;
    float pp;
    sample_one_quad(v, quad, u[s], pol, ii, pp, ll);
    idx_out[s] = ii;
    pos_out[s] = pp;
    if (loads_out) loads_out[s] = ll;
  }
}

// 1-D with a distribution id per sample, one sample per thread.
__global__ void __launch_bounds__(kSampleThreads)
    sample_quad_tagged_kernel(const rtf_node* __restrict__ nodes,
                              const rtf_guide_rec* __restrict__ guide,
                              const rtf_dist* __restrict__ dists, int D,
                              const rtf_quad_rec* __restrict__ quad, const uint32_t* __restrict__ u,
                              const int32_t* __restrict__ dist_id, int64_t count,
                              int32_t* __restrict__ idx_out, float* __restrict__ pos_out,
                              int32_t* __restrict__ loads_out, uint32_t* status) {
  const uint64_t pol = l2_evict_last_policy();
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < count;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int d = __ldcs(dist_id + s);
    int32_t ii = -1, ll = -1;
    float pp = 0.0f;
    if (d >= 0 && d < D) {
      const DistView v = dist_view(dists, d, nodes, guide);
      sample_one_quad(v, quad + __ldg(&dists[d].elem_off), __ldcs(u + s), pol, ii, pp, ll);
    } else {
      raise_status(status, RTF_STATUS_BAD_PLAN);
    }
    __stcs(idx_out + s, ii);
    __stcs(pos_out + s, pp);
    if (loads_out) loads_out[s] = ll;
  }
}

// 2-D: the row through the marginal (last distribution) with u1, the column
// through that row's distribution with u2 (Sec. 5).
__global__ void __launch_bounds__(kSampleThreads)
    sample_quad_2d_kernel(const rtf_node* __restrict__ nodes, const rtf_guide_rec* __restrict__ guide,
                          const rtf_dist* __restrict__ dists, int D,
                          const rtf_quad_rec* __restrict__ quad, const uint2* __restrict__ u,
                          int64_t count, int2* __restrict__ idx_out, float2* __restrict__ pos_out,
                          int2* __restrict__ loads_out) {
  const uint64_t pol = l2_evict_last_policy();
  const DistView marg = dist_view(dists, D - 1, nodes, guide);
  const rtf_quad_rec* mq = quad + __ldg(&dists[D - 1].elem_off);
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < count;
       s += (int64_t)gridDim.x * blockDim.x) {
    const uint2 uu = __ldcs(u + s);
    int32_t r, c = -1, lr, lc = -1;
    float pr, pc = 0.0f;
    sample_one_quad(marg, mq, uu.x, pol, r, pr, lr);
    if (r >= 0 && r < D - 1) {
      const DistView row = dist_view(dists, r, nodes, guide);
      sample_one_quad(row, quad + __ldg(&dists[r].elem_off), uu.y, pol, c, pc, lc);
    }
    __stcs(idx_out + s, make_int2(r, c));
    __stcs(pos_out + s, make_float2(pr, pc));
    if (loads_out) loads_out[s] = make_int2(lr, lc);
  }
}

cudaError_t launch_build_quad(const rtf_forest* f, rtf_quad_rec* quad, cudaStream_t st) {
  const int64_t N = f->num_elems;
  if (N == 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((int64_t)num_sms() * 8,
                                           (N + kQuadThreads - 1) / kQuadThreads);
  quad_kernel<<<(unsigned)blocks, kQuadThreads, 0, st>>>(f->nodes, f->dists, f->num_dists, N,
                                                         quad);
  return cudaGetLastError();
}

cudaError_t launch_sample_quad(const rtf_forest* f, const rtf_quad_rec* quad, const uint32_t* u,
                               const int32_t* dist_id, int64_t count, int mode, int32_t* idx_out,
                               float* pos_out, int32_t* loads_out, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const int sms = num_sms();
  if ((mode & 0xFF) == RTF_SAMPLE_2D) {
    const int64_t blocks =
        std::min<int64_t>((int64_t)sms * 8, (count + kSampleThreads - 1) / kSampleThreads);
    sample_quad_2d_kernel<<<(unsigned)blocks, kSampleThreads, 0, st>>>(
        f->nodes, f->guide_recs, f->dists, f->num_dists, quad, reinterpret_cast<const uint2*>(u),
        count, reinterpret_cast<int2*>(idx_out), reinterpret_cast<float2*>(pos_out),
        reinterpret_cast<int2*>(loads_out));
    return cudaGetLastError();
  }
  if (dist_id != nullptr) {
    const int64_t blocks =
        std::min<int64_t>((int64_t)sms * 8, (count + kSampleThreads - 1) / kSampleThreads);
    sample_quad_tagged_kernel<<<(unsigned)blocks, kSampleThreads, 0, st>>>(
        f->nodes, f->guide_recs, f->dists, f->num_dists, quad, u, dist_id, count, idx_out,
        pos_out, loads_out, f->status);
    return cudaGetLastError();
  }
  // as the binary sampler: fewer resident descents when the records exceed
  // L2 and the samples are scattered
  const bool coherent = (mode & RTF_SAMPLE_COHERENT) != 0;
  const int64_t records = (int64_t)sizeof(rtf_quad_rec) * f->num_elems +
                          (int64_t)sizeof(rtf_guide_rec) * f->num_cells;
  const int per_sm = !coherent && records > l2_bytes() ? 3 : 8;
  const int64_t per_block = (int64_t)kSampleThreads * 4;
  const int64_t blocks = std::min<int64_t>((int64_t)sms * per_sm, (count + per_block - 1) / per_block);
  sample_quad_single_kernel<<<(unsigned)blocks, kSampleThreads, 0, st>>>(
      f->nodes, f->guide_recs, f->dists, quad, u, count, idx_out, pos_out, loads_out);
  return cudaGetLastError();
}

}  // namespace rtf
