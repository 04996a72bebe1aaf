// Device helpers shared by the samplers (the binary radix forest of
// Algorithm 2 and the 4-ary records that collapse two of its levels): record
// loads with an L2 evict-last policy, the scaling of a sample into the integer
// CDF domain and the in-bin position of Sec. 5.
#pragma once

#include <atomic>
#include <cstdint>

#include "rtf_device.cuh"

#ifndef RTF_NODE_PREFETCH
#define RTF_NODE_PREFETCH 0
#endif

namespace rtf {

constexpr int kSampleThreads = 256;

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

__device__ __forceinline__ uint64_t load_cdf(const rtf_node* p, uint64_t pol) {
  uint64_t a;
  asm("ld.global.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(a) : "l"(p), "l"(pol));
  return a;
}

__device__ __forceinline__ int32_t load_child0(const rtf_guide_rec* p, uint64_t pol) {
  int32_t a;
  asm("ld.global.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(a) : "l"(&p->child[0]), "l"(pol));
  return a;
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
// to float32 once each (no fp64 pipe).  The quotient a / b follows Markstein's
// correction of a reciprocal-based quotient (P. Markstein, "Computation of
// elementary functions on the IBM RISC System/6000 processor", IBM J. Res.
// Dev. 34(1), 1990): y ~ 1/b from the hardware reciprocal estimate, q0 = a y,
// the residual e = a - b q0 by one fused multiply-add (exact), q1 = q0 + e y.
// The result is within about 1.5 ulp of the exact value (tested against the
// fp64 oracle within 4 ulp) and clamped below 1.
__device__ __forceinline__ float in_bin_position(uint64_t d, uint32_t r, uint64_t q) {
  // the integer is chosen before its one conversion (the same value either way)
  const bool small = (d >> 32) == 0;
  const float num = u64_to_f32(small ? ((d << 32) | r) : d);
  const float qf = u64_to_f32(q);
  const float den = small ? qf * 4294967296.0f : qf;
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

// Device properties the launchers size their grids by, cached per device
// (host threads may race to fill an entry; they all store the same value).
constexpr int kCachedDevices = 64;

inline int device_attr_cached(std::atomic<int>* cache, cudaDeviceAttr attr, int fallback) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  const bool cacheable = dev >= 0 && dev < kCachedDevices;
  int v = cacheable ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (v == 0) {
    int b = 0;
    if (cudaDeviceGetAttribute(&b, attr, dev) != cudaSuccess || b <= 0) b = fallback;
    v = b;
    if (cacheable) cache[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

inline int64_t l2_bytes() {
  static std::atomic<int> cache[kCachedDevices];
  return device_attr_cached(cache, cudaDevAttrL2CacheSize, 126 << 20);
}

inline int num_sms() {
  static std::atomic<int> cache[kCachedDevices];
  return device_attr_cached(cache, cudaDevAttrMultiProcessorCount, 148);
}

}  // namespace rtf
