// Gradient of the in-bin sample positions with respect to the weights (not in
// the paper; the adjoint of the relaxed forward x = (xi W - C_i) / w_i with the
// bin i of each sample held fixed).
//
//   dL/dw_k = sum_{i in d} c_i  -  sum_{i > k, i in d} a_i  -  b_k
//   a_i = sum_{s -> i} g_s / w_i,  b_i = sum_{s -> i} g_s x_s / w_i,
//   c_i = sum_{s -> i} g_s xi_s / w_i.
//
// Kernels:
//   row_sum_kernel       (2-D) real row totals R_r = sum_c w(r, c), the
//                        weights of the marginal
//   scatter kernels      one vector atomic {a, b, c} per sample into its bin,
//                        runs of equal bins inside a warp merged first
//   dist_total_kernel    G_d = sum_{i in d} c_i per distribution
//   suffix_kernel        reverse decoupled-lookback scan of a per
//                        distribution (fp32 in the tile, fp64 carry), then
//                        dL/dw_k = G_d - S_k - b_k
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
  size_t acc;    // float4 [N]
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
  L.acc = o; o = align256(o + 16 * (size_t)N);
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
__device__ __forceinline__ void scatter_merge(float4* acc, int64_t j, float va, float vb,
                                              float vc, bool valid) {
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  int64_t jprev = __shfl_up_sync(full, j, 1);
  bool head = (lane == 0) || (jprev != j);
  unsigned heads = __ballot_sync(full, head);
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    float pa = __shfl_up_sync(full, va, d);
    float pb = __shfl_up_sync(full, vb, d);
    float pc = __shfl_up_sync(full, vc, d);
    // lane may add lane-d's partial only if no run starts in (lane-d, lane]
    unsigned span = (lane >= d) ? (((1u << lane) << 1) - (1u << (lane - d + 1))) : 0u;
    if (lane >= d && (heads & span) == 0) {
      va += pa;
      vb += pb;
      vc += pc;
    }
  }
  bool tail = (lane == 31) || (((heads >> (lane + 1)) & 1u) != 0);
  if (tail && valid) atomicAdd(acc + j, make_float4(va, vb, vc, 0.0f));
}

__device__ __forceinline__ float u_to_xi(uint32_t u) { return (float)u * 2.3283064365386963e-10f; }

// 1-D samples (dist_id NULL -> distribution 0)
__global__ void __launch_bounds__(kBwThreads)
    scatter_1d_kernel(const float* __restrict__ w, const rtf_dist* __restrict__ dists, int D,
                      const uint32_t* __restrict__ u, const int32_t* __restrict__ dist_id,
                      const int32_t* __restrict__ idx, const float* __restrict__ pos,
                      const float* __restrict__ gpos, int64_t count, float4* acc) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t start = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t iters = (count + stride - 1) / stride;
  for (int64_t it = 0; it < iters; ++it) {
    int64_t s = start + it * stride;
    bool valid = s < count;
    int64_t j = -1 - (int64_t)(threadIdx.x & 31);
    float va = 0.f, vb = 0.f, vc = 0.f;
    if (valid) {
      int d = dist_id ? __ldcs(dist_id + s) : 0;
      int32_t i = __ldcs(idx + s);
      valid = d >= 0 && d < D && i >= 0 && (int64_t)i < dists[d].n;
      if (valid) {
        int64_t off = dists[d].elem_off;
        j = off + i;
        float g = __ldcs(gpos + s);
        float x = __ldcs(pos + s);
        float xi = u_to_xi(__ldcs(u + s));
        float inv = __frcp_rn(w[j]);
        va = g * inv;
        vb = g * x * inv;
        vc = g * xi * inv;
      }
    }
    scatter_merge(acc, j, va, vb, vc, valid);
  }
}

// 2-D samples: the row term into the marginal (weights R), the column term
// into the row.
__global__ void __launch_bounds__(kBwThreads)
    scatter_2d_kernel(const float* __restrict__ w, const rtf_dist* __restrict__ dists, int D,
                      const float* __restrict__ R, const uint2* __restrict__ u,
                      const int2* __restrict__ idx, const float2* __restrict__ pos,
                      const float2* __restrict__ gpos, int64_t count, float4* acc) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t start = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t iters = (count + stride - 1) / stride;
  const int64_t moff = dists[D - 1].elem_off;
  for (int64_t it = 0; it < iters; ++it) {
    int64_t s = start + it * stride;
    bool valid = s < count;
    int64_t jr = -1 - (int64_t)(threadIdx.x & 31), jc = jr;
    float ra = 0.f, rb = 0.f, rc = 0.f, ca = 0.f, cb = 0.f, cc = 0.f;
    if (valid) {
      int2 ii = __ldcs(idx + s);
      uint2 uu = __ldcs(u + s);
      float2 pp = __ldcs(pos + s);
      float2 gg = __ldcs(gpos + s);
      valid = ii.x >= 0 && ii.x < D - 1 && ii.y >= 0 && (int64_t)ii.y < dists[ii.x].n;
      if (valid) {
        jr = moff + ii.x;
        float invr = __frcp_rn(R[ii.x]);
        ra = gg.x * invr;
        rb = gg.x * pp.x * invr;
        rc = gg.x * u_to_xi(uu.x) * invr;
        jc = dists[ii.x].elem_off + ii.y;
        float invc = __frcp_rn(w[jc]);
        ca = gg.y * invc;
        cb = gg.y * pp.y * invc;
        cc = gg.y * u_to_xi(uu.y) * invc;
      }
    }
    scatter_merge(acc, jr, ra, rb, rc, valid);
    scatter_merge(acc, jc, ca, cb, cc, valid);
  }
}

// G_d = sum of c over distribution d (fp32 per thread run, fp64 atomics per run).
__global__ void __launch_bounds__(kBwThreads)
    dist_total_kernel(const float4* __restrict__ acc, const rtf_dist* __restrict__ dists, int D,
                      int64_t N, double* G) {
  __shared__ int dfirst_s;
  const int64_t t0 = (int64_t)blockIdx.x * kBwTile;
  if (threadIdx.x == 0) dfirst_s = find_dist(dists, 0, D - 1, t0);
  __syncthreads();
  const int64_t e0 = t0 + (int64_t)threadIdx.x * kBwPer;
  if (e0 >= N) return;
  int d = find_dist(dists, dfirst_s, min(D - 1, dfirst_s + kBwTile), e0);
  int64_t next = d + 1 < D ? dists[d + 1].elem_off : INT64_MAX;
  float run = 0.f;
  const int64_t e1 = min(e0 + (int64_t)kBwPer, N);
  for (int64_t e = e0; e < e1; ++e) {
    if (e >= next) {
      atomicAdd(G + d, (double)run);
      run = 0.f;
      ++d;
      next = d + 1 < D ? dists[d + 1].elem_off : INT64_MAX;
    }
    run += acc[e].z;
  }
  atomicAdd(G + d, (double)run);
}

// Reverse segmented scan: S_k = sum_{i > k, same distribution} a_i, then the
// gradient.  Tiles are taken from the end by ticket; each tile publishes the
// sum of a over its first piece (the part of dist(t0) inside the tile) and,
// once known, that sum plus everything after it.
__global__ void __launch_bounds__(kBwThreads)
    suffix_kernel(const float4* __restrict__ acc, const rtf_dist* __restrict__ dists, int D,
                  int64_t N, int64_t Nw, const double* __restrict__ G, uint32_t* flags,
                  double* carry, double* incl, uint32_t* ticket, float* grad_w, float* gradR, uint32_t* status) {
  __shared__ uint32_t tick_s;
  __shared__ int dfirst_s;
  __shared__ float agg_s[kBwThreads];
  __shared__ int headf_s[kBwThreads];
  __shared__ float ex_s[kBwThreads];
  __shared__ int exf_s[kBwThreads];
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

  // per-thread reverse runs
  float a[kBwPer], b[kBwPer];
  int dk[kBwPer];
  uint32_t tailmask = 0;  // element k is the last of its distribution
  {
    int d = dfirst;
    if (e0 < t1) d = find_dist(dists, dfirst, min(D - 1, dfirst + kBwTile), e0);
#pragma unroll
    for (int k = 0; k < kBwPer; ++k) {
      int64_t e = e0 + k;
      a[k] = 0.f;
      b[k] = 0.f;
      dk[k] = d;
      if (e < t1) {
        while (d + 1 < D && e >= dists[d + 1].elem_off) ++d;
        dk[k] = d;
        float4 v = acc[e];
        a[k] = v.x;
        b[k] = v.y;
        int64_t end = dists[d].elem_off + dists[d].n;
        if (e + 1 == end) tailmask |= 1u << k;
      }
    }
  }
  // thread aggregate in reverse order: sum of a from its first tail (from the
  // right) to the right end... i.e. the part that continues leftwards
  float tot = 0.f;
#pragma unroll
  for (int k = kBwPer - 1; k >= 0; --k) {
    if (tailmask & (1u << k)) tot = 0.f;
    tot += a[k];
  }
  agg_s[threadIdx.x] = tot;
  headf_s[threadIdx.x] = tailmask ? 1 : 0;
  __syncthreads();
  // forward segmented scan over reversed thread order (thread n-1-tid first)
  {
    const int rt = kBwThreads - 1 - threadIdx.x;  // reversed position of this thread
    (void)rt;
    // simple Hillis-Steele in shared memory over reversed order
    const int me = kBwThreads - 1 - threadIdx.x;  // thread whose value we scan at slot tid
    float v = agg_s[me];
    int f = headf_s[me];
    __syncthreads();
    // slot-ordered arrays
    ex_s[threadIdx.x] = v;
    exf_s[threadIdx.x] = f;
    __syncthreads();
    for (int dlt = 1; dlt < kBwThreads; dlt <<= 1) {
      float pv = 0.f;
      int pf = 0;
      if ((int)threadIdx.x >= dlt) {
        pv = ex_s[threadIdx.x - dlt];
        pf = exf_s[threadIdx.x - dlt];
      }
      __syncthreads();
      if ((int)threadIdx.x >= dlt && !f) {
        v = pv + v;
        f = pf | f;
      } else if ((int)threadIdx.x >= dlt) {
        // a head in this slot: keep own value
      }
      ex_s[threadIdx.x] = v;
      exf_s[threadIdx.x] = f;
      __syncthreads();
    }
    // ex_s[slot] is now inclusive over slots; convert to exclusive per thread
  }
  // exclusive value for thread tid = inclusive at slot (n-1-tid) - 1
  const int slot = kBwThreads - 1 - threadIdx.x;
  float exv = 0.f;
  int exf = 0;
  if (slot > 0) {
    exv = ex_s[slot - 1];
    exf = exf_s[slot - 1];
  }
  // publish: sum over the first piece of the tile (everything from t0 up to
  // the first tail) is the inclusive value of slot n-1 (thread 0)
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
  // lookback for the incoming carry (sum of a beyond t1 in dist(t1-1))
  if (threadIdx.x == 0) {
    double E = 0.0;
    if (continues) {
      int64_t look = tile + 1;
      long long spins = 0;
      while (look < ntiles) {
        uint32_t fl = *((volatile uint32_t*)(flags + look));
        if (fl == 0) {
          if (++spins > kSpinLimit) {
            raise_status(status, RTF_STATUS_TIMEOUT);
            break;
          }
          __nanosleep(32);
          continue;
        }
        __threadfence();
        if (fl == 2) {
          E += *((volatile double*)(incl + look));
          break;
        }
        E += *((volatile double*)(carry + look));
        ++look;
      }
    }
    E_s = E;
    if (!first_piece_closed) {
      incl[tile] = (double)first_piece + E;
      __threadfence();
      atomicExch(flags + tile, 2u);
    }
  }
  __syncthreads();
  const double E = E_s;
  if (e0 >= t1) return;
  // element results: walk the thread's run from the right
  double after = exf ? (double)exv : (double)exv + E;  // sum of a to the right of this thread
  bool cut = false;
  float inrun = 0.f;
#pragma unroll
  for (int k = kBwPer - 1; k >= 0; --k) {
    int64_t e = e0 + k;
    if (e >= t1) continue;
    if (tailmask & (1u << k)) {
      cut = true;
      inrun = 0.f;
    }
    double S = cut ? (double)inrun : after + (double)inrun;  // sum over i > e
    int d = dk[k];
    double gk = G[d] - S - (double)b[k];
    if (e < Nw)
      grad_w[e] = (float)gk;
    else
      gradR[e - Nw] = (float)gk;
    inrun += a[k];
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

cudaError_t launch_backward(const rtf_forest* f, const float* w, const uint32_t* u,
                            const int32_t* dist_id, const int32_t* idx, const float* pos,
                            const float* gpos, int64_t count, int mode, float* grad_w, void* ws,
                            cudaStream_t st) {
  const int64_t N = f->num_elems;
  const int D = f->num_dists;
  const bool two_d = mode == RTF_SAMPLE_2D;
  BwLayout L = bw_layout(N, D);
  char* base = static_cast<char*>(ws);
  float4* acc = reinterpret_cast<float4*>(base + L.acc);
  double* G = reinterpret_cast<double*>(base + L.G);
  uint32_t* flags = reinterpret_cast<uint32_t*>(base + L.flags);
  double* carry = reinterpret_cast<double*>(base + L.carry);
  double* incl = reinterpret_cast<double*>(base + L.incl);
  uint32_t* ticket = reinterpret_cast<uint32_t*>(base + L.ticket);
  float* R = reinterpret_cast<float*>(base + L.R);
  float* gradR = reinterpret_cast<float*>(base + L.gradR);
  const int64_t Nw = two_d ? N - (D - 1) : N;
  cudaError_t e;
  if ((e = cudaMemsetAsync(base, 0, L.zero_end, st))) return e;
  const int sms = bw_sms();
  if (two_d) {
    row_sum_kernel<<<(unsigned)std::min<int64_t>(sms * 4, (D + 7) / 8), 256, 0, st>>>(w, f->dists,
                                                                                 D - 1, R);
  }
  if (count > 0) {
    int64_t blocks = std::min<int64_t>((int64_t)sms * 8, (count + kBwThreads - 1) / kBwThreads);
    if (two_d)
      scatter_2d_kernel<<<(unsigned)blocks, kBwThreads, 0, st>>>(
          w, f->dists, D, R, reinterpret_cast<const uint2*>(u), reinterpret_cast<const int2*>(idx),
          reinterpret_cast<const float2*>(pos), reinterpret_cast<const float2*>(gpos), count, acc);
    else
      scatter_1d_kernel<<<(unsigned)blocks, kBwThreads, 0, st>>>(w, f->dists, D, u, dist_id, idx,
                                                                 pos, gpos, count, acc);
  }
  const int64_t tiles = (N + kBwTile - 1) / kBwTile;
  dist_total_kernel<<<(unsigned)tiles, kBwThreads, 0, st>>>(acc, f->dists, D, N, G);
  suffix_kernel<<<(unsigned)tiles, kBwThreads, 0, st>>>(acc, f->dists, D, N, Nw, G, flags, carry,
                                                        incl, ticket, grad_w, gradR, f->status);
  if (two_d)
    add_row_kernel<<<(unsigned)std::min<int64_t>(sms * 4, D - 1), 256, 0, st>>>(grad_w, f->dists, D - 1,
                                                                         gradR);
  return cudaGetLastError();
}

}  // namespace rtf
