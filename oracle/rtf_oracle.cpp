// Oracle for radix-tree-forest sampling (Binder & Keller, "Massively Parallel
// Construction of Radix Tree Forests for the Efficient Sampling of Discrete or
// Piecewise Constant Probability Distributions").
//
// TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, sequential CPU
// statement of what the GPU path computes.  Only the test suite, the smoke
// check and the CPU-baseline leg of the benchmark may load it.  It shares no
// code, header, table or helper with the CUDA library: it does not include the
// library header and nothing here is linked into the library.
//
// Every function cites the passage of the paper it follows.  Where the paper
// is silent or ambiguous the reading taken is stated in the comment (the same
// readings are listed in the design notes of the repository).
//
// Arithmetic: exact integers (unsigned __int128 where products exceed 64
// bits); the in-bin position and the gradient are computed in fp64.
//
// Parity status per function (what pins it in tests/test_oracle_*.py):
//   orc_scale / orc_quantize / orc_cdf  - exact rational arithmetic (Python
//       fractions) on random and edge-case weights; T < 2^62 bound.
//   orc_index                            - brute-force scan of the definition
//       P_{i-1} <= xi < P_i; sine-64 counts printed in the paper (Fig. 7);
//       stratification bound |count_i - p_i 2^k| < 1.
//   orc_position                         - exact rational arithmetic; n = 1
//       closed form pos = u / 2^32.
//   orc_keys                             - the equivalence u >= K_j <=> t(u) >= C_j
//       checked at K_j - 1 and K_j.
//   orc_forest (Algorithm 1)             - the worked forest of Fig. 11 node
//       for node; an independent top-down (rightmost maximum) recursive
//       definition on random tiny inputs; split-at-highest-differing-bit and
//       in-order invariants; Algorithm 2 over it equals orc_index for every u
//       of a grid.
//   orc_guide                            - Fig. 11 guide cells; brute force of
//       "single interval covers the cell" on tiny inputs.
//   orc_quad / orc_descend_quad          - the 4-ary descent equals orc_index
//       for every u of a grid; its record count is ceil((v - 1) / 2) for v
//       binary visits of Algorithm 2; record splits ascend in key order.
//   orc_descend / orc_descend_steps      - Algorithm 2 equals orc_index for
//       every u of a grid; its visit count equals the depth of the sample's
//       interval in the top-down tree of its cell; at most 1 + (32 - m)
//       visits with 2^m cells.
//   orc_grad_q / orc_grad64              - central finite differences of an
//       independent fp64 relaxed forward at the quantised weights w' (1-D and
//       2-D); the relaxation at w' equals the exact position (it is the
//       function the GPU computes), at the unquantised weights it does not;
//       n = 1 gives zero; two-bin closed form.
//   orc_quantized_weights                - exact rationals: w' = floor(w 2^S) 2^-S.
//   orc_relaxed_position                 - equals an independent fp64
//       restatement of x = (xi W - C_i) / w_i.
//   The 2-D composition (oracle.py: build_env, sample_env) - marginal equal to
//       the exact row totals; rows, columns and positions equal their
//       definition recomputed in Python integers.
//   Table 1's printed statistics         - parity unpinned: the paper gives
//       neither n, the table size nor the "4 spikes" density.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

typedef unsigned __int128 u128;

namespace {

const int ORC_OK = 0;
const int ORC_BAD_WEIGHT = 1;   // negative, NaN or infinite weight
const int ORC_ZERO_TOTAL = 2;   // no positive weight

// "1" of Algorithm 1 (the replacement value at a partition or array
// boundary).  Reading: the replacement stands for the largest possible
// distance, larger than any XOR of two keys in [0, 2^32].
const uint64_t ORC_MAX_DISTANCE = uint64_t(1) << 40;

int ceil_log2(int64_t n) {
  int c = 0;
  while ((int64_t(1) << c) < n) ++c;
  return c;
}

}  // namespace

extern "C" {

// Quantisation scale (the exact fixed-point reading of p_i and P_k, Sec. 1).
// B = 62 - ceil(log2 n_group); e_max = max floor(log2 w_i) over w_i > 0;
// S = B - 1 - e_max, so that every q_i = floor(w_i 2^S) < 2^B and the total
// of n_group such values stays below 2^62.  Sec. 1 assumes p_i > 0; zero
// weights are accepted as unreachable bins, negative / NaN / Inf rejected.
int orc_scale(const float* w, int64_t n, int64_t n_group, int32_t* S_out) {
  int e_max = 0;
  bool any = false;
  for (int64_t i = 0; i < n; ++i) {
    float x = w[i];
    if (std::isnan(x) || std::isinf(x) || x < 0.0f) return ORC_BAD_WEIGHT;
    if (x > 0.0f) {
      int e;
      std::frexp((double)x, &e);  // x = f 2^e, f in [0.5, 1)
      int fl = e - 1;             // floor(log2 x), also for subnormals
      if (!any || fl > e_max) e_max = fl;
      any = true;
    }
  }
  if (!any) return ORC_ZERO_TOTAL;
  int B = 62 - ceil_log2(n_group);
  *S_out = B - 1 - e_max;
  return ORC_OK;
}

// q_i = floor(w_i 2^S).  The product of a float and a power of two is exact
// in double (53-bit significand, no overflow or underflow for these ranges),
// so the floor is exact.
void orc_quantize(const float* w, int64_t n, int32_t S, uint64_t* q) {
  for (int64_t i = 0; i < n; ++i) {
    double v = std::ldexp((double)w[i], S);
    q[i] = (uint64_t)std::floor(v);
  }
}

// Prefix sums, Sec. 1: P_0 = 0, P_k = sum_{i<=k} p_i, here on the integers:
// C[0] = 0, C[k+1] = C[k] + q[k]; C[n] = T.
void orc_cdf(const uint64_t* q, int64_t n, uint64_t* C) {
  C[0] = 0;
  for (int64_t k = 0; k < n; ++k) C[k + 1] = C[k] + q[k];
}

// The uniform variate: a 32-bit sample u stands for xi = u / 2^32 and maps to
// the integer CDF domain as t = floor(u T / 2^32).
static uint64_t t_of(uint32_t u, uint64_t T) {
  return (uint64_t)(((u128)u * (u128)T) >> 32);
}

// Inverse CDF, Sec. 1: P^{-1}(xi) = i  <=>  P_{i-1} <= xi < P_i.  With the
// 0-based integer CDF this is the i with C[i] <= t < C[i+1]; the library
// routine std::upper_bound gives the first C greater than t.
int64_t orc_index(const uint64_t* C, int64_t n, uint32_t u) {
  uint64_t t = t_of(u, C[n]);
  const uint64_t* p = std::upper_bound(C, C + n + 1, t);
  return (int64_t)(p - C) - 1;
}

// In-bin ("sub-pixel") position, Sec. 5: the relative position of xi inside
// the selected interval rescaled to [0, 1):
//   pos = (u T - C_i 2^32) / (q_i 2^32)   with xi = u / 2^32 exactly.
double orc_position(const uint64_t* C, int64_t n, uint32_t u, int64_t i) {
  (void)n;
  u128 num = (u128)u * (u128)C[n] - ((u128)C[i] << 32);
  u128 den = (u128)(C[i + 1] - C[i]) << 32;
  return (double)num / (double)den;
}

// Batched convenience: index and position of each sample.
void orc_sample(const uint64_t* C, int64_t n, const uint32_t* u, int64_t ns,
                int32_t* idx, double* pos) {
  for (int64_t s = 0; s < ns; ++s) {
    int64_t i = orc_index(C, n, u[s]);
    idx[s] = (int32_t)i;
    pos[s] = orc_position(C, n, u[s], i);
  }
}

// Keys in the sample domain.  The interval lower bounds data[j] of
// Algorithm 1 (Sec. 3.2) are taken as 32-bit fixed point: K_j is the smallest
// u with t(u) >= C_j, i.e. K_j = ceil(C_j 2^32 / T); K_0 = 0, K_n = 2^32.
// A key lies in cell floor(K_j M / 2^32) of M equal cells (the guide table of
// the Cutpoint method, Sec. 2.5); K_j = 2^32 falls in the unreachable cell M.
void orc_keys(const uint64_t* C, int64_t n, int64_t M, uint64_t* K,
              int64_t* cell) {
  uint64_t T = C[n];
  for (int64_t j = 0; j <= n; ++j) {
    u128 num = ((u128)C[j] << 32) + (u128)(T - 1);
    K[j] = (uint64_t)(num / (u128)T);
    if (j < n) cell[j] = (int64_t)(((u128)K[j] * (u128)M) >> 32);
  }
}

// Start of guide cell g in the sample domain: the smallest u with
// floor(u M / 2^32) >= g.
static uint64_t cell_start(int64_t g, int64_t M) {
  u128 num = ((u128)g << 32) + (u128)(M - 1);
  return (uint64_t)(num / (u128)M);
}

// Algorithm 1 (Sec. 3.2), run sequentially: the leaves are taken one after the
// other and each climbs until it is the first of two siblings to reach their
// parent; the exchange on otherBounds is a plain read-then-write.  The order of
// the leaves does not change the result (each parent records the two children
// whichever arrives first).
//
// Node enumeration (Sec. 3.1): the node that splits between leaves k-1 and k
// has index k.  Child references: a node index >= 0, or ~i for leaf i.
//
// Distances: valueLow XOR valueNeighborLow against valueHigh XOR
// valueNeighborHigh on the fixed-point keys.  A neighbour outside the array or
// in another cell is replaced by "1", read here as the largest distance
// (ORC_MAX_DISTANCE).  The strict ">" sends equal distances to child 1.
//
// Root convention (caption of Fig. 11): the node of a cell's first leaf j0 is
// the cell root; Algorithm 1 gives it the right child; its left child is set
// to the left neighbour interval ~(j0 - 1), and to ~0 for j0 = 0, where it
// cannot be reached.
void orc_forest(const uint64_t* K, const int64_t* cell, int64_t n,
                int32_t* nodes) {
  std::vector<int64_t> otherBounds(n, -1);
  for (int64_t j = 0; j < 2 * n; ++j) nodes[j] = 0;
  auto distance_low = [&](int64_t lo) -> uint64_t {
    if (lo - 1 < 0 || cell[lo - 1] < cell[lo]) return ORC_MAX_DISTANCE;
    return K[lo] ^ K[lo - 1];
  };
  auto distance_high = [&](int64_t hi) -> uint64_t {
    if (hi + 1 >= n || cell[hi + 1] > cell[hi]) return ORC_MAX_DISTANCE;
    return K[hi] ^ K[hi + 1];
  };
  for (int64_t i = 0; i < n; ++i) {
    int64_t nodeId = ~i;  // leaf_i
    int64_t range[2] = {i, i};
    int64_t otherBound;
    do {
      uint64_t dLow = distance_low(range[0]);
      uint64_t dHigh = distance_high(range[1]);
      int child = (dLow > dHigh) ? 0 : 1;
      int64_t parent = (child == 0) ? range[1] + 1 : range[0];
      nodes[2 * parent + child] = (int32_t)nodeId;
      otherBound = otherBounds[parent];
      otherBounds[parent] = range[child];
      if (otherBound != -1) {
        range[1 - child] = otherBound;
        nodeId = parent;
      }
    } while (otherBound != -1);
  }
  for (int64_t j = 0; j < n; ++j) {
    if (j == 0 || cell[j - 1] != cell[j]) {
      int64_t left = j > 0 ? j - 1 : 0;
      nodes[2 * j + 0] = (int32_t)(~left);
    }
  }
}

// Guide table (Cutpoint method, Sec. 2.5, with the encoding of Sec. 3.2): a
// cell that only one interval overlaps stores ~i (most significant bit set);
// otherwise it stores the root of the cell's tree, which is the cell's first
// leaf.  Reading for zero-width intervals: "only one interval" means one
// interval of non-zero width, i.e. the cell has no key inside it, or all its
// keys equal the cell start (then the last of them covers the whole cell).
void orc_guide(const uint64_t* C, const uint64_t* K, const int64_t* cell,
               int64_t n, int64_t M, int32_t* guide) {
  int64_t j = 0;
  for (int64_t g = 0; g < M; ++g) {
    uint64_t s = cell_start(g, M);
    while (j < n && cell[j] < g) ++j;
    int64_t j0 = j;
    int64_t j1 = j0 - 1;
    while (j1 + 1 < n && cell[j1 + 1] == g) ++j1;
    if (j1 < j0) {
      // no key in the cell: the interval containing the cell start covers it
      int64_t i = orc_index(C, n, (uint32_t)s);
      guide[g] = (int32_t)(~i);
    } else if (K[j1] == s) {
      guide[g] = (int32_t)(~j1);
    } else {
      guide[g] = (int32_t)j0;
    }
  }
}

// Algorithm 2 (Sec. 3.2): g = floor(xi M); j = table[g]; while msb(j) = 0,
// go to child 0 if xi < data[j] else child 1; return ~j.  In the sample
// domain "xi < data[j]" is u < K_j.
int64_t orc_descend(const int32_t* guide, const int32_t* nodes,
                    const uint64_t* K, int64_t M, uint32_t u) {
  int64_t g = (int64_t)(((u128)u * (u128)M) >> 32);
  int32_t j = guide[g];
  while (j >= 0) {
    j = ((uint64_t)u < K[j]) ? nodes[2 * j + 0] : nodes[2 * j + 1];
  }
  return (int64_t)(~j);
}

// Number of node visits of Algorithm 2 for one sample (0 when the guide entry
// already names the interval).
int32_t orc_descend_steps(const int32_t* guide, const int32_t* nodes,
                          const uint64_t* K, int64_t M, uint32_t u) {
  int64_t g = (int64_t)(((u128)u * (u128)M) >> 32);
  int32_t j = guide[g];
  int32_t steps = 0;
  while (j >= 0) {
    j = ((uint64_t)u < K[j]) ? nodes[2 * j + 0] : nodes[2 * j + 1];
    ++steps;
  }
  return steps;
}

// k-ary trees (the section on k-ary trees and the remark on branching factors
// at the end of Sec. 5): a branching factor of four results from collapsing two
// levels of a binary tree.  For node j with children a = child0(j) and
// b = child1(j), the 4-ary record holds the three splits in key order as node
// ids, (a, j, b), and the four grandchildren (child0(a), child1(a), child0(b),
// child1(b)).  Reading: a child that is a leaf has no split of its own, so its
// side repeats the split of j and names the leaf in both of its slots; the
// second comparison on that side then always picks the leaf (u < K_j holds on
// the left, fails on the right).
void orc_quad(const int32_t* nodes, int64_t n, int32_t* split, int32_t* child) {
  for (int64_t j = 0; j < n; ++j) {
    const int32_t a = nodes[2 * j + 0];
    const int32_t b = nodes[2 * j + 1];
    split[3 * j + 1] = (int32_t)j;
    if (a >= 0) {
      split[3 * j + 0] = a;
      child[4 * j + 0] = nodes[2 * a + 0];
      child[4 * j + 1] = nodes[2 * a + 1];
    } else {
      split[3 * j + 0] = (int32_t)j;
      child[4 * j + 0] = a;
      child[4 * j + 1] = a;
    }
    if (b >= 0) {
      split[3 * j + 2] = b;
      child[4 * j + 2] = nodes[2 * b + 0];
      child[4 * j + 3] = nodes[2 * b + 1];
    } else {
      split[3 * j + 2] = (int32_t)j;
      child[4 * j + 2] = b;
      child[4 * j + 3] = b;
    }
  }
}

// Algorithm 2 over the 4-ary records: the guide entry and the decision at the
// cell's root node as in Algorithm 2 (the root's record sits in the guide
// entry), then one 4-ary record per two levels below it: compare with the
// middle split, then with the split of the chosen side.  Returns the interval;
// *records receives the number of 4-ary records read.
int64_t orc_descend_quad(const int32_t* guide, const int32_t* nodes, const int32_t* split,
                         const int32_t* child, const uint64_t* K, int64_t M, uint32_t u,
                         int32_t* records) {
  int64_t g = (int64_t)(((u128)u * (u128)M) >> 32);
  int32_t j = guide[g];
  int32_t r = 0;
  if (j >= 0) j = ((uint64_t)u < K[j]) ? nodes[2 * j + 0] : nodes[2 * j + 1];
  while (j >= 0) {
    const int32_t* s = split + 3 * (int64_t)j;
    const int32_t* c = child + 4 * (int64_t)j;
    if ((uint64_t)u < K[s[1]])
      j = ((uint64_t)u < K[s[0]]) ? c[0] : c[1];
    else
      j = ((uint64_t)u < K[s[2]]) ? c[2] : c[3];
    ++r;
  }
  *records = r;
  return (int64_t)(~j);
}

// Whole build of one distribution: scale, quantise, CDF, keys, forest, guide.
int orc_build(const float* w, int64_t n, int64_t n_group, int64_t M,
              int32_t* S_out, uint64_t* C, int32_t* nodes, int32_t* guide) {
  int32_t S;
  int st = orc_scale(w, n, n_group, &S);
  if (st != ORC_OK) return st;
  *S_out = S;
  std::vector<uint64_t> q(n), K(n + 1);
  std::vector<int64_t> cell(n);
  orc_quantize(w, n, S, q.data());
  orc_cdf(q.data(), n, C);
  if (C[n] == 0) return ORC_ZERO_TOTAL;
  orc_keys(C, n, M, K.data(), cell.data());
  orc_forest(K.data(), cell.data(), n, nodes);
  orc_guide(C, K.data(), cell.data(), n, M, guide);
  return ORC_OK;
}

// Build from integer weights (the marginal of a 2-D map, whose weights are the
// exact row totals; no re-quantisation).
int orc_build_int(const uint64_t* q, int64_t n, int64_t M, uint64_t* C,
                  int32_t* nodes, int32_t* guide) {
  std::vector<uint64_t> K(n + 1);
  std::vector<int64_t> cell(n);
  orc_cdf(q, n, C);
  if (C[n] == 0) return ORC_ZERO_TOTAL;
  orc_keys(C, n, M, K.data(), cell.data());
  orc_forest(K.data(), cell.data(), n, nodes);
  orc_guide(C, K.data(), cell.data(), n, M, guide);
  return ORC_OK;
}

// Gradient of the in-bin position with respect to the weights (not in the
// paper).  Reading: the gradient of the forward that is actually computed,
//   x = (xi T - C_i) / q_i,   q_i = floor(w_i 2^S),
// with the floor of the quantisation passed straight through and the scale S
// held fixed.  In real units this is the relaxation
//   x = (xi W' - C'_i) / w'_i,   w'_k = q_k 2^-S,  W' = sum_k w'_k,
//   C'_i = sum_{k<i} w'_k,
// differentiated at the quantised weights w' (it equals the computed forward
// there), with the bin i held fixed at the one the exact pipeline selected.
// Reverse mode, in fp64, per sample
//   dL/dW'   += g xi / w'_i,   dL/dC'_i += -g / w'_i,   dL/dw'_i += -g x / w'_i,
// then W' = sum w' and C'_i = sum_{k<i} w'_k give
//   dL/dw_k = dL/dW' + sum_{i>k} dL/dC'_i + dL/dw'_k(direct).
// x is taken from the exact integers (orc_position), not recomputed from real
// prefix sums: for bins far narrower than the total that recomputation loses
// most of its digits to cancellation.
//
// Input: the integer CDF C[0..n] of the distribution and its scale S (for the
// marginal of a 2-D map: the CDF of the exact row totals and the map's shared
// scale, so that w'_r = T_r 2^-S is the real total of row r).
void orc_grad_q(const uint64_t* C, int64_t n, int32_t S, const uint32_t* u,
                const int32_t* idx, const float* gx, int64_t ns, double* grad) {
  double dW = 0.0;
  std::vector<double> dC(n, 0.0), dwd(n, 0.0);
  for (int64_t s = 0; s < ns; ++s) {
    int64_t i = idx[s];
    double wq = std::ldexp((double)(C[i + 1] - C[i]), -S);
    double xi = std::ldexp((double)u[s], -32);
    double x = orc_position(C, n, u[s], i);
    double g = (double)gx[s];
    dW += g * xi / wq;
    dC[i] += -g / wq;
    dwd[i] += -g * x / wq;
  }
  double suffix = 0.0;  // sum_{i>k} dL/dC'_i
  for (int64_t k = n - 1; k >= 0; --k) {
    grad[k] = dW + suffix + dwd[k];
    suffix += dC[k];
  }
}

// The quantised weights in real units, w'_k = floor(w_k 2^S) 2^-S (exact in
// fp64: q_k has at most 24 significant bits).
void orc_quantized_weights(const float* w, int64_t n, int32_t S, double* wq) {
  for (int64_t k = 0; k < n; ++k) {
    double v = std::ldexp((double)w[k], S);
    wq[k] = std::ldexp(std::floor(v), -S);
  }
}

// The chain rule of orc_grad_q at arbitrary real weights, with x recomputed
// from them: x = (xi W - C_i) / w_i, W = sum w, C_i = sum_{k<i} w_k.  A
// statement of the relaxation on its own, for the finite-difference pins.
void orc_grad64(const double* w, int64_t n, const uint32_t* u, const int32_t* idx,
                const float* gx, int64_t ns, double* grad) {
  std::vector<double> Creal(n + 1);
  Creal[0] = 0.0;
  for (int64_t k = 0; k < n; ++k) Creal[k + 1] = Creal[k] + w[k];
  double W = Creal[n];
  double dW = 0.0;
  std::vector<double> dC(n, 0.0), dwd(n, 0.0);
  for (int64_t s = 0; s < ns; ++s) {
    int64_t i = idx[s];
    double xi = std::ldexp((double)u[s], -32);
    double x = (xi * W - Creal[i]) / w[i];
    double g = (double)gx[s];
    dW += g * xi / w[i];
    dC[i] += -g / w[i];
    dwd[i] += -g * x / w[i];
  }
  double suffix = 0.0;
  for (int64_t k = n - 1; k >= 0; --k) {
    grad[k] = dW + suffix + dwd[k];
    suffix += dC[k];
  }
}

// The relaxed fp64 forward of the same function (used by the finite
// difference check of orc_grad): x for fixed bins.
void orc_relaxed_position(const double* w, int64_t n, const uint32_t* u,
                          const int32_t* idx, int64_t ns, double* x) {
  double W = 0.0;
  std::vector<double> Creal(n + 1);
  Creal[0] = 0.0;
  for (int64_t k = 0; k < n; ++k) Creal[k + 1] = Creal[k] + w[k];
  W = Creal[n];
  for (int64_t s = 0; s < ns; ++s) {
    int64_t i = idx[s];
    double xi = std::ldexp((double)u[s], -32);
    x[s] = (xi * W - Creal[i]) / w[i];
  }
}

}  // extern "C"
