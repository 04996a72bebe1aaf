/*
 * rtf.h - C interface of the GB300 radix-tree-forest sampler.
 *
 * The library builds, on one GPU, the auxiliary structure of Binder & Keller,
 * "Massively Parallel Construction of Radix Tree Forests for the Efficient
 * Sampling of Discrete or Piecewise Constant Probability Distributions"
 * (arXiv:1901.05423), and maps uniform samples through it:
 *
 *   - the prefix-sum CDF of the weights (Sec. 1: P_0 = 0, P_k = sum p_i),
 *     made exact on 64-bit integers;
 *   - a guide table of 2^m equal cells over [0, 1) (the Cutpoint method,
 *     Sec. 2.5) whose entries use the two's complement encoding of Sec. 3.2;
 *   - one radix tree per cell, all built at once bottom-up (Algorithm 1,
 *     Sec. 3.2);
 *   - the monotone mapping of a sample through its guide cell and a tree
 *     descent (Algorithm 2) to a bin index and an in-bin position (Sec. 5);
 *   - the gradient of the in-bin position with respect to the weights (not in
 *     the paper).
 *
 * Conventions shared by every call:
 *   - Every pointer whose name does not say "host" is DEVICE memory of the
 *     current CUDA device.  The caller allocates and owns all of it; the
 *     library never allocates, frees or synchronises, so every call may be
 *     captured into a CUDA graph.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  All work
 *     is ordered on it.
 *   - The return value reports argument errors and launch errors only.  Errors
 *     that depend on the data (a negative, NaN or infinite weight, a
 *     distribution whose weights are all zero, a bounded wait that ran out)
 *     are OR-ed into the device word `rtf_forest.status` as RTF_STATUS_* bits,
 *     which the caller reads after synchronising.  Outputs are undefined
 *     unless the call returned RTF_OK and the status word is 0.
 *
 * Exact arithmetic (the reading this library takes of P_k and xi):
 *   - weights are float32, w_i >= 0, finite; a zero weight is an empty,
 *     unreachable bin;
 *   - all weights of one distribution (or of one shared-scale group) are
 *     turned into integers q_i = floor(w_i 2^S) with S = B - 1 - e_max,
 *     B = 62 - ceil(log2 n_group), e_max = max floor(log2 w_i); the CDF is the
 *     exact integer prefix sum C_0 = 0, C_{k+1} = C_k + q_k, T = C_n < 2^62;
 *   - a 32-bit sample u stands for xi = u / 2^32 and selects the bin i with
 *     C_i <= t < C_{i+1}, t = floor(u T / 2^32);
 *   - its in-bin position is (u T - C_i 2^32) / (q_i 2^32), returned in
 *     float32 (within a few ulp of the exact value, clamped below 1).
 */
#ifndef RTF_H_
#define RTF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Synchronous return codes. */
typedef enum rtf_status {
  RTF_OK = 0,
  RTF_EINVAL = 1,     /* a null pointer, a size out of range, a misaligned pointer */
  RTF_EWORKSPACE = 2, /* the workspace is smaller than the *_workspace_size call says */
  RTF_ECUDA = 3       /* a CUDA launch or runtime call failed */
} rtf_status;

/* Bits of the device status word (rtf_forest.status). */
#define RTF_STATUS_BAD_WEIGHT 0x1u /* a weight is negative, NaN or infinite */
#define RTF_STATUS_ZERO_TOTAL 0x2u /* a distribution has no positive weight */
#define RTF_STATUS_TIMEOUT 0x4u    /* a bounded wait inside a kernel ran out */
#define RTF_STATUS_BAD_PLAN 0x8u   /* batched plan: n_d < 1, m_d outside [0, 31] */
#define RTF_STATUS_INVARIANT 0x10u /* an internal bound of the forest construction was
                                      exceeded (cannot happen for a valid build; the
                                      forest is incomplete if it is set) */

/* rtf_forest.flags */
#define RTF_FOREST_MARGINAL 0x1 /* the last distribution is the marginal over the
                                   others (2-D map, Sec. 5); see rtf_build_batched */

/* rtf_sample / rtf_sample_backward modes */
#define RTF_SAMPLE_1D 0 /* one sample u per output; dist_id selects the distribution */
#define RTF_SAMPLE_2D 1 /* (u1, u2) pairs; row from the marginal, column from the row */
/* flag OR-ed into the mode of rtf_sample: the cutpoint method with a binary
   search (the paper's comparator, Sec. 2.5) on the same structure instead of
   the radix forest; identical bins and positions */
#define RTF_SAMPLE_BSEARCH 0x100
/* hint OR-ed into the mode of rtf_sample: neighbouring samples are close (a
   sorted or low-discrepancy sequence in order).  For one distribution in 1-D
   with the radix forest, each thread then maps runs of consecutive samples,
   reusing the previous sample's bin or stepping to the next bins and
   descending (Algorithm 2) only where neither holds; otherwise the hint only
   selects the full grid (without it, a structure larger than L2 is sampled by
   fewer resident threads, which keeps more of it in L2 for scattered
   samples).  Results do not depend on the hint: every way finds the unique
   bin with C_i <= t < C_{i+1}. */
#define RTF_SAMPLE_COHERENT 0x200

/*
 * One node record, 16 bytes, in device memory.  Record j of a distribution
 * holds the CDF value C_j and the two children of node j.
 *
 * Node enumeration (Sec. 3.1): node j splits between leaves j-1 and j, so the
 * descent compares against the CDF value with the node's own index (Sec. 3.2,
 * Algorithm 2), which is why the CDF is interleaved with the children (the
 * layout the paper suggests at the end of Sec. 3.2).  A child reference
 * c >= 0 is a node index, c < 0 is the leaf (bin) ~c.  The node of the first
 * leaf j0 of every cell is that cell's root: child[1] is the cell's tree and
 * child[0] the interval overlapping the cell from the left, ~(j0 - 1), or ~0
 * for j0 = 0 (caption of Fig. 11).  Indices are local to the distribution.
 */
typedef struct rtf_node {
  uint64_t cdf;      /* C_j (exact integer CDF, local to the distribution) */
  int32_t child[2];  /* child[0] taken when t < C_j, child[1] otherwise */
} rtf_node;

/*
 * Guide record of one cell, 32 bytes (Sec. 3.2: the guide table points to the
 * root of the cell's tree; here the entry carries the root's decision itself).
 *
 *   cdf, child  a copy of the record of the cell's root, or {C_i, ~i, ~i} for
 *               a cell that one interval i covers.
 *   lo          lower CDF bound of the interval reached through child[0] of
 *               the root: C_{j0-1} (0 for j0 = 0); C_i for a covered cell.
 *   hi          upper CDF bound of the cell's last interval j1: C_{j1+1}, or T
 *               when j1 = n - 1; C_{i+1} for a covered cell.
 *
 * The two neighbours of a leaf in the in-order sequence of a binary tree are
 * its nearest ancestors entered from the right and from the left, so while
 * descending, the lower bound of the final interval is the CDF value of the
 * last node left through child[1] and its upper bound that of the last node
 * left through child[0]; lo and hi stand in where such an ancestor lies
 * outside the cell's tree.  The in-bin position (Sec. 5) thus needs no load
 * after the descent.
 */
typedef struct rtf_guide_rec {
  uint64_t cdf;
  int32_t child[2];
  uint64_t lo;
  uint64_t hi;
} rtf_guide_rec;

/*
 * Per-distribution parameters, 64 bytes, in device memory.  The build writes
 * every field; the caller only allocates the array.
 */
typedef struct rtf_dist {
  int64_t elem_off;  /* first weight / node record of the distribution */
  int64_t n;         /* number of weights (bins) */
  int64_t guide_off; /* first guide cell */
  uint64_t total;    /* T = C_n */
  uint64_t recip;    /* floor((2^128 - 1) / (T << shift)) - 2^64 (key arithmetic) */
  int32_t m;         /* guide bits: the distribution has 2^m cells */
  int32_t scale;     /* S of the fixed-point weights (0 for the marginal) */
  int32_t shift;     /* number of leading zero bits of T */
  int32_t flags;     /* internal */
  int64_t reserved;
} rtf_dist;

/*
 * A forest: the caller fills this host struct with sizes and device pointers
 * (all caller-allocated) before a build, and passes it to the sampler.
 */
typedef struct rtf_forest {
  int32_t num_dists; /* D >= 1 */
  int32_t flags;     /* RTF_FOREST_* */
  int64_t num_elems; /* N = sum of n_d: length of `nodes` */
  int64_t num_cells; /* G = sum of 2^m_d < 2^31: length of `guide` */
  int32_t max_m;     /* largest m_d (host copy; chooses the shared-memory guide path) */
  int32_t reserved;
  rtf_node *nodes;   /* device [N], 16-byte aligned */
  int32_t *guide;    /* device [G] */
  rtf_dist *dists;   /* device [D] */
  uint32_t *status;  /* device [1]: RTF_STATUS_* bits, set to 0 by each build */
  rtf_guide_rec *guide_recs; /* device [G], 32-byte aligned: guide records */
} rtf_forest;

/* Library version string. */
const char *rtf_version(void);

/* Human-readable name of a return code. */
const char *rtf_status_string(rtf_status s);

/*
 * Bytes of workspace rtf_build / rtf_build_batched need for N elements, D
 * distributions and G guide cells.  The workspace needs no initial contents
 * (each build writes or clears every part it reads) and keeps nothing between
 * builds, but it must not serve two builds that run at the same time.
 */
size_t rtf_build_workspace_size(int64_t num_elems, int32_t num_dists,
                                int64_t num_cells);

/*
 * Build the structure of one distribution.
 *
 *   w        device float32[n], 4-byte aligned: the weights (Sec. 1: p up to
 *            normalisation), w_i >= 0, finite, at least one positive.
 *   n        1 <= n <= 2^31 - 2^16.
 *   m        guide bits, 0 <= m <= 30: 2^m cells (Sec. 2.5, Sec. 3.2).
 *   f        f->num_dists == 1, f->num_elems == n, f->num_cells == 2^m,
 *            f->max_m == m; nodes[n], guide[2^m], guide_recs[2^m], dists[1],
 *            status[1] allocated.
 *   ws       device workspace of at least rtf_build_workspace_size(n, 1, 2^m)
 *            bytes, 256-byte aligned.
 *
 * Steps (all on `stream`, no host synchronisation): validation and scale
 * (max exponent), exact integer CDF by a decoupled-lookback scan, keys
 * K_j = ceil(C_j 2^32 / T), Algorithm 1 over all cells at once, guide table.
 * Results: f->nodes, f->guide, f->dists[0] and *f->status.
 */
rtf_status rtf_build(const float *w, int64_t n, int32_t m, rtf_forest *f,
                     void *ws, size_t ws_bytes, void *stream);

/*
 * rtf_build without a caller workspace.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory where
 * they build (a plugin inside a host application that owns the device memory
 * budget, a real-time loop that forbids allocation after start-up, a foreign
 * runtime that hands over raw pointers but cannot reach an allocator).
 * Arguments, results and device status are those of rtf_build; the caller
 * still allocates w and the forest buffers.
 *
 * The scratch is a fixed 10 MiB array inside the library, held on every GPU
 * that loads the library until the process exits.  It fits n <= 2^20 weights
 * and m <= 16 guide bits; larger sizes return RTF_EWORKSPACE without touching
 * the GPU.  The first call in a CUDA context (normally: the first call on a
 * device) looks up the array's device address with that context current, so
 * make that first call before capturing a stream.  The address is kept per
 * context for the rest of the process; it does not survive cudaDeviceReset,
 * after which this entry point must not be called again in the same process.
 * Every call shares the one array and leaves its contents behind (each call
 * clears what must start at zero): calls that overlap on the GPU, from two
 * streams or two threads, race and corrupt each other's results; serialise
 * them.  Nothing here calls cudaMalloc or cudaFree.
 */
rtf_status rtf_build_static(const float *w, int64_t n, int32_t m, rtf_forest *f,
                            void *stream);

/*
 * Build many distributions at once (Sec. 5: several tables and trees are
 * built together by treating the index boundary of every distribution like a
 * cell boundary in Algorithm 1).
 *
 *   w              device float32[offsets[D_w]], 4-byte aligned, where
 *                  D_w = D (independent distributions) or D - 1 (marginal mode).
 *   offsets        device int64[D + 1]: distribution d owns elements
 *                  [offsets[d], offsets[d+1]); offsets[0] = 0, n_d >= 1.
 *   m              device int32[D]: guide bits per distribution, 0..30.
 *   guide_offsets  device int64[D + 1]: guide_offsets[0] = 0,
 *                  guide_offsets[d+1] = guide_offsets[d] + 2^m[d].
 *   f              f->num_dists = D, f->num_elems = offsets[D],
 *                  f->num_cells = guide_offsets[D], f->max_m = max m[d].
 *
 * Without RTF_FOREST_MARGINAL each distribution has its own scale
 * (n_group = n_d).  With RTF_FOREST_MARGINAL in f->flags (a 2-D piecewise
 * constant map, Sec. 5): distributions 0..D-2 are the rows (conditionals) and
 * share one scale (n_group = offsets[D-1]); distribution D-1 has n = D - 1
 * and its integer weights are the exact row totals T_0 .. T_{D-2} (the
 * marginal); w then holds only the offsets[D-1] row weights.
 */
rtf_status rtf_build_batched(const float *w, const int64_t *offsets,
                             const int32_t *m, const int64_t *guide_offsets,
                             rtf_forest *f, void *ws, size_t ws_bytes,
                             void *stream);

/*
 * Map samples to bins (Algorithm 2, Sec. 3.2) and in-bin positions (Sec. 5).
 *
 * RTF_SAMPLE_1D: u is uint32[count]; dist_id is NULL (all samples use
 *   distribution 0) or int32[count] (distribution of each sample, 0..D-1).
 *   idx_out int32[count] receives the bin (local to its distribution),
 *   pos_out float32[count] the position in [0, 1).
 * RTF_SAMPLE_2D: f must carry RTF_FOREST_MARGINAL; u is uint32[2 count] as
 *   (u1, u2) pairs, dist_id must be NULL; u1 selects the row through the
 *   marginal, u2 the column through that row (Sec. 5).  idx_out int32[2 count]
 *   receives (row, column), pos_out float32[2 count] (row position, column
 *   position).
 * RTF_SAMPLE_COHERENT may be OR-ed into either mode (a performance hint).
 * RTF_SAMPLE_BSEARCH may be OR-ed into either mode: each sample is then
 *   found by a binary search over the CDF between the first intervals of its
 *   cell and of the next cell (the cutpoint method), not by a tree descent.
 * u, idx_out and pos_out must be 16-byte aligned; count >= 0.
 */
rtf_status rtf_sample(const rtf_forest *f, const uint32_t *u,
                      const int32_t *dist_id, int64_t count, int32_t mode,
                      int32_t *idx_out, float *pos_out, void *stream);

/*
 * Launch shape of the samplers: the resident blocks of 256 threads per SM
 * that each kind of sampling launch is given (its grid is that times the SM
 * count, capped by the work).  0 keeps the built-in choice, measured on
 * GB300: 3 for one distribution with scattered samples over records larger
 * than L2 (fewer resident descents keep more of the structure in L2), 8 for
 * one distribution otherwise, 8 with a distribution id per sample, 8 in 2-D.
 * (The coherent sampler always runs one wave of resident blocks.)  The
 * setting is process-wide, applies to launches issued after the call and
 * never changes a result.  Each value must lie in [0, 64].
 */
typedef struct rtf_launch_shape {
  int32_t single_large; /* one distribution, records larger than L2, scattered samples */
  int32_t single;       /* one distribution otherwise (without the coherence hint) */
  int32_t tagged;       /* a distribution id per sample */
  int32_t pairs;        /* RTF_SAMPLE_2D */
} rtf_launch_shape;

/* Sets the launch shape; NULL restores the built-in choices. */
rtf_status rtf_set_launch_shape(const rtf_launch_shape *shape);

/* The shape in effect, built-in choices filled in. */
rtf_status rtf_get_launch_shape(rtf_launch_shape *shape);

/*
 * rtf_sample for samples that live in host memory: the samples are copied to
 * the device, mapped and the results copied back in chunks of `chunk` samples
 * (a multiple of 4), with the copies of one chunk overlapping the sampling of
 * another.  Not in the paper: the host-side counterpart of the sampler.
 *
 *   u_host       uint32[count] (2 count in 2-D), or NULL when u_dev already
 *                holds the samples.  Page-locked host memory lets the copies
 *                run asynchronously; pageable memory works but serialises.
 *   u_dev        device uint32[count] (2 count), 16-byte aligned: receives
 *                the samples (when u_host is given), read by the kernels.
 *   dist_id_host / dist_id_dev   as u for the per-sample distribution ids
 *                (1-D only); both NULL for distribution 0.
 *   idx_dev, pos_dev   device outputs as for rtf_sample (16-byte aligned);
 *                they keep the results for later device work (a backward).
 *   idx_host, pos_host host outputs (either may be NULL: no copy back).
 *   mode         as for rtf_sample.
 *
 *   done_event   NULL, or a cudaEvent_t of the caller (see below).
 *
 * Ordering: the copies start after the work already queued on `stream`.
 * With done_event NULL, `stream` waits for the last copy of both directions,
 * so synchronising it makes the host outputs complete.  With an event,
 * `stream` waits for the input copies only and the event is recorded after
 * the last copy back: later work on `stream` overlaps those copies, and the
 * caller waits for the event before it reads the host outputs or reuses
 * idx_dev / pos_dev.  The library keeps two copy streams and four events per
 * device for the rest of the process.
 */
rtf_status rtf_sample_pipelined(const rtf_forest *f, const uint32_t *u_host,
                                uint32_t *u_dev, const int32_t *dist_id_host,
                                int32_t *dist_id_dev, int64_t count, int32_t mode,
                                int32_t *idx_dev, float *pos_dev, int32_t *idx_host,
                                float *pos_host, int64_t chunk, void *done_event,
                                void *stream);

/*
 * Number of loads from the structure that each sample takes under the method
 * of `mode` (RTF_SAMPLE_1D, optionally | RTF_SAMPLE_BSEARCH): guide records
 * plus node records (radix forest) or CDF values (binary search), the
 * quantity of the paper's Table 1.  u and dist_id as for rtf_sample (4-byte
 * alignment suffices); loads_out int32[count] receives the counts, -1 for a
 * sample that found no interval.  One thread per sample, no positions: an
 * analysis aid, not a sampling path.
 */
rtf_status rtf_sample_loads(const rtf_forest *f, const uint32_t *u,
                            const int32_t *dist_id, int64_t count, int32_t mode,
                            int32_t *loads_out, void *stream);

/*
 * 4-ary record, 32 bytes (one L2 sector), in device memory: two levels of a
 * radix tree collapsed into one (the section on k-ary trees; the closing
 * remark on branching factors of Sec. 5).  Record j belongs to node j of the
 * same distribution; with a = child[0] and b = child[1] of node j:
 *
 *   cdf[0..2]  the three splits in order: C_a, C_j, C_b.  A side whose child is
 *              a leaf has no split of its own and repeats C_j.
 *   ref[0..3]  the four grandchildren child[0](a), child[1](a), child[0](b),
 *              child[1](b) (a leaf side names its leaf twice), each relative
 *              to j: 2 (k - j) for node k, 2 (i - j) + 1 for leaf (bin) i.
 *
 * A descent compares t with cdf[1], then with cdf[0] or cdf[2], and moves to
 * ref[0..3]: one load per two levels.  When a reference does not fit in
 * 16 bits (trees over more than 2^14 bins), bit RTF_QUAD_FAR of cdf[1] is set
 * and the descent takes one binary step through the node record instead.
 */
typedef struct rtf_quad_rec {
  uint64_t cdf[3];
  int16_t ref[4];
} rtf_quad_rec;

#define RTF_QUAD_FAR 0x8000000000000000ull

/*
 * Writes the 4-ary records of a built forest: quad must hold f->num_elems
 * records (32 bytes each, 32-byte aligned, device memory).  Stream-ordered
 * after the build that filled f; one thread per node.
 */
rtf_status rtf_build_quad(const rtf_forest *f, rtf_quad_rec *quad, void *stream);

/*
 * rtf_sample through the 4-ary records written by rtf_build_quad: the guide
 * record takes the decision of the cell's root, then each record two levels.
 * Same arguments, modes (RTF_SAMPLE_1D with or without dist_id, RTF_SAMPLE_2D;
 * RTF_SAMPLE_COHERENT is accepted as a hint, RTF_SAMPLE_BSEARCH is not) and
 * results as rtf_sample: the same bins and bit-identical positions.  When
 * loads_out (int32[count], or int32[2 count] in 2-D; 8-byte aligned) is not
 * NULL it receives
 * the structure loads of each sample (guide records plus 4-ary and node
 * records; -1 where no interval was found).
 */
rtf_status rtf_sample_quad(const rtf_forest *f, const rtf_quad_rec *quad,
                           const uint32_t *u, const int32_t *dist_id, int64_t count,
                           int32_t mode, int32_t *idx_out, float *pos_out,
                           int32_t *loads_out, void *stream);

/*
 * Check of the failure path of the library's bounded waits, without any
 * fault: one block runs the decoupled-lookback wait of the scans on a
 * predecessor status word that nothing publishes (scratch: two 64-bit words
 * of device memory, cleared by the call).  After its iteration limit (about
 * a second) the wait gives up, sets RTF_STATUS_TIMEOUT in *status (device
 * memory, not cleared) and the kernel returns; the context stays usable.
 * Stream-ordered.
 */
rtf_status rtf_check_bounded_wait(uint32_t *status, uint64_t *scratch, void *stream);

/* Bytes of workspace rtf_sample_backward needs. */
size_t rtf_backward_workspace_size(int64_t num_elems, int32_t num_dists);

/*
 * Gradient of the in-bin positions with respect to the weights (not in the
 * paper).  With the bin i of each sample held fixed, the position is the
 * real-valued x = (xi W - C_i) / w_i, W = sum_k w_k, C_i = sum_{k<i} w_k, so
 *
 *   dL/dw_k = sum_i Xi_i / w_i - sum_{i>k} A_i / w_i - X_k / w_k
 *
 * with, over the samples s that fell into bin i, A_i = sum g_s,
 * X_i = sum g_s x_s, Xi_i = sum g_s xi_s (g = dL/dx).  The library scatters
 * A_i / w_i and X_i / w_i per bin, sums Xi_i / w_i per distribution and runs a
 * reverse suffix scan per distribution.  In RTF_SAMPLE_2D mode the column
 * positions differentiate through their row and the row positions through the
 * marginal, whose weights are the row sums, so a row's marginal term is added
 * to every weight of that row.
 *
 *   w          the weights the forest was built from (same layout as the build).
 *   u, dist_id, idx, pos   the inputs and outputs of the forward rtf_sample.
 *   grad_pos   float32[count] (1-D) or [2 count] (2-D): dL/dpos.
 *   grad_w     float32[offsets[D_w]] output.
 *   ws         at least rtf_backward_workspace_size(N, D) bytes, 256-byte
 *              aligned; no state is kept between calls.
 */
rtf_status rtf_sample_backward(const rtf_forest *f, const float *w,
                               const uint32_t *u, const int32_t *dist_id,
                               const int32_t *idx, const float *pos,
                               const float *grad_pos, int64_t count,
                               int32_t mode, float *grad_w, void *ws,
                               size_t ws_bytes, void *stream);

/*
 * The backward in three steps, for gradients accumulated over several sample
 * batches or computed while later samples are still being drawn
 * (rtf_sample_backward is the three in a row):
 *
 *   rtf_backward_begin       clears the per-bin sums held in ws.
 *   rtf_backward_accumulate  adds the terms {dL/dpos, dL/dpos * pos} of
 *                            `count` samples (inputs as for
 *                            rtf_sample_backward) to the per-bin sums; any
 *                            number of calls, any split of the samples.
 *   rtf_backward_finish      turns the sums into grad_w (float32[offsets[D_w]]).
 *
 * The calls on one workspace must be ordered (one stream, or events); the
 * workspace holds the sums between them.  Summation order differs between
 * splits, so results agree to float rounding, not bit for bit.
 *
 * Speed: for 1-D samples whose per-bin sums (8 bytes per bin) exceed 3/4 of
 * the L2 cache, an accumulate call that brings at least 4 samples per bin
 * reads its samples twice, adding into one half of the bins per pass so that
 * the sums stay in L2 (2^28 samples into 2^24 bins on GB300: 2.54 ms against
 * 3.17 ms in one pass); smaller calls take one pass.
 */
rtf_status rtf_backward_begin(const rtf_forest *f, void *ws, size_t ws_bytes,
                              void *stream);
rtf_status rtf_backward_accumulate(const rtf_forest *f, const int32_t *dist_id,
                                   const int32_t *idx, const float *pos,
                                   const float *grad_pos, int64_t count,
                                   int32_t mode, void *ws, size_t ws_bytes,
                                   void *stream);
rtf_status rtf_backward_finish(const rtf_forest *f, const float *w, int32_t mode,
                               float *grad_w, void *ws, size_t ws_bytes,
                               void *stream);

#ifdef __cplusplus
} /* extern "C" */
#endif

#endif /* RTF_H_ */
