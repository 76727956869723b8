/*
 * hgmm.h - C ABI of the GB300 (sm_103a) hierarchical-GMM registration path.
 *
 * Method: Eckart, Kim, Kautz, "Fast and Accurate Point Cloud Registration
 * using Trees of Gaussian Mixtures" (arXiv 1807.02587).
 *
 *   - hgmm_build     : the GMM-tree construction the paper relies on
 *                      (Sec. 3 last paragraph, Sec. 4.1 first paragraph): a
 *                      top-down hierarchy of 8-component GMM nodes, each level
 *                      fitted by EM (Eq. 2, Eq. 3) on the points that the
 *                      level above assigned to each parent.
 *   - hgmm_register  : the registration EM loop (Eq. 1, Eq. 4-7): the
 *                      adaptive tree-search E-step of Algorithm 1 with the
 *                      complexity criterion of Sec. 4.1, then the M-step of
 *                      Eq. 9-16 (PCA form of the Mahalanobis distance, weighted
 *                      point-to-plane least squares after Low), solved in FP64.
 *
 * Conventions shared by every entry point
 *   - Return value: 0 (HGMM_OK) or one of the negative HGMM_E* codes below.
 *     hgmm_strerror() gives a one-line message.  A failing call leaves its
 *     outputs unspecified and the tree reusable.
 *   - Points are float32 quadruples (x, y, z, pad): n rows of 16 bytes, the
 *     pointer 16-byte aligned.  "d_" pointers are device memory owned by the
 *     caller; "h_" pointers are host memory owned by the caller.
 *   - Transforms are 4x4 row-major float64 matrices T = [R t; 0 1] that map a
 *     source point z to R z + t in the model (tree) frame: the tree is built
 *     on cloud Z1, the source is Z2 (Eq. 1).
 *   - Streams are passed as void* (a cudaStream_t; NULL = legacy default
 *     stream).  Asynchronous calls only enqueue work; results are valid
 *     after the stream is synchronised.  Calls on one tree must not overlap
 *     (they share the tree's device scratch); different trees are independent.
 *   - The tree lives on the device that was current at hgmm_tree_create and
 *     every call must run with that device current.
 *   - No entry point except hgmm_tree_create / hgmm_tree_destroy allocates or
 *     frees device memory (hgmm_register_pair_host creates the CUDA stream and
 *     graph it replays), so build + register can be captured in a CUDA graph
 *     (the registration is one cooperative launch; two, around an on-device
 *     reorder, for sources of 2^20 points or more).
 *   - Device-side waits are bounded: the registration's arrival and partial-
 *     count waits give up after about a second, record HGMM_ETIMEOUT and
 *     return.
 */
#ifndef HGMM_H
#define HGMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HGMM_OK 0
#define HGMM_EINVAL (-1)      /* bad argument: n < 8, J != 8, depth out of range, misaligned pointer */
#define HGMM_ENOMEM (-2)      /* device allocation failed (hgmm_tree_create only) */
#define HGMM_ECUDA (-3)       /* a CUDA runtime call or kernel launch failed */
#define HGMM_ETIMEOUT (-4)    /* a bounded device-side wait gave up */
#define HGMM_EDEGENERATE (-5) /* the 6x6 normal equations were singular; T kept */
#define HGMM_ENONFINITE (-6)  /* the input cloud holds NaN or Inf coordinates */
#define HGMM_ECAPACITY (-7)   /* n or depth exceeds what the tree was created for */

#define HGMM_J 8          /* components per GMM node (Sec. 4.1) */
#define HGMM_MAX_DEPTH 5  /* deepest supported tree: 8 + 64 + ... + 32768 nodes */

typedef struct hgmm_tree hgmm_tree; /* opaque, device-resident, library-owned */

/* Build parameters.  The paper fixes J = 8 and lambda_c = 0.01 (Sec. 4.1);
 * the others are this library's readings of the build it cites.
 *   em_iters  : EM iterations per tree level (K, default 8).
 *   n_min     : a child whose expected point count falls below n_min dies
 *               (weight 0); a parent whose children all die stays a leaf
 *               and its points ride down with zero posteriors (default 8).
 *   lam_c     : complexity threshold lambda_c of Algorithm 1 (default 0.01).
 *   eps_rel   : covariances get eps*I with eps = (eps_rel * extent)^2, extent
 *               = bounding-box diagonal of the modelled cloud (default 1e-3).
 *   precision : 0 = FP32 moment sums with compensated (Kahan/TwoSum)
 *               accumulation (default); 1 = plain FP32 sums (for comparison).
 *   debug_stop_level, debug_stop_iters : checking aid; 0 = off.  With
 *               debug_stop_level = L + 1 the build finishes levels < L, then
 *               runs only debug_stop_iters EM iterations of level L and stops
 *               (no hand-off), so hgmm_tree_export(L) shows the parameters
 *               after that many iterations (0 = the initial children).
 *   flags     : HGMM_FLAG_* bits (default 0). */
typedef struct hgmm_params {
    int32_t em_iters;
    float n_min;
    float lam_c;
    float eps_rel;
    int32_t precision;
    int32_t debug_stop_level;
    int32_t debug_stop_iters;
    int32_t flags;
} hgmm_params;

/* Run all EM iterations of each multi-launch level of the build in one
 * cooperative launch (arrival counters per parent, the M-step of each parent
 * in a fixed owner CTA) instead of separate E-step and M-step launches per
 * iteration.  The result is the same bit for bit; under a CUDA graph the
 * separate launches are faster on the bench workload, so this is off by
 * default. */
#define HGMM_FLAG_EM_COOPERATIVE 1

/* Per-node record written by hgmm_tree_export: 16 float64 per node,
 * [pi, mu_x, mu_y, mu_z, S_xx, S_xy, S_xz, S_yy, S_yz, S_zz, live, count,
 *  complexity, lambda_1, lambda_2, lambda_3]. */
#define HGMM_NODE_DOUBLES 16

void hgmm_params_default(hgmm_params* p);

/* Allocate a tree able to model up to max_points points with up to max_depth
 * levels, plus all scratch that build and register need (device memory on
 * the current device).  *out receives the handle.  Errors: HGMM_EINVAL,
 * HGMM_ENOMEM, HGMM_ECUDA. */
int hgmm_tree_create(int64_t max_points, int32_t max_depth, hgmm_tree** out);
void hgmm_tree_destroy(hgmm_tree* t);

/* Build the GMM tree of cloud d_points (n x 4 float32, device) with `depth`
 * levels (level l holds 8^(l+1) nodes) and J components per node (must be
 * 8).  p may be NULL for the defaults.  Enqueued on `stream`; non-finite
 * input is reported by hgmm_sync as HGMM_ENONFINITE.
 * Errors: HGMM_EINVAL (n < 8, J != 8, depth not in [1, max_depth],
 * unaligned pointer), HGMM_ECAPACITY, HGMM_ECUDA. */
int hgmm_build(hgmm_tree* t, const float* d_points, int64_t n, int32_t depth,
               int32_t J, const hgmm_params* p, void* stream);

/* Register source cloud d_src (n x 4 float32, device) to the tree: `iters`
 * EM rounds of Algorithm 1 + Eq. 9-16 starting from d_T_init (16 float64,
 * device, row-major; NULL = identity).  lam_c < 0 uses the build's lambda_c;
 * lam_c = 0 disables the early stop (the paper's "GMM-Tree" variant).  The
 * final T is written to d_T_out (16 float64, device).  If d_T_hist is not
 * NULL it receives the T after every round (iters x 16 float64, device).
 * The node moments are exact fixed-point sums of every point's moments, so
 * the result does not depend on the order of the source points, nor on how
 * many CTAs the launch has; a source of 2^20 points or more (up to
 * max_points) is sorted by its first-round nodes into the tree's free point
 * buffer for the remaining rounds, and one of 2^21 points or more runs with
 * three CTAs per SM instead of two (more warps for a throughput-bound
 * descent; the same bits).
 * Errors: HGMM_EINVAL, HGMM_ECUDA; singular normal equations are reported by
 * hgmm_sync as HGMM_EDEGENERATE (T is then left unchanged in that round). */
int hgmm_register(hgmm_tree* t, const float* d_src, int64_t n,
                  const double* d_T_init, int32_t iters, float lam_c,
                  void* stream, double* d_T_out, double* d_T_hist);

/* Eq. 11 objective of the last round of the last hgmm_register, evaluated
 * at the pose that round started from: sum over nodes j with mass of
 * pi*_j sum_l (n_jl^T (mu_j - mu*_j))^2 / lambda_jl (1 float64 to d_obj,
 * device).  0 after a call with iters = 0. */
int hgmm_register_objective(const hgmm_tree* t, double* d_obj, void* stream);

/* Descent variants of the registration E-step (Sec. 4.1: a node's
 * expectation for a point is the sum of its children's expectations, so a
 * child's is its parent's times its posterior among its siblings). */
#define HGMM_DESCENT_ML_LOCAL 0  /* Algorithm 1 as hgmm_register: the maximum-likelihood
                                    path, gamma = the stopping node's sibling posterior */
#define HGMM_DESCENT_ML_GLOBAL 1 /* the maximum-likelihood path, gamma = the product of
                                    the sibling posteriors along the path */
#define HGMM_DESCENT_MULTIPATH 2 /* every live child whose expectation is >= tau is
                                    descended (the others are pruned with their
                                    subtrees); each path stops as Algorithm 1's does and
                                    adds its expectation to the node where it stops */

typedef struct hgmm_descent {
    int32_t mode;     /* HGMM_DESCENT_* */
    float tau;        /* pruning threshold of HGMM_DESCENT_MULTIPATH, in [0, 1] */
    float lam_c;      /* complexity threshold for this call (< 0: the build's) */
    int32_t full_eq7; /* 0: the M-step of Eq. 9-16 (per-node means); 1: the full
                         Eq. 7 (Gauss-Newton over the point contributions, i.e.
                         Eq. 9-16 plus each node's scatter S_j = sum gamma
                         (z' - mu*_j)(z' - mu*_j)^T, which Eq. 8 drops): adds
                         sum_j [d]x P_j [d]x^T-type terms to the rotation block
                         and tr(P_j S_j) / N to the objective */
} hgmm_descent;

/* hgmm_register with the E-step of descent variant d (host struct).  Per
 * round: every (point, stopping node) contribution adds gamma and
 * gamma (z' - mu_j) to the node's 64-bit fixed-point moments; then the same
 * Eq. 9-16 solve (or the full Eq. 7 one, with second moments as well) and
 * T <- dT T.  One launch per round for the descent (a
 * warp-synchronous depth-first search per point with a bounded stack), one
 * for the node terms, one for the solve.  hgmm_register_objective and
 * hgmm_debug_reg_moments report on the last round.  Errors: as hgmm_register;
 * HGMM_EINVAL for an unknown mode or tau outside [0, 1]. */
int hgmm_register_descent(hgmm_tree* t, const float* d_src, int64_t n, const double* d_T_init,
                          int32_t iters, const hgmm_descent* d, void* stream, double* d_T_out,
                          double* d_T_hist);

/* Synchronise `stream` and return the first error the device recorded for
 * this tree since the last hgmm_sync (HGMM_OK if none); clears it. */
int hgmm_sync(hgmm_tree* t, void* stream);

/* End-to-end convenience for callers holding host buffers: copy target and
 * source (n x 4 float32 each, host; pinned memory is fastest) to the tree's
 * device staging buffers, build the target's tree, register the source from
 * h_T_init (NULL = identity) and copy the result to h_T_out (16 float64,
 * host).  The first call of a shape (point counts, depth, parameters, rounds,
 * with or without h_T_init) captures the build and the registration into a
 * CUDA graph on a stream the tree owns; later calls of that shape replay it
 * (one launch instead of about 80); another shape replaces it.  Not while
 * profiling or tracing.  Synchronous.  Errors: as hgmm_build, hgmm_register,
 * hgmm_sync. */
int hgmm_register_pair_host(hgmm_tree* t, const float* h_tgt, int64_t n_tgt,
                            const float* h_src, int64_t n_src, int32_t depth,
                            const hgmm_params* p, const double* h_T_init,
                            int32_t iters, void* stream, double* h_T_out);

/* ---- checking / export (synchronous, host outputs) ---- */

/* Node records of `level` (8^(level+1) nodes x HGMM_NODE_DOUBLES) of the
 * last build; cap = capacity of h_nodes in doubles. */
int hgmm_tree_export(hgmm_tree* t, int32_t level, double* h_nodes, int64_t cap);

/* Node index within `level` of every input point after that level's hand-off
 * (argmax child), in the caller's original point order (n int32). */
int hgmm_debug_labels(hgmm_tree* t, int32_t level, int32_t* h_labels, int64_t cap);

/* Eq. 3 posteriors (Sec. 3) of every input point over the 8 children of its
 * parent at `level`, with the parameters the level ended its EM with: the
 * parent is the point's node of level - 1 (hgmm_debug_labels), or the whole
 * cloud at level 0, and gamma_c = pi_c N(z | c) / sum_k pi_k N(z | k) over
 * those 8 children (dead children 0; all 0 for a parent without a live
 * child).  Computed with the build's FP32 scores.  h_gamma: n x 8 float32
 * (host, caller-owned), row i = input point i, column c = child 8 p + c;
 * cap = its capacity in floats.  Needs a complete build (no debug stop).
 * Errors: HGMM_EINVAL, HGMM_ECAPACITY (cap < 8 n), HGMM_ECUDA. */
int hgmm_debug_posteriors(hgmm_tree* t, int32_t level, float* h_gamma, int64_t cap);

/* Root statistics of the last build: [n, mu(3), Sigma(6 upper), extent, eps]
 * (12 float64). */
int hgmm_debug_root(hgmm_tree* t, double* h_root12);

/* Registration moments of the LAST round of the last hgmm_register: per node
 * of every level (levels concatenated) [M0, M1_x, M1_y, M1_z] float64 with M1
 * = sum gamma z' in the model frame (Algorithm 1, Eq. 9). */
int hgmm_debug_reg_moments(hgmm_tree* t, double* h_m, int64_t cap);

/* Failure-detection check: runs the registration's bounded grid barrier with
 * one of the two arrivals it expects, so the wait must give up after
 * spin_limit polls (~1 us each).  The kernel then records the timeout and
 * returns normally (no fault, no hang): the next hgmm_sync returns
 * HGMM_ETIMEOUT and the tree stays usable.  Enqueued on `stream`. */
int hgmm_debug_barrier_timeout(hgmm_tree* t, int64_t spin_limit, void* stream);

/* ---- per-kernel timing (tracing) ----
 * hgmm_profile(t, 1) clears and starts recording a CUDA event pair around
 * every kernel this tree launches (on the launch stream); hgmm_profile(t, 0)
 * stops.  hgmm_profile_read synchronises the device and returns, for kernel
 * id k in [0, HGMM_PROF_KERNELS), its name, the summed event time in ms and
 * the number of launches recorded.  Recording adds an event pair per launch;
 * it is meant for measurement runs, not for graph capture. */
#define HGMM_PROF_KERNELS 16
int hgmm_profile(hgmm_tree* t, int32_t enable);
int hgmm_profile_read(hgmm_tree* t, int32_t kernel, const char** name, double* total_ms,
                      int64_t* launches);

/* Registration phase trace: with hgmm_trace(t, 1) the next hgmm_register
 * (up to 64 rounds, in one launch: no source reorder while tracing) records,
 * per round and per CTA of its cooperative launch, 6 %globaltimer stamps in
 * ns: round start; descent and moment flush done (the CTA's arrival); all
 * arrivals seen (only the CTAs that own nodes wait for them, 0 elsewhere);
 * node terms published (0 on CTAs without nodes); all partials seen; the
 * CTA's solve and pose update done.  hgmm_trace_read synchronises and copies
 * iters x ctas x 6 int64 (cap = capacity in int64) and reports the
 * dimensions.  Tracing only adds the stamps; results are unchanged. */
int hgmm_trace(hgmm_tree* t, int32_t enable);
int hgmm_trace_read(hgmm_tree* t, int64_t* h_events, int64_t cap, int32_t* iters,
                    int32_t* ctas);

/* Allocation-free fit of one 8-component GMM to a whole cloud: the level-0
 * part of hgmm_build (root statistics, PCA-octant initial children, em_iters
 * EM iterations, FP64 finalize) for callers that cannot allocate device
 * memory at all - code running while someone else captures a CUDA graph on
 * the stream, real-time loops with a memory budget fixed at start-up, or
 * plug-ins whose host owns every allocation.  The paper has no counterpart:
 * this is a deployment variant of the build's first level.
 *   d_points : n x 4 float32, device, 16-byte aligned; 8 <= n <= 1048576
 *              (the capacity of the fixed scratch; larger n -> HGMM_ECAPACITY)
 *   p        : build parameters (NULL = defaults); debug fields ignored
 *   d_out    : 129 float64, device, caller-owned: 8 node records laid out as
 *              in hgmm_tree_export (hard count = -1, no hand-off is run),
 *              then a status word the caller must check once the stream has
 *              run: 0, HGMM_ENONFINITE (NaN/Inf input) or HGMM_ETIMEOUT (a
 *              bounded wait of the E-step gave up), in that order of
 *              precedence, as hgmm_sync reports them; with either error the
 *              nodes are not valid
 * Allocates nothing: its scratch is one static device array (~2.8 MB) that
 * every GPU loading this library holds until exit.  The first call on a
 * device resolves that array's address, so make it before any stream
 * capture; every later call made outside a capture resolves it again (so a
 * call after cudaDeviceReset must also come before any capture).  All calls
 * in the process share the array, so calls that overlap on the GPU (other
 * streams, other threads) race; serialise them.
 * Asynchronous on `stream`.  Errors: HGMM_EINVAL, HGMM_ECAPACITY, HGMM_ECUDA. */
int hgmm_fit_level0_noalloc(const float* d_points, int64_t n, const hgmm_params* p,
                            void* stream, double* d_out);

/* ---- batched form: many independent pairs in one persistent launch ----
 * Every pair (target cloud Z1, source cloud Z2, depth) is built and
 * registered exactly as hgmm_build + hgmm_register do (Sec. 3-4), but all
 * pairs run in one launch: each thread-block cluster takes the next pair
 * from a device queue (largest pairs first) and runs every phase with
 * hardware cluster barriers between them, in its own workspace.  The
 * E-step sums are grouped by how many CTAs share a level, so results match
 * the single-pair path up to FP32 summation order. */
typedef struct hgmm_batch hgmm_batch;

/* Workspaces for clouds of up to max_points points, trees of up to
 * max_depth levels (1..4) and up to max_pairs pairs; one workspace per
 * cluster that can be resident.  Errors: HGMM_EINVAL, HGMM_ENOMEM, HGMM_ECUDA. */
int hgmm_batch_create(int64_t max_points, int32_t max_depth, int32_t max_pairs,
                      hgmm_batch** out);
void hgmm_batch_destroy(hgmm_batch* b);

/* Describe the pairs (host arrays): target of pair i = points
 * [h_tgt_off[i], h_tgt_off[i+1]) of the concatenated cloud buffer, source
 * likewise, tree depth h_depth[i].  Computes the longest-first schedule and
 * uploads it (synchronous).  Errors: HGMM_EINVAL (n_tgt < 8, n_src < 1, bad
 * depth), HGMM_ECAPACITY, HGMM_ECUDA. */
int hgmm_batch_plan(hgmm_batch* b, int32_t n_pairs, const int64_t* h_tgt_off,
                    const int64_t* h_src_off, const int32_t* h_depth);

/* As hgmm_batch_plan with an explicit range per pair: target of pair i =
 * points [h_tgt_rng[2i], h_tgt_rng[2i+1]), source likewise (2 n_pairs int64
 * each).  Ranges may overlap or repeat, so pairs can share a cloud. */
int hgmm_batch_plan_ranges(hgmm_batch* b, int32_t n_pairs, const int64_t* h_tgt_rng,
                           const int64_t* h_src_rng, const int32_t* h_depth);

/* Cluster shape: CTAs (of 256 threads) per pair, 1, 2, 4 or 8 (default 2). */
int hgmm_batch_set_shape(hgmm_batch* b, int32_t cluster_ctas);
int hgmm_batch_get_shape(const hgmm_batch* b, int32_t* cluster_ctas, int32_t* clusters);

/* Build shape of the pairs of one size bucket (by target points: bucket 0
 * below 20,000, bucket 1 below 80,000, bucket 2 the rest): a level runs one
 * warp per E-step work item when it has at least warp_item_parents x
 * (cluster CTAs) parents (else each CTA takes a contiguous chunk of items);
 * a parent's M-step runs on a whole CTA from mstep_cta_runs E-step runs up
 * (else on one warp); its child offsets on a whole CTA from
 * offsets_cta_items items up (else on one warp).  The shapes change only the
 * summation order of the E-step and M-step sums.  Defaults 4, 8, 64.
 * Applies to the current plan and later ones.  Errors: HGMM_EINVAL. */
#define HGMM_BATCH_BUCKETS 3
int hgmm_batch_set_build_shape(hgmm_batch* b, int32_t bucket, int32_t warp_item_parents,
                               int32_t mstep_cta_runs, int32_t offsets_cta_items);
/* The three build-shape values of each bucket (9 int32, bucket-major) and
 * the last autotune's whole-batch times (2 float, ms): default build shape
 * at the chosen cluster shape, tuned build shape (-1 before any autotune). */
int hgmm_batch_get_build_shape(const hgmm_batch* b, int32_t* h_shape9, float* h_ms2);

/* Autotuner over the planned batch (arguments as hgmm_batch_register;
 * synchronous).  (1) Cluster shape: every shape runs the whole batch once
 * untimed and once timed (CUDA events) at the default build shape; the
 * fastest is kept and the four times (ms; -1 if a shape cannot be
 * resident) go to h_ms4.  (2) Build shape per size bucket, one value at a
 * time over a fixed candidate list: each candidate runs on every pair, the
 * launch records each pair's device time, and every bucket keeps the
 * candidate whose pairs took the least total time.  (3) The tuned build
 * shape is kept only if the whole batch is at least as fast as with the
 * default one (both times: hgmm_batch_get_build_shape). */
int hgmm_batch_autotune(hgmm_batch* b, const float* d_points, const hgmm_params* p,
                        const double* d_T_init, int32_t iters, void* stream, double* d_T_out,
                        float* h_ms4);

/* Run the planned batch: d_points = all clouds (float4, device), p = build
 * parameters (NULL = defaults), d_T_init = n_pairs x 16 float64 initial
 * transforms (device; NULL = identity), iters registration rounds.  Writes
 * d_T_out (n_pairs x 16 float64, device), if not NULL d_pair_status
 * (n_pairs int32: 0, HGMM_ENONFINITE, HGMM_ETIMEOUT or HGMM_EDEGENERATE,
 * in that order of precedence), and if not NULL
 * d_T_hist (n_pairs x iters x 16 float64, device: pair i's pose after round
 * k at [16 (i iters + k)]).  One launch on `stream`, graph-capturable.
 * Errors: HGMM_EINVAL, HGMM_ECUDA. */
int hgmm_batch_register(hgmm_batch* b, const float* d_points, const hgmm_params* p,
                        const double* d_T_init, int32_t iters, void* stream, double* d_T_out,
                        int32_t* d_pair_status, double* d_T_hist);

/* Checking: the tree that the last launch built for pair `pair`, level
 * `level` (< the pair's depth), as hgmm_tree_export writes it (cap float64
 * at h_nodes), and its root statistics as hgmm_debug_root writes them.
 * Every cluster's workspace keeps the tree of the last pair it ran, so a
 * pair's tree is available only while no later pair has reused its
 * workspace (a plan of one pair always qualifies).  Synchronous.
 * Errors: HGMM_EINVAL (bad pair or level, or the tree was overwritten),
 * HGMM_ECAPACITY, HGMM_ECUDA. */
int hgmm_batch_debug_tree(const hgmm_batch* b, int32_t pair, int32_t level, double* h_nodes,
                          int64_t cap);
int hgmm_batch_debug_root(const hgmm_batch* b, int32_t pair, double* h_root12);

/* Tracing (no counterpart in the paper): each pair's device run time in the
 * last hgmm_batch_register / hgmm_batch_features launch, nanoseconds of the
 * global timer from the moment its cluster took the pair to the moment it
 * wrote the pair's pose (n_pairs uint64 to h_ns, cap entries at most).
 * Synchronous.  Errors: HGMM_EINVAL, HGMM_ECAPACITY, HGMM_ECUDA. */
int hgmm_batch_pair_ns(const hgmm_batch* b, uint64_t* h_ns, int64_t cap);

/* Per pair of the last hgmm_batch_register: the Eq. 11 objective of its
 * last round (as hgmm_register_objective), n_pairs float64 to d_obj. */
int hgmm_batch_objective(const hgmm_batch* b, double* d_obj, void* stream);

/* Total node count of a tree of `depth` levels (8 + 64 + ... + 8^depth). */
int64_t hgmm_node_count(int32_t depth);

const char* hgmm_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* HGMM_H */
