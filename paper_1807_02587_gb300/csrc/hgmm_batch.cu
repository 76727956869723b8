// Batched form: many independent (target, source) pairs of uneven sizes in
// one persistent launch.  Each thread-block cluster takes the next pair from
// a device queue (pairs ordered largest first), builds the target's GMM tree
// and registers the source, with hardware cluster barriers between phases
// (no spin waits) and its own workspace in HBM; the pair index is broadcast
// to the cluster's CTAs through distributed shared memory.  The phases are
// the shared device functions of hgmm_dev.cuh, so every pair computes what
// hgmm_build + hgmm_register compute (up to the summation order of the
// E-step runs, which depends on how many CTAs share a level).
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/hgmm_proposal.h"
#include "hgmm_dev.cuh"
#include "hgmm_feat.cuh"

namespace cg = cooperative_groups;

namespace hgmm {

// Device pointers of one cluster's workspace.
struct BatchWs {
    NodeEst* est;
    NodeStat* stat;
    float4* rnode;
    int* seg_start;
    int* seg_count;
    RootDev* root;
    float4* pts[2];
    uint32_t* codes;
    Item* items;
    int* item_range;
    int* meta;
    float2* partials;
    int* item_cnt;
    int* item_off;
    float* root_part;
    unsigned long long* acc;
    float2* reg_part;
    double* T;
    float* Rt;
    int* status;
};

struct BatchArgs {
    const float4* points;       // all clouds, concatenated
    const int64_t* tgt_rng;     // [2 n_pairs]: target of pair i = points [rng[2i], rng[2i+1])
    const int64_t* src_rng;     // [2 n_pairs]
    const int* depth;           // [n_pairs]
    const int* order;           // [n_pairs] pair to run k-th
    const double* T_init;       // [n_pairs x 16] or null (identity)
    double* T_out;              // [n_pairs x 16]
    double* T_hist;             // [n_pairs x iters x 16] pose after every round, or null
    int* ws_pair;               // [clusters] pair whose tree each workspace holds
    const int* knobs;           // [n_pairs x 3] build phase shape of each pair (BuildCtx fields)
    unsigned long long* pair_ns;  // [n_pairs] each pair's run time in ns, or null
    int* pair_status;           // [n_pairs] HGMM error code per pair
    double* obj;                // [n_pairs] Eq. 11 objective of the last round, or null
    __nv_bfloat16* feat;        // [n_pairs x 640] target-cloud features, or null
    double* frame;              // [n_pairs x 16] target-cloud frames (with feat)
    const BatchWs* ws;          // [clusters]
    int* queue;                 // next pair to take
    int n_pairs;
    int em_iters;
    float n_min;
    float lam_c;
    float eps_rel;
    int iters;
};

namespace {

static_assert(ACC_REPLICAS == 1, "the batched node terms read one accumulator copy per node");

struct RegSmem {
    double T[12];  // the pair's pose (every CTA of the cluster solves the same system)
    float Rt[12];
    float2 sm[EST_THREADS / 32][NTERM];
    double tot[NTERM];
    double fsm[FRAME_DOUBLES];
};

// dynamic shared memory of k_batch: the staged top levels of the current
// pair's tree (3 float4 per node, padded per block of 8 siblings), then the
// CTA's fixed-point histogram of their registration moments (4 words per node)
constexpr size_t BATCH_DYN_SMEM =
    STAGED_F4 * sizeof(float4) + 4 * STAGED_NODES * sizeof(unsigned long long);

// Sources of at least this many points are reordered by their first-round
// node before the second round (below that the sort costs about what it saves).
constexpr int BATCH_REORDER_MIN = 16384;

// Counting sort of the pair's source points by the node each reached in the
// first round (keys: node id, all ones = none -> key n_nodes), by the
// cluster's CTAs: each CTA counts the keys of its contiguous range into
// shared memory (h, n_nodes + 1 ints), every CTA reads all the cluster's
// counts through distributed shared memory and scans them in key order (key,
// then CTA rank), and each CTA scatters its range to the key's next slot.  The
// order within a key follows shared-memory atomics; the descent's moments are
// exact fixed-point sums, so the pose does not depend on it.
__device__ void sort_source_by_node(const float4* __restrict__ src, int n, int n_nodes,
                                    const uint32_t* __restrict__ keys, float4* __restrict__ dst, int rank,
                                    int cs, cg::cluster_group& cl, int* h) {
    __shared__ int scan_w[EST_THREADS / 32];
    const int nk = n_nodes + 1;
    const int lo = int((int64_t(rank) * n) / cs), hi = int((int64_t(rank + 1) * n) / cs);
    for (int k = threadIdx.x; k < nk; k += blockDim.x) h[k] = 0;
    __syncthreads();
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const uint32_t k = keys[i];
        atomicAdd(&h[k < uint32_t(n_nodes) ? int(k) : n_nodes], 1);
    }
    cl.sync();  // every CTA's counts complete
    // thread t owns keys [t * per, (t + 1) * per): totals over the cluster
    // and the counts of the CTAs before this one
    const int per = (nk + int(blockDim.x) - 1) / int(blockDim.x);
    const int k0 = min(nk, int(threadIdx.x) * per), k1 = min(nk, k0 + per);
    int mine = 0;
    for (int k = k0; k < k1; ++k)
        for (int r = 0; r < cs; ++r) mine += cl.map_shared_rank(h, r)[k];
    // exclusive scan of the threads' totals (warp shuffles, then warp totals)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) scan_w[warp] = incl;
    __syncthreads();
    int base = incl - mine;
    for (int w = 0; w < warp; ++w) base += scan_w[w];
    // first slot of each owned key for this CTA: keys before it (all CTAs),
    // then this key's points in the CTAs before this one
    int pos[32];
    int run = base;
    for (int k = k0, j = 0; k < k1; ++k, ++j) {
        int before = 0, tot = 0;
        for (int r = 0; r < cs; ++r) {
            const int c = cl.map_shared_rank(h, r)[k];
            tot += c;
            if (r < rank) before += c;
        }
        pos[j] = run + before;
        run += tot;
    }
    cl.sync();  // every CTA has read the counts: they may be overwritten
    for (int k = k0, j = 0; k < k1; ++k, ++j) h[k] = pos[j];
    __syncthreads();
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const uint32_t k = keys[i];
        const int slot = atomicAdd(&h[k < uint32_t(n_nodes) ? int(k) : n_nodes], 1);
        if (slot >= 0 && slot < n) dst[slot] = src[i];
    }
    cl.sync();  // the sorted cloud is complete for the whole cluster
}

// One pair, run by all CTAs of this cluster.
template <bool COMP>
__device__ void run_pair(const BatchArgs& a, const BatchWs& w, int cid, int pair, cg::cluster_group& cl,
                         BuildSmem& bs, RegSmem& rgs, float4* sm_est, unsigned long long* hist) {
    const int cs = int(cl.num_blocks());
    const int rank = int(cl.block_rank());
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const float4* tgt = a.points + a.tgt_rng[2 * pair];
    const int n_t = int(a.tgt_rng[2 * pair + 1] - a.tgt_rng[2 * pair]);
    const float4* src = a.points + a.src_rng[2 * pair];
    const int n_s = int(a.src_rng[2 * pair + 1] - a.src_rng[2 * pair]);
    const int depth = a.depth[pair];
    unsigned long long t_start = 0;
    if (rank == 0 && threadIdx.x == 0) {
        a.ws_pair[cid] = pair;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
    }
    double* T_hist = a.T_hist ? a.T_hist + int64_t(16) * a.iters * pair : nullptr;
    // ---- the target's tree (shared with the single-pair build kernel)
    {
        BuildCtx x;
        x.pts = tgt;
        x.n = n_t;
        x.depth = depth;
        x.em_iters = a.em_iters;
        x.n_min = a.n_min;
        x.lam_c = a.lam_c;
        x.eps_rel = a.eps_rel;
        x.stop_level = 0;
        x.stop_iters = 0;
        x.est = w.est;
        x.stat = w.stat;
        x.rnode = w.rnode;
        x.seg_start = w.seg_start;
        x.seg_count = w.seg_count;
        x.root = w.root;
        x.buf[0] = w.pts[0];
        x.buf[1] = w.pts[1];
        for (int l = 0; l < HGMM_MAX_DEPTH; ++l) x.perm[l] = nullptr;
        x.codes = w.codes;
        x.items = w.items;
        x.item_range = w.item_range;
        x.meta = w.meta;
        x.partials = w.partials;
        x.item_cnt = w.item_cnt;
        x.item_off = w.item_off;
        x.root_part = w.root_part;
        x.status = w.status;
        x.warp_item_parents = a.knobs[3 * pair];
        x.mstep_cta_runs = a.knobs[3 * pair + 1];
        x.offsets_cta_items = a.knobs[3 * pair + 2];
        build_levels<COMP>(x, rank, cs, bs, [&]() {
            cl.sync();
            return true;
        });
    }

    // ---- proposal features of the target (levels 0 and 1)
    if (a.feat && rank == 0 && warp == 0 && depth >= 2)
        tree_features_warp(w.root, w.stat, a.feat + int64_t(FEAT_PER_CLOUD) * pair,
                           a.frame + int64_t(FRAME_DOUBLES) * pair, rgs.fsm);

    // ---- registration (Algorithm 1 + Eq. 9-16)
    const int n_nodes = int(level_offset(depth));
    for (int i = rank * blockDim.x + threadIdx.x; i < n_nodes; i += cs * blockDim.x) {
        for (int k = 0; k < 4 * ACC_REPLICAS; ++k) w.acc[4 * ACC_REPLICAS * int64_t(i) + k] = 0ull;
    }
    if (rank == 0 && threadIdx.x < 16) {
        const double v = a.T_init ? a.T_init[16 * pair + threadIdx.x] : ((threadIdx.x % 5 == 0) ? 1.0 : 0.0);
        w.T[threadIdx.x] = v;
        const int r = threadIdx.x >> 2, c = threadIdx.x & 3;
        if (r < 3) w.Rt[c == 3 ? 9 + r : r * 3 + c] = float(v);
    }
    {
        const int ns = n_nodes < STAGED_NODES ? n_nodes : STAGED_NODES;
        stage_nodes(sm_est, w.est, ns);
    }
    cl.sync();
    const double ext = __ldcg(&w.root->extent) > 0.0 ? __ldcg(&w.root->extent) : 1.0;
    const float qscale = float(FIX / ext);
    // large sources: nodes recorded in the first round (the hand-off codes are
    // free after the build), the cloud sorted by them into a ping-pong buffer
    // before the second; the sort borrows the staged nodes' shared memory
    const bool sort_src = a.iters >= 2 && n_s >= BATCH_REORDER_MIN &&
                          n_nodes + 1 <= int(STAGED_F4 * sizeof(float4) / sizeof(int));
    if (threadIdx.x < 12) {
        rgs.T[threadIdx.x] = __ldcg(w.T + threadIdx.x);
        rgs.Rt[threadIdx.x] = __ldcg(w.Rt + threadIdx.x);
    }
    for (int it = 0; it < a.iters; ++it) {
        if (it == 1 && sort_src) {
            sort_source_by_node(src, n_s, n_nodes, w.codes, w.pts[0], rank, cs, cl,
                                reinterpret_cast<int*>(sm_est));
            src = w.pts[0];
            stage_nodes(sm_est, w.est, n_nodes < STAGED_NODES ? n_nodes : STAGED_NODES);
        }
        __syncthreads();
        descend_points<true>(src, n_s, w.est, sm_est, depth, rgs.Rt, qscale, w.acc, rank, cs, hist,
                             it == 0 && sort_src ? w.codes : nullptr);
        __syncthreads();
        flush_node_hist(hist, n_nodes < STAGED_NODES ? n_nodes : STAGED_NODES, w.acc);
        cl.sync();
        float v[32], c[32];  // NTERM terms, padded to a warp's width
#pragma unroll
        for (int k = 0; k < 32; ++k) { v[k] = 0.f; c[k] = 0.f; }
        for (int g = rank * blockDim.x + threadIdx.x; g < n_nodes; g += cs * blockDim.x) {
            // the node's moments and constants in one round trip
            const ulonglong2* ap = reinterpret_cast<const ulonglong2*>(w.acc + 4 * int64_t(g));
            const ulonglong2 q0 = __ldcg(ap), q1 = __ldcg(ap + 1);
            const float4 r0 = __ldcg(w.rnode + 3 * g), r1 = __ldcg(w.rnode + 3 * g + 1);
            const float4 r2 = __ldcg(w.rnode + 3 * g + 2), cm = __ldcg(&w.est[g].a);
            const long long a0 = (long long)q0.x;
            if ((q0.x | q0.y | q1.x | q1.y) == 0ull) continue;
            ulonglong2* wp = reinterpret_cast<ulonglong2*>(w.acc + 4 * int64_t(g));
            wp[0] = make_ulonglong2(0ull, 0ull);
            wp[1] = make_ulonglong2(0ull, 0ull);
            if (a0 <= 0) continue;
            const float M0 = float(a0) * 2.3283064365386963e-10f;  // 2^-32
            const float inv = 1.0f / (qscale * M0);
            float tn[NTERM];
            node_terms(r0, r1, r2, cm, M0, float((long long)q0.y) * inv, float((long long)q1.x) * inv,
                       float((long long)q1.y) * inv, M0 / float(n_s), tn);
#pragma unroll
            for (int k = 0; k < NTERM; ++k) pair_add(v[k], c[k], tn[k], 0.f);
        }
        {
            float ws, we;
            warp_reduce_scatter32(v, c, ws, we);
            if (lane < NTERM) rgs.sm[warp][lane] = make_float2(ws, we);
        }
        __syncthreads();
        if (threadIdx.x < NTERM) {
            float S = 0.f, C = 0.f;
            for (int w2 = 0; w2 < wpb; ++w2) pair_add(S, C, rgs.sm[w2][threadIdx.x].x, rgs.sm[w2][threadIdx.x].y);
            w.reg_part[NTERM * rank + threadIdx.x] = make_float2(S, C);
        }
        cl.sync();
        // every CTA of the cluster reduces the partials in the same order and
        // solves the same system (identical bits), so the new pose needs no
        // hand-over through global memory and no further barrier: the next
        // round's partials are written only after its first barrier, which
        // every CTA reaches after this solve.  Rank 0 keeps the global copies.
        if (threadIdx.x < NTERM) {
            float S = 0.f, C = 0.f;
            for (int b = 0; b < cs; ++b) {
                const float2 x = __ldcg(&w.reg_part[NTERM * b + threadIdx.x]);
                pair_add(S, C, x.x, x.y);
            }
            rgs.tot[threadIdx.x] = double(S) + double(C);
        }
        __syncthreads();
        if (rank == 0 && threadIdx.x == 32 && a.obj && it == a.iters - 1) a.obj[pair] = rgs.tot[NTERM - 1];
        if (warp == 0) {
            const bool solved = warp_solve_update<true>(rgs.tot, rgs.T, rgs.Rt, rank == 0 ? T_hist : nullptr, it,
                                                        rank == 0 ? w.T : nullptr, nullptr);
            if (!solved && rank == 0 && lane == 0) {
                atomicOr(w.status, ST_DEGENERATE);
                if (T_hist)
                    for (int k = 0; k < 16; ++k) T_hist[16 * it + k] = k < 12 ? rgs.T[k] : (k == 15 ? 1.0 : 0.0);
            }
        }
    }
    cl.sync();  // rank 0's final pose is written
    if (rank == 0 && threadIdx.x < 16) {
        a.T_out[16 * pair + threadIdx.x] = __ldcg(w.T + threadIdx.x);
        if (threadIdx.x == 0) {
            const int st = __ldcg(w.status);
            a.pair_status[pair] = (st & ST_NONFINITE)    ? HGMM_ENONFINITE
                                  : (st & ST_TIMEOUT)    ? HGMM_ETIMEOUT
                                  : (st & ST_DEGENERATE) ? HGMM_EDEGENERATE
                                                         : HGMM_OK;
            if (a.pair_ns) {
                unsigned long long t_end;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
                a.pair_ns[pair] = t_end - t_start;
            }
        }
    }
}

template <bool COMP>
__global__ void __launch_bounds__(EST_THREADS, 2) k_batch(BatchArgs a) {
    __shared__ BuildSmem bs;
    __shared__ RegSmem rgs;
    __shared__ int next_pair;
    extern __shared__ float4 batch_dyn[];
    float4* sm_est = batch_dyn;
    unsigned long long* hist = reinterpret_cast<unsigned long long*>(batch_dyn + STAGED_F4);
    for (int i = threadIdx.x; i < 4 * STAGED_NODES; i += blockDim.x) hist[i] = 0ull;
    cg::cluster_group cl = cg::this_cluster();
    const int cs = int(cl.num_blocks());
    const int cid = blockIdx.x / cs;
    const BatchWs w = a.ws[cid];
    for (;;) {
        if (cl.block_rank() == 0 && threadIdx.x == 0) next_pair = atomicAdd(a.queue, 1);
        cl.sync();
        // the pair index from the cluster's first CTA (distributed shared memory)
        const int k = *cl.map_shared_rank(&next_pair, 0);
        cl.sync();
        if (k >= a.n_pairs) break;
        run_pair<COMP>(a, w, cid, a.order[k], cl, bs, rgs, sm_est, hist);
    }
}

}  // namespace

}  // namespace hgmm

using namespace hgmm;

struct hgmm_batch {
    int device = 0;
    int n_sm = 0;
    int64_t max_points = 0;
    int max_depth = 0;
    int max_pairs = 0;
    int max_clusters = 0;      // workspaces allocated
    int cluster_ctas = 2;      // current cluster shape
    int n_pairs = 0;
    std::vector<void*> allocs;
    std::vector<BatchWs> ws;        // host copy of the workspace pointers
    BatchWs* d_ws = nullptr;
    int* d_ws_pair = nullptr;       // per workspace: the pair whose tree it holds (-1: none)
    int64_t* d_tgt_rng = nullptr;
    int64_t* d_src_rng = nullptr;
    int* d_depth = nullptr;
    int* d_order = nullptr;
    int* d_queue = nullptr;
    int* d_pair_status = nullptr;
    double* d_obj = nullptr;        // per pair, last registration's objective
    double* d_T_scratch = nullptr;  // poses of a features-only run
    int min_depth = 0;              // of the current plan
    std::vector<int> h_depth;       // of the current plan, per pair
    std::vector<int> h_bucket;      // of the current plan, per pair (target size bucket)
    // build phase shape per size bucket (warp-item parents factor, M-step CTA
    // runs, child-offset CTA items) and per pair on the device
    int knobs[HGMM_BATCH_BUCKETS][3];
    int* d_knobs = nullptr;
    unsigned long long* d_pair_ns = nullptr;
    float tune_ms[2] = {-1.f, -1.f};  // last autotune: default shape, tuned shape (ms per batch)
};

namespace {

template <typename T>
bool balloc(hgmm_batch* b, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T)) != cudaSuccess) return false;
    b->allocs.push_back(*p);
    return true;
}

// static + dynamic shared memory exceeds the 48 KB default: opt in (once)
bool batch_smem_attr() {
    static const bool ok =
        cudaFuncSetAttribute(k_batch<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(BATCH_DYN_SMEM)) ==
            cudaSuccess &&
        cudaFuncSetAttribute(k_batch<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(BATCH_DYN_SMEM)) ==
            cudaSuccess;
    return ok;
}

int clusters_for(int cs, bool comp) {
    if (!batch_smem_attr()) return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs * 64);
    cfg.blockDim = dim3(EST_THREADS);
    cfg.dynamicSmemBytes = BATCH_DYN_SMEM;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = cs;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    const cudaError_t e = comp ? cudaOccupancyMaxActiveClusters(&n, (void*)k_batch<true>, &cfg)
                               : cudaOccupancyMaxActiveClusters(&n, (void*)k_batch<false>, &cfg);
    return e == cudaSuccess ? n : 0;
}

}  // namespace

extern "C" {

int hgmm_batch_create(int64_t max_points, int32_t max_depth, int32_t max_pairs, hgmm_batch** out) {
    if (!out) return HGMM_EINVAL;
    *out = nullptr;
    if (max_points < 8 || max_points > (int64_t(1) << 28) || max_depth < 1 || max_depth > 4 ||
        max_pairs < 1 || max_pairs > (1 << 20))
        return HGMM_EINVAL;
    hgmm_batch* b = new hgmm_batch();
    if (cudaGetDevice(&b->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) {
        delete b;
        return HGMM_ECUDA;
    }
    b->max_points = max_points;
    b->max_depth = max_depth;
    b->max_pairs = max_pairs;
    // one workspace per cluster that can be resident at the smallest shape
    int mc = 0;
    for (int cs : {1, 2, 4, 8}) mc = std::max(mc, clusters_for(cs, true));
    if (mc < 1) {
        delete b;
        return HGMM_ECUDA;
    }
    b->max_clusters = mc;
    const int64_t nodes = level_offset(max_depth);
    const int64_t parents = max_depth >= 2 ? level_size(max_depth - 2) : 1;
    const int64_t items = (max_points + TILE - 1) / TILE + parents;
    std::vector<BatchWs> ws(mc);
    bool good = true;
    for (int c = 0; c < mc && good; ++c) {
        BatchWs& w = ws[c];
        good &= balloc(b, &w.est, nodes) && balloc(b, &w.stat, nodes) && balloc(b, &w.rnode, 3 * nodes);
        good &= balloc(b, &w.seg_start, nodes) && balloc(b, &w.seg_count, nodes);
        good &= balloc(b, &w.root, 1) && balloc(b, &w.pts[0], max_points) && balloc(b, &w.pts[1], max_points);
        good &= balloc(b, &w.codes, max_points) && balloc(b, &w.item_range, 2 * parents) &&
                balloc(b, &w.items, items);
        good &= balloc(b, &w.meta, 4) && balloc(b, &w.partials, items * NPART);
        good &= balloc(b, &w.item_cnt, items * 8) && balloc(b, &w.item_off, items * 8);
        good &= balloc(b, &w.root_part, 32 * 16) && balloc(b, &w.acc, 4 * ACC_REPLICAS * nodes);
        good &= balloc(b, &w.reg_part, NTERM * 16) && balloc(b, &w.T, 16) && balloc(b, &w.Rt, 12);
        good &= balloc(b, &w.status, 1);
        if (good) good &= cudaMemset(w.seg_count, 0, nodes * sizeof(int)) == cudaSuccess &&
                          cudaMemset(w.stat, 0, nodes * sizeof(NodeStat)) == cudaSuccess;
    }
    good = good && balloc(b, &b->d_ws, mc) && balloc(b, &b->d_tgt_rng, 2 * int64_t(max_pairs)) &&
           balloc(b, &b->d_src_rng, 2 * int64_t(max_pairs)) && balloc(b, &b->d_depth, max_pairs) &&
           balloc(b, &b->d_order, max_pairs) && balloc(b, &b->d_queue, 1) &&
           balloc(b, &b->d_pair_status, max_pairs) && balloc(b, &b->d_obj, max_pairs) &&
           balloc(b, &b->d_T_scratch, 16 * int64_t(max_pairs)) && balloc(b, &b->d_ws_pair, mc) &&
           balloc(b, &b->d_knobs, 3 * int64_t(max_pairs)) && balloc(b, &b->d_pair_ns, max_pairs);
    for (int k = 0; k < HGMM_BATCH_BUCKETS; ++k) {
        b->knobs[k][0] = BUILD_WARP_ITEM_PARENTS;
        b->knobs[k][1] = BUILD_MSTEP_CTA_RUNS;
        b->knobs[k][2] = BUILD_OFFSETS_CTA_ITEMS;
    }
    if (good)
        good = cudaMemcpy(b->d_ws, ws.data(), mc * sizeof(BatchWs), cudaMemcpyHostToDevice) == cudaSuccess &&
               cudaMemset(b->d_ws_pair, 0xff, mc * sizeof(int)) == cudaSuccess;
    b->ws = ws;
    if (!good) {
        hgmm_batch_destroy(b);
        return HGMM_ENOMEM;
    }
    *out = b;
    return HGMM_OK;
}

void hgmm_batch_destroy(hgmm_batch* b) {
    if (!b) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(b->device);
    for (void* p : b->allocs) cudaFree(p);
    cudaSetDevice(cur);
    delete b;
}

}  // extern "C"

namespace {

// Size bucket of a pair by its target cloud: [0, 20k), [20k, 80k), [80k, ...).
int size_bucket(int64_t n_tgt) { return n_tgt < 20000 ? 0 : (n_tgt < 80000 ? 1 : 2); }

// Every planned pair's build shape from its bucket's knobs (synchronous).
int upload_knobs(hgmm_batch* b) {
    if (b->n_pairs < 1) return HGMM_OK;
    std::vector<int> k(3 * size_t(b->n_pairs));
    for (int i = 0; i < b->n_pairs; ++i)
        for (int j = 0; j < 3; ++j) k[3 * i + j] = b->knobs[b->h_bucket[i]][j];
    return cudaMemcpy(b->d_knobs, k.data(), k.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess
               ? HGMM_OK
               : HGMM_ECUDA;
}

}  // namespace

extern "C" {

int hgmm_batch_plan_ranges(hgmm_batch* b, int32_t n_pairs, const int64_t* h_tgt_rng,
                           const int64_t* h_src_rng, const int32_t* h_depth) {
    if (!b || !h_tgt_rng || !h_src_rng || !h_depth || n_pairs < 1 || n_pairs > b->max_pairs)
        return HGMM_EINVAL;
    std::vector<int> order(n_pairs);
    int min_depth = 1 << 30;
    for (int i = 0; i < n_pairs; ++i) {
        min_depth = std::min(min_depth, int(h_depth[i]));
        const int64_t nt = h_tgt_rng[2 * i + 1] - h_tgt_rng[2 * i];
        const int64_t ns = h_src_rng[2 * i + 1] - h_src_rng[2 * i];
        if (nt < 8 || ns < 1 || h_depth[i] < 1 || h_depth[i] > b->max_depth) return HGMM_EINVAL;
        if (nt > b->max_points || ns > b->max_points) return HGMM_ECAPACITY;
        if (h_tgt_rng[2 * i] < 0 || h_src_rng[2 * i] < 0) return HGMM_EINVAL;
        order[i] = i;
    }
    // longest pairs first (LPT): the queue hands the biggest work out early
    auto work = [&](int x) {
        return (h_tgt_rng[2 * x + 1] - h_tgt_rng[2 * x]) + (h_src_rng[2 * x + 1] - h_src_rng[2 * x]);
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
    const size_t rb = size_t(2) * n_pairs * sizeof(int64_t);
    bool good = cudaMemcpy(b->d_tgt_rng, h_tgt_rng, rb, cudaMemcpyHostToDevice) == cudaSuccess;
    good &= cudaMemcpy(b->d_src_rng, h_src_rng, rb, cudaMemcpyHostToDevice) == cudaSuccess;
    good &= cudaMemcpy(b->d_depth, h_depth, n_pairs * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
    good &= cudaMemcpy(b->d_order, order.data(), n_pairs * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!good) return HGMM_ECUDA;
    b->n_pairs = n_pairs;
    b->min_depth = min_depth;
    b->h_depth.assign(h_depth, h_depth + n_pairs);
    b->h_bucket.resize(n_pairs);
    for (int i = 0; i < n_pairs; ++i) b->h_bucket[i] = size_bucket(h_tgt_rng[2 * i + 1] - h_tgt_rng[2 * i]);
    return upload_knobs(b);
}

int hgmm_batch_plan(hgmm_batch* b, int32_t n_pairs, const int64_t* h_tgt_off,
                    const int64_t* h_src_off, const int32_t* h_depth) {
    if (!b || !h_tgt_off || !h_src_off || !h_depth || n_pairs < 1 || n_pairs > b->max_pairs)
        return HGMM_EINVAL;
    std::vector<int64_t> t(2 * size_t(n_pairs)), sr(2 * size_t(n_pairs));
    for (int i = 0; i < n_pairs; ++i) {
        t[2 * i] = h_tgt_off[i];
        t[2 * i + 1] = h_tgt_off[i + 1];
        sr[2 * i] = h_src_off[i];
        sr[2 * i + 1] = h_src_off[i + 1];
    }
    return hgmm_batch_plan_ranges(b, n_pairs, t.data(), sr.data(), h_depth);
}

int hgmm_batch_set_shape(hgmm_batch* b, int32_t cluster_ctas) {
    if (!b || (cluster_ctas != 1 && cluster_ctas != 2 && cluster_ctas != 4 && cluster_ctas != 8))
        return HGMM_EINVAL;
    b->cluster_ctas = cluster_ctas;
    return HGMM_OK;
}

int hgmm_batch_get_shape(const hgmm_batch* b, int32_t* cluster_ctas, int32_t* clusters) {
    if (!b) return HGMM_EINVAL;
    if (cluster_ctas) *cluster_ctas = b->cluster_ctas;
    if (clusters) *clusters = std::min(b->max_clusters, clusters_for(b->cluster_ctas, true));
    return HGMM_OK;
}

}  // extern "C"

namespace {

int launch_batch(hgmm_batch* b, const float* d_points, const hgmm_params* p, const double* d_T_init,
                 int32_t iters, void* stream, double* d_T_out, int32_t* d_pair_status,
                 __nv_bfloat16* d_feat, double* d_frame, double* d_T_hist) {
    if (!b || !d_points || !d_T_out || b->n_pairs < 1 || iters < 0) return HGMM_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_points) & 15u) != 0) return HGMM_EINVAL;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != b->device) return HGMM_EINVAL;
    hgmm_params prm;
    if (p) prm = *p;
    else hgmm_params_default(&prm);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int cs = b->cluster_ctas;
    const bool comp = prm.precision == 0;
    const int nclu = std::min(std::min(b->max_clusters, clusters_for(cs, comp)), b->n_pairs);
    if (nclu < 1) return HGMM_ECUDA;
    BatchArgs a;
    a.points = reinterpret_cast<const float4*>(d_points);
    a.tgt_rng = b->d_tgt_rng;
    a.src_rng = b->d_src_rng;
    a.depth = b->d_depth;
    a.order = b->d_order;
    a.T_init = d_T_init;
    a.T_out = d_T_out;
    a.T_hist = iters > 0 ? d_T_hist : nullptr;
    a.ws_pair = b->d_ws_pair;
    a.knobs = b->d_knobs;
    a.pair_ns = b->d_pair_ns;
    a.pair_status = d_pair_status ? d_pair_status : b->d_pair_status;
    a.obj = b->d_obj;
    a.feat = d_feat;
    a.frame = d_frame;
    a.ws = b->d_ws;
    a.queue = b->d_queue;
    a.n_pairs = b->n_pairs;
    a.em_iters = prm.em_iters;
    a.n_min = prm.n_min;
    a.lam_c = prm.lam_c;
    a.eps_rel = prm.eps_rel;
    a.iters = iters;
    if (cudaMemsetAsync(b->d_queue, 0, sizeof(int), s) != cudaSuccess) return HGMM_ECUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nclu * cs);
    cfg.blockDim = dim3(EST_THREADS);
    cfg.dynamicSmemBytes = BATCH_DYN_SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = cs;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    const cudaError_t e = comp ? cudaLaunchKernelEx(&cfg, k_batch<true>, a)
                               : cudaLaunchKernelEx(&cfg, k_batch<false>, a);
    if (e != cudaSuccess) {
        fprintf(stderr, "hgmm_batch_register: launch failed: %s\n", cudaGetErrorString(e));
        return HGMM_ECUDA;
    }
    return HGMM_OK;
}

}  // namespace

extern "C" {

int hgmm_batch_register(hgmm_batch* b, const float* d_points, const hgmm_params* p,
                        const double* d_T_init, int32_t iters, void* stream, double* d_T_out,
                        int32_t* d_pair_status, double* d_T_hist) {
    return launch_batch(b, d_points, p, d_T_init, iters, stream, d_T_out, d_pair_status, nullptr,
                        nullptr, d_T_hist);
}

namespace {

// The workspace that still holds pair `pair`'s tree after the last launch
// (synchronous), or -1.
int ws_of_pair(const hgmm_batch* b, int pair) {
    std::vector<int> wp(b->max_clusters);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(wp.data(), b->d_ws_pair, wp.size() * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return -2;
    for (int c = 0; c < b->max_clusters; ++c)
        if (wp[c] == pair) return c;
    return -1;
}

}  // namespace

int hgmm_batch_debug_tree(const hgmm_batch* b, int32_t pair, int32_t level, double* h_nodes,
                          int64_t cap) {
    if (!b || !h_nodes || pair < 0 || pair >= b->n_pairs || level < 0 || level >= b->h_depth[pair])
        return HGMM_EINVAL;
    const int64_t m = level_size(level);
    if (cap < m * HGMM_NODE_DOUBLES) return HGMM_ECAPACITY;
    const int c = ws_of_pair(b, pair);
    if (c == -2) return HGMM_ECUDA;
    if (c < 0) return HGMM_EINVAL;
    std::vector<NodeStat> st(m);
    std::vector<int> cnt(m);
    const int64_t off = level_offset(level);
    if (cudaMemcpy(st.data(), b->ws[c].stat + off, m * sizeof(NodeStat), cudaMemcpyDeviceToHost) !=
            cudaSuccess ||
        cudaMemcpy(cnt.data(), b->ws[c].seg_count + off, m * sizeof(int), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
        return HGMM_ECUDA;
    for (int64_t i = 0; i < m; ++i) node_record(st[i], cnt[i], h_nodes + i * HGMM_NODE_DOUBLES);
    return HGMM_OK;
}

int hgmm_batch_debug_root(const hgmm_batch* b, int32_t pair, double* h_root12) {
    if (!b || !h_root12 || pair < 0 || pair >= b->n_pairs) return HGMM_EINVAL;
    const int c = ws_of_pair(b, pair);
    if (c == -2) return HGMM_ECUDA;
    if (c < 0) return HGMM_EINVAL;
    RootDev r;
    if (cudaMemcpy(&r, b->ws[c].root, sizeof(r), cudaMemcpyDeviceToHost) != cudaSuccess) return HGMM_ECUDA;
    root_record(r, h_root12);
    return HGMM_OK;
}

int hgmm_batch_objective(const hgmm_batch* b, double* d_obj, void* stream) {
    if (!b || !d_obj || b->n_pairs < 1) return HGMM_EINVAL;
    return cudaMemcpyAsync(d_obj, b->d_obj, size_t(b->n_pairs) * sizeof(double),
                           cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? HGMM_OK
               : HGMM_ECUDA;
}

int hgmm_batch_features(hgmm_batch* b, const float* d_points, const hgmm_params* p,
                        uint16_t* d_feat, double* d_frame, void* stream) {
    if (!b || !d_feat || !d_frame || b->n_pairs < 1 || b->min_depth < 2) return HGMM_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_feat) & 15u) != 0 || (reinterpret_cast<uintptr_t>(d_frame) & 7u) != 0)
        return HGMM_EINVAL;
    return launch_batch(b, d_points, p, nullptr, 0, stream, b->d_T_scratch, nullptr,
                        reinterpret_cast<__nv_bfloat16*>(d_feat), d_frame, nullptr);
}

int hgmm_batch_autotune(hgmm_batch* b, const float* d_points, const hgmm_params* p,
                        const double* d_T_init, int32_t iters, void* stream, double* d_T_out,
                        float* h_ms4) {
    if (!b || b->n_pairs < 1) return HGMM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HGMM_ECUDA;
    int rc = HGMM_OK;
    // one untimed run, then one timed run of the whole batch (ms; -1 on failure)
    auto timed = [&]() -> float {
        float ms = -1.f;
        rc = hgmm_batch_register(b, d_points, p, d_T_init, iters, stream, d_T_out, nullptr, nullptr);
        if (rc != HGMM_OK) return ms;
        cudaEventRecord(e0, s);
        rc = hgmm_batch_register(b, d_points, p, d_T_init, iters, stream, d_T_out, nullptr, nullptr);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = HGMM_ECUDA;
        else cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    // 1. cluster shape, with every bucket at the default build shape
    int saved[HGMM_BATCH_BUCKETS][3];
    std::memcpy(saved, b->knobs, sizeof(saved));
    for (int k = 0; k < HGMM_BATCH_BUCKETS; ++k) {
        b->knobs[k][0] = BUILD_WARP_ITEM_PARENTS;
        b->knobs[k][1] = BUILD_MSTEP_CTA_RUNS;
        b->knobs[k][2] = BUILD_OFFSETS_CTA_ITEMS;
    }
    if ((rc = upload_knobs(b)) != HGMM_OK) return rc;
    const int shapes[4] = {1, 2, 4, 8};
    float best = 1e30f;
    int best_cs = b->cluster_ctas;
    for (int k = 0; k < 4 && rc == HGMM_OK; ++k) {
        b->cluster_ctas = shapes[k];
        const float ms = clusters_for(shapes[k], true) > 0 ? timed() : -1.f;
        if (h_ms4) h_ms4[k] = ms;
        if (ms > 0.f && ms < best) {
            best = ms;
            best_cs = shapes[k];
        }
    }
    b->cluster_ctas = best_cs;
    b->tune_ms[0] = best;
    // 2. build shape per size bucket, one knob at a time: every candidate runs
    // on all pairs, and each bucket keeps the candidate whose pairs took the
    // least time in total (per-pair device timings of the persistent launch)
    static const int cand[3][5] = {{1, 2, 4, 8, 1 << 20}, {2, 4, 8, 16, 1 << 20}, {16, 32, 64, 256, 1 << 20}};
    std::vector<unsigned long long> ns(b->n_pairs);
    for (int knob = 0; knob < 3 && rc == HGMM_OK; ++knob) {
        double best_t[HGMM_BATCH_BUCKETS];
        int best_v[HGMM_BATCH_BUCKETS];
        for (int k = 0; k < HGMM_BATCH_BUCKETS; ++k) {
            best_t[k] = 1e300;
            best_v[k] = b->knobs[k][knob];
        }
        const int chosen[HGMM_BATCH_BUCKETS] = {b->knobs[0][knob], b->knobs[1][knob], b->knobs[2][knob]};
        for (int c = 0; c < 5 && rc == HGMM_OK; ++c) {
            for (int k = 0; k < HGMM_BATCH_BUCKETS; ++k) b->knobs[k][knob] = cand[knob][c];
            if ((rc = upload_knobs(b)) != HGMM_OK) break;
            if (timed() < 0.f) break;
            if (cudaMemcpy(ns.data(), b->d_pair_ns, ns.size() * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost) != cudaSuccess) {
                rc = HGMM_ECUDA;
                break;
            }
            double tot[HGMM_BATCH_BUCKETS] = {0.0, 0.0, 0.0};
            for (int i = 0; i < b->n_pairs; ++i) tot[b->h_bucket[i]] += double(ns[i]);
            for (int k = 0; k < HGMM_BATCH_BUCKETS; ++k)
                if (tot[k] < best_t[k]) {
                    best_t[k] = tot[k];
                    best_v[k] = cand[knob][c];
                }
        }
        for (int k = 0; k < HGMM_BATCH_BUCKETS; ++k) b->knobs[k][knob] = rc == HGMM_OK ? best_v[k] : chosen[k];
    }
    if (rc == HGMM_OK) rc = upload_knobs(b);
    // 3. the tuned shape against the default one, whole batch; keep the faster
    if (rc == HGMM_OK) {
        const float tuned = timed();
        b->tune_ms[1] = tuned;
        if (rc == HGMM_OK && !(tuned > 0.f && tuned <= best)) {
            for (int k = 0; k < HGMM_BATCH_BUCKETS; ++k) {
                b->knobs[k][0] = BUILD_WARP_ITEM_PARENTS;
                b->knobs[k][1] = BUILD_MSTEP_CTA_RUNS;
                b->knobs[k][2] = BUILD_OFFSETS_CTA_ITEMS;
            }
            rc = upload_knobs(b);
        }
    }
    if (rc != HGMM_OK) {
        std::memcpy(b->knobs, saved, sizeof(saved));
        upload_knobs(b);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int hgmm_batch_set_build_shape(hgmm_batch* b, int32_t bucket, int32_t warp_item_parents,
                               int32_t mstep_cta_runs, int32_t offsets_cta_items) {
    if (!b || bucket < 0 || bucket >= HGMM_BATCH_BUCKETS || warp_item_parents < 1 || mstep_cta_runs < 1 ||
        offsets_cta_items < 1)
        return HGMM_EINVAL;
    b->knobs[bucket][0] = warp_item_parents;
    b->knobs[bucket][1] = mstep_cta_runs;
    b->knobs[bucket][2] = offsets_cta_items;
    return upload_knobs(b);
}

int hgmm_batch_pair_ns(const hgmm_batch* b, uint64_t* h_ns, int64_t cap) {
    if (!b || !h_ns) return HGMM_EINVAL;
    if (cap < b->n_pairs) return HGMM_ECAPACITY;
    if (b->n_pairs == 0) return HGMM_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) return HGMM_ECUDA;
    return cudaMemcpy(h_ns, b->d_pair_ns, size_t(b->n_pairs) * sizeof(unsigned long long),
                      cudaMemcpyDeviceToHost) == cudaSuccess
               ? HGMM_OK
               : HGMM_ECUDA;
}

int hgmm_batch_get_build_shape(const hgmm_batch* b, int32_t* h_shape9, float* h_ms2) {
    if (!b) return HGMM_EINVAL;
    if (h_shape9)
        for (int k = 0; k < HGMM_BATCH_BUCKETS; ++k)
            for (int j = 0; j < 3; ++j) h_shape9[3 * k + j] = b->knobs[k][j];
    if (h_ms2) {
        h_ms2[0] = b->tune_ms[0];
        h_ms2[1] = b->tune_ms[1];
    }
    return HGMM_OK;
}

}  // extern "C"
