// Internal declarations shared by the HGMM CUDA translation units.
//
// Device data layout (all arrays are per tree, indexed by global node id
// g = level_offset(l) + i, level l holding 8^(l+1) nodes; the children of
// node i of level l are nodes 8i .. 8i+7 of level l+1):
//
//   NodeEst  est[g]   48 B, FP32: what the E-step and the descent read.
//                     a = (mu_x, mu_y, mu_z, C), b = (W00, W10, W11, W20),
//                     c = (W21, W22, stop, -) with W = sqrt(log2(e)/2) L^-1
//                     (Sigma = L L^T) and C = log2 pi - 3/2 log2(2 pi)
//                     - sum_i log2 L_ii, so that
//                     log2(pi N(z | mu, Sigma)) = C - |W (z - mu)|^2.
//                     A dead node has C = -inf.
//   NodeStat stat[g]  FP64 parameters (pi, mu, Sigma), eigen-decomposition,
//                     precision matrix P = V diag(1/max(lambda, eps)) V^T and
//                     complexity (Sec. 4.1).
//   seg_start/count   hard segment of each node in the sorted point order.
//
// Points are float4 (x, y, z, pad), re-ordered level by level so that the
// points of every parent are contiguous ("segments"); perm[l] maps sorted
// positions after level l's hand-off back to input indices.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hgmm.h"

namespace hgmm {

constexpr int J = 8;
constexpr int NMOM = 10;              // S0, S1 (3), S2 (6 upper)
constexpr int NPART = J * NMOM;       // 80 moment values per parent run
constexpr int TILE = 256;             // points per build work item
constexpr int EST_THREADS = 256;      // build E-step CTA
constexpr int EST_FOLD = 16;          // E-step points summed in plain FP32 before a compensated fold
constexpr int OFFSET_SLICE_ITEMS = 1024;  // hand-off scan: items per slice of a large parent
constexpr int OFFSET_MAX_SLICES = 64;
constexpr int REG_THREADS = 256;      // registration descent CTA
constexpr int MSTEP_THREADS = 128;    // registration M-step CTA
constexpr int NTERM = 28;             // per-round sums: 21 of H, 6 of g, the objective
constexpr int TRACE_MAX_ITERS = 64;   // rounds the registration trace can hold
constexpr int ACC_REPLICAS = 1;       // copies of each node's registration moments
constexpr int MSTEP_SLICES = 8;        // run slices per parent in the level-wide M-step
constexpr int MSTEP_SLICED_PARENTS = 64;  // levels with at most this many parents are sliced
constexpr int MSTEP_SLICE_MIN_RUNS = 32;  // ... when a parent has about this many runs or more

// Run slices per parent in the level-wide M-step of a level with n_par
// parents over n points, the E-step on `grid` CTAs: a parent's runs are
// about min(items, grid) / n_par; few runs are reduced by one CTA directly.
__host__ __device__ inline int mstep_slices(int n_par, int64_t n, int grid) {
    int64_t items = (n + TILE - 1) / TILE;
    if (items > grid) items = grid;
    const int64_t runs = items / (n_par > 0 ? n_par : 1);
    return n_par <= MSTEP_SLICED_PARENTS && runs >= MSTEP_SLICE_MIN_RUNS ? MSTEP_SLICES : 1;
}

// status bits (device word, OR-ed)
constexpr int ST_NONFINITE = 1;
constexpr int ST_DEGENERATE = 2;
constexpr int ST_CHOL = 4;            // a covariance needed extra regularisation
constexpr int ST_TIMEOUT = 8;

struct NodeEst {
    float4 a, b, c;
};

struct NodeStat {
    double pi;
    double mu[3];
    double S[6];      // xx xy xz yy yz zz
    double lam[3];    // descending
    double V[9];      // eigenvectors in columns, V[r*3+c]
    double P[6];      // precision matrix, same packing as S
    double complexity;
    int live;
    int pad;
};

struct Item {
    int parent;   // parent index within its level (root = 0)
    int start;    // first sorted position
    int count;    // <= TILE
    int pad;
};

struct RootDev {
    double n;
    double mu[3];
    double S[6];
    double extent;
    double eps;
    double lam[3];    // eigen-decomposition of S (descending)
    double V[9];
};

enum KernelId {
    K_ROOT_PARTIAL, K_ROOT_FINAL, K_INIT, K_MAKE_ITEMS, K_FILL_ITEMS, K_ESTEP, K_MSTEP,
    K_ASSIGN, K_OFFSETS, K_SCATTER, K_FINALIZE, K_REG_INIT, K_DESCEND, K_REG_MSTEP, K_COPY_T,
    K_LABELS, K_COUNT
};

struct ProfRecord {
    int id;
    cudaEvent_t a, b;
};

// The exported form of one node (HGMM_NODE_DOUBLES float64, layout in hgmm.h).
inline void node_record(const NodeStat& s, int count, double* o) {
    o[0] = s.live ? s.pi : 0.0;
    for (int a = 0; a < 3; ++a) o[1 + a] = s.mu[a];
    for (int v = 0; v < 6; ++v) o[4 + v] = s.S[v];
    o[10] = s.live ? 1.0 : 0.0;
    o[11] = double(count);
    o[12] = s.complexity;
    for (int a = 0; a < 3; ++a) o[13 + a] = s.lam[a];
}

// The exported form of the root statistics (12 float64, layout in hgmm.h).
inline void root_record(const RootDev& r, double* o) {
    o[0] = r.n;
    for (int a = 0; a < 3; ++a) o[1 + a] = r.mu[a];
    for (int v = 0; v < 6; ++v) o[4 + v] = r.S[v];
    o[10] = r.extent;
    o[11] = r.eps;
}

__host__ __device__ inline int64_t level_size(int l) { return int64_t(1) << (3 * (l + 1)); }
__host__ __device__ inline int64_t level_offset(int l) {
    return ((int64_t(1) << (3 * (l + 1))) - 8) / 7;
}

}  // namespace hgmm

struct hgmm_tree {
    int device = 0;
    int n_sm = 0;
    int64_t cap = 0;
    int max_depth = 0;
    int64_t max_items = 0;
    int64_t max_nodes = 0;
    int est_grid = 0;   // CTAs of the persistent build E-step
    int em_coop_grid = 0;  // co-resident CTAs of the cooperative per-level EM kernel (0: unavailable)
    int reg_grid = 0;       // CTAs of the registration kernel, two per SM
    int reg_grid_wide = 0;  // three per SM, for large sources (0: not co-resident)
    // last build
    int64_t n = 0;
    int depth = 0;
    hgmm_params prm{};
    int64_t reg_n = 0;
    bool built = false;
    // device buffers
    hgmm::NodeEst* est = nullptr;
    hgmm::NodeStat* stat = nullptr;
    int* seg_start = nullptr;
    int* seg_count = nullptr;
    float4* pts[2] = {nullptr, nullptr};
    int* perm[HGMM_MAX_DEPTH] = {};
    uint32_t* codes = nullptr;
    hgmm::Item* items = nullptr;
    int* item_range = nullptr;   // per parent: [begin, end) item indices
    int* meta = nullptr;         // [0] n_items, [1] items per E-step CTA
    float2* partials = nullptr;  // max_items x NPART (sum, compensation)
    int* item_cnt = nullptr;     // max_items x 8
    int* item_off = nullptr;     // max_items x 8
    int* slice_tot = nullptr;    // hand-off of large parents: parents x slices x 8 item-count sums
    int64_t max_slices = 0;      // parents x slices that slice_tot holds
    hgmm::RootDev* root = nullptr;
    float* root_part = nullptr;  // est_grid x 32
    unsigned* root_counter = nullptr;
    unsigned* em_cnt = nullptr;  // cooperative EM: per-parent arrivals + done counter
    float2* mslices = nullptr;   // M-step slice sums (sliced levels: parents x slices x NPART)
    unsigned* mcnt = nullptr;    // M-step slice arrivals per parent (zero between launches)
    int* status = nullptr;
    // registration
    unsigned long long* reg_acc = nullptr;  // nodes x ACC_REPLICAS x 4 fixed point
    unsigned long long* reg_acc2 = nullptr; // nodes x 6 fixed-point second moments (full Eq. 7)
    float2* reg_part = nullptr;             // blocks x 27 (sum, compensation)
    float4* rnode = nullptr;                // nodes x 3: P (6), mu - mu32 (3), FP32
    unsigned* reg_bar = nullptr;            // grid barrier words (8)
    double* reg_T = nullptr;                // 16 doubles current T
    float* reg_Rt = nullptr;                // 12 floats (R row-major, t)
    double* reg_dbg = nullptr;              // nodes x 4 (last round)
    double* reg_obj = nullptr;              // Eq. 11 objective of the last round
    // per-kernel timing and the registration's phase trace
    bool prof_on = false;
    bool trace_on = false;
    int trace_iters = 0;
    int trace_grid = 0;  // CTAs of the traced launch
    unsigned long long* trace = nullptr;  // TRACE_MAX_ITERS x max(reg_grid, reg_grid_wide) x 6
    std::vector<hgmm::ProfRecord> prof;
    // host-API staging
    float4* stage_tgt = nullptr;
    float4* stage_src = nullptr;
    double* stage_T = nullptr;              // 32 doubles: T_init, T_out
    // host API: build + register of the last shape as a CUDA graph (captured
    // on the tree's own stream), replayed by later calls of the same shape
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t pair_exec = nullptr;
    int64_t pair_key[5] = {-1, -1, -1, -1, -1};  // n_tgt, n_src, depth, iters, T_init given
    hgmm_params pair_prm{};
    bool pair_graph_failed = false;
};

// Brackets one kernel launch with a CUDA event pair when profiling is on.
struct ProfScope {
    hgmm_tree* t;
    int id;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(hgmm_tree* t_, int id_, cudaStream_t s_) : t(t_), id(id_), s(s_) {
        if (t->prof_on && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
            cudaEventRecord(a, s);
    }
    ~ProfScope() {
        if (a && b) {
            cudaEventRecord(b, s);
            t->prof.push_back({id, a, b});
        }
    }
};

// Host-side launchers (defined in the .cu files).
int hgmm_build_impl(hgmm_tree* t, const float4* pts, int64_t n, int depth,
                    const hgmm_params& p, cudaStream_t s);
int hgmm_register_impl(hgmm_tree* t, const float4* src, int64_t n,
                       const double* T_init, int iters, float lam_c,
                       cudaStream_t s, double* T_out, double* T_hist);
int hgmm_register_descent_impl(hgmm_tree* t, const float4* src, int64_t n, const double* T_init,
                               int iters, const hgmm_descent& d, cudaStream_t s, double* T_out,
                               double* T_hist);
int hgmm_export_labels_impl(hgmm_tree* t, int level, int* d_out, cudaStream_t s);
int hgmm_debug_posteriors_impl(hgmm_tree* t, int level, float* h_gamma);
int hgmm_register_grid(int n_sm, int per_sm);
int hgmm_em_coop_grid(int n_sm, int est_grid);
bool hgmm_estep_smem_attr();
int hgmm_barrier_timeout_probe_impl(hgmm_tree* t, long long limit, cudaStream_t s);
int hgmm_trace_read_impl(hgmm_tree* t, unsigned long long* h, int64_t cap);
