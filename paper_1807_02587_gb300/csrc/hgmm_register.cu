// Registration EM on the GPU (Sec. 4).
//
// Per round:
//   k_descend   Algorithm 1 for every source point z: z' = R z + t (Eq. 7's
//               T(z)), descend the maximum-likelihood path of the tree from
//               Children(-1) = the 8 level-0 nodes, stop at a node whose
//               complexity is <= lambda_c (Sec. 4.1), at a node without live
//               children or at the leaf level; gamma = the chosen node's
//               posterior among its siblings.  Adds gamma and gamma (z' - mu_j)
//               to the node's moments as 64-bit fixed point (integer adds are
//               exact, so the sums do not depend on the order of the atomics
//               and the result is bit-reproducible).
//   k_mstep     per node with mass: pi* = M0/N, mu* = M1/M0 (Eq. 8-9) and the
//               node's contribution pi* B P B^T, pi* B P (mu_j - mu*) with
//               B = [[mu*]_x; I] to the 6x6 normal equations of Eq. 16 (the
//               three weighted point-to-plane rows of Eq. 13-16 summed in
//               closed form: sum_l (1/lambda_l) n_l n_l^T = P, Eq. 10).
//               Every CTA then reduces the per-CTA sums in the same fixed
//               order, solves the system in FP64 (symmetric elimination) and
//               composes T <- dT T itself: the same inputs and instructions
//               give every CTA the same pose, with no publication step.
#include <algorithm>
#include <cstdio>

#include "hgmm_dev.cuh"

namespace hgmm {

namespace {

__global__ void k_reg_init(const double* __restrict__ T_init, int n_nodes, float lam_c,
                           const NodeStat* __restrict__ stat, NodeEst* __restrict__ est,
                           unsigned long long* __restrict__ acc, double* __restrict__ T,
                           float* __restrict__ Rt, unsigned* __restrict__ bar,
                           double* __restrict__ obj) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_nodes) {
        for (int k = 0; k < 4 * ACC_REPLICAS; ++k) acc[4 * ACC_REPLICAS * int64_t(i) + k] = 0ull;
        if (lam_c >= 0.f)
            est[i].c.z = (stat[i].live && stat[i].complexity <= double(lam_c)) ? 1.f : 0.f;
    }
    if (i == 0) {
        for (int k = 0; k < 16; ++k) T[k] = T_init ? T_init[k] : ((k % 5 == 0) ? 1.0 : 0.0);
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) Rt[r * 3 + c] = float(T[r * 4 + c]);
            Rt[9 + r] = float(T[r * 4 + 3]);
        }
        for (int k = 0; k < 8; ++k)
            if (k != 1) bar[k] = 0u;  // bar[1] is a generation: any start value works
        *obj = 0.0;
    }
}

struct RegArgs {
    const float4* src;
    int n;
    const NodeEst* est;
    const float4* rnode;
    const RootDev* root;
    int depth;
    int n_nodes;
    int iters;
    unsigned long long* acc;
    float2* part;
    unsigned* bar;      // [0] arrivals, [1] generation, [2] partial counter
    double* T;
    float* Rt;
    double* T_hist;
    double* obj;        // Eq. 11 objective of the latest round (pose before its update)
    double* dbg;
    int* status;
    unsigned long long* trace;  // optional: [iter][cta][TRACE_EVENTS] globaltimer ns
    uint32_t* keys;             // k_register<true>: each point's chosen node (one-round launches)
};

constexpr int TRACE_EVENTS = 6;
constexpr size_t REG_DYN_SMEM = STAGED_F4 * sizeof(float4) + 4 * STAGED_NODES * sizeof(unsigned long long);
// three CTAs per SM (dynamic + ~4 KB static + 1 KB reserved each) within 228 KB
static_assert(3 * (REG_DYN_SMEM + 5 * 1024) <= 228 * 1024, "three k_register CTAs must fit on one SM");
// sources from this size on take the three-CTAs-per-SM build (measured: 1M
// points run 10 rounds in 0.65 ms with two CTAs per SM against 0.68 with
// three; 4M in 1.58 against 1.42; 16M in 6.0 against 5.2)
constexpr int REG_WIDE_MIN_POINTS = 1 << 21;

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void trace_mark(unsigned long long* tr, int it, int ev) {
    if (tr && threadIdx.x == 0) tr[(int64_t(it) * gridDim.x + blockIdx.x) * TRACE_EVENTS + ev] = gtimer();
}

// The whole registration loop in one cooperative launch.  Per round:
//   A. Algorithm 1 for every source point (fixed-point node moments)
//   -- every CTA arrives on a counter; only the CTAs that own nodes wait --
//   B. per node with mass: its normal-equation and objective terms (FP32),
//      compensated block sums -> one partial per node-owning CTA, then an
//      arrival on a second counter
//   -- every CTA waits for all partials --
//   C. every CTA reduces the partials in the same fixed order and solves the
//      6x6 system in FP64 itself: identical inputs and instructions give every
//      CTA the same bits, so the new pose needs no publication round trip.
//      CTA 0 keeps the global copies (T, R|t, per-round history, objective).
// Trace events per round and CTA: 0 round start, 1 arrival, 2 all arrivals
// seen (node CTAs), 3 partial published (node CTAs), 4 all partials seen,
// 5 pose solved.  All counters are monotonic over the launch (zeroed by
// k_reg_init), so no CTA resets a word that another may still be reading;
// every wait is bounded.
// KEYS: the launch records each point's chosen node in a.keys (a one-round
// launch before the source reorder).
// MINB: co-resident CTAs per SM the build is register-limited for.  Two (128
// registers) for sources of a few points per thread, where each round is a
// latency chain and the node terms and the solve want the registers; three
// (80) for large sources, whose descent is throughput-bound and gains from
// the extra warps (a few bytes of spills, outside the descent).
template <bool KEYS, int MINB>
__global__ void __launch_bounds__(REG_THREADS, MINB) k_register(RegArgs a) {
    __shared__ float Rt_sm[12];
    __shared__ double T_sm[12];
    __shared__ float2 sm[REG_THREADS / 32][NTERM];
    __shared__ float2 fin[8][NTERM];
    __shared__ double tot[NTERM];
    // dynamic: the staged top levels (3 float4 per node, padded), then the CTA's
    // fixed-point histogram of their moments (4 words per node)
    extern __shared__ float4 reg_dyn[];
    float4* sm_est = reg_dyn;
    unsigned long long* hist = reinterpret_cast<unsigned long long*>(reg_dyn + STAGED_F4);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ns = a.n_nodes < STAGED_NODES ? a.n_nodes : STAGED_NODES;
    const int nb_nodes = (a.n_nodes + blockDim.x - 1) / blockDim.x;
    const bool lead = blockIdx.x == 0;
    // the top levels of the tree are read by every point: stage them once
    // for all rounds (the stop flags were set by k_reg_init before launch);
    // the starting pose (k_reg_init) into shared memory
    {
        stage_nodes(sm_est, a.est, ns);
        for (int i = threadIdx.x; i < 4 * STAGED_NODES; i += blockDim.x) hist[i] = 0ull;
        if (threadIdx.x < 12) {
            T_sm[threadIdx.x] = __ldcg(a.T + threadIdx.x);
            Rt_sm[threadIdx.x] = __ldcg(a.Rt + threadIdx.x);
        }
        __syncthreads();
    }
    const double ext = a.root->extent > 0.0 ? a.root->extent : 1.0;
    const float qscale = float(FIX / ext);  // fixed-point units per metre
    for (int it = 0; it < a.iters; ++it) {
        trace_mark(a.trace, it, 0);
        descend_points<KEYS>(a.src, a.n, a.est, sm_est, a.depth, Rt_sm, qscale, a.acc, blockIdx.x, gridDim.x,
                             hist, a.keys);
        __syncthreads();
        flush_node_hist(hist, ns, a.acc);
        __syncthreads();
        if (threadIdx.x == 0) arrive_release(a.bar + 4);  // this CTA's moment atomics before it
        trace_mark(a.trace, it, 1);
        // ---- B: node terms (only the CTAs that own nodes take part)
        if (blockIdx.x < nb_nodes) {
            if (!wait_acquire(a.bar + 4, unsigned(it + 1) * gridDim.x, a.status, BARRIER_SPIN_LIMIT)) return;
            trace_mark(a.trace, it, 2);
            // at most one node per thread (nb_nodes x blockDim.x >= n_nodes):
            // its terms start the compensated pairs (errors zero)
            float v[32], c[32];  // NTERM terms, padded to a warp's width
#pragma unroll
            for (int k = 0; k < 32; ++k) { v[k] = 0.f; c[k] = 0.f; }
            double* dbg = it == a.iters - 1 ? a.dbg : nullptr;
            const int g = blockIdx.x * blockDim.x + threadIdx.x;
            if (g < a.n_nodes) {
                // the node's constants are loaded with its moments (one L2
                // round trip instead of two)
                const float4 cm = __ldg(&a.est[g].a);
                const float4 r0 = __ldg(a.rnode + 3 * g), r1 = __ldg(a.rnode + 3 * g + 1);
                const float4 r2 = __ldg(a.rnode + 3 * g + 2);
                long long a0 = 0, a1 = 0, a2 = 0, a3 = 0;
                {
                    // integer sums of the replicas: exact, order-free
                    const ulonglong2* rp = reinterpret_cast<const ulonglong2*>(
                        a.acc + 4 * int64_t(g) * ACC_REPLICAS);
                    ulonglong2 q[2 * ACC_REPLICAS];
#pragma unroll
                    for (int r = 0; r < 2 * ACC_REPLICAS; ++r) q[r] = __ldcg(rp + r);
                    unsigned long long any = 0ull;
#pragma unroll
                    for (int r = 0; r < ACC_REPLICAS; ++r) {
                        a0 += (long long)q[2 * r].x;
                        a1 += (long long)q[2 * r].y;
                        a2 += (long long)q[2 * r + 1].x;
                        a3 += (long long)q[2 * r + 1].y;
                        any |= q[2 * r].x | q[2 * r].y | q[2 * r + 1].x | q[2 * r + 1].y;
                    }
                    if (any) {
                        ulonglong2* wp = reinterpret_cast<ulonglong2*>(a.acc + 4 * int64_t(g) * ACC_REPLICAS);
#pragma unroll
                        for (int r = 0; r < 2 * ACC_REPLICAS; ++r) wp[r] = make_ulonglong2(0ull, 0ull);
                    }
                }
                float M0 = 0.f, o0 = 0.f, o1 = 0.f, o2 = 0.f;
                if (a0 > 0) {
                    M0 = float(a0) * 2.3283064365386963e-10f;  // 2^-32
                    const float inv = 1.0f / (qscale * M0);
                    o0 = float(a1) * inv;
                    o1 = float(a2) * inv;
                    o2 = float(a3) * inv;
                    node_terms(r0, r1, r2, cm, M0, o0, o1, o2, M0 / float(a.n), v);
                }
                if (dbg) {
                    dbg[4 * g + 0] = double(a0) * INV_FIX;
                    dbg[4 * g + 1] = double(M0) * (double(cm.x) + double(o0));
                    dbg[4 * g + 2] = double(M0) * (double(cm.y) + double(o1));
                    dbg[4 * g + 3] = double(M0) * (double(cm.z) + double(o2));
                }
            }
            {
                float ws, we;
                warp_reduce_scatter32(v, c, ws, we);
                if (lane < NTERM) sm[warp][lane] = make_float2(ws, we);
            }
            __syncthreads();
            if (threadIdx.x < NTERM) {
                float S = 0.f, C = 0.f;
                for (int w = 0; w < REG_THREADS / 32; ++w) pair_add(S, C, sm[w][threadIdx.x].x, sm[w][threadIdx.x].y);
                a.part[NTERM * blockIdx.x + threadIdx.x] = make_float2(S, C);
            }
            __syncthreads();
            if (threadIdx.x == 0) arrive_release(a.bar + 2);  // partial and cleared moments before it
            trace_mark(a.trace, it, 3);
        }
        // ---- C: every CTA: fixed-order reduction, FP64 solve, pose update
        if (!wait_acquire(a.bar + 2, unsigned(it + 1) * nb_nodes, a.status, BARRIER_SPIN_LIMIT)) return;
        trace_mark(a.trace, it, 4);
        // all partial loads in flight at once (8 groups of NTERM threads),
        // then a fixed-order combine
        if (threadIdx.x < 8 * NTERM) {
            const int k = threadIdx.x % NTERM, q = threadIdx.x / NTERM;
            float S = 0.f, C = 0.f;
            float2 xs[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int b = q + 8 * j;
                xs[j] = b < nb_nodes ? __ldcg(&a.part[NTERM * b + k]) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) pair_add(S, C, xs[j].x, xs[j].y);
            for (int b = q + 64; b < nb_nodes; b += 8) {
                const float2 x = __ldcg(&a.part[NTERM * b + k]);
                pair_add(S, C, x.x, x.y);
            }
            fin[q][k] = make_float2(S, C);
        }
        __syncthreads();
        if (warp == 0) {
            // the eight group sums in order, by the warp that solves
            if (lane < NTERM) {
                float S = 0.f, C = 0.f;
                for (int q = 0; q < 8; ++q) pair_add(S, C, fin[q][lane].x, fin[q][lane].y);
                tot[lane] = double(S) + double(C);
            }
            __syncwarp();
            if (lead && lane == 0 && a.obj) *a.obj = tot[NTERM - 1];
            const bool solved = warp_solve_update<true>(tot, T_sm, Rt_sm, lead ? a.T_hist : nullptr, it,
                                                        lead ? a.T : nullptr, lead ? a.Rt : nullptr);
            if (!solved && lead && lane == 0) {
                atomicOr(a.status, ST_DEGENERATE);  // T kept for this round
                if (a.T_hist)
                    for (int k = 0; k < 16; ++k) a.T_hist[16 * it + k] = k < 12 ? T_sm[k] : (k == 15 ? 1.0 : 0.0);
            }
        }
        __syncthreads();
        trace_mark(a.trace, it, 5);
    }
}

// A wait that nothing ends: the bounded barrier's timeout path, for tests of
// failure detection.  One CTA arrives at a barrier that expects two.
__global__ void k_barrier_timeout_probe(unsigned* bar, int* status, long long limit) {
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = bar + 1;
        const unsigned gen = *vgen;
        atomicAdd(bar, 1u);  // expects 2 arrivals; the second never comes
        long long spins = 0;
        while (*vgen == gen) {
            if (++spins > limit) {
                atomicOr(status, ST_TIMEOUT);
                break;
            }
            __nanosleep(64);
        }
        bar[0] = 0u;
    }
}

// ------------------------------------------------ source reorder (large clouds)
// A large source cloud in arbitrary order sends each warp's 32 points down
// ~20 different paths of the tree, so the descent adds its moments with one
// atomic group per node and warp and its child loads diverge.  Such a cloud
// runs its first round in the caller's order, with every point's chosen node
// recorded; it is then counting-sorted by that node (into a library buffer)
// and runs the remaining rounds in that order, where the 32 points of a warp
// mostly follow one path.  The node moments are exact integer sums of the
// points' fixed-point moments, so the order of the points does not change
// the result at all.
constexpr int REORDER_MIN_POINTS = 1 << 20;
constexpr int REORDER_KEYS = 8192;  // node ids of trees up to depth 4 (4,680 nodes); the last: no node
constexpr int REORDER_THREADS = 256;

// Contiguous range of points of CTA b (of nb).
__device__ __forceinline__ void cta_range(int n, int b, int nb, int& lo, int& hi) {
    lo = int((int64_t(b) * n) / nb);
    hi = int((int64_t(b + 1) * n) / nb);
}

// Pass 1: each CTA's key counts (cnt[b][key]) over its contiguous range.
__global__ void __launch_bounds__(REORDER_THREADS) k_src_count(const uint32_t* __restrict__ keys, int n,
                                                               int* __restrict__ cnt) {
    __shared__ int h[REORDER_KEYS];
    for (int k = threadIdx.x; k < REORDER_KEYS; k += blockDim.x) h[k] = 0;
    __syncthreads();
    int lo, hi;
    cta_range(n, blockIdx.x, gridDim.x, lo, hi);
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) atomicAdd(&h[keys[i] & (REORDER_KEYS - 1)], 1);
    __syncthreads();
    for (int k = threadIdx.x; k < REORDER_KEYS; k += blockDim.x) cnt[int64_t(blockIdx.x) * REORDER_KEYS + k] = h[k];
}

// Pass 2a (one thread per key): cnt[b][key] becomes the exclusive prefix
// over the CTAs b of that key's counts, and tot[key] the key's total.
__global__ void k_src_colscan(int* __restrict__ cnt, int nb, int* __restrict__ tot) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= REORDER_KEYS) return;
    int s = 0;
    for (int b = 0; b < nb; ++b) {
        const int c = cnt[int64_t(b) * REORDER_KEYS + k];
        cnt[int64_t(b) * REORDER_KEYS + k] = s;
        s += c;
    }
    tot[k] = s;
}

// Pass 2b (one CTA of 1024 threads): tot[key] becomes the exclusive prefix
// over the keys (keys in order, CTAs in order within a key).
__global__ void __launch_bounds__(1024) k_src_keyscan(int* __restrict__ tot) {
    constexpr int PER = REORDER_KEYS / 1024;
    __shared__ int part[1024];
    int v[PER], s = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        v[j] = tot[threadIdx.x * PER + j];
        s += v[j];
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int u = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += u;
        __syncthreads();
    }
    int base = part[threadIdx.x] - s;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        tot[threadIdx.x * PER + j] = base;
        base += v[j];
    }
}

// Pass 3: every point to its key's next slot of its CTA (shared-memory
// counters: the order within a CTA's key is not fixed, which the exact
// fixed-point moments of the descent do not see).
__global__ void __launch_bounds__(REORDER_THREADS) k_src_scatter(const float4* __restrict__ src, int n,
                                                                 const uint32_t* __restrict__ keys,
                                                                 const int* __restrict__ cnt,
                                                                 const int* __restrict__ base,
                                                                 float4* __restrict__ dst) {
    __shared__ int pos[REORDER_KEYS];
    for (int k = threadIdx.x; k < REORDER_KEYS; k += blockDim.x)
        pos[k] = base[k] + cnt[int64_t(blockIdx.x) * REORDER_KEYS + k];
    __syncthreads();
    int lo, hi;
    cta_range(n, blockIdx.x, gridDim.x, lo, hi);
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const uint32_t key = keys[i] & (REORDER_KEYS - 1);
        const int slot = atomicAdd(&pos[key], 1);
        if (slot >= 0 && slot < n) dst[slot] = src[i];
    }
}

__global__ void k_copy_T(const double* __restrict__ T, double* __restrict__ out) {
    if (threadIdx.x < 16) out[threadIdx.x] = T[threadIdx.x];
}

// ---------------------------------------------------- descent variants
// One round's E-step under a variant of the descent (Sec. 4.1).  Every warp
// takes 32 points; each lane runs a depth-first search over the tree with a
// stack of (node, level | terminal bit, gamma).  One step pops one entry: a
// terminal entry (a node where its path stops: complexity <= lambda_c or the
// last level) is emitted; any other entry is expanded (the 8 children scored
// as in Algorithm 1) and pushes the child the variant keeps (the
// maximum-likelihood one, or every live child whose expectation reaches
// tau), or, if it has no live child, is emitted itself.  Emissions of the
// warp's step are summed per node (warp_group_sum) and added to the node's
// fixed-point moments.  The stack bound 8 x depth holds for any tau: a step
// removes one entry and adds at most 8, and a level never holds more than 7
// pending siblings.
constexpr int VAR_THREADS = 256;
constexpr int VAR_STACK = 8 * HGMM_MAX_DEPTH;
constexpr int VAR_TERMINAL = 1 << 8;

// Fixed-point units of the second moments gamma (z' - mu_j)_a (z' - mu_j)_b
// per squared extent.
constexpr double FIX2 = 4294967296.0;

template <int MODE, bool M2>
__global__ void __launch_bounds__(VAR_THREADS)
k_descend_var(const float4* __restrict__ src, int n, const NodeEst* __restrict__ est, int depth, float tau,
              const float* __restrict__ Rt, const RootDev* __restrict__ root,
              unsigned long long* __restrict__ acc, unsigned long long* __restrict__ acc2,
              int* __restrict__ status) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the fixed-point scales from the FP64 extent, once per CTA (FP64
    // division is slow on this part)
    __shared__ float s_scale[2];
    if (threadIdx.x == 0) {
        const double ext = root->extent > 0.0 ? root->extent : 1.0;
        s_scale[0] = float(FIX / ext);
        s_scale[1] = float(FIX2 / (ext * ext));
    }
    __syncthreads();
    const float qscale = s_scale[0], q2 = s_scale[1];
    const float r00 = Rt[0], r01 = Rt[1], r02 = Rt[2], r10 = Rt[3], r11 = Rt[4], r12 = Rt[5];
    const float r20 = Rt[6], r21 = Rt[7], r22 = Rt[8], tx = Rt[9], ty = Rt[10], tz = Rt[11];
    const int warps_total = gridDim.x * (VAR_THREADS / 32);
    for (int base = (blockIdx.x * (VAR_THREADS / 32) + warp) * 32; base < n; base += warps_total * 32) {
        const int i = base + lane;
        float4 p = i < n ? src[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        bool valid = i < n;
        if (valid && !(isfinite(p.x) && isfinite(p.y) && isfinite(p.z))) {
            atomicOr(status, ST_NONFINITE);
            valid = false;
        }
        const float x = fmaf(r00, p.x, fmaf(r01, p.y, fmaf(r02, p.z, tx)));
        const float y = fmaf(r10, p.x, fmaf(r11, p.y, fmaf(r12, p.z, ty)));
        const float w = fmaf(r20, p.x, fmaf(r21, p.y, fmaf(r22, p.z, tz)));
        int sn[VAR_STACK], sm[VAR_STACK];
        float sg[VAR_STACK];
        int sp = 0;
        if (valid) {  // the root: its children are the level-0 nodes
            sn[0] = -1;
            sm[0] = -1 & 0xff;
            sg[0] = 1.f;
            sp = 1;
        }
        while (__any_sync(FULL, sp > 0)) {
            int out_node = -1;
            float out_g = 0.f;
            if (sp > 0) {
                --sp;
                const int g = sn[sp], meta = sm[sp];
                const float gam = sg[sp];
                const int l = (meta & 0xff) == 0xff ? -1 : (meta & 0xff);
                if (meta & VAR_TERMINAL) {
                    out_node = g;
                    out_g = gam;
                } else {
                    const int cl = l + 1;
                    const int64_t first = d_level_offset(cl) + 8 * (l < 0 ? 0 : int64_t(g) - d_level_offset(l));
                    float sc8[8], st8[8];
                    float best = -CUDART_INF_F;
                    int bi = -1;
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const NodeEst* e = est + first + c;
                        const float4 ea = __ldg(&e->a), eb = __ldg(&e->b), ec = __ldg(&e->c);
                        const float ex = x - ea.x, ey = y - ea.y, ez = w - ea.z;
                        const float d0 = eb.x * ex;
                        const float d1 = fmaf(eb.z, ey, eb.y * ex);
                        const float d2 = fmaf(ec.y, ez, fmaf(ec.x, ey, eb.w * ex));
                        float sc = fmaf(-d0, d0, ea.w);
                        sc = fmaf(-d1, d1, sc);
                        sc = fmaf(-d2, d2, sc);
                        sc8[c] = sc;
                        st8[c] = ec.z;
                        if (sc > best) {
                            best = sc;
                            bi = c;
                        }
                    }
                    if (bi < 0) {  // no live child: the path ends here
                        if (l >= 0) {
                            out_node = g;
                            out_g = gam;
                        }
                    } else {
                        float sum = 0.f;
#pragma unroll
                        for (int c = 0; c < 8; ++c) sum += exp2f(sc8[c] - best);
                        const float inv = 1.0f / sum;
                        const bool last = cl == depth - 1;
                        if (MODE == HGMM_DESCENT_MULTIPATH) {
                            for (int c = 7; c >= 0; --c) {
                                const float cg = gam * (exp2f(sc8[c] - best) * inv);
                                if (sc8[c] > -CUDART_INF_F && cg >= tau && sp < VAR_STACK) {
                                    sn[sp] = int(first + c);
                                    sm[sp] = cl | ((last || st8[c] != 0.f) ? VAR_TERMINAL : 0);
                                    sg[sp] = cg;
                                    ++sp;
                                }
                            }
                        } else {
                            const float pc = inv;  // the best child's posterior: 2^0 / sum
                            sn[sp] = int(first + bi);
                            sm[sp] = cl | ((last || st8[bi] != 0.f) ? VAR_TERMINAL : 0);
                            sg[sp] = MODE == HGMM_DESCENT_ML_GLOBAL ? gam * pc : pc;
                            ++sp;
                        }
                    }
                }
            }
            constexpr int NV = M2 ? 10 : 4;
            float v[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) v[q] = 0.f;
            if (out_node >= 0) {
                const float4 a = __ldg(&est[out_node].a);
                const float dx = x - a.x, dy = y - a.y, dz = w - a.z;
                v[0] = out_g;
                v[1] = out_g * dx;
                v[2] = out_g * dy;
                v[3] = out_g * dz;
                if (M2) {
                    v[4] = v[1] * dx;
                    v[5] = v[1] * dy;
                    v[6] = v[1] * dz;
                    v[7] = v[2] * dy;
                    v[8] = v[2] * dz;
                    v[9] = v[3] * dz;
                }
            }
            const int rank = warp_group_sum<NV>(out_node, v);
            if (out_node >= 0 && rank == 0) {
                unsigned long long* dst = acc + 4 * int64_t(out_node) * ACC_REPLICAS;
                atomicAdd(dst + 0, (unsigned long long)to_fix(v[0] * 4294967296.0f));
                atomicAdd(dst + 1, (unsigned long long)to_fix(v[1] * qscale));
                atomicAdd(dst + 2, (unsigned long long)to_fix(v[2] * qscale));
                atomicAdd(dst + 3, (unsigned long long)to_fix(v[3] * qscale));
                if (M2) {
                    unsigned long long* d2 = acc2 + 6 * int64_t(out_node);
#pragma unroll
                    for (int q = 0; q < 6; ++q) atomicAdd(d2 + q, (unsigned long long)to_fix(v[4 + q] * q2));
                }
            }
        }
    }
}

// Levi-Civita symbol on indices 0..2.
__host__ __device__ constexpr int lc3(int i, int j, int k) { return (i - j) * (j - k) * (k - i) / 2; }

// The full Eq. 7 additions of one node from its scatter S = sum gamma d d^T
// (d = z' - mu*): the rotation block gains sum gamma [d]x P [d]x^T, i.e.
// entry (a, b) = sum eps(a,j,k) eps(b,n,m) P_km S_jn, the rotation part of
// the right-hand side gains -sum gamma d x (P d), i.e. entry a =
// -sum eps(a,j,k) P_km S_jm, and the objective tr(P S); all times 1 / N.
__device__ __forceinline__ void scatter_terms(const float (&P)[3][3], const float (&S)[3][3], float inv_n,
                                              float* w) {
    const int rr[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    const int slot[6] = {0, 1, 2, 6, 7, 11};  // upper-packed 6x6 positions of the rotation block
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        const int a = rr[e][0], b = rr[e][1];
        float h = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (lc3(a, j, k) == 0) continue;
#pragma unroll
                for (int nn = 0; nn < 3; ++nn)
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        if (lc3(b, nn, m) == 0) continue;
                        h = fmaf(float(lc3(a, j, k) * lc3(b, nn, m)) * P[k][m], S[j][nn], h);
                    }
            }
        w[slot[e]] += inv_n * h;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float gsum = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (lc3(a, j, k) == 0) continue;
#pragma unroll
                for (int m = 0; m < 3; ++m) gsum = fmaf(float(lc3(a, j, k)) * P[k][m], S[j][m], gsum);
            }
        w[21 + a] -= inv_n * gsum;
    }
    float tr = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int m = 0; m < 3; ++m) tr = fmaf(P[k][m], S[k][m], tr);
    w[27] += inv_n * tr;
}

// Node terms of one round from the fixed-point moments (256 nodes per CTA,
// a warp reduce-scatter per 32 nodes, the CTA's eight warp sums in order);
// the accumulators are cleared for the next round.  FULL adds the scatter
// terms of the full Eq. 7 from the second moments.
template <bool FULL>
__global__ void __launch_bounds__(VAR_THREADS)
k_var_terms(int n_nodes, int n, const NodeEst* __restrict__ est, const float4* __restrict__ rnode,
            const RootDev* __restrict__ root, unsigned long long* __restrict__ acc,
            unsigned long long* __restrict__ acc2, float2* __restrict__ part, double* __restrict__ dbg) {
    __shared__ float2 sm[VAR_THREADS / 32][NTERM];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = blockIdx.x * VAR_THREADS + threadIdx.x;
    __shared__ float s_scale[2];
    if (threadIdx.x == 0) {
        const double ext = root->extent > 0.0 ? root->extent : 1.0;
        s_scale[0] = float(FIX / ext);
        s_scale[1] = float(FIX2 / (ext * ext));
    }
    __syncthreads();
    const float qscale = s_scale[0];
    float v[32], c[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) { v[k] = 0.f; c[k] = 0.f; }
    if (g < n_nodes) {
        unsigned long long* ap = acc + 4 * int64_t(g) * ACC_REPLICAS;
        const long long a0 = (long long)ap[0], a1 = (long long)ap[1], a2 = (long long)ap[2],
                        a3 = (long long)ap[3];
        if (a0 | a1 | a2 | a3) ap[0] = ap[1] = ap[2] = ap[3] = 0ull;
        const float4 cm = est[g].a;
        float M0 = 0.f, o0 = 0.f, o1 = 0.f, o2 = 0.f;
        if (a0 > 0) {
            float wv[NTERM];
            M0 = float(a0) * 2.3283064365386963e-10f;  // 2^-32
            const float inv = 1.0f / (qscale * M0);
            o0 = float(a1) * inv;
            o1 = float(a2) * inv;
            o2 = float(a3) * inv;
            node_terms(rnode[3 * g], rnode[3 * g + 1], rnode[3 * g + 2], cm, M0, o0, o1, o2, M0 / float(n), wv);
            if (FULL) {
                // scatter about mu*: S = M2 - M1 M1^T / M0 (moments centred on
                // the FP32 mean), formed in FP64
                unsigned long long* bp = acc2 + 6 * int64_t(g);
                const double i1 = 1.0 / double(qscale), i2 = 1.0 / double(s_scale[1]);
                const double m0 = double(a0) * INV_FIX;
                const double m1[3] = {double(a1) * i1, double(a2) * i1, double(a3) * i1};
                double m2[6];
                for (int q = 0; q < 6; ++q) m2[q] = double((long long)bp[q]) * i2;
                const int ij[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
                float Sm[3][3];
                for (int q = 0; q < 6; ++q) {
                    const int r = ij[q][0], cc = ij[q][1];
                    const float sv = float(m2[q] - m1[r] * m1[cc] / m0);
                    Sm[r][cc] = sv;
                    Sm[cc][r] = sv;
                }
                const float4 p0 = rnode[3 * g], p1 = rnode[3 * g + 1];
                const float Pm[3][3] = {{p0.x, p0.y, p0.z}, {p0.y, p0.w, p1.x}, {p0.z, p1.x, p1.y}};
                scatter_terms(Pm, Sm, 1.0f / float(n), wv);
            }
#pragma unroll
            for (int k = 0; k < NTERM; ++k) pair_add(v[k], c[k], wv[k], 0.f);
        }
        if (FULL) {
            unsigned long long* bp = acc2 + 6 * int64_t(g);
            for (int q = 0; q < 6; ++q) bp[q] = 0ull;
        }
        dbg[4 * g + 0] = double(a0) * INV_FIX;
        dbg[4 * g + 1] = double(M0) * (double(cm.x) + double(o0));
        dbg[4 * g + 2] = double(M0) * (double(cm.y) + double(o1));
        dbg[4 * g + 3] = double(M0) * (double(cm.z) + double(o2));
    }
    float ws, we;
    warp_reduce_scatter32(v, c, ws, we);
    if (lane < NTERM) sm[warp][lane] = make_float2(ws, we);
    __syncthreads();
    if (threadIdx.x < NTERM) {
        float S = 0.f, C = 0.f;
        for (int k = 0; k < VAR_THREADS / 32; ++k) pair_add(S, C, sm[k][threadIdx.x].x, sm[k][threadIdx.x].y);
        part[NTERM * blockIdx.x + threadIdx.x] = make_float2(S, C);
    }
}

__global__ void __launch_bounds__(VAR_THREADS)
k_var_solve(const float2* __restrict__ part, int nb, int it, double* __restrict__ T, float* __restrict__ Rt,
            double* __restrict__ T_hist, double* __restrict__ obj, int* __restrict__ status) {
    sum_terms_and_solve(part, nb, it, T, Rt, T_hist, obj, status);
}

}  // namespace

}  // namespace hgmm

using namespace hgmm;

int hgmm_register_impl(hgmm_tree* t, const float4* src, int64_t n64, const double* T_init,
                       int iters, float lam_c, cudaStream_t s, double* T_out, double* T_hist) {
    const int n = int(n64);
    const int n_nodes = int(hgmm_node_count(t->depth));
    {
        ProfScope ps_(t, K_REG_INIT, s);
        // lam_c < 0: the build's threshold (set here too, so that an earlier
        // call with another threshold does not leave its stop flags behind)
        if (lam_c < 0.f) lam_c = t->prm.lam_c;
        k_reg_init<<<(n_nodes + 255) / 256, 256, 0, s>>>(T_init, n_nodes, lam_c, t->stat, t->est,
                                                          t->reg_acc, t->reg_T, t->reg_Rt,
                                                          t->reg_bar, t->reg_obj);
    }
    // a large source that fits the tree's free point buffer is reordered
    // after its first round: node keys in the dead hand-off codes, per-CTA
    // counts and key totals in the build's partials (both free after the
    // build); CTAs: two per SM, fewer if the counts would not fit
    const int reorder_ctas =
        int(std::min<int64_t>(2 * t->n_sm, t->max_items * NPART * 2 / REORDER_KEYS - 1));
    const bool reorder = iters > 1 && n >= REORDER_MIN_POINTS && n64 <= t->cap && reorder_ctas >= 32 &&
                         n_nodes < REORDER_KEYS && !t->trace_on;
    const bool wide = n >= REG_WIDE_MIN_POINTS && t->reg_grid_wide > 0;
    const int grid = wide ? t->reg_grid_wide : t->reg_grid;
    auto launch = [&](const float4* pts, int rounds, double* hist, uint32_t* keys) -> int {
        RegArgs a;
        a.src = pts;
        a.n = n;
        a.est = t->est;
        a.rnode = t->rnode;
        a.root = t->root;
        a.depth = t->depth;
        a.n_nodes = n_nodes;
        a.iters = rounds;
        a.acc = t->reg_acc;
        a.part = t->reg_part;
        a.bar = t->reg_bar;
        a.T = t->reg_T;
        a.Rt = t->reg_Rt;
        a.T_hist = hist;
        a.dbg = t->reg_dbg;
        a.obj = t->reg_obj;
        a.status = t->status;
        a.keys = keys;
        a.trace = (t->trace_on && rounds <= TRACE_MAX_ITERS) ? t->trace : nullptr;
        if (a.trace) cudaMemsetAsync(t->trace, 0, size_t(rounds) * grid * TRACE_EVENTS * 8, s);
        t->trace_iters = a.trace ? rounds : 0;
        t->trace_grid = a.trace ? grid : 0;
        void* args[] = {&a};
        ProfScope ps_(t, K_DESCEND, s);
        const void* fn = wide ? (keys ? (const void*)k_register<true, 3> : (const void*)k_register<false, 3>)
                              : (keys ? (const void*)k_register<true, 2> : (const void*)k_register<false, 2>);
        const cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(REG_THREADS), args,
                                                          REG_DYN_SMEM, s);
        if (e != cudaSuccess) {
            fprintf(stderr, "hgmm: cooperative launch failed: %s\n", cudaGetErrorString(e));
            return HGMM_ECUDA;
        }
        return HGMM_OK;
    };
    if (reorder) {
        // round 1 in the caller's order, recording each point's node
        if (int rc = launch(src, 1, T_hist, t->codes)) return rc;
        {
            ProfScope ps_(t, K_REG_INIT, s);
            float4* sorted = t->pts[t->depth & 1];
            int* cnt = reinterpret_cast<int*>(t->partials);
            int* tot = cnt + int64_t(reorder_ctas) * REORDER_KEYS;
            k_src_count<<<reorder_ctas, REORDER_THREADS, 0, s>>>(t->codes, n, cnt);
            k_src_colscan<<<REORDER_KEYS / 256, 256, 0, s>>>(cnt, reorder_ctas, tot);
            k_src_keyscan<<<1, 1024, 0, s>>>(tot);
            k_src_scatter<<<reorder_ctas, REORDER_THREADS, 0, s>>>(src, n, t->codes, cnt, tot, sorted);
            src = sorted;
            // the remaining rounds start from the pose after round 1
            k_reg_init<<<(n_nodes + 255) / 256, 256, 0, s>>>(t->reg_T, n_nodes, lam_c, t->stat, t->est,
                                                              t->reg_acc, t->reg_T, t->reg_Rt,
                                                              t->reg_bar, t->reg_obj);
        }
        if (int rc = launch(src, iters - 1, T_hist ? T_hist + 16 : nullptr, nullptr)) return rc;
    } else if (iters > 0) {
        if (int rc = launch(src, iters, T_hist, nullptr)) return rc;
    }
    if (T_out) {
        ProfScope ps_(t, K_COPY_T, s);
        k_copy_T<<<1, 32, 0, s>>>(t->reg_T, T_out);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "hgmm: launch failed: %s\n", cudaGetErrorString(e));
        return HGMM_ECUDA;
    }
    return HGMM_OK;
}

int hgmm_register_descent_impl(hgmm_tree* t, const float4* src, int64_t n64, const double* T_init,
                               int iters, const hgmm_descent& d, cudaStream_t s, double* T_out,
                               double* T_hist) {
    const int n = int(n64);
    const int n_nodes = int(hgmm_node_count(t->depth));
    const float lam_c = d.lam_c >= 0.f ? d.lam_c : t->prm.lam_c;
    k_reg_init<<<(n_nodes + 255) / 256, 256, 0, s>>>(T_init, n_nodes, lam_c, t->stat, t->est, t->reg_acc,
                                                      t->reg_T, t->reg_Rt, t->reg_bar, t->reg_obj);
    const int tgrid = (n_nodes + VAR_THREADS - 1) / VAR_THREADS;
    const int dgrid = std::max(1, std::min(4 * t->n_sm, (n + VAR_THREADS - 1) / VAR_THREADS));
    const bool full = d.full_eq7 != 0;
    if (full) cudaMemsetAsync(t->reg_acc2, 0, size_t(6) * n_nodes * sizeof(unsigned long long), s);
    for (int it = 0; it < iters; ++it) {
#define HGMM_DESCEND(M, F)                                                                          \
    k_descend_var<M, F><<<dgrid, VAR_THREADS, 0, s>>>(src, n, t->est, t->depth, d.tau, t->reg_Rt, t->root, \
                                                      t->reg_acc, t->reg_acc2, t->status)
        if (d.mode == HGMM_DESCENT_ML_LOCAL) {
            if (full) HGMM_DESCEND(HGMM_DESCENT_ML_LOCAL, true); else HGMM_DESCEND(HGMM_DESCENT_ML_LOCAL, false);
        } else if (d.mode == HGMM_DESCENT_ML_GLOBAL) {
            if (full) HGMM_DESCEND(HGMM_DESCENT_ML_GLOBAL, true); else HGMM_DESCEND(HGMM_DESCENT_ML_GLOBAL, false);
        } else {
            if (full) HGMM_DESCEND(HGMM_DESCENT_MULTIPATH, true); else HGMM_DESCEND(HGMM_DESCENT_MULTIPATH, false);
        }
#undef HGMM_DESCEND
        if (full)
            k_var_terms<true><<<tgrid, VAR_THREADS, 0, s>>>(n_nodes, n, t->est, t->rnode, t->root, t->reg_acc,
                                                            t->reg_acc2, t->reg_part, t->reg_dbg);
        else
            k_var_terms<false><<<tgrid, VAR_THREADS, 0, s>>>(n_nodes, n, t->est, t->rnode, t->root, t->reg_acc,
                                                             t->reg_acc2, t->reg_part, t->reg_dbg);
        k_var_solve<<<1, VAR_THREADS, 0, s>>>(t->reg_part, tgrid, it, t->reg_T, t->reg_Rt, T_hist, t->reg_obj,
                                              t->status);
    }
    if (T_out) k_copy_T<<<1, 32, 0, s>>>(t->reg_T, T_out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "hgmm: launch failed: %s\n", cudaGetErrorString(e));
        return HGMM_ECUDA;
    }
    return HGMM_OK;
}

int hgmm_register_grid(int n_sm, int per_sm) {
    // static + dynamic shared memory exceeds the 48 KB default: opt in; the
    // grid must be co-resident for both variants (KEYS) of the build asked
    // for; 0 if that build does not reach per_sm CTAs per SM (the caller then
    // keeps to the two-per-SM build)
    if (per_sm != 2 && per_sm != 3) return 0;
    const void* fns[2] = {per_sm == 3 ? (const void*)k_register<false, 3> : (const void*)k_register<false, 2>,
                          per_sm == 3 ? (const void*)k_register<true, 3> : (const void*)k_register<true, 2>};
    int got = per_sm;
    for (const void* fn : fns) {
        int k = 0;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(REG_DYN_SMEM)) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, fn, REG_THREADS, REG_DYN_SMEM) != cudaSuccess || k < 1)
            return 0;
        got = std::min(got, k);
    }
    if (per_sm == 3 && got < 3) return 0;
    return n_sm * got;  // <= co-resident CTAs (cooperative launch)
}

int hgmm_trace_read_impl(hgmm_tree* t, unsigned long long* h, int64_t cap) {
    const int64_t need = int64_t(t->trace_iters) * t->trace_grid * TRACE_EVENTS;
    if (cap < need) return HGMM_ECAPACITY;
    if (need == 0) return HGMM_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) return HGMM_ECUDA;
    return cudaMemcpy(h, t->trace, need * 8, cudaMemcpyDeviceToHost) == cudaSuccess ? HGMM_OK
                                                                                     : HGMM_ECUDA;
}

int hgmm_barrier_timeout_probe_impl(hgmm_tree* t, long long limit, cudaStream_t s) {
    k_barrier_timeout_probe<<<1, 32, 0, s>>>(t->reg_bar + 4, t->status, limit);
    return cudaGetLastError() == cudaSuccess ? HGMM_OK : HGMM_ECUDA;
}
