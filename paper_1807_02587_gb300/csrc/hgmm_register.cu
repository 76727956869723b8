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
//               closed form: sum_l (1/lambda_l) n_l n_l^T = P, Eq. 10).  FP64.
//               The last CTA to finish reduces the per-CTA sums in a fixed
//               order, solves (Cholesky) and composes T <- dT T.
#include <cstdio>

#include "hgmm_internal.cuh"
#include "hgmm_math.cuh"

namespace hgmm {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr double FIX = 4294967296.0;      // 2^32
constexpr double INV_FIX = 1.0 / 4294967296.0;
constexpr float FIX_CLAMP = 1.0995116e12f;  // 2^40

__device__ __forceinline__ int64_t d_level_offset(int l) {
    return ((int64_t(1) << (3 * (l + 1))) - 8) / 7;
}

__global__ void k_reg_init(const double* __restrict__ T_init, int n_nodes, float lam_c,
                           const NodeStat* __restrict__ stat, NodeEst* __restrict__ est,
                           unsigned long long* __restrict__ acc, double* __restrict__ T,
                           float* __restrict__ Rt, unsigned* __restrict__ bar) {
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
        bar[0] = 0u;
        bar[2] = 0u;
    }
}

__device__ __forceinline__ long long to_fix(float v) {
    const float c = fminf(fmaxf(v, -FIX_CLAMP), FIX_CLAMP);
    return __float2ll_rn(c);
}

// Algorithm 1 for the points of this CTA (grid-stride by warps) with the
// current transform; adds each point's (gamma, gamma (z' - mu_j)) to the
// chosen node's fixed-point moments.
constexpr int STAGED_NODES = 584;  // levels 0..2 (8 + 64 + 512 nodes) live in shared memory

__device__ __forceinline__ void load_node(const NodeEst* __restrict__ est, const float4* sm_est,
                                          int64_t g, float4& ea, float4& eb, float4& ec) {
    if (g < STAGED_NODES) {
        ea = sm_est[3 * g];
        eb = sm_est[3 * g + 1];
        ec = sm_est[3 * g + 2];
    } else {
        const NodeEst* e = est + g;
        ea = __ldg(&e->a);
        eb = __ldg(&e->b);
        ec = __ldg(&e->c);
    }
}

__device__ __forceinline__ void descend_points(const float4* __restrict__ src, int n,
                                               const NodeEst* __restrict__ est, const float4* sm_est,
                                               int depth, const float* Rt_sm, float qscale,
                                               unsigned long long* __restrict__ acc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float r00 = Rt_sm[0], r01 = Rt_sm[1], r02 = Rt_sm[2], r10 = Rt_sm[3], r11 = Rt_sm[4];
    const float r12 = Rt_sm[5], r20 = Rt_sm[6], r21 = Rt_sm[7], r22 = Rt_sm[8];
    const float tx = Rt_sm[9], ty = Rt_sm[10], tz = Rt_sm[11];
    const int wpb = blockDim.x >> 5;
    const int warps_total = gridDim.x * wpb;
    for (int base = (blockIdx.x * wpb + warp) * 32; base < n; base += warps_total * 32) {
        const int i = base + lane;
        const bool valid = i < n;
        float4 z = valid ? src[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float x = fmaf(r00, z.x, fmaf(r01, z.y, fmaf(r02, z.z, tx)));
        const float y = fmaf(r10, z.x, fmaf(r11, z.y, fmaf(r12, z.z, ty)));
        const float w = fmaf(r20, z.x, fmaf(r21, z.y, fmaf(r22, z.z, tz)));
        int chosen = -1;
        float gamma = 0.f, cmx = 0.f, cmy = 0.f, cmz = 0.f;
        int local = 0;  // index within its level of the current search node
        for (int l = 0; l < depth && valid; ++l) {
            const int64_t first = d_level_offset(l) + 8 * int64_t(local);
            float sc8[8];
            float best = -CUDART_INF_F;
            int bi = -1;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                float4 ea, eb, ec;
                load_node(est, sm_est, first + c, ea, eb, ec);
                const float ex = x - ea.x, ey = y - ea.y, ez = w - ea.z;
                const float d0 = eb.x * ex;
                const float d1 = fmaf(eb.z, ey, eb.y * ex);
                const float d2 = fmaf(ec.y, ez, fmaf(ec.x, ey, eb.w * ex));
                float sc = fmaf(-d0, d0, ea.w);
                sc = fmaf(-d1, d1, sc);
                sc = fmaf(-d2, d2, sc);
                sc8[c] = sc;
                if (sc > best) { best = sc; bi = c; }
            }
            if (bi < 0) break;  // the current node has no live children
            float sum = 0.f;
#pragma unroll
            for (int c = 0; c < 8; ++c) sum += exp2f(sc8[c] - best);
            gamma = 1.0f / sum;
            chosen = int(first + bi);
            local = 8 * local + bi;
            float4 ea, eb, ec;
            load_node(est, sm_est, chosen, ea, eb, ec);
            cmx = ea.x; cmy = ea.y; cmz = ea.z;
            if (ec.z != 0.f) break;  // Complexity <= lambda_c
        }
        // Sum (gamma, gamma (z' - mu_j)) over the lanes of this warp that chose
        // the same node j: a pairwise tree over the members' ranks (fixed order,
        // so deterministic), then one fixed-point atomic per value and group.
        // Integer adds are exact, so the node totals do not depend on the
        // order in which groups arrive.
        const bool has = chosen >= 0;
        float v0 = has ? gamma : 0.f;
        float v1 = has ? gamma * (x - cmx) : 0.f;
        float v2 = has ? gamma * (y - cmy) : 0.f;
        float v3 = has ? gamma * (w - cmz) : 0.f;
        const unsigned peers = __match_any_sync(FULL, chosen);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        const int gsize = __popc(peers);
        const unsigned higher = lane == 31 ? 0u : (peers & ~((2u << lane) - 1u));
#pragma unroll
        for (int st = 1; st < 32; st <<= 1) {
            unsigned h = higher;  // lane holding rank + st within my group
            for (int k = 1; k < st; ++k) h &= h - 1u;
            const int srcl = h ? __ffs(h) - 1 : lane;
            const float o0 = __shfl_sync(FULL, v0, srcl);
            const float o1 = __shfl_sync(FULL, v1, srcl);
            const float o2 = __shfl_sync(FULL, v2, srcl);
            const float o3 = __shfl_sync(FULL, v3, srcl);
            if ((rank & (2 * st - 1)) == 0 && rank + st < gsize) {
                v0 += o0; v1 += o1; v2 += o2; v3 += o3;
            }
        }
        if (has && rank == 0) {
            // one of ACC_REPLICAS copies per CTA spreads the atomics on hot
            // nodes (a ground plane collects a large share of the points)
            unsigned long long* dst =
                acc + 4 * (int64_t(chosen) * ACC_REPLICAS + (blockIdx.x & (ACC_REPLICAS - 1)));
            atomicAdd(dst + 0, (unsigned long long)to_fix(v0 * 4294967296.0f));
            atomicAdd(dst + 1, (unsigned long long)to_fix(v1 * qscale));
            atomicAdd(dst + 2, (unsigned long long)to_fix(v2 * qscale));
            atomicAdd(dst + 3, (unsigned long long)to_fix(v3 * qscale));
        }
    }
}

// Per-node contribution to the 6x6 normal equations in FP32; the sums over
// nodes are compensated (TwoSum pairs), so the 27 totals that reach the FP64
// solve carry ~2x FP32 precision.  Per node j with mass (M0 > 0):
//   mu* = mu_j32 + o,  o = (M1 rel. to mu_j32) / M0,   d = mu_j - mu* = dmu_j - o
//   H_j = pi* [[A [mu*]x^T, A], [A^T, P]],  A = [mu*]x P,   g_j = pi* [mu* x P d; P d]
__device__ __forceinline__ void node_terms(const float4 p0, const float4 p1, const float4 dm,
                                           const float4 cm, float M0, float o0, float o1,
                                           float o2, float pis, float* v) {
    const float P[3][3] = {{p0.x, p0.y, p0.z}, {p0.y, p0.w, p1.x}, {p0.z, p1.x, p1.y}};
    const float m0 = cm.x + o0, m1 = cm.y + o1, m2 = cm.z + o2;
    const float d0 = dm.x - o0, d1 = dm.y - o1, d2 = dm.z - o2;
    float A[3][3], Bm[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        A[0][k] = m1 * P[2][k] - m2 * P[1][k];
        A[1][k] = m2 * P[0][k] - m0 * P[2][k];
        A[2][k] = m0 * P[1][k] - m1 * P[0][k];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        Bm[i][0] = m1 * A[i][2] - m2 * A[i][1];
        Bm[i][1] = m2 * A[i][0] - m0 * A[i][2];
        Bm[i][2] = m0 * A[i][1] - m1 * A[i][0];
    }
    float Pd[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) Pd[i] = P[i][0] * d0 + P[i][1] * d1 + P[i][2] * d2;
    const float top[3] = {m1 * Pd[2] - m2 * Pd[1], m2 * Pd[0] - m0 * Pd[2], m0 * Pd[1] - m1 * Pd[0]};
    int k = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i; j < 6; ++j) {
            float h;
            if (i < 3 && j < 3) h = Bm[i][j];
            else if (i < 3) h = A[i][j - 3];
            else h = P[i - 3][j - 3];
            v[k++] = pis * h;
        }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        v[21 + i] = pis * top[i];
        v[24 + i] = pis * Pd[i];
    }
    (void)M0;
}

// T <- dT T with dT = (Rodrigues(w), t); FP64.  sin(th)/th and
// (1 - cos th)/th^2 by their Taylor series for th < 0.5 (truncation < 1e-15).
__device__ inline void compose_update(const double x[6], double* T) {
    const double th2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    double a, b;
    if (th2 < 0.25) {
        a = 1.0 + th2 * (-1.0 / 6 + th2 * (1.0 / 120 + th2 * (-1.0 / 5040 + th2 * (1.0 / 362880 +
            th2 * (-1.0 / 39916800 + th2 * (1.0 / 6227020800.0))))));
        b = 0.5 + th2 * (-1.0 / 24 + th2 * (1.0 / 720 + th2 * (-1.0 / 40320 + th2 * (1.0 / 3628800 +
            th2 * (-1.0 / 479001600 + th2 * (1.0 / 87178291200.0))))));
    } else {
        const double th = sqrt(th2);
        a = sin(th) / th;
        b = (1.0 - cos(th)) / th2;
    }
    const double K[9] = {0, -x[2], x[1], x[2], 0, -x[0], -x[1], x[0], 0};
    double dR[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double kk = 0.0;
            for (int m = 0; m < 3; ++m) kk += K[i * 3 + m] * K[m * 3 + j];
            dR[i * 3 + j] = (i == j ? 1.0 : 0.0) + a * K[i * 3 + j] + b * kk;
        }
    double Tn[12];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 4; ++c)
            Tn[r * 4 + c] = dR[r * 3 + 0] * T[c] + dR[r * 3 + 1] * T[4 + c] + dR[r * 3 + 2] * T[8 + c];
        Tn[r * 4 + 3] += x[3 + r];
    }
    for (int k = 0; k < 12; ++k) T[k] = Tn[k];
}

// FP64 solve of the 6x6 normal equations and the pose update by one warp.
// Lane i < 6 owns row i; the right-looking Cholesky updates all rows with
// one instruction per column, so the FP64 instruction count of the critical
// path (~70 cycles each on this part) is about a third of a one-thread
// solve.  L is kept in shared memory for the back substitution.  Returns
// false (uniformly) for a non-positive pivot.
__device__ bool warp_solve_update(const double* tot, double (*Lsm)[6], double* T,
                                  float* Rt, double* T_hist, int iter) {
    const int lane = threadIdx.x & 31;
    const int row = lane < 6 ? lane : 5;
    auto H = [&](int i, int j) {  // upper-packed 21 entries
        if (i > j) { const int t = i; i = j; j = t; }
        return tot[i * 6 - (i * (i - 1)) / 2 + (j - i)];
    };
    double a[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) a[j] = H(row, j);
    double g = tot[21 + row];
    double dmax = 0.0;
#pragma unroll
    for (int j = 0; j < 6; ++j) dmax = fmax(dmax, H(j, j));
    double r[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double dk = __shfl_sync(FULL, a[k], k);
        if (!(dk > 1e-15 * dmax)) return false;
        r[k] = rsqrt_f64(dk);
        const double lik = a[k] * r[k];  // L_ik for rows i >= k
        if (lane < 6) Lsm[k][lane] = lik;
#pragma unroll
        for (int j = k + 1; j < 6; ++j) {
            const double ljk = __shfl_sync(FULL, lik, j);
            a[j] = fma(-lik, ljk, a[j]);
        }
    }
    __syncwarp();
    // forward: L y = g (column k: y_k = g_k r_k, then rows i > k lose L_ik y_k)
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double yk = __shfl_sync(FULL, g, k) * r[k];
        if (lane == k) g = yk;
        else if (lane > k) g = fma(-Lsm[k][row], yk, g);
    }
    // backward: L^T x = y (x_k = y_k r_k, then rows j < k lose L_kj x_k)
    double x[6];
#pragma unroll
    for (int k = 5; k >= 0; --k) {
        const double xk = __shfl_sync(FULL, g, k) * r[k];
        x[k] = xk;
        if (lane < k) g = fma(-Lsm[lane][k], xk, g);
    }
    // dT = (Rodrigues(w), t); lane e < 12 computes entry e of the new [R|t]
    const double th2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    double ca, cb;
    if (th2 < 0.25) {
        ca = 1.0 + th2 * (-1.0 / 6 + th2 * (1.0 / 120 + th2 * (-1.0 / 5040 + th2 * (1.0 / 362880 +
             th2 * (-1.0 / 39916800 + th2 * (1.0 / 6227020800.0))))));
        cb = 0.5 + th2 * (-1.0 / 24 + th2 * (1.0 / 720 + th2 * (-1.0 / 40320 + th2 * (1.0 / 3628800 +
             th2 * (-1.0 / 479001600 + th2 * (1.0 / 87178291200.0))))));
    } else {
        const double th = sqrt(th2);
        ca = sin(th) / th;
        cb = (1.0 - cos(th)) / th2;
    }
    const int e = lane < 12 ? lane : 11;
    const int rr = e >> 2, cc = e & 3;
    // row rr of dR = I + a K + b K^2, K = [w]x, (K^2)_{rm} = w_r w_m - |w|^2 delta_rm
    const double kr[3] = {rr == 0 ? 0.0 : (rr == 1 ? x[2] : -x[1]),
                          rr == 0 ? -x[2] : (rr == 1 ? 0.0 : x[0]),
                          rr == 0 ? x[1] : (rr == 1 ? -x[0] : 0.0)};
    double acc = cc == 3 ? x[3 + rr] : 0.0;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const double drm = (m == rr ? 1.0 - cb * th2 : 0.0) + ca * kr[m] + cb * x[rr] * x[m];
        acc = fma(drm, __ldcg(T + m * 4 + cc), acc);
    }
    __syncwarp();
    if (lane < 12) {
        T[e] = acc;
        Rt[cc == 3 ? 9 + rr : rr * 3 + cc] = float(acc);
        if (T_hist) T_hist[16 * iter + e] = acc;
    }
    if (T_hist && lane >= 12 && lane < 16) T_hist[16 * iter + lane] = lane == 15 ? 1.0 : 0.0;
    return true;
}

// Bounded grid-wide barrier for a cooperative launch (all CTAs co-resident):
// generation counter, spin with a sleep and an iteration limit; on timeout
// it records ST_TIMEOUT and returns false so the kernel can exit.
constexpr long long BARRIER_SPIN_LIMIT = 1000000;  // about a second

__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* status, long long limit) {
    __shared__ int ok_sm;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = bar + 1;
        const unsigned gen = *vgen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long spins = 0;
            while (*vgen == gen) {
                if (++spins > limit) {
                    atomicOr(status, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_sm = ok;
    }
    __syncthreads();
    return ok_sm != 0;
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
    double* dbg;
    int* status;
    unsigned long long* trace;  // optional: [iter][cta][TRACE_EVENTS] globaltimer ns
};

constexpr int TRACE_EVENTS = 6;

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
//   -- grid barrier --
//   B. per node with mass: its 27 normal-equation terms (FP32), compensated
//      block sums -> one partial per CTA; the last CTA to finish
//   C. reduces the partials in a fixed order, solves the 6x6 system in FP64
//      and composes T <- dT T
//   -- grid barrier --  (everyone reads the new T)
__global__ void __launch_bounds__(REG_THREADS, 2) k_register(RegArgs a) {
    __shared__ float Rt_sm[12];
    __shared__ float2 sm[REG_THREADS / 32][27];
    __shared__ float2 fin[8][27];
    __shared__ double tot[27];
    __shared__ double Lsm[6][6];
    __shared__ bool last;
    __shared__ float4 sm_est[3 * STAGED_NODES];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the top levels of the tree are read by every point: stage them once
    // for all rounds (the stop flags were set by k_reg_init before launch)
    {
        const int ns = a.n_nodes < STAGED_NODES ? a.n_nodes : STAGED_NODES;
        const float4* gsrc = reinterpret_cast<const float4*>(a.est);
        for (int i = threadIdx.x; i < 3 * ns; i += blockDim.x) sm_est[i] = gsrc[i];
        __syncthreads();
    }
    const double ext = a.root->extent > 0.0 ? a.root->extent : 1.0;
    const float qscale = float(FIX / ext);  // fixed-point units per metre
    for (int it = 0; it < a.iters; ++it) {
        trace_mark(a.trace, it, 0);
        if (threadIdx.x < 12) Rt_sm[threadIdx.x] = __ldcg(a.Rt + threadIdx.x);
        __syncthreads();
        descend_points(a.src, a.n, a.est, sm_est, a.depth, Rt_sm, qscale, a.acc);
        trace_mark(a.trace, it, 1);
        if (!grid_barrier(a.bar, a.status, BARRIER_SPIN_LIMIT)) return;
        trace_mark(a.trace, it, 2);
        // ---- B: node terms (only the CTAs that own nodes take part)
        const int nb_nodes = (a.n_nodes + blockDim.x - 1) / blockDim.x;
        if (blockIdx.x < nb_nodes) {
        float v[27], c[27];
#pragma unroll
        for (int k = 0; k < 27; ++k) { v[k] = 0.f; c[k] = 0.f; }
        double* dbg = it == a.iters - 1 ? a.dbg : nullptr;
        for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.n_nodes; g += nb_nodes * blockDim.x) {
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
            const float4 cm = a.est[g].a;
            float M0 = 0.f, o0 = 0.f, o1 = 0.f, o2 = 0.f;
            if (a0 > 0) {
                float w[27];
                M0 = float(a0) * 2.3283064365386963e-10f;  // 2^-32
                const float inv = 1.0f / (qscale * M0);
                o0 = float(a1) * inv;
                o1 = float(a2) * inv;
                o2 = float(a3) * inv;
                node_terms(a.rnode[3 * g], a.rnode[3 * g + 1], a.rnode[3 * g + 2], cm, M0, o0, o1,
                           o2, M0 / float(a.n), w);
#pragma unroll
                for (int k = 0; k < 27; ++k) pair_add(v[k], c[k], w[k], 0.f);
            }
            if (dbg) {
                dbg[4 * g + 0] = double(a0) * INV_FIX;
                dbg[4 * g + 1] = double(M0) * (double(cm.x) + double(o0));
                dbg[4 * g + 2] = double(M0) * (double(cm.y) + double(o1));
                dbg[4 * g + 3] = double(M0) * (double(cm.z) + double(o2));
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int k = 0; k < 27; ++k) {
                const float s2 = __shfl_xor_sync(FULL, v[k], off);
                const float c2 = __shfl_xor_sync(FULL, c[k], off);
                pair_add(v[k], c[k], s2, c2);
            }
        if (lane == 0)
            for (int k = 0; k < 27; ++k) sm[warp][k] = make_float2(v[k], c[k]);
        __syncthreads();
        if (threadIdx.x < 27) {
            float S = 0.f, C = 0.f;
            for (int w = 0; w < REG_THREADS / 32; ++w) pair_add(S, C, sm[w][threadIdx.x].x, sm[w][threadIdx.x].y);
            a.part[27 * blockIdx.x + threadIdx.x] = make_float2(S, C);
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) last = (atomicAdd(a.bar + 2, 1u) == unsigned(nb_nodes) - 1);
        __syncthreads();
        trace_mark(a.trace, it, 3);
        if (last) {
            // ---- C: fixed-order reduction, FP64 solve, pose update
            __threadfence();
            const int nb = nb_nodes;
            // all partial loads in flight at once (8 groups of 27 threads),
            // then a fixed-order combine
            if (threadIdx.x < 216) {
                const int k = threadIdx.x % 27, q = threadIdx.x / 27;
                float S = 0.f, C = 0.f;
                float2 xs[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int b = q + 8 * j;
                    xs[j] = b < nb ? __ldcg(&a.part[27 * b + k]) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) pair_add(S, C, xs[j].x, xs[j].y);
                for (int b = q + 64; b < nb; b += 8) {
                    const float2 x = __ldcg(&a.part[27 * b + k]);
                    pair_add(S, C, x.x, x.y);
                }
                fin[q][k] = make_float2(S, C);
            }
            __syncthreads();
            if (threadIdx.x < 27) {
                float S = 0.f, C = 0.f;
                for (int q = 0; q < 8; ++q) pair_add(S, C, fin[q][threadIdx.x].x, fin[q][threadIdx.x].y);
                tot[threadIdx.x] = double(S) + double(C);
            }
            __syncthreads();
            if (warp == 0) {
                const bool solved = warp_solve_update(tot, Lsm, a.T, a.Rt, a.T_hist, it);
                if (!solved && lane == 0) {
                    atomicOr(a.status, ST_DEGENERATE);  // T kept for this round
                    if (a.T_hist)
                        for (int k = 0; k < 16; ++k) a.T_hist[16 * it + k] = __ldcg(a.T + k);
                }
                if (lane == 0) a.bar[2] = 0u;
                __threadfence();
            }
            trace_mark(a.trace, it, 4);
        }
        }  // node-owning CTAs
        if (!grid_barrier(a.bar, a.status, BARRIER_SPIN_LIMIT)) return;
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

__global__ void k_copy_T(const double* __restrict__ T, double* __restrict__ out) {
    if (threadIdx.x < 16) out[threadIdx.x] = T[threadIdx.x];
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
        k_reg_init<<<(n_nodes + 255) / 256, 256, 0, s>>>(T_init, n_nodes, lam_c, t->stat, t->est,
                                                          t->reg_acc, t->reg_T, t->reg_Rt,
                                                          t->reg_bar);
    }
    if (iters > 0) {
        RegArgs a;
        a.src = src;
        a.n = n;
        a.est = t->est;
        a.rnode = t->rnode;
        a.root = t->root;
        a.depth = t->depth;
        a.n_nodes = n_nodes;
        a.iters = iters;
        a.acc = t->reg_acc;
        a.part = t->reg_part;
        a.bar = t->reg_bar;
        a.T = t->reg_T;
        a.Rt = t->reg_Rt;
        a.T_hist = T_hist;
        a.dbg = t->reg_dbg;
        a.status = t->status;
        a.trace = (t->trace_on && iters <= TRACE_MAX_ITERS) ? t->trace : nullptr;
        if (a.trace) cudaMemsetAsync(t->trace, 0, size_t(iters) * t->reg_grid * TRACE_EVENTS * 8, s);
        t->trace_iters = a.trace ? iters : 0;
        void* args[] = {&a};
        ProfScope ps_(t, K_DESCEND, s);
        const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_register, dim3(t->reg_grid),
                                                          dim3(REG_THREADS), args, 0, s);
        if (e != cudaSuccess) {
            fprintf(stderr, "hgmm: cooperative launch failed: %s\n", cudaGetErrorString(e));
            return HGMM_ECUDA;
        }
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

int hgmm_register_grid(int n_sm) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_register, REG_THREADS, 0) != cudaSuccess ||
        per_sm < 1)
        return 0;
    return n_sm * (per_sm < 2 ? per_sm : 2);  // <= co-resident CTAs (cooperative launch)
}

int hgmm_trace_read_impl(hgmm_tree* t, unsigned long long* h, int64_t cap) {
    const int64_t need = int64_t(t->trace_iters) * t->reg_grid * TRACE_EVENTS;
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
