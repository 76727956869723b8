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
                           float* __restrict__ Rt, unsigned* __restrict__ counter) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_nodes) {
        acc[4 * i + 0] = 0ull;
        acc[4 * i + 1] = 0ull;
        acc[4 * i + 2] = 0ull;
        acc[4 * i + 3] = 0ull;
        if (lam_c >= 0.f)
            est[i].c.z = (stat[i].live && stat[i].complexity <= double(lam_c)) ? 1.f : 0.f;
    }
    if (i == 0) {
        for (int k = 0; k < 16; ++k) T[k] = T_init ? T_init[k] : ((k % 5 == 0) ? 1.0 : 0.0);
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) Rt[r * 3 + c] = float(T[r * 4 + c]);
            Rt[9 + r] = float(T[r * 4 + 3]);
        }
        *counter = 0u;
    }
}

__device__ __forceinline__ long long to_fix(float v) {
    const float c = fminf(fmaxf(v, -FIX_CLAMP), FIX_CLAMP);
    return __float2ll_rn(c);
}

__global__ void __launch_bounds__(REG_THREADS) k_descend(const float4* __restrict__ src, int n,
                                                        const NodeEst* __restrict__ est, int depth,
                                                        const float* __restrict__ Rt,
                                                        const RootDev* __restrict__ root,
                                                        unsigned long long* __restrict__ acc) {
    __shared__ unsigned long long slot[REG_THREADS / 32][32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v = 0; v < 4; ++v) slot[warp][lane][v] = 0ull;
    __syncwarp();
    const float r00 = Rt[0], r01 = Rt[1], r02 = Rt[2], r10 = Rt[3], r11 = Rt[4], r12 = Rt[5];
    const float r20 = Rt[6], r21 = Rt[7], r22 = Rt[8], tx = Rt[9], ty = Rt[10], tz = Rt[11];
    // fixed-point units per metre (a zero-extent cloud uses unit scale)
    const float qscale = float(FIX / (root->extent > 0.0 ? root->extent : 1.0));
    const int warps_total = gridDim.x * (REG_THREADS / 32);
    for (int base = (blockIdx.x * (REG_THREADS / 32) + warp) * 32; base < n; base += warps_total * 32) {
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
            float s[8];
            float best = -CUDART_INF_F;
            int bi = -1;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const NodeEst* e = est + first + c;
                const float4 a = __ldg(&e->a), b = __ldg(&e->b), cc = __ldg(&e->c);
                const float ex = x - a.x, ey = y - a.y, ez = w - a.z;
                const float d0 = b.x * ex;
                const float d1 = fmaf(b.z, ey, b.y * ex);
                const float d2 = fmaf(cc.y, ez, fmaf(cc.x, ey, b.w * ex));
                float sc = fmaf(-d0, d0, a.w);
                sc = fmaf(-d1, d1, sc);
                sc = fmaf(-d2, d2, sc);
                s[c] = sc;
                if (sc > best) { best = sc; bi = c; }
            }
            if (bi < 0) break;  // the current node has no live children
            float sum = 0.f;
#pragma unroll
            for (int c = 0; c < 8; ++c) sum += exp2f(s[c] - best);
            gamma = 1.0f / sum;
            chosen = int(first + bi);
            local = 8 * local + bi;
            const float4 a = __ldg(&est[chosen].a);
            cmx = a.x; cmy = a.y; cmz = a.z;
            if (__ldg(&est[chosen].c).z != 0.f) break;  // Complexity <= lambda_c
        }
        // accumulate (M0, M1 relative to the node's FP32 mean) as fixed point
        const bool has = chosen >= 0;
        long long v0 = 0, v1 = 0, v2 = 0, v3 = 0;
        if (has) {
            v0 = to_fix(gamma * 4294967296.0f);
            v1 = to_fix(gamma * (x - cmx) * qscale);
            v2 = to_fix(gamma * (y - cmy) * qscale);
            v3 = to_fix(gamma * (w - cmz) * qscale);
        }
        const unsigned active = __ballot_sync(FULL, has);
        if (has) {
            const unsigned peers = __match_any_sync(active, chosen);
            const int leader = __ffs(peers) - 1;
            unsigned long long* dst = acc + 4 * int64_t(chosen);
            if (peers == (1u << lane)) {
                atomicAdd(dst + 0, (unsigned long long)v0);
                atomicAdd(dst + 1, (unsigned long long)v1);
                atomicAdd(dst + 2, (unsigned long long)v2);
                atomicAdd(dst + 3, (unsigned long long)v3);
            } else {
                atomicAdd(&slot[warp][leader][0], (unsigned long long)v0);
                atomicAdd(&slot[warp][leader][1], (unsigned long long)v1);
                atomicAdd(&slot[warp][leader][2], (unsigned long long)v2);
                atomicAdd(&slot[warp][leader][3], (unsigned long long)v3);
                __syncwarp(peers);
                if (lane == leader) {
                    for (int v = 0; v < 4; ++v) {
                        atomicAdd(dst + v, slot[warp][lane][v]);
                        slot[warp][lane][v] = 0ull;
                    }
                }
                __syncwarp(peers);
            }
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

__global__ void __launch_bounds__(MSTEP_THREADS) k_mstep(int n_nodes, int n_src, int iter,
                                                        const float4* __restrict__ rnode,
                                                        const NodeEst* __restrict__ est,
                                                        const RootDev* __restrict__ root,
                                                        unsigned long long* __restrict__ acc,
                                                        float2* __restrict__ part,
                                                        unsigned* __restrict__ counter,
                                                        double* __restrict__ T, float* __restrict__ Rt,
                                                        double* __restrict__ T_hist,
                                                        double* __restrict__ dbg,
                                                        int* __restrict__ status) {
    __shared__ float2 sm[MSTEP_THREADS / 32][27];
    __shared__ float2 fin[4][27];
    __shared__ bool last;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float v[27], c[27];
#pragma unroll
    for (int k = 0; k < 27; ++k) { v[k] = 0.f; c[k] = 0.f; }
    if (g < n_nodes) {
        const long long a0 = (long long)acc[4 * g + 0];
        const long long a1 = (long long)acc[4 * g + 1];
        const long long a2 = (long long)acc[4 * g + 2];
        const long long a3 = (long long)acc[4 * g + 3];
        acc[4 * g + 0] = 0ull;
        acc[4 * g + 1] = 0ull;
        acc[4 * g + 2] = 0ull;
        acc[4 * g + 3] = 0ull;
        const float4 cm = est[g].a;
        float M0 = 0.f, o0 = 0.f, o1 = 0.f, o2 = 0.f;
        if (a0 > 0) {
            M0 = float(a0) * 2.3283064365386963e-10f;  // 2^-32
            const float qs = float(FIX / (root->extent > 0.0 ? root->extent : 1.0));
            const float inv = 1.0f / (qs * M0);
            o0 = float(a1) * inv;
            o1 = float(a2) * inv;
            o2 = float(a3) * inv;
            node_terms(rnode[3 * g], rnode[3 * g + 1], rnode[3 * g + 2], cm, M0, o0, o1, o2,
                       M0 / float(n_src), v);
        }
        if (dbg) {
            dbg[4 * g + 0] = double(a0) * INV_FIX;
            dbg[4 * g + 1] = double(M0) * (double(cm.x) + double(o0));
            dbg[4 * g + 2] = double(M0) * (double(cm.y) + double(o1));
            dbg[4 * g + 3] = double(M0) * (double(cm.z) + double(o2));
        }
    }
    // compensated warp + block reduction, fixed order
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
        for (int w = 0; w < MSTEP_THREADS / 32; ++w) pair_add(S, C, sm[w][threadIdx.x].x, sm[w][threadIdx.x].y);
        part[27 * blockIdx.x + threadIdx.x] = make_float2(S, C);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the last CTA: 4 groups of 27 threads sum the block partials (fixed order)
    const int nb = gridDim.x;
    if (threadIdx.x < 108) {
        const int k = threadIdx.x % 27, q = threadIdx.x / 27;
        float S = 0.f, C = 0.f;
        for (int b = q; b < nb; b += 4) {
            const float2 x = __ldcg(&part[27 * b + k]);
            pair_add(S, C, x.x, x.y);
        }
        fin[q][k] = make_float2(S, C);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot[27];
        for (int k = 0; k < 27; ++k) {
            float S = 0.f, C = 0.f;
            for (int q = 0; q < 4; ++q) pair_add(S, C, fin[q][k].x, fin[q][k].y);
            tot[k] = double(S) + double(C);
        }
        double x[6];
        double Tl[16];
        for (int k = 0; k < 16; ++k) Tl[k] = T[k];
        if (chol_solve6(tot, tot + 21, x)) {
            compose_update(x, Tl);
        } else {
            atomicOr(status, ST_DEGENERATE);
        }
        for (int k = 0; k < 16; ++k) T[k] = Tl[k];
        for (int r = 0; r < 3; ++r) {
            for (int cc = 0; cc < 3; ++cc) Rt[r * 3 + cc] = float(Tl[r * 4 + cc]);
            Rt[9 + r] = float(Tl[r * 4 + 3]);
        }
        if (T_hist)
            for (int k = 0; k < 16; ++k) T_hist[16 * iter + k] = Tl[k];
        *counter = 0u;
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
    const int nb = (n_nodes + MSTEP_THREADS - 1) / MSTEP_THREADS;
    {
        ProfScope ps_(t, K_REG_INIT, s);
        k_reg_init<<<(n_nodes + 255) / 256, 256, 0, s>>>(T_init, n_nodes, lam_c, t->stat, t->est,
                                                          t->reg_acc, t->reg_T, t->reg_Rt,
                                                          t->reg_counter);
    }
    for (int it = 0; it < iters; ++it) {
        {
            ProfScope ps_(t, K_DESCEND, s);
            k_descend<<<t->reg_grid, REG_THREADS, 0, s>>>(src, n, t->est, t->depth, t->reg_Rt, t->root,
                                                         t->reg_acc);
        }
        {
            ProfScope ps_(t, K_REG_MSTEP, s);
            k_mstep<<<nb, MSTEP_THREADS, 0, s>>>(n_nodes, n, it, t->rnode, t->est, t->root, t->reg_acc,
                                                 t->reg_part, t->reg_counter, t->reg_T, t->reg_Rt,
                                                 T_hist, t->reg_dbg, t->status);
        }
    }
    {
        ProfScope ps_(t, K_COPY_T, s);
        if (T_out) k_copy_T<<<1, 32, 0, s>>>(t->reg_T, T_out);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "hgmm: launch failed: %s\n", cudaGetErrorString(e));
        return HGMM_ECUDA;
    }
    return HGMM_OK;
}
