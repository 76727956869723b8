// Flat "GMM J=n" variant (Sec. 5, variant 3): a single-level GMM whose J
// components every point is associated with (Eq. 3 over all J), the moments
// of Eq. 8 over every (point, component) pair, and the tree's M-step
// (Eq. 9-16) and pose update.
//
// One round is four launches:
//   k_flat_lse      four lanes per two points (each lane every fourth
//                   component), components staged in shared memory:
//                   log2 sum_j pi_j N(z'|Theta_j) of every point (chunks of
//                   8 components share one rescale of the running sum; the
//                   four partial sums are combined by shuffles).  FP32, log2
//                   domain.
//   k_flat_moments  thread per component, a slice of points staged in shared
//                   memory: gamma_ij = 2^(s_ij - lse_i) and its moments
//                   centred on the component's FP32 mean, plain FP32 sums
//                   over 16 points folded into compensated pairs; one partial
//                   per (slice, component).  The same kernel with 10 moments
//                   is the E-step of the flat EM fit.
//   k_flat_terms    32 components per CTA, eight warps splitting the
//                   slices: fixed-order sums, then per component the Eq. 12-16
//                   normal-equation and objective terms (node_terms) and a
//                   warp reduce-scatter to one partial per CTA.
//   k_flat_solve    fixed-order sum of the CTA partials, FP64 solve and
//                   T <- dT T by one warp (warp_solve_update).
// Every sum has a fixed order, so a registration is bit-reproducible.
#include <cstdio>
#include <cstring>

#include "hgmm_dev.cuh"
#include "../../include/hgmm_flat.h"

namespace hgmm {

struct FlatComp {
    double pi;
    double mu[3];
    double S[6];     // xx xy xz yy yz zz
    double lam[3];   // descending
    double V[9];     // eigenvectors in columns
    double P[6];     // V diag(1 / max(lambda, eps)) V^T
    int live;
    int level, index;
    int pad;
};

namespace {

constexpr int FROM_TREE_THREADS = 1024;
constexpr int LSE_THREADS = 256;
constexpr int LSE_PPT = 2;       // points per thread
constexpr int LSE_SPLIT = 4;     // lanes sharing one point group (each takes every 4th component)
constexpr int LSE_POINTS = LSE_THREADS / LSE_SPLIT * LSE_PPT;  // points per CTA
constexpr int LSE_TILE = 512;    // components staged per pass
constexpr int MOM_THREADS = 256; // one component per thread
constexpr int MOM_STAGE = 256;   // points staged per pass
constexpr int NMOM_MAX = 10;

// ------------------------------------------------------------ from the tree
// One CTA.  Candidates are the nodes of levels 0..L-1 (global id order);
// thread t takes a contiguous run of them, so the block scan of the run
// counts gives the components in (level, index) order.
__global__ void __launch_bounds__(FROM_TREE_THREADS)
k_flat_from_tree(const NodeStat* __restrict__ st, const RootDev* __restrict__ root, int L, int n_cand,
                 FlatComp* __restrict__ comp, NodeEst* __restrict__ est, float4* __restrict__ rterm,
                 int* __restrict__ meta, double* __restrict__ eps_out, int* __restrict__ status) {
    __shared__ int wcount[FROM_TREE_THREADS / 32];
    __shared__ double wsum[FROM_TREE_THREADS / 32];
    __shared__ double total_sh;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int per = (n_cand + FROM_TREE_THREADS - 1) / FROM_TREE_THREADS;
    const int g0 = min(n_cand, t * per), g1 = min(n_cand, g0 + per);
    // pass 1: flags, weights, counts
    int cnt = 0;
    double wsum_t = 0.0;
    for (int g = g0; g < g1; ++g) {
        int l = 0;
        while (l + 1 < L && g >= d_level_offset(l + 1)) ++l;
        const int64_t i = g - d_level_offset(l);
        if (!st[g].live) continue;
        bool child = false;
        if (l + 1 < L) {
            const int64_t c0 = d_level_offset(l + 1) + 8 * i;
            for (int c = 0; c < 8; ++c) child = child || st[c0 + c].live;
        }
        if (child) continue;
        double w = 1.0;
        for (int k = 0; k <= l; ++k) w = st[d_level_offset(k) + (i >> (3 * (l - k)))].pi * w;
        wsum_t += w;
        ++cnt;
    }
    // block scan of the counts, block sum of the weights (fixed order)
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += v;
    }
    double ws = wsum_t;
    for (int o = 16; o > 0; o >>= 1) ws += __shfl_down_sync(FULL, ws, o);
    if (lane == 31) wcount[warp] = incl;
    if (lane == 0) wsum[warp] = ws;
    __syncthreads();
    if (t == 0) {
        int run = 0;
        double tot = 0.0;
        for (int w = 0; w < FROM_TREE_THREADS / 32; ++w) {
            const int c = wcount[w];
            wcount[w] = run;
            run += c;
            tot += wsum[w];
        }
        total_sh = tot;
        meta[0] = run;
        *eps_out = root->eps;
        if (!(tot > 0.0)) atomicOr(status, ST_DEGENERATE);
    }
    __syncthreads();
    const double inv_total = total_sh > 0.0 ? 1.0 / total_sh : 0.0;
    const double eps = root->eps;
    int j = wcount[warp] + incl - cnt;
    // pass 2: write the components
    for (int g = g0; g < g1; ++g) {
        int l = 0;
        while (l + 1 < L && g >= d_level_offset(l + 1)) ++l;
        const int64_t i = g - d_level_offset(l);
        const NodeStat& s = st[g];
        if (!s.live) continue;
        bool child = false;
        if (l + 1 < L) {
            const int64_t c0 = d_level_offset(l + 1) + 8 * i;
            for (int c = 0; c < 8; ++c) child = child || st[c0 + c].live;
        }
        if (child) continue;
        double w = 1.0;
        for (int k = 0; k <= l; ++k) w = st[d_level_offset(k) + (i >> (3 * (l - k)))].pi * w;
        FlatComp& f = comp[j];
        f.pi = w * inv_total;
        for (int a = 0; a < 3; ++a) f.mu[a] = s.mu[a];
        for (int v = 0; v < 6; ++v) f.S[v] = s.S[v];
        for (int a = 0; a < 3; ++a) f.lam[a] = s.lam[a];
        for (int v = 0; v < 9; ++v) f.V[v] = s.V[v];
        for (int v = 0; v < 6; ++v) f.P[v] = s.P[v];
        f.live = 1;
        f.level = l;
        f.index = int(i);
        if (!pack_est(f.pi, f.mu, f.S, eps, 0.f, est[j])) atomicOr(status, ST_CHOL);
        const float4 a = est[j].a;
        rterm[3 * j] = make_float4(float(s.P[0]), float(s.P[1]), float(s.P[2]), float(s.P[3]));
        rterm[3 * j + 1] = make_float4(float(s.P[4]), float(s.P[5]), 0.f, 0.f);
        rterm[3 * j + 2] = make_float4(float(s.mu[0] - double(a.x)), float(s.mu[1] - double(a.y)),
                                       float(s.mu[2] - double(a.z)), 0.f);
        ++j;
    }
}

// ------------------------------------------------------------- E-step parts
__device__ __forceinline__ void load_rt(const float* Rt, float (&r)[12]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) r[k] = Rt[k];
}

// z' = R z + t (the descent's arithmetic); a point with a non-finite
// coordinate is excluded (it gets lse = +inf, so gamma = 0) and reported
// to `status` if that is not NULL.
template <bool XF>
__device__ __forceinline__ bool load_point(const float4* __restrict__ pts, int i, const float (&r)[12],
                                           float& x, float& y, float& z, int* status) {
    const float4 p = pts[i];
    if (XF) {
        x = fmaf(r[0], p.x, fmaf(r[1], p.y, fmaf(r[2], p.z, r[9])));
        y = fmaf(r[3], p.x, fmaf(r[4], p.y, fmaf(r[5], p.z, r[10])));
        z = fmaf(r[6], p.x, fmaf(r[7], p.y, fmaf(r[8], p.z, r[11])));
    } else {
        x = p.x;
        y = p.y;
        z = p.z;
    }
    const bool fin = isfinite(p.x) && isfinite(p.y) && isfinite(p.z);
    if (!fin) {
        if (status) atomicOr(status, ST_NONFINITE);
        x = y = z = 0.f;
    }
    return fin;
}

__device__ __forceinline__ void comp_from_smem(const float4* sc, int c, ChildRegs& r) {
    const float4 a = sc[3 * c], b = sc[3 * c + 1], d = sc[3 * c + 2];
    r.mx = a.x; r.my = a.y; r.mz = a.z; r.C = a.w;
    r.w00 = b.x; r.w10 = b.y; r.w11 = b.z; r.w20 = b.w;
    r.w21 = d.x; r.w22 = d.y;
}

// Running log2-sum-exp2 of one point over a chunk of K scores: one rescale
// of the running sum per chunk.  -inf scores (dead components) add nothing.
template <int K>
__device__ __forceinline__ void lse_chunk(const float (&s)[K], float& m, float& sum) {
    float cm = s[0];
#pragma unroll
    for (int k = 1; k < K; ++k) cm = fmaxf(cm, s[k]);
    const float nm = fmaxf(m, cm);
    const float ref = nm == -CUDART_INF_F ? 0.f : nm;
    float acc = sum * exp2f(m - ref);
#pragma unroll
    for (int k = 0; k < K; ++k) acc += exp2f(s[k] - ref);
    sum = acc;
    m = nm;
}

template <bool XF>
__global__ void __launch_bounds__(LSE_THREADS)
k_flat_lse(const float4* __restrict__ pts, int n, const float* __restrict__ Rt,
           const NodeEst* __restrict__ est, const int* __restrict__ meta, float* __restrict__ lse,
           int* __restrict__ status) {
    __shared__ float4 sc[3 * LSE_TILE];
    const int J = meta[0];
    // lane = 4 * (point group within the warp) + phase; the four lanes of a
    // group take components phase, phase + 4, ... of the same points
    const int phase = threadIdx.x % LSE_SPLIT, grp = threadIdx.x / LSE_SPLIT;
    constexpr int GROUPS = LSE_THREADS / LSE_SPLIT;
    float r[12];
    if (XF) load_rt(Rt, r);
    float zx[LSE_PPT], zy[LSE_PPT], zz[LSE_PPT], m[LSE_PPT], sum[LSE_PPT];
    bool ok[LSE_PPT];
#pragma unroll
    for (int k = 0; k < LSE_PPT; ++k) {
        const int i = blockIdx.x * LSE_POINTS + k * GROUPS + grp;
        // only phase 0 reports a non-finite point (once)
        ok[k] = i < n && load_point<XF>(pts, i < n ? i : 0, r, zx[k], zy[k], zz[k], phase == 0 ? status : nullptr);
        if (i >= n) zx[k] = zy[k] = zz[k] = 0.f;
        m[k] = -CUDART_INF_F;
        sum[k] = 0.f;
    }
    for (int j0 = 0; j0 < J; j0 += LSE_TILE) {
        const int cnt = min(LSE_TILE, J - j0);
        __syncthreads();
        const float4* src = reinterpret_cast<const float4*>(est + j0);
        for (int q = threadIdx.x; q < 3 * cnt; q += LSE_THREADS) sc[q] = src[q];
        __syncthreads();
        int c = phase;
        for (; c + 7 * LSE_SPLIT < cnt; c += 8 * LSE_SPLIT) {
            float s[LSE_PPT][8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                ChildRegs cr;
                comp_from_smem(sc, c + u * LSE_SPLIT, cr);
#pragma unroll
                for (int k = 0; k < LSE_PPT; ++k) {
                    float ex, ey, ez;
                    s[k][u] = child_score(cr, zx[k], zy[k], zz[k], ex, ey, ez);
                }
            }
#pragma unroll
            for (int k = 0; k < LSE_PPT; ++k) lse_chunk<8>(s[k], m[k], sum[k]);
        }
        for (; c < cnt; c += LSE_SPLIT) {
            ChildRegs cr;
            comp_from_smem(sc, c, cr);
#pragma unroll
            for (int k = 0; k < LSE_PPT; ++k) {
                float ex, ey, ez;
                float s1[1] = {child_score(cr, zx[k], zy[k], zz[k], ex, ey, ez)};
                lse_chunk<1>(s1, m[k], sum[k]);
            }
        }
    }
    // combine the four partial (max, sum) pairs of each point group
#pragma unroll
    for (int k = 0; k < LSE_PPT; ++k) {
#pragma unroll
        for (int o = 1; o < LSE_SPLIT; o <<= 1) {
            const float mo = __shfl_xor_sync(FULL, m[k], o);
            const float so = __shfl_xor_sync(FULL, sum[k], o);
            const float nm = fmaxf(m[k], mo);
            const float ref = nm == -CUDART_INF_F ? 0.f : nm;
            sum[k] = sum[k] * exp2f(m[k] - ref) + so * exp2f(mo - ref);
            m[k] = nm;
        }
        const int i = blockIdx.x * LSE_POINTS + k * GROUPS + grp;
        if (i < n && phase == 0) lse[i] = (ok[k] && sum[k] > 0.f) ? m[k] + log2f(sum[k]) : CUDART_INF_F;
    }
}

// Work split of one moment pass, computed on the device from the live
// component count J (the host only knows an upper bound): component tiles
// of MOM_THREADS x point slices, at most max_ctas CTAs in all.
struct FlatPlan {
    int tiles, slices, slice_len, jpad;
};

__device__ __forceinline__ FlatPlan flat_plan(int J, int n, int max_ctas) {
    FlatPlan p;
    p.tiles = J > 0 ? (J + MOM_THREADS - 1) / MOM_THREADS : 1;
    p.jpad = p.tiles * MOM_THREADS;
    const int want = max_ctas / p.tiles > 1 ? max_ctas / p.tiles : 1;
    const int most = (n + 63) / 64;
    int sl = want < most ? want : most;
    if (sl < 1) sl = 1;
    p.slice_len = (n + sl - 1) / sl;
    p.slices = (n + p.slice_len - 1) / p.slice_len;
    return p;
}

template <int NM>
__device__ __forceinline__ void fold_mom(float (&in)[NM], float (&s)[NM], float (&c)[NM]) {
#pragma unroll
    for (int v = 0; v < NM; ++v) {
        float t, e;
        two_sum(s[v], in[v], t, e);
        s[v] = t;
        c[v] += e;
        in[v] = 0.f;
    }
}

// Partial moments of components [tile*256, tile*256 + 256) over the points
// of one slice; NM = 4 (gamma, gamma e) or 10 (and gamma e e^T), e = z' - mu32.
template <int NM, bool XF>
__global__ void __launch_bounds__(MOM_THREADS)
k_flat_moments(const float4* __restrict__ pts, int n, const float* __restrict__ Rt,
               const float* __restrict__ lse, const NodeEst* __restrict__ est,
               const int* __restrict__ meta, int max_ctas, float2* __restrict__ part) {
    __shared__ float4 sp[MOM_STAGE];
    const int J = meta[0];
    const FlatPlan pl = flat_plan(J, n, max_ctas);
    const int tile = blockIdx.x % pl.tiles, slice = blockIdx.x / pl.tiles;
    if (slice >= pl.slices) return;  // uniform over the CTA
    const int slice_len = pl.slice_len, jpad = pl.jpad;
    const int j = tile * MOM_THREADS + threadIdx.x;
    const bool own = j < J;
    ChildRegs cr;
    if (own) {
        load_child(est + j, cr);
    } else {
        cr.mx = cr.my = cr.mz = 0.f;
        cr.C = -CUDART_INF_F;
        cr.w00 = cr.w10 = cr.w11 = cr.w20 = cr.w21 = cr.w22 = 0.f;
    }
    float r[12];
    if (XF) load_rt(Rt, r);
    const int i0 = slice * slice_len, i1 = min(n, i0 + slice_len);
    float in[NM], s[NM], c[NM];
#pragma unroll
    for (int v = 0; v < NM; ++v) { in[v] = 0.f; s[v] = 0.f; c[v] = 0.f; }
    auto pair = [&](const float4 p) {
        float ex, ey, ez;
        const float sc = child_score(cr, p.x, p.y, p.z, ex, ey, ez);
        const float g = exp2f(sc - p.w);
        if (NM == 4) {
            in[0] += g;
            in[1] = fmaf(g, ex, in[1]);
            in[2] = fmaf(g, ey, in[2]);
            in[3] = fmaf(g, ez, in[3]);
        } else {
            accum10(in, g, ex, ey, ez);
        }
    };
    for (int b = i0; b < i1; b += MOM_STAGE) {
        const int cnt = min(MOM_STAGE, i1 - b);
        __syncthreads();
        if (threadIdx.x < cnt) {
            const int i = b + threadIdx.x;
            float x, y, z;
            const bool fin = load_point<XF>(pts, i, r, x, y, z, nullptr);  // reported by k_flat_lse
            sp[threadIdx.x] = make_float4(x, y, z, fin ? __ldg(lse + i) : CUDART_INF_F);
        }
        __syncthreads();
        // plain FP32 sums over 16 points, then one compensated fold
        int q = 0;
        for (; q + 16 <= cnt; q += 16) {
#pragma unroll
            for (int u = 0; u < 16; ++u) pair(sp[q + u]);
            fold_mom<NM>(in, s, c);
        }
        for (; q < cnt; ++q) pair(sp[q]);
        fold_mom<NM>(in, s, c);
    }
    if (own) {
#pragma unroll
        for (int v = 0; v < NM; ++v) part[(int64_t(slice) * NM + v) * jpad + j] = make_float2(s[v], c[v]);
    }
}

// The slice partials of 32 components (one per lane) summed by a CTA of
// MOM_THREADS: warp w takes slices w, w + 8, ...; warp 0 then adds the eight
// warp sums in a fixed order.  Lane l of warp 0 returns the totals of
// component blockIdx.x * 32 + l (zero beyond J).
constexpr int RED_COMPS = 32;
constexpr int RED_WARPS = MOM_THREADS / 32;

template <int NM>
__device__ __forceinline__ void reduce_slices(const float2* __restrict__ part, const FlatPlan& pl, int J,
                                              float2 (*red)[NM][RED_COMPS], float (&S)[NM], float (&C)[NM]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = blockIdx.x * RED_COMPS + lane;
#pragma unroll
    for (int v = 0; v < NM; ++v) { S[v] = 0.f; C[v] = 0.f; }
    if (j < J) {
        for (int sl = warp; sl < pl.slices; sl += RED_WARPS) {
#pragma unroll
            for (int v = 0; v < NM; ++v) {
                const float2 x = part[(int64_t(sl) * NM + v) * pl.jpad + j];
                pair_add(S[v], C[v], x.x, x.y);
            }
        }
    }
#pragma unroll
    for (int v = 0; v < NM; ++v) red[warp][v][lane] = make_float2(S[v], C[v]);
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int v = 0; v < NM; ++v) { S[v] = 0.f; C[v] = 0.f; }
        for (int w = 0; w < RED_WARPS; ++w) {
#pragma unroll
            for (int v = 0; v < NM; ++v) pair_add(S[v], C[v], red[w][v][lane].x, red[w][v][lane].y);
        }
    }
}

// ------------------------------------------------------------ registration
__global__ void k_flat_reg_init(const double* __restrict__ T_init, double* __restrict__ T,
                                float* __restrict__ Rt, double* __restrict__ obj) {
    if (threadIdx.x == 0) {
        for (int k = 0; k < 16; ++k) T[k] = T_init ? T_init[k] : ((k % 5 == 0) ? 1.0 : 0.0);
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) Rt[r * 3 + c] = float(T[r * 4 + c]);
            Rt[9 + r] = float(T[r * 4 + 3]);
        }
        *obj = 0.0;
    }
}

__global__ void __launch_bounds__(MOM_THREADS)
k_flat_terms(const float2* __restrict__ part, int max_ctas, const int* __restrict__ meta,
             const NodeEst* __restrict__ est, const float4* __restrict__ rterm, int n,
             float2* __restrict__ tpart, double* __restrict__ dbg) {
    __shared__ float2 red[RED_WARPS][4][RED_COMPS];
    const int J = meta[0];
    if (blockIdx.x * RED_COMPS >= J) return;  // uniform over the CTA
    const FlatPlan pl = flat_plan(J, n, max_ctas);
    float S[4], C[4];
    reduce_slices<4>(part, pl, J, red, S, C);
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x, j = blockIdx.x * RED_COMPS + lane;
    float v[32], c[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) { v[k] = 0.f; c[k] = 0.f; }
    if (j < J) {
        const float4 cm = est[j].a;
        const float M0 = S[0] + C[0];
        float o0 = 0.f, o1 = 0.f, o2 = 0.f;
        if (M0 > 0.f) {
            const float inv = 1.0f / M0;
            o0 = (S[1] + C[1]) * inv;
            o1 = (S[2] + C[2]) * inv;
            o2 = (S[3] + C[3]) * inv;
            float w[NTERM];
            node_terms(rterm[3 * j], rterm[3 * j + 1], rterm[3 * j + 2], cm, M0, o0, o1, o2, M0 / float(n), w);
#pragma unroll
            for (int k = 0; k < NTERM; ++k) pair_add(v[k], c[k], w[k], 0.f);
        }
        dbg[4 * j + 0] = double(M0);
        dbg[4 * j + 1] = double(M0) * (double(cm.x) + double(o0));
        dbg[4 * j + 2] = double(M0) * (double(cm.y) + double(o1));
        dbg[4 * j + 3] = double(M0) * (double(cm.z) + double(o2));
    }
    float ws, we;
    warp_reduce_scatter32(v, c, ws, we);
    if (lane < NTERM) tpart[NTERM * blockIdx.x + lane] = make_float2(ws, we);
}

__global__ void __launch_bounds__(MOM_THREADS)
k_flat_solve(const float2* __restrict__ tpart, const int* __restrict__ meta, int it,
             double* __restrict__ T, float* __restrict__ Rt, double* __restrict__ T_hist,
             double* __restrict__ obj, int* __restrict__ status) {
    sum_terms_and_solve(tpart, (meta[0] + RED_COMPS - 1) / RED_COMPS, it, T, Rt, T_hist, obj, status);
}

__global__ void k_flat_copy_T(const double* __restrict__ T, double* __restrict__ out) {
    if (threadIdx.x < 16) out[threadIdx.x] = T[threadIdx.x];
}

// ------------------------------------------------------------------ EM fit
// M-step of component j from its 10 moments (centred on its FP32 mean):
// S0, d = S1 / S0, Sigma = S2 / S0 - d d^T + eps I, pi = S0 / n; a component
// below n_min expected points dies and keeps its parameters.
__global__ void __launch_bounds__(MOM_THREADS)
k_flat_mstep(const float2* __restrict__ part, int max_ctas, const int* __restrict__ meta, int n,
             float n_min, const double* __restrict__ eps_p, FlatComp* __restrict__ comp,
             NodeEst* __restrict__ est, int* __restrict__ status) {
    __shared__ float2 red[RED_WARPS][10][RED_COMPS];
    const int J = meta[0];
    if (blockIdx.x * RED_COMPS >= J) return;  // uniform over the CTA
    const FlatPlan pl = flat_plan(J, n, max_ctas);
    float Sf[10], Cf[10];
    reduce_slices<10>(part, pl, J, red, Sf, Cf);
    const int j = blockIdx.x * RED_COMPS + threadIdx.x;
    if (threadIdx.x >= 32 || j >= J) return;
    double m[10];
    for (int v = 0; v < 10; ++v) m[v] = double(Sf[v]) + double(Cf[v]);
    FlatComp& f = comp[j];
    NodeEst& e = est[j];
    const double S0 = m[0];
    if (!(f.live && S0 >= double(n_min) && S0 > 0.0)) {
        f.live = 0;
        f.pi = 0.0;
        dead_est(f.mu, e);
        return;
    }
    const double eps = *eps_p;
    const double inv = rcp_f64(S0);
    const double d[3] = {m[1] * inv, m[2] * inv, m[3] * inv};
    const double mu[3] = {double(e.a.x) + d[0], double(e.a.y) + d[1], double(e.a.z) + d[2]};
    double S[6];
    S[0] = m[4] * inv - d[0] * d[0] + eps;
    S[1] = m[5] * inv - d[0] * d[1];
    S[2] = m[6] * inv - d[0] * d[2];
    S[3] = m[7] * inv - d[1] * d[1] + eps;
    S[4] = m[8] * inv - d[1] * d[2];
    S[5] = m[9] * inv - d[2] * d[2] + eps;
    f.pi = S0 / double(n);
    for (int a = 0; a < 3; ++a) f.mu[a] = mu[a];
    for (int v = 0; v < 6; ++v) f.S[v] = S[v];
    if (!pack_est(f.pi, f.mu, f.S, eps, 0.f, e)) atomicOr(status, ST_CHOL);
}

// Eigen-decomposition, precision matrix and FP32 registration constants of
// every component after a fit.
__global__ void __launch_bounds__(MOM_THREADS)
k_flat_finalize(const int* __restrict__ meta, const double* __restrict__ eps_p, FlatComp* __restrict__ comp,
                const NodeEst* __restrict__ est, float4* __restrict__ rterm) {
    const int J = meta[0];
    const int j = blockIdx.x * MOM_THREADS + threadIdx.x;
    if (j >= J) return;
    FlatComp& f = comp[j];
    if (!f.live) {
        for (int v = 0; v < 6; ++v) f.P[v] = 0.0;
        rterm[3 * j] = rterm[3 * j + 1] = rterm[3 * j + 2] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    double lam[3], V[9];
    eig3(f.S, lam, V);
    const double eps = *eps_p;
    double il[3];
    for (int a = 0; a < 3; ++a) {
        f.lam[a] = lam[a];
        il[a] = rcp_f64(fmax(lam[a], eps));
    }
    for (int v = 0; v < 9; ++v) f.V[v] = V[v];
    const int ij[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    for (int v = 0; v < 6; ++v) {
        const int r = ij[v][0], c = ij[v][1];
        double acc = 0.0;
        for (int k = 0; k < 3; ++k) acc += V[r * 3 + k] * il[k] * V[c * 3 + k];
        f.P[v] = acc;
    }
    const float4 a = est[j].a;
    rterm[3 * j] = make_float4(float(f.P[0]), float(f.P[1]), float(f.P[2]), float(f.P[3]));
    rterm[3 * j + 1] = make_float4(float(f.P[4]), float(f.P[5]), 0.f, 0.f);
    rterm[3 * j + 2] = make_float4(float(f.mu[0] - double(a.x)), float(f.mu[1] - double(a.y)),
                                   float(f.mu[2] - double(a.z)), 0.f);
}

}  // namespace
}  // namespace hgmm

using namespace hgmm;

struct hgmm_flat {
    int device = 0;
    int n_sm = 0;
    int64_t cap = 0;
    int cap_comp = 0;
    int jcap = 0;          // upper bound of J since the last hgmm_flat_from_tree
    bool have = false;
    int max_ctas = 0;      // moment CTAs per pass (slices x component tiles)
    FlatComp* comp = nullptr;
    NodeEst* est = nullptr;
    float4* rterm = nullptr;
    int* meta = nullptr;
    double* eps = nullptr;
    float* lse = nullptr;
    float2* part = nullptr;
    float2* tpart = nullptr;
    double* T = nullptr;
    float* Rt = nullptr;
    double* obj = nullptr;
    double* dbg = nullptr;
    int* status = nullptr;
};

namespace {

void free_flat(hgmm_flat* f) {
    if (!f) return;
    void* ptrs[] = {f->comp, f->est, f->rterm, f->meta, f->eps, f->lse, f->part, f->tpart,
                    f->T, f->Rt, f->obj, f->dbg, f->status};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete f;
}

template <typename T>
bool falloc(T** p, size_t count) {
    *p = nullptr;
    return cudaMalloc(reinterpret_cast<void**>(p), (count ? count : 1) * sizeof(T)) == cudaSuccess;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool on_device(const hgmm_flat* f) {
    int cur = -1;
    return cudaGetDevice(&cur) == cudaSuccess && cur == f->device;
}

// Grid of a moment pass: enough CTAs for the device-side plan of any J up
// to the bound (max_ctas, or more tiles than that at one slice each).
int moment_grid(const hgmm_flat* f) {
    const int tiles = (f->jcap + MOM_THREADS - 1) / MOM_THREADS;
    return tiles > f->max_ctas ? tiles : f->max_ctas;
}

int launched() { return cudaGetLastError() == cudaSuccess ? HGMM_OK : HGMM_ECUDA; }

}  // namespace

extern "C" {

int hgmm_flat_create(int64_t max_points, int32_t max_components, hgmm_flat** out) {
    if (!out || max_points < 1 || max_points > (int64_t(1) << 30) || max_components < 1) return HGMM_EINVAL;
    *out = nullptr;
    hgmm_flat* f = new hgmm_flat();
    cudaGetDevice(&f->device);
    cudaDeviceGetAttribute(&f->n_sm, cudaDevAttrMultiProcessorCount, f->device);
    f->cap = max_points;
    f->cap_comp = max_components;
    f->max_ctas = 4 * (f->n_sm > 0 ? f->n_sm : 1);
    const int tiles_max = (max_components + MOM_THREADS - 1) / MOM_THREADS;
    const size_t part_ctas = size_t(f->max_ctas > tiles_max ? f->max_ctas : tiles_max);
    const bool good = falloc(&f->comp, max_components) && falloc(&f->est, max_components) &&
                      falloc(&f->rterm, 3 * size_t(max_components)) && falloc(&f->meta, 4) &&
                      falloc(&f->eps, 1) && falloc(&f->lse, size_t(max_points)) &&
                      falloc(&f->part, part_ctas * MOM_THREADS * NMOM_MAX) &&
                      falloc(&f->tpart, size_t((max_components + RED_COMPS - 1) / RED_COMPS) * NTERM) && falloc(&f->T, 16) && falloc(&f->Rt, 12) &&
                      falloc(&f->obj, 1) && falloc(&f->dbg, 4 * size_t(max_components)) &&
                      falloc(&f->status, 1);
    if (!good || cudaMemset(f->status, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(f->meta, 0, 4 * sizeof(int)) != cudaSuccess || cudaMemset(f->obj, 0, sizeof(double)) != cudaSuccess) {
        free_flat(f);
        cudaGetLastError();
        return HGMM_ENOMEM;
    }
    *out = f;
    return HGMM_OK;
}

void hgmm_flat_destroy(hgmm_flat* f) { free_flat(f); }

int hgmm_flat_from_tree(hgmm_flat* f, const hgmm_tree* t, int32_t level, void* stream) {
    if (!f || !t || !t->built || !on_device(f) || t->device != f->device) return HGMM_EINVAL;
    if (level < -1 || level >= t->depth) return HGMM_EINVAL;
    const int L = level < 0 ? t->depth : level + 1;
    const int64_t n_cand = level_offset(L);
    if (n_cand > f->cap_comp) return HGMM_ECAPACITY;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_flat_from_tree<<<1, FROM_TREE_THREADS, 0, s>>>(t->stat, t->root, L, int(n_cand), f->comp, f->est,
                                                    f->rterm, f->meta, f->eps, f->status);
    f->jcap = int(n_cand);
    f->have = true;
    return launched();
}

int hgmm_flat_fit(hgmm_flat* f, const float* d_points, int64_t n, int32_t em_iters, float n_min, void* stream) {
    if (!f || !f->have || !d_points || n < 1 || em_iters < 0 || !aligned16(d_points) || !on_device(f))
        return HGMM_EINVAL;
    if (n > f->cap) return HGMM_ECAPACITY;
    if (em_iters == 0) return HGMM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float4* pts = reinterpret_cast<const float4*>(d_points);
    const int tiles = (f->jcap + MOM_THREADS - 1) / MOM_THREADS;
    const int rgrid = (f->jcap + RED_COMPS - 1) / RED_COMPS;
    const int mgrid = moment_grid(f);
    const int lse_grid = int((n + LSE_POINTS - 1) / LSE_POINTS);
    for (int it = 0; it < em_iters; ++it) {
        k_flat_lse<false><<<lse_grid, LSE_THREADS, 0, s>>>(pts, int(n), nullptr, f->est, f->meta, f->lse, f->status);
        k_flat_moments<10, false><<<mgrid, MOM_THREADS, 0, s>>>(pts, int(n), nullptr, f->lse, f->est, f->meta,
                                                               mgrid, f->part);
        k_flat_mstep<<<rgrid, MOM_THREADS, 0, s>>>(f->part, mgrid, f->meta, int(n), n_min, f->eps, f->comp,
                                                   f->est, f->status);
    }
    k_flat_finalize<<<tiles, MOM_THREADS, 0, s>>>(f->meta, f->eps, f->comp, f->est, f->rterm);
    return launched();
}

int hgmm_flat_register(hgmm_flat* f, const float* d_src, int64_t n, const double* d_T_init, int32_t iters,
                       void* stream, double* d_T_out, double* d_T_hist) {
    if (!f || !f->have || !d_src || n < 1 || iters < 0 || !aligned16(d_src) || !on_device(f)) return HGMM_EINVAL;
    if (n > f->cap) return HGMM_ECAPACITY;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float4* pts = reinterpret_cast<const float4*>(d_src);
    const int rgrid = (f->jcap + RED_COMPS - 1) / RED_COMPS;
    const int mgrid = moment_grid(f);
    const int lse_grid = int((n + LSE_POINTS - 1) / LSE_POINTS);
    k_flat_reg_init<<<1, 32, 0, s>>>(d_T_init, f->T, f->Rt, f->obj);
    for (int it = 0; it < iters; ++it) {
        k_flat_lse<true><<<lse_grid, LSE_THREADS, 0, s>>>(pts, int(n), f->Rt, f->est, f->meta, f->lse, f->status);
        k_flat_moments<4, true><<<mgrid, MOM_THREADS, 0, s>>>(pts, int(n), f->Rt, f->lse, f->est, f->meta, mgrid,
                                                             f->part);
        k_flat_terms<<<rgrid, MOM_THREADS, 0, s>>>(f->part, mgrid, f->meta, f->est, f->rterm, int(n),
                                                   f->tpart, f->dbg);
        k_flat_solve<<<1, MOM_THREADS, 0, s>>>(f->tpart, f->meta, it, f->T, f->Rt, d_T_hist, f->obj, f->status);
    }
    if (d_T_out) k_flat_copy_T<<<1, 32, 0, s>>>(f->T, d_T_out);
    return launched();
}

int hgmm_flat_objective(const hgmm_flat* f, double* d_obj, void* stream) {
    if (!f || !d_obj) return HGMM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(d_obj, f->obj, sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return HGMM_ECUDA;
    return HGMM_OK;
}

int hgmm_flat_export(hgmm_flat* f, double* h_out, int64_t cap, int32_t* h_count, int32_t* h_node) {
    if (!f || !h_count || (cap > 0 && !h_out) || cap < 0) return HGMM_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) return HGMM_ECUDA;
    int J = 0;
    if (cudaMemcpy(&J, f->meta, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HGMM_ECUDA;
    *h_count = J;
    const int64_t m = J < cap ? J : cap;
    if (m > 0) {
        FlatComp* hc = new FlatComp[m];
        if (cudaMemcpy(hc, f->comp, size_t(m) * sizeof(FlatComp), cudaMemcpyDeviceToHost) != cudaSuccess) {
            delete[] hc;
            return HGMM_ECUDA;
        }
        for (int64_t j = 0; j < m; ++j) {
            double* o = h_out + 10 * j;
            o[0] = hc[j].live ? hc[j].pi : 0.0;
            for (int a = 0; a < 3; ++a) o[1 + a] = hc[j].mu[a];
            for (int v = 0; v < 6; ++v) o[4 + v] = hc[j].S[v];
            if (h_node) {
                h_node[2 * j] = hc[j].level;
                h_node[2 * j + 1] = hc[j].index;
            }
        }
        delete[] hc;
    }
    return HGMM_OK;
}

int hgmm_flat_debug_moments(hgmm_flat* f, double* h_out, int64_t cap, int32_t* h_count) {
    if (!f || !h_out || !h_count || cap < 0) return HGMM_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) return HGMM_ECUDA;
    int J = 0;
    if (cudaMemcpy(&J, f->meta, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HGMM_ECUDA;
    *h_count = J;
    const int64_t m = J < cap ? J : cap;
    if (m > 0 && cudaMemcpy(h_out, f->dbg, size_t(m) * 4 * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        return HGMM_ECUDA;
    return HGMM_OK;
}

int hgmm_flat_sync(hgmm_flat* f, void* stream) {
    if (!f) return HGMM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int st = 0;
    if (cudaMemcpyAsync(&st, f->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return HGMM_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return HGMM_ECUDA;
    if (st) {
        const int zero = 0;
        if (cudaMemcpy(f->status, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return HGMM_ECUDA;
    }
    if (st & ST_NONFINITE) return HGMM_ENONFINITE;
    if (st & ST_DEGENERATE) return HGMM_EDEGENERATE;
    return HGMM_OK;
}

}  // extern "C"
