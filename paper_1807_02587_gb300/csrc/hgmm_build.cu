// GMM-tree build on the GPU (the model construction Sec. 3 takes from its
// reference [33]; 8-component nodes, Sec. 4.1).
//
// Per level l (children = the 8^(l+1) nodes of level l, parents = level l-1
// or the root):
//   k_init_children   PCA-octant initial children of every parent (FP64 eigen)
//   k_make_items      split each parent's contiguous point segment into work
//                     items of <= TILE points, laid out parent by parent
//   K x ( k_estep     per point: Eq. 3 posteriors over the 8 children of its
//                     parent (FP32, log2 domain, max-subtracted exp2) and the
//                     gamma-weighted moments S0, S1, S2 of every child,
//                     centred on the child's current mean; compensated sums;
//                     one partial per (CTA, parent) run
//    + k_mstep        per parent: fixed-order reduction of its runs, FP64
//                     M-step and Cholesky, dead-child rule, new FP32 E-step
//                     constants )
//   k_assign          argmax hand-off (ties -> lowest index) with in-item ranks
//   k_child_offsets   per parent: child segment starts and per-item offsets
//   k_scatter         stable 8-way partition of every parent's segment
//   k_finalize        FP64 eigen, complexity, precision matrix of level l
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "hgmm_internal.cuh"
#include "hgmm_math.cuh"

namespace hgmm {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int64_t d_level_offset(int l) {
    return ((int64_t(1) << (3 * (l + 1))) - 8) / 7;
}

// ---------------------------------------------------------------- root stats
// Whole-cloud mean, covariance and bounding box (the root of the tree, whose
// children are Children(-1) of Algorithm 1).  Sums of (z - z0) and
// (z - z0)(z - z0)^T with z0 = the first point, FP32 with compensated
// accumulation.  Each CTA writes a partial (32 floats: [0..17] 9 (sum, err)
// pairs, [18..20] min, [21..23] max, [24] non-finite count); the last CTA to
// finish reduces them in a fixed order and writes the FP64 root record.
__device__ __forceinline__ void root_combine(float* f, const float* o) {
#pragma unroll
    for (int v = 0; v < 9; ++v) pair_add(f[2 * v], f[2 * v + 1], o[2 * v], o[2 * v + 1]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        f[18 + a] = fminf(f[18 + a], o[18 + a]);
        f[21 + a] = fmaxf(f[21 + a], o[21 + a]);
    }
    f[24] = __int_as_float(__float_as_int(f[24]) + __float_as_int(o[24]));
}

__device__ __forceinline__ void root_identity(float* f) {
#pragma unroll
    for (int v = 0; v < 18; ++v) f[v] = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) { f[18 + a] = CUDART_INF_F; f[21 + a] = -CUDART_INF_F; }
    f[24] = __int_as_float(0);
}

__global__ void __launch_bounds__(256) k_root(const float4* __restrict__ pts, int n,
                                              float eps_rel, float* __restrict__ part,
                                              unsigned* __restrict__ counter,
                                              RootDev* __restrict__ root, int* __restrict__ status) {
    __shared__ float sm[8][25];
    __shared__ bool last;
    const float4 z0 = pts[0];
    float in[9] = {}, s[9] = {}, c[9] = {};
    float mn[3] = {CUDART_INF_F, CUDART_INF_F, CUDART_INF_F};
    float mx[3] = {-CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F};
    int bad = 0, cnt = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 z = pts[i];
        if (!(isfinite(z.x) && isfinite(z.y) && isfinite(z.z))) {
            ++bad;
            continue;
        }
        const float dx = z.x - z0.x, dy = z.y - z0.y, dz = z.z - z0.z;
        in[0] += dx; in[1] += dy; in[2] += dz;
        in[3] = fmaf(dx, dx, in[3]); in[4] = fmaf(dx, dy, in[4]); in[5] = fmaf(dx, dz, in[5]);
        in[6] = fmaf(dy, dy, in[6]); in[7] = fmaf(dy, dz, in[7]); in[8] = fmaf(dz, dz, in[8]);
        mn[0] = fminf(mn[0], z.x); mn[1] = fminf(mn[1], z.y); mn[2] = fminf(mn[2], z.z);
        mx[0] = fmaxf(mx[0], z.x); mx[1] = fmaxf(mx[1], z.y); mx[2] = fmaxf(mx[2], z.z);
        if (++cnt == 16) {
#pragma unroll
            for (int v = 0; v < 9; ++v) { pair_add(s[v], c[v], in[v], 0.f); in[v] = 0.f; }
            cnt = 0;
        }
    }
#pragma unroll
    for (int v = 0; v < 9; ++v) pair_add(s[v], c[v], in[v], 0.f);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int v = 0; v < 9; ++v) {
            const float s2 = __shfl_xor_sync(FULL, s[v], off);
            const float c2 = __shfl_xor_sync(FULL, c[v], off);
            pair_add(s[v], c[v], s2, c2);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(FULL, mn[a], off));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(FULL, mx[a], off));
        }
        bad += __shfl_xor_sync(FULL, bad, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        for (int v = 0; v < 9; ++v) { sm[warp][2 * v] = s[v]; sm[warp][2 * v + 1] = c[v]; }
        for (int a = 0; a < 3; ++a) { sm[warp][18 + a] = mn[a]; sm[warp][21 + a] = mx[a]; }
        sm[warp][24] = __int_as_float(bad);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float f[25];
        root_identity(f);
        for (int w = 0; w < 8; ++w) root_combine(f, sm[w]);
        float* o = part + 32 * blockIdx.x;
        for (int v = 0; v < 25; ++v) o[v] = f[v];
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // last CTA: 16 half-warp groups each reduce every 16th partial (lane i of
    // a group owns item i: 9 (sum, err) pairs, 3 min, 3 max, count), then one
    // thread combines the 16 group results in order
    __shared__ float gs[16][25];
    {
        const int grp = threadIdx.x >> 4, it = threadIdx.x & 15;
        float a = 0.f, b = 0.f;
        if (it >= 9 && it < 12) a = CUDART_INF_F;
        if (it >= 12 && it < 15) a = -CUDART_INF_F;
        int cntb = 0;
#pragma unroll 4
        for (int blk = grp; blk < (int)gridDim.x; blk += 16) {
            const float* o = part + 32 * blk;
            if (it < 9) pair_add(a, b, __ldcg(o + 2 * it), __ldcg(o + 2 * it + 1));
            else if (it < 12) a = fminf(a, __ldcg(o + 18 + it - 9));
            else if (it < 15) a = fmaxf(a, __ldcg(o + 21 + it - 12));
            else cntb += __float_as_int(__ldcg(o + 24));
        }
        if (it < 9) { gs[grp][2 * it] = a; gs[grp][2 * it + 1] = b; }
        else if (it < 12) gs[grp][18 + it - 9] = a;
        else if (it < 15) gs[grp][21 + it - 12] = a;
        else gs[grp][24] = __int_as_float(cntb);
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    float F[25];
    root_identity(F);
    for (int w = 0; w < 16; ++w) root_combine(F, gs[w]);
    *counter = 0u;
    if (__float_as_int(F[24]) > 0) atomicOr(status, ST_NONFINITE);
    const double nn = double(n);
    double m1[3], m2[6];
    for (int a = 0; a < 3; ++a) m1[a] = (double(F[2 * a]) + double(F[2 * a + 1])) / nn;
    for (int v = 0; v < 6; ++v) m2[v] = (double(F[6 + 2 * v]) + double(F[7 + 2 * v])) / nn;
    root->n = nn;
    root->mu[0] = double(z0.x) + m1[0];
    root->mu[1] = double(z0.y) + m1[1];
    root->mu[2] = double(z0.z) + m1[2];
    double S[6];
    S[0] = m2[0] - m1[0] * m1[0];
    S[1] = m2[1] - m1[0] * m1[1];
    S[2] = m2[2] - m1[0] * m1[2];
    S[3] = m2[3] - m1[1] * m1[1];
    S[4] = m2[4] - m1[1] * m1[2];
    S[5] = m2[5] - m1[2] * m1[2];
    for (int v = 0; v < 6; ++v) root->S[v] = S[v];
    double e2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double d = double(F[21 + a]) - double(F[18 + a]);
        e2 += d * d;
    }
    root->extent = sqrt(e2);
    const double e = double(eps_rel) * root->extent;
    root->eps = e * e;
    eig3(S, root->lam, root->V);
}

// ---------------------------------------------------------------- init
// One CTA per parent; threads 0..7 build child c.
__global__ void k_init_children(int level, const RootDev* __restrict__ root,
                                NodeStat* __restrict__ stat, NodeEst* __restrict__ est,
                                const int* __restrict__ seg_count, int* __restrict__ status) {
    __shared__ double lam[3], V[9], mu_p[3], S_p[6];
    __shared__ int alive;
    const int p = blockIdx.x;
    const int64_t child0 = d_level_offset(level) + 8 * int64_t(p);
    if (threadIdx.x == 0) {
        // the parent's eigen-decomposition was computed when it was finalised
        if (level == 0) {
            for (int a = 0; a < 3; ++a) { mu_p[a] = root->mu[a]; lam[a] = root->lam[a]; }
            for (int v = 0; v < 6; ++v) S_p[v] = root->S[v];
            for (int v = 0; v < 9; ++v) V[v] = root->V[v];
            alive = 1;
        } else {
            const int64_t g = d_level_offset(level - 1) + p;
            const NodeStat& ps = stat[g];
            for (int a = 0; a < 3; ++a) { mu_p[a] = ps.mu[a]; lam[a] = ps.lam[a]; }
            for (int v = 0; v < 6; ++v) S_p[v] = ps.S[v];
            for (int v = 0; v < 9; ++v) V[v] = ps.V[v];
            alive = (ps.live && seg_count[g] > 0) ? 1 : 0;
        }
    }
    __syncthreads();
    const int c = threadIdx.x;
    if (c >= 8) return;
    NodeStat& cs = stat[child0 + c];
    NodeEst& ce = est[child0 + c];
    if (!alive) {
        cs.live = 0;
        cs.pi = 0.0;
        for (int a = 0; a < 3; ++a) cs.mu[a] = mu_p[a];
        for (int v = 0; v < 6; ++v) cs.S[v] = 0.0;
        dead_est(mu_p, ce);
        return;
    }
    const double eps = root->eps;
    double mu[3];
    for (int a = 0; a < 3; ++a) {
        double acc = mu_p[a];
        for (int b = 0; b < 3; ++b) {
            const double sgn = ((c >> b) & 1) ? 1.0 : -1.0;
            const double lb = fmax(lam[b], 0.0);
            acc += sgn * 0.5 * (lb > 0.0 ? lb * rsqrt_f64(lb) : 0.0) * V[a * 3 + b];
        }
        mu[a] = acc;
    }
    double S[6];
    for (int v = 0; v < 6; ++v) S[v] = S_p[v] * 0.25;
    S[0] += eps; S[3] += eps; S[5] += eps;
    cs.live = 1;
    cs.pi = 0.125;
    for (int a = 0; a < 3; ++a) cs.mu[a] = mu[a];
    for (int v = 0; v < 6; ++v) cs.S[v] = S[v];
    if (!pack_est(0.125, mu, S, eps, 0.f, ce)) atomicOr(status, ST_CHOL);
}

// ---------------------------------------------------------------- items
// Single CTA of 1024 threads: exclusive scan over parents of their item counts.
__global__ void __launch_bounds__(1024) k_make_items(int level, int n, int n_parents,
                                                     const int* __restrict__ seg_start,
                                                     const int* __restrict__ seg_count,
                                                     const NodeStat* __restrict__ stat,
                                                     Item* __restrict__ items,
                                                     int* __restrict__ item_range,
                                                     int* __restrict__ meta, int est_grid) {
    __shared__ int warp_tot[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int64_t poff = level == 0 ? 0 : d_level_offset(level - 1);
    for (int base = 0; base < n_parents; base += blockDim.x) {
        const int p = base + threadIdx.x;
        int count = 0;
        if (p < n_parents) {
            // every parent segment that holds points gets items, live or not:
            // points under a leaf parent (no live children) are carried down on
            // its first child's segment with zero posteriors
            count = level == 0 ? n : seg_count[poff + p];
        }
        const int k = (count + TILE - 1) / TILE;
        // block exclusive scan of k
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        int x = k;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(FULL, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(FULL, w, off);
                if (lane >= off) w += y;
            }
            warp_tot[lane] = w;  // inclusive
        }
        __syncthreads();
        const int excl = carry + (warp ? warp_tot[warp - 1] : 0) + x - k;
        if (p < n_parents) {
            item_range[2 * p] = excl;
            item_range[2 * p + 1] = excl + k;
            // the item list itself is written in parallel by k_fill_items
        }
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_tot[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // items per E-step CTA (contiguous chunks, so a parent's runs are few)
        meta[0] = carry;
        meta[1] = max(1, (carry + est_grid - 1) / est_grid);
    }
}

// One thread per item: locate its parent (largest p with begin(p) <= j; an
// empty parent shares its begin with the next one, which owns j) and write it.
__global__ void k_fill_items(int level, int n, int n_parents, const int* __restrict__ seg_start,
                             const int* __restrict__ seg_count,
                             const int* __restrict__ item_range, const int* __restrict__ meta,
                             Item* __restrict__ items) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= meta[0]) return;
    int lo = 0, hi = n_parents - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (item_range[2 * mid] <= j) lo = mid;
        else hi = mid - 1;
    }
    const int p = lo;
    const int r = j - item_range[2 * p];
    int start = 0, count = n;
    if (level > 0) {
        const int64_t g = d_level_offset(level - 1) + p;
        start = seg_start[g];
        count = seg_count[g];
    }
    Item it;
    it.parent = p;
    it.start = start + r * TILE;
    it.count = min(TILE, count - r * TILE);
    it.pad = 0;
    items[j] = it;
}

// ---------------------------------------------------------------- M-step
// M-step of parent p (Sec. 3 EM on the parent's points): reduce the parent's
// run partials in a fixed order (8 warps over the runs, then in order),
// then threads 0..7 build child c in FP64: S0, mean shift d = S1/S0 from the
// FP32 mean the E-step used, Sigma = S2/S0 - d d^T + eps I, pi = S0 / n_p;
// a child below n_min expected points dies (a parent whose children all die
// stays a leaf).  Runs with 256 threads.
struct MstepSmem {
    double mom[NPART];
    float2 grp[8][NPART];
};

template <bool COMP>
__device__ void mstep_parent(int level, int n, int p, int i0, int i1, int C,
                             const float2* __restrict__ partials,
                             const int* __restrict__ seg_count, const RootDev* __restrict__ root,
                             float n_min, NodeStat* __restrict__ stat,
                             NodeEst* __restrict__ est, int* __restrict__ status, MstepSmem& sm) {
    const int nruns = (i1 - 1) / C - i0 / C + 1;
    {
        // warp w sums runs w, w+8, ...; lane l owns values l, l+32, l+64
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int nw = blockDim.x >> 5;
        float S[3] = {0.f, 0.f, 0.f}, Cc[3] = {0.f, 0.f, 0.f};
        for (int r0 = warp; r0 < nruns; r0 += 4 * nw) {
            float2 x[4][3];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int r = r0 + u * nw;
                const int slot = r == 0 ? i0 : (i0 / C + r) * C;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const int v = lane + 32 * j;
                    x[u][j] = (r < nruns && v < NPART)
                                  ? __ldcg(&partials[int64_t(slot) * NPART + v])
                                  : make_float2(0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    if (COMP) pair_add(S[j], Cc[j], x[u][j].x, x[u][j].y);
                    else S[j] += x[u][j].x;
                }
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int v = lane + 32 * j;
            if (v < NPART) sm.grp[warp][v] = make_float2(S[j], Cc[j]);
        }
    }
    __syncthreads();
    if (threadIdx.x < NPART) {
        float S = 0.f, Cc = 0.f;
        for (int q = 0; q < int(blockDim.x >> 5); ++q) {
            if (COMP) pair_add(S, Cc, sm.grp[q][threadIdx.x].x, sm.grp[q][threadIdx.x].y);
            else S += sm.grp[q][threadIdx.x].x;
        }
        sm.mom[threadIdx.x] = double(S) + double(Cc);
    }
    __syncthreads();
    const int cidx = threadIdx.x;
    if (cidx < 8) {
        const int64_t g = d_level_offset(level) + 8 * int64_t(p) + cidx;
        NodeStat& cs = stat[g];
        NodeEst& ce = est[g];
        const double* m = sm.mom + cidx * NMOM;
        const double S0 = m[0];
        const double n_p = level == 0 ? double(n) : double(seg_count[d_level_offset(level - 1) + p]);
        const bool live = cs.live && S0 >= double(n_min) && S0 > 0.0;
        if (!live) {
            cs.live = 0;
            cs.pi = 0.0;
            ce.a.w = -CUDART_INF_F;
            ce.b = make_float4(0.f, 0.f, 0.f, 0.f);
            ce.c.x = 0.f;
            ce.c.y = 0.f;
        } else {
            const double eps = root->eps;
            const double inv = rcp_f64(S0);
            const double d[3] = {m[1] * inv, m[2] * inv, m[3] * inv};
            const double mu[3] = {double(ce.a.x) + d[0], double(ce.a.y) + d[1], double(ce.a.z) + d[2]};
            double S[6];
            S[0] = m[4] * inv - d[0] * d[0] + eps;
            S[1] = m[5] * inv - d[0] * d[1];
            S[2] = m[6] * inv - d[0] * d[2];
            S[3] = m[7] * inv - d[1] * d[1] + eps;
            S[4] = m[8] * inv - d[1] * d[2];
            S[5] = m[9] * inv - d[2] * d[2] + eps;
            const double pi = S0 * rcp_f64(n_p);
            cs.pi = pi;
            for (int a = 0; a < 3; ++a) cs.mu[a] = mu[a];
            for (int v = 0; v < 6; ++v) cs.S[v] = S[v];
            if (!pack_est(pi, mu, S, eps, 0.f, ce)) atomicOr(status, ST_CHOL);
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- E-step
// Lane layout: a quad of 4 lanes handles one point, lane k of the quad owns
// children 2k and 2k+1 (their constants live in registers); a warp handles 8
// points per step, the CTA 64.  Each lane accumulates the 10 moments of its
// two children: plain FP32 over up to 16 points, then folded into a
// compensated (sum, error) pair.
struct ChildRegs {
    float mx, my, mz, C, w00, w10, w11, w20, w21, w22;
};

__device__ __forceinline__ void load_child(const NodeEst* __restrict__ e, ChildRegs& r) {
    const float4 a = e->a, b = e->b, c = e->c;
    r.mx = a.x; r.my = a.y; r.mz = a.z; r.C = a.w;
    r.w00 = b.x; r.w10 = b.y; r.w11 = b.z; r.w20 = b.w;
    r.w21 = c.x; r.w22 = c.y;
}

// log2(pi N(z | child)) and the centred offset e = z - mu.
__device__ __forceinline__ float child_score(const ChildRegs& r, float zx, float zy, float zz,
                                             float& ex, float& ey, float& ez) {
    ex = zx - r.mx;
    ey = zy - r.my;
    ez = zz - r.mz;
    const float d0 = r.w00 * ex;
    const float d1 = fmaf(r.w11, ey, r.w10 * ex);
    const float d2 = fmaf(r.w22, ez, fmaf(r.w21, ey, r.w20 * ex));
    float s = fmaf(-d0, d0, r.C);
    s = fmaf(-d1, d1, s);
    s = fmaf(-d2, d2, s);
    return s;
}

__device__ __forceinline__ void accum10(float* a, float g, float ex, float ey, float ez) {
    const float gx = g * ex, gy = g * ey, gz = g * ez;
    a[0] += g;
    a[1] += gx;
    a[2] += gy;
    a[3] += gz;
    a[4] = fmaf(gx, ex, a[4]);
    a[5] = fmaf(gx, ey, a[5]);
    a[6] = fmaf(gx, ez, a[6]);
    a[7] = fmaf(gy, ey, a[7]);
    a[8] = fmaf(gy, ez, a[8]);
    a[9] = fmaf(gz, ez, a[9]);
}

template <bool COMP>
__device__ __forceinline__ void fold20(float* in, float* s, float* c) {
#pragma unroll
    for (int v = 0; v < 20; ++v) {
        if (COMP) {
            float t, e;
            two_sum(s[v], in[v], t, e);
            s[v] = t;
            c[v] += e;
        } else {
            s[v] += in[v];
        }
        in[v] = 0.f;
    }
}

// Block-wide reduction of the (s, c) accumulators into partial slot `run`.
template <bool COMP>
__device__ __forceinline__ void flush_run(float* s, float* c, float2 (*red)[NPART],
                                          float2* __restrict__ out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, k = lane & 3;
#pragma unroll
    for (int off = 4; off < 32; off <<= 1) {
#pragma unroll
        for (int v = 0; v < 20; ++v) {
            const float s2 = __shfl_xor_sync(FULL, s[v], off);
            const float c2 = __shfl_xor_sync(FULL, c[v], off);
            if (COMP) pair_add(s[v], c[v], s2, c2);
            else s[v] += s2;
        }
    }
    if (lane < 4) {
#pragma unroll
        for (int v = 0; v < 20; ++v) red[warp][k * 20 + v] = make_float2(s[v], COMP ? c[v] : 0.f);
    }
    __syncthreads();
    if (threadIdx.x < NPART) {
        float S = 0.f, Cc = 0.f;
        for (int w = 0; w < EST_THREADS / 32; ++w) {
            const float2 x = red[w][threadIdx.x];
            if (COMP) pair_add(S, Cc, x.x, x.y);
            else S += x.x;
        }
        out[threadIdx.x] = make_float2(S, Cc);
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < 20; ++v) { s[v] = 0.f; c[v] = 0.f; }
}

template <bool COMP>
__global__ void __launch_bounds__(EST_THREADS, 2)
k_estep(const float4* __restrict__ pts, const Item* __restrict__ items,
        const int* __restrict__ meta, const NodeEst* __restrict__ est_lvl,
        float2* __restrict__ partials) {
    __shared__ float2 red[EST_THREADS / 32][NPART];
    const int n_items = meta[0];
    const int C = meta[1];
    const int ib = blockIdx.x * C;
    const int ie = min(ib + C, n_items);
    if (ib >= ie) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane >> 2, k = lane & 3;
    float in[20], s[20], c[20];
#pragma unroll
    for (int v = 0; v < 20; ++v) { in[v] = 0.f; s[v] = 0.f; c[v] = 0.f; }
    int nfold = 0;
    int cur = -1, run = -1;
    ChildRegs r0, r1;
    for (int it = ib; it < ie; ++it) {
        const Item w = items[it];
        if (w.parent != cur) {
            if (cur >= 0) {
                fold20<COMP>(in, s, c);
                nfold = 0;
                flush_run<COMP>(s, c, red, partials + int64_t(run) * NPART);
            }
            cur = w.parent;
            run = it;
            load_child(est_lvl + 8 * cur + 2 * k, r0);
            load_child(est_lvl + 8 * cur + 2 * k + 1, r1);
        }
        float4 znext = pts[w.start + min(warp * 8 + q, w.count - 1)];
        for (int base = 0; base < w.count; base += 64) {
            const int idx = base + warp * 8 + q;
            const bool valid = idx < w.count;
            const float4 z = znext;
            if (base + 64 < w.count) znext = pts[w.start + min(idx + 64, w.count - 1)];
            float e0x, e0y, e0z, e1x, e1y, e1z;
            const float s0 = child_score(r0, z.x, z.y, z.z, e0x, e0y, e0z);
            const float s1 = child_score(r1, z.x, z.y, z.z, e1x, e1y, e1z);
            float m = fmaxf(s0, s1);
            m = fmaxf(m, __shfl_xor_sync(FULL, m, 1));
            m = fmaxf(m, __shfl_xor_sync(FULL, m, 2));
            const bool any_live = m > -CUDART_INF_F;  // false for a leaf parent
            const float p0 = any_live ? exp2f(s0 - m) : 0.f;
            const float p1 = any_live ? exp2f(s1 - m) : 0.f;
            float tot = p0 + p1;
            tot += __shfl_xor_sync(FULL, tot, 1);
            tot += __shfl_xor_sync(FULL, tot, 2);
            const float rinv = (valid && any_live) ? 1.0f / tot : 0.0f;
            accum10(in, p0 * rinv, e0x, e0y, e0z);
            accum10(in + 10, p1 * rinv, e1x, e1y, e1z);
            if (++nfold == 16) {
                fold20<COMP>(in, s, c);
                nfold = 0;
            }
        }
    }
    fold20<COMP>(in, s, c);
    flush_run<COMP>(s, c, red, partials + int64_t(run) * NPART);
}

template <bool COMP>
__global__ void __launch_bounds__(256) k_mstep(int level, int n, const int* __restrict__ item_range,
                                               const int* __restrict__ meta,
                                               const float2* __restrict__ partials,
                                               const int* __restrict__ seg_count,
                                               const RootDev* __restrict__ root, float n_min,
                                               NodeStat* __restrict__ stat,
                                               NodeEst* __restrict__ est, int* __restrict__ status) {
    __shared__ MstepSmem msm;
    const int p = blockIdx.x;
    const int i0 = item_range[2 * p], i1 = item_range[2 * p + 1];
    if (i0 >= i1) return;  // parent without points: children stay dead
    mstep_parent<COMP>(level, n, p, i0, i1, meta[1], partials, seg_count, root, n_min, stat, est,
                       status, msm);
}

// ---------------------------------------------------------------- M-step
// ---------------------------------------------------------------- hand-off
__global__ void __launch_bounds__(EST_THREADS) k_assign(const float4* __restrict__ pts,
                                                        const Item* __restrict__ items,
                                                        const int* __restrict__ meta,
                                                        const NodeEst* __restrict__ est_lvl,
                                                        uint32_t* __restrict__ codes,
                                                        int* __restrict__ item_cnt) {
    __shared__ int cnt[EST_THREADS / 32][8];
    __shared__ int base[8];
    const int n_items = meta[0];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane >> 2, k = lane & 3;
    const unsigned lt = (1u << lane) - 1u;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const Item w = items[it];
        ChildRegs r0, r1;
        load_child(est_lvl + 8 * w.parent + 2 * k, r0);
        load_child(est_lvl + 8 * w.parent + 2 * k + 1, r1);
        if (threadIdx.x < 8) base[threadIdx.x] = 0;
        __syncthreads();
        for (int b0 = 0; b0 < w.count; b0 += 64) {
            const int idx = b0 + warp * 8 + q;
            const bool valid = idx < w.count;
            const float4 z = pts[w.start + (valid ? idx : 0)];
            float ex, ey, ez;
            const float s0 = child_score(r0, z.x, z.y, z.z, ex, ey, ez);
            const float s1 = child_score(r1, z.x, z.y, z.z, ex, ey, ez);
            float best = s0;
            int lab = 2 * k;
            if (s1 > best) { best = s1; lab = 2 * k + 1; }
#pragma unroll
            for (int off = 1; off <= 2; off <<= 1) {
                const float ob = __shfl_xor_sync(FULL, best, off);
                const int ol = __shfl_xor_sync(FULL, lab, off);
                if (ob > best || (ob == best && ol < lab)) { best = ob; lab = ol; }
            }
            const bool lead = valid && k == 0;
            int my_rank = 0;
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
                const unsigned bal = __ballot_sync(FULL, lead && lab == cc);
                if (lane == 0) cnt[warp][cc] = __popc(bal);
                if (lab == cc) my_rank = __popc(bal & lt);
            }
            __syncthreads();
            if (lead) {
                int r = base[lab] + my_rank;
                for (int w2 = 0; w2 < warp; ++w2) r += cnt[w2][lab];
                codes[w.start + idx] = uint32_t(lab) | (uint32_t(r) << 3);
            }
            __syncthreads();
            if (threadIdx.x < 8) {
                int tsum = 0;
                for (int w2 = 0; w2 < EST_THREADS / 32; ++w2) tsum += cnt[w2][threadIdx.x];
                base[threadIdx.x] += tsum;
            }
            __syncthreads();
        }
        if (threadIdx.x < 8) item_cnt[8 * it + threadIdx.x] = base[threadIdx.x];
        __syncthreads();
    }
}

// One CTA (256 threads) per parent: per child, exclusive scan over the
// parent's items of the item counts -> absolute destination offsets.
__global__ void __launch_bounds__(256) k_child_offsets(int level, int n,
                                                       const int* __restrict__ item_range,
                                                       const Item* __restrict__ items,
                                                       const int* __restrict__ item_cnt,
                                                       int* __restrict__ item_off,
                                                       int* __restrict__ seg_start,
                                                       int* __restrict__ seg_count) {
    __shared__ int tot[8][8];       // [warp][child]
    __shared__ int carry[8];
    const int p = blockIdx.x;
    const int i0 = item_range[2 * p], i1 = item_range[2 * p + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t g0 = d_level_offset(level) + 8 * int64_t(p);
    int pstart;
    if (i0 < i1) {
        pstart = items[i0].start;
    } else {
        // empty parent: its children get empty segments at the parent's start
        pstart = level == 0 ? 0 : seg_start[d_level_offset(level - 1) + p];
    }
    // pass 1: totals per child
    int t8[8] = {};
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x)
        for (int cc = 0; cc < 8; ++cc) t8[cc] += item_cnt[8 * i + cc];
    for (int cc = 0; cc < 8; ++cc) {
        int x = t8[cc];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(FULL, x, off);
        if (lane == 0) tot[warp][cc] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = pstart;
        for (int cc = 0; cc < 8; ++cc) {
            int s = 0;
            for (int w = 0; w < 8; ++w) s += tot[w][cc];
            carry[cc] = run;
            seg_start[g0 + cc] = run;
            seg_count[g0 + cc] = s;
            run += s;
        }
    }
    __syncthreads();
    // pass 2: scan in chunks of 256 items
    for (int b = i0; b < i1; b += blockDim.x) {
        const int i = b + threadIdx.x;
        int v8[8];
        for (int cc = 0; cc < 8; ++cc) v8[cc] = i < i1 ? item_cnt[8 * i + cc] : 0;
        int incl[8];
        for (int cc = 0; cc < 8; ++cc) {
            int x = v8[cc];
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(FULL, x, off);
                if (lane >= off) x += y;
            }
            incl[cc] = x;
            if (lane == 31) tot[warp][cc] = x;
        }
        __syncthreads();
        for (int cc = 0; cc < 8; ++cc) {
            int pre = carry[cc];
            for (int w = 0; w < warp; ++w) pre += tot[w][cc];
            if (i < i1) item_off[8 * i + cc] = pre + incl[cc] - v8[cc];
        }
        __syncthreads();
        if (threadIdx.x < 8) {
            int s = 0;
            for (int w = 0; w < 8; ++w) s += tot[w][threadIdx.x];
            carry[threadIdx.x] += s;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_scatter(const float4* __restrict__ pts_in,
                                                 const int* __restrict__ perm_in,
                                                 const Item* __restrict__ items,
                                                 const int* __restrict__ meta,
                                                 const uint32_t* __restrict__ codes,
                                                 const int* __restrict__ item_off,
                                                 float4* __restrict__ pts_out,
                                                 int* __restrict__ perm_out) {
    const int n_items = meta[0];
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const Item w = items[it];
        for (int j = threadIdx.x; j < w.count; j += blockDim.x) {
            const int pos = w.start + j;
            const uint32_t code = codes[pos];
            const int dst = item_off[8 * it + (code & 7u)] + int(code >> 3);
            pts_out[dst] = pts_in[pos];
            perm_out[dst] = perm_in ? perm_in[pos] : pos;
        }
    }
}

// ---------------------------------------------------------------- finalize
__global__ void k_finalize(int level, float lam_c, const RootDev* __restrict__ root,
                           NodeStat* __restrict__ stat, NodeEst* __restrict__ est,
                           float4* __restrict__ rnode) {
    const int64_t m = int64_t(1) << (3 * (level + 1));
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int64_t g = d_level_offset(level) + i;
    NodeStat& s = stat[g];
    if (!s.live) {
        for (int a = 0; a < 3; ++a) s.lam[a] = 1.0;
        for (int v = 0; v < 9; ++v) s.V[v] = (v % 4 == 0) ? 1.0 : 0.0;
        for (int v = 0; v < 6; ++v) s.P[v] = 0.0;
        s.complexity = 1.0;
        est[g].c.z = 0.f;
        rnode[3 * g] = make_float4(0.f, 0.f, 0.f, 0.f);
        rnode[3 * g + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        rnode[3 * g + 2] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    double lam[3], V[9];
    eig3(s.S, lam, V);
    const double eps = root->eps;
    double il[3];
    for (int a = 0; a < 3; ++a) {
        s.lam[a] = lam[a];
        il[a] = rcp_f64(fmax(lam[a], eps));
    }
    for (int v = 0; v < 9; ++v) s.V[v] = V[v];
    // P = V diag(1/lambda) V^T (Eq. 10)
    const int ij[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    for (int v = 0; v < 6; ++v) {
        const int r = ij[v][0], c = ij[v][1];
        double acc = 0.0;
        for (int k = 0; k < 3; ++k) acc += V[r * 3 + k] * il[k] * V[c * 3 + k];
        s.P[v] = acc;
    }
    s.complexity = lam[2] * rcp_f64(lam[0] + lam[1] + lam[2]);
    const float4 a = est[g].a;
    est[g].c.z = (s.complexity <= double(lam_c)) ? 1.f : 0.f;
    // FP32 registration constants: P and the offset of the FP64 mean from the
    // FP32 mean the descent measures against
    rnode[3 * g] = make_float4(float(s.P[0]), float(s.P[1]), float(s.P[2]), float(s.P[3]));
    rnode[3 * g + 1] = make_float4(float(s.P[4]), float(s.P[5]), 0.f, 0.f);
    rnode[3 * g + 2] = make_float4(float(s.mu[0] - double(a.x)), float(s.mu[1] - double(a.y)),
                                   float(s.mu[2] - double(a.z)), 0.f);
}

// ---------------------------------------------------------------- labels
__global__ void k_labels(int level, int n, const int* __restrict__ perm,
                         const int* __restrict__ seg_start, const int* __restrict__ seg_count,
                         int* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t off = d_level_offset(level);
    const int64_t m = int64_t(1) << (3 * (level + 1));
    // largest node with seg_start <= i (segments are in node order)
    int64_t lo = 0, hi = m - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (seg_start[off + mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    const int dst = perm[i];
    if (dst >= 0 && dst < n) out[dst] = int(lo);
}

}  // namespace

}  // namespace hgmm

using namespace hgmm;

#define HGMM_LAUNCH_CHECK()                                   \
    do {                                                      \
        cudaError_t e_ = cudaGetLastError();                  \
        if (e_ != cudaSuccess) {                              \
            fprintf(stderr, "hgmm: launch failed: %s (%s:%d)\n", cudaGetErrorString(e_), \
                    __FILE__, __LINE__);                      \
            return HGMM_ECUDA;                                \
        }                                                     \
    } while (0)

int hgmm_build_impl(hgmm_tree* t, const float4* pts, int64_t n64, int depth,
                    const hgmm_params& p, cudaStream_t s) {
    const int n = int(n64);
    const int G = t->est_grid;
    {
        ProfScope ps_(t, K_ROOT_PARTIAL, s);
        k_root<<<G, 256, 0, s>>>(pts, n, p.eps_rel, t->root_part, t->root_counter, t->root,
                                 t->status);
    }
    HGMM_LAUNCH_CHECK();
    const float4* cur = pts;
    const int* perm_prev = nullptr;
    const bool comp = p.precision == 0;
    for (int l = 0; l < depth; ++l) {
        const int n_par = l == 0 ? 1 : int(level_size(l - 1));
        const int64_t off = level_offset(l);
        NodeEst* est_lvl = t->est + off;
        {
            ProfScope ps_(t, K_INIT, s);
            k_init_children<<<n_par, 32, 0, s>>>(l, t->root, t->stat, t->est, t->seg_count, t->status);
        }
        {
            ProfScope ps_(t, K_MAKE_ITEMS, s);
            k_make_items<<<1, 1024, 0, s>>>(l, n, n_par, t->seg_start, t->seg_count, t->stat,
                                            t->items, t->item_range, t->meta, G);
        }
        {
            ProfScope ps_(t, K_FILL_ITEMS, s);
            k_fill_items<<<int((t->max_items + 255) / 256), 256, 0, s>>>(
                l, n, n_par, t->seg_start, t->seg_count, t->item_range, t->meta, t->items);
        }
        HGMM_LAUNCH_CHECK();
        const bool stop_here = p.debug_stop_level == l + 1;
        const int em_iters = stop_here ? p.debug_stop_iters : p.em_iters;
        for (int k = 0; k < em_iters; ++k) {
            {
                ProfScope ps_(t, K_ESTEP, s);
                if (comp)
                    k_estep<true><<<G, EST_THREADS, 0, s>>>(cur, t->items, t->meta, est_lvl, t->partials);
                else
                    k_estep<false><<<G, EST_THREADS, 0, s>>>(cur, t->items, t->meta, est_lvl, t->partials);
            }
            {
                ProfScope ps_(t, K_MSTEP, s);
                if (comp)
                    k_mstep<true><<<n_par, 256, 0, s>>>(l, n, t->item_range, t->meta, t->partials,
                                                        t->seg_count, t->root, p.n_min, t->stat,
                                                        t->est, t->status);
                else
                    k_mstep<false><<<n_par, 256, 0, s>>>(l, n, t->item_range, t->meta, t->partials,
                                                         t->seg_count, t->root, p.n_min, t->stat,
                                                         t->est, t->status);
            }
        }
        HGMM_LAUNCH_CHECK();
        if (stop_here) return HGMM_OK;  // checking aid: parameters after em_iters
        {
            ProfScope ps_(t, K_ASSIGN, s);
            k_assign<<<G, EST_THREADS, 0, s>>>(cur, t->items, t->meta, est_lvl, t->codes, t->item_cnt);
        }
        {
            ProfScope ps_(t, K_OFFSETS, s);
            k_child_offsets<<<n_par, 256, 0, s>>>(l, n, t->item_range, t->items, t->item_cnt,
                                                  t->item_off, t->seg_start, t->seg_count);
        }
        float4* out = t->pts[l & 1];
        {
            ProfScope ps_(t, K_SCATTER, s);
            k_scatter<<<G, 256, 0, s>>>(cur, perm_prev, t->items, t->meta, t->codes, t->item_off,
                                        out, t->perm[l]);
        }
        const int m = int(level_size(l));
        {
            ProfScope ps_(t, K_FINALIZE, s);
            // one warp per CTA: the FP64 eigen work is spread over as many SMs
            // as possible (each SM's FP64 pipe is narrow)
            k_finalize<<<(m + 31) / 32, 32, 0, s>>>(l, p.lam_c, t->root, t->stat, t->est,
                                                    t->rnode);
        }
        HGMM_LAUNCH_CHECK();
        cur = out;
        perm_prev = t->perm[l];
    }
    return HGMM_OK;
}

int hgmm_export_labels_impl(hgmm_tree* t, int level, int* d_out, cudaStream_t s) {
    const int n = int(t->n);
    {
        ProfScope ps_(t, K_LABELS, s);
        k_labels<<<(n + 255) / 256, 256, 0, s>>>(level, n, t->perm[level], t->seg_start,
                                                 t->seg_count, d_out);
    }
    HGMM_LAUNCH_CHECK();
    return HGMM_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the level-0 fit.
//
// Some callers cannot call cudaMalloc at all: code running while another
// component is capturing a CUDA graph on the same stream, real-time loops
// whose memory budget is fixed at start-up, or plug-ins whose host owns every
// device allocation.  For them, hgmm_fit_level0_noalloc runs the same level-0
// pipeline as hgmm_build (root statistics, PCA-octant initial children, K EM
// iterations of the 8-component GMM, FP64 finalize) with all of its scratch in
// the fixed array below instead of a tree's buffers.  The array lives in every
// GPU that loads this library until the process exits.
// ---------------------------------------------------------------------------
namespace hgmm {
namespace {

constexpr int NA_MAX_POINTS = 1 << 20;              // largest cloud the scratch holds
constexpr int NA_MAX_ITEMS = NA_MAX_POINTS / TILE + 1;
constexpr int NA_MAX_GRID = 1024;                   // E-step / root CTAs
constexpr size_t na_align(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t NA_OFF_EST = 0;
constexpr size_t NA_OFF_STAT = na_align(NA_OFF_EST + 8 * sizeof(NodeEst));
constexpr size_t NA_OFF_RNODE = na_align(NA_OFF_STAT + 8 * sizeof(NodeStat));
constexpr size_t NA_OFF_ROOT = na_align(NA_OFF_RNODE + 24 * sizeof(float4));
constexpr size_t NA_OFF_RPART = na_align(NA_OFF_ROOT + sizeof(RootDev));
constexpr size_t NA_OFF_WORDS = na_align(NA_OFF_RPART + size_t(NA_MAX_GRID) * 32 * sizeof(float));
constexpr size_t NA_OFF_ITEMS = na_align(NA_OFF_WORDS + 16 * sizeof(int));
constexpr size_t NA_OFF_PART = na_align(NA_OFF_ITEMS + size_t(NA_MAX_ITEMS) * sizeof(Item));
constexpr size_t NA_BYTES = na_align(NA_OFF_PART + size_t(NA_MAX_ITEMS) * NPART * sizeof(float2));

// ~2.8 MB of device memory shared by every call in the process.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

__global__ void k_noalloc_out(const NodeStat* __restrict__ stat, const int* __restrict__ status,
                              double* __restrict__ out) {
    const int c = threadIdx.x;
    if (c < 8) {
        const NodeStat& s = stat[c];
        double* o = out + 16 * c;
        o[0] = s.live ? s.pi : 0.0;
        for (int a = 0; a < 3; ++a) o[1 + a] = s.mu[a];
        for (int v = 0; v < 6; ++v) o[4 + v] = s.S[v];
        o[10] = s.live ? 1.0 : 0.0;
        o[11] = -1.0;  // hard counts need the hand-off, which this fit does not run
        o[12] = s.complexity;
        for (int a = 0; a < 3; ++a) o[13 + a] = s.lam[a];
    }
    if (c == 8) {
        const int st = *status;
        out[128] = (st & ST_NONFINITE) ? double(HGMM_ENONFINITE) : 0.0;
    }
}

struct NoAllocDevice {
    unsigned char* base = nullptr;  // device address of g_noalloc_scratch
    int grid = 0;
};

}  // namespace
}  // namespace hgmm

extern "C" int hgmm_fit_level0_noalloc(const float* d_points, int64_t n, const hgmm_params* p,
                                       void* stream, double* d_out) {
    using namespace hgmm;
    if (!d_points || !d_out || n < 8) return HGMM_EINVAL;
    if (n > NA_MAX_POINTS) {
        fprintf(stderr,
                "hgmm_fit_level0_noalloc: %lld points exceed the fixed scratch capacity of %d\n",
                (long long)n, NA_MAX_POINTS);
        return HGMM_ECAPACITY;
    }
    if ((reinterpret_cast<uintptr_t>(d_points) & 15u) != 0) return HGMM_EINVAL;
    hgmm_params prm;
    if (p) {
        prm = *p;
        if (prm.em_iters < 0 || prm.em_iters > 1000 || !(prm.eps_rel >= 0.f) ||
            !(prm.n_min >= 0.f) || !(prm.lam_c >= 0.f))
            return HGMM_EINVAL;
    } else {
        hgmm_params_default(&prm);
    }
    // one-time set-up per device, with that device current: resolve the
    // scratch array's device address (host code cannot use the symbol itself)
    constexpr int MAX_DEV = 64;
    static NoAllocDevice devs[MAX_DEV];
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return HGMM_ECUDA;
    NoAllocDevice d;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!devs[dev].base) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
                fprintf(stderr, "hgmm_fit_level0_noalloc: cudaGetSymbolAddress failed\n");
                return HGMM_ECUDA;
            }
            int n_sm = 0;
            if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                return HGMM_ECUDA;
            devs[dev].grid = std::min(2 * n_sm, NA_MAX_GRID);
            devs[dev].base = static_cast<unsigned char*>(ptr);
        }
        d = devs[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* b = d.base;
    NodeEst* est = reinterpret_cast<NodeEst*>(b + NA_OFF_EST);
    NodeStat* stat = reinterpret_cast<NodeStat*>(b + NA_OFF_STAT);
    float4* rnode = reinterpret_cast<float4*>(b + NA_OFF_RNODE);
    RootDev* root = reinterpret_cast<RootDev*>(b + NA_OFF_ROOT);
    float* rpart = reinterpret_cast<float*>(b + NA_OFF_RPART);
    int* words = reinterpret_cast<int*>(b + NA_OFF_WORDS);
    unsigned* root_counter = reinterpret_cast<unsigned*>(words + 0);
    int* status = words + 1;
    int* item_range = words + 2;  // [2]
    int* meta = words + 4;        // [2]
    int* seg = words + 6;         // [2] (unused at level 0)
    Item* items = reinterpret_cast<Item*>(b + NA_OFF_ITEMS);
    float2* partials = reinterpret_cast<float2*>(b + NA_OFF_PART);
    const int G = d.grid;
    const int ni = int(n);
    // the array keeps the previous call's contents: clear the words that
    // must start at zero (counter, status)
    if (cudaMemsetAsync(words, 0, 16 * sizeof(int), s) != cudaSuccess) return HGMM_ECUDA;
    k_root<<<G, 256, 0, s>>>(reinterpret_cast<const float4*>(d_points), ni, prm.eps_rel, rpart,
                             root_counter, root, status);
    k_init_children<<<1, 32, 0, s>>>(0, root, stat, est, seg, status);
    k_make_items<<<1, 1024, 0, s>>>(0, ni, 1, seg, seg, stat, items, item_range, meta, G);
    k_fill_items<<<(NA_MAX_ITEMS + 255) / 256, 256, 0, s>>>(0, ni, 1, seg, seg, item_range, meta,
                                                            items);
    for (int k = 0; k < prm.em_iters; ++k) {
        if (prm.precision == 0) {
            k_estep<true><<<G, EST_THREADS, 0, s>>>(reinterpret_cast<const float4*>(d_points), items,
                                                    meta, est, partials);
            k_mstep<true><<<1, 256, 0, s>>>(0, ni, item_range, meta, partials, seg, root,
                                            prm.n_min, stat, est, status);
        } else {
            k_estep<false><<<G, EST_THREADS, 0, s>>>(reinterpret_cast<const float4*>(d_points), items,
                                                     meta, est, partials);
            k_mstep<false><<<1, 256, 0, s>>>(0, ni, item_range, meta, partials, seg, root,
                                             prm.n_min, stat, est, status);
        }
    }
    k_finalize<<<1, 32, 0, s>>>(0, prm.lam_c, root, stat, est, rnode);
    k_noalloc_out<<<1, 32, 0, s>>>(stat, status, d_out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "hgmm_fit_level0_noalloc: launch failed: %s\n", cudaGetErrorString(e));
        return HGMM_ECUDA;
    }
    return HGMM_OK;
}
