// Device-side building blocks of the HGMM path, shared by the single-cloud
// kernels (one launch per phase, or one cooperative launch), the batched
// engine (one thread-block cluster per pair) and the allocation-free fit.
// Every phase takes the index and count of the CTAs that share it, so the
// same arithmetic runs under any of those schedules.
#pragma once

#include "hgmm_internal.cuh"
#include "hgmm_math.cuh"

namespace hgmm {

constexpr unsigned FULL = 0xffffffffu;
constexpr double FIX = 4294967296.0;      // 2^32
constexpr double INV_FIX = 1.0 / 4294967296.0;
constexpr float FIX_CLAMP = 1.0995116e12f;  // 2^40

__device__ __forceinline__ int64_t d_level_offset(int l) {
    return ((int64_t(1) << (3 * (l + 1))) - 8) / 7;
}

// ===================================================================== root
// Whole-cloud mean, covariance and bounding box (the root of the tree, whose
// children are Children(-1) of Algorithm 1).  Sums of (z - z0) and
// (z - z0)(z - z0)^T with z0 = the first point, FP32 with compensated
// accumulation.  A CTA partial is 25 floats: [0..17] 9 (sum, err) pairs,
// [18..20] min, [21..23] max, [24] non-finite count.
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


struct RootSmem {
    float sm[8][25];
    float gs[16][25];
};

// CTA `cta` of `ncta` sums its share of the points into out[0..24].
__device__ __forceinline__ void root_partial_cta(const float4* __restrict__ pts, int n, int cta,
                                                 int ncta, float* __restrict__ out, RootSmem& rs) {
    const float4 z0 = pts[0];
    float in[9] = {}, s[9] = {}, c[9] = {};
    float mn[3] = {CUDART_INF_F, CUDART_INF_F, CUDART_INF_F};
    float mx[3] = {-CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F};
    int bad = 0, cnt = 0;
    for (int i = cta * blockDim.x + threadIdx.x; i < n; i += ncta * blockDim.x) {
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
        for (int v = 0; v < 9; ++v) { rs.sm[warp][2 * v] = s[v]; rs.sm[warp][2 * v + 1] = c[v]; }
        for (int a = 0; a < 3; ++a) { rs.sm[warp][18 + a] = mn[a]; rs.sm[warp][21 + a] = mx[a]; }
        rs.sm[warp][24] = __int_as_float(bad);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float f[25];
        root_identity(f);
        for (int w = 0; w < int(blockDim.x >> 5); ++w) root_combine(f, rs.sm[w]);
        for (int v = 0; v < 25; ++v) out[v] = f[v];
    }
    __syncthreads();
}

// One CTA (>= 256 threads) reduces the `nparts` partials (stride 32 floats)
// in a fixed order -- 16 half-warp groups, then one thread -- and writes the
// FP64 root record with its eigen-decomposition.
__device__ __forceinline__ void root_final_cta(const float* __restrict__ part, int nparts,
                                               const float4* __restrict__ pts, int n, float eps_rel,
                                               RootDev* __restrict__ root, int* __restrict__ status,
                                               RootSmem& rs) {
    if (threadIdx.x < 256) {
        const int grp = threadIdx.x >> 4, it = threadIdx.x & 15;
        float a = 0.f, b = 0.f;
        if (it >= 9 && it < 12) a = CUDART_INF_F;
        if (it >= 12 && it < 15) a = -CUDART_INF_F;
        int cntb = 0;
#pragma unroll 4
        for (int blk = grp; blk < nparts; blk += 16) {
            const float* o = part + 32 * blk;
            if (it < 9) pair_add(a, b, __ldcg(o + 2 * it), __ldcg(o + 2 * it + 1));
            else if (it < 12) a = fminf(a, __ldcg(o + 18 + it - 9));
            else if (it < 15) a = fmaxf(a, __ldcg(o + 21 + it - 12));
            else cntb += __float_as_int(__ldcg(o + 24));
        }
        if (it < 9) { rs.gs[grp][2 * it] = a; rs.gs[grp][2 * it + 1] = b; }
        else if (it < 12) rs.gs[grp][18 + it - 9] = a;
        else if (it < 15) rs.gs[grp][21 + it - 12] = a;
        else rs.gs[grp][24] = __int_as_float(cntb);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float F[25];
        root_identity(F);
        for (int w = 0; w < 16; ++w) root_combine(F, rs.gs[w]);
        if (__float_as_int(F[24]) > 0) atomicOr(status, ST_NONFINITE);
        const float4 z0 = pts[0];
        const double nn = double(n);
        const double rn = rcp_f64(nn);  // one reciprocal instead of nine divisions
        double m1[3], m2[6];
        for (int a = 0; a < 3; ++a) m1[a] = (double(F[2 * a]) + double(F[2 * a + 1])) * rn;
        for (int v = 0; v < 6; ++v) m2[v] = (double(F[6 + 2 * v]) + double(F[7 + 2 * v])) * rn;
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
    __syncthreads();
}

// ===================================================================== init
// PCA-octant initial child c of parent p (level-0 parent = the root): mean
// mu_p + 1/2 sum_a s_a sqrt(lambda_a) v_a (s_a = +1 iff bit a of c), covariance
// Sigma_p / 4 + eps I, weight 1/8.  Children of a parent that is dead or
// holds no points are dead.  The parent's eigen-decomposition was computed
// when it was finalised.
__device__ __forceinline__ void init_child(int level, int p, int c, const RootDev* __restrict__ root,
                                           NodeStat* __restrict__ stat, NodeEst* __restrict__ est,
                                           const int* __restrict__ seg_count,
                                           int* __restrict__ status) {
    double lam[3], V[9], mu_p[3], S_p[6];
    bool alive;
    if (level == 0) {
        for (int a = 0; a < 3; ++a) { mu_p[a] = root->mu[a]; lam[a] = root->lam[a]; }
        for (int v = 0; v < 6; ++v) S_p[v] = root->S[v];
        for (int v = 0; v < 9; ++v) V[v] = root->V[v];
        alive = true;
    } else {
        const int64_t g = d_level_offset(level - 1) + p;
        const NodeStat& ps = stat[g];
        for (int a = 0; a < 3; ++a) { mu_p[a] = ps.mu[a]; lam[a] = ps.lam[a]; }
        for (int v = 0; v < 6; ++v) S_p[v] = ps.S[v];
        for (int v = 0; v < 9; ++v) V[v] = ps.V[v];
        alive = ps.live && seg_count[g] > 0;
    }
    const int64_t gc = d_level_offset(level) + 8 * int64_t(p) + c;
    NodeStat& cs = stat[gc];
    NodeEst& ce = est[gc];
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

// ==================================================================== items
// One CTA: exclusive scan over the level's parents of ceil(count / TILE);
// item_range[2p..2p+1] = [begin, end) item indices of parent p, meta[0] =
// item count, meta[1] = items per CTA for `nchunks` contiguous chunks.
// Every parent segment that holds points gets items, live or not: points
// under a leaf parent are carried down on its first child's segment with
// zero posteriors.
__device__ __forceinline__ void make_items_cta(int level, int n, int n_parents,
                                               const int* __restrict__ seg_count,
                                               int* __restrict__ item_range, int* __restrict__ meta,
                                               int nchunks, int* warp_tot /* smem[33] */) {
    int& carry = warp_tot[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int64_t poff = level == 0 ? 0 : d_level_offset(level - 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    for (int base = 0; base < n_parents; base += blockDim.x) {
        const int p = base + threadIdx.x;
        int count = 0;
        if (p < n_parents) count = level == 0 ? n : seg_count[poff + p];
        const int k = (count + TILE - 1) / TILE;
        int x = k;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(FULL, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = lane < nw ? warp_tot[lane] : 0;
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
        }
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_tot[nw - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // items per CTA (contiguous chunks, so a parent's runs are few)
        meta[0] = carry;
        meta[1] = max(1, (carry + nchunks - 1) / nchunks);
    }
    __syncthreads();
}

// Item j of a level: its parent is the largest p with begin(p) <= j (an
// empty parent shares its begin with the next one, which owns j).
__device__ __forceinline__ Item item_at(int j, int level, int n, int n_parents,
                                        const int* __restrict__ item_range,
                                        const int* __restrict__ seg_start,
                                        const int* __restrict__ seg_count) {
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
    return it;
}

// Item sources for the phases below: a materialised list, or computed on
// the fly from the per-parent ranges.
struct ItemList {
    const Item* items;
    __device__ __forceinline__ Item operator()(int j) const { return items[j]; }
};

struct ItemCalc {
    int level, n, n_parents;
    const int* item_range;
    const int* seg_start;
    const int* seg_count;
    __device__ __forceinline__ Item operator()(int j) const {
        return item_at(j, level, n, n_parents, item_range, seg_start, seg_count);
    }
};

// =================================================================== E-step
// Lane layout: a quad of 4 lanes handles one point, lane k of the quad owns
// children 2k and 2k+1 (their constants live in registers); a warp handles 8
// points per step, the CTA (EST_THREADS) 64.  Each lane accumulates the 10
// moments of its two children: plain FP32 over up to EST_FOLD points, then
// folded into a compensated (sum, error) pair.
struct ChildRegs {
    float mx, my, mz, C, w00, w10, w11, w20, w21, w22;
};

// CG: read through L2 only (constants that other CTAs of a persistent
// launch rewrite between uses).
template <bool CG = false>
__device__ __forceinline__ void load_child(const NodeEst* __restrict__ e, ChildRegs& r) {
    const float4 a = CG ? __ldcg(&e->a) : e->a, b = CG ? __ldcg(&e->b) : e->b, c = CG ? __ldcg(&e->c) : e->c;
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

// ---- packed pair of children (Blackwell FP32x2 arithmetic) -----------------
// Children 2k and 2k + 1 of a parent in the .x and .y halves: every packed
// instruction performs the two lanes' IEEE round-to-nearest operations, so
// the results are those of the scalar code (child_score, accum10, two_sum)
// bit for bit, in half the instructions.  The means and log-normalisers are
// stored negated so that subtractions become packed additions.
struct ChildPair {
    float2 nmx, nmy, nmz, nC, w00, w10, w11, w20, w21, w22;
};

template <bool CG = false>
__device__ __forceinline__ void load_child_pair(const NodeEst* __restrict__ e, ChildPair& p) {
    ChildRegs a, b;
    load_child<CG>(e, a);
    load_child<CG>(e + 1, b);
    p.nmx = make_float2(-a.mx, -b.mx);
    p.nmy = make_float2(-a.my, -b.my);
    p.nmz = make_float2(-a.mz, -b.mz);
    p.nC = make_float2(-a.C, -b.C);
    p.w00 = make_float2(a.w00, b.w00);
    p.w10 = make_float2(a.w10, b.w10);
    p.w11 = make_float2(a.w11, b.w11);
    p.w20 = make_float2(a.w20, b.w20);
    p.w21 = make_float2(a.w21, b.w21);
    p.w22 = make_float2(a.w22, b.w22);
}

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
// x - y, rounded once (as __fsub_rn)
__device__ __forceinline__ float2 sub2(float2 x, float2 y) { return __ffma2_rn(y, f2(-1.f), x); }

// u = -log2(pi N(z | child)) of both children (exactly the negated
// child_score) and the offsets e = z - mu.
__device__ __forceinline__ float2 neg_score_pair(const ChildPair& p, float zx, float zy, float zz, float2& ex,
                                                 float2& ey, float2& ez) {
    ex = __fadd2_rn(f2(zx), p.nmx);
    ey = __fadd2_rn(f2(zy), p.nmy);
    ez = __fadd2_rn(f2(zz), p.nmz);
    const float2 d0 = __fmul2_rn(p.w00, ex);
    const float2 d1 = __ffma2_rn(p.w11, ey, __fmul2_rn(p.w10, ex));
    const float2 d2 = __ffma2_rn(p.w22, ez, __ffma2_rn(p.w21, ey, __fmul2_rn(p.w20, ex)));
    float2 u = __ffma2_rn(d0, d0, p.nC);
    u = __ffma2_rn(d1, d1, u);
    return __ffma2_rn(d2, d2, u);
}

// accum10 of both children: a[v].x / .y = moment v of child 2k / 2k + 1.
__device__ __forceinline__ void accum_pair(float2 (&a)[10], float2 g, float2 ex, float2 ey, float2 ez) {
    const float2 gx = __fmul2_rn(g, ex), gy = __fmul2_rn(g, ey), gz = __fmul2_rn(g, ez);
    a[0] = __fadd2_rn(a[0], g);
    a[1] = __fadd2_rn(a[1], gx);
    a[2] = __fadd2_rn(a[2], gy);
    a[3] = __fadd2_rn(a[3], gz);
    a[4] = __ffma2_rn(gx, ex, a[4]);
    a[5] = __ffma2_rn(gx, ey, a[5]);
    a[6] = __ffma2_rn(gx, ez, a[6]);
    a[7] = __ffma2_rn(gy, ey, a[7]);
    a[8] = __ffma2_rn(gy, ez, a[8]);
    a[9] = __ffma2_rn(gz, ez, a[9]);
}

// fold20 on packed accumulators (two_sum per half).
template <bool COMP>
__device__ __forceinline__ void fold_pair(float2 (&in)[10], float2 (&s)[10], float2 (&c)[10]) {
#pragma unroll
    for (int v = 0; v < 10; ++v) {
        if (COMP) {
            const float2 t = __fadd2_rn(s[v], in[v]);
            const float2 bp = sub2(t, s[v]);
            const float2 e = __fadd2_rn(sub2(s[v], sub2(t, bp)), sub2(in[v], bp));
            s[v] = t;
            c[v] = __fadd2_rn(c[v], e);
        } else {
            s[v] = __fadd2_rn(s[v], in[v]);
        }
        in[v] = make_float2(0.f, 0.f);
    }
}

// Whether the parent whose children this quad lane holds (cp) has a live
// child: all lanes of the warp work on the same parent, so a warp vote
// answers for the quad.  A parent without one (a leaf) carries its points
// down with zero posteriors, so its items need no E-step arithmetic.
__device__ __forceinline__ bool parent_has_live_child(const ChildPair& cp) {
    return __any_sync(FULL, cp.nC.x < CUDART_INF_F || cp.nC.y < CUDART_INF_F);
}

// One E-step point of a quad lane (parent with a live child): Eq. 3
// posteriors of the point over the parent's 8 children (this lane holds two,
// its quad the rest: max and sum by shuffles) and the lane's two children's
// moments.
__device__ __forceinline__ void estep_point_pair(const ChildPair& cp, const float4 z, bool valid, float2 (&in)[10]) {
    float2 ex, ey, ez;
    const float2 u = neg_score_pair(cp, z.x, z.y, z.z, ex, ey, ez);
    float umin = fminf(u.x, u.y);
    umin = fminf(umin, __shfl_xor_sync(FULL, umin, 1));
    umin = fminf(umin, __shfl_xor_sync(FULL, umin, 2));
    const float2 arg = sub2(f2(umin), u);  // = score - max score
    const float p0 = ex2_fast(arg.x);
    const float p1 = ex2_fast(arg.y);
    float tot = p0 + p1;
    tot += __shfl_xor_sync(FULL, tot, 1);
    tot += __shfl_xor_sync(FULL, tot, 2);
    const float rinv = valid ? rcp_fast(tot) : 0.0f;
    accum_pair(in, __fmul2_rn(make_float2(p0, p1), f2(rinv)), ex, ey, ez);
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

// One level of the flush's reduce-scatter over the eight lanes of a warp
// that hold the same children (lanes k, k + 4, ..., k + 28): of the lane's
// first 2H values (H = N / 2 rounded up) it keeps the half chosen by bit O
// of its lane index (the first H, or the remaining N - H) and adds the
// partner's copy of that half, which lands at positions 0.. of s and c.
template <bool COMP, int N, int O>
__device__ __forceinline__ void flush_rs_level(float* s, float* c, int lane) {
    constexpr int H = (N + 1) / 2, L = N - H;  // kept by the lower / upper lane
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        // lower lane keeps i < H and sends i + H (i < L); upper keeps H + i (i < L), sends i
        const float ss = up ? s[i] : (i < L ? s[H + i] : 0.f);
        const float cs = up ? c[i] : (i < L ? c[H + i] : 0.f);
        float sk = up ? (i < L ? s[H + i] : 0.f) : s[i];
        float ck = up ? (i < L ? c[H + i] : 0.f) : c[i];
        const float sr = __shfl_xor_sync(FULL, ss, O);
        const float cr = __shfl_xor_sync(FULL, cs, O);
        if (COMP) pair_add(sk, ck, sr, cr);
        else sk += sr;
        s[i] = sk;
        c[i] = ck;
    }
}

// Block-wide reduction of the (s, c) accumulators into partial slot `run`.
// Within a warp the eight lanes of each child pair reduce-scatter their 20
// values (18 compensated additions and 36 shuffles per lane instead of 60
// and 120 for a butterfly); each value's warp total then sits in exactly
// one lane, which stores it for the fixed-order sum over the warps.
template <bool COMP>
__device__ __forceinline__ void flush_run(float* s, float* c, float2 (*red)[NPART],
                                          float2* __restrict__ out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, k = lane & 3;
    flush_rs_level<COMP, 20, 16>(s, c, lane);  // 10 values left
    flush_rs_level<COMP, 10, 8>(s, c, lane);   // 5
    flush_rs_level<COMP, 5, 4>(s, c, lane);    // 3 (lower lane) or 2 (upper lane)
    {
        // the values this lane now holds: a half of 20 by lane bit 4, of
        // that a half of 10 by bit 3, of that the first 3 or last 2 by bit 2
        const int base = ((lane & 16) ? 10 : 0) + ((lane & 8) ? 5 : 0) + ((lane & 4) ? 3 : 0);
        const int cnt = (lane & 4) ? 2 : 3;
#pragma unroll
        for (int i = 0; i < 3; ++i)
            if (i < cnt) red[warp][k * 20 + base + i] = make_float2(s[i], COMP ? c[i] : 0.f);
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


// flush_run of packed accumulators (child 2k's ten values, then child
// 2k + 1's, as flush_run expects), which are cleared.
template <bool COMP>
__device__ __forceinline__ void flush_pair(float2 (&s2)[10], float2 (&c2)[10], float2 (*red)[NPART],
                                           float2* __restrict__ out) {
    float s[20], c[20];
#pragma unroll
    for (int v = 0; v < 10; ++v) {
        s[v] = s2[v].x;
        s[10 + v] = s2[v].y;
        c[v] = c2[v].x;
        c[10 + v] = c2[v].y;
        s2[v] = make_float2(0.f, 0.f);
        c2[v] = make_float2(0.f, 0.f);
    }
    flush_run<COMP>(s, c, red, out);
}

// E-step of items [ib, ie) by one CTA: Eq. 3 posteriors of every point over
// the 8 children of its parent (log2 domain, max subtracted), gamma-weighted
// moments of each child centred on the child's current FP32 mean, one
// partial per run of consecutive items with the same parent, stored at the
// run's first item (ONE_RUN: the items are one parent's, and its single
// partial goes to partials[0..NPART), e.g. in shared memory).
template <bool COMP, class Items, bool CG = false, bool ONE_RUN = false>
__device__ __forceinline__ void estep_range(const float4* __restrict__ pts, Items items, int ib,
                                            int ie, const NodeEst* __restrict__ est_lvl,
                                            float2* __restrict__ partials,
                                            float2 (*red)[NPART]) {
    if (ib >= ie) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane >> 2, k = lane & 3;
    float2 in[10], s[10], c[10];
#pragma unroll
    for (int v = 0; v < 10; ++v) { in[v] = make_float2(0.f, 0.f); s[v] = in[v]; c[v] = in[v]; }
    int nfold = 0;
    int cur = -1, run = -1;
    bool live = false;
    ChildPair cp;
    for (int it = ib; it < ie; ++it) {
        const Item w = items(it);
        if (w.parent != cur) {
            if (cur >= 0) {
                fold_pair<COMP>(in, s, c);
                nfold = 0;
                flush_pair<COMP>(s, c, red, ONE_RUN ? partials : partials + int64_t(run) * NPART);
            }
            cur = w.parent;
            run = it;
            load_child_pair<CG>(est_lvl + 8 * cur + 2 * k, cp);
            live = parent_has_live_child(cp);
        }
        if (!live) continue;  // zero posteriors: nothing to add
        float4 znext = pts[w.start + min(warp * 8 + q, w.count - 1)];
        for (int base = 0; base < w.count; base += 64) {
            const int idx = base + warp * 8 + q;
            const bool valid = idx < w.count;
            const float4 z = znext;
            if (base + 64 < w.count) znext = pts[w.start + min(idx + 64, w.count - 1)];
            estep_point_pair(cp, z, valid, in);
            if (++nfold == EST_FOLD) {
                fold_pair<COMP>(in, s, c);
                nfold = 0;
            }
        }
    }
    fold_pair<COMP>(in, s, c);
    flush_pair<COMP>(s, c, red, ONE_RUN ? partials : partials + int64_t(run) * NPART);
}

// The E-step of whole items by single warps (items first, first + stride,
// ...): the same arithmetic as estep_range, but each item's moments are
// reduced inside its warp (quads of lanes: 8 points per step) and stored as
// the item's own partial, with no block-wide step.  For levels whose parents
// are many and small, where a CTA's chunk would cross a parent boundary at
// almost every item.
template <bool COMP, class Items>
__device__ __forceinline__ void estep_items_warp(const float4* __restrict__ pts, Items items, int first,
                                                 int stride, int n_items,
                                                 const NodeEst* __restrict__ est_lvl,
                                                 float2* __restrict__ partials) {
    const int lane = threadIdx.x & 31;
    const int q = lane >> 2, k = lane & 3;
    for (int it = first; it < n_items; it += stride) {
        const Item w = items(it);
        ChildRegs r0, r1;
        load_child(est_lvl + 8 * w.parent + 2 * k, r0);
        load_child(est_lvl + 8 * w.parent + 2 * k + 1, r1);
        float in[20], s[20], c[20];
#pragma unroll
        for (int v = 0; v < 20; ++v) { in[v] = 0.f; s[v] = 0.f; c[v] = 0.f; }
        int nfold = 0;
        // a parent without a live child: zero posteriors, zero partial
        const bool live = __any_sync(FULL, r0.C > -CUDART_INF_F || r1.C > -CUDART_INF_F);
        float4 znext = pts[w.start + min(q, w.count - 1)];
        for (int base = 0; live && base < w.count; base += 8) {
            const int idx = base + q;
            const bool valid = idx < w.count;
            const float4 z = znext;
            if (base + 8 < w.count) znext = pts[w.start + min(idx + 8, w.count - 1)];
            float e0x, e0y, e0z, e1x, e1y, e1z;
            const float s0 = child_score(r0, z.x, z.y, z.z, e0x, e0y, e0z);
            const float s1 = child_score(r1, z.x, z.y, z.z, e1x, e1y, e1z);
            float m = fmaxf(s0, s1);
            m = fmaxf(m, __shfl_xor_sync(FULL, m, 1));
            m = fmaxf(m, __shfl_xor_sync(FULL, m, 2));
            const float p0 = ex2_fast(s0 - m);
            const float p1 = ex2_fast(s1 - m);
            float tot = p0 + p1;
            tot += __shfl_xor_sync(FULL, tot, 1);
            tot += __shfl_xor_sync(FULL, tot, 2);
            const float rinv = valid ? rcp_fast(tot) : 0.0f;
            accum10(in, p0 * rinv, e0x, e0y, e0z);
            accum10(in + 10, p1 * rinv, e1x, e1y, e1z);
            if (++nfold == EST_FOLD) {
                fold20<COMP>(in, s, c);
                nfold = 0;
            }
        }
        fold20<COMP>(in, s, c);
        // the reduce-scatter of flush_run: each value's warp total lands in one lane
        flush_rs_level<COMP, 20, 16>(s, c, lane);
        flush_rs_level<COMP, 10, 8>(s, c, lane);
        flush_rs_level<COMP, 5, 4>(s, c, lane);
        const int base = ((lane & 16) ? 10 : 0) + ((lane & 8) ? 5 : 0) + ((lane & 4) ? 3 : 0);
        const int cnt = (lane & 4) ? 2 : 3;
        float2* out = partials + int64_t(it) * NPART + k * 20 + base;
#pragma unroll
        for (int i = 0; i < 3; ++i)
            if (i < cnt) out[i] = make_float2(s[i], COMP ? c[i] : 0.f);
    }
}

// =================================================================== M-step
// The M-step of the 8 children of parent p by one warp, a quad of lanes per
// child (lane 4c + r: child c, role r): the two reciprocals share one
// instruction stream (role 1 takes the parent's count), the mean offset,
// the six covariance entries and the FP32 constants are split over the
// roles and gathered by shuffles, and only the 3x3 Cholesky (which needs
// all six entries) runs on every lane of the quad.  One FP64 warp
// instruction holds the SMSP's FP64 pipe ~64 cycles whatever the active
// mask, so this issues about half the FP64 instructions of one lane per
// child.  Same rules as before: S0 below n_min kills the child; Sigma =
// S2/S0 - d d^T + eps I with d = S1/S0 (moments about the child's FP32
// mean); pi = S0 / n_p.  mom: 80 doubles (child c's ten at c * NMOM), shared
// or global.  All 32 lanes of the warp call it.
__device__ __forceinline__ void child_mstep_quad(int level, int n, int p, const double* mom,
                                                 const int* __restrict__ seg_count,
                                                 const RootDev* __restrict__ root, float n_min,
                                                 NodeStat* __restrict__ stat, NodeEst* __restrict__ est,
                                                 int* __restrict__ status) {
    const int lane = threadIdx.x & 31, c = lane >> 2, r = lane & 3, q0 = lane & ~3;
    const unsigned qm = 0xFu << q0;
    const int64_t g = d_level_offset(level) + 8 * int64_t(p) + c;
    NodeStat& cs = stat[g];
    NodeEst& ce = est[g];
    const double* m = mom + c * NMOM;
    const double S0 = m[0];
    const double n_p = level == 0 ? double(n) : double(seg_count[d_level_offset(level - 1) + p]);
    // a child below n_min expected points dies; if all eight die the parent
    // stays a leaf (its points keep zero posteriors from then on)
    const bool live = cs.live && S0 >= double(n_min) && S0 > 0.0;  // the same on the quad
    if (!live) {
        if (r == 0) {
            cs.live = 0;
            cs.pi = 0.0;
            ce.a.w = -CUDART_INF_F;
            ce.b = make_float4(0.f, 0.f, 0.f, 0.f);
            ce.c.x = 0.f;
            ce.c.y = 0.f;
        }
        return;
    }
    const double eps = root->eps;
    const double rx = rcp_f64(r == 1 ? n_p : S0);
    const double inv = __shfl_sync(qm, rx, q0);
    const double rnp = __shfl_sync(qm, rx, q0 | 1);
    // role a < 3: the mean offset d_a and the new mean mu_a
    const float4 ca = ce.a;
    const int a = r < 3 ? r : 2;
    const double da = m[1 + a] * inv;
    const double mua = double(a == 0 ? ca.x : (a == 1 ? ca.y : ca.z)) + da;
    const double d0 = __shfl_sync(qm, da, q0), d1 = __shfl_sync(qm, da, q0 | 1), d2 = __shfl_sync(qm, da, q0 | 2);
    // role r: covariance entries r and (r < 2) r + 4; packing xx xy xz yy yz zz
    auto entry = [&](int v) {
        const double di = v < 3 ? d0 : (v < 5 ? d1 : d2);
        const double dj = v == 0 ? d0 : (v == 1 || v == 3 ? d1 : d2);
        double e = fma(-di, dj, m[4 + v] * inv);
        if (v == 0 || v == 3 || v == 5) e += eps;
        return e;
    };
    const double e0 = entry(r), e1 = entry(r < 2 ? r + 4 : 5);
    double S[6];
    S[0] = __shfl_sync(qm, e0, q0);
    S[1] = __shfl_sync(qm, e0, q0 | 1);
    S[2] = __shfl_sync(qm, e0, q0 | 2);
    S[3] = __shfl_sync(qm, e0, q0 | 3);
    S[4] = __shfl_sync(qm, e1, q0);
    S[5] = __shfl_sync(qm, e1, q0 | 1);
    const double pi = S0 * rnp;
    if (r == 0) cs.pi = pi;
    if (r < 3) cs.mu[r] = mua;
    cs.S[r] = e0;
    if (r < 2) cs.S[r + 4] = e1;
    // Cholesky of Sigma (every lane of the quad), with the diagonal loading
    // of pack_est when it is not positive definite
    double L[6], R[3];
    bool clean = true;
    double boost = eps > 0.0 ? eps : 1e-30;
    bool ok = chol3(S, L, R);
    for (int tries = 0; tries < 8 && !ok; ++tries) {
        clean = false;
        S[0] += boost; S[3] += boost; S[5] += boost;
        boost *= 10.0;
        ok = chol3(S, L, R);
    }
    if (!ok) {  // hopeless (NaN input): make it an isotropic unit Gaussian
        L[0] = 1; L[1] = 0; L[2] = 1; L[3] = 0; L[4] = 0; L[5] = 1;
        R[0] = 1; R[1] = 1; R[2] = 1;
        clean = false;
    }
    if (!clean && r == 0) atomicOr(status, ST_CHOL);
    // W = sqrt(log2(e) / 2) L^-1: role r forms entries r and (r < 2) r + 4 of
    // (m00, m10, m11, m20, m21, m22)
    const double k = 0.8493218002880191;  // sqrt(log2(e) / 2)
    const double m00 = R[0], m11 = R[1], m22 = R[2];
    const double m10 = -L[1] * m00 * m11;
    const double m21 = -L[4] * m11 * m22;
    const double m20 = -(L[3] * m00 + L[4] * m10) * m22;
    const double wa = r == 0 ? m00 : (r == 1 ? m10 : (r == 2 ? m11 : m20));
    const double wb = r == 0 ? m21 : m22;
    const float f0 = float(k * wa), f1 = float(k * wb);
    const float w00 = __shfl_sync(qm, f0, q0), w10 = __shfl_sync(qm, f0, q0 | 1);
    const float w11 = __shfl_sync(qm, f0, q0 | 2), w20 = __shfl_sync(qm, f0, q0 | 3);
    const float w21 = __shfl_sync(qm, f1, q0), w22 = __shfl_sync(qm, f1, q0 | 1);
    const float mf = float(mua);
    const float mx = __shfl_sync(qm, mf, q0), my = __shfl_sync(qm, mf, q0 | 1), mz = __shfl_sync(qm, mf, q0 | 2);
    if (r == 0) {
        // log-normaliser in FP32: log2 det(L) from the FP64 product split
        // into exponent and mantissa
        int ex = 0;
        const double mant = frexp(L[0] * L[2] * L[5], &ex);
        const float C = log2f(float(pi)) - 3.9547135f /* 1.5 log2(2 pi) */ -
                        (float(ex) + log2f(float(mant)));
        ce.a = make_float4(mx, my, mz, C);
        ce.b = make_float4(w00, w10, w11, w20);
        ce.c = make_float4(w21, w22, 0.f, 0.f);
    }
}

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
    if (threadIdx.x < 32) child_mstep_quad(level, n, p, sm.mom, seg_count, root, n_min, stat, est, status);
    __syncthreads();
}

// The runs of a parent split into MSTEP_SLICES slices (slice j: runs
// [j * nruns / S, (j + 1) * nruns / S)), each reduced by one CTA in the order
// of mstep_parent's first phase; the slice sums are then combined in slice
// order.  The level-wide M-step reduces the slices of a parent in parallel
// CTAs; the cooperative EM's owner reduces them one after another: the same
// arithmetic either way.
template <bool COMP>
__device__ void reduce_run_slice(int i0, int i1, int C, int j, int n_slices, const float2* __restrict__ partials,
                                 MstepSmem& sm, float2* out) {
    const int nruns = (i1 - 1) / C - i0 / C + 1;
    const int ra = int((int64_t(j) * nruns) / n_slices), rb = int((int64_t(j + 1) * nruns) / n_slices);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    float S[3] = {0.f, 0.f, 0.f}, Cc[3] = {0.f, 0.f, 0.f};
    for (int r0 = ra + warp; r0 < rb; r0 += 4 * nw) {
        float2 x[4][3];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = r0 + u * nw;
            const int slot = r == 0 ? i0 : (i0 / C + r) * C;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int v = lane + 32 * q;
                x[u][q] = (r < rb && v < NPART) ? __ldcg(&partials[int64_t(slot) * NPART + v])
                                                 : make_float2(0.f, 0.f);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                if (COMP) pair_add(S[q], Cc[q], x[u][q].x, x[u][q].y);
                else S[q] += x[u][q].x;
            }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int v = lane + 32 * q;
        if (v < NPART) sm.grp[warp][v] = make_float2(S[q], Cc[q]);
    }
    __syncthreads();
    if (threadIdx.x < NPART) {
        float Sx = 0.f, Cx = 0.f;
        for (int w = 0; w < nw; ++w) {
            if (COMP) pair_add(Sx, Cx, sm.grp[w][threadIdx.x].x, sm.grp[w][threadIdx.x].y);
            else Sx += sm.grp[w][threadIdx.x].x;
        }
        out[threadIdx.x] = make_float2(Sx, Cx);
    }
    __syncthreads();
}

// Combine the n_slices slice sums (NPART each; GLOBAL: written by other
// CTAs, read through L2; else shared memory) in slice order and run the
// M-step of the parent's 8 children.
template <bool COMP, bool GLOBAL>
__device__ void mstep_from_slices(int level, int n, int p, const float2* slices, int n_slices,
                                  const int* __restrict__ seg_count, const RootDev* __restrict__ root,
                                  float n_min, NodeStat* __restrict__ stat, NodeEst* __restrict__ est,
                                  int* __restrict__ status, MstepSmem& sm) {
    if (threadIdx.x < NPART) {
        float S = 0.f, Cc = 0.f;
        for (int j = 0; j < n_slices; ++j) {
            const float2 x = GLOBAL ? __ldcg(&slices[j * NPART + threadIdx.x]) : slices[j * NPART + threadIdx.x];
            if (COMP) pair_add(S, Cc, x.x, x.y);
            else S += x.x;
        }
        sm.mom[threadIdx.x] = double(S) + double(Cc);
    }
    __syncthreads();
    if (threadIdx.x < 32) child_mstep_quad(level, n, p, sm.mom, seg_count, root, n_min, stat, est, status);
    __syncthreads();
}

// The same M-step for a parent with few runs, by one warp (no block
// barriers): lane l sums values l, l+32, l+64 over the runs in order; lanes
// 0..7 then build the children.  mom = 80 doubles of shared memory per warp.
template <bool COMP>
__device__ void mstep_parent_warp(int level, int n, int p, int i0, int i1, int C,
                                  const float2* __restrict__ partials,
                                  const int* __restrict__ seg_count, const RootDev* __restrict__ root,
                                  float n_min, NodeStat* __restrict__ stat,
                                  NodeEst* __restrict__ est, int* __restrict__ status, double* mom) {
    const int lane = threadIdx.x & 31;
    const int nruns = (i1 - 1) / C - i0 / C + 1;
    float S[3] = {0.f, 0.f, 0.f}, Cc[3] = {0.f, 0.f, 0.f};
    for (int r = 0; r < nruns; ++r) {
        const int slot = r == 0 ? i0 : (i0 / C + r) * C;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int v = lane + 32 * j;
            if (v < NPART) {
                const float2 x = __ldcg(&partials[int64_t(slot) * NPART + v]);
                if (COMP) pair_add(S[j], Cc[j], x.x, x.y);
                else S[j] += x.x;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int v = lane + 32 * j;
        if (v < NPART) mom[v] = double(S[j]) + double(Cc[j]);
    }
    __syncwarp();
    child_mstep_quad(level, n, p, mom, seg_count, root, n_min, stat, est, status);
    __syncwarp();
}


// ================================================================= hand-off
static_assert(TILE % 64 == 0 && EST_THREADS == 256, "an item is whole CTA steps of 64 points");
struct AssignSmem {
    int cnt[TILE / 64][EST_THREADS / 32][8];  // [step][warp][child]
};

// Argmax hand-off (ties -> lowest index) of one item's points by one CTA,
// with each point's rank among the item's points that chose the same child
// (ballots, so deterministic and stable): codes[pos] = child | rank << 3 and
// item_cnt[8 it + c] = the item's count per child.  All of the item's
// points (up to TILE, 64 per CTA step) are loaded and labelled first, with
// the per-step, per-warp child counts in shared memory, so one barrier
// serves the whole item: a point's rank is the counts of the steps before
// its own, plus those of the warps before its own, plus its rank in its warp.
__device__ __forceinline__ void assign_item(const float4* __restrict__ pts, const Item w, int it,
                                            const NodeEst* __restrict__ est_lvl,
                                            uint32_t* __restrict__ codes,
                                            int* __restrict__ item_cnt, AssignSmem& as) {
    constexpr int NS = TILE / 64;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane >> 2, k = lane & 3;
    const unsigned lt = (1u << lane) - 1u;
    ChildRegs r0, r1;
    load_child(est_lvl + 8 * w.parent + 2 * k, r0);
    load_child(est_lvl + 8 * w.parent + 2 * k + 1, r1);
    float4 z[NS];
#pragma unroll
    for (int st = 0; st < NS; ++st) z[st] = pts[w.start + min(64 * st + warp * 8 + q, w.count - 1)];
    int lab_s[NS], rank_s[NS];
#pragma unroll
    for (int st = 0; st < NS; ++st) {
        const bool valid = 64 * st + warp * 8 + q < w.count;
        float ex, ey, ez;
        const float s0 = child_score(r0, z[st].x, z[st].y, z[st].z, ex, ey, ez);
        const float s1 = child_score(r1, z[st].x, z[st].y, z[st].z, ex, ey, ez);
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
            if (lane == 0) as.cnt[st][warp][cc] = __popc(bal);
            if (lab == cc) my_rank = __popc(bal & lt);
        }
        lab_s[st] = lab;
        rank_s[st] = my_rank;
    }
    __syncthreads();
#pragma unroll
    for (int st = 0; st < NS; ++st) {
        const int idx = 64 * st + warp * 8 + q;
        if (k == 0 && idx < w.count) {
            const int lab = lab_s[st];
            int r = rank_s[st];
            for (int s2 = 0; s2 < st; ++s2)
#pragma unroll
                for (int w2 = 0; w2 < EST_THREADS / 32; ++w2) r += as.cnt[s2][w2][lab];
            for (int w2 = 0; w2 < warp; ++w2) r += as.cnt[st][w2][lab];
            codes[w.start + idx] = uint32_t(lab) | (uint32_t(r) << 3);
        }
    }
    if (threadIdx.x < 8) {
        int tsum = 0;
        for (int s2 = 0; s2 < NS; ++s2)
#pragma unroll
            for (int w2 = 0; w2 < EST_THREADS / 32; ++w2) tsum += as.cnt[s2][w2][threadIdx.x];
        item_cnt[8 * it + threadIdx.x] = tsum;
    }
    __syncthreads();
}

struct OffsetSmem {
    int tot[8][8];  // [warp][child]
    int carry[8];
};

__device__ __forceinline__ void child_offsets_scan(int ia, int ib, const int* __restrict__ item_cnt,
                                                   int* __restrict__ item_off, OffsetSmem& os);

// Child segments of parent p (items [i0, i1), segment start pstart) by one
// CTA of 256 threads: per child, an exclusive scan over the parent's items
// of the item counts -> absolute destination offsets; children's seg_start /
// seg_count.
__device__ __forceinline__ void child_offsets_cta(int level, int p, int i0, int i1, int pstart,
                                                  const int* __restrict__ item_cnt,
                                                  int* __restrict__ item_off,
                                                  int* __restrict__ seg_start,
                                                  int* __restrict__ seg_count, OffsetSmem& os) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t g0 = d_level_offset(level) + 8 * int64_t(p);
    int t8[8] = {};
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x)
        for (int cc = 0; cc < 8; ++cc) t8[cc] += item_cnt[8 * i + cc];
    for (int cc = 0; cc < 8; ++cc) {
        int x = t8[cc];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(FULL, x, off);
        if (lane == 0) os.tot[warp][cc] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = pstart;
        for (int cc = 0; cc < 8; ++cc) {
            int s = 0;
            for (int w = 0; w < 8; ++w) s += os.tot[w][cc];
            os.carry[cc] = run;
            seg_start[g0 + cc] = run;
            seg_count[g0 + cc] = s;
            run += s;
        }
    }
    __syncthreads();
    child_offsets_scan(i0, i1, item_cnt, item_off, os);
}

// Items [ia, ib) of a parent by one CTA of 256 threads, os.carry[c] = the
// destination of child c's first point in item ia (set and synchronised by
// the caller): per child, an exclusive scan of the item counts ->
// item_off.  carry ends past the range.
__device__ __forceinline__ void child_offsets_scan(int ia, int ib, const int* __restrict__ item_cnt,
                                                   int* __restrict__ item_off, OffsetSmem& os) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i1 = ib;
    for (int b = ia; b < i1; b += blockDim.x) {
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
            if (lane == 31) os.tot[warp][cc] = x;
        }
        __syncthreads();
        for (int cc = 0; cc < 8; ++cc) {
            int pre = os.carry[cc];
            for (int w = 0; w < warp; ++w) pre += os.tot[w][cc];
            if (i < i1) item_off[8 * i + cc] = pre + incl[cc] - v8[cc];
        }
        __syncthreads();
        if (threadIdx.x < 8) {
            int s = 0;
            for (int w = 0; w < 8; ++w) s += os.tot[w][threadIdx.x];
            os.carry[threadIdx.x] += s;
        }
        __syncthreads();
    }
}

// The same by one warp (for parents with few items): lanes scan 32 items at
// a time per child in a fixed order.
__device__ __forceinline__ void child_offsets_warp(int level, int p, int i0, int i1, int pstart,
                                                   const int* __restrict__ item_cnt,
                                                   int* __restrict__ item_off,
                                                   int* __restrict__ seg_start,
                                                   int* __restrict__ seg_count) {
    const int lane = threadIdx.x & 31;
    const int64_t g0 = d_level_offset(level) + 8 * int64_t(p);
    int tot8[8] = {};
    for (int i = i0 + lane; i < i1; i += 32)
        for (int cc = 0; cc < 8; ++cc) tot8[cc] += item_cnt[8 * i + cc];
    int carry8[8];
    int run = pstart;
    for (int cc = 0; cc < 8; ++cc) {
        int x = tot8[cc];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(FULL, x, off);
        carry8[cc] = run;
        if (lane == 0) {
            seg_start[g0 + cc] = run;
            seg_count[g0 + cc] = x;
        }
        run += x;
    }
    for (int b = i0; b < i1; b += 32) {
        const int i = b + lane;
        for (int cc = 0; cc < 8; ++cc) {
            const int v = i < i1 ? item_cnt[8 * i + cc] : 0;
            int x = v;
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(FULL, x, off);
                if (lane >= off) x += y;
            }
            if (i < i1) item_off[8 * i + cc] = carry8[cc] + x - v;
            carry8[cc] += __shfl_sync(FULL, x, 31);
        }
    }
}

// Stable 8-way partition of one item's points by one CTA (or any group of
// threads striding by `stride` from `first`).
__device__ __forceinline__ void scatter_item(const float4* __restrict__ pts_in,
                                             const int* __restrict__ perm_in, const Item w, int it,
                                             const uint32_t* __restrict__ codes,
                                             const int* __restrict__ item_off,
                                             float4* __restrict__ pts_out,
                                             int* __restrict__ perm_out, int first, int stride) {
    for (int j = first; j < w.count; j += stride) {
        const int pos = w.start + j;
        const uint32_t code = codes[pos];
        const int dst = item_off[8 * it + (code & 7u)] + int(code >> 3);
        pts_out[dst] = pts_in[pos];
        if (perm_out) perm_out[dst] = perm_in ? perm_in[pos] : pos;
    }
}

// =================================================================== finalize
// Node i of a level: FP64 eigen-decomposition of its covariance,
// complexity lambda_3 / (lambda_1 + lambda_2 + lambda_3) and the stop flag
// (<= lambda_c, Sec. 4.1), precision P = V diag(1/max(lambda, eps)) V^T
// (Eq. 10) and the FP32 registration constants.
__device__ __forceinline__ void finalize_node(int level, int64_t i, float lam_c,
                                              const RootDev* __restrict__ root,
                                              NodeStat* __restrict__ stat, NodeEst* __restrict__ est,
                                              float4* __restrict__ rnode) {
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

// ============================================================ whole build
// Scratch of one build phase at a time.
struct BuildSmem {
    union {
        float2 red[EST_THREADS / 32][NPART];
        MstepSmem msm;
        double wmom[EST_THREADS / 32][NPART];
        AssignSmem as;
        OffsetSmem os;
        RootSmem rs;
        int warp_tot[33];
    };
};

// Device buffers of one tree build (the target's points are read, the
// ping-pong buffers receive each level's sorted order).
struct BuildCtx {
    const float4* pts;
    int n, depth, em_iters;
    float n_min, lam_c, eps_rel;
    int stop_level, stop_iters;  // stop after stop_iters EM iterations of level stop_level - 1
    NodeEst* est;
    NodeStat* stat;
    float4* rnode;
    int* seg_start;
    int* seg_count;
    RootDev* root;
    float4* buf[2];
    int* perm[HGMM_MAX_DEPTH];   // per level, or null (no input-order labels kept)
    uint32_t* codes;
    Item* items;                 // the level's work items, filled once per level
    int* item_range;
    int* meta;
    float2* partials;
    int* item_cnt;
    int* item_off;
    float* root_part;            // cs x 32
    int* status;
    // shape of the phases (the batched form tunes them per cloud size):
    int warp_item_parents;       // one warp per E-step item when parents >= this x CTAs
    int mstep_cta_runs;          // a parent's M-step on a whole CTA from this many runs
    int offsets_cta_items;       // a parent's child offsets on a whole CTA from this many items
};

// Default phase shape of build_levels.
constexpr int BUILD_WARP_ITEM_PARENTS = 4;
constexpr int BUILD_MSTEP_CTA_RUNS = 8;
constexpr int BUILD_OFFSETS_CTA_ITEMS = 64;

// The top-down build (Sec. 3, Sec. 4.1 and the readings of the hot path) run
// by cs CTAs of rank 0..cs-1 that meet at sync() between phases: root
// statistics, then per level the child init, the work items, K EM
// iterations (E-step over the items, M-step per parent: a whole CTA for
// parents with many runs, one warp for the others), the argmax hand-off,
// the stable partition into the other point buffer and the per-node
// finalisation.  sync() returns false when a bounded wait gave up; the
// build then stops.  Returns the buffer holding the last level's order.
template <bool COMP, typename Sync>
__device__ bool build_levels(const BuildCtx& x, int rank, int cs, BuildSmem& bs, Sync sync) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    if (rank == 0 && threadIdx.x == 0) *x.status = 0;
    root_partial_cta(x.pts, x.n, rank, cs, x.root_part + 32 * rank, bs.rs);
    if (!sync()) return false;
    if (rank == 0) root_final_cta(x.root_part, cs, x.pts, x.n, x.eps_rel, x.root, x.status, bs.rs);
    if (!sync()) return false;
    const float4* cur = x.pts;
    const int* perm_prev = nullptr;
    for (int l = 0; l < x.depth; ++l) {
        const int n_par = l == 0 ? 1 : int(level_size(l - 1));
        // per-parent work goes to CTA (p + 1) mod cs, warp p / cs: the FP64
        // chains of the parents land on every SM (one SM's FP64 pipe is
        // narrow) and level 0's single parent runs beside CTA 0's item scan
        const int prank = rank == 0 ? cs - 1 : rank - 1;  // parents p = prank + cs * j
        for (int p = prank + cs * warp; p < n_par; p += cs * wpb)
            if (lane < 8) init_child(l, p, lane, x.root, x.stat, x.est, x.seg_count, x.status);
        if (rank == 0)
            make_items_cta(l, x.n, n_par, x.seg_count, x.item_range, x.meta, cs, bs.warp_tot);
        if (!sync()) return false;
        const int n_items = __ldcg(x.meta);
        const int C = __ldcg(x.meta + 1);
        {
            // materialise the items once: every later phase of the level reads them
            const ItemCalc calc{l, x.n, n_par, x.item_range, x.seg_start, x.seg_count};
            for (int j = rank * blockDim.x + threadIdx.x; j < n_items; j += cs * blockDim.x)
                x.items[j] = calc(j);
        }
        if (!sync()) return false;
        const ItemList items{x.items};
        NodeEst* est_lvl = x.est + level_offset(l);
        const bool stop_here = x.stop_level == l + 1;
        const int K = stop_here ? x.stop_iters : x.em_iters;
        // many small parents per CTA: one warp per item, every item its own
        // run (C = 1); otherwise each CTA takes a chunk of C items
        const bool warp_items = n_par >= x.warp_item_parents * cs;
        const int Crun = warp_items ? 1 : C;
        for (int k = 0; k < K; ++k) {
            if (warp_items)
                estep_items_warp<COMP>(cur, items, rank * wpb + warp, cs * wpb, n_items, est_lvl,
                                       x.partials);
            else
                estep_range<COMP>(cur, items, rank * C, min(rank * C + C, n_items), est_lvl, x.partials,
                                  bs.red);
            if (!sync()) return false;
            for (int p = prank; p < n_par; p += cs) {
                const int i0 = __ldcg(x.item_range + 2 * p), i1 = __ldcg(x.item_range + 2 * p + 1);
                if (i0 < i1 && (i1 - 1) / Crun - i0 / Crun + 1 >= x.mstep_cta_runs)
                    mstep_parent<COMP>(l, x.n, p, i0, i1, Crun, x.partials, x.seg_count, x.root,
                                       x.n_min, x.stat, x.est, x.status, bs.msm);
            }
            __syncthreads();
            for (int p = prank + cs * warp; p < n_par; p += cs * wpb) {
                const int i0 = __ldcg(x.item_range + 2 * p), i1 = __ldcg(x.item_range + 2 * p + 1);
                if (i0 < i1 && (i1 - 1) / Crun - i0 / Crun + 1 < x.mstep_cta_runs)
                    mstep_parent_warp<COMP>(l, x.n, p, i0, i1, Crun, x.partials, x.seg_count, x.root,
                                            x.n_min, x.stat, x.est, x.status, bs.wmom[warp]);
            }
            if (!sync()) return false;
        }
        if (stop_here) return true;  // checking aid: parameters after K iterations
        // hand-off: argmax, per-parent child offsets, stable partition
        for (int it = rank; it < n_items; it += cs)
            assign_item(cur, items(it), it, est_lvl, x.codes, x.item_cnt, bs.as);
        if (!sync()) return false;
        for (int p = prank; p < n_par; p += cs) {  // parents with many items: a whole CTA
            const int i0 = __ldcg(x.item_range + 2 * p), i1 = __ldcg(x.item_range + 2 * p + 1);
            if (i1 - i0 >= x.offsets_cta_items) child_offsets_cta(l, p, i0, i1, items(i0).start, x.item_cnt, x.item_off,
                                                 x.seg_start, x.seg_count, bs.os);
        }
        __syncthreads();
        for (int p = prank + cs * warp; p < n_par; p += cs * wpb) {
            const int i0 = __ldcg(x.item_range + 2 * p), i1 = __ldcg(x.item_range + 2 * p + 1);
            if (i1 - i0 >= x.offsets_cta_items) continue;
            const int pstart = i0 < i1 ? items(i0).start
                                       : (l == 0 ? 0 : __ldcg(x.seg_start + level_offset(l - 1) + p));
            child_offsets_warp(l, p, i0, i1, pstart, x.item_cnt, x.item_off, x.seg_start, x.seg_count);
        }
        if (!sync()) return false;
        float4* out = x.buf[l & 1];
        int* perm_out = x.perm[l];
        for (int it = rank; it < n_items; it += cs)
            scatter_item(cur, perm_prev, items(it), it, x.codes, x.item_off, out, perm_out,
                         threadIdx.x, blockDim.x);
        // per-node finalisation: node r + cs t for thread t of CTA r, so the
        // FP64 eigen chains spread over every CTA (each SM's FP64 pipe is narrow)
        const int64_t m = level_size(l);
        for (int64_t i = int64_t(threadIdx.x) * cs + rank; i < m; i += int64_t(cs) * blockDim.x)
            finalize_node(l, i, x.lam_c, x.root, x.stat, x.est, x.rnode);
        if (!sync()) return false;
        cur = out;
        perm_prev = perm_out;
    }
    return true;
}

// ============================================================ registration
__device__ __forceinline__ long long to_fix(float v) {
    const float c = fminf(fmaxf(v, -FIX_CLAMP), FIX_CLAMP);
    return __float2ll_rn(c);
}

// Algorithm 1 for the points of this CTA (grid-stride by warps) with the
// current transform; adds each point's (gamma, gamma (z' - mu_j)) to the
// chosen node's fixed-point moments.
constexpr int STAGED_NODES = 584;  // levels 0..2 (8 + 64 + 512 nodes) live in shared memory
// Staged layout: node g at float4 slot 3 g + g / 8, i.e. one float4 of padding
// after each block of 8 siblings (100 words), so that the same child of
// different parents falls on different banks (block b starts at bank 4 b mod
// 32): the lanes of a warp descending under different parents load without
// conflicts between up to 8 consecutive parents.
constexpr int STAGED_F4 = 3 * STAGED_NODES + STAGED_NODES / 8;
static_assert(STAGED_NODES % 8 == 0, "whole sibling blocks are staged");

__device__ __forceinline__ int staged_slot(int g) { return 3 * g + (g >> 3); }

// Copy the first ns nodes (ns <= STAGED_NODES) of est to the staged layout
// (all threads of the CTA; the caller synchronises).
__device__ __forceinline__ void stage_nodes(float4* sm_est, const NodeEst* __restrict__ est, int ns) {
    const float4* g = reinterpret_cast<const float4*>(est);
    for (int i = threadIdx.x; i < 3 * ns; i += blockDim.x) {
        const int node = i / 3;
        sm_est[i + (node >> 3)] = __ldcg(g + i);
    }
}

// Child c of the sibling block that starts at node `first` (a multiple of 8:
// level offsets and 8 x parent index are); `staged` = the block lies in the
// staged levels, and `blk` is its first slot there (staged_slot(first)).
__device__ __forceinline__ void load_child(const NodeEst* __restrict__ est, const float4* blk, bool staged,
                                           int64_t first, int c, float4& ea, float4& eb, float4& ec) {
    if (staged) {
        ea = blk[3 * c];
        eb = blk[3 * c + 1];
        ec = blk[3 * c + 2];
    } else {
        const NodeEst* e = est + first + c;
        ea = __ldg(&e->a);
        eb = __ldg(&e->b);
        ec = __ldg(&e->c);
    }
}

// Sums (v[0..NV)) over the lanes of the warp that hold the same key (all 32
// lanes call it): a pairwise tree over the members' ranks (fixed order, so
// deterministic).  Returns the lane's rank in its group; rank 0 holds the
// group's sums.  The registration descent sums 64-bit fixed-point values
// (exact: the node totals depend neither on the order in which groups arrive
// nor on how the points are grouped into warps).
template <int NV, typename V = float>
__device__ __forceinline__ int warp_group_sum(int key, V (&v)[NV]) {
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(FULL, key);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    const int gsize = __popc(peers);
    const int gmax = __reduce_max_sync(FULL, unsigned(gsize));
    const unsigned higher = lane == 31 ? 0u : (peers & ~((2u << lane) - 1u));
    // the member st ranks above this lane (this lane if there is none): the
    // next member, then doubled by one shuffle per step (the member 2 st
    // above is the one st above the member st above), valid wherever it is
    // used (rank + st < gsize)
    int nxt = higher ? __ffs(higher) - 1 : lane;
#pragma unroll
    for (int st = 1; st < 32; st <<= 1) {
        if (st >= gmax) break;  // warp-uniform: no group has a member st above
        V o[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) o[q] = __shfl_sync(FULL, v[q], nxt);
        if ((rank & (2 * st - 1)) == 0 && rank + st < gsize) {
#pragma unroll
            for (int q = 0; q < NV; ++q) v[q] += o[q];
        }
        nxt = __shfl_sync(FULL, nxt, nxt);
    }
    return rank;
}

// KEYS: key_out (if not null) receives each point's chosen node (all ones:
// none), for the source reorder between the first and the second round.
// hist (shared memory, 4 x STAGED_NODES fixed-point words, zero on entry, or
// null): the groups whose node is one of the staged top levels add into the
// CTA's own histogram instead of global memory; flush_node_hist then moves it
// to the global accumulators with one atomic per touched word.  The top
// levels are where most points stop on large planar structures, so this
// keeps thousands of warps from serialising on a few hot addresses.
template <bool KEYS = false>
__device__ __forceinline__ void descend_points(const float4* __restrict__ src, int n,
                                               const NodeEst* __restrict__ est, const float4* sm_est,
                                               int depth, const float* Rt_sm, float qscale,
                                               unsigned long long* __restrict__ acc, int cta, int ncta,
                                               unsigned long long* hist = nullptr,
                                               uint32_t* __restrict__ key_out = nullptr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float r00 = Rt_sm[0], r01 = Rt_sm[1], r02 = Rt_sm[2], r10 = Rt_sm[3], r11 = Rt_sm[4];
    const float r12 = Rt_sm[5], r20 = Rt_sm[6], r21 = Rt_sm[7], r22 = Rt_sm[8];
    const float tx = Rt_sm[9], ty = Rt_sm[10], tz = Rt_sm[11];
    const int wpb = blockDim.x >> 5;
    // 32-point chunks dealt round-robin to the CTAs (chunk j to CTA j mod
    // ncta), then to the CTA's warps: every CTA, and so every SM, gets the
    // same number of chunks to within one, drawn from the whole cloud (the
    // descent's depth, and so a chunk's cost, varies along a scan)
    const int nchunk = (n + 31) >> 5;
    for (int ch = cta + ncta * warp; ch < nchunk; ch += ncta * wpb) {
        const int base = ch * 32;
        const int i = base + lane;
        const bool valid = i < n;
        float4 z = valid ? src[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float x = fmaf(r00, z.x, fmaf(r01, z.y, fmaf(r02, z.z, tx)));
        const float y = fmaf(r10, z.x, fmaf(r11, z.y, fmaf(r12, z.z, ty)));
        const float w = fmaf(r20, z.x, fmaf(r21, z.y, fmaf(r22, z.z, tz)));
        int chosen = -1;
        float gamma = 0.f, cmx = 0.f, cmy = 0.f, cmz = 0.f;
        int local = 0;  // index within its level of the current search node
        int off = 0;    // first node of the level (32-bit: a depth-5 tree has 37,448 nodes)
        for (int l = 0; l < depth && valid; ++l) {
            const int first = off + 8 * local;
            off = 8 * off + 8;  // the next level's first node
            float sc8[8];
            float best = -CUDART_INF_F;
            int bi = -1;
            float bstop = 0.f;  // the best child's stop flag (its mean is read once, after the descent)
            // one child's log2 score from its three records, and the running argmax
            auto score = [&](int c, const float4 ea, const float4 eb, const float4 ec) {
                const float ex = x - ea.x, ey = y - ea.y, ez = w - ea.z;
                const float d0 = eb.x * ex;
                const float d1 = fmaf(eb.z, ey, eb.y * ex);
                const float d2 = fmaf(ec.y, ez, fmaf(ec.x, ey, eb.w * ex));
                float sc = fmaf(-d0, d0, ea.w);
                sc = fmaf(-d1, d1, sc);
                sc = fmaf(-d2, d2, sc);
                sc8[c] = sc;
                if (sc > best) {
                    best = sc;
                    bi = c;
                    bstop = ec.z;
                }
            };
            // the staged levels (the same level for every lane still
            // descending) read shared memory, deeper levels the cache
            if (first < STAGED_NODES) {
                const float4* blk = sm_est + staged_slot(first);
#pragma unroll
                for (int c = 0; c < 8; ++c) score(c, blk[3 * c], blk[3 * c + 1], blk[3 * c + 2]);
            } else {
                const NodeEst* e = est + first;
#pragma unroll
                for (int c = 0; c < 8; ++c) score(c, __ldg(&e[c].a), __ldg(&e[c].b), __ldg(&e[c].c));
            }
            if (bi < 0) break;  // the current node has no live children
            float sum = 0.f;
#pragma unroll
            for (int c = 0; c < 8; ++c) sum += ex2_fast(sc8[c] - best);
            gamma = rcp_fast(sum);
            chosen = first + bi;
            local = 8 * local + bi;
            if (bstop != 0.f) break;  // Complexity <= lambda_c
        }
        const bool has = chosen >= 0;
        if (has) {
            const float4 cm = chosen < STAGED_NODES ? sm_est[staged_slot(chosen)] : __ldg(&est[chosen].a);
            cmx = cm.x; cmy = cm.y; cmz = cm.z;
        }
        if (KEYS && key_out && valid) key_out[i] = has ? uint32_t(chosen) : 0xFFFFFFFFu;  // the point's node
        // each point's moments as fixed-point integers before any sum: the
        // per-warp group sums and the node totals are then exact integer
        // sums, independent of the order of the points
        long long q[4] = {0, 0, 0, 0};
        if (has) {
            q[0] = to_fix(gamma * 4294967296.0f);
            q[1] = to_fix(gamma * (x - cmx) * qscale);
            q[2] = to_fix(gamma * (y - cmy) * qscale);
            q[3] = to_fix(gamma * (w - cmz) * qscale);
        }
        int rank;
        if (__all_sync(FULL, chosen == __shfl_sync(FULL, chosen, 0))) {
            // one group (every point of the warp chose the same node, as
            // most do once the source is in node order): warp reductions of
            // two biased limbs per value, q + 2^40 = l0 + 2^21 l1 with
            // l0 < 2^21, l1 <= 2^20, so the 32-lane sums stay below 2^26:
            // the same exact integer totals as the group tree
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const unsigned long long u = (unsigned long long)(q[v] + (1ll << 40));
                const unsigned s0 = __reduce_add_sync(FULL, unsigned(u) & 0x1FFFFFu);
                const unsigned s1 = __reduce_add_sync(FULL, unsigned(u >> 21));
                q[v] = (long long)s0 + ((long long)s1 << 21) - (32ll << 40);
            }
            rank = lane;
        } else {
            rank = warp_group_sum<4, long long>(chosen, q);
        }
        if (has && rank == 0) {
            unsigned long long* dst =
                (hist && chosen < STAGED_NODES)
                    ? hist + 4 * chosen
                    : acc + 4 * (int64_t(chosen) * ACC_REPLICAS + (cta & (ACC_REPLICAS - 1)));
            atomicAdd(dst + 0, (unsigned long long)q[0]);
            atomicAdd(dst + 1, (unsigned long long)q[1]);
            atomicAdd(dst + 2, (unsigned long long)q[2]);
            atomicAdd(dst + 3, (unsigned long long)q[3]);
        }
    }
}

// Add the CTA's histogram of the staged levels to the global accumulators
// (integer adds: exact and order-free) and clear it.  Call after a
// __syncthreads that follows descend_points.
__device__ __forceinline__ void flush_node_hist(unsigned long long* hist, int n_staged,
                                                unsigned long long* __restrict__ acc) {
    static_assert(ACC_REPLICAS == 1, "one accumulator copy per node");
    for (int i = threadIdx.x; i < 4 * n_staged; i += blockDim.x) {
        const unsigned long long v = hist[i];
        if (v) {
            atomicAdd(acc + i, v);
            hist[i] = 0ull;
        }
    }
}

// Per-node contribution to the 6x6 normal equations in FP32; the sums over
// nodes are compensated (TwoSum pairs), so the totals that reach the FP64
// solve carry ~2x FP32 precision.  Per node j with mass (M0 > 0):
//   mu* = mu_j32 + o,  o = (M1 rel. to mu_j32) / M0,   d = mu_j - mu* = dmu_j - o
//   H_j = pi* [[A [mu*]x^T, A], [A^T, P]],  A = [mu*]x P,   g_j = pi* [mu* x P d; P d]
// and the node's share of the Eq. 11 objective at the current pose,
//   pi* d^T P d = pi* sum_l (n_l^T d)^2 / lambda_l.
// Layout of v (NTERM floats): 21 upper-packed H entries, 6 of g, the objective.

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
    v[27] = pis * (d0 * Pd[0] + d1 * Pd[1] + d2 * Pd[2]);
    (void)M0;
}

// One level of a warp reduce-scatter of 32 compensated (sum, error) pairs:
// the lane keeps the half of its 2*O-long valid prefix selected by
// bit O of its lane index and adds the partner's copy of that half.
template <int O>
__device__ __forceinline__ void rs_level(float (&v)[32], float (&c)[32], int lane) {
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < O; ++i) {
        const float ss = up ? v[i] : v[i + O];
        const float cs = up ? c[i] : c[i + O];
        float sk = up ? v[i + O] : v[i];
        float ck = up ? c[i + O] : c[i];
        const float sr = __shfl_xor_sync(FULL, ss, O);
        const float cr = __shfl_xor_sync(FULL, cs, O);
        pair_add(sk, ck, sr, cr);
        v[i] = sk;
        c[i] = ck;
    }
}

// Warp totals of 32 per-lane (sum, error) pairs (term t in v[t], c[t]): after
// the five levels lane l holds the warp total of term l in (s, e).  31 pair
// additions per lane instead of 160 for a butterfly over every term; the
// tree over lanes is fixed, so the result is deterministic.
__device__ __forceinline__ void warp_reduce_scatter32(float (&v)[32], float (&c)[32], float& s, float& e) {
    const int lane = threadIdx.x & 31;
    rs_level<16>(v, c, lane);
    rs_level<8>(v, c, lane);
    rs_level<4>(v, c, lane);
    rs_level<2>(v, c, lane);
    rs_level<1>(v, c, lane);
    s = v[0];
    e = c[0];
}

__host__ __device__ constexpr int up6(int i, int j) { return i * 6 - (i * (i - 1)) / 2 + (j - i); }

// FP64 solve of the 6x6 normal equations H x = g (Eq. 16) and the pose update
// by one warp.  One FP64 warp instruction holds this part's FP64 pipe for ~70
// cycles whatever the active mask, so the solve is laid out to issue few of
// them: lane L < 21 holds upper-packed entry L of H, lanes 21..26 hold g (the
// layout of tot), and symmetric Gaussian elimination without pivoting (H is
// positive definite) updates every entry of the trailing block and of g with
// one multiply and one FMA per pivot; back substitution runs on the g lanes
// (rows scaled by their pivot's reciprocal: one FMA per step).  Pivots are
// checked with integer compares of their bit patterns (positive, finite,
// above 1e-15 of the largest diagonal, inside [2^-1000, 2^1000]).
// T <- dR T + dt with dR from Rodrigues' formula, all in FP64.  Returns false
// (uniformly) for a failed pivot, leaving T unchanged.
// T_SHARED: T (and Rt) live in this CTA's shared memory (every CTA of the
// registration solves the same system itself, so the pose needs no
// publication); T_copy / Rt_copy, if given, receive the new pose too (the
// global copies one CTA keeps for the caller).
template <bool T_SHARED = false>
__device__ __forceinline__ bool warp_solve_update(const double* tot, double* T, float* Rt, double* T_hist,
                                         int iter, double* T_copy = nullptr, float* Rt_copy = nullptr) {
    const int lane = threadIdx.x & 31;
    // (row, column) of this lane's entry; column 6 = right-hand side, row -1 = idle
    int ri = -1, rj = 0;
    if (lane < 21) {
        int k = lane;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            if (ri < 0 && k < 6 - i) {
                ri = i;
                rj = i + k;
            }
            if (ri < 0) k -= 6 - i;
        }
    } else if (lane < 27) {
        ri = lane - 21;
        rj = 6;
    }
    double a = lane < 27 ? tot[lane] : 0.0;
    // this lane's column of the current pose, loaded now so that the L2
    // latency overlaps the elimination (entry (rr, cc) below)
    // (lanes 16..27 hold the same entries as lanes 0..11: the pose update
    // below splits its dot products and series between the two halves)
    const int e = (lane & 15) < 12 ? (lane & 15) : 11;
    const int rr = e >> 2, cc = e & 3;
    const double t0 = T_SHARED ? T[cc] : __ldcg(T + cc);
    const double t1 = T_SHARED ? T[4 + cc] : __ldcg(T + 4 + cc);
    const double t2 = T_SHARED ? T[8 + cc] : __ldcg(T + 8 + cc);
    // pivot threshold from the largest diagonal entry, in FP32
    float dm = (ri >= 0 && rj == ri) ? float(a) : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dm = fmaxf(dm, __shfl_xor_sync(FULL, dm, o));
    const long long thr = __double_as_longlong(double(1e-15f * dm));
    double r[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double p = __shfl_sync(FULL, a, up6(k, k));
        const long long pb = __double_as_longlong(p);
        // a pivot must be positive, above the threshold and inside
        // [2^-1000, 2^1000] (far beyond any scale the terms reach)
        if (!(pb > thr && pb > 0x0170000000000000LL && pb < 0x7E70000000000000LL)) return false;
        // reciprocal: the multi-function unit's FP64 approximation
        // (rcp.approx.ftz.f64; measured on this part: relative error below
        // 2^-19.9) refined by one third-order step of the iteration for 1/p,
        // r (1 + e + e^2) with e = 1 - p r (error e^3 < 2^-59, below FP64
        // rounding; a Newton step, r (1 + e), would stop at 2^-39.8): no
        // FP32 <-> FP64 conversions and no division subroutine on the
        // elimination's critical path
        double rp;
        asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(rp) : "d"(p));
        {
            const double e = fma(-p, rp, 1.0);
            rp = fma(rp, fma(e, e, e), rp);
        }
        r[k] = rp;
        const bool upd = ri > k;
        const int s1 = upd ? up6(k, ri) : 0;
        const int s2 = upd ? (rj < 6 ? up6(k, rj) : 21 + k) : 0;
        const double aki = __shfl_sync(FULL, a, s1);
        const double akj = __shfl_sync(FULL, a, s2);
        // a_ij -= (a_ki a_kj) / p: the product does not wait for the
        // reciprocal, so one FMA follows it on the chain
        const double t = aki * akj;
        if (upd) a = fma(-t, rp, a);
    }
    // back substitution on rows scaled by their pivot's reciprocal (one
    // multiply on every lane): W_ik = U_ik / U_ii, c_i = b'_i / U_ii, then
    // x_k = c_k and c_i -= W_ik x_k (i < k), one FMA per step
    double rri = r[0];
#pragma unroll
    for (int k = 1; k < 6; ++k) rri = ri == k ? r[k] : rri;
    a *= rri;
    double x[6];
#pragma unroll
    for (int k = 5; k >= 0; --k) {
        const double xk = __shfl_sync(FULL, a, 21 + k);
        x[k] = xk;
        const bool upd = rj == 6 && ri < k;
        const double wik = __shfl_sync(FULL, a, upd ? up6(ri, k) : 0);
        if (upd) a = fma(-wik, xk, a);
    }
    // dR = I + a K + b K^2 (Rodrigues), K = [w]x, K^2 = w w^T - |w|^2 I, in
    // FP64: a and b must keep their exact trigonometric relation or dR drifts
    // off the rotation group.  Lane e < 12 forms entry (r, c) of
    // dR T + dt = T + a K T + b (w (w^T T) - |w|^2 T) + dt without forming dR.
    // Every FP64 warp instruction costs the same whatever its lanes do, so
    // the three dot products share one FMA chain (lanes 0..11: (w^T T)_c,
    // lanes 16..27: (K T)_rc, lane 12: |w|^2) and a and b one series
    // (lanes 0..15: a, lanes 16..31: b).
    const bool hi = lane >= 16;
    const double trc = rr == 0 ? t0 : (rr == 1 ? t1 : t2);
    double p0, p1, p2, q0, q1, q2;
    if (lane == 12) {
        p0 = q0 = x[0]; p1 = q1 = x[1]; p2 = q2 = x[2];
    } else if (hi) {
        // (K T)_rc: row r of K = [w]x has one zero
        p0 = rr == 0 ? -x[2] : (rr == 1 ? x[2] : -x[1]);
        p1 = rr == 0 ? x[1] : (rr == 1 ? -x[0] : x[0]);
        q0 = rr == 0 ? t1 : t0;
        q1 = rr == 0 ? t2 : (rr == 1 ? t2 : t1);
        p2 = 0.0; q2 = 0.0;
    } else {
        p0 = x[0]; p1 = x[1]; p2 = x[2];
        q0 = t0; q1 = t1; q2 = t2;
    }
    const double dot = fma(p0, q0, fma(p1, q1, p2 * q2));
    const double th2 = __shfl_sync(FULL, dot, 12);
    const double kt = __shfl_sync(FULL, dot, e + 16);
    const double wt = dot;  // (w^T T)_c on lanes 0..11
    double ser;
    if (th2 < 1e-4) {  // series truncated after th2^2: error < th2^3 / 5040
        ser = fma(th2, fma(th2, hi ? 1.0 / 720 : 1.0 / 120, hi ? -1.0 / 24 : -1.0 / 6), hi ? 0.5 : 1.0);
    } else if (th2 < 0.25) {
        // a = sum_k (-th2)^k / (2k+1)!, b = sum_k (-th2)^k / (2k+2)!, k <= 6
        ser = hi ? 1.0 / 87178291200.0 : 1.0 / 6227020800.0;
        ser = fma(th2, ser, hi ? -1.0 / 479001600 : -1.0 / 39916800);
        ser = fma(th2, ser, hi ? 1.0 / 3628800 : 1.0 / 362880);
        ser = fma(th2, ser, hi ? -1.0 / 40320 : -1.0 / 5040);
        ser = fma(th2, ser, hi ? 1.0 / 720 : 1.0 / 120);
        ser = fma(th2, ser, hi ? -1.0 / 24 : -1.0 / 6);
        ser = fma(th2, ser, hi ? 0.5 : 1.0);
    } else {
        const double th = sqrt(th2);
        ser = hi ? (1.0 - cos(th)) / th2 : sin(th) / th;
    }
    const double ca = ser;
    const double cb = __shfl_sync(FULL, ser, e + 16);
    const double wr = rr == 0 ? x[0] : (rr == 1 ? x[1] : x[2]);
    const double u = fma(wr, wt, -th2 * trc);
    const double xt = rr == 0 ? x[3] : (rr == 1 ? x[4] : x[5]);
    double acc = trc + (cc == 3 ? xt : 0.0);
    acc = fma(ca, kt, acc);
    acc = fma(cb, u, acc);
    __syncwarp();
    if (lane < 12) {
        T[e] = acc;
        Rt[cc == 3 ? 9 + rr : rr * 3 + cc] = float(acc);
        if (T_copy) T_copy[e] = acc;
        if (Rt_copy) Rt_copy[cc == 3 ? 9 + rr : rr * 3 + cc] = float(acc);
        if (T_hist) T_hist[16 * iter + e] = acc;
    }
    if (T_hist && lane >= 12 && lane < 16) T_hist[16 * iter + lane] = lane == 15 ? 1.0 : 0.0;
    return true;
}

// Fixed-order sum of nb per-CTA partials of the NTERM normal-equation and
// objective terms (compensated pairs) by a CTA of at least 8 warps (warp w
// takes partials w, w + 8, ...; then the eight group sums in order), the
// objective to *obj, and the FP64 solve and pose update by warp 0.  A
// singular system records ST_DEGENERATE and keeps T (also in T_hist).
__device__ inline void sum_terms_and_solve(const float2* __restrict__ tpart, int nb, int it, double* T,
                                           float* Rt, double* T_hist, double* obj, int* status) {
    __shared__ float2 fin[8][32];
    __shared__ double tot[NTERM];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < 8) {
        float S = 0.f, C = 0.f;
        if (lane < NTERM)
            for (int b = warp; b < nb; b += 8) {
                const float2 x = tpart[NTERM * b + lane];
                pair_add(S, C, x.x, x.y);
            }
        fin[warp][lane] = make_float2(S, C);
    }
    __syncthreads();
    if (warp != 0) return;
    if (lane < NTERM) {
        float S = 0.f, C = 0.f;
        for (int w = 0; w < 8; ++w) pair_add(S, C, fin[w][lane].x, fin[w][lane].y);
        tot[lane] = double(S) + double(C);
    }
    __syncwarp();
    if (lane == 0 && obj) *obj = tot[NTERM - 1];
    const bool solved = warp_solve_update(tot, T, Rt, T_hist, it);
    if (!solved && lane == 0) {
        atomicOr(status, ST_DEGENERATE);
        if (T_hist)
            for (int k = 0; k < 16; ++k) T_hist[16 * it + k] = T[k];
    }
}

// Thread 0 waits (bounded) until *word - target >= 0 (a monotonic counter or
// generation), then the CTA proceeds; on timeout it records ST_TIMEOUT and
// every thread of the CTA gets false.  The acquire side of a release made by
// the CTA that advanced the word (a fence before its atomic or store).
// sleep_ns > 0 backs off between polls (many CTAs polling one word slow
// down the CTA that will advance it); the limit then counts polls.
__device__ __forceinline__ bool wait_at_least(const unsigned* word, unsigned target, int* status,
                                              long long limit, unsigned sleep_ns = 0) {
    __shared__ int ok_wait;
    if (threadIdx.x == 0) {
        const volatile unsigned* v = word;
        int ok = 1;
        long long spins = 0;
        while (int(*v - target) < 0) {
            if (++spins > limit) {
                atomicOr(status, ST_TIMEOUT);
                ok = 0;
                break;
            }
            if (sleep_ns) __nanosleep(sleep_ns);
        }
        __threadfence();
        ok_wait = ok;
    }
    __syncthreads();
    return ok_wait != 0;
}

// One thread adds one to a monotonic counter as a release (after a
// __syncthreads): the CTA's earlier global writes and atomics are visible to
// any thread that sees the new count through wait_acquire.  fence.acq_rel is
// the lighter release fence of the PTX memory model (no sequentially
// consistent order is needed here); it is cumulative over the barrier.
__device__ __forceinline__ void arrive_release(unsigned* word) {
    asm volatile("fence.acq_rel.gpu;\n\tred.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(word) : "memory");
}

// wait_at_least with relaxed polls and one acquire fence once the count is
// reached (the counterpart of arrive_release); bounded, ST_TIMEOUT on expiry.
__device__ __forceinline__ bool wait_acquire(const unsigned* word, unsigned target, int* status,
                                             long long limit) {
    __shared__ int ok_acq;
    if (threadIdx.x == 0) {
        int ok = 1;
        long long spins = 0;
        unsigned v;
        for (;;) {
            asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(word) : "memory");
            if (int(v - target) >= 0) break;
            if (++spins > limit) {
                atomicOr(status, ST_TIMEOUT);
                ok = 0;
                break;
            }
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        ok_acq = ok;
    }
    __syncthreads();
    return ok_acq != 0;
}

// Grid-wide barrier of a cooperative launch on a monotonic arrival counter
// (zeroed before the launch): every CTA adds one and waits until the counter
// reaches target = (barriers passed so far) x gridDim.x.  Arrivals are
// non-returning atomics and no word is ever reset, so no CTA can miss a
// release; the wait is bounded (wait_at_least).
__device__ __forceinline__ bool grid_sync_count(unsigned* ctr, unsigned target, int* status,
                                                long long limit) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
    }
    return wait_at_least(ctr, target, status, limit);
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


}  // namespace hgmm
