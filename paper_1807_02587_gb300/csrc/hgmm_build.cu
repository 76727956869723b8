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
//                     (parents of many items: per slice of their items, after
//                     k_offset_slices has summed each slice's counts)
//   k_scatter         stable 8-way partition of every parent's segment
//   k_finalize        FP64 eigen, complexity, precision matrix of level l
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "hgmm_dev.cuh"
#include "hgmm_async.cuh"

namespace hgmm {

namespace {

// Whole-cloud root statistics: every CTA writes a partial; the last CTA to
// finish reduces them in a fixed order and writes the FP64 root record.
__global__ void __launch_bounds__(256) k_root(const float4* __restrict__ pts, int n,
                                              float eps_rel, float* __restrict__ part,
                                              unsigned* __restrict__ counter,
                                              RootDev* __restrict__ root, int* __restrict__ status) {
    __shared__ RootSmem rs;
    __shared__ bool last;
    root_partial_cta(pts, n, blockIdx.x, gridDim.x, part + 32 * blockIdx.x, rs);
    if (threadIdx.x == 0) {
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    root_final_cta(part, gridDim.x, pts, n, eps_rel, root, status, rs);
    if (threadIdx.x == 0) *counter = 0u;
}

// One CTA per parent; threads 0..7 build child c.
__global__ void k_init_children(int level, const RootDev* __restrict__ root,
                                NodeStat* __restrict__ stat, NodeEst* __restrict__ est,
                                const int* __restrict__ seg_count, int* __restrict__ status) {
    if (threadIdx.x < 8) init_child(level, blockIdx.x, threadIdx.x, root, stat, est, seg_count, status);
}

__global__ void __launch_bounds__(1024) k_make_items(int level, int n, int n_parents,
                                                     const int* __restrict__ seg_count,
                                                     int* __restrict__ item_range,
                                                     int* __restrict__ meta, int est_grid) {
    __shared__ int warp_tot[33];
    make_items_cta(level, n, n_parents, seg_count, item_range, meta, est_grid, warp_tot);
}

// One thread per item: materialise the item list.
__global__ void k_fill_items(int level, int n, int n_parents, const int* __restrict__ seg_start,
                             const int* __restrict__ seg_count,
                             const int* __restrict__ item_range, const int* __restrict__ meta,
                             Item* __restrict__ items) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= meta[0]) return;
    items[j] = item_at(j, level, n, n_parents, item_range, seg_start, seg_count);
}

// The level-wide E-step: the arithmetic of estep_range (so the result is
// the same bit for bit), with each item's points (one contiguous run of at
// most TILE float4) brought into shared memory by one bulk asynchronous copy,
// ESTEP_STAGES items ahead of the compute, so that no warp waits on a global
// load.  One thread issues the copies; each completes on its stage's
// mbarrier; a stage is refilled after the CTA's barrier at the end of the
// item that used it (with an async-proxy fence).  All waits are bounded: on
// a timeout the CTA records ST_TIMEOUT, waits (bounded) for its copies in
// flight and stops.
constexpr int ESTEP_STAGES = 4;
// Dynamic shared memory of k_estep: the compensated sums (s, c) of every
// lane's ten packed moment pairs, [value][thread], kept out of the register
// file so that three CTAs fit on an SM.
constexpr size_t ESTEP_DYN_SMEM = size_t(2) * 10 * EST_THREADS * sizeof(float2);

// fold_pair with the compensated sums in shared memory (the same arithmetic).
template <bool COMP>
__device__ __forceinline__ void fold_pair_smem(float2 (&in)[10], float2* acc_s, float2* acc_c) {
    const int t = threadIdx.x;
#pragma unroll
    for (int v = 0; v < 10; ++v) {
        float2 sv = acc_s[v * EST_THREADS + t];
        if (COMP) {
            float2 cv = acc_c[v * EST_THREADS + t];
            const float2 tt = __fadd2_rn(sv, in[v]);
            const float2 bp = sub2(tt, sv);
            const float2 e = __fadd2_rn(sub2(sv, sub2(tt, bp)), sub2(in[v], bp));
            sv = tt;
            cv = __fadd2_rn(cv, e);
            acc_c[v * EST_THREADS + t] = cv;
        } else {
            sv = __fadd2_rn(sv, in[v]);
        }
        acc_s[v * EST_THREADS + t] = sv;
        in[v] = make_float2(0.f, 0.f);
    }
}

template <bool COMP>
__device__ __forceinline__ void flush_pair_smem(float2* acc_s, float2* acc_c, float2 (*red)[NPART],
                                                float2* __restrict__ out) {
    float2 s2[10], c2[10];
    const int t = threadIdx.x;
#pragma unroll
    for (int v = 0; v < 10; ++v) {
        s2[v] = acc_s[v * EST_THREADS + t];
        c2[v] = COMP ? acc_c[v * EST_THREADS + t] : make_float2(0.f, 0.f);
        acc_s[v * EST_THREADS + t] = make_float2(0.f, 0.f);
        acc_c[v * EST_THREADS + t] = make_float2(0.f, 0.f);
    }
    flush_pair<COMP>(s2, c2, red, out);
}

// The level-wide E-step: the arithmetic of estep_range (so the result is
// the same bit for bit), with each item's points (one contiguous run of at
// most TILE float4) brought into shared memory by one bulk asynchronous copy,
// ESTEP_STAGES items ahead of the compute, so that no warp waits on a global
// load, and the compensated sums in shared memory.  One thread issues the
// copies; each completes on its stage's mbarrier; a stage is refilled after
// the CTA's barrier at the end of the item that used it (with an async-proxy
// fence).  All waits are bounded: on a timeout the CTA records ST_TIMEOUT,
// waits (bounded) for its copies in flight and stops.
template <bool COMP>
__global__ void __launch_bounds__(EST_THREADS, 3)
k_estep(const float4* __restrict__ pts, const Item* __restrict__ items,
        const int* __restrict__ meta, const NodeEst* __restrict__ est_lvl,
        float2* __restrict__ partials, int* __restrict__ status) {
    __shared__ float2 red[EST_THREADS / 32][NPART];
    __shared__ __align__(16) float4 stage[ESTEP_STAGES][TILE];
    __shared__ __align__(8) uint64_t full[ESTEP_STAGES];
    extern __shared__ float2 estep_dyn[];
    float2* acc_s = estep_dyn;
    float2* acc_c = estep_dyn + 10 * EST_THREADS;
    const int n_items = meta[0];
    const int C = meta[1];
    const int ib = blockIdx.x * C, ie = min(ib + C, n_items);
    if (ib >= ie) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane >> 2, k = lane & 3;
    for (int v = 0; v < 10; ++v) {
        acc_s[v * EST_THREADS + threadIdx.x] = make_float2(0.f, 0.f);
        acc_c[v * EST_THREADS + threadIdx.x] = make_float2(0.f, 0.f);
    }
    if (threadIdx.x == 0) {
        for (int st = 0; st < ESTEP_STAGES; ++st) tc::mbar_init(&full[st], 1);
        tc::fence_mbar_init();
        for (int it = ib; it < min(ie, ib + ESTEP_STAGES); ++it) {
            const Item w = items[it];
            const int st = (it - ib) % ESTEP_STAGES;
            tc::mbar_arrive_expect_tx(&full[st], uint32_t(w.count) * 16u);
            tc::bulk_g2s(tc::smem_u32(stage[st]), pts + w.start, uint32_t(w.count) * 16u, &full[st]);
        }
    }
    __syncthreads();
    float2 in[10];
#pragma unroll
    for (int v = 0; v < 10; ++v) in[v] = make_float2(0.f, 0.f);
    int nfold = 0;
    int cur = -1, run = -1;
    bool live = false;
    ChildPair cp;
    int it = ib;
    for (; it < ie; ++it) {
        const Item w = items[it];
        if (w.parent != cur) {
            if (cur >= 0) {
                fold_pair_smem<COMP>(in, acc_s, acc_c);
                nfold = 0;
                flush_pair_smem<COMP>(acc_s, acc_c, red, partials + int64_t(run) * NPART);
            }
            cur = w.parent;
            run = it;
            load_child_pair(est_lvl + 8 * cur + 2 * k, cp);
            live = parent_has_live_child(cp);
        }
        const int st = (it - ib) % ESTEP_STAGES;
        const uint32_t parity = uint32_t((it - ib) / ESTEP_STAGES) & 1u;
        // a thread whose wait ran out computes on whatever the stage holds
        // (in bounds, discarded): the CTA's vote at the end of the item stops it
        const bool landed = tc::mbar_wait_bounded(&full[st], parity, tc::MBAR_SPIN_LIMIT);
        const float4* zs = stage[st];
        // a parent without a live child: zero posteriors, nothing to add
        for (int base = 0; live && base < w.count; base += 64) {
            const int idx = base + warp * 8 + q;
            const bool valid = idx < w.count;
            const float4 z = zs[min(idx, w.count - 1)];
            estep_point_pair(cp, z, valid, in);
            if (++nfold == EST_FOLD) {
                fold_pair_smem<COMP>(in, acc_s, acc_c);
                nfold = 0;
            }
        }
        // every thread is done with this stage (one barrier per item, which
        // also carries the timeout vote)
        if (__syncthreads_or(!landed)) {
            if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
            break;
        }
        if (threadIdx.x == 0 && it + ESTEP_STAGES < ie) {
            const Item wn = items[it + ESTEP_STAGES];
            tc::fence_proxy_async();
            tc::mbar_arrive_expect_tx(&full[st], uint32_t(wn.count) * 16u);
            tc::bulk_g2s(tc::smem_u32(stage[st]), pts + wn.start, uint32_t(wn.count) * 16u, &full[st]);
        }
    }
    if (it < ie) {
        // timed out: let the copies in flight land (bounded) before the CTA
        // and its shared memory go away
        if (threadIdx.x == 0)
            for (int j = it; j < min(ie, it + ESTEP_STAGES); ++j)
                tc::mbar_wait_bounded(&full[(j - ib) % ESTEP_STAGES], uint32_t((j - ib) / ESTEP_STAGES) & 1u,
                                      tc::MBAR_SPIN_LIMIT);
        return;
    }
    fold_pair_smem<COMP>(in, acc_s, acc_c);
    flush_pair_smem<COMP>(acc_s, acc_c, red, partials + int64_t(run) * NPART);
}

// The level-wide M-step: CTA (p, j) reduces slice j of parent p's runs into
// the slice buffer; the last of the parent's n_slices CTAs to finish
// (arrival counter, reset by that CTA) combines the slices in order and runs
// the FP64 M-step of the 8 children.
template <bool COMP>
__global__ void __launch_bounds__(256) k_mstep(int level, int n, const int* __restrict__ item_range,
                                               const int* __restrict__ meta,
                                               const float2* __restrict__ partials,
                                               const int* __restrict__ seg_count,
                                               const RootDev* __restrict__ root, float n_min,
                                               NodeStat* __restrict__ stat,
                                               NodeEst* __restrict__ est, int* __restrict__ status,
                                               float2* __restrict__ slices, unsigned* __restrict__ mcnt) {
    __shared__ MstepSmem msm;
    __shared__ float2 own[NPART];
    __shared__ bool last;
    const int p = blockIdx.x, j = blockIdx.y, ns = gridDim.y;
    const int i0 = item_range[2 * p], i1 = item_range[2 * p + 1];
    if (i0 >= i1) return;  // parent without points: children stay dead
    if (ns == 1) {
        reduce_run_slice<COMP>(i0, i1, meta[1], 0, 1, partials, msm, own);
        mstep_from_slices<COMP, false>(level, n, p, own, 1, seg_count, root, n_min, stat, est, status, msm);
        return;
    }
    float2* mine = slices + (int64_t(p) * ns + j) * NPART;
    reduce_run_slice<COMP>(i0, i1, meta[1], j, ns, partials, msm, mine);
    if (threadIdx.x < NPART) __threadfence();  // each writer's slice values before the arrival
    __syncthreads();
    if (threadIdx.x == 0) {
        last = atomicAdd(mcnt + p, 1u) == unsigned(ns - 1);
        if (last) {
            mcnt[p] = 0u;  // every slice has arrived: ready for the next launch
            __threadfence();
        }
    }
    __syncthreads();
    if (!last) return;
    mstep_from_slices<COMP, true>(level, n, p, slices + int64_t(p) * ns * NPART, ns, seg_count, root, n_min, stat,
                                  est, status, msm);
}

// All K EM iterations of one parent by one CTA (blockIdx.x = parent): the
// E-step over the parent's items as a single run (its moments kept in shared
// memory), then the M-step of its 8 children, with nothing but
// __syncthreads between them (the parents of a
// level are independent during EM).  For levels with many small parents,
// where the level-wide E-step / M-step launches would be mostly latency.
template <bool COMP>
__global__ void __launch_bounds__(EST_THREADS, 2) k_em_local(int level, int n, int K,
                                                            const float4* __restrict__ pts,
                                                            const Item* __restrict__ items,
                                                            const int* __restrict__ item_range,
                                                            const int* __restrict__ seg_count,
                                                            const RootDev* __restrict__ root, float n_min,
                                                            NodeStat* __restrict__ stat,
                                                            NodeEst* __restrict__ est,
                                                            int* __restrict__ status) {
    __shared__ union {
        float2 red[EST_THREADS / 32][NPART];
        MstepSmem msm;
    } sm;
    __shared__ float2 run_sm[NPART];
    const int p = blockIdx.x;
    const int i0 = item_range[2 * p], i1 = item_range[2 * p + 1];
    if (i0 >= i1) return;  // parent without points: children stay dead
    const NodeEst* est_lvl = est + level_offset(level);
    for (int k = 0; k < K; ++k) {
        // [i0, i1) is one run: its partial stays in shared memory (the
        // flush ends with a block barrier)
        estep_range<COMP, ItemList, false, true>(pts, ItemList{items}, i0, i1, est_lvl, run_sm, sm.red);
        // the moments mstep_parent forms from a single run: sum + compensation
        if (threadIdx.x < NPART) sm.msm.mom[threadIdx.x] = double(run_sm[threadIdx.x].x) + double(run_sm[threadIdx.x].y);
        __syncthreads();
        if (threadIdx.x < 32)
            child_mstep_quad(level, n, p, sm.msm.mom, seg_count, root, n_min, stat, est, status);
        __syncthreads();
    }
}

// All K EM iterations of one level in one cooperative launch (levels whose
// parents are few, or large).  Per iteration every CTA runs the E-step of
// its chunk of items, reading the children's constants through L2 (they
// change between iterations), and adds one arrival to each parent its chunk
// touched; the CTA owning parent p (p mod gridDim) waits for all of p's runs,
// runs the same fixed-order reduction and FP64 M-step as k_mstep and counts
// p as done; the next iteration starts once every parent is done.  The
// arithmetic is that of k_estep + k_mstep, so the result is the same bit
// for bit.  cnt: n_par arrival counters, then the done counter, all zero at
// launch and monotonic; every wait is bounded (ST_TIMEOUT, then return).
template <bool COMP>
__global__ void __launch_bounds__(EST_THREADS, 2)
k_em_coop(int level, int n, int n_par, int K, int n_chunks, const float4* __restrict__ pts,
          const Item* __restrict__ items, const int* __restrict__ meta, const int* __restrict__ item_range,
          float2* __restrict__ partials, const int* __restrict__ seg_count, const RootDev* __restrict__ root,
          float n_min, NodeStat* __restrict__ stat, NodeEst* __restrict__ est, unsigned* __restrict__ cnt,
          int* __restrict__ status) {
    __shared__ union {
        float2 red[EST_THREADS / 32][NPART];
        struct {
            MstepSmem msm;
            float2 slice[MSTEP_SLICES][NPART];
        };
    } sm;
    const int n_items = meta[0], C = meta[1];
    const NodeEst* est_lvl = est + level_offset(level);
    unsigned* done = cnt + n_par;
    for (int k = 0; k < K; ++k) {
        if (k > 0 && !wait_at_least(done, unsigned(k) * unsigned(n_par), status, BARRIER_SPIN_LIMIT, 128)) return;
        // the item chunks of the level-wide E-step (n_chunks of C items),
        // each an E-step over its items and one arrival per parent it touches
        for (int b = blockIdx.x; b < n_chunks; b += gridDim.x) {
            const int ib = b * C, ie = min(ib + C, n_items);
            if (ib >= ie) continue;
            estep_range<COMP, ItemList, true>(pts, ItemList{items}, ib, ie, est_lvl, partials, sm.red);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();  // the partials before the arrivals
                for (int p = items[ib].parent; p <= items[ie - 1].parent; ++p) atomicAdd(cnt + p, 1u);
            }
        }
        for (int p = blockIdx.x; p < n_par; p += gridDim.x) {
            const int i0 = item_range[2 * p], i1 = item_range[2 * p + 1];
            if (i0 < i1) {  // a parent without points has no runs; its children stay dead
                const unsigned runs = unsigned((i1 - 1) / C - i0 / C + 1);
                if (!wait_at_least(cnt + p, unsigned(k + 1) * runs, status, BARRIER_SPIN_LIMIT)) return;
                // the level-wide M-step's slices, reduced one after another
                const int ns = mstep_slices(n_par, n, n_chunks);
                for (int j = 0; j < ns; ++j)
                    reduce_run_slice<COMP>(i0, i1, C, j, ns, partials, sm.msm, sm.slice[j]);
                mstep_from_slices<COMP, false>(level, n, p, &sm.slice[0][0], ns, seg_count, root, n_min, stat, est,
                                               status, sm.msm);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();  // the children's new constants before the count
                atomicAdd(done, 1u);
            }
        }
    }
}

__global__ void __launch_bounds__(EST_THREADS) k_assign(const float4* __restrict__ pts,
                                                        const Item* __restrict__ items,
                                                        const int* __restrict__ meta,
                                                        const NodeEst* __restrict__ est_lvl,
                                                        uint32_t* __restrict__ codes,
                                                        int* __restrict__ item_cnt) {
    __shared__ AssignSmem as;
    const int n_items = meta[0];
    for (int it = blockIdx.x; it < n_items; it += gridDim.x)
        assign_item(pts, items[it], it, est_lvl, codes, item_cnt, as);
}

// Slice j of the nsl slices of a parent's items [i0, i1).
__device__ __forceinline__ void offset_slice(int i0, int i1, int nsl, int j, int& a, int& b) {
    const int per = (i1 - i0 + nsl - 1) / nsl;
    a = min(i1, i0 + j * per);
    b = min(i1, a + per);
}

// Parents with many items (the hand-off of large clouds' top levels): CTA
// (p, j) sums the item counts of slice j of parent p per child.
__global__ void __launch_bounds__(256) k_offset_slices(const int* __restrict__ item_range,
                                                       const int* __restrict__ item_cnt, int nsl,
                                                       int* __restrict__ slice_tot) {
    __shared__ int tot[8][8];
    const int p = blockIdx.x, j = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int a, b;
    offset_slice(item_range[2 * p], item_range[2 * p + 1], nsl, j, a, b);
    int t8[8] = {};
    for (int i = a + threadIdx.x; i < b; i += blockDim.x)
        for (int cc = 0; cc < 8; ++cc) t8[cc] += item_cnt[8 * i + cc];
    for (int cc = 0; cc < 8; ++cc) {
        int x = t8[cc];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(FULL, x, off);
        if (lane == 0) tot[warp][cc] = x;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        int x = 0;
        for (int w = 0; w < 8; ++w) x += tot[w][threadIdx.x];
        slice_tot[(int64_t(p) * nsl + j) * 8 + threadIdx.x] = x;
    }
}

// CTA (p, j) of 256 threads: the child segments of parent p and the item
// offsets of slice j of its items (nsl = 1: the whole parent in one CTA;
// nsl > 1: the slices' sums from k_offset_slices give each slice's start).
__global__ void __launch_bounds__(256) k_child_offsets(int level, int n,
                                                       const int* __restrict__ item_range,
                                                       const Item* __restrict__ items,
                                                       const int* __restrict__ item_cnt,
                                                       int* __restrict__ item_off,
                                                       int* __restrict__ seg_start,
                                                       int* __restrict__ seg_count, int nsl,
                                                       const int* __restrict__ slice_tot) {
    __shared__ OffsetSmem os;
    const int p = blockIdx.x, j = blockIdx.y;
    const int i0 = item_range[2 * p], i1 = item_range[2 * p + 1];
    // an empty parent's children get empty segments at the parent's start
    const int pstart = i0 < i1 ? items[i0].start
                               : (level == 0 ? 0 : seg_start[d_level_offset(level - 1) + p]);
    if (nsl == 1) {
        child_offsets_cta(level, p, i0, i1, pstart, item_cnt, item_off, seg_start, seg_count, os);
        return;
    }
    if (threadIdx.x == 0) {
        const int* st = slice_tot + int64_t(p) * nsl * 8;
        const int64_t g0 = d_level_offset(level) + 8 * int64_t(p);
        int run = pstart;
        for (int cc = 0; cc < 8; ++cc) {
            int tot = 0, pre = 0;
            for (int jj = 0; jj < nsl; ++jj) {
                if (jj == j) pre = tot;
                tot += st[8 * jj + cc];
            }
            os.carry[cc] = run + pre;
            if (j == 0) {
                seg_start[g0 + cc] = run;
                seg_count[g0 + cc] = tot;
            }
            run += tot;
        }
    }
    __syncthreads();
    int a, b;
    offset_slice(i0, i1, nsl, j, a, b);
    child_offsets_scan(a, b, item_cnt, item_off, os);
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
    for (int it = blockIdx.x; it < n_items; it += gridDim.x)
        scatter_item(pts_in, perm_in, items[it], it, codes, item_off, pts_out, perm_out,
                     threadIdx.x, blockDim.x);
}

__global__ void k_finalize(int level, float lam_c, const RootDev* __restrict__ root,
                           NodeStat* __restrict__ stat, NodeEst* __restrict__ est,
                           float4* __restrict__ rnode) {
    const int64_t m = int64_t(1) << (3 * (level + 1));
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < m) finalize_node(level, i, lam_c, root, stat, est, rnode);
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

// ------------------------------------------------------------ posteriors
// Eq. 3 posteriors of every point over the 8 children of its parent at
// `level` (the parent being the point's node of level - 1, or the root),
// from the level's final parameters, with the build's own FP32 scores
// (log2 domain, maximum subtracted).  A parent without a live child gives
// zero posteriors, as in the build's E-step.  The points are read in the
// order of the deepest level's hand-off (pts, perm); children [4 half,
// 4 half + 4) of input point perm[i] go to out[perm[i]] (float4).
__global__ void k_posteriors(int level, int depth, int half, int n, const float4* __restrict__ pts,
                             const int* __restrict__ perm, const int* __restrict__ seg_start,
                             const NodeEst* __restrict__ est, float4* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int leaf = depth - 1;
    const int64_t off = d_level_offset(leaf);
    // node of the deepest level holding sorted position i
    int64_t lo = 0, hi = (int64_t(1) << (3 * depth)) - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (seg_start[off + mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    const int64_t parent = level == 0 ? 0 : (lo >> (3 * (leaf - level + 1)));
    const NodeEst* ch = est + d_level_offset(level) + 8 * parent;
    const float4 z = pts[i];
    float sc[8];
    float mx = -CUDART_INF_F;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        ChildRegs r;
        load_child(ch + c, r);
        float ex, ey, ez;
        sc[c] = child_score(r, z.x, z.y, z.z, ex, ey, ez);
        mx = fmaxf(mx, sc[c]);
    }
    float g[8];
    float tot = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        g[c] = mx > -CUDART_INF_F ? ex2_fast(sc[c] - mx) : 0.f;
        tot += g[c];
    }
    const float rinv = tot > 0.f ? rcp_fast(tot) : 0.f;
    const int dst = perm[i];
    if (dst >= 0 && dst < n)
        out[dst] = half ? make_float4(g[4] * rinv, g[5] * rinv, g[6] * rinv, g[7] * rinv)
                        : make_float4(g[0] * rinv, g[1] * rinv, g[2] * rinv, g[3] * rinv);
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

// levels with at least this many parents, of at most LOCAL_EM_POINTS points
// on average, run their EM parent-locally (one CTA per parent)
constexpr int LOCAL_EM_PARENTS = 256;
constexpr int64_t LOCAL_EM_POINTS = 2048;

// Whether est_grid CTAs of the cooperative EM kernel fit on the device at
// once (a cooperative launch needs them co-resident).
// k_estep's dynamic shared memory plus its static part exceeds the 48 KB
// default: opt in (per device, before the first launch).
bool hgmm_estep_smem_attr() {
    return cudaFuncSetAttribute(k_estep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ESTEP_DYN_SMEM)) ==
               cudaSuccess &&
           cudaFuncSetAttribute(k_estep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ESTEP_DYN_SMEM)) ==
               cudaSuccess;
}

// CTAs of the cooperative EM kernel that fit on the device at once (a
// cooperative launch needs them co-resident), at most est_grid; 0 if none.
int hgmm_em_coop_grid(int n_sm, int est_grid) {
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_em_coop<true>, EST_THREADS, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_em_coop<false>, EST_THREADS, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return std::min(std::min(a, b) * n_sm, est_grid);
}

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
            k_make_items<<<1, 1024, 0, s>>>(l, n, n_par, t->seg_count, t->item_range, t->meta, G);
        }
        {
            ProfScope ps_(t, K_FILL_ITEMS, s);
            k_fill_items<<<int((t->max_items + 255) / 256), 256, 0, s>>>(
                l, n, n_par, t->seg_start, t->seg_count, t->item_range, t->meta, t->items);
        }
        HGMM_LAUNCH_CHECK();
        const bool stop_here = p.debug_stop_level == l + 1;
        const int em_iters = stop_here ? p.debug_stop_iters : p.em_iters;
        const bool local_em = n_par >= LOCAL_EM_PARENTS && n64 <= LOCAL_EM_POINTS * n_par;
        if (local_em && em_iters > 0) {
            ProfScope ps_(t, K_ESTEP, s);
            if (comp)
                k_em_local<true><<<n_par, EST_THREADS, 0, s>>>(l, n, em_iters, cur, t->items, t->item_range,
                                                              t->seg_count, t->root, p.n_min,
                                                              t->stat, t->est, t->status);
            else
                k_em_local<false><<<n_par, EST_THREADS, 0, s>>>(l, n, em_iters, cur, t->items, t->item_range,
                                                               t->seg_count, t->root, p.n_min,
                                                               t->stat, t->est, t->status);
        }
        const bool coop_em = !local_em && em_iters > 0 && t->em_coop_grid > 0 && (p.flags & HGMM_FLAG_EM_COOPERATIVE);
        if (coop_em) {
            ProfScope ps_(t, K_ESTEP, s);
            cudaMemsetAsync(t->em_cnt, 0, size_t(n_par + 1) * sizeof(unsigned), s);
            int lv = l, nn = n, np = n_par, K = em_iters, chunks = G;
            float nmin = p.n_min;
            void* args[] = {&lv, &nn, &np, &K, &chunks, &cur, &t->items, &t->meta, &t->item_range, &t->partials,
                            &t->seg_count, &t->root, &nmin, &t->stat, &t->est, &t->em_cnt, &t->status};
            const void* fn = comp ? (const void*)k_em_coop<true> : (const void*)k_em_coop<false>;
            if (cudaLaunchCooperativeKernel(fn, dim3(t->em_coop_grid), dim3(EST_THREADS), args, 0, s) != cudaSuccess) {
                fprintf(stderr, "hgmm: cooperative EM launch failed\n");
                return HGMM_ECUDA;
            }
        }
        for (int k = 0; k < (local_em || coop_em ? 0 : em_iters); ++k) {
            {
                ProfScope ps_(t, K_ESTEP, s);
                if (comp)
                    k_estep<true><<<G, EST_THREADS, ESTEP_DYN_SMEM, s>>>(cur, t->items, t->meta, est_lvl, t->partials, t->status);
                else
                    k_estep<false><<<G, EST_THREADS, ESTEP_DYN_SMEM, s>>>(cur, t->items, t->meta, est_lvl, t->partials, t->status);
            }
            {
                ProfScope ps_(t, K_MSTEP, s);
                if (comp)
                    k_mstep<true><<<dim3(n_par, mstep_slices(n_par, n64, G)), 256, 0, s>>>(
                        l, n, t->item_range, t->meta, t->partials, t->seg_count, t->root, p.n_min, t->stat,
                        t->est, t->status, t->mslices, t->mcnt);
                else
                    k_mstep<false><<<dim3(n_par, mstep_slices(n_par, n64, G)), 256, 0, s>>>(
                        l, n, t->item_range, t->meta, t->partials, t->seg_count, t->root, p.n_min, t->stat,
                        t->est, t->status, t->mslices, t->mcnt);
            }
        }
        HGMM_LAUNCH_CHECK();
        if (stop_here) return HGMM_OK;  // checking aid: parameters after em_iters
        {
            ProfScope ps_(t, K_ASSIGN, s);
            k_assign<<<t->n_sm * 4, EST_THREADS, 0, s>>>(cur, t->items, t->meta, est_lvl, t->codes, t->item_cnt);
        }
        {
            ProfScope ps_(t, K_OFFSETS, s);
            // parents of many items (top levels of large clouds) are scanned
            // in slices of about OFFSET_SLICE_ITEMS items by parallel CTAs
            const int64_t items_est = (n64 + TILE - 1) / TILE + n_par;
            int nsl = int(std::min<int64_t>(OFFSET_MAX_SLICES, std::max<int64_t>(1, items_est / n_par / OFFSET_SLICE_ITEMS)));
            while (nsl > 1 && int64_t(n_par) * nsl > t->max_slices) --nsl;
            if (nsl > 1)
                k_offset_slices<<<dim3(n_par, nsl), 256, 0, s>>>(t->item_range, t->item_cnt, nsl, t->slice_tot);
            k_child_offsets<<<dim3(n_par, nsl), 256, 0, s>>>(l, n, t->item_range, t->items, t->item_cnt,
                                                             t->item_off, t->seg_start, t->seg_count, nsl,
                                                             t->slice_tot);
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

int hgmm_debug_posteriors_impl(hgmm_tree* t, int level, float* h_gamma) {
    const int n = int(t->n);
    const int d = t->depth;
    // the deepest level's hand-off left the points in pts[(d - 1) & 1]; the
    // other ping-pong buffer (n float4) is free after the build
    const float4* pts = t->pts[(d - 1) & 1];
    float4* buf = t->pts[d & 1];
    for (int half = 0; half < 2; ++half) {
        k_posteriors<<<(n + 255) / 256, 256>>>(level, d, half, n, pts, t->perm[d - 1], t->seg_start, t->est,
                                               buf);
        HGMM_LAUNCH_CHECK();
        if (cudaMemcpy2D(h_gamma + 4 * half, 8 * sizeof(float), buf, sizeof(float4), sizeof(float4), size_t(n),
                         cudaMemcpyDeviceToHost) != cudaSuccess)
            return HGMM_ECUDA;
    }
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
        // the codes hgmm_sync reports for a tree, in the same order
        const int st = *status;
        out[128] = (st & ST_NONFINITE)    ? double(HGMM_ENONFINITE)
                   : (st & ST_TIMEOUT)    ? double(HGMM_ETIMEOUT)
                   : (st & ST_DEGENERATE) ? double(HGMM_EDEGENERATE)
                                          : 0.0;
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
    // set-up per device, with that device current: resolve the scratch
    // array's device address (host code cannot use the symbol itself).  Done
    // on every call made outside a stream capture (cheap; it also picks up a
    // new context after cudaDeviceReset); a call made while the stream is
    // being captured uses the address the last such call resolved.
    constexpr int MAX_DEV = 64;
    static NoAllocDevice devs[MAX_DEV];
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return HGMM_ECUDA;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cap) != cudaSuccess) return HGMM_ECUDA;
    NoAllocDevice d;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!devs[dev].base || cap == cudaStreamCaptureStatusNone) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
                fprintf(stderr, "hgmm_fit_level0_noalloc: cudaGetSymbolAddress failed\n");
                return HGMM_ECUDA;
            }
            int n_sm = 0;
            if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                return HGMM_ECUDA;
            if (!hgmm_estep_smem_attr()) return HGMM_ECUDA;
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
    k_make_items<<<1, 1024, 0, s>>>(0, ni, 1, seg, item_range, meta, G);
    k_fill_items<<<(NA_MAX_ITEMS + 255) / 256, 256, 0, s>>>(0, ni, 1, seg, seg, item_range, meta,
                                                            items);
    for (int k = 0; k < prm.em_iters; ++k) {
        if (prm.precision == 0) {
            k_estep<true><<<G, EST_THREADS, ESTEP_DYN_SMEM, s>>>(reinterpret_cast<const float4*>(d_points), items,
                                                    meta, est, partials, status);
            k_mstep<true><<<dim3(1, 1), 256, 0, s>>>(0, ni, item_range, meta, partials, seg, root,
                                            prm.n_min, stat, est, status, nullptr, nullptr);
        } else {
            k_estep<false><<<G, EST_THREADS, ESTEP_DYN_SMEM, s>>>(reinterpret_cast<const float4*>(d_points), items,
                                                     meta, est, partials, status);
            k_mstep<false><<<dim3(1, 1), 256, 0, s>>>(0, ni, item_range, meta, partials, seg, root,
                                             prm.n_min, stat, est, status, nullptr, nullptr);
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
