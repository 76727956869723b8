// C ABI of the HGMM library: tree lifetime, argument checking, the
// host-buffer convenience call and the export / checking entry points.
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <vector>

#include "hgmm_internal.cuh"

using namespace hgmm;

namespace {

bool ok(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return true;
    fprintf(stderr, "hgmm: %s: %s\n", what, cudaGetErrorString(e));
    return false;
}

template <typename T>
bool dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return true;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T)) == cudaSuccess;
}

void clear_prof(hgmm_tree* t) {
    for (auto& r : t->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    t->prof.clear();
}

const char* const kKernelNames[HGMM_PROF_KERNELS] = {
    "root_partial", "root_final", "init_children", "make_items", "fill_items", "estep",
    "mstep", "assign", "child_offsets", "scatter", "finalize", "reg_init", "register",
    "reg_mstep", "copy_T", "labels"};

void free_tree(hgmm_tree* t) {
    if (!t) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(t->device);
    clear_prof(t);
    if (t->pair_exec) cudaGraphExecDestroy(t->pair_exec);
    if (t->cap_stream) cudaStreamDestroy(t->cap_stream);
    void* ptrs[] = {t->est, t->stat, t->seg_start, t->seg_count, t->pts[0], t->pts[1],
                    t->codes, t->items, t->item_range, t->meta, t->partials, t->item_cnt,
                    t->item_off, t->slice_tot, t->root, t->root_part, t->root_counter, t->em_cnt, t->mslices, t->mcnt, t->status, t->reg_acc, t->reg_acc2, t->reg_part,
                    t->reg_bar, t->reg_T, t->reg_Rt, t->reg_dbg, t->reg_obj, t->rnode, t->trace, t->stage_tgt,
                    t->stage_src, t->stage_T};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int l = 0; l < HGMM_MAX_DEPTH; ++l)
        if (t->perm[l]) cudaFree(t->perm[l]);
    cudaSetDevice(cur);
    delete t;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int check_device(const hgmm_tree* t) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return HGMM_ECUDA;
    return cur == t->device ? HGMM_OK : HGMM_EINVAL;
}

}  // namespace

extern "C" {

int64_t hgmm_node_count(int32_t depth) {
    if (depth < 1 || depth > HGMM_MAX_DEPTH) return 0;
    return level_offset(depth);  // sum of 8^(l+1) for l < depth
}

void hgmm_params_default(hgmm_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->em_iters = 8;
    p->n_min = 8.0f;
    p->lam_c = 0.01f;
    p->eps_rel = 1e-3f;
    p->precision = 0;
}

const char* hgmm_strerror(int code) {
    switch (code) {
        case HGMM_OK: return "ok";
        case HGMM_EINVAL: return "invalid argument";
        case HGMM_ENOMEM: return "device allocation failed";
        case HGMM_ECUDA: return "CUDA error";
        case HGMM_ETIMEOUT: return "device wait timed out";
        case HGMM_EDEGENERATE: return "singular normal equations";
        case HGMM_ENONFINITE: return "non-finite input coordinates";
        case HGMM_ECAPACITY: return "size exceeds the tree's capacity";
        default: return "unknown error";
    }
}

int hgmm_tree_create(int64_t max_points, int32_t max_depth, hgmm_tree** out) {
    if (!out) return HGMM_EINVAL;
    *out = nullptr;
    if (max_points < 8 || max_points > (int64_t(1) << 30) || max_depth < 1 ||
        max_depth > HGMM_MAX_DEPTH)
        return HGMM_EINVAL;
    hgmm_tree* t = new hgmm_tree();
    if (!ok(cudaGetDevice(&t->device), "cudaGetDevice")) { delete t; return HGMM_ECUDA; }
    cudaDeviceProp prop;
    if (!ok(cudaGetDeviceProperties(&prop, t->device), "cudaGetDeviceProperties")) {
        delete t;
        return HGMM_ECUDA;
    }
    t->n_sm = prop.multiProcessorCount;
    t->cap = max_points;
    t->max_depth = max_depth;
    t->max_nodes = level_offset(max_depth);
    // widest parent level: level max_depth-2 (8^(max_depth-1) nodes), or the root
    const int64_t parents = max_depth >= 2 ? level_size(max_depth - 2) : 1;
    t->max_items = (max_points + TILE - 1) / TILE + parents;
    t->est_grid = t->n_sm * 3;  // three k_estep CTAs fit on an SM
    t->reg_grid = hgmm_register_grid(t->n_sm, 2);
    t->reg_grid_wide = hgmm_register_grid(t->n_sm, 3);
    if (t->reg_grid_wide == 0) cudaGetLastError();  // large sources keep the two-per-SM build
    t->em_coop_grid = hgmm_em_coop_grid(t->n_sm, t->est_grid);
    if (!hgmm_estep_smem_attr()) {
        cudaGetLastError();
        delete t;
        return HGMM_ECUDA;
    }
    if (t->reg_grid < 1) {
        delete t;
        return HGMM_ECUDA;
    }
    // one normal-equation partial per registration CTA, or per 32 nodes in
    // the descent variants
    const int64_t nb = std::max<int64_t>(std::max(t->reg_grid, t->reg_grid_wide), (t->max_nodes + 31) / 32);
    bool good = true;
    good &= dalloc(&t->est, t->max_nodes);
    good &= dalloc(&t->stat, t->max_nodes);
    good &= dalloc(&t->seg_start, t->max_nodes);
    good &= dalloc(&t->seg_count, t->max_nodes);
    good &= dalloc(&t->pts[0], max_points);
    good &= dalloc(&t->pts[1], max_points);
    for (int l = 0; l < max_depth; ++l) good &= dalloc(&t->perm[l], max_points);
    good &= dalloc(&t->codes, max_points);
    good &= dalloc(&t->items, t->max_items);
    good &= dalloc(&t->item_range, 2 * std::max<int64_t>(parents, 1));
    good &= dalloc(&t->meta, 4);
    good &= dalloc(&t->partials, t->max_items * NPART);
    good &= dalloc(&t->item_cnt, t->max_items * 8);
    good &= dalloc(&t->item_off, t->max_items * 8);
    t->max_slices = t->max_items / OFFSET_SLICE_ITEMS + 2;
    good &= dalloc(&t->slice_tot, t->max_slices * 8);
    good &= dalloc(&t->root, 1);
    good &= dalloc(&t->root_part, int64_t(t->est_grid) * 32);
    good &= dalloc(&t->root_counter, 1);
    good &= dalloc(&t->em_cnt, level_size(std::max(0, max_depth - 1)) + 1);
    good &= dalloc(&t->mslices, int64_t(MSTEP_SLICED_PARENTS) * MSTEP_SLICES * NPART);
    good &= dalloc(&t->mcnt, MSTEP_SLICED_PARENTS);
    good &= dalloc(&t->status, 1);
    good &= dalloc(&t->reg_acc, 4 * ACC_REPLICAS * t->max_nodes);
    good &= dalloc(&t->reg_acc2, 6 * t->max_nodes);
    good &= dalloc(&t->reg_part, NTERM * nb);
    good &= dalloc(&t->rnode, 3 * t->max_nodes);
    good &= dalloc(&t->trace, int64_t(TRACE_MAX_ITERS) * std::max(t->reg_grid, t->reg_grid_wide) * 6);
    good &= dalloc(&t->reg_bar, 8);
    good &= dalloc(&t->reg_T, 16);
    good &= dalloc(&t->reg_Rt, 12);
    good &= dalloc(&t->reg_dbg, 4 * t->max_nodes);
    good &= dalloc(&t->reg_obj, 1);
    good &= dalloc(&t->stage_tgt, max_points);
    good &= dalloc(&t->stage_src, max_points);
    good &= dalloc(&t->stage_T, 32);
    if (!good) {
        free_tree(t);
        return HGMM_ENOMEM;
    }
    good &= ok(cudaMemset(t->status, 0, sizeof(int)), "cudaMemset");
    good &= ok(cudaMemset(t->reg_bar, 0, 8 * sizeof(unsigned)), "cudaMemset");
    good &= ok(cudaMemset(t->root_counter, 0, sizeof(unsigned)), "cudaMemset");
    good &= ok(cudaMemset(t->mcnt, 0, MSTEP_SLICED_PARENTS * sizeof(unsigned)), "cudaMemset");
    good &= ok(cudaMemset(t->reg_acc, 0, 4 * ACC_REPLICAS * t->max_nodes * sizeof(unsigned long long)),
               "cudaMemset");
    good &= ok(cudaMemset(t->stat, 0, t->max_nodes * sizeof(NodeStat)), "cudaMemset");
    good &= ok(cudaMemset(t->seg_count, 0, t->max_nodes * sizeof(int)), "cudaMemset");
    good &= ok(cudaMemset(t->seg_start, 0, t->max_nodes * sizeof(int)), "cudaMemset");
    good &= ok(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    if (!good) {
        free_tree(t);
        return HGMM_ECUDA;
    }
    *out = t;
    return HGMM_OK;
}

void hgmm_tree_destroy(hgmm_tree* t) { free_tree(t); }

int hgmm_build(hgmm_tree* t, const float* d_points, int64_t n, int32_t depth, int32_t J,
               const hgmm_params* p, void* stream) {
    if (!t || !d_points) return HGMM_EINVAL;
    if (J != HGMM_J || n < 8 || depth < 1 || depth > HGMM_MAX_DEPTH) return HGMM_EINVAL;
    if (!aligned16(d_points)) return HGMM_EINVAL;
    if (n > t->cap || depth > t->max_depth) return HGMM_ECAPACITY;
    if (int rc = check_device(t)) return rc;
    hgmm_params prm;
    if (p) {
        prm = *p;
        if (prm.em_iters < 0 || prm.em_iters > 1000 || !(prm.eps_rel >= 0.f) ||
            !(prm.n_min >= 0.f) || !(prm.lam_c >= 0.f) || prm.debug_stop_level < 0 ||
            prm.debug_stop_level > depth || prm.debug_stop_iters < 0 ||
            prm.debug_stop_iters > prm.em_iters)
            return HGMM_EINVAL;
    } else {
        hgmm_params_default(&prm);
    }
    t->n = n;
    t->depth = depth;
    t->prm = prm;
    t->built = true;
    return hgmm_build_impl(t, reinterpret_cast<const float4*>(d_points), n, depth, prm,
                           static_cast<cudaStream_t>(stream));
}

int hgmm_register(hgmm_tree* t, const float* d_src, int64_t n, const double* d_T_init,
                  int32_t iters, float lam_c, void* stream, double* d_T_out, double* d_T_hist) {
    if (!t || !d_src || n < 1 || iters < 0 || !t->built) return HGMM_EINVAL;
    if (!aligned16(d_src)) return HGMM_EINVAL;
    if (n > (int64_t(1) << 31) - 1) return HGMM_ECAPACITY;
    if (int rc = check_device(t)) return rc;
    t->reg_n = n;
    return hgmm_register_impl(t, reinterpret_cast<const float4*>(d_src), n, d_T_init, iters,
                              lam_c, static_cast<cudaStream_t>(stream), d_T_out, d_T_hist);
}

int hgmm_register_descent(hgmm_tree* t, const float* d_src, int64_t n, const double* d_T_init,
                          int32_t iters, const hgmm_descent* d, void* stream, double* d_T_out,
                          double* d_T_hist) {
    if (!t || !d_src || !d || n < 1 || iters < 0 || !t->built) return HGMM_EINVAL;
    if (d->mode < HGMM_DESCENT_ML_LOCAL || d->mode > HGMM_DESCENT_MULTIPATH) return HGMM_EINVAL;
    if (d->full_eq7 != 0 && d->full_eq7 != 1) return HGMM_EINVAL;
    if (!(d->tau >= 0.0f && d->tau <= 1.0f)) return HGMM_EINVAL;
    if (!aligned16(d_src)) return HGMM_EINVAL;
    if (n > (int64_t(1) << 31) - 1) return HGMM_ECAPACITY;
    if (int rc = check_device(t)) return rc;
    t->reg_n = n;
    return hgmm_register_descent_impl(t, reinterpret_cast<const float4*>(d_src), n, d_T_init, iters, *d,
                                      static_cast<cudaStream_t>(stream), d_T_out, d_T_hist);
}

int hgmm_sync(hgmm_tree* t, void* stream) {
    if (!t) return HGMM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int st = 0;
    if (!ok(cudaMemcpyAsync(&st, t->status, sizeof(int), cudaMemcpyDeviceToHost, s), "status copy"))
        return HGMM_ECUDA;
    if (!ok(cudaStreamSynchronize(s), "cudaStreamSynchronize")) return HGMM_ECUDA;
    if (st) {
        const int zero = 0;
        if (!ok(cudaMemcpy(t->status, &zero, sizeof(int), cudaMemcpyHostToDevice), "status reset"))
            return HGMM_ECUDA;
    }
    if (st & ST_NONFINITE) return HGMM_ENONFINITE;
    if (st & ST_TIMEOUT) return HGMM_ETIMEOUT;
    if (st & ST_DEGENERATE) return HGMM_EDEGENERATE;
    return HGMM_OK;
}

int hgmm_register_pair_host(hgmm_tree* t, const float* h_tgt, int64_t n_tgt, const float* h_src,
                            int64_t n_src, int32_t depth, const hgmm_params* p,
                            const double* h_T_init, int32_t iters, void* stream,
                            double* h_T_out) {
    if (!t || !h_tgt || !h_src || !h_T_out) return HGMM_EINVAL;
    if (n_tgt > t->cap || n_src > t->cap) return HGMM_ECAPACITY;
    if (n_tgt < 8 || n_src < 1) return HGMM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!ok(cudaMemcpyAsync(t->stage_tgt, h_tgt, size_t(n_tgt) * 16, cudaMemcpyHostToDevice, s), "H2D"))
        return HGMM_ECUDA;
    if (!ok(cudaMemcpyAsync(t->stage_src, h_src, size_t(n_src) * 16, cudaMemcpyHostToDevice, s), "H2D"))
        return HGMM_ECUDA;
    const double* dTi = nullptr;
    if (h_T_init) {
        if (!ok(cudaMemcpyAsync(t->stage_T, h_T_init, 16 * sizeof(double), cudaMemcpyHostToDevice, s), "H2D"))
            return HGMM_ECUDA;
        dTi = t->stage_T;
    }
    hgmm_params prm;
    if (p) prm = *p;
    else hgmm_params_default(&prm);
    auto enqueue = [&](void* st) -> int {
        int rc = hgmm_build(t, reinterpret_cast<const float*>(t->stage_tgt), n_tgt, depth, HGMM_J, &prm, st);
        if (rc) return rc;
        return hgmm_register(t, reinterpret_cast<const float*>(t->stage_src), n_src, dTi, iters, -1.f, st,
                             t->stage_T + 16, nullptr);
    };
    // the build and the registration as one CUDA graph, captured for this
    // shape on the tree's own stream (the caller's may be the legacy default
    // stream, which cannot be captured) and replayed on the caller's stream:
    // the ~80 kernels of a step cost one launch.  Not while profiling or
    // tracing (their events and stamps are per launch).
    const int64_t key[5] = {n_tgt, n_src, depth, iters, h_T_init ? 1 : 0};
    bool use_graph = !t->prof_on && !t->trace_on && !t->pair_graph_failed;
    if (use_graph) {
        const bool same = t->pair_exec && std::memcmp(key, t->pair_key, sizeof(key)) == 0 &&
                          std::memcmp(&prm, &t->pair_prm, sizeof(prm)) == 0;
        if (!same) {
            if (t->pair_exec) {
                cudaGraphExecDestroy(t->pair_exec);
                t->pair_exec = nullptr;
            }
            if (!t->cap_stream && !ok(cudaStreamCreateWithFlags(&t->cap_stream, cudaStreamNonBlocking), "stream"))
                return HGMM_ECUDA;
            // the staging copies above (on s) come before the captured work
            if (!ok(cudaStreamSynchronize(s), "sync")) return HGMM_ECUDA;
            cudaGraph_t g = nullptr;
            if (!ok(cudaStreamBeginCapture(t->cap_stream, cudaStreamCaptureModeThreadLocal), "capture"))
                return HGMM_ECUDA;
            const int rc = enqueue(t->cap_stream);
            const cudaError_t ec = cudaStreamEndCapture(t->cap_stream, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (ec != cudaSuccess || !g || cudaGraphInstantiate(&t->pair_exec, g, 0) != cudaSuccess) {
                (void)cudaGetLastError();
                if (g) cudaGraphDestroy(g);
                t->pair_exec = nullptr;
                t->pair_graph_failed = true;  // this tree runs the host API eagerly from now on
                use_graph = false;
            } else {
                cudaGraphDestroy(g);
                std::memcpy(t->pair_key, key, sizeof(key));
                t->pair_prm = prm;
            }
        }
    }
    if (use_graph) {
        if (!ok(cudaGraphLaunch(t->pair_exec, s), "graph launch")) return HGMM_ECUDA;
    } else if (int rc = enqueue(stream)) {
        return rc;
    }
    if (!ok(cudaMemcpyAsync(h_T_out, t->stage_T + 16, 16 * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H"))
        return HGMM_ECUDA;
    return hgmm_sync(t, stream);
}

int hgmm_tree_export(hgmm_tree* t, int32_t level, double* h_nodes, int64_t cap) {
    if (!t || !h_nodes || !t->built || level < 0 || level >= t->depth) return HGMM_EINVAL;
    const int64_t m = level_size(level);
    if (cap < m * HGMM_NODE_DOUBLES) return HGMM_ECAPACITY;
    std::vector<NodeStat> st(m);
    std::vector<int> cnt(m);
    const int64_t off = level_offset(level);
    if (!ok(cudaDeviceSynchronize(), "sync")) return HGMM_ECUDA;
    if (!ok(cudaMemcpy(st.data(), t->stat + off, m * sizeof(NodeStat), cudaMemcpyDeviceToHost), "D2H"))
        return HGMM_ECUDA;
    if (!ok(cudaMemcpy(cnt.data(), t->seg_count + off, m * sizeof(int), cudaMemcpyDeviceToHost), "D2H"))
        return HGMM_ECUDA;
    for (int64_t i = 0; i < m; ++i) node_record(st[i], cnt[i], h_nodes + i * HGMM_NODE_DOUBLES);
    return HGMM_OK;
}

int hgmm_debug_labels(hgmm_tree* t, int32_t level, int32_t* h_labels, int64_t cap) {
    if (!t || !h_labels || !t->built || level < 0 || level >= t->depth) return HGMM_EINVAL;
    if (cap < t->n) return HGMM_ECAPACITY;
    // the hand-off codes are dead after the build: reuse them as the output
    int* d = reinterpret_cast<int*>(t->codes);
    int rc = hgmm_export_labels_impl(t, level, d, nullptr);
    if (rc == HGMM_OK &&
        !ok(cudaMemcpy(h_labels, d, size_t(t->n) * sizeof(int), cudaMemcpyDeviceToHost), "D2H"))
        rc = HGMM_ECUDA;
    return rc;
}

int hgmm_debug_posteriors(hgmm_tree* t, int32_t level, float* h_gamma, int64_t cap) {
    if (!t || !h_gamma || !t->built || level < 0 || level >= t->depth || t->prm.debug_stop_level != 0)
        return HGMM_EINVAL;
    if (cap < 8 * t->n) return HGMM_ECAPACITY;
    if (int rc = check_device(t)) return rc;
    if (!ok(cudaDeviceSynchronize(), "sync")) return HGMM_ECUDA;
    return hgmm_debug_posteriors_impl(t, level, h_gamma);
}

int hgmm_debug_root(hgmm_tree* t, double* h_root12) {
    if (!t || !h_root12 || !t->built) return HGMM_EINVAL;
    RootDev r;
    if (!ok(cudaDeviceSynchronize(), "sync")) return HGMM_ECUDA;
    if (!ok(cudaMemcpy(&r, t->root, sizeof(r), cudaMemcpyDeviceToHost), "D2H")) return HGMM_ECUDA;
    root_record(r, h_root12);
    return HGMM_OK;
}

int hgmm_debug_reg_moments(hgmm_tree* t, double* h_m, int64_t cap) {
    if (!t || !h_m || !t->built) return HGMM_EINVAL;
    const int64_t m = hgmm_node_count(t->depth);
    if (cap < 4 * m) return HGMM_ECAPACITY;
    if (!ok(cudaDeviceSynchronize(), "sync")) return HGMM_ECUDA;
    if (!ok(cudaMemcpy(h_m, t->reg_dbg, size_t(4 * m) * sizeof(double), cudaMemcpyDeviceToHost), "D2H"))
        return HGMM_ECUDA;
    return HGMM_OK;
}

int hgmm_register_objective(const hgmm_tree* t, double* d_obj, void* stream) {
    if (!t || !d_obj || !t->built) return HGMM_EINVAL;
    if (!ok(cudaMemcpyAsync(d_obj, t->reg_obj, sizeof(double), cudaMemcpyDeviceToDevice,
                            static_cast<cudaStream_t>(stream)), "D2D"))
        return HGMM_ECUDA;
    return HGMM_OK;
}

int hgmm_debug_barrier_timeout(hgmm_tree* t, int64_t spin_limit, void* stream) {
    if (!t || spin_limit < 1 || spin_limit > 100000000) return HGMM_EINVAL;
    if (int rc = check_device(t)) return rc;
    return hgmm_barrier_timeout_probe_impl(t, spin_limit, static_cast<cudaStream_t>(stream));
}

int hgmm_trace(hgmm_tree* t, int32_t enable) {
    if (!t) return HGMM_EINVAL;
    t->trace_on = enable != 0;
    return HGMM_OK;
}

int hgmm_trace_read(hgmm_tree* t, int64_t* h_events, int64_t cap, int32_t* iters,
                    int32_t* ctas) {
    if (!t || !h_events) return HGMM_EINVAL;
    if (iters) *iters = t->trace_iters;
    if (ctas) *ctas = t->trace_grid;
    return hgmm_trace_read_impl(t, reinterpret_cast<unsigned long long*>(h_events), cap);
}

int hgmm_profile(hgmm_tree* t, int32_t enable) {
    if (!t) return HGMM_EINVAL;
    if (enable) {
        if (!ok(cudaDeviceSynchronize(), "sync")) return HGMM_ECUDA;
        clear_prof(t);
    }
    t->prof_on = enable != 0;
    return HGMM_OK;
}

int hgmm_profile_read(hgmm_tree* t, int32_t kernel, const char** name, double* total_ms,
                      int64_t* launches) {
    static_assert(K_COUNT == HGMM_PROF_KERNELS, "kernel table");
    if (!t || kernel < 0 || kernel >= HGMM_PROF_KERNELS) return HGMM_EINVAL;
    if (!ok(cudaDeviceSynchronize(), "sync")) return HGMM_ECUDA;
    double ms = 0.0;
    int64_t cnt = 0;
    for (const auto& r : t->prof) {
        if (r.id != kernel) continue;
        float x = 0.f;
        if (!ok(cudaEventElapsedTime(&x, r.a, r.b), "cudaEventElapsedTime")) return HGMM_ECUDA;
        ms += x;
        ++cnt;
    }
    if (name) *name = kKernelNames[kernel];
    if (total_ms) *total_ms = ms;
    if (launches) *launches = cnt;
    return HGMM_OK;
}

}  // extern "C"
