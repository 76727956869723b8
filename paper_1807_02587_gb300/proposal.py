"""Learned pose proposal: data generation, training and evaluation on the GPU.

Every step of the proposal path runs in the library's kernels through the C
ABI (``binding``): tree builds and canonical-frame features
(hgmm_batch_features), the network (hgmm_mlp_*), pose decode / encode /
select, and the refinement by the plain method (hgmm_batch_register).
PyTorch here only holds device buffers, uploads the synthetic clouds and
draws shuffled batch indices.

Labels come from the plain method itself: every training pair is registered
from several starts (the identity and the four frame alignments
R = V_t S V_s^T, S a proper diagonal sign matrix); the start whose
refinement ends with the lowest Eq. 11 objective gives the label, and labels
further than ``label_tol_deg`` from the known ground truth are dropped (and
counted).  At test time the network's proposal is refined by the plain
method and the plain method from the identity stays the fallback: of the
two refinements the one with the lower objective is kept.
"""
from __future__ import annotations

import time

import numpy as np

from . import binding as B
from . import synth

# 6-D codes (first two columns) of the proper diagonal sign matrices
FLIP_CODES = np.array([[1, 0, 0, 0, 1, 0], [1, 0, 0, 0, -1, 0], [-1, 0, 0, 0, 1, 0],
                       [-1, 0, 0, 0, -1, 0]], np.float32)


def _torch():
    import torch
    return torch


def rotation_error_deg(Ra, Rb) -> float:
    c = (np.trace(np.asarray(Ra).T @ np.asarray(Rb)) - 1.0) / 2.0
    return float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights from the seeded generator; the last layer scaled
    by 0.1 and its bias set to the 6-D code of the identity, so the untrained
    network proposes the frame alignment with S = I."""
    p = synth.mlp_init(seed).astype(np.float32)
    w3 = 256 * 1280 + 256 + 256 * 256 + 256
    p[w3:w3 + 9 * 256] *= 0.1
    p[w3 + 9 * 256:] = np.array([1, 0, 0, 0, 1, 0, 0, 0, 0], np.float32)
    return p


class PairSet:
    """Clouds of many pairs in one device buffer (float4) with per-pair
    point ranges; pairs may share a source cloud."""

    def __init__(self, clouds, src_of, tgt_of, T_gt):
        torch = _torch()
        f4 = [synth.to_float4(c) for c in clouds]
        sizes = np.array([c.shape[0] for c in f4], np.int64)
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        rng = np.stack([off[:-1], off[1:]], axis=1)
        self.src_rng = rng[np.asarray(src_of)]
        self.tgt_rng = rng[np.asarray(tgt_of)]
        self.n = len(src_of)
        self.points = torch.from_numpy(np.concatenate(f4)).cuda()
        self.T_gt = np.asarray(T_gt, np.float64).reshape(self.n, 4, 4)
        self.max_points = int(sizes.max())


def scene_pairs(seed: int, n_scenes: int, per_scene: int, n: int) -> PairSet:
    """Training pairs: source sample i against per_scene SO(3)-uniform poses
    of the second sample of scene i (the source cloud is stored once)."""
    sc = synth.so3_scene_set(seed, n_scenes, per_scene, n)
    clouds, src_of, tgt_of, T = [], [], [], []
    for i in range(n_scenes):
        si = len(clouds)
        clouds.append(sc["src"][i])
        for j in range(per_scene):
            tgt_of.append(len(clouds))
            src_of.append(si)
            clouds.append(synth.apply(sc["T"][i, j], sc["tgt_base"][i].astype(np.float64)))
            T.append(sc["T"][i, j])
    return PairSet(clouds, src_of, tgt_of, np.array(T))


def so3_test_pairs(seed: int, count: int, n: int) -> PairSet:
    ps = synth.so3_pairs(seed, count, n)
    clouds = [c for p in ps for c in (p["src"], p["tgt"])]
    return PairSet(clouds, np.arange(0, 2 * count, 2), np.arange(1, 2 * count, 2),
                   np.array([p["T_gt"] for p in ps]))


class Engine:
    """Batch engines for one PairSet: feature builds (source of pair i as
    entry 2i, target as 2i+1, depth 2) and registrations (depth ``depth``)."""

    def __init__(self, ps: PairSet, depth: int, cluster_ctas: int = 8):
        torch = _torch()
        self.ps, self.depth, n = ps, depth, ps.n
        self.fb = B.Batch(ps.max_points, 2, 2 * n)
        ent = np.empty((2 * n, 2), np.int64)
        ent[0::2], ent[1::2] = ps.src_rng, ps.tgt_rng
        B.hgmm_batch_plan_ranges(self.fb.handle, ent, ent, [2] * (2 * n))
        B.hgmm_batch_set_shape(self.fb.handle, cluster_ctas)
        self.rb = B.Batch(ps.max_points, depth, n)
        B.hgmm_batch_plan_ranges(self.rb.handle, ps.tgt_rng, ps.src_rng, [depth] * n)
        B.hgmm_batch_set_shape(self.rb.handle, cluster_ctas)
        self.X = torch.zeros((n, 1280), dtype=torch.bfloat16, device="cuda")
        self.frames = torch.zeros((n, 32), dtype=torch.float64, device="cuda")

    def features(self, stream=None):
        B.hgmm_batch_features(self.fb.handle, self.ps.points, self.X, self.frames, stream=stream)
        return self.X, self.frames

    def register(self, T_init, iters: int, T_out=None, obj=None, status=None, stream=None):
        torch = _torch()
        n = self.ps.n
        T_out = T_out if T_out is not None else torch.zeros((n, 16), dtype=torch.float64, device="cuda")
        obj = obj if obj is not None else torch.zeros(n, dtype=torch.float64, device="cuda")
        B.hgmm_batch_register(self.rb.handle, self.ps.points, T_out, T_init=T_init, iters=iters,
                              stream=stream, pair_status=status)
        B.hgmm_batch_objective(self.rb.handle, obj, stream=stream)
        return T_out, obj

    def flip_starts(self):
        """The four frame alignments of every pair (4, n, 16)."""
        torch = _torch()
        n = self.ps.n
        out = torch.zeros((4, n, 16), dtype=torch.float64, device="cuda")
        y = torch.zeros((n, 9), dtype=torch.float32, device="cuda")
        for k in range(4):
            y[:, :6] = torch.from_numpy(FLIP_CODES[k]).cuda()
            B.hgmm_pose_decode(y, self.frames, out[k])
        return out


def label_pairs(ps: PairSet, depth: int = 3, iters: int = 30, label_tol_deg: float = 1.0,
                cluster_ctas: int = 8):
    """Features, multi-start labels of the plain method, and the check of
    each label against the ground truth.  Returns (X, labels, keep, stats)."""
    torch = _torch()
    eng = Engine(ps, depth, cluster_ctas)
    n = ps.n
    t0 = time.perf_counter()
    eng.features()
    starts = [None] + list(eng.flip_starts())
    best = torch.zeros((n, 16), dtype=torch.float64, device="cuda")
    best_obj = torch.full((n,), float("inf"), dtype=torch.float64, device="cuda")
    for k, T0 in enumerate(starts):
        T, o = eng.register(T0, iters)
        B.hgmm_pose_select(best, best_obj, T, o, best, obj_out=best_obj)
    labels = torch.zeros((n, 12), dtype=torch.float32, device="cuda")
    B.hgmm_pose_encode(best, eng.frames, labels)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    Tb = best.cpu().numpy().reshape(n, 4, 4)
    err = np.array([rotation_error_deg(Tb[i, :3, :3], ps.T_gt[i, :3, :3]) for i in range(n)])
    keep = err <= label_tol_deg
    stats = {"pairs": n, "label_within_tol": float(keep.mean()), "label_tol_deg": label_tol_deg,
             "starts": len(starts), "seconds": secs, "median_label_err_deg": float(np.median(err))}
    return eng.X.clone(), labels, keep, stats


def train(net, X, labels, keep, epochs: int = 40, batch: int = 512, lr: float = 1e-3,
          w_t: float = 1.0, seed: int = 0, log=None):
    """Adam on the kept rows; cosine learning-rate decay; returns the mean
    loss of the last epoch."""
    torch = _torch()
    rows = torch.from_numpy(np.nonzero(keep)[0].astype(np.int32)).cuda()
    n = int(rows.shape[0])
    if n < 1:
        raise ValueError("no labelled rows to train on")
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    steps = max(1, n // batch)
    total = epochs * steps
    last = []
    k = 0
    for ep in range(epochs):
        perm = rows[torch.randperm(n, device="cuda", generator=g)]
        ep_loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        for s in range(steps):
            cur = lr * 0.5 * (1.0 + np.cos(np.pi * k / total))
            idx = perm[s * batch:(s + 1) * batch]
            B.hgmm_mlp_train_step(net.handle, X, labels, int(idx.shape[0]), index=idx, w_t=w_t,
                                  lr=float(cur), loss=loss)
            ep_loss += loss
            k += 1
        if log is not None and (ep % 10 == 0 or ep == epochs - 1):
            log(f"epoch {ep}: loss {ep_loss.item() / steps:.4f}")
        if ep == epochs - 1:
            last.append(ep_loss.item() / steps)
    B.hgmm_mlp_sync(net.handle)
    return last[-1]


def propose(net, eng: Engine, y=None, T=None, stream=None):
    """Network proposal (n, 16) for every pair of the engine's set."""
    torch = _torch()
    n = eng.ps.n
    y = y if y is not None else torch.zeros((n, 9), dtype=torch.float32, device="cuda")
    T = T if T is not None else torch.zeros((n, 16), dtype=torch.float64, device="cuda")
    eng.features(stream=stream)
    B.hgmm_mlp_forward(net.handle, eng.X, y, stream=stream)
    B.hgmm_pose_decode(y, eng.frames, T, stream=stream)
    return T


def success(ps: PairSet, T, tol_deg: float = 0.1):
    Tn = T.cpu().numpy().reshape(ps.n, 4, 4)
    err = np.array([rotation_error_deg(Tn[i, :3, :3], ps.T_gt[i, :3, :3]) for i in range(ps.n)])
    return float((err <= tol_deg).mean()), err


def evaluate(net, ps: PairSet, depth: int = 4, iters: int = 30, cluster_ctas: int = 8, reps: int = 3):
    """Success rate (<= 0.1 deg) and pairs/s of the plain method from the
    identity and of the proposal + refinement with the identity fallback,
    both timed with CUDA events over the whole pipeline (inputs resident)."""
    torch = _torch()
    eng = Engine(ps, depth, cluster_ctas)
    n = ps.n
    ident = torch.zeros((n, 16), dtype=torch.float64, device="cuda")
    ident[:, [0, 5, 10, 15]] = 1.0
    T_id = torch.zeros((n, 16), dtype=torch.float64, device="cuda")
    o_id = torch.zeros(n, dtype=torch.float64, device="cuda")
    T_pr = torch.zeros((n, 16), dtype=torch.float64, device="cuda")
    o_pr = torch.zeros(n, dtype=torch.float64, device="cuda")
    T_sel = torch.zeros((n, 16), dtype=torch.float64, device="cuda")
    choice = torch.zeros(n, dtype=torch.int32, device="cuda")
    y = torch.zeros((n, 9), dtype=torch.float32, device="cuda")
    T_prop = torch.zeros((n, 16), dtype=torch.float64, device="cuda")

    def plain():
        eng.register(ident, iters, T_out=T_id, obj=o_id)

    def learned():
        propose(net, eng, y=y, T=T_prop)
        eng.register(T_prop, iters, T_out=T_pr, obj=o_pr)
        eng.register(ident, iters, T_out=T_id, obj=o_id)
        B.hgmm_pose_select(T_pr, o_pr, T_id, o_id, T_sel, choice)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps / 1e3

    t_plain = timed(plain)
    s_plain, err_plain = success(ps, T_id)
    t_learn = timed(learned)
    s_learn, err_learn = success(ps, T_sel)
    s_prop_only, _ = success(ps, T_pr)
    _, err_prop = success(ps, T_prop, 1e9)
    return {
        "pairs": n, "depth": depth, "iters": iters,
        "plain_success_le_0p1deg": s_plain, "plain_pairs_per_s": n / t_plain,
        "plain_within_1deg": float((err_plain <= 1.0).mean()),
        "learned_success_le_0p1deg": s_learn, "learned_pairs_per_s": n / t_learn,
        "learned_within_1deg": float((err_learn <= 1.0).mean()),
        "learned_median_final_err_deg": float(np.median(err_learn)),
        "learned_without_fallback_success_le_0p1deg": s_prop_only,
        "fallback_taken": float(choice.float().mean().item()),
        "proposal_median_err_deg": float(np.median(err_prop)),
        "proposal_within_30deg": float((err_prop <= 30.0).mean()),
    }
