"""Shared helpers of the GPU-vs-oracle parity tests.

The tolerances are the ones the target of this path states: component means
and covariances within 1e-4 relative, final rotation within 0.01 degrees and
translation within 1e-4 of the scene extent.  Argmax decisions (the level
hand-off, the descent) are compared by what is unique: a point may only be
assigned differently where the oracle's own top-two log-likelihood margin is
a near-tie that FP32 cannot resolve.
"""
import numpy as np

from oracle import hgmm_oracle as O
from paper_1807_02587_gb300 import synth

MEAN_TOL = 1e-4
COV_TOL = 1e-4
PI_TOL = 1e-4
ROT_TOL_DEG = 0.01
TRANS_TOL_REL = 1e-4
TIE_MARGIN = 1e-3  # nats


def device_cloud(P):
    """(N,3) float64 -> (CUDA (N,4) float32 tensor, float64 copy of exactly
    the float32 values the GPU sees, for the oracle)."""
    import torch
    f4 = synth.to_float4(P)
    return torch.from_numpy(f4).cuda(), f4[:, :3].astype(np.float64)


def oracle_params(prm_gpu=None, depth=3):
    p = O.Params(depth=depth)
    if prm_gpu is not None:
        p.em_iters = prm_gpu.em_iters
        p.n_min = float(prm_gpu.n_min)
        p.lam_c = float(np.float32(prm_gpu.lam_c))
        p.eps_rel = float(np.float32(prm_gpu.eps_rel))
    return p


def safe_sigma(d):
    S = d["Sigma"].copy()
    S[~d["live"]] = np.eye(3)
    return S


def node_errors(g, o):
    """Relative errors of GPU node params g vs oracle level o over nodes live in both."""
    live = g["live"] & o.live
    scale = np.maximum(np.linalg.norm(o.mu[live], axis=1),
                       np.sqrt(np.trace(o.Sigma[live], axis1=1, axis2=2)))
    e_mu = np.linalg.norm(g["mu"][live] - o.mu[live], axis=1) / scale
    e_S = (np.linalg.norm(g["Sigma"][live] - o.Sigma[live], axis=(1, 2))
           / np.linalg.norm(o.Sigma[live], axis=(1, 2)))
    e_pi = np.abs(g["pi"][live] - o.pi[live])
    return e_mu, e_S, e_pi


def handoff_check(Z, parent, g):
    """GPU labels of a level vs the oracle's argmax under the GPU's own final
    parameters (teacher forcing).  Returns (reference labels, top-two margin
    per point).  A point whose parent has no live child has no decision to
    make: it rides down on the parent's first child (margin +inf, so any
    disagreement there counts as a real one); a point with one live child
    gets +inf too."""
    pi = np.where(g["live"], g["pi"], 0.0)
    S = O.child_scores(Z, parent, pi, g["mu"], safe_sigma(g))
    srt = np.sort(S, axis=1)
    with np.errstate(invalid="ignore"):
        margin = srt[:, -1] - srt[:, -2]
    margin = np.where(np.isfinite(srt[:, -1]), margin, np.inf)
    ref = parent * 8 + np.argmax(S, axis=1)
    return ref, margin


AMBIG_REL = 1e-4     # an expected count this close to n_min (or to the runner-up) is a near-tie
COND_PERTURB = 1e-7  # relative input perturbation used to find ill-conditioned EM fits
COND_TOL = 2e-5      # oracle response to that perturbation beyond which a fit is ill-conditioned


def ambiguous_parents(s0_hist, n_par, n_min):
    """Parents whose dead-child decisions were near-ties at some iteration:
    an expected count within AMBIG_REL (relative) of n_min."""
    amb = np.zeros(n_par, bool)
    for S0 in s0_hist:
        S = S0.reshape(n_par, 8)
        amb |= np.any(np.abs(S - n_min) <= AMBIG_REL * max(n_min, 1.0), axis=1)
    return amb


def ill_conditioned_parents(Z, parent, n_par, p_mu, p_S, p_cnt, prm_o, eps, o, seed=0):
    """Parents whose 8-child EM fit moves by more than COND_TOL when the input
    coordinates are perturbed by COND_PERTURB relative: their K-iteration
    result is not determined to FP32 precision by the data."""
    rng = np.random.default_rng(seed)
    Zp = Z * (1.0 + COND_PERTURB * rng.standard_normal(Z.shape))
    o2 = O.build_level(Zp, parent, n_par, p_mu, p_S, p_cnt, prm_o, eps)
    live = o.live & o2.live
    bad = np.zeros(o.pi.shape[0], bool)
    bad[o.live != o2.live] = True
    e_mu, e_S, e_pi = node_errors({"mu": o2.mu, "Sigma": o2.Sigma, "pi": o2.pi, "live": o2.live}, o)
    idx = np.nonzero(live)[0]
    bad[idx] |= (e_mu > COND_TOL) | (e_S > COND_TOL) | (e_pi > COND_TOL)
    return bad.reshape(n_par, 8).any(axis=1)


def check_build(tree, Z, prm_o, report=None, conditioning=True):
    """Teacher-forced level-by-level comparison of a GPU tree with the oracle.
    Children of parents with near-tie decisions or an ill-conditioned EM fit
    are excluded from the parameter comparison (and counted)."""
    N = Z.shape[0]
    r = tree.root()
    mu0, S0, extent = O.root_stats(Z)
    out = {"root_mu": float(np.linalg.norm(r["mu"] - mu0) / max(np.linalg.norm(mu0), extent)),
           "root_S": float(np.linalg.norm(r["Sigma"] - S0) / np.linalg.norm(S0)),
           "extent": float(abs(r["extent"] - extent) / extent), "levels": []}
    eps = (prm_o.eps_rel * extent) ** 2
    parent = np.zeros(N, np.int64)
    p_mu, p_S, p_cnt = mu0[None], S0[None], np.array([N])
    for l in range(prm_o.depth):
        n_par = p_mu.shape[0]
        g = tree.export(l)
        o = O.build_level(Z, parent, n_par, p_mu, p_S, p_cnt, prm_o, eps)
        excl = ambiguous_parents(o.s0_hist, n_par, prm_o.n_min)
        n_amb = int(excl.sum())
        if conditioning:
            excl |= ill_conditioned_parents(Z, parent, n_par, p_mu, p_S, p_cnt, prm_o, eps, o)
        keep = ~np.repeat(excl, 8)
        gk = {k: v[keep] for k, v in g.items()}
        ok = o.__class__(pi=o.pi[keep], mu=o.mu[keep], Sigma=o.Sigma[keep], live=o.live[keep],
                         labels=None, count=None)
        e_mu, e_S, e_pi = node_errors(gk, ok)
        lab = tree.labels(l).astype(np.int64)
        ref, margin = handoff_check(Z, parent, g)
        dis = lab != ref
        pt_keep = ~excl[parent]
        cnt_gpu = np.bincount(lab, minlength=g["pi"].shape[0])
        out["levels"].append({
            "live_mismatch": int(np.sum(gk["live"] != ok.live)),
            "mu": float(e_mu.max(initial=0)), "S": float(e_S.max(initial=0)),
            "pi": float(e_pi.max(initial=0)),
            "mu_p99": float(np.percentile(e_mu, 99)) if e_mu.size else 0.0,
            "label_disagree": int(dis.sum()),
            "label_disagree_not_tie": int(np.sum(dis & (margin >= TIE_MARGIN) & pt_keep)),
            "count_mismatch": int(np.sum(cnt_gpu != g["count"])),
            "n_live": int(g["live"].sum()),
            "excluded_parents": int(excl.sum()), "near_tie_parents": n_amb,
            "parents_with_points": int(np.sum(p_cnt > 0)),
        })
        parent = lab
        p_mu, p_S = g["mu"], safe_sigma(g)
        p_cnt = np.where(g["live"], g["count"], 0)
    if report is not None:
        report.append(out)
    return out


def check_em_steps(B, dev, Z, depth, steps, prm=None):
    """Single-iteration teacher forcing: for each (level, k) the GPU build is
    stopped after k-1 and after k EM iterations of that level; the oracle runs
    one EM iteration from the GPU's k-1 parameters and is compared with the
    GPU's k-th.  Returns a list of per-step error records."""
    import torch  # noqa: F401  (device tensors)
    prm = prm or B.params()
    N = Z.shape[0]
    mu0, S0, extent = O.root_stats(Z)
    prm_o = oracle_params(prm, depth)
    eps = (prm_o.eps_rel * extent) ** 2
    tree = B.Tree(N, depth)
    res = []
    def stop_at(level, iters):
        q = B.params(em_iters=prm.em_iters, n_min=prm.n_min, lam_c=prm.lam_c,
                     eps_rel=prm.eps_rel, precision=prm.precision,
                     debug_stop_level=level, debug_stop_iters=iters)
        return q

    for (l, k) in steps:
        pa = stop_at(l + 1, k - 1)
        tree.build(dev, depth, pa)
        tree.sync()
        A = tree.export(l)
        if l == 0:
            parent = np.zeros(N, np.int64)
            p_cnt = np.array([N])
        else:
            parent = tree.labels(l - 1).astype(np.int64)
            p_cnt = np.bincount(parent, minlength=8 ** l)
        pb = stop_at(l + 1, k)
        tree.build(dev, depth, pb)
        tree.sync()
        G = tree.export(l)
        n_par = A["pi"].shape[0] // 8
        pi = np.where(A["live"], A["pi"], 0.0)
        pi_n, mu_n, Sig_n, live_n, S0n, _ = O.em_iteration(
            Z, parent, n_par, p_cnt, pi, A["mu"], safe_sigma(A), eps, prm_o.n_min)
        amb = ambiguous_parents([S0n], n_par, prm_o.n_min)
        keep = ~np.repeat(amb, 8)
        o = O.Level(pi=pi_n[keep], mu=mu_n[keep], Sigma=Sig_n[keep], live=live_n[keep],
                    labels=None, count=None)
        gk = {kk: v[keep] for kk, v in G.items()}
        e_mu, e_S, e_pi = node_errors(gk, o)
        res.append({"level": l, "iter": k, "live_mismatch": int(np.sum(gk["live"] != o.live)),
                    "mu": float(e_mu.max(initial=0)), "S": float(e_S.max(initial=0)),
                    "pi": float(e_pi.max(initial=0)), "near_tie_parents": int(amb.sum())})
    return res


def tree_from_gpu(tree, prm_o, extent):
    levels = []
    for l in range(prm_o.depth):
        d = tree.export(l)
        d["Sigma"] = safe_sigma(d)
        levels.append(d)
    return O.tree_from_arrays(prm_o, extent, levels)


def pose_errors(Ta, Tb, extent):
    return (O.rotation_error_deg(Ta[:3, :3], Tb[:3, :3]),
            float(np.linalg.norm(Ta[:3, 3] - Tb[:3, 3]) / extent))


def per_round_teacher_forced(ot, Zs, hist, extent, rounds=None, T0=None):
    """Registration with per-round teacher forcing: for each round k (0-based)
    the oracle runs one round of Algorithm 1 + Eq. 9-16 on tree ``ot`` from
    the GPU's pose after round k-1 (``T0``, default identity, for k = 0) and
    is compared with the GPU's pose after round k.  Works whether or not the
    trajectory converges.  Returns [(k, rot_deg, trans_rel)]."""
    n = hist.shape[0]
    rounds = range(n) if rounds is None else rounds
    out = []
    for k in rounds:
        Tprev = (np.eye(4) if T0 is None else T0) if k == 0 else hist[k - 1]
        T_o = O.register(ot, Zs, T_init=Tprev, iters=1)
        r, t = pose_errors(hist[k], T_o, extent)
        out.append((k, r, t))
    return out
