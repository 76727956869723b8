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
    parameters (teacher forcing).  Returns (n_disagree, n_disagree_not_tie)."""
    pi = np.where(g["live"], g["pi"], 0.0)
    S = O.child_scores(Z, parent, pi, g["mu"], safe_sigma(g))
    srt = np.sort(S, axis=1)
    margin = srt[:, -1] - srt[:, -2]
    ref = parent * 8 + np.argmax(S, axis=1)
    return ref, margin


def check_build(tree, Z, prm_o, report=None):
    """Teacher-forced level-by-level comparison of a GPU tree with the oracle.
    Returns a dict of maximum errors per level."""
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
        g = tree.export(l)
        o = O.build_level(Z, parent, p_mu.shape[0], p_mu, p_S, p_cnt, prm_o, eps)
        e_mu, e_S, e_pi = node_errors(g, o)
        lab = tree.labels(l).astype(np.int64)
        ref, margin = handoff_check(Z, parent, g)
        dis = lab != ref
        cnt_gpu = np.bincount(lab, minlength=g["pi"].shape[0])
        out["levels"].append({
            "live_mismatch": int(np.sum(g["live"] != o.live)),
            "mu": float(e_mu.max(initial=0)), "S": float(e_S.max(initial=0)),
            "pi": float(e_pi.max(initial=0)),
            "label_disagree": int(dis.sum()),
            "label_disagree_not_tie": int(np.sum(dis & (margin >= TIE_MARGIN))),
            "count_mismatch": int(np.sum(cnt_gpu != g["count"])),
            "n_live": int(g["live"].sum()),
        })
        parent = lab
        p_mu, p_S = g["mu"], safe_sigma(g)
        p_cnt = np.where(g["live"], g["count"], 0)
    if report is not None:
        report.append(out)
    return out


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
