"""Plain FP64 CPU oracle of hierarchical-GMM (HGMM) registration.

TEST INFRASTRUCTURE ONLY.  This module exists so that the CUDA path can be
checked against an obviously-correct restatement of the method.  Only the
test suite, the package smoke check and the benchmark's CPU-baseline leg may
import it; the library itself never does.  It shares no code with the CUDA
path: its only inputs are float64 numpy arrays.

Everything is float64 numpy, vectorised over points ("for z_i in parallel",
Algorithm 1) and written to be read against the paper:

* Eq. 2  GMM density, Eq. 3 posterior (E-step of the tree build and of the
  registration), computed as a log-sum-exp with the maximum subtracted.
* Sec. 3 / Sec. 4.1  GMM-tree build: a top-down hierarchy of 8-component GMM
  nodes.  The paper defers the build to its reference [33]; the steps below
  are this project's stated reading (PCA-octant child init, K fixed EM
  iterations per level on the hard-assigned points of each parent, dead
  children below ``n_min`` expected points, a parent whose children all die
  stays a leaf, argmax hand-off).
* Algorithm 1  E_STEP_ADAPTIVE: max-likelihood descent with the PCA
  complexity early stop (Sec. 4.1, lambda_c = 0.01), accumulation of the
  zeroth and first moments M0, M1 (and M2 for checking).
* Eq. 8-9  per-cluster reduction (pi*, mu*), Eq. 10-11 PCA form of the
  Mahalanobis distance, Eq. 12-16 the stacked weighted linear least-squares
  system of Low's point-to-plane linearisation, solved here with
  ``numpy.linalg.lstsq``; the update is T <- dT T with dT from the
  axis-angle (Rodrigues) map of the solved small rotation.

Readings where the paper is silent or garbled (each is listed in the design
notes of the repository):

* Eq. 14 prints b = n^T (mu* - mu); with the small-angle linearisation
  R mu* ~ mu* + w x mu* the right-hand side that drives T(mu*) toward mu is
  n^T (mu - mu*).  That sign is used (``test_mstep_reduces_objective`` pins it).
* Eq. 13's last weight is garbled (lambda_{J_1}); w_l = sqrt(pi*_j/lambda_{j,l})
  is used for every l.
* gamma[searchID] in Algorithm 1 is the posterior of the chosen node among the
  live children of its parent at the level where the descent stopped.
* A point whose current node has no live children stops there.
* Complexity(Theta) <= lambda_c stops the descent ("<=" as printed).
* Sec. 4.1's remark that a parent's expectation is the sum of its children's
  gives the variants of e_step_descent: gamma as the product of the sibling
  posteriors along the path, and the threshold-pruned multi-path descent
  (a child below tau is dropped with its subtree; each path stops as
  Algorithm 1's does).
* Eq. 8 replaces Eq. 7's double sum by one term per cluster and so drops the
  scatter of each cluster's points about mu*_j, which depends on R unless
  Sigma_j is isotropic; register_eq7 keeps it (Gauss-Newton over the point
  contributions).
* The flat "GMM J=n" variant (Sec. 5) does not say how its J components are
  obtained: here they are the leaves of the tree (weights = products of the
  within-parent weights), optionally refined by plain EM over all J, and the
  registration associates every point with every component softly (Eq. 3
  over all J, Eq. 8 moments), which is what removing the tree leaves.

Parity pins: every function here is checked by ``tests/test_oracle_*.py``
against closed forms, invariants and brute force (posteriors summing to one,
sibling mass equal to the parent's point count, EM monotonicity, recovery of
known blob mixtures, weighted Kabsch on isotropic clusters, brute-force flat
GMM association, recovery of a known transform).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

J = 8  # components per GMM node (Sec. 4.1: 8-component GMM nodes)
LOG_2PI = np.log(2.0 * np.pi)


@dataclass
class Params:
    """depth: number of tree levels L (level l holds 8^(l+1) nodes).
    em_iters: EM iterations per level (K).  n_min: a child whose expected
    point count drops below this dies.  lam_c: complexity threshold of
    Sec. 4.1.  eps_rel: covariance regulariser eps = (eps_rel * extent)^2."""
    depth: int = 3
    em_iters: int = 8
    n_min: float = 8.0
    lam_c: float = 0.01
    eps_rel: float = 1e-3


@dataclass
class Level:
    pi: np.ndarray        # (m,)   mixing weight within the parent's GMM
    mu: np.ndarray        # (m,3)
    Sigma: np.ndarray     # (m,3,3)
    live: np.ndarray      # (m,)   bool
    labels: np.ndarray    # (N,)   node index (within this level) of each point
    count: np.ndarray     # (m,)   hard point count after the hand-off
    lam: np.ndarray = None         # (m,3) eigenvalues, descending
    vec: np.ndarray = None         # (m,3,3) eigenvectors in columns
    complexity: np.ndarray = None  # (m,)
    loglik: list = field(default_factory=list)  # per EM iteration, per parent


@dataclass
class Tree:
    params: Params
    root_mu: np.ndarray
    root_Sigma: np.ndarray
    extent: float
    eps: float
    levels: list


# --------------------------------------------------------------------------
# Gaussian terms (Eq. 2, Eq. 3)
# --------------------------------------------------------------------------
def gauss_terms(Sigma):
    """Inverse and log-determinant of each covariance in a (m,3,3) stack."""
    inv = np.linalg.inv(Sigma)
    sign, logdet = np.linalg.slogdet(Sigma)
    return inv, logdet


def log_gauss(Z, mu, inv, logdet):
    """log N(z_i | mu_i, Sigma_i) for row-aligned stacks."""
    d = Z - mu
    q = np.einsum("ni,nij,nj->n", d, inv, d)
    return -0.5 * (q + logdet + 3.0 * LOG_2PI)


def sym_eig(S):
    """Eigen-decomposition of symmetric 3x3 stacks: eigenvalues descending
    (lambda_1 >= lambda_2 >= lambda_3, Sec. 4.1), eigenvector columns with the
    sign chosen so that the entry of largest magnitude is positive."""
    w, V = np.linalg.eigh(S)
    w = w[..., ::-1]
    V = V[..., ::-1]
    k = np.argmax(np.abs(V), axis=-2)  # (..., 3): row of largest |entry|
    s = np.take_along_axis(V, k[..., None, :], axis=-2)[..., 0, :]
    V = V * np.where(s < 0, -1.0, 1.0)[..., None, :]
    return w, V


def complexity(lam):
    """Complexity(Theta) = lambda_3 / (lambda_1 + lambda_2 + lambda_3), Sec. 4.1."""
    return lam[..., 2] / lam.sum(axis=-1)


# --------------------------------------------------------------------------
# GMM-tree build (Sec. 3, Sec. 4.1; construction after reference [33])
# --------------------------------------------------------------------------
def root_stats(Z):
    """Mean and (population) covariance of the whole cloud, and its extent
    (bounding-box diagonal)."""
    mu = Z.mean(axis=0)
    d = Z - mu
    Sigma = d.T @ d / Z.shape[0]
    extent = float(np.linalg.norm(Z.max(axis=0) - Z.min(axis=0)))
    return mu, Sigma, extent


def octant_children(mu_p, Sigma_p, eps):
    """Initial 8 children of a parent Gaussian: child k with sign bits
    s_a = +1 if bit a of k is set else -1 sits at
    mu_p + 1/2 sum_a s_a sqrt(lambda_a) v_a with covariance Sigma_p/4 + eps I
    and weight 1/8."""
    lam, V = sym_eig(Sigma_p)
    half = 0.5 * np.sqrt(np.maximum(lam, 0.0))
    mus = np.empty((J, 3))
    for k in range(J):
        s = np.array([1.0 if (k >> a) & 1 else -1.0 for a in range(3)])
        mus[k] = mu_p + V @ (s * half)
    Sig = np.repeat((Sigma_p / 4.0 + eps * np.eye(3))[None], J, axis=0)
    return mus, Sig, np.full(J, 1.0 / J)


def child_scores(Z, parent, pi, mu, Sigma):
    """(N, 8) matrix of log(pi_c N(z_i | Theta_c)) over the 8 children of each
    point's parent; -inf for dead children (pi_c = 0)."""
    inv, logdet = gauss_terms(Sigma)
    with np.errstate(divide="ignore"):
        logpi = np.log(pi)
    S = np.empty((Z.shape[0], J))
    for c in range(J):
        node = parent * J + c
        S[:, c] = logpi[node] + log_gauss(Z, mu[node], inv[node], logdet[node])
    return S


def posteriors(S):
    """Eq. 3 evaluated as a log-sum-exp with the row maximum subtracted.
    Returns the posteriors and the per-point log-likelihood log p(z_i).  A
    row without any live component (a leaf parent) gets zero posteriors."""
    m = S.max(axis=1, keepdims=True)
    none = ~np.isfinite(m)
    e = np.exp(S - np.where(none, 0.0, m))
    e[none[:, 0]] = 0.0
    tot = e.sum(axis=1, keepdims=True)
    with np.errstate(invalid="ignore", divide="ignore"):
        g = np.where(none, 0.0, e / np.where(none, 1.0, tot))
        ll = np.where(none, -np.inf, m + np.log(tot))
    return g, ll[:, 0]


def mstep_children(Z, parent, gamma, n_parents, n_points_parent, eps, n_min):
    """Maximisation step of every child GMM from the posteriors: expected
    counts S0_c, means, covariances (+ eps I) and weights pi_c = S0_c / n_p.
    A child whose expected count is below n_min dies (pi = 0); when all eight
    die the parent is not split (it stays a leaf).  Children of a parent
    without points are dead."""
    m = n_parents * J
    node = (parent[:, None] * J + np.arange(J)[None, :]).ravel()
    g = gamma.ravel()
    Zr = np.repeat(Z, J, axis=0)
    S0 = np.bincount(node, weights=g, minlength=m)
    S1 = np.stack([np.bincount(node, weights=g * Zr[:, a], minlength=m)
                   for a in range(3)], axis=1)
    with np.errstate(invalid="ignore", divide="ignore"):
        mu = S1 / S0[:, None]
    d = Zr - mu[node]
    Sigma = np.empty((m, 3, 3))
    for a in range(3):
        for b in range(3):
            Sigma[:, a, b] = np.bincount(node, weights=g * d[:, a] * d[:, b],
                                         minlength=m)
    with np.errstate(invalid="ignore", divide="ignore"):
        Sigma = Sigma / S0[:, None, None] + eps * np.eye(3)
        pi = S0 / np.repeat(n_points_parent, J)
    S0p = S0.reshape(n_parents, J)
    dead = S0p < n_min
    dead[n_points_parent == 0, :] = True
    live = ~dead.ravel()
    pi = np.where(live, pi, 0.0)
    return pi, mu, Sigma, live, S0


def init_children(n_parents, parent_mu, parent_Sigma, parent_count, eps):
    """Initial (pi, mu, Sigma, live) of all children: PCA octants of every
    parent that holds points; children of empty parents are dead."""
    m = n_parents * J
    pi = np.zeros(m)
    mu = np.zeros((m, 3))
    Sigma = np.repeat(np.eye(3)[None], m, axis=0)
    live = np.zeros(m, bool)
    for p in range(n_parents):
        if parent_count[p] == 0:
            continue
        cm, cS, cp = octant_children(parent_mu[p], parent_Sigma[p], eps)
        sl = slice(p * J, (p + 1) * J)
        mu[sl], Sigma[sl], pi[sl], live[sl] = cm, cS, cp, True
    return pi, mu, Sigma, live


def em_iteration(Z, parent, n_parents, parent_count, pi, mu, Sigma, eps, n_min):
    """One EM iteration of every parent's 8-child GMM on its own points:
    E-step (Eq. 3) with the current parameters, then the M-step.  Dead
    children keep their last parameters (they are never used again).
    Returns the new (pi, mu, Sigma, live), the expected counts S0 and the
    per-parent log-likelihood under the parameters the E-step used."""
    S = child_scores(Z, parent, pi, mu, Sigma)
    gamma, ll = posteriors(S)
    pi_n, mu_n, Sig_n, live_n, S0 = mstep_children(
        Z, parent, gamma, n_parents, parent_count, eps, n_min)
    mu = np.where(live_n[:, None], mu_n, mu)
    Sigma = np.where(live_n[:, None, None], Sig_n, Sigma)
    return pi_n, mu, Sigma, live_n, S0, np.bincount(parent, weights=ll, minlength=n_parents)


def build_level(Z, parent, n_parents, parent_mu, parent_Sigma, parent_count,
                params, eps):
    """One level of the top-down build.  ``parent`` gives each point's parent
    node (index within the previous level, 0 for the root).  Runs K EM
    iterations of every parent's 8-child GMM on that parent's points, then the
    argmax hand-off (ties to the lowest index)."""
    m = n_parents * J
    pi, mu, Sigma, live = init_children(n_parents, parent_mu, parent_Sigma, parent_count, eps)
    history, s0_hist = [], []
    for _ in range(params.em_iters):
        pi, mu, Sigma, live, S0, ll = em_iteration(
            Z, parent, n_parents, parent_count, pi, mu, Sigma, eps, params.n_min)
        history.append(ll)
        s0_hist.append(S0)
    S = child_scores(Z, parent, pi, mu, Sigma)
    _, ll = posteriors(S)
    history.append(np.bincount(parent, weights=ll, minlength=n_parents))
    labels = parent * J + np.argmax(S, axis=1)
    count = np.bincount(labels, minlength=m)
    lam = np.ones((m, 3))
    vec = np.repeat(np.eye(3)[None], m, axis=0)
    lam[live], vec[live] = sym_eig(Sigma[live])
    lv = Level(pi=pi, mu=mu, Sigma=Sigma, live=live, labels=labels,
               count=count, lam=lam, vec=vec, complexity=complexity(lam),
               loglik=history)
    lv.s0_hist = s0_hist
    return lv


def build_tree(Z, params: Params) -> Tree:
    """Top-down GMM-tree build of cloud Z (N,3), levels 0..depth-1."""
    Z = np.asarray(Z, dtype=np.float64)
    mu0, S0, extent = root_stats(Z)
    eps = (params.eps_rel * extent) ** 2
    parent = np.zeros(Z.shape[0], dtype=np.int64)
    p_mu, p_S, p_cnt = mu0[None], S0[None], np.array([Z.shape[0]])
    levels = []
    for _ in range(params.depth):
        lv = build_level(Z, parent, p_mu.shape[0], p_mu, p_S, p_cnt, params, eps)
        levels.append(lv)
        parent = lv.labels
        p_mu, p_S = lv.mu, lv.Sigma
        p_cnt = np.where(lv.live, lv.count, 0)
    return Tree(params=params, root_mu=mu0, root_Sigma=S0, extent=extent,
                eps=eps, levels=levels)


# --------------------------------------------------------------------------
# Registration E-step: Algorithm 1 (E_STEP_ADAPTIVE)
# --------------------------------------------------------------------------
def e_step_adaptive(tree: Tree, Zp, lam_c=None, want_m2=False):
    """Per point: descend the maximum-likelihood path from Children(-1) = the
    8 level-0 nodes; stop at the first chosen node whose complexity is at most
    lambda_c, or at the leaf level, or at a node without live children.  The
    point contributes gamma = its posterior among the siblings at the stopping
    level to the moments of the chosen node.

    Returns per level: M0 (m,), M1 (m,3) [, M2 (m,3,3)], and per point the
    (level, node, gamma) of its association."""
    lam_c = tree.params.lam_c if lam_c is None else lam_c
    N = Zp.shape[0]
    L = len(tree.levels)
    search = np.full(N, -1, dtype=np.int64)
    level_of = np.full(N, -1, dtype=np.int64)
    gamma = np.zeros(N)
    active = np.ones(N, bool)
    for l in range(L):
        lv = tree.levels[l]
        idx = np.nonzero(active)[0]
        if idx.size == 0:
            break
        base = np.zeros(idx.size, np.int64) if l == 0 else search[idx] * J
        cand = base[:, None] + np.arange(J)[None, :]
        has_live = lv.live[cand].any(axis=1)
        stopped = idx[~has_live]
        active[stopped] = False
        idx, base, cand = idx[has_live], base[has_live], cand[has_live]
        if idx.size == 0:
            break
        S = child_scores(Zp[idx], base // J, lv.pi, lv.mu, lv.Sigma)
        g, _ = posteriors(S)
        j = np.argmax(S, axis=1)
        search[idx] = cand[np.arange(idx.size), j]
        level_of[idx] = l
        gamma[idx] = g[np.arange(idx.size), j]
        stop = lv.complexity[search[idx]] <= lam_c
        active[idx[stop]] = False
    M0, M1, M2 = [], [], []
    for l in range(L):
        m = tree.levels[l].pi.shape[0]
        sel = level_of == l
        node = search[sel]
        g = gamma[sel]
        z = Zp[sel]
        M0.append(np.bincount(node, weights=g, minlength=m))
        M1.append(np.stack([np.bincount(node, weights=g * z[:, a], minlength=m)
                            for a in range(3)], axis=1))
        if want_m2:
            q = np.empty((m, 3, 3))
            for a in range(3):
                for b in range(3):
                    q[:, a, b] = np.bincount(node, weights=g * z[:, a] * z[:, b],
                                             minlength=m)
            M2.append(q)
    out = {"M0": M0, "M1": M1, "level": level_of, "node": search, "gamma": gamma}
    if want_m2:
        out["M2"] = M2
    return out


def e_step_descent(tree: Tree, Zp, mode: str, tau: float = 0.0, lam_c=None):
    """Variants of Algorithm 1's descent (Sec. 4.1).  A node's expectation
    for a point is the sum of its children's, so the expectation of a child
    is its parent's times the child's posterior among its siblings.

    mode "local":     the maximum-likelihood path; gamma = the stopping
                      node's posterior among its siblings (e_step_adaptive).
    mode "global":    the maximum-likelihood path; gamma = the product of the
                      sibling posteriors along the path (the expectation).
    mode "multipath": every live child whose expectation is >= tau is
                      descended, the others are pruned with their subtrees;
                      each path stops as Algorithm 1's does (complexity <=
                      lambda_c, the leaf level, or no live children) and adds
                      its expectation to the node where it stops.

    Returns M0, M1 per level and the contributions as arrays (point, level,
    node, gamma), one row per (point, stopping node)."""
    lam_c = tree.params.lam_c if lam_c is None else lam_c
    N = Zp.shape[0]
    L = len(tree.levels)
    # frontier: points whose search continues below node `par` (index within
    # level l - 1; -1 = the root) with expectation g_par
    pt = np.arange(N)
    par = np.full(N, -1, np.int64)
    g_par = np.ones(N)
    out_i, out_l, out_n, out_g = [], [], [], []

    def emit(i, l, node, g):
        out_i.append(i), out_l.append(np.full(i.size, l)), out_n.append(node), out_g.append(g)

    for l in range(L):
        if pt.size == 0:
            break
        lv = tree.levels[l]
        base = np.zeros(pt.size, np.int64) if l == 0 else par * J
        cand = base[:, None] + np.arange(J)[None, :]
        has_live = lv.live[cand].any(axis=1)
        if l > 0:  # a node without live children stops its path
            dead_end = ~has_live
            emit(pt[dead_end], l - 1, par[dead_end], g_par[dead_end])
        pt, par, g_par, cand = pt[has_live], par[has_live], g_par[has_live], cand[has_live]
        if pt.size == 0:
            break
        S = child_scores(Zp[pt], np.maximum(par, 0), lv.pi, lv.mu, lv.Sigma)
        post, _ = posteriors(S)
        if mode in ("local", "global"):
            k = np.argmax(S, axis=1)
            rows = np.arange(pt.size)
            child = cand[rows, k]
            g = post[rows, k] * (g_par if mode == "global" else 1.0)
            nxt_pt, nxt_child, nxt_g = pt, child, g
        elif mode == "multipath":
            g_all = post * g_par[:, None]
            keep = lv.live[cand] & (g_all >= tau)
            r, k = np.nonzero(keep)
            nxt_pt, nxt_child, nxt_g = pt[r], cand[r, k], g_all[r, k]
        else:
            raise ValueError(mode)
        stop = (lv.complexity[nxt_child] <= lam_c) | (l == L - 1)
        emit(nxt_pt[stop], l, nxt_child[stop], nxt_g[stop])
        go = ~stop
        # g_par: what the path adds if it ends at this node (local mode: the
        # node's own sibling posterior, as Algorithm 1 keeps it)
        pt, par, g_par = nxt_pt[go], nxt_child[go], nxt_g[go]
    ci, cl, cn, cg = (np.concatenate(a) if a else np.zeros(0) for a in (out_i, out_l, out_n, out_g))
    ci, cl, cn = ci.astype(np.int64), cl.astype(np.int64), cn.astype(np.int64)
    M0, M1 = [], []
    for l in range(L):
        m = tree.levels[l].pi.shape[0]
        sel = cl == l
        M0.append(np.bincount(cn[sel], weights=cg[sel], minlength=m))
        M1.append(np.stack([np.bincount(cn[sel], weights=cg[sel] * Zp[ci[sel], a], minlength=m)
                            for a in range(3)], axis=1))
    return {"M0": M0, "M1": M1, "point": ci, "level": cl, "node": cn, "gamma": cg}


# --------------------------------------------------------------------------
# Registration M-step: Eq. 8-16
# --------------------------------------------------------------------------
def cluster_stats(M0, M1, N):
    """Eq. 8-9: pi*_j = M0_j / N and mu*_j = M1_j / M0_j for clusters with mass."""
    used = M0 > 0
    return used, M0[used] / N, M1[used] / M0[used][:, None]


def stacked_system(mu_star, pi_star, mu, lam, vec):
    """Eq. 13-16: rows w_l [mu* x n_l, n_l] and right-hand sides
    w_l n_l^T (mu_j - mu*_j) for l = 1..3 and every used cluster j, with
    w_l = sqrt(pi*_j / lambda_{j,l})."""
    rows, rhs = [], []
    for l in range(3):
        n = vec[:, :, l]
        w = np.sqrt(pi_star / lam[:, l])
        b = np.einsum("ji,ji->j", n, mu - mu_star)
        a = np.concatenate([np.cross(mu_star, n), n], axis=1)
        rows.append(w[:, None] * a)
        rhs.append(w * b)
    return np.concatenate(rows), np.concatenate(rhs)


def rodrigues(w):
    th = np.linalg.norm(w)
    K = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])
    if th < 1e-300:
        return np.eye(3) + K
    return (np.eye(3) + np.sin(th) / th * K
            + (1.0 - np.cos(th)) / (th * th) * (K @ K))


def solve_increment(mu_star, pi_star, mu, lam, vec):
    """Least-squares solution x = (alpha, beta, gamma, tx, ty, tz) of Eq. 16."""
    A, b = stacked_system(mu_star, pi_star, mu, lam, vec)
    x, *_ = np.linalg.lstsq(A, b, rcond=None)
    return x


def increment_matrix(x):
    dT = np.eye(4)
    dT[:3, :3] = rodrigues(x[:3])
    dT[:3, 3] = x[3:]
    return dT


def objective(T, mu_star, pi_star, mu, lam, vec):
    """Eq. 11 / Eq. 12: sum_j sum_l pi*_j / lambda_jl (n_jl^T (T(mu*_j) - mu_j))^2."""
    y = mu_star @ T[:3, :3].T + T[:3, 3]
    r = np.einsum("jil,ji->jl", vec, y - mu)
    return float(np.sum(pi_star[:, None] / lam * r * r))


def model_eigen(tree: Tree, level: int, node):
    lv = tree.levels[level]
    lam = np.maximum(lv.lam[node], tree.eps)
    return lv.mu[node], lam, lv.vec[node]


def register_descent(tree: Tree, Z2, mode: str, tau: float = 0.0, T_init=None, iters=30,
                     lam_c=None, history=False):
    """`register` with the E-step of e_step_descent(mode, tau); the M-step
    (Eq. 8-16) and the update are the same."""
    Z2 = np.asarray(Z2, dtype=np.float64)
    T = np.eye(4) if T_init is None else np.array(T_init, dtype=np.float64)
    N = Z2.shape[0]
    hist = []
    for _ in range(iters):
        Zp = Z2 @ T[:3, :3].T + T[:3, 3]
        E = e_step_descent(tree, Zp, mode, tau, lam_c)
        ms, ps, mus, lams, vecs = [], [], [], [], []
        for l in range(len(tree.levels)):
            used, pstar, mstar = cluster_stats(E["M0"][l], E["M1"][l], N)
            node = np.nonzero(used)[0]
            mu, lam, vec = model_eigen(tree, l, node)
            ms.append(mstar), ps.append(pstar), mus.append(mu)
            lams.append(lam), vecs.append(vec)
        mstar, pstar = np.concatenate(ms), np.concatenate(ps)
        mu, lam, vec = np.concatenate(mus), np.concatenate(lams), np.concatenate(vecs)
        x = solve_increment(mstar, pstar, mu, lam, vec)
        if history:
            hist.append({"T_start": T.copy(), "x": x, "M0": E["M0"], "M1": E["M1"],
                         "objective": objective(np.eye(4), mstar, pstar, mu, lam, vec)})
        T = increment_matrix(x) @ T
    return (T, hist) if history else T


def eq7_objective(T, Z2, contrib, mu, P):
    """Eq. 7: sum over (point i, node j) contributions of
    gamma_ij (T(z_i) - mu_j)^T Sigma_j^-1 (T(z_i) - mu_j), with Sigma_j^-1
    taken as P_j = V diag(1 / max(lambda, eps)) V^T; contrib = (point, row,
    gamma) with `row` indexing mu / P."""
    i, r, g = contrib
    y = Z2[i] @ T[:3, :3].T + T[:3, 3] - mu[r]
    return float(np.sum(g * np.einsum("ka,kab,kb->k", y, P[r], y)))


def eq7_increment(Zp, contrib, mu, lam, vec):
    """Gauss-Newton step of Eq. 7 at the current pose (the points already
    moved, Zp = T(Z2)): for every contribution and every eigen-direction l a
    point-to-plane row w [z'_i x n_l, n_l] with right-hand side
    w n_l^T (mu_j - z'_i), w = sqrt(gamma_ij / lambda_jl) (Eq. 10 applied to
    each point instead of to mu*_j), solved by least squares."""
    i, r, g = contrib
    rows, rhs = [], []
    for l in range(3):
        n = vec[r, :, l]
        w = np.sqrt(g / lam[r, l])
        rows.append(w[:, None] * np.concatenate([np.cross(Zp[i], n), n], axis=1))
        rhs.append(w * np.einsum("ka,ka->k", n, mu[r] - Zp[i]))
    x, *_ = np.linalg.lstsq(np.concatenate(rows), np.concatenate(rhs), rcond=None)
    return x


def _node_table(tree):
    """Every node of the tree stacked level by level: mu, eigen (lambda
    floored at eps), precision P."""
    mus, lams, vecs = [], [], []
    for l, lv in enumerate(tree.levels):
        idx = np.arange(lv.pi.shape[0])
        mu, lam, vec = model_eigen(tree, l, idx)
        mus.append(mu), lams.append(lam), vecs.append(vec)
    mu, lam, vec = np.concatenate(mus), np.concatenate(lams), np.concatenate(vecs)
    P = np.einsum("kal,kl,kbl->kab", vec, 1.0 / lam, vec)
    offs = np.cumsum([0] + [lv.pi.shape[0] for lv in tree.levels])
    return mu, lam, vec, P, offs


def register_eq7(tree: Tree, Z2, mode: str = "local", tau: float = 0.0, T_init=None, iters=30,
                 lam_c=None, history=False):
    """EM registration with the full Eq. 7 M-step: the E-step of
    e_step_descent(mode, tau), then one Gauss-Newton step of Eq. 7 over the
    (point, node) contributions (keeping the scatter of each node's points
    that Eq. 8-9 drop) and T <- dT T."""
    Z2 = np.asarray(Z2, dtype=np.float64)
    T = np.eye(4) if T_init is None else np.array(T_init, dtype=np.float64)
    mu, lam, vec, P, offs = _node_table(tree)
    hist = []
    for _ in range(iters):
        Zp = Z2 @ T[:3, :3].T + T[:3, 3]
        E = e_step_descent(tree, Zp, mode, tau, lam_c)
        contrib = (E["point"], offs[E["level"]] + E["node"], E["gamma"])
        x = eq7_increment(Zp, contrib, mu, lam, vec)
        if history:
            hist.append({"T_start": T.copy(), "x": x,
                         "objective": eq7_objective(np.eye(4), Zp, contrib, mu, P) / Z2.shape[0]})
        T = increment_matrix(x) @ T
    return (T, hist) if history else T


def register(tree: Tree, Z2, T_init=None, iters=30, lam_c=None, history=False):
    """EM registration of source Z2 (N,3) into the tree's frame (Eq. 1):
    alternate Algorithm 1 and the M-step of Eq. 9-16 for ``iters`` rounds.
    Returns T (4x4) and, if requested, the per-iteration transforms and
    moments."""
    Z2 = np.asarray(Z2, dtype=np.float64)
    T = np.eye(4) if T_init is None else np.array(T_init, dtype=np.float64)
    N = Z2.shape[0]
    hist = []
    for _ in range(iters):
        Zp = Z2 @ T[:3, :3].T + T[:3, 3]
        E = e_step_adaptive(tree, Zp, lam_c)
        ms, ps, mus, lams, vecs = [], [], [], [], []
        for l in range(len(tree.levels)):
            used, pstar, mstar = cluster_stats(E["M0"][l], E["M1"][l], N)
            node = np.nonzero(used)[0]
            mu, lam, vec = model_eigen(tree, l, node)
            ms.append(mstar), ps.append(pstar), mus.append(mu)
            lams.append(lam), vecs.append(vec)
        mstar, pstar = np.concatenate(ms), np.concatenate(ps)
        mu, lam, vec = np.concatenate(mus), np.concatenate(lams), np.concatenate(vecs)
        x = solve_increment(mstar, pstar, mu, lam, vec)
        T = increment_matrix(x) @ T
        if history:
            hist.append({"T": T.copy(), "x": x, "M0": E["M0"], "M1": E["M1"]})
    return (T, hist) if history else T


# --------------------------------------------------------------------------
# Flat "GMM J=n" association (Sec. 5 variant 3), for cross-checking
# --------------------------------------------------------------------------
def flat_associate(Zp, pi, mu, Sigma):
    """Linear search over all components of a single-level GMM: Eq. 3
    posteriors and the argmax association of every point."""
    n = Zp.shape[0]
    inv, logdet = gauss_terms(Sigma)
    with np.errstate(divide="ignore"):
        lp = np.log(pi)
    S = np.stack([lp[c] + log_gauss(Zp, np.broadcast_to(mu[c], Zp.shape),
                                    np.broadcast_to(inv[c], (n, 3, 3)),
                                    np.full(n, logdet[c]))
                  for c in range(pi.shape[0])], axis=1)
    g, _ = posteriors(S)
    return g, np.argmax(S, axis=1)


# --------------------------------------------------------------------------
# Flat "GMM J=n" variant (Sec. 5, variant 3): a single-level GMM, every
# point associated with every component (O(NJ)), the same Eq. 9-16 M-step
# --------------------------------------------------------------------------
@dataclass
class Flat:
    pi: np.ndarray      # (J,) mixing weights over the whole cloud (0 = dead)
    mu: np.ndarray      # (J,3)
    Sigma: np.ndarray   # (J,3,3)
    node: np.ndarray    # (J,2) (level, index) of the tree node each started from
    eps: float

    @property
    def live(self):
        return self.pi > 0.0


def flat_from_tree(tree: Tree, level=None) -> Flat:
    """The single-level GMM a tree defines at the scale of `level` (default:
    its deepest level).  Components: every live node of that level and every
    live node of a shallower level without a live child (the leaves of the
    tree cut below `level`).  Weight: the product of the within-parent
    weights pi along the node's path from level 0 (the mixture weight the
    hierarchy gives it), the weights renormalised to sum to one.  Ordered by
    level, then by index within the level."""
    L = len(tree.levels) if level is None else level + 1
    glob = []
    for l in range(L):
        lv = tree.levels[l]
        up = np.ones(lv.pi.shape[0]) if l == 0 else np.repeat(glob[l - 1], J)
        glob.append(np.where(lv.live, lv.pi * up, 0.0))
    pis, mus, Sigs, nodes = [], [], [], []
    for l in range(L):
        lv = tree.levels[l]
        if l + 1 < L:
            has_child = tree.levels[l + 1].live.reshape(-1, J).any(axis=1)
        else:
            has_child = np.zeros(lv.pi.shape[0], bool)
        sel = np.nonzero(lv.live & ~has_child)[0]
        pis.append(glob[l][sel])
        mus.append(lv.mu[sel])
        Sigs.append(lv.Sigma[sel])
        nodes.append(np.stack([np.full(sel.size, l), sel], axis=1))
    pi = np.concatenate(pis)
    return Flat(pi=pi / pi.sum(), mu=np.concatenate(mus), Sigma=np.concatenate(Sigs),
                node=np.concatenate(nodes), eps=tree.eps)


def flat_scores(Zp, flat: Flat):
    """(N, J) matrix of log(pi_j N(z_i | Theta_j)) (Eq. 2 terms); -inf for
    dead components."""
    inv, logdet = gauss_terms(flat.Sigma)
    with np.errstate(divide="ignore"):
        lp = np.log(flat.pi)
    n = Zp.shape[0]
    S = np.empty((n, flat.pi.shape[0]))
    for c in range(flat.pi.shape[0]):
        S[:, c] = lp[c] + log_gauss(Zp, np.broadcast_to(flat.mu[c], Zp.shape),
                                    np.broadcast_to(inv[c], (n, 3, 3)), np.full(n, logdet[c]))
    return S


def flat_em(Z, flat: Flat, iters: int, n_min: float = 8.0):
    """`iters` EM iterations of the flat GMM on cloud Z: Eq. 3 posteriors of
    every point over all components, then pi_j = S0_j / N, mu_j = S1_j / S0_j,
    Sigma_j = sum_i gamma_ij (z_i - mu_j)(z_i - mu_j)^T / S0_j + eps I.  A
    component below n_min expected points dies (pi = 0) and keeps its last
    parameters.  Returns the new Flat and the log-likelihood sum_i log p(z_i)
    under the parameters each E-step used."""
    Z = np.asarray(Z, np.float64)
    pi, mu, Sigma = flat.pi.copy(), flat.mu.copy(), flat.Sigma.copy()
    lls = []
    for _ in range(iters):
        g, ll = posteriors(flat_scores(Z, Flat(pi, mu, Sigma, flat.node, flat.eps)))
        lls.append(float(ll.sum()))
        S0 = g.sum(axis=0)
        live = (pi > 0.0) & (S0 >= n_min) & (S0 > 0.0)
        with np.errstate(invalid="ignore", divide="ignore"):
            mu_n = (g.T @ Z) / S0[:, None]
        Sig_n = np.empty_like(Sigma)
        for c in range(pi.shape[0]):
            d = Z - mu_n[c]
            with np.errstate(invalid="ignore", divide="ignore"):
                Sig_n[c] = (g[:, c, None] * d).T @ d / S0[c] + flat.eps * np.eye(3)
        mu = np.where(live[:, None], mu_n, mu)
        Sigma = np.where(live[:, None, None], Sig_n, Sigma)
        pi = np.where(live, S0 / Z.shape[0], 0.0)
    return Flat(pi=pi, mu=mu, Sigma=Sigma, node=flat.node, eps=flat.eps), lls


def flat_moments(flat: Flat, Zp):
    """Eq. 8 with the flat model: M0_j = sum_i gamma_ij, M1_j = sum_i
    gamma_ij z'_i over every point and component."""
    g, _ = posteriors(flat_scores(Zp, flat))
    return g.sum(axis=0), g.T @ Zp


def register_flat(flat: Flat, Z2, T_init=None, iters=30, history=False):
    """EM registration of source Z2 to the flat GMM (Eq. 1): each round the
    flat moments at the current pose, then the same M-step as the tree
    (Eq. 9-16 with lambda clamped at eps) and T <- dT T."""
    Z2 = np.asarray(Z2, dtype=np.float64)
    T = np.eye(4) if T_init is None else np.array(T_init, dtype=np.float64)
    N = Z2.shape[0]
    lam_all, vec_all = sym_eig(flat.Sigma)
    lam_all = np.maximum(lam_all, flat.eps)
    hist = []
    for _ in range(iters):
        Zp = Z2 @ T[:3, :3].T + T[:3, 3]
        M0, M1 = flat_moments(flat, Zp)
        used, pstar, mstar = cluster_stats(M0, M1, N)
        x = solve_increment(mstar, pstar, flat.mu[used], lam_all[used], vec_all[used])
        if history:
            hist.append({"T_start": T.copy(), "x": x, "M0": M0, "M1": M1,
                         "objective": objective(np.eye(4), mstar, pstar, flat.mu[used],
                                                lam_all[used], vec_all[used])})
        T = increment_matrix(x) @ T
    return (T, hist) if history else T


# --------------------------------------------------------------------------
# Helpers for parity checks against exported trees
# --------------------------------------------------------------------------
def tree_from_arrays(params: Params, extent: float, levels: list) -> Tree:
    """Build an oracle Tree from exported per-level arrays (pi, mu, Sigma,
    live); eigen-decompositions are recomputed here in float64."""
    eps = (params.eps_rel * extent) ** 2
    out = []
    for d in levels:
        pi = np.asarray(d["pi"], np.float64)
        mu = np.asarray(d["mu"], np.float64)
        Sigma = np.asarray(d["Sigma"], np.float64)
        live = np.asarray(d["live"], bool)
        lam = np.ones((pi.shape[0], 3))
        vec = np.repeat(np.eye(3)[None], pi.shape[0], axis=0)
        if live.any():
            lam[live], vec[live] = sym_eig(Sigma[live])
        pi = np.where(live, pi, 0.0)
        out.append(Level(pi=pi, mu=mu, Sigma=Sigma, live=live,
                         labels=d.get("labels"), count=d.get("count"),
                         lam=lam, vec=vec, complexity=complexity(lam)))
    return Tree(params=params, root_mu=None, root_Sigma=None, extent=extent,
                eps=eps, levels=out)


def rotation_error_deg(R_a, R_b):
    c = (np.trace(R_a.T @ R_b) - 1.0) / 2.0
    return float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))
