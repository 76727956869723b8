"""Pins of the FP64 oracle against closed forms, invariants, independent
library routines and brute force (no GPU).

Each test names the passage of the paper it checks.  A plausible mistake in
the oracle (a dropped term, a wrong sign, a transposed operand, a wrong index
into the tree) makes at least one of these fail; ``test_planted_*`` shows it
for the two readings that are easiest to get wrong.
"""
import numpy as np
import pytest
from scipy.stats import multivariate_normal

from oracle import hgmm_oracle as O
from paper_1807_02587_gb300 import synth as S


def _rand_spd(rng, scale=1.0):
    A = rng.normal(size=(3, 3))
    return scale * (A @ A.T + 0.3 * np.eye(3))


# ------------------------------------------------- root statistics (Sec. 3)
def test_root_stats_closed_form_box_vertices():
    """The whole-cloud Gaussian that seeds the tree (Children(-1) of
    Algorithm 1 are fitted inside it) and the extent that sets the
    regulariser: the 8 vertices of an axis-aligned box with sides (2, 4, 6)
    centred at c, each repeated k times, have mean c, population covariance
    diag(1, 4, 9) (every coordinate is +-half a side with equal weight;
    the N-1 sample form would give 8k/(8k-1) times that) and bounding-box
    diagonal sqrt(2^2 + 4^2 + 6^2) = sqrt(56); a rigid motion moves the mean
    with it, rotates the covariance to R diag R^T and leaves the extent of
    an axis-aligned box's bounding box unchanged under a translation."""
    c = np.array([0.3, -1.2, 5.0])
    half = np.array([1.0, 2.0, 3.0])
    V = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)], float)
    for k in (1, 3):
        Z = np.repeat(c + V * half, k, axis=0)
        mu, Sig, ext = O.root_stats(Z)
        assert np.allclose(mu, c, atol=1e-14)
        assert np.allclose(Sig, np.diag([1.0, 4.0, 9.0]), atol=1e-13)
        assert abs(ext - np.sqrt(56.0)) < 1e-13
    # rotated box: covariance R diag R^T; the bounding box of the rotated
    # vertices is wider than the box (extent = diagonal of that box)
    R = S.axis_angle_matrix(np.array([0.0, 0.0, 1.0]), np.pi / 2)
    Z = (c + V * half) @ R.T
    mu, Sig, ext = O.root_stats(Z)
    assert np.allclose(mu, R @ c, atol=1e-13)
    assert np.allclose(Sig, np.diag([4.0, 1.0, 9.0]), atol=1e-13)  # x and y sides swapped
    assert abs(ext - np.sqrt(56.0)) < 1e-13
    R45 = S.axis_angle_matrix(np.array([0.0, 0.0, 1.0]), np.pi / 4)
    _, _, ext45 = O.root_stats((V * half) @ R45.T)
    # extents of the rotated rectangle's bounding box along x and y: (2 + 4)/sqrt(2) each
    assert abs(ext45 - np.sqrt(2 * (6.0 / np.sqrt(2)) ** 2 + 6.0 ** 2)) < 1e-12


# ---------------------------------------------------------------- Eq. 2 / Eq. 3
def test_log_gauss_matches_scipy_density():
    """Eq. 2: the oracle's Gaussian log-density equals scipy's independent
    multivariate-normal implementation."""
    rng = np.random.default_rng(0)
    for _ in range(5):
        mu = rng.normal(size=3)
        Sig = _rand_spd(rng)
        Z = rng.normal(size=(50, 3)) * 2
        inv, logdet = O.gauss_terms(Sig[None])
        got = O.log_gauss(Z, np.broadcast_to(mu, Z.shape),
                          np.broadcast_to(inv[0], (50, 3, 3)),
                          np.full(50, logdet[0]))
        ref = multivariate_normal(mu, Sig).logpdf(Z)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_posterior_is_bayes_rule_bruteforce():
    """Eq. 3 by brute force: pi_j N_j / sum_k pi_k N_k with densities from
    scipy, one point and one component at a time."""
    rng = np.random.default_rng(1)
    pi = rng.uniform(0.1, 1.0, size=8)
    pi /= pi.sum()
    mu = rng.normal(size=(8, 3))
    Sig = np.stack([_rand_spd(rng, 0.5) for _ in range(8)])
    Z = rng.normal(size=(20, 3))
    g, lab = O.flat_associate(Z, pi, mu, Sig)
    for i in range(Z.shape[0]):
        dens = [pi[c] * multivariate_normal(mu[c], Sig[c]).pdf(Z[i]) for c in range(8)]
        tot = sum(dens)
        for c in range(8):
            assert abs(g[i, c] - dens[c] / tot) < 1e-12
        assert lab[i] == int(np.argmax(dens))
    np.testing.assert_allclose(g.sum(axis=1), 1.0, atol=1e-13)


def test_posteriors_sum_to_one_with_dead_children():
    rng = np.random.default_rng(2)
    S_ = rng.normal(size=(100, 8)) * 30
    S_[:, 3] = -np.inf
    g, ll = O.posteriors(S_)
    np.testing.assert_allclose(g.sum(1), 1.0, atol=1e-13)
    assert np.all(g[:, 3] == 0)
    np.testing.assert_allclose(ll, np.log(np.exp(S_ - 50).sum(1)) + 50, rtol=1e-12)


# ---------------------------------------------------------------- eigen / PCA
def test_sym_eig_closed_form():
    """lambda_1 >= lambda_2 >= lambda_3 (Sec. 4.1) of R diag(3, 2, 0.5) R^T are
    3, 2, 0.5 with eigenvectors the columns of R (largest entry positive)."""
    rng = S.make_rng(3)
    R = S.random_rotation(rng, 180)
    Sig = R @ np.diag([3.0, 2.0, 0.5]) @ R.T
    lam, V = O.sym_eig(Sig[None])
    np.testing.assert_allclose(lam[0], [3.0, 2.0, 0.5], rtol=1e-13)
    for a in range(3):
        v = V[0][:, a]
        r = R[:, a] * np.sign(R[np.argmax(np.abs(R[:, a])), a])
        np.testing.assert_allclose(v, r, atol=1e-12)
        assert v[np.argmax(np.abs(v))] > 0
    np.testing.assert_allclose(V[0] @ np.diag(lam[0]) @ V[0].T, Sig, atol=1e-13)


def test_complexity_closed_form():
    """Complexity = lambda_3 / (lambda_1 + lambda_2 + lambda_3) (Sec. 4.1)."""
    assert O.complexity(np.array([1.0, 1.0, 0.01])) == pytest.approx(0.01 / 2.01)
    assert O.complexity(np.array([1.0, 1.0, 1.0])) == pytest.approx(1.0 / 3.0)


def test_octant_init_closed_form():
    """PCA-octant child init: child k sits at mu_p + 1/2 sum_a s_a sqrt(l_a) v_a."""
    mu_p = np.array([1.0, -2.0, 0.5])
    Sig_p = np.diag([4.0, 1.0, 0.25])
    mus, Sig, pi = O.octant_children(mu_p, Sig_p, eps=1e-6)
    for k in range(8):
        s = np.array([1 if k & 1 else -1, 1 if k & 2 else -1, 1 if k & 4 else -1])
        np.testing.assert_allclose(mus[k], mu_p + 0.5 * s * np.array([2.0, 1.0, 0.5]))
        np.testing.assert_allclose(Sig[k], Sig_p / 4 + 1e-6 * np.eye(3))
    np.testing.assert_allclose(pi, 1 / 8)


# ---------------------------------------------------------------- tree build
def test_sibling_mass_equals_parent_count():
    """Sec. 4.1: a parent's expectation is the sum of its children's; with
    posteriors over the 8 siblings, sum_c S0_c equals the parent's point count."""
    Z = S.corner_scene(S.make_rng(4), 3000)
    tree = O.build_tree(Z, O.Params(depth=2))
    prev = np.zeros(Z.shape[0], np.int64)
    for lv in tree.levels:
        n_par = lv.pi.shape[0] // 8
        Sx = O.child_scores(Z, prev, lv.pi, lv.mu, lv.Sigma)
        g, _ = O.posteriors(Sx)
        *_, S0 = O.mstep_children(Z, prev, g, n_par,
                                  np.bincount(prev, minlength=n_par), tree.eps, 8)
        split = lv.live.reshape(n_par, 8).any(1)  # leaf parents keep zero posteriors
        np.testing.assert_allclose(S0.reshape(n_par, 8).sum(1),
                                   np.where(split, np.bincount(prev, minlength=n_par), 0),
                                   rtol=1e-12)
        assert lv.count.sum() == Z.shape[0]
        prev = lv.labels


def test_em_loglik_monotone_per_parent():
    """EM never decreases the likelihood (Sec. 3): with no regulariser and no
    child removal, every parent's log-likelihood is non-decreasing."""
    Z = S.corner_scene(S.make_rng(5), 4000)
    tree = O.build_tree(Z, O.Params(depth=2, em_iters=10, eps_rel=0.0, n_min=0.0))
    for lv in tree.levels:
        ll = np.array(lv.loglik)
        d = np.diff(ll, axis=0)
        assert np.all(d >= -1e-9 * np.abs(ll[1:]).max()), d.min()


def _octant_blobs(seed, n_per=400):
    rng = S.make_rng(seed)
    centers = [np.array([4.0 * (1 if k & 1 else -1), 2.0 * (1 if k & 2 else -1),
                         1.0 * (1 if k & 4 else -1)]) for k in range(8)]
    covs = []
    for _ in range(8):
        R = S.random_rotation(rng, 180)
        covs.append(R @ np.diag([0.02, 0.005, 0.0005]) @ R.T)
    return S.blob_cloud(seed, n_per, centers, covs), centers


def test_blob_mixture_recovery():
    """With 8 well separated anisotropic blobs the level-0 EM fixed point is
    the blobs' own sample means and covariances (posteriors are 0/1)."""
    (Z, y), centers = _octant_blobs(6)
    tree = O.build_tree(Z, O.Params(depth=1, em_iters=15, eps_rel=0.0))
    lv = tree.levels[0]
    assert lv.live.all()
    for c in range(8):
        k = int(np.argmin([np.linalg.norm(lv.mu[c] - ce) for ce in centers]))
        P = Z[y == k]
        np.testing.assert_allclose(lv.mu[c], P.mean(0), atol=1e-10)
        np.testing.assert_allclose(lv.Sigma[c], np.cov(P.T, bias=True), atol=1e-10)
        assert lv.pi[c] == pytest.approx(1 / 8, abs=1e-12)
        assert np.all(lv.labels[y == k] == c)


def test_dead_children_and_terminal_nodes():
    """Children with fewer than n_min expected points get pi = 0 and never
    receive points; a parent without points, or whose children all fall below
    n_min, has no live children; a parent with >= 8 n_min points always has
    one (pigeonhole)."""
    Z = S.corner_scene(S.make_rng(7), 600)
    tree = O.build_tree(Z, O.Params(depth=3, n_min=8))
    for l, lv in enumerate(tree.levels):
        assert np.all(lv.pi[~lv.live] == 0)
        n_par = lv.pi.shape[0] // 8
        live_par = lv.live.reshape(n_par, 8).any(1)
        # points of a leaf parent stay on its (dead) first child's segment
        assert np.all(lv.count[~lv.live & ~np.repeat(~live_par, 8)] == 0)
        par_count = (np.where(tree.levels[l - 1].live, tree.levels[l - 1].count, 0)
                     if l else np.array([Z.shape[0]]))
        assert np.all(live_par[par_count >= 64])
        assert not np.any(live_par[par_count == 0])
        tot = lv.pi.reshape(n_par, 8).sum(1)[live_par]
        assert np.all(tot <= 1.0 + 1e-12) and np.all(tot > 0.5)


# ---------------------------------------------------------------- Algorithm 1
def _bruteforce_descent(tree, Zp, lam_c):
    out = []
    for z in Zp:
        parent, res = None, None
        for l, lv in enumerate(tree.levels):
            cand = list(range(8)) if parent is None else list(range(parent * 8, parent * 8 + 8))
            live = [c for c in cand if lv.live[c]]
            if not live:
                break
            dens = {c: lv.pi[c] * multivariate_normal(lv.mu[c], lv.Sigma[c]).pdf(z)
                    for c in live}
            tot = sum(dens.values())
            j = max(live, key=lambda c: (dens[c], -c))
            res = (l, j, dens[j] / tot)
            parent = j
            if lv.complexity[j] <= lam_c:
                break
        out.append(res)
    return out


@pytest.mark.parametrize("lam_c", [0.0, 0.01, 0.03])
def test_descent_matches_bruteforce(lam_c):
    """Algorithm 1 line by line for each point with scipy densities: level,
    node and gamma[searchID] of every point's association."""
    Z = S.corner_scene(S.make_rng(8), 2500)
    tree = O.build_tree(Z, O.Params(depth=3))
    Zp = S.corner_scene(S.make_rng(9), 60)
    E = O.e_step_adaptive(tree, Zp, lam_c=lam_c)
    ref = _bruteforce_descent(tree, Zp, lam_c)
    for i, (l, j, g) in enumerate(ref):
        assert E["level"][i] == l and E["node"][i] == j
        assert E["gamma"][i] == pytest.approx(g, rel=1e-9)
    # M0/M1 are the gamma-weighted sums of the associated points (Alg. 1 L14)
    for l in range(3):
        m0 = np.zeros(tree.levels[l].pi.shape[0])
        for i, (li, j, g) in enumerate(ref):
            if li == l:
                m0[j] += g
        np.testing.assert_allclose(E["M0"][l], m0, atol=1e-12)


def test_flat_tree_descent_is_flat_gmm_association():
    """Depth 1 with lambda_c = 0 is a flat 8-GMM ("GMM J=n", Sec. 5): the
    descent association equals the linear-search argmax."""
    Z = S.corner_scene(S.make_rng(10), 2000)
    tree = O.build_tree(Z, O.Params(depth=1, lam_c=0.0))
    lv = tree.levels[0]
    Zp = S.corner_scene(S.make_rng(11), 500)
    E = O.e_step_adaptive(tree, Zp, lam_c=0.0)
    g, lab = O.flat_associate(Zp, lv.pi, lv.mu, lv.Sigma)
    assert np.array_equal(E["node"], lab)
    np.testing.assert_allclose(E["gamma"], g[np.arange(500), lab], rtol=1e-12)


# ---------------------------------------------------------------- Eq. 8-16
def _weighted_kabsch(P, Q, w):
    """argmin_R,t sum_j w_j |R p_j + t - q_j|^2 by SVD (closed form)."""
    w = w / w.sum()
    pc, qc = w @ P, w @ Q
    H = (P - pc).T @ (w[:, None] * (Q - qc))
    U, _, Vt = np.linalg.svd(H)
    D = np.diag([1, 1, np.sign(np.linalg.det(Vt.T @ U.T))])
    R = Vt.T @ D @ U.T
    return R, qc - R @ pc


def test_isotropic_mstep_converges_to_weighted_kabsch():
    """With Sigma_j = I, Eq. 11 is weighted point-to-point least squares; the
    iterated linearised solve of Eq. 16 converges to the SVD solution."""
    rng = np.random.default_rng(12)
    J_ = 30
    ms = rng.normal(size=(J_, 3))
    R = S.random_rotation(rng, 25)
    mu = ms @ R.T + np.array([0.2, -0.1, 0.05]) + 0.05 * rng.normal(size=(J_, 3))
    pi = rng.uniform(0.2, 1.0, J_)
    lam = np.ones((J_, 3))
    vec = np.repeat(S.random_rotation(rng, 180)[None], J_, axis=0)
    T = np.eye(4)
    for _ in range(25):
        x = O.solve_increment(ms @ T[:3, :3].T + T[:3, 3], pi, mu, lam, vec)
        T = O.increment_matrix(x) @ T
    Rk, tk = _weighted_kabsch(ms, mu, pi)
    np.testing.assert_allclose(T[:3, :3], Rk, atol=1e-10)
    np.testing.assert_allclose(T[:3, 3], tk, atol=1e-10)


def _aniso_clusters(seed, J_=40):
    rng = np.random.default_rng(seed)
    ms = rng.uniform(-1, 1, size=(J_, 3))
    vec = np.stack([S.random_rotation(rng, 180) for _ in range(J_)])
    lam = np.stack([np.sort(rng.uniform(1e-4, 1e-1, 3))[::-1] for _ in range(J_)])
    pi = rng.uniform(0.2, 1.0, J_) / J_
    return rng, ms, vec, lam, pi


def test_exact_correspondence_is_fixed_point():
    """If mu_j = T(mu*_j) exactly, Eq. 16's solution at that T is zero."""
    rng, ms, vec, lam, pi = _aniso_clusters(13)
    T = S.rigid(S.random_rotation(rng, 20), [0.1, 0.2, -0.3])
    mu = S.apply(T, ms)
    x = O.solve_increment(S.apply(T, ms), pi, mu, lam, vec)
    assert np.abs(x).max() < 1e-12


def test_pca_rows_equal_mahalanobis():
    """Eq. 10: sum_l (1/lambda_l) (n_l^T d)^2 = d^T Sigma^-1 d, so at x = 0 the
    stacked residual of Eq. 16 is the pi*-weighted Mahalanobis sum of Eq. 8."""
    rng, ms, vec, lam, pi = _aniso_clusters(14)
    mu = ms + 0.05 * rng.normal(size=ms.shape)
    A, b = O.stacked_system(ms, pi, mu, lam, vec)
    Sig = np.einsum("jal,jl,jbl->jab", vec, lam, vec)
    d = mu - ms
    maha = np.einsum("ja,jab,jb->j", d, np.linalg.inv(Sig), d)
    assert float(b @ b) == pytest.approx(float(np.sum(pi * maha)), rel=1e-12)
    assert O.objective(np.eye(4), ms, pi, mu, lam, vec) == pytest.approx(float(b @ b), rel=1e-12)


def test_mstep_reduces_objective():
    """One solve of Eq. 16 lowers Eq. 11's objective (pins the sign of b)."""
    rng, ms, vec, lam, pi = _aniso_clusters(15)
    T_true = S.rigid(S.random_rotation(rng, 3), [0.01, -0.02, 0.01])
    mu = S.apply(T_true, ms) + 0.001 * rng.normal(size=ms.shape)
    f0 = O.objective(np.eye(4), ms, pi, mu, lam, vec)
    x = O.solve_increment(ms, pi, mu, lam, vec)
    f1 = O.objective(O.increment_matrix(x), ms, pi, mu, lam, vec)
    assert f1 < 0.05 * f0


def test_planted_sign_error_is_caught():
    """Eq. 14 taken literally (b = n^T (mu* - mu)) raises the objective: the
    sign test above fails for that mistake."""
    rng, ms, vec, lam, pi = _aniso_clusters(15)
    T_true = S.rigid(S.random_rotation(rng, 3), [0.01, -0.02, 0.01])
    mu = S.apply(T_true, ms) + 0.001 * rng.normal(size=ms.shape)
    A, b = O.stacked_system(ms, pi, mu, lam, vec)
    x_bad, *_ = np.linalg.lstsq(A, -b, rcond=None)
    f0 = O.objective(np.eye(4), ms, pi, mu, lam, vec)
    assert O.objective(O.increment_matrix(x_bad), ms, pi, mu, lam, vec) > f0


def test_planted_transposed_cross_is_caught():
    """Using n x mu* in place of mu* x n in Eq. 16 breaks the fixed point."""
    rng, ms, vec, lam, pi = _aniso_clusters(16)
    T = S.rigid(S.random_rotation(rng, 10), [0.1, 0.0, 0.0])
    mu = S.apply(T, ms)
    A, b = O.stacked_system(ms, pi, mu, lam, vec)
    A_bad = A.copy()
    A_bad[:, :3] *= -1
    x_good, *_ = np.linalg.lstsq(A, b, rcond=None)
    x_bad, *_ = np.linalg.lstsq(A_bad, b, rcond=None)
    Tg = O.increment_matrix(x_good)
    Tb = O.increment_matrix(x_bad)
    assert O.rotation_error_deg(Tg[:3, :3], T[:3, :3]) < O.rotation_error_deg(Tb[:3, :3], T[:3, :3])


def test_rodrigues_closed_form():
    w = np.array([0.3, -0.2, 0.5])
    R = O.rodrigues(w)
    np.testing.assert_allclose(R, S.axis_angle_matrix(w, np.linalg.norm(w)), atol=1e-14)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)


# ---------------------------------------------------------------- whole method
def test_blob_registration_recovers_known_transform():
    """Eq. 1 on a cloud of 8 tight anisotropic blobs: the source is the target
    moved by a known rigid motion drawn with the Sec. 5 protocol (+-15 deg per
    axis, +-0.05 translation); registration recovers it."""
    (Z, _), _ = _octant_blobs(17, n_per=150)
    rng = S.make_rng(18)
    T_gt = S.rigid(S.euler_xyz_rotation(rng, 15), rng.uniform(-0.05, 0.05, 3))
    src = S.apply(np.linalg.inv(T_gt), Z)
    tree = O.build_tree(Z, O.Params(depth=1, em_iters=15))
    T = O.register(tree, src, iters=20)
    assert O.rotation_error_deg(T[:3, :3], T_gt[:3, :3]) < 0.01
    assert np.linalg.norm(T[:3, 3] - T_gt[:3, 3]) < 1e-4


def test_self_registration_small_perturbation():
    """A 2 degree perturbation of the model cloud itself is undone to within
    the method's fixed-point bias (10k points, depth 3)."""
    Z = S.corner_scene(S.make_rng(0), 10000)
    tree = O.build_tree(Z, O.Params(depth=3))
    T0 = S.rigid(S.axis_angle_matrix([1, 2, 3], np.deg2rad(2.0)), [0.0, 0, 0])
    T = O.register(tree, Z, T_init=T0, iters=20)
    assert O.rotation_error_deg(T[:3, :3], np.eye(3)) < 0.2
    assert np.linalg.norm(T[:3, 3]) < 5e-3
