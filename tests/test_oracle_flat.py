"""Pins of the oracle's flat "GMM J=n" variant (Sec. 5, variant 3) against a
hand-worked tree, the labels of a real build, scipy's densities, scikit-
learn's EM step, the EM invariants and known transforms (no GPU)."""
import numpy as np
import pytest
from scipy.stats import multivariate_normal

from oracle import hgmm_oracle as O
from paper_1807_02587_gb300 import synth as S


def _level(pi, live, mu=None):
    m = len(pi)
    mu = np.zeros((m, 3)) if mu is None else mu
    Sig = np.repeat(np.eye(3)[None], m, axis=0)
    return O.Level(pi=np.asarray(pi, float), mu=mu, Sigma=Sig, live=np.asarray(live, bool),
                   labels=None, count=None)


def test_flat_from_tree_hand_example():
    """Two levels worked by hand.  Level 0: nodes 0 and 1 live (pi 0.6, 0.4).
    Level 1: node 0's children 0 and 1 live (pi 0.25, 0.75); node 1 has no
    live child.  Components: level-0 node 1 (a leaf, weight 0.4) and level-1
    nodes 0 and 1 (weights 0.6 x 0.25 = 0.15 and 0.6 x 0.75 = 0.45)."""
    pi0 = [0.6, 0.4] + [0.0] * 6
    live0 = [1, 1] + [0] * 6
    pi1 = [0.25, 0.75] + [0.0] * 62
    live1 = [1, 1] + [0] * 62
    mu1 = np.arange(64 * 3, dtype=float).reshape(64, 3)
    tree = O.Tree(params=O.Params(depth=2), root_mu=None, root_Sigma=None, extent=1.0,
                  eps=1e-6, levels=[_level(pi0, live0), _level(pi1, live1, mu1)])
    f = O.flat_from_tree(tree)
    assert f.node.tolist() == [[0, 1], [1, 0], [1, 1]]
    np.testing.assert_allclose(f.pi, [0.4, 0.15, 0.45], rtol=0, atol=1e-15)
    np.testing.assert_array_equal(f.mu[1:], mu1[:2])
    # cut at level 0: the two level-0 nodes, renormalised
    f0 = O.flat_from_tree(tree, level=0)
    assert f0.node.tolist() == [[0, 0], [0, 1]]
    np.testing.assert_allclose(f0.pi, [0.6, 0.4], atol=1e-15)
    # weights that do not sum to one are renormalised
    tree.levels[1].pi[:2] = [0.2, 0.6]
    np.testing.assert_allclose(O.flat_from_tree(tree).pi, np.array([0.4, 0.12, 0.36]) / 0.88, atol=1e-15)


def test_flat_components_are_the_ends_of_the_hard_paths():
    """On a real build, the components with points are exactly the deepest
    live nodes of the points' hard-assignment paths (a point never stops at
    a live node that has a live child: the argmax hand-off picks a live
    child), computed here from the labels alone."""
    Z = S.corner_scene(S.make_rng(7), 3000)
    tree = O.build_tree(Z, O.Params(depth=3, n_min=8))
    f = O.flat_from_tree(tree)
    ends = set()
    for i in range(Z.shape[0]):
        last = None
        for l, lv in enumerate(tree.levels):
            node = int(lv.labels[i])
            if not lv.live[node]:
                break
            last = (l, node)
        ends.add(last)
    comp = {(int(l), int(j)) for l, j in f.node}
    assert ends <= comp
    with_pts = {(l, j) for l, j in comp if tree.levels[l].count[j] > 0}
    assert with_pts == ends
    assert f.pi.sum() == pytest.approx(1.0, abs=1e-12) and np.all(f.pi > 0)


def test_flat_scores_match_scipy_mixture():
    """Eq. 2 / Eq. 3 over all components: log pi_j + log N(z | Theta_j) from
    scipy's multivariate normal, posteriors by Bayes' rule."""
    rng = np.random.default_rng(3)
    Jn = 5
    mu = rng.normal(size=(Jn, 3))
    Sig = np.stack([(lambda A: A @ A.T + 0.2 * np.eye(3))(rng.normal(size=(3, 3))) for _ in range(Jn)])
    pi = rng.uniform(0.1, 1.0, Jn)
    pi /= pi.sum()
    f = O.Flat(pi=pi, mu=mu, Sigma=Sig, node=np.zeros((Jn, 2), int), eps=0.0)
    Z = rng.normal(size=(40, 3)) * 1.5
    S_ = O.flat_scores(Z, f)
    ref = np.stack([np.log(pi[c]) + multivariate_normal(mu[c], Sig[c]).logpdf(Z) for c in range(Jn)], axis=1)
    np.testing.assert_allclose(S_, ref, rtol=1e-12, atol=1e-12)
    M0, M1 = O.flat_moments(f, Z)
    dens = np.exp(ref)
    g = dens / dens.sum(axis=1, keepdims=True)
    np.testing.assert_allclose(M0, g.sum(axis=0), rtol=1e-12)
    np.testing.assert_allclose(M1, g.T @ Z, rtol=1e-12, atol=1e-12)


def test_flat_em_step_matches_sklearn():
    """One EM iteration equals scikit-learn's GaussianMixture step (full
    covariances, reg_covar = eps) from the same initial parameters."""
    mixture = pytest.importorskip("sklearn.mixture")
    Z = S.corner_scene(S.make_rng(2), 1500)
    tree = O.build_tree(Z, O.Params(depth=1, em_iters=3))
    f = O.flat_from_tree(tree)
    eps = 1e-4
    f = O.Flat(pi=f.pi, mu=f.mu, Sigma=f.Sigma, node=f.node, eps=eps)
    got, _ = O.flat_em(Z, f, 1, n_min=0.0)
    gm = mixture.GaussianMixture(n_components=f.pi.size, covariance_type="full", reg_covar=eps,
                                 max_iter=1, tol=0.0, weights_init=f.pi, means_init=f.mu,
                                 precisions_init=np.linalg.inv(f.Sigma))
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        gm.fit(Z)
    np.testing.assert_allclose(got.pi, gm.weights_, rtol=1e-9)
    np.testing.assert_allclose(got.mu, gm.means_, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(got.Sigma, gm.covariances_, rtol=1e-8, atol=1e-12)


def test_flat_em_loglik_monotone_and_blob_recovery():
    """EM never lowers the log-likelihood (eps = 0, no deaths); with eight
    well separated blobs its fixed point is the blobs' sample means,
    covariances and proportions."""
    rng = S.make_rng(6)
    centers = [np.array([4.0 * (1 if k & 1 else -1), 2.0 * (1 if k & 2 else -1),
                         1.0 * (1 if k & 4 else -1)]) for k in range(8)]
    covs = []
    for _ in range(8):
        R = S.random_rotation(rng, 180)
        covs.append(R @ np.diag([0.02, 0.005, 0.0005]) @ R.T)
    Z, y = S.blob_cloud(6, 300, centers, covs)
    tree = O.build_tree(Z, O.Params(depth=1, em_iters=2, eps_rel=0.0))
    f = O.flat_from_tree(tree)
    got, lls = O.flat_em(Z, f, 25, n_min=0.0)
    assert np.all(np.diff(lls) >= -1e-9 * abs(lls[0]))
    for c in range(8):
        k = int(np.argmin([np.linalg.norm(got.mu[c] - ce) for ce in centers]))
        P = Z[y == k]
        np.testing.assert_allclose(got.mu[c], P.mean(0), atol=1e-9)
        np.testing.assert_allclose(got.Sigma[c], np.cov(P.T, bias=True), atol=1e-9)
        assert got.pi[c] == pytest.approx(1 / 8, abs=1e-12)


def _soft_blobs(seed, n_per=200):
    """Eight anisotropic blobs that overlap (about 6 % of the points have no
    posterior above 0.99), so flat EM converges quickly to a fixed point
    whose posteriors are not all 0 or 1."""
    rng = S.make_rng(6)
    centers = [np.array([2.0 * (1 if k & 1 else -1), 1.5 * (1 if k & 2 else -1),
                         1.0 * (1 if k & 4 else -1)]) for k in range(8)]
    covs = []
    for _ in range(8):
        R = S.random_rotation(rng, 180)
        covs.append(R @ np.diag([0.6, 0.2, 0.04]) @ R.T)
    Z, _ = S.blob_cloud(seed, n_per, centers, covs)
    tree = O.build_tree(Z, O.Params(depth=1, em_iters=2))
    return Z, O.flat_from_tree(tree)


def test_flat_em_fixed_point_registers_to_identity():
    """At an EM fixed point of the flat GMM on Z, Z itself has mu*_j = mu_j
    for every component (Eq. 8-9), so Eq. 16's right-hand side vanishes and
    registering Z from the identity leaves it there (away from the fixed
    point the first increment is of order 1e-3)."""
    Z, f0 = _soft_blobs(4)
    f, _ = O.flat_em(Z, f0, 150, n_min=0.0)
    f2, _ = O.flat_em(Z, f, 1, n_min=0.0)
    assert np.max(np.abs(f2.mu - f.mu)) < 1e-12  # converged
    g, _ = O.posteriors(O.flat_scores(Z, f))
    assert np.mean(g.max(axis=1) < 0.99) > 0.03  # soft association
    T, hist = O.register_flat(f, Z, iters=2, history=True)
    assert np.max(np.abs(hist[0]["x"])) < 1e-12
    np.testing.assert_allclose(T, np.eye(4), atol=1e-12)
    _, h0 = O.register_flat(f0, Z, iters=1, history=True)
    assert np.max(np.abs(h0[0]["x"])) > 1e-4


def test_flat_registration_recovers_known_transform():
    """The source is the model cloud moved by a known motion (Sec. 5
    protocol: +-15 deg per axis, +-0.05 translation); with the flat GMM at
    an EM fixed point of the model cloud the true pose is a fixed point of
    the registration, and 40 rounds from the identity reach it."""
    Z, f0 = _soft_blobs(5)
    f, _ = O.flat_em(Z, f0, 150, n_min=0.0)
    rng = S.make_rng(8)
    T_gt = S.rigid(S.euler_xyz_rotation(rng, 15), rng.uniform(-0.05, 0.05, 3))
    src = S.apply(np.linalg.inv(T_gt), Z)
    T = O.register_flat(f, src, iters=40)
    assert O.rotation_error_deg(T[:3, :3], T_gt[:3, :3]) < 1e-6
    assert np.linalg.norm(T[:3, 3] - T_gt[:3, 3]) < 1e-8


def test_planted_flat_rhs_sign_error_is_caught():
    """The sign reading of Eq. 14, planted wrong in the flat registration,
    makes the known-transform recovery fail."""
    Z, f0 = _soft_blobs(5)
    f, _ = O.flat_em(Z, f0, 150, n_min=0.0)
    T_gt = S.rigid(S.axis_angle_matrix([1, -2, 1], np.deg2rad(6.0)), [0.02, -0.01, 0.03])
    src = S.apply(np.linalg.inv(T_gt), Z)
    orig = O.stacked_system
    try:
        def flipped(*a):
            A, b = orig(*a)
            return A, -b
        O.stacked_system = flipped
        T = O.register_flat(f, src, iters=20)
    finally:
        O.stacked_system = orig
    assert O.rotation_error_deg(T[:3, :3], T_gt[:3, :3]) > 1.0
