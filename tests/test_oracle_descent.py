"""Pins of the oracle's descent variants (Sec. 4.1: a node's expectation is
the sum of its children's; the maximum-likelihood path with local or
path-product gamma; threshold-pruned multi-path descent) against the pinned
Algorithm 1 E-step, the pinned flat GMM, mass conservation, a brute-force
enumeration and a known transform (no GPU)."""
import numpy as np
import pytest

from oracle import hgmm_oracle as O
from paper_1807_02587_gb300 import synth as S


@pytest.fixture(scope="module")
def corner():
    Z = S.corner_scene(S.make_rng(7), 2500)
    return Z, O.build_tree(Z, O.Params(depth=3))


@pytest.mark.parametrize("lam_c", [0.01, 0.0])
def test_local_mode_is_algorithm_1(corner, lam_c):
    Z, tree = corner
    a = O.e_step_adaptive(tree, Z, lam_c)
    b = O.e_step_descent(tree, Z, "local", lam_c=lam_c)
    for l in range(3):
        np.testing.assert_array_equal(a["M0"][l], b["M0"][l])
        np.testing.assert_array_equal(a["M1"][l], b["M1"][l])


def test_multipath_on_one_level_is_the_soft_gmm(corner):
    """Depth 1, no pruning: every level-0 node receives the point's Eq. 3
    posterior over the level-0 GMM, i.e. the flat GMM's moments (pinned
    against scipy's densities)."""
    Z, _ = corner
    tree = O.build_tree(Z, O.Params(depth=1))
    m = O.e_step_descent(tree, Z, "multipath", tau=0.0)
    M0, M1 = O.flat_moments(O.flat_from_tree(tree), Z)
    live = np.nonzero(tree.levels[0].live)[0]
    np.testing.assert_allclose(m["M0"][0][live], M0, rtol=1e-12)
    np.testing.assert_allclose(m["M1"][0][live], M1, rtol=1e-10, atol=1e-12)


def test_multipath_conserves_each_subtree_mass(corner):
    """No pruning and no early stop: a point's expectations over the nodes
    where its paths end sum to one, and over the ends inside the subtree of
    level-0 node p to its level-0 posterior of p (the sum rule of Sec. 4.1)."""
    Z, tree = corner
    m = O.e_step_descent(tree, Z, "multipath", tau=0.0, lam_c=0.0)
    tot = np.zeros(Z.shape[0])
    np.add.at(tot, m["point"], m["gamma"])
    np.testing.assert_allclose(tot, 1.0, atol=1e-12)
    g0, _ = O.posteriors(O.child_scores(Z, np.zeros(Z.shape[0], np.int64), tree.levels[0].pi,
                                        tree.levels[0].mu, tree.levels[0].Sigma))
    top = m["node"] >> (3 * m["level"])  # level-0 ancestor of each end node
    per = np.zeros((Z.shape[0], 8))
    np.add.at(per, (m["point"], top), m["gamma"])
    np.testing.assert_allclose(per, g0, atol=1e-12)


def _brute_force(tree, z, tau, lam_c):
    """Recursive enumeration from the root: a live node whose expectation
    (product of sibling posteriors along its path) reaches tau is an end if
    it stops (complexity <= lam_c, last level, or no live child); otherwise
    its children are visited.  A node below tau is skipped with its subtree,
    and a node whose live children all fall below tau ends nothing."""
    ends = {}
    L = len(tree.levels)

    def visit(l, parent, g_parent):
        lv = tree.levels[l]
        kids = np.arange(8) + 8 * parent
        if not lv.live[kids].any():
            return False
        post, _ = O.posteriors(O.child_scores(z[None], np.array([parent]), lv.pi, lv.mu, lv.Sigma))
        for k, c in enumerate(kids):
            if not lv.live[c]:
                continue
            g = g_parent * post[0, k]
            if g < tau:
                continue
            if lv.complexity[c] <= lam_c or l == L - 1 or not visit(l + 1, c, g):
                ends[(l, int(c))] = g
        return True

    visit(0, 0, 1.0)
    return ends


def test_multipath_pruning_matches_enumeration(corner):
    Z, tree = corner
    pts = Z[:25]
    for tau in (0.02, 0.2):
        m = O.e_step_descent(tree, pts, "multipath", tau=tau)
        for i in range(pts.shape[0]):
            sel = m["point"] == i
            got = {(int(l), int(n)): g for l, n, g in zip(m["level"][sel], m["node"][sel], m["gamma"][sel])}
            want = _brute_force(tree, pts[i], tau, tree.params.lam_c)
            assert got.keys() == want.keys()
            for k in got:
                assert got[k] == pytest.approx(want[k], rel=1e-12)


def test_multipath_above_one_half_is_the_global_path(corner):
    """With tau > 1/2 at most one child of a node can pass, and it is the
    maximum-likelihood one: the multi-path ends are exactly the global-mode
    ends whose expectation reaches tau, and pruning only removes mass."""
    Z, tree = corner
    g = O.e_step_descent(tree, Z, "global")
    m = O.e_step_descent(tree, Z, "multipath", tau=0.51)
    keep = g["gamma"] >= 0.51
    got = sorted(zip(m["point"], m["level"], m["node"], m["gamma"]))
    want = sorted(zip(g["point"][keep], g["level"][keep], g["node"][keep], g["gamma"][keep]))
    assert len(got) == len(want)
    for a, b in zip(got, want):
        assert a[:3] == b[:3] and a[3] == pytest.approx(b[3], rel=1e-14)
    loc = O.e_step_descent(tree, Z, "local")
    assert np.all(g["gamma"] <= loc["gamma"][np.argsort(loc["point"])][g["point"]] + 1e-15)
    masses = [sum(x.sum() for x in O.e_step_descent(tree, Z, "multipath", tau=t)["M0"])
              for t in (0.0, 1e-3, 1e-2, 0.1, 0.5)]
    assert all(a >= b - 1e-9 for a, b in zip(masses, masses[1:]))


def _blobs(seed):
    rng = S.make_rng(6)
    centers = [np.array([2.0 * (1 if k & 1 else -1), 1.5 * (1 if k & 2 else -1),
                         1.0 * (1 if k & 4 else -1)]) for k in range(8)]
    covs = []
    for _ in range(8):
        R = S.random_rotation(rng, 180)
        covs.append(R @ np.diag([0.3, 0.1, 0.02]) @ R.T)
    Z, _ = S.blob_cloud(seed, 300, centers, covs)
    return Z


@pytest.mark.parametrize("mode,tau", [("global", 0.0), ("multipath", 0.01)])
def test_descent_variants_recover_known_transform(mode, tau):
    """Sec. 5 protocol (+-15 deg per axis, +-0.05): the source is the model
    cloud moved by a known motion; each variant recovers it to the accuracy
    the tree's fixed-point bias allows on 2400 points."""
    Z = _blobs(3)
    tree = O.build_tree(Z, O.Params(depth=2, em_iters=8))
    rng = S.make_rng(9)
    T_gt = S.rigid(S.euler_xyz_rotation(rng, 15), rng.uniform(-0.05, 0.05, 3))
    src = S.apply(np.linalg.inv(T_gt), Z)
    T = O.register_descent(tree, src, mode, tau, iters=40)
    assert O.rotation_error_deg(T[:3, :3], T_gt[:3, :3]) < 0.2
    assert np.linalg.norm(T[:3, 3] - T_gt[:3, 3]) < 5e-3
    T_l = O.register(tree, src, iters=40)
    print(mode, O.rotation_error_deg(T[:3, :3], T_gt[:3, :3]), O.rotation_error_deg(T_l[:3, :3], T_gt[:3, :3]))
