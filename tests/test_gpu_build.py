"""GPU tree build vs the FP64 oracle, level by level with teacher forcing
(the oracle re-runs each level's EM from the GPU's parent assignment and
parent parameters) - GMM-tree build of Sec. 3 / Sec. 4.1, Eq. 2-3."""
import numpy as np
import pytest

from oracle import hgmm_oracle as O
from paper_1807_02587_gb300 import synth
from tests import parity as PT

pytestmark = pytest.mark.gpu


def _cases():
    return {
        "corner10k_d3": (lambda: synth.corner_pair(0)["tgt"], 3),
        "corner4099_d2": (lambda: synth.corner_pair(1, n=4099)["tgt"], 2),
        "lidar_d4": (lambda: synth.lidar_pair(0)["tgt"], 4),
        "primitive50k_d4": (lambda: synth.primitive_pair(3, 50001)["tgt"], 4),
    }


@pytest.fixture(scope="module")
def B():
    from paper_1807_02587_gb300 import binding
    return binding


@pytest.mark.parametrize("case", list(_cases()))
def test_build_matches_oracle_teacher_forced(B, case):
    make, depth = _cases()[case]
    P = make()
    dev, Z = PT.device_cloud(P)
    prm = B.params()
    tree = B.Tree(Z.shape[0], depth)
    tree.build(dev, depth, prm)
    tree.sync()
    res = PT.check_build(tree, Z, PT.oracle_params(prm, depth))
    print(case, res)
    assert res["root_mu"] < 1e-6 and res["root_S"] < 1e-5 and res["extent"] < 1e-6
    for l, r in enumerate(res["levels"]):
        assert r["count_mismatch"] == 0, (l, r)
        assert r["live_mismatch"] == 0, (l, r)
        assert r["mu"] < PT.MEAN_TOL, (l, r)
        assert r["S"] < PT.COV_TOL, (l, r)
        assert r["pi"] < PT.PI_TOL, (l, r)
        assert r["label_disagree_not_tie"] == 0, (l, r)
        assert r["label_disagree"] <= max(3, 1e-3 * Z.shape[0]), (l, r)
        # near-tie / ill-conditioned parents are few
        assert r["excluded_parents"] <= max(2, 0.02 * r["parents_with_points"]), (l, r)


@pytest.mark.parametrize("case", ["corner10k_d3", "lidar_d4"])
def test_em_iteration_teacher_forced(B, case):
    """One EM iteration at a time: GPU parameters after iteration k against
    the oracle's iteration from the GPU's parameters after k-1 (every level;
    first, middle and last iteration)."""
    make, depth = _cases()[case]
    dev, Z = PT.device_cloud(make())
    steps = [(l, k) for l in range(depth) for k in (1, 4, 8)]
    res = PT.check_em_steps(B, dev, Z, depth, steps)
    for r in res:
        print(case, r)
        assert r["live_mismatch"] == 0, r
        assert r["mu"] < 1e-5 and r["S"] < 1e-5 and r["pi"] < 1e-5, r


def test_build_is_deterministic(B):
    P = synth.corner_pair(2)["tgt"]
    dev, Z = PT.device_cloud(P)
    tree = B.Tree(Z.shape[0], 3)
    outs = []
    for _ in range(2):
        tree.build(dev, 3)
        tree.sync()
        outs.append([tree.export(l) for l in range(3)] + [tree.labels(2)])
    for a, b in zip(outs[0][:3], outs[1][:3]):
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(outs[0][3], outs[1][3])


def test_plain_fp32_sums_differ_but_stay_close(B):
    """precision = 1 (plain FP32 moment sums) builds the same tree up to
    rounding; the compensated default is the one checked above."""
    P = synth.primitive_pair(5, 60000)["tgt"]
    dev, Z = PT.device_cloud(P)
    tree = B.Tree(Z.shape[0], 2)
    tree.build(dev, 2, B.params(precision=1))
    tree.sync()
    res = PT.check_build(tree, Z, PT.oracle_params(B.params(), 2))
    for r in res["levels"]:
        assert r["live_mismatch"] == 0
        assert r["mu"] < 1e-3 and r["S"] < 1e-3


@pytest.mark.parametrize("case", list(_cases()))
def test_cooperative_em_equals_per_iteration_launches(B, case):
    """One cooperative launch per level for all EM iterations performs the
    same E-step and M-step arithmetic as the per-iteration launches: the
    trees, their labels and a stopped build agree bit for bit."""
    make, depth = _cases()[case]
    dev, Z = PT.device_cloud(make())
    out = []
    for flags in (0, B.HGMM_FLAG_EM_COOPERATIVE):
        tree = B.Tree(Z.shape[0], depth)
        tree.build(dev, depth, B.params(flags=flags))
        tree.sync()
        levels = [tree.export(l) for l in range(depth)]
        labels = [tree.labels(l) for l in range(depth)]
        stopped = B.Tree(Z.shape[0], depth)
        stopped.build(dev, depth, B.params(flags=flags, debug_stop_level=depth, debug_stop_iters=3))
        stopped.sync()
        out.append((levels, labels, stopped.export(depth - 1)))
    for l in range(depth):
        for k in ("pi", "mu", "Sigma", "live", "count"):
            np.testing.assert_array_equal(out[0][0][l][k], out[1][0][l][k])
        np.testing.assert_array_equal(out[0][1][l], out[1][1][l])
    for k in ("pi", "mu", "Sigma", "live"):
        np.testing.assert_array_equal(out[0][2][k], out[1][2][k])


@pytest.mark.parametrize("case", ["corner10k_d3", "lidar_d4"])
def test_node_eigen_decomposition_is_fp64_accurate(B, case):
    """Every live node's eigenvalues (Sec. 4.1 complexity, Eq. 10 PCA form)
    against numpy's eigh of the same exported FP64 covariance: the FP32
    Jacobi + FP64 refinement must be accurate to FP64 level."""
    make, depth = _cases()[case]
    dev, Z = PT.device_cloud(make())
    tree = B.Tree(Z.shape[0], depth)
    tree.build(dev, depth)
    tree.sync()
    worst_l = worst_c = 0.0
    for l in range(depth):
        e = tree.export(l)
        live = e["live"]
        w = np.linalg.eigvalsh(e["Sigma"][live])[:, ::-1]
        err = np.abs(e["lam"][live] - w) / w[:, :1]
        cplx = w[:, 2] / w.sum(axis=1)
        worst_l = max(worst_l, float(err.max(initial=0)))
        worst_c = max(worst_c, float(np.abs(e["complexity"][live] - cplx).max(initial=0)))
    print(case, "eigenvalue rel err", worst_l, "complexity err", worst_c)
    assert worst_l < 1e-11 and worst_c < 1e-11


@pytest.mark.parametrize("name", ["corner", "lidar"])
def test_debug_posteriors_match_oracle(B, name):
    """hgmm_debug_posteriors: the Eq. 3 posteriors of every point over its
    parent's children at every level, element by element against the
    oracle's (log-sum-exp in FP64) under the GPU's own parameters and parent
    labels (teacher forcing).  FP32 scores carry an absolute error of about
    1e-7 of the squared Mahalanobis distance, which moves a posterior by at
    most a quarter of it."""
    if name == "corner":
        P, depth = synth.corner_pair(2)["tgt"], 3
    else:
        P, depth = synth.lidar_pair(0)["tgt"], 4
    dev, Z = PT.device_cloud(P)
    tree = B.Tree(Z.shape[0], depth)
    tree.build(dev, depth)
    tree.sync()
    N = Z.shape[0]
    parent = np.zeros(N, np.int64)
    for l in range(depth):
        g = tree.export(l)
        got = tree.posteriors(l).astype(np.float64)
        pi = np.where(g["live"], g["pi"], 0.0)
        ref, _ = O.posteriors(O.child_scores(Z, parent, pi, g["mu"], PT.safe_sigma(g)))
        err = np.abs(got - ref)
        leaf = ~np.isfinite(O.child_scores(Z, parent, pi, g["mu"], PT.safe_sigma(g)).max(axis=1))
        print(f"{name} level {l}: max |dgamma| {err.max():.2e}, p99.9 {np.percentile(err, 99.9):.2e}, "
              f"leaf-parent points {int(leaf.sum())}")
        assert np.all(got[leaf] == 0.0)
        sums = got[~leaf].sum(axis=1)
        assert np.all(np.abs(sums - 1.0) < 1e-5)
        assert err.max() < 1e-3 and np.percentile(err, 99.9) < 1e-5, (l, err.max())
        parent = tree.labels(l).astype(np.int64)
