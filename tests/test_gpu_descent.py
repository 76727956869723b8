"""Descent variants of the registration E-step (Sec. 4.1) on the GPU vs the
FP64 oracle on the GPU's own tree: Algorithm 1 through the variant kernel
(against hgmm_register too), the path-product gamma, and the threshold-pruned
multi-path descent; first-round moments, 30 rounds, the LiDAR workload's
first round, mass conservation and determinism; and the full Eq. 7 M-step
(second moments, scatter terms) against the oracle's Gauss-Newton step over
the point contributions."""
import numpy as np
import pytest

from oracle import hgmm_oracle as O
from paper_1807_02587_gb300 import synth
from tests import parity as PT

pytestmark = pytest.mark.gpu

MODES = {"local": 0, "global": 1, "multipath": 2}


@pytest.fixture(scope="module")
def B():
    from paper_1807_02587_gb300 import binding
    return binding


def _setup(B, p, depth):
    tgt, Zt = PT.device_cloud(p["tgt"])
    src, Zs = PT.device_cloud(p["src"])
    tree = B.Tree(max(Zt.shape[0], Zs.shape[0]), depth)
    tree.build(tgt, depth)
    tree.sync()
    ot = PT.tree_from_gpu(tree, PT.oracle_params(B.params(), depth), tree.root()["extent"])
    return tree, ot, src, Zs


def _small():
    return synth.corner_pair(7, max_deg=3.0, max_t=0.02)


def _first_round(B, tree, ot, src, Zs, mode, tau):
    T1 = tree.register_descent(src, MODES[mode], tau, iters=1).cpu().numpy()
    tree.sync()
    g = tree.reg_moments()
    E = O.e_step_descent(ot, Zs, mode, tau)
    M0 = np.concatenate(E["M0"])
    M1 = np.concatenate(E["M1"])
    N = Zs.shape[0]
    extent = ot.extent
    dM0 = np.abs(g[:, 0] - M0)
    big = M0 > 5.0
    err = np.linalg.norm(M1[big] / M0[big, None] - g[big, 1:] / g[big, :1], axis=1) / extent
    T_o = O.register_descent(ot, Zs, mode, tau, iters=1)
    r, t = PT.pose_errors(T1, T_o, extent)
    print(mode, tau, "sum|dM0|", dM0.sum(), "of", M0.sum(), "mu* median", np.median(err), "pose", r, t)
    # posteriors in FP32; argmax and threshold decisions can flip only at
    # near-ties, each moving at most one point's share
    assert dM0.sum() <= 1e-4 * N + 2.0
    assert np.median(err) < 1e-6
    assert r < 2e-3 and t < 2e-5


@pytest.mark.parametrize("mode,tau", [("local", 0.0), ("global", 0.0), ("multipath", 0.01), ("multipath", 0.1)])
def test_first_round_matches_oracle(B, mode, tau):
    tree, ot, src, Zs = _setup(B, _small(), 3)
    _first_round(B, tree, ot, src, Zs, mode, tau)


@pytest.mark.parametrize("mode,tau", [("global", 0.0), ("multipath", 0.01)])
def test_first_round_on_lidar_workload(B, mode, tau):
    tree, ot, src, Zs = _setup(B, synth.lidar_pair(0), 4)
    _first_round(B, tree, ot, src, Zs, mode, tau)


@pytest.mark.parametrize("mode,tau", [("global", 0.0), ("multipath", 0.01)])
def test_thirty_rounds_match_oracle(B, mode, tau):
    p = _small()
    tree, ot, src, Zs = _setup(B, p, 3)
    T = tree.register_descent(src, MODES[mode], tau, iters=30).cpu().numpy()
    tree.sync()
    T_o = O.register_descent(ot, Zs, mode, tau, iters=30)
    r, t = PT.pose_errors(T, T_o, ot.extent)
    print(mode, "GPU vs oracle", r, t, "GPU vs truth", PT.pose_errors(T, p["T_gt"], ot.extent))
    assert r < PT.ROT_TOL_DEG and t < PT.TRANS_TOL_REL


def test_local_variant_equals_register(B):
    """Algorithm 1 through the variant kernels and through k_register: the
    same fixed-point node sums up to the FP32 order of the warp-group sums."""
    tree, ot, src, Zs = _setup(B, _small(), 3)
    a = tree.register(src, iters=30).cpu().numpy()
    b = tree.register_descent(src, 0, 0.0, iters=30).cpu().numpy()
    tree.sync()
    r, t = PT.pose_errors(a, b, ot.extent)
    assert r < 1e-4 and t < 1e-6, (r, t)


def test_multipath_conserves_mass(B):
    """No pruning, no early stop: each point's expectations over the ends of
    its paths sum to one, so M0 over all nodes is the point count."""
    tree, ot, src, Zs = _setup(B, _small(), 2)
    tree.register_descent(src, 2, 0.0, iters=1, lam_c=0.0)
    tree.sync()
    g = tree.reg_moments()
    assert g[:, 0].sum() == pytest.approx(Zs.shape[0], rel=1e-5)


def test_descent_is_deterministic(B):
    tree, ot, src, Zs = _setup(B, _small(), 3)
    a = tree.register_descent(src, 2, 0.01, iters=8).cpu().numpy()
    b = tree.register_descent(src, 2, 0.01, iters=8).cpu().numpy()
    tree.sync()
    assert np.array_equal(a, b)


def test_threshold_override_does_not_persist(B):
    """A registration with lambda_c = 0 sets the stop flags for that call
    only: the next call with the build's threshold gives the same pose as a
    fresh one."""
    tree, ot, src, Zs = _setup(B, _small(), 3)
    a = tree.register(src, iters=10).cpu().numpy()
    tree.register(src, iters=10, lam_c=0.0)
    tree.register_descent(src, 1, 0.0, iters=3, lam_c=0.0)
    b = tree.register(src, iters=10).cpu().numpy()
    tree.sync()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("mode,tau,name", [("local", 0.0, "corner"), ("multipath", 0.01, "corner"),
                                           ("local", 0.0, "lidar")])
def test_full_eq7_first_round_matches_oracle(B, mode, tau, name):
    """The full Eq. 7 M-step (scatter kept): the first round's pose and
    objective against the oracle's Gauss-Newton step over the point
    contributions."""
    import torch
    p, depth = (_small(), 3) if name == "corner" else (synth.lidar_pair(0), 4)
    tree, ot, src, Zs = _setup(B, p, depth)
    T1 = tree.register_descent(src, MODES[mode], tau, iters=1, full_eq7=True).cpu().numpy()
    obj = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.hgmm_register_objective(tree.handle, obj)
    tree.sync()
    T_o, h = O.register_eq7(ot, Zs, mode, tau, iters=1, history=True)
    r, t = PT.pose_errors(T1, T_o, ot.extent)
    T9 = O.register_descent(ot, Zs, mode, tau, iters=1)
    print(name, mode, "eq7 GPU vs oracle", r, t, "objective", obj.item(), h[0]["objective"],
          "eq7 vs eq9 step", PT.pose_errors(T_o, T9, ot.extent))
    assert r < 2e-3 and t < 2e-5
    assert obj.item() == pytest.approx(h[0]["objective"], rel=1e-3)


def test_full_eq7_thirty_rounds_match_oracle(B):
    p = _small()
    tree, ot, src, Zs = _setup(B, p, 3)
    T = tree.register_descent(src, 0, 0.0, iters=30, full_eq7=True).cpu().numpy()
    tree.sync()
    T_o = O.register_eq7(ot, Zs, "local", 0.0, iters=30)
    r, t = PT.pose_errors(T, T_o, ot.extent)
    print("eq7 30 rounds GPU vs oracle", r, t, "GPU vs truth", PT.pose_errors(T, p["T_gt"], ot.extent))
    assert r < PT.ROT_TOL_DEG and t < PT.TRANS_TOL_REL
