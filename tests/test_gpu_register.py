"""GPU registration (Algorithm 1 + Eq. 9-16) vs the FP64 oracle.

* teacher-forced tree: the oracle registers on the GPU's exported tree, so
  only the registration arithmetic is compared;
* first-round moments M0, M1 per node (Algorithm 1, Eq. 9);
* free-running: oracle build + register against GPU build + register.
"""
import numpy as np
import pytest

from oracle import hgmm_oracle as O
from paper_1807_02587_gb300 import synth
from tests import parity as PT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1807_02587_gb300 import binding
    return binding


def _pair(name):
    if name == "lidar":
        return synth.lidar_pair(0), 4
    if name == "corner_small":
        return synth.corner_pair(7, max_deg=3.0, max_t=0.02), 3
    if name == "depth":
        return synth.depth_pair(0), 4
    raise KeyError(name)


def _gpu_run(B, p, depth, iters, T_init=None, lam_c=-1.0):
    import torch
    tgt, Zt = PT.device_cloud(p["tgt"])
    src, Zs = PT.device_cloud(p["src"])
    tree = B.Tree(max(Zt.shape[0], Zs.shape[0]), depth)
    tree.build(tgt, depth)
    Ti = None if T_init is None else torch.tensor(T_init, dtype=torch.float64, device="cuda")
    hist = torch.zeros((max(iters, 1), 4, 4), dtype=torch.float64, device="cuda")
    T = tree.register(src, Ti, iters=iters, lam_c=lam_c, T_hist=hist)
    tree.sync()
    return tree, Zt, Zs, T.cpu().numpy(), hist.cpu().numpy()


@pytest.mark.parametrize("name", ["lidar", "corner_small"])
def test_register_on_gpu_tree_matches_oracle(B, name):
    p, depth = _pair(name)
    tree, Zt, Zs, T_gpu, hist = _gpu_run(B, p, depth, 30)
    extent = tree.root()["extent"]
    ot = PT.tree_from_gpu(tree, PT.oracle_params(B.params(), depth), extent)
    T_or, h_or = O.register(ot, Zs, iters=30, history=True)
    errs = [PT.pose_errors(hist[k], h_or[k]["T"], extent) for k in range(30)]
    print(name, "per-iteration (deg, rel t):", [(round(a, 5), f"{b:.1e}") for a, b in errs[::5]])
    r, t = PT.pose_errors(T_gpu, T_or, extent)
    assert r < PT.ROT_TOL_DEG and t < PT.TRANS_TOL_REL, (r, t)


@pytest.mark.parametrize("name", ["lidar", "corner_small"])
def test_first_round_moments_match_oracle(B, name):
    p, depth = _pair(name)
    tree, Zt, Zs, T_gpu, _ = _gpu_run(B, p, depth, 1)
    extent = tree.root()["extent"]
    ot = PT.tree_from_gpu(tree, PT.oracle_params(B.params(), depth), extent)
    E = O.e_step_adaptive(ot, Zs)
    M0 = np.concatenate(E["M0"])
    M1 = np.concatenate(E["M1"])
    g = tree.reg_moments()
    N = Zs.shape[0]
    # points whose descent could flip between FP32 and FP64: near-tie margins
    dM0 = np.abs(g[:, 0] - M0)
    assert dM0.sum() <= 1e-4 * N + 1.0, dM0.sum()
    assert np.isclose(g[:, 0].sum(), M0.sum(), rtol=1e-5)
    big = M0 > 5.0
    mstar_o = M1[big] / M0[big, None]
    mstar_g = g[big, 1:] / g[big, :1]
    err = np.linalg.norm(mstar_o - mstar_g, axis=1) / extent
    assert np.median(err) < 1e-6, np.median(err)


@pytest.mark.parametrize("name", ["lidar"])
def test_free_running_matches_oracle(B, name):
    p, depth = _pair(name)
    tree, Zt, Zs, T_gpu, _ = _gpu_run(B, p, depth, 30)
    prm_o = PT.oracle_params(B.params(), depth)
    ot = O.build_tree(Zt, prm_o)
    T_or = O.register(ot, Zs, iters=30)
    r, t = PT.pose_errors(T_gpu, T_or, ot.extent)
    print(name, "free-running GPU vs oracle:", r, t,
          "GPU vs truth:", PT.pose_errors(T_gpu, p["T_gt"], ot.extent))
    assert r < PT.ROT_TOL_DEG and t < PT.TRANS_TOL_REL, (r, t)


def test_register_is_deterministic(B):
    p, depth = _pair("corner_small")
    a = _gpu_run(B, p, depth, 10)[3]
    b = _gpu_run(B, p, depth, 10)[3]
    assert np.array_equal(a, b)


def test_gmm_tree_variant_lambda_zero(B):
    """lam_c = 0 at registration time is the paper's GMM-Tree Ln variant (no
    early stop, Sec. 5); it must match the oracle run with lambda_c = 0."""
    p, depth = _pair("corner_small")
    tree, Zt, Zs, T_gpu, _ = _gpu_run(B, p, depth, 10, lam_c=0.0)
    extent = tree.root()["extent"]
    ot = PT.tree_from_gpu(tree, PT.oracle_params(B.params(), depth), extent)
    T_or = O.register(ot, Zs, iters=10, lam_c=0.0)
    r, t = PT.pose_errors(T_gpu, T_or, extent)
    assert r < PT.ROT_TOL_DEG and t < PT.TRANS_TOL_REL, (r, t)
