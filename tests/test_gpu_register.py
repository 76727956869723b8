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


@pytest.mark.parametrize("name", ["lidar", "corner_small", "depth"])
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


# ---- configs as stated: corner scene at <= 30 deg / t <= 0.1 (10k points,
# depth 3), and the structured-light depth pair (~276k points, depth 4)
def _per_round(B, p, depth, iters=30, rounds=None):
    tree, Zt, Zs, T_gpu, hist = _gpu_run(B, p, depth, iters)
    extent = tree.root()["extent"]
    ot = PT.tree_from_gpu(tree, PT.oracle_params(B.params(), depth), extent)
    errs = PT.per_round_teacher_forced(ot, Zs, hist, extent, rounds)
    return tree, Zt, Zs, T_gpu, errs, extent


@pytest.mark.parametrize("seed", range(10))
def test_corner_30deg_per_round_teacher_forced(B, seed):
    """Every one of 30 rounds, started from the GPU's own previous pose on the
    GPU's tree, matches one oracle round (Algorithm 1 + Eq. 9-16) within
    0.01 deg / 1e-4 extent, whether or not the trajectory converges."""
    p = synth.corner_pair(seed)
    _, _, _, T_gpu, errs, extent = _per_round(B, p, 3)
    worst_r = max(e[1] for e in errs)
    worst_t = max(e[2] for e in errs)
    print(f"corner seed {seed}: worst per-round {worst_r:.2e} deg / {worst_t:.2e};"
          f" GPU vs truth {PT.pose_errors(T_gpu, p['T_gt'], extent)}")
    assert worst_r < PT.ROT_TOL_DEG and worst_t < PT.TRANS_TOL_REL, errs


def test_corner_30deg_free_running_where_well_conditioned(B):
    """Free-running (oracle build + register against GPU build + register)
    on the seeds 0..9 of the 30-degree corner configuration whose trajectory
    is determined to FP32 precision: the oracle run on the input perturbed
    by 1e-7 relative (about FP32 rounding) ends within a quarter of the
    tolerance of the unperturbed oracle run.  On this scene the method as
    read does not reach the ground truth from these poses (its fixed point
    moves even with source = target), and most trajectories amplify a 1e-7
    perturbation to 0.01-0.3 deg over 30 rounds; those seeds are compared
    round by round by the teacher-forced test instead."""
    prm_o = PT.oracle_params(B.params(), 3)
    compared = 0
    for seed in range(10):
        p = synth.corner_pair(seed)
        tree, Zt, Zs, T_gpu, _ = _gpu_run(B, p, 3, 30)
        ot = O.build_tree(Zt, prm_o)
        T_or = O.register(ot, Zs, iters=30)
        rng = np.random.default_rng(seed)
        Ztp = Zt * (1.0 + PT.COND_PERTURB * rng.standard_normal(Zt.shape))
        Zsp = Zs * (1.0 + PT.COND_PERTURB * rng.standard_normal(Zs.shape))
        T_p = O.register(O.build_tree(Ztp, prm_o), Zsp, iters=30)
        cr, ct = PT.pose_errors(T_or, T_p, ot.extent)
        r, t = PT.pose_errors(T_gpu, T_or, ot.extent)
        print(f"corner seed {seed}: oracle response to 1e-7 input perturbation {cr:.1e} deg / {ct:.1e}; "
              f"GPU vs oracle {r:.1e} deg / {t:.1e}")
        if cr > PT.ROT_TOL_DEG / 4 or ct > PT.TRANS_TOL_REL / 4:
            continue
        compared += 1
        assert r < PT.ROT_TOL_DEG and t < PT.TRANS_TOL_REL, (seed, r, t)
    assert compared >= 1


def test_depth_pair_per_round_teacher_forced(B):
    """Config-3 structured-light pair (depth 4, ~276k points): every round of
    30 against one oracle round from the GPU's previous pose."""
    p = synth.depth_pair(0)
    _, _, _, T_gpu, errs, extent = _per_round(B, p, 4)
    worst_r = max(e[1] for e in errs)
    worst_t = max(e[2] for e in errs)
    print(f"depth pair: worst per-round {worst_r:.2e} deg / {worst_t:.2e};"
          f" GPU vs truth {PT.pose_errors(T_gpu, p['T_gt'], extent)}")
    assert worst_r < PT.ROT_TOL_DEG and worst_t < PT.TRANS_TOL_REL, errs


def test_depth_pair_free_running(B):
    """Config-3 pair free-running: oracle build + register against GPU build +
    register (final pose)."""
    p = synth.depth_pair(0)
    tree, Zt, Zs, T_gpu, _ = _gpu_run(B, p, 4, 30)
    prm_o = PT.oracle_params(B.params(), 4)
    ot = O.build_tree(Zt, prm_o)
    T_or = O.register(ot, Zs, iters=30)
    r, t = PT.pose_errors(T_gpu, T_or, ot.extent)
    print("depth pair free-running GPU vs oracle:", r, t, "oracle vs truth:",
          PT.pose_errors(T_or, p["T_gt"], ot.extent))
    assert r < PT.ROT_TOL_DEG and t < PT.TRANS_TOL_REL, (r, t)


def test_registration_does_not_depend_on_the_order_of_the_source_points(B):
    """Every point's moments become 64-bit fixed-point integers before they
    are summed (per warp, per CTA, per node), so the registration is the same
    bit for bit whatever the order of the source points: the LiDAR source in
    its scan order and in two random orders, 30 rounds."""
    import torch
    p = synth.lidar_pair(0)
    tgt, _ = PT.device_cloud(p["tgt"])
    src4 = synth.to_float4(p["src"])
    tree = B.Tree(max(tgt.shape[0], src4.shape[0]), 4)
    tree.build(tgt, 4)
    rng = np.random.default_rng(7)
    outs = []
    for perm in (np.arange(src4.shape[0]), rng.permutation(src4.shape[0]), rng.permutation(src4.shape[0])):
        src = torch.from_numpy(np.ascontiguousarray(src4[perm])).cuda()
        hist = torch.zeros((30, 4, 4), dtype=torch.float64, device="cuda")
        tree.register(src, iters=30, T_hist=hist)
        tree.sync()
        outs.append(hist.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


@pytest.mark.parametrize("n", [1_200_000, 2_200_000])
def test_large_unordered_source_is_reordered_without_changing_the_result(B, n):
    """A source of at least 2^20 points runs its first round in the given
    order, recording each point's node, and is then counting-sorted by that
    node for the remaining rounds (from 2^21 points with three registration
    CTAs per SM instead of two).  The node moments are exact integer sums
    of the points' fixed-point moments, so the order of the source points
    does not change the pose: the same cloud in two random orders gives the
    same 3 rounds bit for bit; the first round matches one oracle round on
    the GPU's tree, and so does the second (after the reorder) from the GPU's
    pose after the first."""
    import torch
    rng = np.random.default_rng(5)
    p = synth.primitive_pair(17, n, max_deg=3.0, max_t=0.02)
    tgt, Zt = PT.device_cloud(p["tgt"])
    src4 = synth.to_float4(p["src"])
    tree = B.Tree(src4.shape[0], 4)
    tree.build(tgt, 4)
    outs = []
    for perm in (rng.permutation(src4.shape[0]), rng.permutation(src4.shape[0])):
        src = torch.from_numpy(np.ascontiguousarray(src4[perm])).cuda()
        hist = torch.zeros((3, 4, 4), dtype=torch.float64, device="cuda")
        tree.register(src, iters=3, T_hist=hist)
        tree.sync()
        outs.append(hist.cpu().numpy())
    extent = tree.root()["extent"]
    assert np.array_equal(outs[0], outs[1])
    ot = PT.tree_from_gpu(tree, PT.oracle_params(B.params(), 4), extent)
    Zs = src4[:, :3].astype(np.float64)
    T_o = O.register(ot, Zs, iters=1)
    r, t = PT.pose_errors(outs[0][0], T_o, extent)
    assert r < PT.ROT_TOL_DEG and t < PT.TRANS_TOL_REL, (r, t)
    T_o2 = O.register(ot, Zs, T_init=outs[0][0], iters=1)
    r, t = PT.pose_errors(outs[0][1], T_o2, extent)
    assert r < PT.ROT_TOL_DEG and t < PT.TRANS_TOL_REL, (r, t)
