"""Flat "GMM J=n" variant (Sec. 5, variant 3) on the GPU vs the FP64 oracle.

* components made from the GPU's own tree: the same nodes (exact), weights
  and parameters;
* flat EM, one iteration at a time from the GPU's previous parameters;
* registration: per-component moments of the first round, the Eq. 11
  objective, and 30 rounds against the oracle on the GPU's own components;
* the bench's LiDAR workload (93k points, depth 4, ~3000 components): the
  first round's moments and pose;
* edge cases: a ragged cloud, a one-point source (singular normal
  equations), non-finite input and the capacity checks.
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


def _setup(B, p, depth, em_iters=0, level=-1):
    tgt, Zt = PT.device_cloud(p["tgt"])
    src, Zs = PT.device_cloud(p["src"])
    n = max(Zt.shape[0], Zs.shape[0])
    tree = B.Tree(n, depth)
    tree.build(tgt, depth)
    flat = B.Flat(n, int(B.hgmm_node_count(depth)))
    flat.from_tree(tree, level)
    if em_iters:
        flat.fit(tgt, em_iters)
    flat.sync()
    return tree, flat, tgt, Zt, src, Zs


def _oracle_flat(flat, eps):
    e = flat.export()
    return O.Flat(pi=e["pi"], mu=e["mu"], Sigma=e["Sigma"], node=e["node"], eps=eps)


def _small():
    return synth.corner_pair(7, max_deg=3.0, max_t=0.02)


@pytest.mark.parametrize("depth,level", [(3, -1), (3, 1), (4, -1)])
def test_components_from_gpu_tree_match_oracle(B, depth, level):
    p = _small()
    tree, flat, *_ = _setup(B, p, depth, level=level)
    ot = PT.tree_from_gpu(tree, PT.oracle_params(B.params(), depth), tree.root()["extent"])
    of = O.flat_from_tree(ot, None if level < 0 else level)
    g = flat.export()
    assert g["J"] == of.pi.shape[0]
    np.testing.assert_array_equal(g["node"], of.node)
    np.testing.assert_allclose(g["pi"], of.pi, rtol=1e-12)
    np.testing.assert_array_equal(g["mu"], of.mu)
    np.testing.assert_array_equal(g["Sigma"], of.Sigma)


@pytest.mark.parametrize("depth", [2, 3])
def test_flat_em_steps_match_oracle(B, depth):
    """Teacher forcing: the oracle runs one EM iteration from the GPU's
    parameters after k-1 iterations and is compared with the GPU's k-th."""
    p = _small()
    tgt, Zt = PT.device_cloud(p["tgt"])
    n = Zt.shape[0]
    tree = B.Tree(n, depth)
    tree.build(tgt, depth)
    eps = tree.root()["eps"]
    prev = None
    for k in range(0, 4):
        flat = B.Flat(n, int(B.hgmm_node_count(depth)))
        flat.from_tree(tree)
        flat.fit(tgt, k)
        flat.sync()
        cur = _oracle_flat(flat, eps)
        if prev is not None:
            want, _ = O.flat_em(Zt, prev, 1, n_min=8.0)
            live = want.pi > 0
            assert np.array_equal(live, cur.pi > 0), k
            scale = np.maximum(np.linalg.norm(want.mu[live], axis=1),
                               np.sqrt(np.trace(want.Sigma[live], axis1=1, axis2=2)))
            e_mu = np.linalg.norm(cur.mu[live] - want.mu[live], axis=1) / scale
            e_S = (np.linalg.norm(cur.Sigma[live] - want.Sigma[live], axis=(1, 2))
                   / np.linalg.norm(want.Sigma[live], axis=(1, 2)))
            e_pi = np.abs(cur.pi[live] - want.pi[live])
            print(depth, k, "J", live.sum(), "mu", e_mu.max(), "S", e_S.max(), "pi", e_pi.max())
            assert e_mu.max() < PT.MEAN_TOL and e_S.max() < PT.COV_TOL and e_pi.max() < PT.PI_TOL
        prev = cur


def _first_round_check(B, flat, Zs, T0, extent, eps):
    import torch
    of = _oracle_flat(flat, eps)
    T_init = torch.from_numpy(T0.reshape(16).copy()).cuda()
    T1 = flat.register(PT.device_cloud(Zs)[0], T_init=T_init, iters=1).cpu().numpy()
    obj = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.hgmm_flat_objective(flat.handle, obj)
    flat.sync()
    g = flat.moments()
    Zp = Zs @ T0[:3, :3].T + T0[:3, 3]
    M0, M1 = O.flat_moments(of, Zp)
    N = Zs.shape[0]
    assert abs(g[:, 0].sum() - M0.sum()) < 1e-5 * N
    big = M0 > 1.0
    rel0 = np.abs(g[big, 0] - M0[big]) / M0[big]
    mstar_o = M1[big] / M0[big, None]
    mstar_g = g[big, 1:] / g[big, :1]
    err = np.linalg.norm(mstar_o - mstar_g, axis=1) / extent
    T_o, h = O.register_flat(of, Zs, T_init=T0, iters=1, history=True)
    r, t = PT.pose_errors(T1, T_o, extent)
    print("J", of.pi.size, "M0 rel max", rel0.max(), "mu* max", err.max(), "pose", r, t,
          "objective", obj.item(), h[0]["objective"])
    assert rel0.max() < 1e-4 and err.max() < 1e-5
    assert r < 1e-4 and t < 1e-5
    assert obj.item() == pytest.approx(h[0]["objective"], rel=1e-4)


def test_first_round_matches_oracle(B):
    p = _small()
    tree, flat, tgt, Zt, src, Zs = _setup(B, p, 3, em_iters=2)
    rng = np.random.default_rng(1)
    T0 = synth.rigid(synth.random_rotation(rng, 2.0), rng.uniform(-0.01, 0.01, 3))
    _first_round_check(B, flat, Zs, T0, tree.root()["extent"], tree.root()["eps"])


def test_first_round_on_lidar_workload(B):
    """The bench's workload: 93k-point LiDAR scans, depth 4 (~3000
    components), one round from the identity."""
    p = synth.lidar_pair(0)
    tree, flat, tgt, Zt, src, Zs = _setup(B, p, 4)
    _first_round_check(B, flat, Zs, np.eye(4), tree.root()["extent"], tree.root()["eps"])


@pytest.mark.parametrize("em_iters", [0, 2])
def test_registration_matches_oracle(B, em_iters):
    import torch
    p = _small()
    tree, flat, tgt, Zt, src, Zs = _setup(B, p, 3, em_iters=em_iters)
    extent = tree.root()["extent"]
    of = _oracle_flat(flat, tree.root()["eps"])
    hist = torch.zeros((30, 4, 4), dtype=torch.float64, device="cuda")
    T = flat.register(src, iters=30, T_hist=hist).cpu().numpy()
    flat.sync()
    T_o, h = O.register_flat(of, Zs, iters=30, history=True)
    hist = hist.cpu().numpy()
    errs = [PT.pose_errors(hist[k], h[k + 1]["T_start"] if k + 1 < 30 else T_o, extent) for k in range(30)]
    print("per round (deg, rel t):", [(f"{a:.1e}", f"{b:.1e}") for a, b in errs[::5]])
    r, t = PT.pose_errors(T, T_o, extent)
    assert r < PT.ROT_TOL_DEG and t < PT.TRANS_TOL_REL, (r, t)
    print("GPU vs truth", PT.pose_errors(T, p["T_gt"], extent))


def test_registration_is_deterministic(B):
    p = _small()
    out = []
    for _ in range(2):
        tree, flat, tgt, Zt, src, Zs = _setup(B, p, 3, em_iters=1)
        out.append(flat.register(src, iters=8).cpu().numpy())
        flat.sync()
    assert np.array_equal(out[0], out[1])


def test_edge_cases(B):
    import torch
    p = _small()
    tree, flat, tgt, Zt, src, Zs = _setup(B, p, 3)
    # a one-point source: rank-deficient normal equations (rank 3 up to
    # rounding); either the pivot check reports them or T stays finite
    one = src[:1].contiguous()
    T = flat.register(one, iters=2).cpu().numpy()
    try:
        flat.sync()
    except B.HgmmError as e:
        assert e.code == B.HGMM_EDEGENERATE
    assert np.isfinite(T).all()
    # a ragged source of 1001 points still registers
    T = flat.register(src[:1001].contiguous(), iters=3).cpu().numpy()
    flat.sync()
    assert np.isfinite(T).all()
    # non-finite input is reported
    bad = src[:2000].clone()
    bad[7, 1] = float("nan")
    flat.register(bad, iters=1)
    with pytest.raises(B.HgmmError) as e:
        flat.sync()
    assert e.value.code == B.HGMM_ENONFINITE
    # capacity and argument checks
    big = torch.zeros((Zt.shape[0] + 10, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(B.HgmmError) as e:
        flat.register(big, iters=1)
    assert e.value.code == B.HGMM_ECAPACITY
    small = B.Flat(1000, 64)
    with pytest.raises(B.HgmmError) as e:
        small.from_tree(tree)  # 584 candidate nodes at depth 3
    assert e.value.code == B.HGMM_ECAPACITY
    with pytest.raises(B.HgmmError) as e:
        flat.from_tree(tree, level=3)
    assert e.value.code == B.HGMM_EINVAL
    fresh = B.Flat(1000, 64)
    with pytest.raises(B.HgmmError) as e:
        fresh.register(src[:100].contiguous(), iters=1)
    assert e.value.code == B.HGMM_EINVAL
