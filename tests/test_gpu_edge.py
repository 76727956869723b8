"""Edge cases and error behaviour of the C ABI on the GPU: smallest clouds,
deep sparse trees, degenerate geometry, non-finite input, invalid arguments,
capacity limits, the host-buffer entry point."""
import numpy as np
import pytest

from paper_1807_02587_gb300 import synth
from tests import parity as PT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1807_02587_gb300 import binding
    return binding


def _consistent(tree, n, depth):
    for l in range(depth):
        g = tree.export(l)
        lab = tree.labels(l)
        assert lab.min() >= 0 and lab.max() < 8 ** (l + 1)
        assert np.array_equal(np.bincount(lab, minlength=8 ** (l + 1)), g["count"])
        assert g["count"].sum() == n
        # a dead node holds points only as child 0 of a parent without live
        # children (a leaf parent's points are carried down there)
        split = g["live"].reshape(-1, 8).any(axis=1)
        carrier = np.zeros(g["live"].shape[0], bool)
        carrier[0::8] = ~split
        assert np.all(g["count"][~g["live"] & ~carrier] == 0)
        assert np.all(np.isfinite(g["mu"][g["live"]]))
        assert np.all(np.isfinite(g["Sigma"][g["live"]]))
        if l:
            assert np.array_equal(lab // 8, tree.labels(l - 1))


@pytest.mark.parametrize("n,depth", [(8, 1), (8, 3), (9, 2), (300, 5), (30001, 5)])
def test_small_and_deep_trees(B, n, depth):
    P = synth.corner_scene(synth.make_rng(n), n)
    dev, Z = PT.device_cloud(P)
    tree = B.Tree(n, depth)
    tree.build(dev, depth)
    tree.sync()
    _consistent(tree, n, depth)
    if n >= 300:
        res = PT.check_build(tree, Z, PT.oracle_params(B.params(), depth))
        for r in res["levels"]:
            assert r["live_mismatch"] == 0 and r["mu"] < PT.MEAN_TOL and r["S"] < PT.COV_TOL, r
            assert r["excluded_parents"] <= max(2, 0.02 * r["parents_with_points"]), r


def test_coincident_points(B):
    import torch
    P = np.tile(np.array([[1.0, 2.0, 3.0]]), (1000, 1))
    dev, Z = PT.device_cloud(P)
    tree = B.Tree(1000, 3)
    tree.build(dev, 3)
    tree.sync()
    _consistent(tree, 1000, 3)
    T = tree.register(dev, iters=3)
    try:
        tree.sync()
    except B.HgmmError as e:
        assert e.code == B.HGMM_EDEGENERATE
    assert np.all(np.isfinite(T.cpu().numpy()))


def test_nonfinite_input_is_reported(B):
    P = synth.corner_scene(synth.make_rng(1), 2000)
    P[123, 1] = np.nan
    dev, _ = PT.device_cloud(P)
    tree = B.Tree(2000, 2)
    tree.build(dev, 2)
    with pytest.raises(B.HgmmError) as ei:
        tree.sync()
    assert ei.value.code == B.HGMM_ENONFINITE
    # the tree stays usable
    P[123, 1] = 0.5
    dev, _ = PT.device_cloud(P)
    tree.build(dev, 2)
    tree.sync()


def test_invalid_arguments(B):
    import torch
    P = synth.corner_scene(synth.make_rng(2), 1000)
    dev, _ = PT.device_cloud(P)
    tree = B.Tree(1000, 3)
    with pytest.raises(B.HgmmError) as e:
        B.hgmm_build(tree.handle, dev, 3, J=7)
    assert e.value.code == B.HGMM_EINVAL
    for d in (0, 6):
        with pytest.raises(B.HgmmError):
            B.hgmm_build(tree.handle, dev, d)
    with pytest.raises(B.HgmmError) as e:
        B.hgmm_build(tree.handle, dev, 4)  # deeper than the tree was created for
    assert e.value.code == B.HGMM_ECAPACITY
    big = torch.zeros((1001, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(B.HgmmError) as e:
        B.hgmm_build(tree.handle, big, 2)
    assert e.value.code == B.HGMM_ECAPACITY
    flat = torch.zeros(4 * 100 + 1, dtype=torch.float32, device="cuda")
    mis = flat[1:].view(100, 4)
    with pytest.raises(B.HgmmError) as e:
        B.hgmm_build(tree.handle, mis, 2)
    assert e.value.code == B.HGMM_EINVAL
    tiny = torch.zeros((7, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(B.HgmmError) as e:
        B.hgmm_build(tree.handle, tiny, 1)
    assert e.value.code == B.HGMM_EINVAL


def test_host_entry_point_matches_device_path(B):
    """The host-buffer entry point captures the build and the registration
    of a shape into a CUDA graph on its first call and replays it later: the
    first call, a replay, a call of another shape (a new capture) and the
    first shape again all give the device path's bits."""
    import torch
    p = synth.corner_pair(11, n=6000, max_deg=3.0, max_t=0.02)
    q = synth.corner_pair(12, n=5000, max_deg=3.0, max_t=0.02)
    tree = B.Tree(6000, 3)

    def host(pair):
        return B.hgmm_register_pair_host(tree.handle, synth.to_float4(pair["tgt"]),
                                         synth.to_float4(pair["src"]), 3, B.params(), None, 12)

    outs = [host(p), host(p), host(q), host(p)]

    def device(pair):
        tgt, _ = PT.device_cloud(pair["tgt"])
        src, _ = PT.device_cloud(pair["src"])
        tree.build(tgt, 3)
        T = tree.register(src, iters=12).cpu().numpy()
        tree.sync()
        return T

    T_p, T_q = device(p), device(q)
    for k in (0, 1, 3):
        assert np.array_equal(outs[k], T_p), k
    assert np.array_equal(outs[2], T_q)
    assert not np.array_equal(T_p, T_q)


def test_bounded_wait_times_out_without_fault(B):
    """Failure detection on the GPU: a grid-barrier wait that nothing ends
    gives up after its spin limit, records HGMM_ETIMEOUT and returns; the
    context and the tree stay usable."""
    tree = B.Tree(2000, 2)
    B.hgmm_debug_barrier_timeout(tree.handle, 20000)
    with pytest.raises(B.HgmmError) as e:
        tree.sync()
    assert e.value.code == B.HGMM_ETIMEOUT
    P = synth.corner_scene(synth.make_rng(3), 2000)
    dev, _ = PT.device_cloud(P)
    tree.build(dev, 2)
    tree.register(dev, iters=2)
    tree.sync()


def test_large_parent_handoff_in_slices(B):
    """A level-0 parent of ~2,100 items: its hand-off scan runs in two slices
    on parallel CTAs; the partition stays consistent (every point once, in
    its chosen child's segment) and level 1, built from those segments,
    matches the oracle."""
    n = 530_001
    P = synth.primitive_pair(5, n)["tgt"]
    dev, Z = PT.device_cloud(P)
    tree = B.Tree(n, 2)
    tree.build(dev, 2)
    tree.sync()
    _consistent(tree, n, 2)
    res = PT.check_build(tree, Z, PT.oracle_params(B.params(), 2), conditioning=False)
    for r in res["levels"]:
        assert r["count_mismatch"] == 0 and r["live_mismatch"] == 0, r
        assert r["mu"] < PT.MEAN_TOL and r["S"] < PT.COV_TOL, r
        assert r["label_disagree_not_tie"] == 0, r
