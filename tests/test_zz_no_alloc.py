"""The allocation-free level-0 fit (hgmm_fit_level0_noalloc) against the
regular build of a depth-1 tree (hgmm_build + hgmm_tree_export).

Callers that cannot allocate device memory (another component capturing a
CUDA graph on their stream, fixed-budget real-time loops, plug-ins whose host
owns all allocations) use the variant whose scratch is a static device
array.  Three calls in a row (30k, 93k, then 2k points) check that the
shared array's leftover contents from a larger call do not leak into a
smaller one, for both moment-sum precisions.  This file is named to be
collected last.
"""
import numpy as np
import pytest

from paper_1807_02587_gb300 import synth
from tests import parity as PT

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_level0_matches_regular_build(precision):
    import torch
    from paper_1807_02587_gb300 import binding as B
    prm = B.params(precision=precision)
    clouds = [synth.corner_scene(synth.make_rng(21), 30001),
              synth.lidar_pair(1)["tgt"],
              synth.corner_scene(synth.make_rng(22), 2000)]
    out = torch.zeros(129, dtype=torch.float64, device="cuda")
    for P in clouds:  # calls in a row: larger, then smaller clouds
        dev, _ = PT.device_cloud(P)
        out.fill_(np.nan)
        B.hgmm_fit_level0_noalloc(dev, prm, out=out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got[128] == 0.0
        tree = B.Tree(dev.shape[0], 1)
        tree.build(dev, 1, prm)
        tree.sync()
        ref = B.hgmm_tree_export(tree.handle, 0, 8)
        g = got[:128].reshape(8, 16)
        assert np.array_equal(g[:, 10], ref[:, 10])  # live flags
        live = ref[:, 10] > 0.5
        assert live.any()
        scale = np.maximum(np.linalg.norm(ref[live, 1:4], axis=1), 1e-6)
        assert np.all(np.linalg.norm(g[live, 1:4] - ref[live, 1:4], axis=1) / scale < PT.MEAN_TOL)
        nS = np.linalg.norm(ref[live, 4:10], axis=1)
        assert np.all(np.linalg.norm(g[live, 4:10] - ref[live, 4:10], axis=1) / nS < PT.COV_TOL)
        assert np.all(np.abs(g[live, 0] - ref[live, 0]) < PT.PI_TOL)
        assert np.allclose(g[live, 12:16], ref[live, 12:16], rtol=1e-4, atol=1e-12)
        assert np.all(g[:, 11] == -1.0)


def test_noalloc_reports_nonfinite_input():
    import torch
    from paper_1807_02587_gb300 import binding as B
    P = synth.corner_scene(synth.make_rng(23), 5000)
    P[17, 1] = np.inf
    dev, _ = PT.device_cloud(P)
    out = torch.zeros(129, dtype=torch.float64, device="cuda")
    B.hgmm_fit_level0_noalloc(dev, out=out)
    torch.cuda.synchronize()
    assert out[128].item() == B.HGMM_ENONFINITE
    # the next call on clean input is not affected by the previous status
    dev2, _ = PT.device_cloud(synth.corner_scene(synth.make_rng(24), 5000))
    B.hgmm_fit_level0_noalloc(dev2, out=out)
    torch.cuda.synchronize()
    assert out[128].item() == 0.0


def test_noalloc_rejects_too_many_points():
    import torch
    from paper_1807_02587_gb300 import binding as B
    big = torch.zeros(((1 << 20) + 1, 4), dtype=torch.float32, device="cuda")
    out = torch.zeros(129, dtype=torch.float64, device="cuda")
    with pytest.raises(B.HgmmError) as e:
        B.hgmm_fit_level0_noalloc(big, out=out)
    assert e.value.code == B.HGMM_ECAPACITY
