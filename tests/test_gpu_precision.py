"""Precision form: FP32 E-step with compensated (TwoSum) moment sums against
plain FP32 sums, each measured against the FP64 oracle level by level on the
structured-light depth pair (~276k points, depth 4).

One EM iteration at a time (teacher forced, so the comparison isolates the
arithmetic of that iteration): the oracle runs the iteration from the GPU's
own previous parameters.  The printed table is the per-level error report.
"""
import numpy as np
import pytest

from paper_1807_02587_gb300 import synth
from tests import parity as PT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1807_02587_gb300 import binding
    return binding


def test_compensated_vs_plain_per_level(B):
    p = synth.depth_pair(0)
    dev, Z = PT.device_cloud(p["tgt"])
    steps = [(l, k) for l in range(4) for k in (1, 8)]
    rows = {}
    for name, prec in (("compensated", 0), ("plain", 1)):
        res = PT.check_em_steps(B, dev, Z, 4, steps, B.params(precision=prec))
        rows[name] = res
    print("\nlevel iter | compensated mu / Sigma / pi | plain mu / Sigma / pi")
    for a, b in zip(rows["compensated"], rows["plain"]):
        print(f"{a['level']:5d} {a['iter']:4d} | {a['mu']:.2e} {a['S']:.2e} {a['pi']:.2e} | "
              f"{b['mu']:.2e} {b['S']:.2e} {b['pi']:.2e}")
    for r in rows["compensated"]:
        assert r["live_mismatch"] == 0, r
        assert r["mu"] < PT.MEAN_TOL and r["S"] < PT.COV_TOL and r["pi"] < PT.PI_TOL, r
    for r in rows["plain"]:
        assert r["mu"] < 1e-3 and r["S"] < 1e-3, r
    # the compensated sums are never worse than the plain ones at level 0,
    # where a single parent sums every point
    l0c = [r for r in rows["compensated"] if r["level"] == 0]
    l0p = [r for r in rows["plain"] if r["level"] == 0]
    assert max(r["S"] for r in l0c) <= 1.5 * max(r["S"] for r in l0p) + 1e-9
