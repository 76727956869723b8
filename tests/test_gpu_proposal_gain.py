"""What the trained proposal gains over the method without it, on held-out
pairs whose rotations are uniform over SO(3), refined by the plain method at
depth 4 (success = final rotation within 0.1 deg):

* the shipped network (trained by ``train_proposal`` on 100k pairs that the
  plain method generated and labelled) against the plain method from the
  identity and against the frame alignment alone (the untrained network);
* a network trained here from scratch on the GPU (8000 labelled pairs)
  against the same two baselines.

The held-out pairs come from seeds that training does not use."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

W3_BIAS = 396032  # index of b3 in the flat parameter vector


def _frame_only(B, P, seed):
    base = B.Mlp(256)
    B.hgmm_mlp_set_params(base.handle, P.init_params(seed) * (np.arange(B.HGMM_MLP_PARAMS) >= W3_BIAS))
    return base


def test_shipped_proposal_gain():
    from paper_1807_02587_gb300 import binding as B
    from paper_1807_02587_gb300 import proposal as P
    path = os.path.join(os.path.dirname(P.__file__), "weights", "proposal_mlp.npz")
    net = B.Mlp(256)
    B.hgmm_mlp_set_params(net.handle, np.load(path)["params"])
    test = P.so3_test_pairs(4242, 128, 30000)
    res = P.evaluate(net, test, depth=4, iters=30, reps=1)
    print("shipped", res)
    res0 = P.evaluate(_frame_only(B, P, 0), test, depth=4, iters=30, reps=1)
    print("frame alignment only", res0)
    assert res["learned_success_le_0p1deg"] >= 0.85
    assert res["learned_success_le_0p1deg"] >= res["plain_success_le_0p1deg"] + 0.6
    assert res["learned_success_le_0p1deg"] >= res0["learned_success_le_0p1deg"] + 0.4


def test_training_from_scratch_gains():
    import torch
    from paper_1807_02587_gb300 import binding as B
    from paper_1807_02587_gb300 import proposal as P
    Xs, Ls, Ks = [], [], []
    for c in range(4):
        train = P.scene_pairs(500 + c, 250, 8, 8000)
        X, L, keep, st = P.label_pairs(train, depth=3, iters=30)
        print("labels", st)
        assert st["label_within_tol"] > 0.8
        Xs.append(X), Ls.append(L), Ks.append(keep)
        del train
    net = B.Mlp(512)
    B.hgmm_mlp_set_params(net.handle, P.init_params(1))
    P.train(net, torch.cat(Xs), torch.cat(Ls), np.concatenate(Ks), epochs=60, batch=512, lr=1e-3, seed=1)
    test = P.so3_test_pairs(600, 96, 20000)
    res = P.evaluate(net, test, depth=4, iters=30, reps=1)
    print("trained here", res)
    res0 = P.evaluate(_frame_only(B, P, 1), test, depth=4, iters=30, reps=1)
    print("frame alignment only", res0)
    assert res["learned_success_le_0p1deg"] >= res["plain_success_le_0p1deg"] + 0.3
    assert res["learned_success_le_0p1deg"] >= res0["learned_success_le_0p1deg"] + 0.15
    assert res["proposal_median_err_deg"] < 0.5 * res0["proposal_median_err_deg"]
