"""The FP64 oracle against the hand-worked fixtures in tests/golden/ (no GPU).

Each fixture file states, in its header, the passage of the paper whose
definition it works through and how its values were obtained (by hand, as
exact fractions or values of elementary functions): none comes from the
oracle or from the CUDA path.
"""
import os

import numpy as np

from oracle import hgmm_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    assert rows, name
    return rows


def _rot_z(deg):
    c, s = np.cos(np.deg2rad(deg)), np.sin(np.deg2rad(deg))
    if deg == 90:
        c, s = 0.0, 1.0  # exact
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def test_complexity_fixture_sec4_1():
    """Sec. 4.1: Complexity of covariances with the fixture's eigenvalues
    (placed along a fixed rotation, so the oracle's eigen-decomposition is
    part of what is checked) and the stop decision at lambda_C = 0.01."""
    R = np.array([[0.36, 0.48, -0.8], [-0.8, 0.6, 0.0], [0.48, 0.64, 0.6]])  # orthonormal (3-4-5 entries)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-15)
    for l1, l2, l3, num, den, stop in _rows("complexity_sec4_1.txt"):
        lam_true = np.array([float(l1), float(l2), float(l3)])
        Sig = R @ np.diag(lam_true) @ R.T
        lam, _ = O.sym_eig(Sig[None])
        c = float(O.complexity(lam)[0])
        assert abs(c - float(num) / float(den)) < 1e-13, (l1, l2, l3, c)
        assert (c <= 0.01) == bool(int(stop)), (l1, l2, l3, c)


def test_posterior_fixture_eq3():
    """Eq. 3: two live unit-covariance children at (+-1, 0, 0) with equal
    weights give the logistic function of 2x; the six dead children get 0."""
    rows = _rows("posterior_eq3.txt")
    Z = np.array([[float(r[0]), float(r[1]), float(r[2])] for r in rows])
    pi = np.zeros(8)
    pi[:2] = 0.5
    mu = np.zeros((8, 3))
    mu[0, 0], mu[1, 0] = 1.0, -1.0
    Sigma = np.repeat(np.eye(3)[None], 8, axis=0)
    S = O.child_scores(Z, np.zeros(len(rows), dtype=np.int64), pi, mu, Sigma)
    g, _ = O.posteriors(S)
    for i, r in enumerate(rows):
        np.testing.assert_allclose(g[i, :2], [float(r[3]), float(r[4])], rtol=1e-14, atol=1e-16)
        assert np.all(g[i, 2:] == 0.0)


def test_objective_fixture_eq12():
    """Eq. 11 / Eq. 12 for one cluster, summed by hand for five poses."""
    mu = np.zeros((1, 3))
    mu_star = np.ones((1, 3))
    pi_star = np.array([0.5])
    lam = np.array([[4.0, 1.0, 0.25]])
    vec = np.eye(3)[None]  # column l = eigenvector n_l
    for ang, tx, ty, tz, val in _rows("objective_eq12.txt"):
        T = np.eye(4)
        T[:3, :3] = _rot_z(int(ang))
        T[:3, 3] = [float(tx), float(ty), float(tz)]
        assert abs(O.objective(T, mu_star, pi_star, mu, lam, vec) - float(val)) < 1e-14, (ang, tx, ty, tz)


def test_mstep_shift_fixture_eq16():
    """Eq. 13-16: a pure shift of every weighted mean is solved exactly
    (no rotation, the shift as the translation)."""
    rows = _rows("mstep_shift_eq16.txt")
    cl = [r for r in rows if r[0] == "c"]
    t0 = np.array([float(v) for v in next(r for r in rows if r[0] == "t")[1:]])
    mu = np.array([[float(v) for v in r[1:4]] for r in cl])
    lam = np.array([[float(v) for v in r[4:7]] for r in cl])
    pi_star = np.array([float(r[7]) for r in cl])
    vec = np.repeat(np.eye(3)[None], len(cl), axis=0)
    x = O.solve_increment(mu - t0, pi_star, mu, lam, vec)
    np.testing.assert_allclose(x[:3], 0.0, atol=1e-14)
    np.testing.assert_allclose(x[3:], t0, atol=1e-14)
