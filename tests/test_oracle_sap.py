"""Pins of the oracle's string-averaging projections (Sec. II-D, SAP) to
things other than itself: the projection onto one row's hyperplane (lambda =
1 satisfies the row exactly), Cimmino's simultaneous projection (every row a
string of its own) written as one sparse-matrix formula, and Fejer
monotonicity of the iterates towards any solution of a consistent system."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2108_12369_gb300 import workloads as W


def _small_system(orc, n=48, angles=12, ppa=40, noise=0.0):
    w = W.neo2_2d_spline(n_angles=angles, paths_per_angle=ppa, n=n, h=204.8 / n, noise_rel=noise)
    ref = orc.simulate(w["phantom"], w["angles"], w["paths_per_angle"], w["model"], w["seed"])
    return w, ref


def test_one_row_with_unit_relaxation_lands_on_its_hyperplane(orc):
    w, ref = _small_system(orc)
    rp, col, val = ref["row_ptr"], ref["col"], ref["val"]
    i = int(np.argmax(np.diff(rp)))
    r0, r1 = rp[i], rp[i + 1]
    rp1 = np.array([0, r1 - r0])
    rng = np.random.default_rng(3)
    x0 = rng.uniform(0.5, 1.5, n := 48 * 48)
    x = orc.sap(rp1, col[r0:r1], val[r0:r1], [5.0], n, 1, 1.0, 1, x0)
    a = np.zeros(n)
    np.add.at(a, col[r0:r1], val[r0:r1])
    assert abs(a @ x - 5.0) < 1e-12 * max(1.0, np.abs(a) @ np.abs(x))
    d = x - x0  # the move is along a
    assert np.allclose(d, (d @ a) / (a @ a) * a, rtol=0, atol=1e-12)
    # half relaxation goes half way
    xh = orc.sap(rp1, col[r0:r1], val[r0:r1], [5.0], n, 1, 0.5, 1, x0)
    assert abs(a @ xh - 0.5 * (5.0 + a @ x0)) < 1e-12 * max(1.0, np.abs(a) @ np.abs(x0))


def test_every_row_its_own_string_is_cimmino(orc):
    w, ref = _small_system(orc)
    rp, col, val, b = ref["row_ptr"], ref["col"], ref["val"], ref["b"]
    m, n = len(rp) - 1, 48 * 48
    A = sp.csr_matrix((val, col, rp), shape=(m, n))
    rng = np.random.default_rng(4)
    x0 = rng.uniform(0.0, 2.0, n)
    lam = 0.7
    nrm = np.asarray(A.multiply(A).sum(axis=1)).ravel()
    live = nrm > 0
    coef = np.zeros(m)
    coef[live] = lam * (b[live] - A[live] @ x0) / nrm[live]
    # strings of one row: the empty ones (rows missing the grid) leave x0
    want = x0 + (A.T @ coef) / m
    got = orc.sap(rp, col, val, b, n, m, lam, 1, x0)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("M,lam", [(1, 1.0), (7, 0.1), (40, 1.9)])
def test_iterates_approach_any_solution_of_a_consistent_system(orc, M, lam):
    """For b = A x_true and 0 < lambda < 2 every projection, hence every
    string sweep and their average, moves no farther from x_true."""
    w, ref = _small_system(orc)
    rp, col, val = ref["row_ptr"], ref["col"], ref["val"]
    n = 48 * 48
    A = sp.csr_matrix((val, col, rp), shape=(len(rp) - 1, n))
    x_true = ref["x_true"].astype(np.float64)
    b = A @ x_true
    x = np.zeros(n)
    dist = [np.linalg.norm(x - x_true)]
    res = [np.linalg.norm(A @ x - b)]
    for _ in range(6):
        x = orc.sap(rp, col, val, b, n, M, lam, 1, x)
        dist.append(np.linalg.norm(x - x_true))
        res.append(np.linalg.norm(A @ x - b))
    assert all(d1 <= d0 * (1 + 1e-12) for d0, d1 in zip(dist[:-1], dist[1:])), dist
    assert res[-1] < 0.5 * res[0]


def test_weights_pick_strings(orc):
    """All weight on string t gives that string's sweep alone: the same as a
    single string over its rows."""
    w, ref = _small_system(orc)
    rp, col, val, b = ref["row_ptr"], ref["col"], ref["val"], ref["b"]
    n, M, t = 48 * 48, 5, 3
    wts = np.zeros(M)
    wts[t] = 1.0
    got = orc.sap(rp, col, val, b, n, M, 0.3, 1, None, weights=wts)
    rows = np.arange(t, len(rp) - 1, M)
    A = sp.csr_matrix((val, col, rp), shape=(len(rp) - 1, n))[rows]
    want = orc.sap(A.indptr, A.indices, A.data, b[rows], n, 1, 0.3, 1, None)
    assert np.array_equal(got, want)
