"""Pins of the oracle's smoothed subproblems (feature table, read as the
soft-min -a log sum_x exp(-<lambda,x>/a)): brute-force enumeration of each
subproblem's feasible set, the limit a -> 0 (within a log|X_j| of E^j),
marginals in [0, 1] that are the gradient (central differences)."""
import numpy as np
import pytest

import oracle
import workloads
from tests import brute


def _rows_problem(seed, n=16, rows=10, kmax=8):
    good = []
    for r in workloads.random_rows(6 * rows, kmax=kmax, n=n, seed=seed):
        try:
            oracle.Oracle(workloads.single_rows_problem([r], n, np.zeros(n)))
            good.append(r)
        except oracle.OracleError:
            pass
        if len(good) == rows:
            break
    return workloads.single_rows_problem(good, n, np.zeros(n)), good


@pytest.mark.parametrize("a", [0.3, 1.0, 10.0, 100.0])
def test_smoothed_vs_enumeration(a):
    prob, rows = _rows_problem(5)
    P = oracle.Oracle(prob)
    rng = np.random.default_rng(1)
    lam = rng.normal(size=P.num_slots) * 3
    E, mg = P.smoothed(lam, a)
    for j, (v, coef, sense, rhs) in enumerate(rows):
        sl = slice(P.row_ptr[j], P.row_ptr[j + 1])
        X = brute.row_feasible(coef, sense, rhs).astype(np.float64)
        z = -(X @ lam[sl]) / a
        mz = z.max()
        logZ = mz + np.log(np.exp(z - mz).sum())
        assert abs(E[j] - (-a * logZ)) < 1e-9 * max(1.0, abs(E[j]))
        p = np.exp(z - logZ)
        np.testing.assert_allclose(mg[sl], p @ X, atol=1e-12)


def test_smoothed_limit_and_gradient():
    prob, rows = _rows_problem(7)
    P = oracle.Oracle(prob)
    rng = np.random.default_rng(2)
    lam = rng.normal(size=P.num_slots)
    _, Emin = P.lower_bound(lam, np.zeros(P.num_slots), energies=True)
    for a in (1e-3, 1e-2):
        E, mg = P.smoothed(lam, a)
        for j, (v, coef, sense, rhs) in enumerate(rows):
            nX = len(brute.row_feasible(coef, sense, rhs))
            assert Emin[j] - a * np.log(nX) - 1e-12 <= E[j] <= Emin[j] + 1e-12
        assert np.all(mg >= 0) and np.all(mg <= 1 + 1e-12)
    a = 2.0
    E, mg = P.smoothed(lam, a)
    h = 1e-6
    for q in rng.choice(P.num_slots, size=20, replace=False):
        e = np.zeros(P.num_slots)
        e[q] = h
        fd = (P.smoothed(lam + e, a)[0].sum() - P.smoothed(lam - e, a)[0].sum()) / (2 * h)
        assert abs(fd - mg[q]) < 1e-7
