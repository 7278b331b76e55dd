"""Pins of the oracle's min-marginals (Alg. 1 line "min-marginal difference",
computed through the shortest-path formula of App. B) against brute-force
enumeration of each subproblem and against closed forms."""
import numpy as np
import pytest

import oracle
import workloads
from tests import brute


@pytest.mark.parametrize("seed", [11, 12])
def test_min_marginals_vs_enumeration(seed):
    rng = np.random.default_rng(seed)
    checked = 0
    for (v, a, sense, b) in workloads.random_rows(80, kmax=12, seed=seed):
        k = len(v)
        prob = workloads.single_rows_problem([(np.arange(k), a, sense, b)], k, np.zeros(k))
        try:
            P = oracle.Oracle(prob)
        except oracle.OracleError:
            continue
        lam = rng.normal(size=k)
        m0, m1 = P.min_marginals(lam)
        b0, b1 = brute.row_min_marginals(a, sense, b, lam)
        np.testing.assert_allclose(m0, b0, rtol=0, atol=1e-12)
        np.testing.assert_allclose(m1, b1, rtol=0, atol=1e-12)
        # E^j = min(m0, m1) for every variable
        E = P.lower_bound(lam, np.zeros(k), energies=True)[1][0]
        assert abs(E - min(m0[0], m1[0])) < 1e-12
        checked += 1
    assert checked > 30


def test_multi_row_problem_vs_enumeration():
    rows = workloads.random_rows(30, kmax=9, n=20, seed=5)
    rng = np.random.default_rng(0)
    good = []
    for r in rows:
        try:
            oracle.Oracle(workloads.single_rows_problem([r], 20, np.zeros(20)))
            good.append(r)
        except oracle.OracleError:
            pass
    P = oracle.Oracle(workloads.single_rows_problem(good, 20, np.zeros(20)))
    lam = rng.normal(size=P.num_slots)
    m0, m1 = P.min_marginals(lam)
    for j, (v, a, s, b) in enumerate(good):
        sl = slice(P.row_ptr[j], P.row_ptr[j + 1])
        b0, b1 = brute.row_min_marginals(a, s, b, lam[sl])
        np.testing.assert_allclose(m0[sl], b0, atol=1e-12)
        np.testing.assert_allclose(m1[sl], b1, atol=1e-12)


def test_independent_set_row_closed_form():
    """x_u + x_v <= 1: m1_u = lam_u, m0_u = min(0, lam_v)."""
    P = oracle.Oracle(workloads.single_rows_problem([(np.array([0, 1]), np.array([1, 1]), 0, 1)], 2, np.zeros(2)))
    rng = np.random.default_rng(3)
    for _ in range(50):
        lam = rng.normal(size=2)
        m0, m1 = P.min_marginals(lam)
        assert m1[0] == lam[0] and m1[1] == lam[1]
        assert m0[0] == min(0.0, lam[1]) and m0[1] == min(0.0, lam[0])


@pytest.mark.parametrize("k", [2, 3, 5, 8, 300])
def test_at_most_one_closed_form(k):
    """sum x <= 1: m1_i = lam_i, m0_i = min(0, min_{p != i} lam_p)."""
    P = oracle.Oracle(workloads.single_rows_problem([(np.arange(k), np.ones(k), 0, 1)], k, np.zeros(k)))
    rng = np.random.default_rng(k)
    for _ in range(20):
        lam = rng.normal(size=k)
        m0, m1 = P.min_marginals(lam)
        for i in range(k):
            others = np.delete(lam, i)
            assert abs(m1[i] - lam[i]) < 1e-15
            assert abs(m0[i] - min(0.0, others.min())) < 1e-15


@pytest.mark.parametrize("k", [2, 3, 6, 9, 300])
def test_at_least_one_closed_form(k):
    """sum x >= 1: m1_i = lam_i + sum_{p!=i} min(0, lam_p);
    m0_i = sum_{p!=i} min(0, lam_p) + (min_{p!=i} lam_p if no lam_p < 0 else 0)."""
    P = oracle.Oracle(workloads.single_rows_problem([(np.arange(k), np.ones(k), 1, 1)], k, np.zeros(k)))
    rng = np.random.default_rng(100 + k)
    for t in range(30):
        lam = rng.normal(size=k) + (1.5 if t % 3 == 0 else 0.0)  # some all-positive draws
        m0, m1 = P.min_marginals(lam)
        for i in range(k):
            o = np.delete(lam, i)
            neg = np.minimum(o, 0.0).sum()
            assert abs(m1[i] - (lam[i] + neg)) < 1e-12
            want0 = neg + (o.min() if (o >= 0).all() else 0.0)
            assert abs(m0[i] - want0) < 1e-12


def test_minimiser_vs_enumeration():
    """The minimising vectors s^j(i, beta) of Alg. 2 equal the brute-force
    argmin when the minimum is unique."""
    rng = np.random.default_rng(21)
    checked = 0
    for (v, a, sense, b) in workloads.random_rows(60, kmax=10, seed=21):
        k = len(v)
        try:
            P = oracle.Oracle(workloads.single_rows_problem([(np.arange(k), a, sense, b)], k, np.zeros(k)))
        except oracle.OracleError:
            continue
        lam = rng.normal(size=k)
        for h in range(k):
            for beta in (0, 1):
                xb, gap = brute.row_argmin(a, sense, b, lam, h, beta)
                if gap < 1e-9:
                    continue
                np.testing.assert_array_equal(P.minimiser(0, lam, h, beta), xb)
                checked += 1
    assert checked > 100


def test_minimiser_tie_rules():
    """With all-zero costs every feasible vector ties, so the tie rules alone
    decide.  For sum x <= 1 the canonical order puts the "one already taken"
    node first on every level below the root (its key (lo, hi) = (., bottom)
    sorts before (., .)), so:
      * h = 0: x = beta * e_0 (root, then 0-arcs);
      * h > 0, beta = 0: the smallest-rank node of level h is "taken", whose
        only in-arc path is the root's 1-arc followed by 0-arcs: x = e_0;
      * h > 0, beta = 1: only the "free" node has a 1-arc; its prefix is all
        0-arcs: x = e_h."""
    k = 5
    P = oracle.Oracle(workloads.single_rows_problem([(np.arange(k), np.ones(k), 0, 1)], k, np.zeros(k)))
    for h in range(k):
        for beta in (0, 1):
            x = P.minimiser(0, np.zeros(k), h, beta)
            want = np.zeros(k, np.int32)
            if h == 0:
                want[0] = beta
            elif beta == 0:
                want[0] = 1
            else:
                want[h] = 1
            np.testing.assert_array_equal(x, want)


def _smallest(v, r, negative_only):
    """Sum of the r smallest entries of v (only the negative ones among them
    when negative_only)."""
    w = np.sort(v)[:r]
    return float(np.minimum(w, 0.0).sum() if negative_only else w.sum())


@pytest.mark.parametrize("k,sense,b", [(40, workloads.LE, 3), (500, workloads.LE, 10), (300, workloads.EQ, 25),
                                       (64, workloads.EQ, 1)])
def test_cardinality_closed_form(k, sense, b):
    """Long cardinality rows (the sizes the long-BDD path runs): for sum x <= b
    the cheapest assignment takes the at most b most negative costs, so
    m1_i = lam_i + (b - 1 smallest negatives of the others), m0_i = (b
    smallest negatives of the others); for sum x = b exactly b are taken:
    m1_i = lam_i + (b - 1 smallest of the others), m0_i = (b smallest of the
    others)."""
    P = oracle.Oracle(workloads.single_rows_problem([(np.arange(k), np.ones(k), sense, b)], k, np.zeros(k)))
    rng = np.random.default_rng(7 * k + b)
    neg_only = sense == workloads.LE
    for _ in range(3):
        lam = rng.normal(size=k)
        m0, m1 = P.min_marginals(lam)
        for i in range(0, k, max(1, k // 40)):
            o = np.delete(lam, i)
            assert abs(m1[i] - (lam[i] + _smallest(o, b - 1, neg_only))) < 1e-12
            assert abs(m0[i] - _smallest(o, b, neg_only)) < 1e-12
