"""Pins of the oracle's Alg. 1 (generalized min-marginal averaging, Sec. 3.2)
against what the paper and the mathematics fix: the feasibility invariant and
monotone bound of Prop. 1, weak duality against a brute-force optimum, exact
special cases and an independent closed-form restatement for independent-set
rows."""
import numpy as np
import pytest

import oracle
import workloads
from tests import brute


def _feasibility_residual(P, lam, M):
    tot = np.zeros(P.n)
    np.add.at(tot, P.col, lam + M)
    covered = P.deg > 0
    return np.abs(tot - P.c)[covered].max() / max(1.0, np.abs(P.c).max())


def _random_feasible_problem(seed, n=16, rows=14, kmax=7):
    good = []
    for r in workloads.random_rows(4 * rows, kmax=kmax, n=n, seed=seed):
        try:
            oracle.Oracle(workloads.single_rows_problem([r], n, np.zeros(n)))
            good.append(r)
        except oracle.OracleError:
            pass
        if len(good) == rows:
            break
    rng = np.random.default_rng(seed)
    return workloads.single_rows_problem(good, n, rng.normal(size=n))


@pytest.mark.parametrize("make", [lambda: workloads.set_cover(), lambda: _random_feasible_problem(3),
                                  lambda: workloads.independent_set(n=300, seed=9),
                                  lambda: workloads.long_rows_mix(seed=3, n_short=20)])
def test_prop1_feasibility_and_monotone_per_sweep(make):
    """Prop. 1: sum_j (lambda_ij + M_ij) = c_i after every sweep (reading of the
    garbled invariant in its proof) and the bound never decreases."""
    P = oracle.Oracle(make())
    rng = np.random.default_rng(0)
    lam, M = P.init_lambda()
    omega = rng.uniform(0.0, 1.0, P.num_slots)
    alpha = rng.uniform(0.1, 1.0, P.num_slots)
    s = np.zeros(P.n)
    np.add.at(s, P.col, alpha)
    alpha = alpha / s[P.col]  # convex weights per variable
    prev = P.lower_bound(lam, M)
    for k in range(12):
        lam, M = P.sweep(lam, M, forward=(k % 2 == 0), omega=omega, alpha=alpha)
        assert _feasibility_residual(P, lam, M) < 1e-12
        lb = P.lower_bound(lam, M)
        assert lb >= prev - 1e-9 * max(1.0, abs(prev))
        prev = lb


def test_weak_duality_config1_bruteforce():
    """Config 1: 100 plain iterations, the bound stays <= the brute-force ILP
    optimum over all 2^24 assignments and never decreases."""
    prob = workloads.set_cover()
    opt, _ = brute.problem_opt(prob)
    P = oracle.Oracle(prob)
    lam, M = P.init_lambda()
    lam, M, tr = P.iterate(lam, M, 0.5, None, 100, trace=True)
    assert np.all(np.diff(tr) >= -1e-9)
    assert tr[-1] <= opt + 1e-9
    assert tr[-1] > P.lower_bound(*P.init_lambda())


def test_disjoint_rows_bound_is_optimum():
    """Every variable in exactly one row: the dual is tight at the uniform
    split and stays at the optimum."""
    rows = [(np.array([0, 1, 2]), np.array([1, 1, 1]), 1, 1),
            (np.array([3, 4]), np.array([1, -1]), 0, 0),
            (np.array([5, 6, 7, 8]), np.array([2, 1, 1, 3]), 0, 4)]
    rng = np.random.default_rng(4)
    prob = workloads.single_rows_problem(rows, 10, rng.normal(size=10))  # var 9 uncovered
    opt, _ = brute.problem_opt(prob)
    P = oracle.Oracle(prob)
    lam, M = P.init_lambda()
    assert abs(P.lower_bound(lam, M) - opt) < 1e-12
    lam, M, tr = P.iterate(lam, M, 0.5, None, 5, trace=True)
    np.testing.assert_allclose(tr, opt, atol=1e-12)


def test_single_row_bound():
    rng = np.random.default_rng(8)
    for (v, a, s, b) in workloads.random_rows(30, kmax=10, seed=8):
        k = len(v)
        prob = workloads.single_rows_problem([(np.arange(k), a, s, b)], k, rng.normal(size=k))
        try:
            P = oracle.Oracle(prob)
        except oracle.OracleError:
            continue
        opt, _ = brute.problem_opt(prob)
        assert abs(P.lower_bound(*P.init_lambda()) - opt) < 1e-12


@pytest.mark.parametrize("k,sense,b", [(300, workloads.LE, 1), (500, workloads.LE, 10), (300, workloads.EQ, 25),
                                       (300, workloads.GE, 1)])
def test_single_long_row_bound(k, sense, b):
    """One cardinality row over hundreds of variables (a long BDD): the bound
    at the uniform split is the row's optimum, which sorting gives: the b
    smallest costs for sum x = b, the at most b negative ones among the b
    smallest for sum x <= b, and for sum x >= 1 every negative cost or, if
    there is none, the smallest one."""
    rng = np.random.default_rng(k + b)
    c = rng.normal(size=k)
    P = oracle.Oracle(workloads.single_rows_problem([(np.arange(k), np.ones(k), sense, b)], k, c))
    w = np.sort(c)
    if sense == workloads.EQ:
        opt = w[:b].sum()
    elif sense == workloads.LE:
        opt = np.minimum(w[:b], 0.0).sum()
    else:
        opt = np.minimum(c, 0.0).sum() if (c < 0).any() else w[0]
    assert abs(P.lower_bound(*P.init_lambda()) - opt) < 1e-12


def test_omega_zero_is_identity():
    """omega = 0 extracts nothing, so S stays 0 and lambda never moves."""
    P = oracle.Oracle(workloads.set_cover())
    lam0, M0 = P.init_lambda()
    lam, M, tr = P.iterate(lam0, M0, 0.0, None, 4, trace=True)
    np.testing.assert_array_equal(lam, lam0)
    assert np.all(M == 0)
    np.testing.assert_allclose(tr, P.lower_bound(lam0, M0), atol=0)


def _is_iteration_closed_form(prob, lam, M, omega):
    """One plain iteration on x_u + x_v <= 1 rows, written out from the closed
    form of the row's min-marginals: m1 = lambda_own, m0 = min(0, lambda_other)."""
    col = prob["col"].reshape(-1, 2)
    n = prob["n"]
    deg = np.bincount(prob["col"], minlength=n)
    lam = lam.reshape(-1, 2).copy()
    M = M.reshape(-1, 2).copy()
    for order in ((0, 1), (1, 0)):      # forward sweep, then backward sweep
        S = np.zeros(n)
        np.add.at(S, col.reshape(-1), M.reshape(-1))
        for e in range(len(col)):
            for h in order:
                o = 1 - h
                Mn = omega * (lam[e, h] - min(0.0, lam[e, o]))
                lam[e, h] = lam[e, h] - Mn + S[col[e, h]] / deg[col[e, h]]
                M[e, h] = Mn
    return lam.reshape(-1), M.reshape(-1)


def test_independent_set_iteration_closed_form():
    prob = workloads.independent_set(n=200, seed=31)
    P = oracle.Oracle(prob)
    lam, M = P.init_lambda()
    for it in range(3):
        want_l, want_M = _is_iteration_closed_form(prob, lam, M, 0.5)
        lam, M = P.iterate(lam, M, 0.5, None, 1)
        np.testing.assert_allclose(lam, want_l, atol=1e-12)
        np.testing.assert_allclose(M, want_M, atol=1e-12)


def test_fastdog_special_case_defaults():
    """The plain method is omega = 0.5 and alpha = 1/|J_i| (remark in Sec. 3.2):
    passing them explicitly equals the defaults."""
    P = oracle.Oracle(workloads.set_cover())
    lam, M = P.init_lambda()
    a = P.iterate(lam, M, 0.5, None, 3)
    b = P.iterate(lam, M, np.full(P.num_slots, 0.5), 1.0 / P.deg[P.col], 3)
    np.testing.assert_array_equal(a[0], b[0])


def test_init_split():
    P = oracle.Oracle(workloads.set_cover())
    lam, M = P.init_lambda()
    np.testing.assert_allclose(lam, P.c[P.col] / P.deg[P.col])
    assert _feasibility_residual(P, lam, M) < 1e-15


def test_lb_seed_is_minimiser():
    """Gradient of the loss (eq. 3) = a minimising assignment of each
    subproblem; the unary term gives [S_i < 0]."""
    rng = np.random.default_rng(17)
    prob = _random_feasible_problem(17)
    P = oracle.Oracle(prob)
    lam = rng.normal(size=P.num_slots)
    M = rng.normal(size=P.num_slots)
    gl, gM = P.lb_seed(lam, M)
    _, E = P.lower_bound(lam, M, energies=True)
    for j in range(P.m):
        sl = slice(P.row_ptr[j], P.row_ptr[j + 1])
        a = prob["coef"][sl]
        X = brute.row_feasible(a, int(prob["sense"][j]), int(prob["rhs"][j]))
        assert any((X == gl[sl]).all(axis=1))
        assert abs(gl[sl] @ lam[sl] - E[j]) < 1e-12
    S = np.zeros(P.n)
    np.add.at(S, P.col, M)
    np.testing.assert_array_equal(gM, (S[P.col] < 0).astype(float))


def test_openmp_build_is_bit_identical():
    """The oracle built with OpenMP (sweeps over the BDDs in parallel, the S
    sums afterwards in the fixed order) gives the single-threaded oracle's
    lambda, M and bound bit for bit; it only times the all-cores baseline."""
    prob = workloads.tracking(frames=4, dets=300, seed=17)
    P1 = oracle.Oracle(prob)
    P2 = oracle.Oracle(prob, openmp=True)
    l1, m1 = P1.init_lambda()
    l2, m2 = P2.init_lambda()
    l1, m1 = P1.iterate(l1, m1, 0.5, None, 5)
    l2, m2 = P2.iterate(l2, m2, 0.5, None, 5)
    assert np.array_equal(l1, l2) and np.array_equal(m1, m2)
    assert P1.lower_bound(l1, m1) == P2.lower_bound(l2, m2)
