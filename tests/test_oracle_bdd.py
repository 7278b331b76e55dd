"""Pins of the oracle's BDD builder against brute force (App. B: the r-T paths
of a subproblem's BDD are exactly its feasible assignments; every r-T path
meets one node per variable)."""
import numpy as np
import pytest

import oracle
import workloads
from tests import brute


def _one_row_problem(v, a, sense, b):
    k = len(v)
    return workloads.single_rows_problem([(np.arange(k), a, sense, b)], k, np.zeros(k))


def _rows(seed, num=120, kmax=12):
    return workloads.random_rows(num, kmax=kmax, seed=seed)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_paths_equal_feasible_set(seed):
    checked = 0
    for (v, a, sense, b) in _rows(seed):
        feas = brute.row_feasible(a, sense, b)
        try:
            P = oracle.Oracle(_one_row_problem(v, a, sense, b))
        except oracle.OracleError as e:
            # infeasible (4) or forcing (5): confirm by enumeration
            if e.status == 4:
                assert len(feas) == 0
            else:
                assert e.status == 5
                assert len(feas) > 0
                assert ((feas == 0).all(axis=0) | (feas == 1).all(axis=0)).any()
            continue
        ls, lo, hi = P.bdd(0)
        paths = brute.bdd_paths(ls, lo, hi)
        got = {tuple(p) for p in paths}
        want = {tuple(x) for x in feas}
        assert got == want
        assert len(paths) == len(got)  # every assignment exactly one path
        checked += 1
    assert checked > 40


@pytest.mark.parametrize("seed", [4, 5])
def test_canonical_and_reduced(seed):
    """Quasi-reduced and canonical: per level no two nodes share (lo, hi), the
    nodes are sorted by (lo, hi) with bottom=-2 < top=-1 < ranks, no node has
    two bottom children, every node is reachable from the root, and two
    different feasible sets never give the same structure."""
    for (v, a, sense, b) in _rows(seed):
        try:
            P = oracle.Oracle(_one_row_problem(v, a, sense, b))
        except oracle.OracleError:
            continue
        ls, lo, hi = P.bdd(0)
        k = len(ls) - 1
        assert ls[0] == 0 and ls[1] == 1  # a single root
        reach = {0}
        for h in range(k):
            keys = list(zip(lo[ls[h]:ls[h + 1]], hi[ls[h]:ls[h + 1]]))
            assert keys == sorted(keys)
            assert len(set(keys)) == len(keys)
            assert all(not (x == -2 and y == -2) for x, y in keys)
            for r, (x, y) in enumerate(keys):
                assert r in reach
                if h < k - 1:
                    assert x not in (-1,) and y not in (-1,)
                else:
                    assert x in (-1, -2) and y in (-1, -2)
            reach = {x for x, _ in keys if x >= 0} | {y for _, y in keys if y >= 0}
            if h < k - 1:
                assert reach == set(range(ls[h + 2] - ls[h + 1]))


def test_minimal_width_matches_distinct_residual_functions():
    """The node count of each level equals the number of distinct residual
    feasible sets of the reachable prefixes (brute force over prefixes)."""
    rng = np.random.default_rng(7)
    for _ in range(40):
        k = int(rng.integers(2, 9))
        a = rng.integers(-3, 4, size=k)
        sense = int(rng.integers(0, 3))
        b = int(rng.integers(np.minimum(a, 0).sum(), np.maximum(a, 0).sum() + 1))
        feas = brute.row_feasible(a, sense, b)
        if len(feas) == 0:
            continue
        try:
            P = oracle.Oracle(_one_row_problem(np.arange(k), a, sense, b))
        except oracle.OracleError:
            continue
        ls, _, _ = P.bdd(0)
        fs = {tuple(x) for x in feas}
        for h in range(k):
            classes = set()
            for prefix in {x[:h] for x in fs}:
                rest = frozenset(x[h:] for x in fs if x[:h] == prefix)
                classes.add(rest)
            assert ls[h + 1] - ls[h] == len(classes)


def test_status_codes():
    with pytest.raises(oracle.OracleError) as e:  # 2 x0 + 2 x1 = 1: infeasible
        oracle.Oracle(workloads.single_rows_problem([(np.array([0, 1]), np.array([2, 2]), 2, 1)], 2, np.zeros(2)))
    assert e.value.status == 4
    with pytest.raises(oracle.OracleError) as e:  # x0 + x1 >= 2 forces both
        oracle.Oracle(workloads.single_rows_problem([(np.array([0, 1]), np.array([1, 1]), 1, 2)], 2, np.zeros(2)))
    assert e.value.status == 5
    bad = workloads.single_rows_problem([(np.array([0, 1]), np.array([1, 1]), 0, 1)], 2, np.zeros(2))
    bad["col"] = bad["col"][::-1].copy()
    with pytest.raises(oracle.OracleError) as e:
        oracle.Oracle(bad)
    assert e.value.status == 1


def test_config_sizes():
    """Node and slot counts of the small configurations (stated in the design notes)."""
    P = oracle.Oracle(workloads.independent_set())
    m = len(P.row_ptr) - 1
    assert P.num_slots == 2 * m
    assert P.num_nodes == 3 * m  # root, two second-level nodes per edge row
