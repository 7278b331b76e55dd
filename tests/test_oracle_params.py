"""Pins of the oracle's non-parametric update (eq. 2) and of the output
transforms of Alg. 3 (softmax of alpha-hat over J_i, sigmoid of omega-hat,
centring of theta-hat) against what they must satisfy: dual feasibility is
kept (Prop. 1 / eq. 2's stated purpose), the weights are convex, the
transforms' invariances, and FP64 central differences for the backward."""
import numpy as np
import pytest

import oracle
import workloads


@pytest.fixture(scope="module")
def P():
    return oracle.Oracle(workloads.matching_quadratic(L=20, R=20, pairs=150, seed=3))


def _sum_by_var(P, x):
    s = np.zeros(P.n)
    np.add.at(s, P.col, x)
    return s


def test_nonparam_update_keeps_dual_feasibility(P):
    rng = np.random.default_rng(0)
    lam, _ = P.init_lambda()
    theta = rng.normal(size=P.num_slots) * 3
    lam2 = P.nonparam_update(lam, theta)
    np.testing.assert_allclose(_sum_by_var(P, lam2), _sum_by_var(P, lam), atol=1e-12)
    # a theta that already sums to 0 over every J_i is added unchanged
    th0 = theta - (_sum_by_var(P, theta) / np.maximum(P.deg, 1))[P.col]
    np.testing.assert_allclose(P.nonparam_update(lam, th0), lam + th0, atol=1e-12)
    # a theta constant over J_i changes nothing
    const = rng.normal(size=P.n)[P.col]
    np.testing.assert_allclose(P.nonparam_update(lam, const), lam, atol=1e-12)


def test_transforms_invariants(P):
    rng = np.random.default_rng(1)
    ah, wh, th = (rng.normal(size=P.num_slots) * 2 for _ in range(3))
    a, w, t = P.param_transform(ah, wh, th)
    np.testing.assert_allclose(_sum_by_var(P, a)[P.deg > 0], 1.0, atol=1e-12)
    assert np.all(a > 0) and np.all((w > 0) & (w < 1))
    np.testing.assert_allclose(_sum_by_var(P, t), 0.0, atol=1e-12)
    # shift invariance of the softmax per variable, sigmoid symmetry
    a2, w2, _ = P.param_transform(ah + rng.normal(size=P.n)[P.col], -wh, th)
    np.testing.assert_allclose(a2, a, atol=1e-12)
    np.testing.assert_allclose(w2, 1.0 - w, atol=1e-12)
    # alpha-hat equal over J_i gives the plain method's 1/|J_i|; omega-hat 0 gives 0.5
    a3, w3, _ = P.param_transform(np.zeros(P.num_slots), np.zeros(P.num_slots), th)
    np.testing.assert_allclose(a3, 1.0 / P.deg[P.col], atol=1e-15)
    np.testing.assert_allclose(w3, 0.5, atol=1e-15)
    # the transformed parameters satisfy Prop. 1's conditions
    assert np.all(w >= 0) and np.all(w <= 1)


def test_transforms_backward_fd(P):
    rng = np.random.default_rng(2)
    ah, wh, th = (rng.normal(size=P.num_slots) for _ in range(3))
    ga, gw, gt = (rng.normal(size=P.num_slots) for _ in range(3))

    def L(ah_, wh_, th_):
        a, w, t = P.param_transform(ah_, wh_, th_)
        return ga @ a + gw @ w + gt @ t

    a, w, _ = P.param_transform(ah, wh, th)
    gah, gwh, gth = P.param_transform_backward(a, w, ga, gw, gt)
    h = 1e-6
    for x, g, which in ((ah, gah, 0), (wh, gwh, 1), (th, gth, 2)):
        for q in rng.choice(P.num_slots, size=25, replace=False):
            e = np.zeros(P.num_slots)
            e[q] = h
            args_p = [ah, wh, th]
            args_m = [ah, wh, th]
            args_p = [v + e if k == which else v for k, v in enumerate(args_p)]
            args_m = [v - e if k == which else v for k, v in enumerate(args_m)]
            fd = (L(*args_p) - L(*args_m)) / (2 * h)
            assert abs(fd - g[q]) < 1e-6 * max(1.0, abs(fd))
