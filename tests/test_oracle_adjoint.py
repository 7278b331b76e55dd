"""Pins of the oracle's backpropagation (Alg. 2, Prop. 2) against FP64
central finite differences of the forward iteration on tiny instances.

The map of Alg. 1 is piecewise linear; a coordinate is compared only where
two step sizes agree (away from kinks)."""
import numpy as np
import pytest

import oracle
import workloads


def _tiny(seed, n=10, rows=8, kmax=5):
    good = []
    for r in workloads.random_rows(6 * rows, kmax=kmax, n=n, seed=seed):
        try:
            oracle.Oracle(workloads.single_rows_problem([r], n, np.zeros(n)))
            good.append(r)
        except oracle.OracleError:
            pass
        if len(good) == rows:
            break
    rng = np.random.default_rng(seed)
    return oracle.Oracle(workloads.single_rows_problem(good, n, rng.normal(size=n)))


def _inputs(P, seed):
    rng = np.random.default_rng(seed)
    lam = rng.normal(size=P.num_slots)
    M = 0.3 * rng.normal(size=P.num_slots)
    omega = rng.uniform(0.2, 0.8, P.num_slots)
    alpha = rng.uniform(0.1, 1.0, P.num_slots)
    s = np.zeros(P.n)
    np.add.at(s, P.col, alpha)
    alpha = alpha / s[P.col]
    return lam, M, omega, alpha


def _fd_check(f, x, g, h=1e-6, min_checked=5):
    checked = 0
    for q in range(len(x)):
        e = np.zeros_like(x)
        e[q] = 1.0
        d1 = (f(x + h * e) - f(x - h * e)) / (2 * h)
        d2 = (f(x + 0.25 * h * e) - f(x - 0.25 * h * e)) / (0.5 * h)
        if abs(d1 - d2) > 1e-6 * max(1.0, abs(d1)):
            continue  # a kink inside the stencil
        assert abs(g[q] - d1) < 1e-5 * max(1.0, abs(d1)), (q, g[q], d1)
        checked += 1
    assert checked >= min_checked


@pytest.mark.parametrize("seed,iters", [(1, 1), (2, 2), (3, 3)])
def test_linear_loss_fd(seed, iters):
    """L = <a, lambda_T> + <b, M_T>: analytic gradients w.r.t. lambda_0, M_0,
    omega and alpha equal finite differences."""
    P = _tiny(seed)
    lam, M, omega, alpha = _inputs(P, seed)
    rng = np.random.default_rng(100 + seed)
    a = rng.normal(size=P.num_slots)
    b = rng.normal(size=P.num_slots)

    def loss(l0, M0, om, al):
        lT, MT = P.iterate(l0, M0, om, al, iters)
        return a @ lT + b @ MT

    gl, gM, gw, ga = P.backward(lam, M, omega, alpha, iters, a, b)
    _fd_check(lambda x: loss(x, M, omega, alpha), lam, gl)
    _fd_check(lambda x: loss(lam, x, omega, alpha), M, gM)
    _fd_check(lambda x: loss(lam, M, x, alpha), omega, gw)
    _fd_check(lambda x: loss(lam, M, omega, x), alpha, ga)


@pytest.mark.parametrize("seed", [5, 6])
def test_lower_bound_loss_fd(seed):
    """The training loss (eq. 3 plus the unary term of the bound) through 2
    iterations: seeds from the minimising assignments."""
    P = _tiny(seed, n=9, rows=7)
    lam, M, omega, alpha = _inputs(P, seed)
    iters = 2

    def loss(l0, M0, om, al):
        lT, MT = P.iterate(l0, M0, om, al, iters)
        return P.lower_bound(lT, MT)

    lT, MT = P.iterate(lam, M, omega, alpha, iters)
    sl, sM = P.lb_seed(lT, MT)
    gl, gM, gw, ga = P.backward(lam, M, omega, alpha, iters, sl, sM)
    _fd_check(lambda x: loss(x, M, omega, alpha), lam, gl, min_checked=3)
    _fd_check(lambda x: loss(lam, M, x, alpha), omega, gw, min_checked=3)
    _fd_check(lambda x: loss(lam, M, omega, x), alpha, ga, min_checked=3)


def test_gradient_of_M0_is_shared_per_variable():
    """Alg. 2 (reading of its first line): the gradient of M^old_ij is the same
    for every j in J_i."""
    P = _tiny(8)
    lam, M, omega, alpha = _inputs(P, 8)
    rng = np.random.default_rng(0)
    _, gM, _, _ = P.backward(lam, M, omega, alpha, 2, rng.normal(size=P.num_slots), rng.normal(size=P.num_slots))
    for i in range(P.n):
        v = gM[P.col == i]
        if len(v):
            assert np.ptp(v) == 0.0


@pytest.mark.parametrize("seed,iters", [(21, 1), (22, 2)])
def test_oracle_backward_equals_dense_autograd(seed, iters):
    """The oracle's Alg. 2 (minimiser vectors from its BDDs) against torch
    autograd through a dense restatement of Alg. 1 (brute-force min-marginals):
    two implementations with nothing in common."""
    import torch

    from tests import dense_ref

    good = []
    for r in workloads.random_rows(6 * 8, kmax=5, n=10, seed=seed):
        try:
            oracle.Oracle(workloads.single_rows_problem([r], 10, np.zeros(10)))
            good.append(r)
        except oracle.OracleError:
            pass
        if len(good) == 8:
            break
    rng = np.random.default_rng(seed)
    prob = workloads.single_rows_problem(good, 10, rng.normal(size=10))
    O = oracle.Oracle(prob)
    lam, M, omega, alpha = _inputs(O, seed)
    rng2 = np.random.default_rng(500 + seed)
    a = rng2.normal(size=O.num_slots)
    b = rng2.normal(size=O.num_slots)
    gl, gM, gw, ga = O.backward(lam, M, omega, alpha, iters, a, b)
    t = [torch.tensor(x, dtype=torch.float64, requires_grad=True) for x in (lam, M, omega, alpha)]
    lT, MT = dense_ref.iterate(prob, *t, iters)
    loss = (lT * torch.as_tensor(a)).sum() + (MT * torch.as_tensor(b)).sum()
    loss.backward()
    for mine, ref in zip((gl, gM, gw, ga), t):
        np.testing.assert_allclose(mine, ref.grad.numpy(), atol=1e-9, rtol=1e-9)
