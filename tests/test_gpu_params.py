"""GPU parity of the non-parametric update (eq. 2), the output transforms of
Alg. 3 and their adjoints against the FP64 oracle, and of one whole DOGE
round (transforms -> eq. 2 -> T iterations of Alg. 1 -> lower bound) end to
end through the autograd Functions.  Tolerances as for the solver: 1e-5
relative on values, 1e-4 absolute on O(1) gradients."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_2205_11638_gb300 import build, solver
from paper_2205_11638_gb300.solver import DualIterate, LowerBound, NonParamUpdate, ParamTransform

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _np(t):
    return t.detach().double().cpu().numpy()


def _f32(x):
    return np.float32(x).astype(np.float64)


def test_nonparam_and_transforms_vs_oracle():
    prob = workloads.matching_quadratic(L=60, R=60, pairs=3000, seed=6)
    O = oracle.Oracle(prob)
    A = solver.plan(prob).bind()
    rng = np.random.default_rng(0)
    lam = _f32(rng.normal(size=O.num_slots))
    th, ah, wh = (_f32(rng.normal(size=O.num_slots) * 2) for _ in range(3))
    lam_g = A.from_csr(lam)
    A.nonparam_update(lam_g, A.from_csr(th))
    np.testing.assert_allclose(_np(A.to_csr(lam_g)), O.nonparam_update(lam, th), atol=1e-5)
    got = A.param_transform(A.from_csr(ah), A.from_csr(wh), A.from_csr(th))
    want = O.param_transform(ah, wh, th)
    for g, w in zip(got, want):
        np.testing.assert_allclose(_np(A.to_csr(g)), w, atol=1e-5, rtol=1e-5)
    ga, gw, gt = (_f32(rng.normal(size=O.num_slots)) for _ in range(3))
    gotb = A.param_transform_backward(got[0], got[1], A.from_csr(ga), A.from_csr(gw), A.from_csr(gt))
    wantb = O.param_transform_backward(want[0], want[1], ga, gw, gt)
    for g, w in zip(gotb, wantb):
        np.testing.assert_allclose(_np(A.to_csr(g)), w, atol=1e-5)
    g_th = A.nonparam_backward(A.from_csr(gt))
    np.testing.assert_allclose(_np(A.to_csr(g_th)), wantb[2], atol=1e-5)


def _tiny(seed, n=14, rows=12, kmax=6):
    good = []
    for r in workloads.random_rows(8 * rows, kmax=kmax, n=n, seed=seed):
        try:
            oracle.Oracle(workloads.single_rows_problem([r], n, np.zeros(n)))
            good.append(r)
        except oracle.OracleError:
            pass
        if len(good) == rows:
            break
    rng = np.random.default_rng(seed)
    return workloads.single_rows_problem(good, n, rng.normal(size=n))


@pytest.mark.parametrize("seed", [31, 32])
def test_doge_round_end_to_end_gradients(seed):
    """alpha-hat, omega-hat, theta-hat -> Alg. 3 transforms -> eq. 2 ->
    2 iterations of Alg. 1 -> lower bound; gradients of the bound with respect
    to the predictor outputs, GPU autograd chain vs the oracle's chain."""
    prob = _tiny(seed)
    O = oracle.Oracle(prob)
    A = solver.plan(prob).bind()
    rng = np.random.default_rng(seed)
    lam0, M0 = O.init_lambda()
    lam0 = _f32(lam0)
    ah, wh, th = (_f32(rng.normal(size=O.num_slots)) for _ in range(3))
    T = 2
    # oracle chain
    a, w, t = O.param_transform(ah, wh, th)
    lam1 = O.nonparam_update(lam0, t)
    lT, MT = O.iterate(lam1, M0, w, a, T)
    sl, sM = O.lb_seed(lT, MT)
    gl1, _, gw, ga = O.backward(lam1, M0, w, a, T, sl, sM)
    g_t = gl1 - (np.bincount(O.col, weights=gl1, minlength=O.n) / np.maximum(O.deg, 1))[O.col]
    want = O.param_transform_backward(a, w, ga, gw, g_t)
    # GPU chain through autograd
    leaves = [A.from_csr(x).requires_grad_(True) for x in (ah, wh, th)]
    a_g, w_g, t_g = ParamTransform.apply(*leaves, A)
    lam1_g = NonParamUpdate.apply(A.from_csr(lam0), t_g, A)
    lT_g, MT_g = DualIterate.apply(lam1_g, A.from_csr(M0), w_g, a_g, A, T, 1)
    lb = LowerBound.apply(lT_g, MT_g, A).sum()
    lb.backward()
    v = float(lb.detach())
    assert abs(v - O.lower_bound(lT, MT)) < 1e-4 * max(1.0, abs(v))
    for leaf, wv in zip(leaves, want):
        np.testing.assert_allclose(_np(A.to_csr(leaf.grad)), wv, atol=1e-4)


@pytest.mark.parametrize("a", [1.0, 10.0, 100.0])
def test_smoothed_dual_vs_oracle(a):
    """Smoothed-dual features for the three smoothing factors of the feature
    table, FP32 log-sum-exp on the GPU against the FP64 oracle."""
    prob = workloads.matching_quadratic(L=60, R=60, pairs=3000, seed=8)
    O = oracle.Oracle(prob)
    A = solver.plan(prob).bind()
    rng = np.random.default_rng(int(a))
    lam = _f32(rng.normal(size=O.num_slots) * 2)
    E, mg = A.smoothed_dual(A.from_csr(lam), a)
    oE, omg = O.smoothed(lam, a)
    np.testing.assert_allclose(_np(E), oE, rtol=1e-5, atol=1e-5 * a)
    np.testing.assert_allclose(_np(A.to_csr(mg)), omg, atol=1e-4)
