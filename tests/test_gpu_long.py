"""GPU parity of the long-BDD execution model (one warp per BDD, a level's
nodes over the lanes) against the FP64 oracle, through the C ABI.

Rows whose BDD exceeds a tile lane (more than 254 nodes, or a level wider
than 128) are swept by these kernels; the oracle builds and sweeps them like
any other row.  Bars as for the tiles: lambda and M after one iteration
within 1e-5 * max|c|, the bound after 100 iterations within 1e-5 relative,
min-marginals and energies within 1e-5 * max|c|, minimising assignments
exact on tie-free inputs, gradients of unrolls of up to 3 iterations within
1e-4 on tie-free inputs."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_2205_11638_gb300 import build, solver

pytestmark = pytest.mark.gpu

TOL_LAM = 1e-5
TOL_LB = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _np(t):
    return t.detach().double().cpu().numpy()


def _softmax_alpha(col, n, rng):
    e = np.exp(rng.normal(size=len(col)))
    s = np.zeros(n)
    np.add.at(s, col, e)
    return e / s[col]


def _parity(prob, iters_lb=100, per_slot=False, seed=0, **opts):
    O = oracle.Oracle(prob)
    A = solver.plan(prob, **opts).bind()
    assert A.plan.sizes.num_long_bdds > 0
    cmax = np.abs(prob["c"]).max()
    rng = np.random.default_rng(seed)
    omega = alpha = om_t = al_t = None
    if per_slot:
        alpha = np.float32(_softmax_alpha(prob["col"], prob["n"], rng)).astype(np.float64)
        omega = np.float32(1.0 / (1.0 + np.exp(-rng.normal(size=len(prob["col"]))))).astype(np.float64)
        om_t, al_t = A.from_csr(omega), A.from_csr(alpha)
    lam, M = A.init_lambda()
    ol, oM = O.init_lambda()
    A.iterate(lam, M, om_t, al_t, iters=1)
    ol, oM = O.iterate(ol, oM, 0.5 if omega is None else omega, alpha, 1)
    assert float(np.abs(_np(A.to_csr(lam)) - ol).max()) <= TOL_LAM * cmax
    assert float(np.abs(_np(A.to_csr(M)) - oM).max()) <= TOL_LAM * cmax
    lb = A.iterate(lam, M, om_t, al_t, iters=iters_lb - 1, lb=True)
    assert torch.isfinite(lam).all() and torch.isfinite(lb).all()
    ol, oM = O.iterate(ol, oM, 0.5 if omega is None else omega, alpha, iters_lb - 1)
    want = O.lower_bound(ol, oM, per_instance=True)[1]
    rel = np.abs(lb.cpu().numpy() - want) / np.maximum(1.0, np.abs(want))
    assert rel.max() <= TOL_LB, (lb, want)
    return A, O


@pytest.mark.parametrize("per_slot", [False, True])
def test_long_rows_mixed_with_short_rows(per_slot):
    """Cardinality rows over 500 variables (<= 1, <= 10, = 25), >= 1 over 300,
    a knapsack row with a level of 169 nodes, and 40 short rows in one arena."""
    _parity(workloads.long_rows_mix(seed=3), per_slot=per_slot, seed=4)


def test_long_rows_only():
    """An arena of long BDDs only (no tiles): the long launch runs alone."""
    prob = workloads.long_rows_mix(seed=8, n_short=0)
    A, _ = _parity(prob, iters_lb=60)
    assert A.plan.sizes.num_tiles == 0


@pytest.mark.parametrize("lanes", [0, 2])
def test_assignment_instance(lanes):
    """The assignment workload's shape at 400 x 400 with 300 candidates per
    left node: 800 rows of about 300 variables, every BDD a long one (swept
    one to a warp, and 16 to a warp with two lanes each)."""
    _parity(workloads.assignment(L=400, R=400, cand=300, seed=12), iters_lb=100, long_lanes=lanes)


@pytest.mark.parametrize("per_slot", [False, True])
@pytest.mark.parametrize("name,lanes", [("mix", 0), ("assignment", 0), ("assignment", 2), ("assignment", 8)])
def test_plain_sweeps_equal_recording_sweeps(name, lanes, per_slot):
    """dg_iterate's plain sweeps (the long BDDs whose levels have at most 32
    nodes swept 32 / G to a warp, G lanes each, path costs in registers)
    against the recording sweeps of a one-segment dg_iterate_checkpointed
    (every long BDD through the general level loop, one warp each): lambda,
    M and the bound bit for bit, at the lane count dg_bind picks (32 for
    both instances: the mix's widest narrow level has 26 nodes, and the
    assignment instance has too few BDDs to fill the SMs at fewer lanes) and
    at forced ones (several BDDs of different lengths to a warp)."""
    if name == "mix":
        prob = workloads.long_rows_mix(seed=21)
    else:
        prob = workloads.assignment(L=120, R=300, cand=280, seed=22)
    A = solver.plan(prob, long_lanes=lanes).bind()
    assert A.plan.sizes.num_long_bdds > 0
    om = al = None
    if per_slot:
        rng = np.random.default_rng(5)
        al = A.from_csr(_softmax_alpha(prob["col"], prob["n"], rng))
        om = A.from_csr(rng.uniform(0.2, 0.8, size=len(prob["col"])))
    lam0, M0 = A.init_lambda()
    T = 6
    l1, m1 = lam0.clone(), M0.clone()
    lb1 = A.iterate(l1, m1, om, al, iters=T, lb=True)
    l2, m2 = lam0.clone(), M0.clone()
    _, lb2 = A.iterate_checkpointed(l2, m2, om, al, iters=T, ckpt_every=T, lb=True)
    assert torch.equal(l1, l2) and torch.equal(m1, m2) and torch.equal(lb1, lb2)


def test_long_min_marginals_energies_and_seed():
    prob = workloads.long_rows_mix(seed=6)
    O = oracle.Oracle(prob)
    A = solver.plan(prob).bind()
    rng = np.random.default_rng(2)
    lam = A.from_csr(rng.normal(size=O.num_slots))
    M = A.from_csr(0.1 * rng.normal(size=O.num_slots))
    lam_c, M_c = _np(A.to_csr(lam)), _np(A.to_csr(M))
    cmax = 4.0
    m0, m1 = A.min_marginals(lam)
    o0, o1 = O.min_marginals(lam_c)
    np.testing.assert_allclose(_np(A.to_csr(m0)), o0, atol=TOL_LAM * cmax * 10, rtol=0)
    np.testing.assert_allclose(_np(A.to_csr(m1)), o1, atol=TOL_LAM * cmax * 10, rtol=0)
    lb, E = A.lower_bound(lam, M, energies=True)
    want, oE = O.lower_bound(lam_c, M_c, energies=True)
    np.testing.assert_allclose(_np(E), oE, atol=TOL_LAM * cmax * 10, rtol=0)
    assert abs(float(lb[0]) - want) <= TOL_LB * max(1.0, abs(want))
    gl, gM = A.lb_seed(lam, M)
    ol, oM = O.lb_seed(lam_c, M_c)
    np.testing.assert_array_equal(_np(A.to_csr(gl)), ol)
    np.testing.assert_array_equal(_np(A.to_csr(gM)), oM)


@pytest.mark.parametrize("a", [1.0, 10.0])
def test_long_smoothed_dual(a):
    prob = workloads.long_rows_mix(seed=7)
    O = oracle.Oracle(prob)
    A = solver.plan(prob).bind()
    rng = np.random.default_rng(3)
    lam = A.from_csr(rng.normal(size=O.num_slots))
    E, mg = A.smoothed_dual(lam, a)
    oE, omg = O.smoothed(_np(A.to_csr(lam)), a)
    np.testing.assert_allclose(_np(E), oE, rtol=1e-5, atol=1e-4)
    np.testing.assert_allclose(_np(A.to_csr(mg)), omg, rtol=0, atol=1e-4)


@pytest.mark.parametrize("iters,per_slot", [(1, True), (2, True), (2, False)])
def test_long_adjoint_vs_oracle(iters, per_slot):
    """Alg. 2 through the long-BDD sweeps (and the tiles' of the short rows)
    from random tie-free (lambda, M), against the oracle's explicit
    minimiser vectors."""
    prob = workloads.long_rows_mix(seed=9, n_short=20)
    O = oracle.Oracle(prob)
    A = solver.plan(prob).bind()
    rng = np.random.default_rng(20 + iters)
    f32 = lambda x: np.float32(x).astype(np.float64)  # noqa: E731
    lam, M = f32(rng.normal(size=O.num_slots)), f32(0.3 * rng.normal(size=O.num_slots))
    if per_slot:
        omega = f32(rng.uniform(0.2, 0.8, O.num_slots))
        alpha = f32(_softmax_alpha(O.col, O.n, rng))
    else:
        omega, alpha = 0.5, None
    a, b = f32(rng.normal(size=O.num_slots)), f32(rng.normal(size=O.num_slots))
    want = O.backward(lam, M, omega, alpha, iters, a, b)
    om_t = A.from_csr(omega) if per_slot else None
    al_t = A.from_csr(alpha) if per_slot else None
    got = A.backward(A.from_csr(lam), A.from_csr(M), om_t, al_t, iters, 1, A.from_csr(a), A.from_csr(b))
    for g, w in zip(got if per_slot else got[:2], want):
        np.testing.assert_allclose(_np(A.to_csr(g)), w, atol=1e-4, rtol=0)


def test_long_adjoint_checkpoint_interval_bit_identical():
    prob = workloads.long_rows_mix(seed=10, n_short=20)
    A = solver.plan(prob).bind()
    lam, M = A.init_lambda()
    rng = np.random.default_rng(0)
    gl = A.from_csr(rng.normal(size=A.plan.sizes.num_lambda))
    gM = A.from_csr(rng.normal(size=A.plan.sizes.num_lambda))
    outs = [A.backward(lam, M, None, None, 5, ck, gl, gM) for ck in (1, 2, 5)]
    for o in outs[1:]:
        for x, y in zip(o, outs[0]):
            assert torch.equal(x, y)
