"""GPU parity of libdg's sweeps against the FP64 oracle (through the C ABI).

Tolerances (float32 kernels vs the float64 oracle): lambda and M after one
iteration within 1e-5 * max|c| (max abs), the lower bound after 100 (or the
stated number of) iterations within 1e-5 relative; min-marginals within
1e-5 * max|c|.  Integer/structural outputs (minimising assignments) are
compared exactly on tie-free inputs."""
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


def _arena(prob, **opts):
    return solver.plan(prob, **opts).bind()


def _softmax_alpha(col, n, rng):
    z = rng.normal(size=len(col))
    e = np.exp(z)
    s = np.zeros(n)
    np.add.at(s, col, e)
    return e / s[col]


def _check_iterations(prob, iters_lam=1, iters_lb=100, omega=None, alpha=None, **opts):
    O = oracle.Oracle(prob)
    A = _arena(prob, **opts)
    cmax = np.abs(prob["c"]).max()
    lam, M = A.init_lambda()
    ol, oM = O.init_lambda()
    np.testing.assert_allclose(_np(A.to_csr(lam)), ol, rtol=0, atol=1e-6 * cmax)
    om_t = al_t = None
    if omega is not None:
        om_t, al_t = A.from_csr(omega), A.from_csr(alpha)
    A.iterate(lam, M, om_t, al_t, iters=iters_lam)
    assert torch.isfinite(lam).all() and torch.isfinite(M).all()
    ol1, oM1 = O.iterate(ol, oM, 0.5 if omega is None else omega, alpha, iters_lam)
    err_l = np.abs(_np(A.to_csr(lam)) - ol1).max()
    err_M = np.abs(_np(A.to_csr(M)) - oM1).max()
    assert err_l <= TOL_LAM * cmax, err_l
    assert err_M <= TOL_LAM * cmax, err_M
    lb = A.iterate(lam, M, om_t, al_t, iters=iters_lb - iters_lam, lb=True)
    assert torch.isfinite(lam).all() and torch.isfinite(M).all() and torch.isfinite(lb).all()
    olT, oMT = O.iterate(ol1, oM1, 0.5 if omega is None else omega, alpha, iters_lb - iters_lam)
    want = O.lower_bound(olT, oMT, per_instance=True)[1]
    got = lb.cpu().numpy()
    rel = np.abs(got - want) / np.maximum(1.0, np.abs(want))
    assert rel.max() <= TOL_LB, (got, want)
    return A, O, lam, M


def test_config1_set_cover_parity_and_weak_duality():
    from tests import brute
    prob = workloads.set_cover()
    A, O, lam, M = _check_iterations(prob, 1, 100)
    opt, _ = brute.problem_opt(prob)
    assert float(A.lower_bound(lam, M)[0]) <= opt + 1e-4


def test_config2_independent_set_parity():
    _check_iterations(workloads.independent_set(), 1, 200)


@pytest.mark.parametrize("per_slot", [False, True])
def test_variables_with_many_slots(per_slot):
    # every variable in more than 32 rows: S and the per-slot terms come from
    # the warp-per-variable reduction
    prob = workloads.independent_set(n=800, avg_deg=48.0, seed=7)
    if not per_slot:
        _check_iterations(prob, 1, 60)
        return
    rng = np.random.default_rng(8)
    omega = rng.uniform(0.2, 0.8, size=len(prob["col"]))
    _check_iterations(prob, 1, 60, omega=omega, alpha=_softmax_alpha(prob["col"], prob["n"], rng))


def test_config3_matching_per_slot_parameters():
    prob = workloads.matching_quadratic()
    rng = np.random.default_rng(3)
    alpha = _softmax_alpha(prob["col"], prob["n"], rng)
    omega = 1.0 / (1.0 + np.exp(-rng.normal(size=len(prob["col"]))))
    _check_iterations(prob, 1, 20, omega=omega, alpha=alpha)


def test_config4_batched_instances():
    prob, kinds = workloads.batched_mix(num=12, scale=0.03)
    assert len(set(kinds.tolist())) >= 2
    _check_iterations(prob, 1, 30)


def test_config5_tracking_scaled_100_iterations():
    _check_iterations(workloads.tracking(frames=50, dets=400), 1, 100)


def test_config5_full_size_sampled():
    """Full tracking instance in the benchmark's launch configuration: the
    invariants of Prop. 1 hold at any size, and sampled rows' min-marginals
    equal the oracle's evaluated row by row."""
    prob = workloads.tracking()
    A = _arena(prob)
    lam, M = A.init_lambda()
    n = prob["n"]
    col = torch.as_tensor(prob["col"], dtype=torch.int64, device=A.device)
    c = torch.as_tensor(prob["c"], device=A.device)
    covered = torch.bincount(col, minlength=n) > 0
    prev = float(A.lower_bound(lam, M)[0])
    for it in range(5):
        lb = float(A.iterate(lam, M, iters=1, lb=True)[0])
        assert lb >= prev - 1e-5 * abs(prev)
        prev = lb
        tot = torch.zeros(n, dtype=torch.float64, device=A.device)
        tot.index_add_(0, col, (A.to_csr(lam) + A.to_csr(M)).double())
        resid = (tot - c)[covered].abs().max().item()
        assert resid <= TOL_LAM * float(c.abs().max())
    m0, m1 = A.min_marginals(lam)
    lam_csr, m0c, m1c = _np(A.to_csr(lam)), _np(A.to_csr(m0)), _np(A.to_csr(m1))
    rng = np.random.default_rng(0)
    rows = rng.choice(len(prob["row_ptr"]) - 1, size=300, replace=False)
    cmax = np.abs(prob["c"]).max()
    for j in rows:
        b, e = prob["row_ptr"][j], prob["row_ptr"][j + 1]
        k = int(e - b)
        one = workloads.single_rows_problem([(np.arange(k), prob["coef"][b:e], int(prob["sense"][j]),
                                             int(prob["rhs"][j]))], k, np.zeros(k))
        o0, o1 = oracle.Oracle(one).min_marginals(lam_csr[b:e])
        assert np.abs(o0 - m0c[b:e]).max() <= TOL_LAM * cmax
        assert np.abs(o1 - m1c[b:e]).max() <= TOL_LAM * cmax


def test_min_marginals_energy_and_seed_vs_oracle():
    prob = workloads.matching_quadratic(L=60, R=60, pairs=3000, seed=9)
    O = oracle.Oracle(prob)
    A = _arena(prob)
    rng = np.random.default_rng(1)
    lam_c = rng.normal(size=O.num_slots)
    M_c = rng.normal(size=O.num_slots) * 0.1
    lam = A.from_csr(lam_c)
    M = A.from_csr(M_c)
    m0, m1 = A.min_marginals(lam)
    o0, o1 = O.min_marginals(_np(A.to_csr(lam)))
    np.testing.assert_allclose(_np(A.to_csr(m0)), o0, atol=1e-5 * 4)
    np.testing.assert_allclose(_np(A.to_csr(m1)), o1, atol=1e-5 * 4)
    lb, E = A.lower_bound(lam, M, energies=True)
    want, oE = O.lower_bound(_np(A.to_csr(lam)), _np(A.to_csr(M)), energies=True)
    np.testing.assert_allclose(_np(E), oE, atol=1e-5 * 4)
    assert abs(float(lb[0]) - want) <= 1e-5 * max(1.0, abs(want))
    gl, gM = A.lb_seed(lam, M)
    ol, oM = O.lb_seed(_np(A.to_csr(lam)), _np(A.to_csr(M)))
    np.testing.assert_array_equal(_np(A.to_csr(gl)), ol)
    np.testing.assert_array_equal(_np(A.to_csr(gM)), oM)


def test_layout_and_block_size_independent_bit_exact():
    """The arithmetic of every BDD does not depend on how BDDs are packed into
    tiles or on the CTA size: results are bit-identical."""
    prob = workloads.tracking(frames=6, dets=300, seed=4)
    outs = []
    for tn, ts, bt in [(2048, 1024, 256), (256, 128, 64), (8192, 4096, 512), (1024, 512, 128)]:
        A = _arena(prob, tile_nodes=tn, tile_slots=ts, block_threads=bt)
        lam, M = A.init_lambda()
        lb = A.iterate(lam, M, iters=7, lb=True)
        outs.append((_np(A.to_csr(lam)), _np(A.to_csr(M)), float(lb[0])))
    for o in outs[1:]:
        np.testing.assert_array_equal(o[0], outs[0][0])
        np.testing.assert_array_equal(o[1], outs[0][1])
        assert o[2] == outs[0][2]


def test_graph_replay_equals_iterate():
    prob = workloads.matching_quadratic(L=50, R=50, pairs=2500, seed=2)
    A = _arena(prob)
    lam, M = A.init_lambda()
    lam2, M2 = lam.clone(), M.clone()
    lb_out = torch.zeros(1, dtype=torch.float64, device=A.device)
    g = A.graph(lam2, M2, iters=5, lb_out=lb_out)
    torch.cuda.synchronize()
    for _ in range(3):
        A.iterate(lam, M, iters=5)
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(lam, lam2) and torch.equal(M, M2)
    assert float(lb_out[0]) == float(A.lower_bound(lam, M)[0]) or abs(
        float(lb_out[0]) - float(A.lower_bound(lam, M)[0])) < 1e-9


def _wide_row(rng, lo_w=17, hi_w=32, amax=25, kmax=13):
    while True:
        k = int(rng.integers(8, kmax))
        a = rng.integers(1, amax, size=k)
        b = int(a.sum() // 2)
        try:
            O = oracle.Oracle(workloads.single_rows_problem([(np.arange(k), a, 0, b)], k, np.zeros(k)))
        except oracle.OracleError:
            continue
        ls, lo, _ = O.bdd(0)
        w = np.diff(ls).max()
        if lo_w <= w <= hi_w and len(lo) <= 254:
            return a, b


def test_edge_cases_vs_oracle():
    """Single-variable rows, a level of 17..32 nodes (full warp segment),
    uncovered variables, equality rows, and a ragged mix of lengths."""
    rng = np.random.default_rng(5)
    a, b = _wide_row(rng)
    k = len(a)
    rows = [(np.arange(k), a, 0, b),                      # wide knapsack level
            (np.array([k]), np.array([1]), 0, 1),           # single variable, x <= 1
            (np.array([k, k + 1, k + 2]), np.array([1, 1, -1]), 2, 0),
            (np.array([0, k + 3]), np.array([1, 1]), 1, 1)]
    n = k + 6  # last two variables are in no row
    for _ in range(40):
        rows.append(workloads.random_rows(1, kmax=6, n=n - 2, seed=int(rng.integers(1 << 30)))[0])
    good = []
    for r in rows:
        try:
            oracle.Oracle(workloads.single_rows_problem([r], n, np.zeros(n)))
            good.append(r)
        except oracle.OracleError:
            pass
    prob = workloads.single_rows_problem(good, n, rng.normal(size=n))
    _check_iterations(prob, 1, 40)
    _check_iterations(prob, 1, 40, tile_nodes=64, tile_slots=32, block_threads=32)


def test_renorm_keeps_invariant_in_fp64():
    prob = workloads.independent_set(n=5000, seed=8)
    A = _arena(prob, renorm_every=1)
    lam, M = A.init_lambda()
    A.iterate(lam, M, iters=50)
    n = prob["n"]
    col = torch.as_tensor(prob["col"], dtype=torch.int64, device=A.device)
    tot = torch.zeros(n, dtype=torch.float64, device=A.device)
    tot.index_add_(0, col, A.to_csr(lam).double() + A.to_csr(M).double())
    c = torch.as_tensor(prob["c"], device=A.device)
    cov = torch.bincount(col, minlength=n) > 0
    assert (tot - c)[cov].abs().max().item() < 2e-6


def test_config4_full_batch_per_instance_bounds():
    """All 64 uneven instances of the batching configuration in one arena:
    lambda after one iteration and every instance's bound after 10."""
    prob, kinds = workloads.batched_mix(num=64)
    assert len(prob["inst_row_ptr"]) == 65
    _check_iterations(prob, 1, 10)


def test_batched_uncovered_variables_per_instance():
    """Variables that no row covers add min(0, c_i) to their own instance's
    bound only (Def. 2 with the unary term): three instances, uncovered
    variables of negative and positive cost in the first and last."""
    rng = np.random.default_rng(17)
    insts = []
    for k, extra in enumerate(((-3.0, 2.0), (), (0.5, -7.25, -1.0))):
        n0 = 12
        rows = []
        for r in workloads.random_rows(40, kmax=5, n=n0, seed=300 + k):
            try:
                oracle.Oracle(workloads.single_rows_problem([r], n0, np.zeros(n0)))
                rows.append(r)
            except oracle.OracleError:
                pass
        c = np.concatenate([rng.normal(size=n0), np.asarray(extra, dtype=np.float64)])
        insts.append(workloads.single_rows_problem(rows[:10], n0 + len(extra), c))
    prob = workloads.concat(insts)
    A, O, lam, M = _check_iterations(prob, 1, 30)
    got = A.lower_bound(lam, M).cpu().numpy()
    ol, oM = O.init_lambda()
    ol, oM = O.iterate(ol, oM, 0.5, None, 30)
    want = O.lower_bound(ol, oM, per_instance=True)[1]
    np.testing.assert_allclose(got, want, rtol=TOL_LB, atol=TOL_LB)


def test_resume_from_saved_state_is_bit_identical():
    """Solver resume: the arena is rebuilt from the rows and the saved (lambda,
    M) continue exactly where they stopped: 6 + 4 iterations through a second,
    independently planned arena equal 10 iterations in one call."""
    prob = workloads.independent_set(n=3000, seed=21)
    A = _arena(prob)
    lam, M = A.init_lambda()
    lb10 = A.iterate(lam, M, iters=10, lb=True)
    B = _arena(prob)
    l2, m2 = B.init_lambda()
    B.iterate(l2, m2, iters=6)
    saved = (l2.cpu(), m2.cpu())
    C = _arena(prob)
    l3, m3 = saved[0].to(C.device), saved[1].to(C.device)
    lb6_4 = C.iterate(l3, m3, iters=4, lb=True)
    assert torch.equal(l3, lam) and torch.equal(m3, M) and torch.equal(lb6_4, lb10)


def test_largest_bdd_and_widest_level_vs_oracle():
    """The largest BDD the layout takes (254 nodes, 30 levels of width up to
    15) next to levels of 17..32 and of more than 40 nodes and ordinary rows:
    lambda after one iteration and the bound after 60 against the oracle."""
    rng = np.random.default_rng(33)
    a, b = _wide_row(rng)
    k = len(a)
    a2, b2 = _wide_row(rng, lo_w=40, hi_w=128, amax=40, kmax=14)
    k2 = len(a2)
    n = 40
    rows = [(np.arange(30), np.ones(30, np.int64), 0, 14),     # 254 nodes
            (np.arange(k) + 20, a, 0, b),                        # level of 17..32 nodes
            (np.arange(k2) + 5, a2, 0, b2)]                      # level of more than 40 nodes
    for r in workloads.random_rows(60, kmax=6, n=n, seed=34):
        try:
            oracle.Oracle(workloads.single_rows_problem([r], n, np.zeros(n)))
            rows.append(r)
        except oracle.OracleError:
            pass
    prob = workloads.single_rows_problem(rows, n, rng.normal(size=n))
    assert len(solver.plan(prob).bdd(0)[1]) == 254
    _check_iterations(prob, 1, 60)


def test_problem_without_rows():
    """Zero rows: iterating is a no-op and the bound is sum_i min(0, c_i)."""
    c = np.array([1.0, -2, 3, -0.5, 0])
    prob = dict(n=5, row_ptr=np.zeros(1, np.int64), col=np.zeros(0, np.int32), coef=np.zeros(0, np.int32),
                sense=np.zeros(0, np.int8), rhs=np.zeros(0, np.int32), c=c)
    A = _arena(prob)
    lam, M = A.init_lambda()
    lb = A.iterate(lam, M, iters=3, lb=True)
    assert float(lb[0]) == float(np.minimum(c, 0).sum())
    assert float(A.lower_bound(lam, M)[0]) == float(np.minimum(c, 0).sum())


def test_degenerate_parameters():
    """omega = 0 moves nothing (M stays 0, so alpha S = 0 and lambda is
    unchanged bit for bit); with every variable in one row (alpha = 1) the
    bound at the initial split already equals the optimum and stays there."""
    prob = workloads.matching_quadratic(L=20, R=20, pairs=200, seed=41)
    A = _arena(prob)
    lam0, M0 = A.init_lambda()
    lam, M = lam0.clone(), M0.clone()
    omega = torch.zeros_like(lam)
    alpha = A.from_csr(1.0 / np.bincount(prob["col"], minlength=prob["n"])[prob["col"]])
    A.iterate(lam, M, omega, alpha, iters=5)
    assert torch.equal(lam, lam0) and torch.equal(M, M0)
    # disjoint rows: x_{2r} + x_{2r+1} <= 1 for r < 20, random costs
    rng = np.random.default_rng(42)
    rows = [(np.array([2 * r, 2 * r + 1]), np.array([1, 1]), 0, 1) for r in range(20)]
    c = rng.normal(size=40)
    dis = workloads.single_rows_problem(rows, 40, c)
    B = _arena(dis)
    l, m = B.init_lambda()
    opt = sum(min(0.0, c[2 * r], c[2 * r + 1]) for r in range(20))
    assert abs(float(B.lower_bound(l, m)[0]) - opt) < 1e-5
    lb = B.iterate(l, m, iters=10, lb=True)
    assert abs(float(lb[0]) - opt) < 1e-5
