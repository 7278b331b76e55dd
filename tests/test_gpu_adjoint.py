"""GPU adjoint (Alg. 2, dg_backward) against the FP64 oracle's Alg. 2, the
dense PyTorch autograd reference, and itself under different checkpoint
intervals.

Tolerance: float32 kernels against float64 references, 1e-4 absolute on
gradients of O(1) magnitude for unrolls of up to 3 iterations on tie-free
inputs.  Long unrolls (20 iterations of the matching instance) also cross
near-ties whose float32 and float64 argmins differ; there the bar is a
relative L2 error below 1e-3 with at least 99% of the entries within 1e-4:
a near-tie whose winner differs between the two precisions legitimately
routes a gradient term along another path."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_2205_11638_gb300 import build, solver
from paper_2205_11638_gb300.solver import DualIterate, LowerBound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _np(t):
    return t.detach().double().cpu().numpy()


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


def _params(O, seed):
    rng = np.random.default_rng(seed)
    lam = rng.normal(size=O.num_slots)
    M = 0.3 * rng.normal(size=O.num_slots)
    omega = rng.uniform(0.2, 0.8, O.num_slots)
    alpha = rng.uniform(0.1, 1.0, O.num_slots)
    s = np.zeros(O.n)
    np.add.at(s, O.col, alpha)
    return lam, M, omega, alpha / s[O.col]


@pytest.mark.parametrize("seed,iters", [(1, 1), (2, 2), (3, 3), (4, 2)])
def test_gpu_adjoint_vs_oracle_tiny(seed, iters):
    prob = _tiny(seed)
    O = oracle.Oracle(prob)
    A = solver.plan(prob).bind()
    lam, M, omega, alpha = _params(O, seed)
    # float32 round trip so that both sides start from the same values
    lam, M, omega, alpha = (np.float32(x).astype(np.float64) for x in (lam, M, omega, alpha))
    rng = np.random.default_rng(100 + seed)
    a = np.float32(rng.normal(size=O.num_slots)).astype(np.float64)
    b = np.float32(rng.normal(size=O.num_slots)).astype(np.float64)
    want = O.backward(lam, M, omega, alpha, iters, a, b)
    t = [A.from_csr(x) for x in (lam, M, omega, alpha, a, b)]
    got = A.backward(t[0], t[1], t[2], t[3], iters, 2, t[4], t[5])
    for g, w in zip(got, want):
        np.testing.assert_allclose(_np(A.to_csr(g)), w, atol=1e-4, rtol=0)


def test_gpu_adjoint_plain_mode_vs_oracle():
    prob = _tiny(7)
    O = oracle.Oracle(prob)
    A = solver.plan(prob).bind()
    lam, M, _, _ = _params(O, 7)
    lam, M = np.float32(lam).astype(np.float64), np.float32(M).astype(np.float64)
    rng = np.random.default_rng(3)
    a = np.float32(rng.normal(size=O.num_slots)).astype(np.float64)
    b = np.float32(rng.normal(size=O.num_slots)).astype(np.float64)
    want = O.backward(lam, M, 0.5, None, 2, a, b)
    got = A.backward(A.from_csr(lam), A.from_csr(M), None, None, 2, 1, A.from_csr(a), A.from_csr(b))
    for g, w in zip(got, want):
        np.testing.assert_allclose(_np(A.to_csr(g)), w, atol=1e-4, rtol=0)


def test_gpu_adjoint_vs_dense_autograd():
    from tests import dense_ref
    prob = _tiny(11, n=10, rows=8, kmax=5)
    O = oracle.Oracle(prob)
    A = solver.plan(prob).bind()
    lam, M, omega, alpha = (np.float32(x).astype(np.float64) for x in _params(O, 11))
    t = [torch.tensor(x, dtype=torch.float64, requires_grad=True) for x in (lam, M, omega, alpha)]
    lT, MT = dense_ref.iterate(prob, *t, 2)
    dense_ref.lower_bound(prob, lT, MT).backward()
    lam_g, M_g, om_g, al_g = (A.from_csr(x) for x in (lam, M, omega, alpha))
    for x in (lam_g, M_g, om_g, al_g):
        x.requires_grad_(True)
    lT2, MT2 = DualIterate.apply(lam_g, M_g, om_g, al_g, A, 2, 1)
    LowerBound.apply(lT2, MT2, A).sum().backward()
    for mine, ref in zip((lam_g, M_g, om_g, al_g), t):
        np.testing.assert_allclose(_np(A.to_csr(mine.grad)), ref.grad.numpy(), atol=1e-4, rtol=0)


def test_checkpoint_interval_does_not_change_gradients():
    prob = workloads.matching_quadratic(L=40, R=40, pairs=1600, seed=5)
    A = solver.plan(prob).bind()
    lam, M = A.init_lambda()
    rng = np.random.default_rng(0)
    gl = A.from_csr(rng.normal(size=A.plan.sizes.num_lambda))
    gM = A.from_csr(rng.normal(size=A.plan.sizes.num_lambda))
    outs = [A.backward(lam, M, None, None, 6, ck, gl, gM) for ck in (1, 4, 6, 50)]
    for o in outs[1:]:
        for x, y in zip(o, outs[0]):
            assert torch.equal(x, y)


@pytest.mark.parametrize("with_long", [False, True])
def test_parameter_gradients_are_optional(with_long):
    # g_omega / g_alpha may be NULL: not computed, the other gradients unchanged
    prob = workloads.long_rows_mix(seed=41) if with_long else workloads.matching_quadratic(L=40, R=40, pairs=1600, seed=6)
    A = solver.plan(prob).bind()
    lam, M = A.init_lambda()
    rng = np.random.default_rng(1)
    nl = A.plan.sizes.num_lambda
    gl, gM = A.from_csr(rng.normal(size=nl)), A.from_csr(rng.normal(size=nl))
    om = A.from_csr(rng.uniform(0.2, 0.8, size=nl))
    al = A.from_csr(np.full(nl, 0.5))
    full = A.backward(lam, M, om, al, 4, 2, gl, gM)
    for keep in ((0, 1), (0, 1, 2), (0, 1, 3)):
        outs = [A.zeros() if k in keep else None for k in range(4)]
        A.backward_into(lam, M, om, al, 4, 2, gl, gM, outs)
        torch.cuda.synchronize()
        for k in keep:
            assert torch.equal(outs[k], full[k])


def test_config3_matching_20_unrolled_iterations_lb_loss():
    """Matching with linearised quadratic terms, per-slot omega (sigmoid) and
    alpha (softmax per variable), 20 unrolled iterations, gradient of the
    final lower bound, against the oracle."""
    prob = workloads.matching_quadratic()
    O = oracle.Oracle(prob)
    A = solver.plan(prob).bind()
    rng = np.random.default_rng(3)
    z = np.exp(rng.normal(size=O.num_slots))
    s = np.zeros(O.n)
    np.add.at(s, O.col, z)
    alpha = np.float32(z / s[O.col]).astype(np.float64)
    omega = np.float32(1.0 / (1.0 + np.exp(-rng.normal(size=O.num_slots)))).astype(np.float64)
    lam0, M0 = O.init_lambda()
    lam0 = np.float32(lam0).astype(np.float64)
    T = 20
    lT, MT = O.iterate(lam0, M0, omega, alpha, T)
    sl, sM = O.lb_seed(lT, MT)
    want = O.backward(lam0, M0, omega, alpha, T, sl, sM)
    lam_g, M_g, om_g, al_g = (A.from_csr(x) for x in (lam0, M0, omega, alpha))
    for x in (lam_g, M_g, om_g, al_g):
        x.requires_grad_(True)
    lT2, MT2 = DualIterate.apply(lam_g, M_g, om_g, al_g, A, T, 10)
    LowerBound.apply(lT2, MT2, A).sum().backward()
    for mine, w in zip((lam_g, M_g, om_g, al_g), want):
        g = _np(A.to_csr(mine.grad))
        rel = np.linalg.norm(g - w) / max(1e-12, np.linalg.norm(w))
        frac = np.mean(np.abs(g - w) <= 1e-4)
        assert rel < 1e-3 and frac >= 0.99, (rel, frac)


@pytest.mark.parametrize("per_slot", [False, True])
def test_checkpointed_forward_and_backward_are_bit_identical(per_slot):
    """dg_iterate_checkpointed leaves (lam, M, bound) exactly as dg_iterate,
    and dg_backward_checkpointed from its checkpoints gives exactly
    dg_backward's gradients (the same kernels in the same order)."""
    prob = workloads.matching_quadratic(L=40, R=40, pairs=1600, seed=9)
    A = solver.plan(prob).bind()
    lam0, M0 = A.init_lambda()
    rng = np.random.default_rng(4)
    om = al = None
    if per_slot:
        col = prob["col"]
        z = np.exp(rng.normal(size=len(col)))
        s = np.zeros(prob["n"])
        np.add.at(s, col, z)
        al = A.from_csr(z / s[col])
        om = A.from_csr(1.0 / (1.0 + np.exp(-rng.normal(size=len(col)))))
    T, ck = 7, 3
    l1, m1 = lam0.clone(), M0.clone()
    lb1 = A.iterate(l1, m1, om, al, iters=T, lb=True)
    l2, m2 = lam0.clone(), M0.clone()
    ws, lb2 = A.iterate_checkpointed(l2, m2, om, al, iters=T, ckpt_every=ck, lb=True)
    assert torch.equal(l1, l2) and torch.equal(m1, m2) and torch.equal(lb1, lb2)
    gl = A.from_csr(rng.normal(size=A.plan.sizes.num_lambda))
    gM = A.from_csr(rng.normal(size=A.plan.sizes.num_lambda))
    want = A.backward(lam0, M0, om, al, T, ck, gl, gM)
    got = A.backward_checkpointed(om, al, T, ck, gl, gM, ws)
    for x, y in zip(got, want):
        assert torch.equal(x, y)


def test_checkpointed_forward_rejects_renorm():
    """The FP64 re-projection is not differentiated: both the checkpointing
    forward and dg_backward refuse options that ask for it."""
    prob = workloads.matching_quadratic(L=20, R=20, pairs=200, seed=2)
    A = solver.plan(prob, renorm_every=5).bind()
    lam, M = A.init_lambda()
    with pytest.raises(RuntimeError, match="re-projection"):
        A.iterate_checkpointed(lam, M, iters=3, ckpt_every=2)
    with pytest.raises(RuntimeError, match="re-projection"):
        A.backward(lam, M, None, None, 3, 2, A.zeros(), A.zeros())


@pytest.mark.parametrize("T,ck", [(0, 3), (2, 50), (5, 1)])
def test_checkpointed_edge_intervals(T, ck):
    """No iterations (gradients pass through, bound of the initial state), a
    checkpoint interval longer than the unroll, and one checkpoint per
    iteration: the checkpointed pair still equals dg_iterate + dg_backward."""
    prob = workloads.matching_quadratic(L=30, R=30, pairs=900, seed=12)
    A = solver.plan(prob).bind()
    lam0, M0 = A.init_lambda()
    l1, m1 = lam0.clone(), M0.clone()
    lb1 = A.iterate(l1, m1, iters=T, lb=True)
    l2, m2 = lam0.clone(), M0.clone()
    ws, lb2 = A.iterate_checkpointed(l2, m2, iters=T, ckpt_every=ck, lb=True)
    assert torch.equal(l1, l2) and torch.equal(m1, m2) and torch.equal(lb1, lb2)
    rng = np.random.default_rng(T + 10 * ck)
    gl = A.from_csr(rng.normal(size=A.plan.sizes.num_lambda))
    gM = A.from_csr(rng.normal(size=A.plan.sizes.num_lambda))
    want = A.backward(lam0, M0, None, None, T, ck, gl, gM)
    got = A.backward_checkpointed(None, None, T, ck, gl, gM, ws)
    for x, y in zip(got, want):
        assert torch.equal(x, y)
    if T == 0:
        assert torch.equal(got[0], gl) and torch.equal(got[1], gM)


def test_gpu_adjoint_wide_levels_vs_oracle():
    """Alg. 2 through BDDs with a level wider than a warp (a knapsack row with
    more than 40 nodes on one level) and the 30-level cardinality row at the
    node limit, next to ordinary rows; per-slot parameters, 2 iterations."""
    rng = np.random.default_rng(61)
    while True:
        k = int(rng.integers(8, 14))
        a = rng.integers(1, 40, size=k)
        b = int(a.sum() // 2)
        try:
            Ow = oracle.Oracle(workloads.single_rows_problem([(np.arange(k), a, 0, b)], k, np.zeros(k)))
        except oracle.OracleError:
            continue
        ls, lo, _ = Ow.bdd(0)
        if np.diff(ls).max() > 40 and len(lo) <= 254:
            break
    n = 36
    rows = [(np.arange(k) + 3, a, 0, b), (np.arange(30) + 6, np.ones(30, np.int64), 0, 14)]
    for r in workloads.random_rows(40, kmax=5, n=n, seed=62):
        try:
            oracle.Oracle(workloads.single_rows_problem([r], n, np.zeros(n)))
            rows.append(r)
        except oracle.OracleError:
            pass
    prob = workloads.single_rows_problem(rows, n, rng.normal(size=n))
    O = oracle.Oracle(prob)
    A = solver.plan(prob).bind()
    lam, M, omega, alpha = (np.float32(x).astype(np.float64) for x in _params(O, 63))
    a_ = np.float32(rng.normal(size=O.num_slots)).astype(np.float64)
    b_ = np.float32(rng.normal(size=O.num_slots)).astype(np.float64)
    want = O.backward(lam, M, omega, alpha, 2, a_, b_)
    t = [A.from_csr(x) for x in (lam, M, omega, alpha, a_, b_)]
    got = A.backward(t[0], t[1], t[2], t[3], 2, 1, t[4], t[5])
    for g, w in zip(got, want):
        np.testing.assert_allclose(_np(A.to_csr(g)), w, atol=1e-4, rtol=0)


def test_batched_adjoint_equals_per_instance():
    """Batching changes only which tile and lane a BDD lands on, never the
    arithmetic of a BDD or the order of a variable's sums: the gradients of a
    3-instance arena equal, bit for bit, those of each instance alone."""
    insts = [workloads.matching_quadratic(L=15, R=15, pairs=120, seed=71),
             workloads.independent_set(n=400, seed=72),
             workloads.set_cover(n=30, m=20, seed=73)]
    prob = workloads.concat(insts)
    T, ck = 3, 2
    A = solver.plan(prob).bind()
    rng = np.random.default_rng(74)
    ga = rng.normal(size=A.plan.sizes.num_lambda)
    gb = rng.normal(size=A.plan.sizes.num_lambda)
    lam0, M0 = A.init_lambda()
    outs = A.backward(lam0, M0, None, None, T, ck, A.from_csr(ga), A.from_csr(gb))
    batch = [_np(A.to_csr(o)) for o in outs]
    nnz0 = 0
    for inst in insts:
        B = solver.plan(inst).bind()
        nnz = B.plan.sizes.num_lambda
        l0, m0 = B.init_lambda()
        one = B.backward(l0, m0, None, None, T, ck, B.from_csr(ga[nnz0:nnz0 + nnz]), B.from_csr(gb[nnz0:nnz0 + nnz]))
        for x, y in zip(one, batch):
            assert np.array_equal(_np(B.to_csr(x)), y[nnz0:nnz0 + nnz])
        nnz0 += nnz


def test_forward_and_adjoint_replay_from_a_cuda_graph():
    """dg_iterate_checkpointed, dg_lb_seed and dg_backward_checkpointed only
    enqueue stream-ordered work (no host synchronisation, no allocation), so a
    whole DOGE training step's solver part can be captured once and
    replayed; the replay's gradients equal the eager ones bit for bit."""
    prob = workloads.matching_quadratic(L=30, R=30, pairs=900, seed=81)
    A = solver.plan(prob).bind()
    col, n = prob["col"], prob["n"]
    rng = np.random.default_rng(82)
    z = np.exp(rng.normal(size=len(col)))
    s = np.zeros(n)
    np.add.at(s, col, z)
    alpha = A.from_csr(z / s[col])
    omega = A.from_csr(1.0 / (1.0 + np.exp(-rng.normal(size=len(col)))))
    lam0, M0 = A.init_lambda()
    T, ck = 6, 4
    ws = torch.empty(A.backward_workspace_bytes(T, ck), dtype=torch.uint8, device=A.device)
    outs = [A.zeros() for _ in range(4)]
    gl, gM = A.zeros(), A.zeros()
    lam, M = lam0.clone(), M0.clone()

    def step():
        lam.copy_(lam0)
        M.copy_(M0)
        A.iterate_checkpointed(lam, M, omega, alpha, iters=T, ckpt_every=ck, workspace=ws)
        A.lb_seed_into(lam, M, gl, gM)
        A.backward_checkpointed(omega, alpha, T, ck, gl, gM, ws, outs)

    step()
    torch.cuda.synchronize()
    eager = [o.clone() for o in outs]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for o in outs:
        o.zero_()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(eager, outs):
        assert torch.equal(a, b)
