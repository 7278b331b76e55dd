"""Long BDDs together with the other parts of the path: several instances of
uneven size in one arena, some with rows beyond a tile lane (per-instance
bounds against the FP64 oracle, Def. 2 with the unary term), the iteration
loop captured in a CUDA graph (replay equal to dg_iterate bit for bit), the
launch-shape autotuner (results unchanged), and the autograd functions over
an arena with long BDDs (against the oracle's Alg. 2)."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_2205_11638_gb300 import autotune, build, solver
from paper_2205_11638_gb300.solver import DualIterate, LowerBound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _batch():
    return workloads.concat([workloads.long_rows_mix(seed=21, n_short=30),
                             workloads.independent_set(n=800, seed=22),
                             workloads.assignment(L=300, R=300, cand=280, seed=23),
                             workloads.matching_quadratic(L=30, R=30, pairs=600, seed=24)])


def test_batched_arena_with_long_bdds_per_instance_bounds():
    prob = _batch()
    A = solver.plan(prob).bind()
    assert A.plan.sizes.num_long_bdds > 0 and A.num_inst == 4
    lam, M = A.init_lambda()
    lb = A.iterate(lam, M, iters=30, lb=True)
    O = oracle.Oracle(prob)
    ol, oM = O.init_lambda()
    ol, oM = O.iterate(ol, oM, 0.5, None, 30)
    want = O.lower_bound(ol, oM, per_instance=True)[1]
    rel = np.abs(lb.cpu().numpy() - want) / np.maximum(1.0, np.abs(want))
    assert rel.max() <= 1e-5, (lb, want)


def test_graph_replay_and_autotune_with_long_bdds():
    prob = workloads.long_rows_mix(seed=25, n_short=40)
    A = solver.plan(prob).bind()
    lam, M = A.init_lambda()
    lam2, M2 = lam.clone(), M.clone()
    stream = torch.cuda.Stream()
    lb = torch.zeros(1, dtype=torch.float64, device=A.device)
    with torch.cuda.stream(stream):
        g = A.graph(lam2, M2, iters=4, lb_out=lb, stream=stream)
    torch.cuda.synchronize()
    for _ in range(3):
        # both on the current stream: they share the arena's scratch
        A.iterate(lam, M, iters=4)
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(lam, lam2) and torch.equal(M, M2)
    # the autotuner changes launch shapes only
    B = solver.plan(prob).bind()
    autotune.tune_launch(B, reps=1)
    l3, m3 = B.init_lambda()
    B.iterate(l3, m3, iters=12)
    assert torch.equal(l3, lam) and torch.equal(m3, M)


def test_autograd_through_long_bdds_vs_oracle():
    prob = workloads.long_rows_mix(seed=26, n_short=20)
    O = oracle.Oracle(prob)
    A = solver.plan(prob).bind()
    rng = np.random.default_rng(5)
    f32 = lambda x: np.float32(x).astype(np.float64)  # noqa: E731
    lam0 = f32(rng.normal(size=O.num_slots))
    M0 = f32(0.2 * rng.normal(size=O.num_slots))
    omega = f32(rng.uniform(0.2, 0.8, O.num_slots))
    e = np.exp(rng.normal(size=O.num_slots))
    s = np.zeros(O.n)
    np.add.at(s, O.col, e)
    alpha = f32(e / s[O.col])
    T = 2
    lT, MT = O.iterate(lam0, M0, omega, alpha, T)
    sl, sM = O.lb_seed(lT, MT)
    want = O.backward(lam0, M0, omega, alpha, T, sl, sM)
    leaves = [A.from_csr(x) for x in (lam0, M0, omega, alpha)]
    for x in leaves:
        x.requires_grad_(True)
    lT2, MT2 = DualIterate.apply(*leaves, A, T, 1)
    LowerBound.apply(lT2, MT2, A).sum().backward()
    for x, w in zip(leaves, want):
        np.testing.assert_allclose(A.to_csr(x.grad).double().cpu().numpy(), w, atol=1e-4, rtol=0)
