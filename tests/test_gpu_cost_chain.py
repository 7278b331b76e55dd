"""Path costs handed from one sweep to the next (DG_SWEEP_COSTS_OUT /
DG_SWEEP_COSTS_IN, and dg_iterate's own hand-off): a sweep that reads SP(., T)
or SP(r, .) (App. B's two recursions) from the sweep before it instead of
recomputing them must give bit for bit the lambda and M of the sweep that
recomputes them, and the arena must refuse the hand-off whenever lambda may
have changed in between."""
import ctypes

import numpy as np
import pytest
import torch

import workloads
from paper_2205_11638_gb300 import _lib, build, solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _softmax_alpha(col, n, rng):
    e = np.exp(rng.normal(size=len(col)))
    s = np.zeros(n)
    np.add.at(s, col, e)
    return e / s[col]


def _mode1(prob, A, seed=3):
    rng = np.random.default_rng(seed)
    omega = rng.uniform(0.1, 0.9, size=len(prob["col"]))
    alpha = _softmax_alpha(prob["col"], len(prob["c"]), rng)
    return A.from_csr(omega), A.from_csr(alpha)


def _manual(A, lam, M, iters, om=None, al=None, handoff=True, renorm_every=0):
    """dg_iterate's schedule spelled out with dg_sum_M / dg_sweep."""
    A.sum_M(M, alpha=al)
    handed = False
    for it in range(iters):
        rn = renorm_every > 0 and (it + 1) % renorm_every == 0
        A.sweep(lam, M, forward=True, omega=om, alpha=al, costs_in=handoff and handed, costs_out=handoff)
        A.sum_M(M, alpha=al)
        A.sweep(lam, M, forward=False, omega=om, alpha=al, costs_in=handoff, costs_out=handoff and not rn)
        A.sum_M(M, lam=lam, alpha=al, renorm=rn)
        handed = not rn


def _free_random_rows(num, seed, n=500):
    rows = [r for r in workloads.random_rows(3 * num, kmax=12, n=n, seed=seed) if workloads._free_row(r)][:num]
    return workloads.single_rows_problem(rows, n, np.random.default_rng(seed).normal(size=n))


CASES = {
    "tracking_40x400": lambda: workloads.tracking(frames=40, dets=400, seed=31),
    "matching": lambda: workloads.matching_quadratic(L=60, R=60, pairs=3000, seed=32),
    "with_long_bdds": lambda: workloads.long_rows_mix(seed=33),
    "random_rows": lambda: _free_random_rows(2000, seed=34),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("mode", [0, 1])
def test_handed_on_costs_bit_identical(name, mode):
    prob = CASES[name]()
    A = solver.plan(prob).bind()
    om = al = None
    if mode == 1:
        om, al = _mode1(prob, A)
    lam0, M0 = A.init_lambda()
    outs = []
    for how in ("iterate", "handoff", "recompute"):
        lam, M = lam0.clone(), M0.clone()
        if how == "iterate":
            A.iterate(lam, M, om, al, iters=6)
        else:
            _manual(A, lam, M, 6, om, al, handoff=how == "handoff")
        torch.cuda.synchronize()
        assert torch.isfinite(lam).all() and torch.isfinite(M).all()
        outs.append((lam.cpu(), M.cpu()))
    for lam, M in outs[1:]:
        assert torch.equal(lam, outs[0][0]) and torch.equal(M, outs[0][1])


def test_renorm_iterations_bit_identical():
    prob = workloads.tracking(frames=30, dets=300, seed=35)
    A = solver.plan(prob, renorm_every=2).bind()
    lam0, M0 = A.init_lambda()
    lam, M = lam0.clone(), M0.clone()
    A.iterate(lam, M, iters=5)
    lam2, M2 = lam0.clone(), M0.clone()
    _manual(A, lam2, M2, 5, handoff=False, renorm_every=2)
    torch.cuda.synchronize()
    assert torch.equal(lam.cpu(), lam2.cpu()) and torch.equal(M.cpu(), M2.cpu())


def test_checkpoint_recompute_gradients_independent_of_interval():
    # the backward pass recomputes its checkpoints with plain sweeps that hand
    # their costs on; gradients must not depend on the checkpoint interval
    prob = workloads.tracking(frames=12, dets=200, seed=36)
    A = solver.plan(prob).bind()
    lam0, M0 = A.init_lambda()
    A.iterate(lam0, M0, iters=2)
    g = torch.randn(A.num_slots, device=A.device, generator=torch.Generator(A.device).manual_seed(7))
    g = g * (A.slot_instance() >= 0)
    om, al = _mode1(prob, A)
    res = []
    for ck in (1, 3, 8):
        out = A.backward(lam0, M0, om, al, iters=8, ckpt_every=ck, g_lamT=g, g_MT=torch.zeros_like(g))
        torch.cuda.synchronize()
        res.append([t.cpu() for t in out])
    for r in res[1:]:
        for a, b in zip(r, res[0]):
            assert torch.equal(a, b)


def test_costs_in_refused_without_a_matching_costs_out():
    prob = workloads.matching_quadratic(L=30, R=30, pairs=800, seed=37)
    A = solver.plan(prob).bind()
    lam, M = A.init_lambda()
    other = lam.clone()

    def refused(fn, what="DG_SWEEP_COSTS_IN"):
        with pytest.raises(_lib.DgError) as e:
            fn()
        assert what in str(e.value)

    A.sum_M(M)
    refused(lambda: A.sweep(lam, M, forward=False, costs_in=True))            # nothing handed on yet
    refused(lambda: A.sweep(lam, M, forward=True, costs_in=True))
    A.sweep(lam, M, forward=True, costs_out=True)
    refused(lambda: A.sweep(lam, M, forward=True, costs_in=True))             # same direction
    A.sweep(lam, M, forward=True, costs_out=True)
    refused(lambda: A.sweep(other, M, forward=False, costs_in=True))          # another lambda
    A.sweep(lam, M, forward=True, costs_out=True)
    A.sum_M(M, lam=lam, renorm=True)
    refused(lambda: A.sweep(lam, M, forward=False, costs_in=True))            # re-projected lambda
    A.sweep(lam, M, forward=True, costs_out=True)
    A.min_marginals(lam)
    refused(lambda: A.sweep(lam, M, forward=False, costs_in=True))            # another call in between
    A.sweep(lam, M, forward=True, costs_out=True)
    A.sweep(lam, M, forward=False)
    refused(lambda: A.sweep(lam, M, forward=False, costs_in=True))            # a backward sweep in between
    A.sweep(lam, M, forward=True, costs_out=True)
    A.sum_M(M)
    A.sweep(lam, M, forward=False, costs_in=True, costs_out=True)             # allowed
    A.sum_M(M)
    lb = torch.zeros(A.num_inst, dtype=torch.float64, device=A.device)
    A.bound_from_energies(lb)
    A.sweep(lam, M, forward=True, costs_in=True)                              # allowed
    torch.cuda.synchronize()
    assert torch.isfinite(lam).all()
    p = [ctypes.c_void_p(t.data_ptr()) for t in (lam, M)]
    st = _lib.load().dg_sweep(A._h, None, p[0], p[1], None, None, 0, 1, 8, None)  # unknown flag
    assert st == _lib.DG_EINVAL and b"unknown flag" in _lib.load().dg_last_error()


def test_sweep_mode_must_match_the_last_reduction():
    prob = workloads.matching_quadratic(L=30, R=30, pairs=800, seed=38)
    A = solver.plan(prob).bind()
    om, al = _mode1(prob, A)
    lam, M = A.init_lambda()
    A.sum_M(M)                                  # mode 0 averaging terms
    with pytest.raises(_lib.DgError) as e:
        A.sweep(lam, M, forward=True, omega=om, alpha=al)
    assert "mode" in str(e.value)
    A.sum_M(M, alpha=al)                        # mode 1
    A.sweep(lam, M, forward=True, omega=om, alpha=al)
    torch.cuda.synchronize()


def test_graph_replay_counts_as_a_call_on_the_arena():
    prob = workloads.matching_quadratic(L=30, R=30, pairs=800, seed=39)
    A = solver.plan(prob).bind()
    om, al = _mode1(prob, A)
    lam, M = A.init_lambda()
    lam_g, M_g = lam.clone(), M.clone()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = A.graph(lam_g, M_g, om, al, iters=2, stream=stream)   # a mode-1 iteration loop
    torch.cuda.synchronize()
    A.sum_M(M)
    A.sweep(lam, M, forward=True, costs_out=True)
    A.sum_M(M)
    g.replay()                                                    # rewrites the handed-on costs
    with pytest.raises(_lib.DgError) as e:
        A.sweep(lam, M, forward=False, costs_in=True)
    assert "DG_SWEEP_COSTS_IN" in str(e.value)
    with pytest.raises(_lib.DgError) as e:                        # its averaging terms are mode 1 now
        A.sweep(lam, M, forward=False)
    assert "mode" in str(e.value)
    A.sum_M(M)
    A.sweep(lam, M, forward=False)
    torch.cuda.synchronize()
    assert torch.isfinite(lam).all()
