"""dg_lower_bound_noalloc, the bound for callers that cannot give libdg
scratch memory (see include/dg.h): through the C ABI it must return what
dg_lower_bound returns, on consecutive calls sharing the static array.

This file is collected last on purpose: it runs after every other test in a
full session, and also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

import workloads
from paper_2205_11638_gb300 import _lib, build, solver

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make", [lambda: workloads.matching_quadratic(L=80, R=80, pairs=4000, seed=11),
                                  lambda: workloads.long_rows_mix(seed=5)], ids=["tiles", "with_long_bdds"])
def test_noalloc_bound_matches_lower_bound_twice(make):
    build.build()
    lib = _lib.load()
    prob = make()
    A = solver.plan(prob).bind()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    lam, M = A.init_lambda()
    for call in range(2):
        A.iterate(lam, M, iters=3 + call)
        want = A.lower_bound(lam, M)
        got = torch.full((A.num_inst,), float("nan"), dtype=torch.float64, device=A.device)
        st = lib.dg_lower_bound_noalloc(A._h, stream, ctypes.c_void_p(lam.data_ptr()),
                                        ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(got.data_ptr()))
        assert st == _lib.DG_OK, lib.dg_last_error()
        torch.cuda.synchronize()
        w, g = want.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.abs(g - w) <= 1e-5 * np.maximum(1.0, np.abs(w))), (call, g, w)


def test_noalloc_bound_captured_in_a_cuda_graph():
    # the reason for the entry point: a bound inside a stream capture (after a
    # first eager call has looked up the static array), replayed later
    build.build()
    lib = _lib.load()
    prob = workloads.matching_quadratic(L=60, R=60, pairs=2500, seed=12)
    A = solver.plan(prob).bind()
    lam, M = A.init_lambda()
    A.iterate(lam, M, iters=2)
    out = torch.zeros(A.num_inst, dtype=torch.float64, device=A.device)
    args = [ctypes.c_void_p(t.data_ptr()) for t in (lam, M, out)]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        st = lib.dg_lower_bound_noalloc(A._h, ctypes.c_void_p(side.cuda_stream), *args)  # eager first call
        assert st == _lib.DG_OK, lib.dg_last_error()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            st = lib.dg_lower_bound_noalloc(A._h, ctypes.c_void_p(side.cuda_stream), *args)
        assert st == _lib.DG_OK, lib.dg_last_error()
    torch.cuda.current_stream().wait_stream(side)
    for k in range(2):
        A.iterate(lam, M, iters=1)   # new state; the graph reads the same buffers
        out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        want = A.lower_bound(lam, M).cpu().numpy()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - want) <= 1e-5 * np.maximum(1.0, np.abs(want))), (k, got, want)


def test_noalloc_rejects_arena_beyond_static_limit():
    build.build()
    lib = _lib.load()
    prob = workloads.independent_set(n=400_000, avg_deg=4.0, seed=3)  # 4 m + 8 n > 4 MiB
    A = solver.plan(prob).bind()
    lam, M = A.init_lambda()
    out = torch.zeros(A.num_inst, dtype=torch.float64, device=A.device)
    st = lib.dg_lower_bound_noalloc(A._h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                    ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(M.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()))
    assert st == _lib.DG_EINVAL
    assert b"static array" in lib.dg_last_error()
