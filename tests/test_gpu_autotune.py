"""The autotuner changes launch shapes and the layout of tiles, never the
arithmetic of a BDD: tuned and untuned arenas give bit-identical results; the
layout search caches its choice per (GPU, problem statistics)."""
import json

import pytest
import torch

import workloads
from paper_2205_11638_gb300 import autotune, build, solver

pytestmark = pytest.mark.gpu


def _run(A, iters=6):
    lam, M = A.init_lambda()
    lb = A.iterate(lam, M, iters=iters, lb=True)
    return A.to_csr(lam), A.to_csr(M), float(lb[0])


def test_launch_tuning_keeps_results_bit_identical():
    build.build()
    prob = workloads.tracking(frames=8, dets=400, seed=2)
    A = solver.plan(prob).bind()
    ref = _run(A)
    ms = autotune.tune_launch(A, reps=2)
    assert ms > 0
    got = _run(A)
    assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1]) and ref[2] == got[2]


def test_layout_search_and_cache(tmp_path, monkeypatch):
    build.build()
    monkeypatch.setenv("DG_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    prob = workloads.matching_quadratic(L=60, R=60, pairs=3000, seed=4)
    ref = _run(solver.plan(prob).bind())
    opts, A = autotune.tune(prob, reps=2, chunks=(1024, 16384), ratios=(60, 90))
    got = _run(A)
    assert torch.equal(ref[0], got[0]) and ref[2] == got[2]
    cache = json.load(open(tmp_path / "cache.json"))
    assert len(cache) == 1 and list(cache.values())[0]["options"] == opts
    opts2, _ = autotune.tune(prob, reps=1)
    assert opts2 == opts
