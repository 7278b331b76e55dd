"""Failure paths on the GPU that fault nothing: a bounded host wait that runs
out while work is still queued (DG_ETIMEOUT), then completes; invalid
arguments rejected before any launch."""
import pytest
import torch

import workloads
from paper_2205_11638_gb300 import _lib, build, solver

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_then_completes():
    build.build()
    A = solver.plan(workloads.tracking(frames=60, dets=1000)).bind()
    lam, M = A.init_lambda()
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        A.iterate(lam, M, iters=300, stream=s)       # tens of milliseconds of queued work
        assert solver.wait(s, timeout_ms=0) == _lib.DG_ETIMEOUT
        assert b"still running" in _lib.load().dg_last_error()
        assert solver.wait(s, timeout_ms=60_000) == _lib.DG_OK
    assert torch.isfinite(lam).all()


def test_invalid_arguments_rejected_before_launch():
    build.build()
    A = solver.plan(workloads.set_cover()).bind()
    lam, M = A.init_lambda()
    with pytest.raises((ValueError, _lib.DgError)):
        A.iterate(lam, M, omega=A.zeros(), alpha=None)  # mode 1 needs alpha
    off = torch.zeros(A.num_slots + 1, device=A.device)[1:]  # 4-byte aligned, not 16
    with pytest.raises(_lib.DgError) as e:
        A.iterate(off, M, iters=1)
    assert e.value.status == _lib.DG_EINVAL
