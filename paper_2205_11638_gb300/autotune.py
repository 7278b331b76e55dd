"""Autotuner of the arena layout and launch shapes.

Two levels:

* launch shapes (native, ``dg_autotune``): per launch group and sweep
  direction the CTA size (1, 2 or 4 warps), then the number of concurrent
  streams, each timed with CUDA events on the arena itself;
* layout (here): the locality chunk of the tile sort and the footprint ratio
  of the launch groups, each candidate planned, bound, launch-tuned and timed
  on whole sweeps.  The winner is cached per (GPU, problem statistics) in a
  JSON file (``$DG_AUTOTUNE_CACHE``, default ``~/.cache/dg_autotune.json``).

Tuning changes only how tiles are grouped and launched, never the arithmetic
of a BDD: results are bit-identical under every choice.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os

import numpy as np
import torch

from . import _lib, solver

CHUNKS = (4096, 16384, 65536)
RATIOS = (60, 75, 90)


def cache_path() -> str:
    return os.environ.get("DG_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "dg_autotune.json"))


def problem_key(rows: dict, device=None) -> str:
    """(GPU name, shape statistics of the instance) as a cache key."""
    rp = np.asarray(rows["row_ptr"])
    lens = np.diff(rp)
    hist = np.bincount(np.minimum(lens, 63), minlength=64)
    h = hashlib.sha256()
    h.update(np.asarray([rows["n"], len(rp) - 1, rp[-1]], np.int64).tobytes())
    h.update(hist.astype(np.int64).tobytes())
    h.update(np.asarray(rows["coef"][: min(4096, len(rows["coef"]))], np.int32).tobytes())
    name = torch.cuda.get_device_name(device) if torch.cuda.is_available() else "cpu"
    return f"{name}|{h.hexdigest()[:24]}"


def tune_launch(arena: "solver.Arena", reps: int = 5, stream=None) -> float:
    """dg_autotune on the arena (work buffers allocated here); returns the
    tuned milliseconds of one forward plus one backward sweep."""
    lam, M = arena.init_lambda(stream)
    ms = ctypes.c_float(0.0)
    _lib.check(_lib.load().dg_autotune(arena._h, solver._stream_handle(stream), solver._ptr(lam), solver._ptr(M),
                                       int(reps), ctypes.byref(ms)), "dg_autotune")
    return float(ms.value)


def tune(rows: dict, reps: int = 5, chunks=CHUNKS, ratios=RATIOS, use_cache: bool = True, **plan_opts):
    """Searches the layout knobs; returns (options dict, tuned arena)."""
    key = problem_key(rows)
    path = cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except Exception:
            cache = {}
    if use_cache and key in cache:
        opts = cache[key]["options"]
        A = solver.plan(rows, **plan_opts, **opts).bind()
        tune_launch(A, reps)
        return opts, A
    best = None
    for cr in chunks:
        for ratio in ratios:
            opts = dict(chunk_rows=cr, group_ratio_pct=ratio)
            A = solver.plan(rows, **plan_opts, **opts).bind()
            ms = tune_launch(A, reps)
            if best is None or ms < best[0]:
                best = (ms, opts, A)
            else:
                del A
    ms, opts, A = best
    if use_cache:
        cache[key] = {"options": opts, "sweep_pair_ms": ms}
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        json.dump(cache, open(tmp, "w"), indent=1)
        os.replace(tmp, path)
    return opts, A
