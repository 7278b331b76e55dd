"""Brute-force enumeration used to pin the oracle (pure numpy, no solver code).

Everything here enumerates assignments explicitly; nothing is shared with the
oracle or the CUDA path.
"""
from __future__ import annotations

import numpy as np


def assignments(k: int) -> np.ndarray:
    """All 2^k binary vectors as a [2^k, k] int8 array (bit h of the index = x_h)."""
    idx = np.arange(1 << k, dtype=np.int64)
    return ((idx[:, None] >> np.arange(k)) & 1).astype(np.int8)


def satisfies(act: np.ndarray, sense: int, rhs: int) -> np.ndarray:
    if sense == 0:
        return act <= rhs
    if sense == 1:
        return act >= rhs
    return act == rhs


def row_feasible(coefs, sense, rhs) -> np.ndarray:
    """Feasible assignments of one row, as a [F, k] int8 array."""
    X = assignments(len(coefs))
    act = X.astype(np.int64) @ np.asarray(coefs, np.int64)
    return X[satisfies(act, sense, rhs)]


def row_min_marginals(coefs, sense, rhs, lam):
    """min over feasible x with x_h = beta of <lam, x>, for every h and beta."""
    X = row_feasible(coefs, sense, rhs)
    val = X.astype(np.float64) @ np.asarray(lam, np.float64)
    k = len(coefs)
    m0 = np.full(k, np.inf)
    m1 = np.full(k, np.inf)
    for h in range(k):
        z = X[:, h] == 0
        if z.any():
            m0[h] = val[z].min()
        if (~z).any():
            m1[h] = val[~z].min()
    return m0, m1


def row_argmin(coefs, sense, rhs, lam, h=None, beta=None):
    """The unique minimiser (the caller guarantees no ties) of <lam, x> over
    the row's feasible set, optionally with x_h = beta."""
    X = row_feasible(coefs, sense, rhs)
    if h is not None:
        X = X[X[:, h] == beta]
    val = X.astype(np.float64) @ np.asarray(lam, np.float64)
    o = np.argsort(val, kind="stable")
    return X[o[0]], (val[o[1]] - val[o[0]]) if len(o) > 1 else np.inf


def bdd_paths(level_start, lo, hi) -> np.ndarray:
    """All root-to-top paths of an exported BDD as a [P, k] int8 array."""
    k = len(level_start) - 1
    out = []

    def walk(h, rank, prefix):
        v = level_start[h] + rank
        for beta, ch in ((0, lo[v]), (1, hi[v])):
            if ch == -2:
                continue
            if h == k - 1:
                if ch == -1:
                    out.append(prefix + [beta])
                continue
            walk(h + 1, ch, prefix + [beta])

    walk(0, 0, [])
    return np.array(out, np.int8).reshape(-1, k)


def problem_opt(P: dict, chunk_bits: int = 20):
    """min <c, x> over x in {0,1}^n satisfying every row (n <= 26)."""
    n = int(P["n"])
    assert n <= 26
    m = len(P["row_ptr"]) - 1
    A = np.zeros((m, n), np.int64)
    for j in range(m):
        s, e = P["row_ptr"][j], P["row_ptr"][j + 1]
        A[j, P["col"][s:e]] = P["coef"][s:e]
    best, arg = np.inf, None
    total = 1 << n
    step = 1 << min(chunk_bits, n)
    for base in range(0, total, step):
        idx = np.arange(base, min(base + step, total), dtype=np.int64)
        X = ((idx[:, None] >> np.arange(n)) & 1).astype(np.int8)
        act = X.astype(np.int64) @ A.T
        ok = np.ones(len(idx), bool)
        for j in range(m):
            ok &= satisfies(act[:, j], int(P["sense"][j]), int(P["rhs"][j]))
        if ok.any():
            val = X[ok].astype(np.float64) @ P["c"]
            q = int(np.argmin(val))
            if val[q] < best:
                best, arg = float(val[q]), X[ok][q]
    return best, arg
