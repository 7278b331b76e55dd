"""Seeded synthetic binary programs shaped like DOGE-Train's workloads.

This module only draws random instances; it contains none of the solver's
arithmetic and is shared by the oracle's tests, the CUDA path's tests, the
smoke check and ``bench.py``.

The paper's datasets (Sec. 4.2: cell tracking, graph matching, independent
set, QAPLib) are not available, so these generators stand in for them with
the sizes and value distributions of the benchmark configurations:

* :func:`set_cover`       -- tiny random set cover (brute-force checkable)
* :func:`independent_set` -- Erdos-Renyi graph, one ``x_u + x_v <= 1`` per edge
* :func:`matching_quadratic` -- assignment rows plus linearised quadratic terms
* :func:`batched_mix`     -- many uneven instances of the three kinds above
* :func:`tracking`        -- frames of detections joined by flow constraints

Every instance is a dict of CSR arrays: ``n``, ``row_ptr`` (int64[m+1]),
``col`` (int32, strictly ascending within a row), ``coef`` (int32), ``sense``
(int8: 0 ``<=``, 1 ``>=``, 2 ``=``), ``rhs`` (int32), ``c`` (float64[n]), and
for batches ``inst_row_ptr`` / ``inst_var_ptr``.
"""
from __future__ import annotations

import numpy as np

LE, GE, EQ = 0, 1, 2
BASE_SEED = 20221205


def _pack(n, rows_vars, rows_coef, sense, rhs, c):
    """Packs python lists of per-row (vars, coefs) into sorted CSR arrays."""
    row_ptr = np.zeros(len(rows_vars) + 1, np.int64)
    cols, coefs = [], []
    for j, (v, a) in enumerate(zip(rows_vars, rows_coef)):
        v = np.asarray(v, np.int64)
        a = np.asarray(a, np.int64)
        o = np.argsort(v, kind="stable")
        cols.append(v[o])
        coefs.append(a[o])
        row_ptr[j + 1] = row_ptr[j] + len(v)
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    coef = np.concatenate(coefs).astype(np.int32) if coefs else np.zeros(0, np.int32)
    return dict(n=int(n), row_ptr=row_ptr, col=col, coef=coef,
                sense=np.asarray(sense, np.int8), rhs=np.asarray(rhs, np.int32),
                c=np.asarray(c, np.float64))


def _csr_from_flat(n, row_of, var, coef, sense, rhs, c):
    """Vectorised CSR assembly: entries (row_of, var, coef) in any order."""
    order = np.lexsort((var, row_of))
    row_of = row_of[order]
    m = len(sense)
    counts = np.bincount(row_of, minlength=m)
    row_ptr = np.zeros(m + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return dict(n=int(n), row_ptr=row_ptr, col=var[order].astype(np.int32),
                coef=coef[order].astype(np.int32), sense=np.asarray(sense, np.int8),
                rhs=np.asarray(rhs, np.int32), c=np.asarray(c, np.float64))


def set_cover(n=24, m=16, kmin=3, kmax=8, seed=BASE_SEED + 1, cmin=1.0, cmax=10.0):
    """Random set cover: rows sum_{j in S_i} x_j >= 1, |S_i| ~ U{kmin..kmax} drawn
    without replacement, costs c ~ U[cmin, cmax]."""
    rng = np.random.default_rng(seed)
    rows_v, rows_a = [], []
    for _ in range(m):
        k = int(rng.integers(kmin, kmax + 1))
        v = rng.choice(n, size=k, replace=False)
        rows_v.append(v)
        rows_a.append(np.ones(k, np.int64))
    c = rng.uniform(cmin, cmax, size=n)
    return _pack(n, rows_v, rows_a, [GE] * m, [1] * m, c)


def _er_edges(n, avg_deg, rng):
    p = avg_deg / (n - 1)
    npairs = n * (n - 1) // 2
    ne = int(rng.binomial(npairs, p))
    seen = np.zeros(0, np.int64)
    while len(seen) < ne:
        need = ne - len(seen)
        u = rng.integers(0, n, size=2 * need + 16)
        v = rng.integers(0, n, size=2 * need + 16)
        keep = u != v
        a = np.minimum(u[keep], v[keep]).astype(np.int64)
        b = np.maximum(u[keep], v[keep]).astype(np.int64)
        key = a * n + b
        seen = np.unique(np.concatenate([seen, key]))
    if len(seen) > ne:
        seen = rng.permutation(seen)[:ne]
        seen.sort()
    return (seen // n).astype(np.int64), (seen % n).astype(np.int64)


def independent_set(n=10_000, avg_deg=8.0, seed=BASE_SEED + 2):
    """Independent set on G(n, p = avg_deg/(n-1)): one row x_u + x_v <= 1 per
    edge, costs c = -w with w ~ U[0, 1]."""
    rng = np.random.default_rng(seed)
    u, v = _er_edges(n, avg_deg, rng)
    m = len(u)
    row_of = np.repeat(np.arange(m), 2)
    var = np.stack([u, v], 1).reshape(-1)
    coef = np.ones(2 * m, np.int64)
    c = -rng.uniform(0.0, 1.0, size=n)
    return _csr_from_flat(n, row_of, var, coef, np.full(m, LE), np.ones(m), c)


def matching_quadratic(L=200, R=200, cand=10, pairs=20_000, seed=BASE_SEED + 3, sigma_y=0.5):
    """Graph matching with linearised quadratic terms.

    Each left node picks ``cand`` distinct right nodes: one assignment variable
    x per pick with cost N(0,1).  Rows: sum over a left node's x <= 1 and sum
    over a right node's x <= 1.  ``pairs`` distinct unordered pairs (a, b) of x
    variables each get an auxiliary y_ab with cost N(0, sigma_y^2) and rows
    y <= x_a, y <= x_b, y >= x_a + x_b - 1."""
    rng = np.random.default_rng(seed)
    right = np.stack([rng.choice(R, size=cand, replace=False) for _ in range(L)])  # [L, cand]
    nx = L * cand
    cx = rng.normal(0.0, 1.0, size=nx)
    npair_max = nx * (nx - 1) // 2
    pairs = min(pairs, npair_max)
    keys = np.zeros(0, np.int64)
    while len(keys) < pairs:
        need = pairs - len(keys)
        a = rng.integers(0, nx, size=2 * need + 16)
        b = rng.integers(0, nx, size=2 * need + 16)
        keep = a != b
        lo = np.minimum(a[keep], b[keep]).astype(np.int64)
        hi = np.maximum(a[keep], b[keep]).astype(np.int64)
        keys = np.unique(np.concatenate([keys, lo * nx + hi]))
    if len(keys) > pairs:
        keys = np.sort(rng.permutation(keys)[:pairs])
    pa, pb = keys // nx, keys % nx
    cy = rng.normal(0.0, sigma_y, size=pairs)
    n = nx + pairs
    row_of, var, coef, sense, rhs = [], [], [], [], []
    r = 0
    xid = np.arange(nx).reshape(L, cand)
    for a in range(L):                       # sum of a left node's x <= 1
        row_of.append(np.full(cand, r)); var.append(xid[a]); coef.append(np.ones(cand, np.int64))
        sense.append(LE); rhs.append(1); r += 1
    flat_right = right.reshape(-1)
    for b in range(R):                       # sum of a right node's x <= 1
        xs = np.nonzero(flat_right == b)[0]
        if len(xs) == 0:
            continue
        row_of.append(np.full(len(xs), r)); var.append(xs); coef.append(np.ones(len(xs), np.int64))
        sense.append(LE); rhs.append(1); r += 1
    # per pair p, rows r+3p: y - x_a <= 0, r+3p+1: y - x_b <= 0, r+3p+2: x_a + x_b - y <= 1
    y = nx + np.arange(pairs)
    r1 = r + 3 * np.arange(pairs)
    row_of += [np.repeat(r1, 2), np.repeat(r1 + 1, 2), np.repeat(r1 + 2, 3)]
    var += [np.stack([pa, y], 1).reshape(-1), np.stack([pb, y], 1).reshape(-1),
            np.stack([pa, pb, y], 1).reshape(-1)]
    coef += [np.tile([-1, 1], pairs), np.tile([-1, 1], pairs), np.tile([1, 1, -1], pairs)]
    sense_arr = np.concatenate([np.array(sense, np.int64), np.full(3 * pairs, LE)])
    rhs_arr = np.concatenate([np.array(rhs, np.int64), np.tile([0, 0, 1], pairs)])
    c = np.concatenate([cx, cy])
    return _csr_from_flat(n, np.concatenate(row_of).astype(np.int64), np.concatenate(var).astype(np.int64),
                          np.concatenate(coef).astype(np.int64), sense_arr, rhs_arr, c)


def tracking(frames=500, dets=2000, cand=4, seed=BASE_SEED + 5):
    """Tracking-like flow instance.

    Every detection in frames 0..frames-2 has ``cand`` distinct random target
    detections in the next frame (edge variables, cost N(0,1)); every detection
    has an appearance and a disappearance variable.  Rows per detection:
    sum(in) <= 1, sum(out) <= 1 and sum(in) + appear - sum(out) - disappear = 0
    (rows with an empty sum are dropped).  The detection cost c_d ~ U[-2, 0] is
    put on the appearance variable and on every incoming edge, so that a
    detection pays it once whenever it is active.

    Variable ids are laid out frame by frame: appear and disappear variables of
    frame f, then the edges leaving frame f."""
    rng = np.random.default_rng(seed)
    F, D, K = frames, dets, cand
    assert D >= K and F >= 2
    cd = rng.uniform(-2.0, 0.0, size=(F, D))
    targets = np.empty((F - 1, D, K), np.int64)
    for f in range(F - 1):
        t = rng.integers(0, D, size=(D, K))
        for _ in range(64):
            s = np.sort(t, axis=1)
            dup = (s[:, 1:] == s[:, :-1]).any(axis=1)
            if not dup.any():
                break
            t[dup] = rng.integers(0, D, size=(int(dup.sum()), K))
        else:
            for d in np.nonzero(dup)[0]:
                t[d] = rng.choice(D, size=K, replace=False)
        targets[f] = t
    block = 2 * D + K * D          # variables of one frame with outgoing edges
    n = (F - 1) * block + 2 * D
    c = np.zeros(n)
    fi, di = np.meshgrid(np.arange(F), np.arange(D), indexing="ij")
    c[fi * block + di] = cd                                   # appear
    f3 = np.arange(F - 1)[:, None, None]
    d3 = np.arange(D)[None, :, None]
    k3 = np.arange(K)[None, None, :]
    eid = f3 * block + 2 * D + d3 * K + k3
    c[eid] = rng.normal(0.0, 1.0, size=(F - 1, D, K)) + cd[f3 + 1, targets]
    tgt_det = ((f3 + 1) * D + targets).reshape(-1)
    src_det = np.broadcast_to(f3 * D + d3, (F - 1, D, K)).reshape(-1)
    eid = eid.reshape(-1)
    ndet = F * D
    has_in = np.bincount(tgt_det, minlength=ndet) > 0
    has_out = np.bincount(src_det, minlength=ndet) > 0
    per = has_in.astype(np.int64) + has_out.astype(np.int64) + 1   # rows per detection
    start = np.zeros(ndet, np.int64)
    np.cumsum(per[:-1], out=start[1:])
    in_row = start
    out_row = start + has_in
    flow_row = start + has_in + has_out
    m = int(per.sum())
    sense = np.full(m, LE, np.int8)
    rhs = np.ones(m, np.int32)
    sense[flow_row] = EQ
    rhs[flow_row] = 0
    alld = np.arange(ndet)
    a_var = (alld // D) * block + alld % D
    z_var = a_var + D
    ne = len(eid)
    row_of = np.concatenate([in_row[tgt_det], out_row[src_det], flow_row[tgt_det], flow_row[src_det],
                             flow_row, flow_row])
    var = np.concatenate([eid, eid, eid, eid, a_var, z_var])
    coef = np.concatenate([np.ones(ne), np.ones(ne), np.ones(ne), -np.ones(ne),
                           np.ones(ndet), -np.ones(ndet)]).astype(np.int64)
    return _csr_from_flat(n, row_of, var.astype(np.int64), coef, sense, rhs, c)


def concat(instances):
    """Packs several instances into one batched problem (variables and rows
    renumbered, instance boundaries in inst_row_ptr / inst_var_ptr)."""
    ns = [int(x["n"]) for x in instances]
    ms = [len(x["row_ptr"]) - 1 for x in instances]
    var_off = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    row_off = np.concatenate([[0], np.cumsum(ms)]).astype(np.int64)
    nnz_off = np.concatenate([[0], np.cumsum([x["row_ptr"][-1] for x in instances])]).astype(np.int64)
    row_ptr = np.concatenate([[0]] + [x["row_ptr"][1:] + nnz_off[k] for k, x in enumerate(instances)])
    col = np.concatenate([x["col"].astype(np.int64) + var_off[k] for k, x in enumerate(instances)])
    return dict(n=int(var_off[-1]), row_ptr=row_ptr.astype(np.int64), col=col.astype(np.int32),
                coef=np.concatenate([x["coef"] for x in instances]).astype(np.int32),
                sense=np.concatenate([x["sense"] for x in instances]).astype(np.int8),
                rhs=np.concatenate([x["rhs"] for x in instances]).astype(np.int32),
                c=np.concatenate([x["c"] for x in instances]),
                inst_row_ptr=row_off, inst_var_ptr=var_off.astype(np.int32))


def batched_mix(num=64, seed=BASE_SEED + 4, scale=1.0):
    """``num`` instances of uneven size, kind drawn uniformly: independent set
    (n ~ U[1k, 50k], average degree 8), set cover (n ~ U[500, 20k], m = n/2,
    |S| ~ U{3..12}) and matching (L = R ~ U[50, 300], 10 candidates per left
    node, 100*L quadratic pairs).  Instance k draws from seed + 1000*k.
    ``scale`` shrinks every size (tests use small scales)."""
    rng = np.random.default_rng(seed)
    kinds = rng.integers(0, 3, size=num)
    out = []
    for k in range(num):
        s = seed + 1000 * k
        r = np.random.default_rng(s)
        if kinds[k] == 0:
            n = max(16, int(r.integers(1000, 50_001) * scale))
            out.append(independent_set(n=n, avg_deg=8.0, seed=s))
        elif kinds[k] == 1:
            n = max(16, int(r.integers(500, 20_001) * scale))
            out.append(set_cover(n=n, m=max(1, n // 2), kmin=3, kmax=12, seed=s))
        else:
            Lr = max(12, int(r.integers(50, 301) * scale))
            out.append(matching_quadratic(L=Lr, R=Lr, cand=10, pairs=100 * Lr, seed=s))
    return concat(out), kinds


def random_rows(num, kmax=14, n=None, amax=3, seed=0, allow_eq=True):
    """Random integer rows for the oracle's pins: k ~ U{1..kmax} distinct
    variables, coefficients in [-amax, amax], random sense and a right-hand side
    drawn inside the reachable range.  Returns a list of (vars, coefs, sense,
    rhs); rows may be infeasible or force a variable -- callers filter."""
    rng = np.random.default_rng(seed)
    n = n or kmax
    rows = []
    for _ in range(num):
        k = int(rng.integers(1, kmax + 1))
        v = np.sort(rng.choice(n, size=k, replace=False))
        a = rng.integers(-amax, amax + 1, size=k)
        lo = int(np.minimum(a, 0).sum())
        hi = int(np.maximum(a, 0).sum())
        sense = int(rng.integers(0, 3 if allow_eq else 2))
        b = int(rng.integers(lo, hi + 1))
        rows.append((v, a, sense, b))
    return rows


def _free_row(row):
    """True if every variable of a short row takes both values in some
    feasible assignment (enumeration of its 2^k assignments)."""
    _, a, sense, b = row
    a = np.asarray(a, np.int64)
    k = len(a)
    x = (np.arange(1 << k)[:, None] >> np.arange(k)[None, :]) & 1
    act = x @ a
    ok = act <= b if sense == LE else (act >= b if sense == GE else act == b)
    if not ok.any():
        return False
    feas = x[ok]
    return bool(np.all(feas.min(axis=0) == 0) and np.all(feas.max(axis=0) == 1))


def long_rows_mix(seed=BASE_SEED + 6, n_short=40):
    """Rows whose BDDs are too large for a tile lane, mixed with short ones:
    cardinality rows over 500 variables (sum <= 1, sum <= 10, sum = 25),
    sum >= 1 over 300 variables, a knapsack row sum_i i * x_i <= 200 over 30
    variables (a level of more than 128 nodes), and random short rows over
    the first 40 variables.  Costs N(0, 1)."""
    rng = np.random.default_rng(seed)
    n = 700
    rows = [(np.sort(rng.choice(n, size=500, replace=False)), np.ones(500, np.int64), LE, 1),
            (np.sort(rng.choice(n, size=500, replace=False)), np.ones(500, np.int64), LE, 10),
            (np.sort(rng.choice(n, size=500, replace=False)), np.ones(500, np.int64), EQ, 25),
            (np.sort(rng.choice(n, size=300, replace=False)), np.ones(300, np.int64), GE, 1),
            (np.arange(600, 630), np.arange(1, 31), LE, 200)]
    short = []
    for r in random_rows(8 * n_short, kmax=6, n=40, seed=seed + 1):
        if _free_row(r):
            short.append(r)
        if len(short) == n_short:
            break
    return single_rows_problem(rows + short, n, rng.normal(size=n))


def assignment(L=2000, R=2000, cand=300, seed=BASE_SEED + 7):
    """Sparse assignment (graph-matching-like) instance with long rows: every
    left node has ``cand`` distinct random right candidates (variable x_lr,
    cost N(0, 1)); rows sum_r x_lr <= 1 per left node and sum_l x_lr <= 1 per
    right node (about ``cand`` variables each)."""
    rng = np.random.default_rng(seed)
    rights = np.stack([np.sort(rng.choice(R, size=cand, replace=False)) for _ in range(L)])
    n = L * cand
    var = np.arange(n, dtype=np.int64)
    left = np.repeat(np.arange(L), cand)
    right = rights.reshape(-1)
    row_of = np.concatenate([left, L + right])
    vv = np.concatenate([var, var])
    m = L + R
    sense = np.full(m, LE, np.int8)
    rhs = np.ones(m, np.int32)
    keep = np.bincount(row_of, minlength=m) > 0
    remap = np.cumsum(keep) - 1
    return _csr_from_flat(n, remap[row_of], vv, np.ones(len(vv), np.int64), sense[keep], rhs[keep],
                          rng.normal(size=n))


def single_rows_problem(rows, n, c):
    """One problem from a list of (vars, coefs, sense, rhs) rows."""
    return _pack(n, [r[0] for r in rows], [r[1] for r in rows], [r[2] for r in rows],
                 [r[3] for r in rows], c)


CONFIGS = {
    "set_cover_24": lambda: set_cover(),
    "independent_set_10k": lambda: independent_set(),
    "matching_quadratic_200": lambda: matching_quadratic(),
    "batched_mix_64": lambda: batched_mix()[0],
    "tracking_500x2000": lambda: tracking(),
    "assignment_2000x300": lambda: assignment(),
}
