"""CPU-side checks of libdg: the library loads and exports every function of
include/dg.h, and the host builder (dg_plan) produces the canonical BDDs the
oracle builds independently, bit for bit, with the documented status codes.
No kernel is launched here."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import workloads
from paper_2205_11638_gb300 import _lib, build, solver

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "dg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[A-Za-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol():
    lib = _lib.load()
    names = _declared_functions()
    assert len(names) >= 20
    for nm in names:
        assert hasattr(lib, nm), nm
    assert set(names) == set(_lib.SIGNATURES)


def test_struct_layouts(tmp_path):
    """The ctypes mirrors have the C layout of include/dg.h (sizes and offsets
    printed by a C program compiled against the header)."""
    src = tmp_path / "layout.c"
    src.write_text(
        "#include <stdio.h>\n#include <stddef.h>\n#include \"dg.h\"\n"
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(dg_rows), sizeof(dg_options),"
        " sizeof(dg_sizes), sizeof(dg_stats), offsetof(dg_rows, m), offsetof(dg_sizes, m),"
        " offsetof(dg_stats, hop_histogram)); return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(_lib.dg_rows), ctypes.sizeof(_lib.dg_options), ctypes.sizeof(_lib.dg_sizes),
            ctypes.sizeof(_lib.dg_stats), _lib.dg_rows.m.offset, _lib.dg_sizes.m.offset,
            _lib.dg_stats.hop_histogram.offset]
    assert got == want


@pytest.mark.parametrize("make", [lambda: workloads.set_cover(), lambda: workloads.independent_set(n=1500, seed=4),
                                  lambda: workloads.matching_quadratic(L=30, R=30, pairs=900, seed=5),
                                  lambda: workloads.tracking(frames=4, dets=40, seed=6),
                                  lambda: workloads.batched_mix(num=6, scale=0.01)[0]])
def test_plan_structure_bit_exact_vs_oracle(make):
    prob = make()
    P = solver.plan(prob)
    O = oracle.Oracle(prob)
    assert P.sizes.num_nodes == O.num_nodes
    assert P.sizes.num_lambda == O.num_slots
    for j in range(P.m):
        for a, b in zip(P.bdd(j), O.bdd(j)):
            np.testing.assert_array_equal(a, b)


def test_plan_random_rows_bit_exact():
    rows = []
    for r in workloads.random_rows(400, kmax=12, n=40, seed=77):
        try:
            oracle.Oracle(workloads.single_rows_problem([r], 40, np.zeros(40)))
        except oracle.OracleError:
            continue
        rows.append(r)
    prob = workloads.single_rows_problem(rows, 40, np.random.default_rng(0).normal(size=40))
    P = solver.plan(prob)
    O = oracle.Oracle(prob)
    for j in range(P.m):
        for a, b in zip(P.bdd(j), O.bdd(j)):
            np.testing.assert_array_equal(a, b)


def test_plan_wide_coefficient_rows_bit_exact():
    """Rows with coefficients in [-12, 12] (the builder clamps partial sums to
    the window where residual functions still differ) keep the oracle's BDDs,
    bit for bit, for every sense."""
    rows = []
    for r in workloads.random_rows(700, kmax=14, n=40, amax=12, seed=91):
        try:
            oracle.Oracle(workloads.single_rows_problem([r], 40, np.zeros(40)))
        except oracle.OracleError:
            continue
        rows.append(r)
    assert len({r[2] for r in rows}) == 3
    prob = workloads.single_rows_problem(rows, 40, np.zeros(40))
    P = solver.plan(prob)
    O = oracle.Oracle(prob)
    for j in range(P.m):
        for a, b in zip(P.bdd(j), O.bdd(j)):
            np.testing.assert_array_equal(a, b)
    P.validate()


def test_slot_map_is_permutation():
    prob = workloads.matching_quadratic(L=30, R=30, pairs=900, seed=5)
    P = solver.plan(prob, tile_nodes=256, tile_slots=128)
    sm = P.slot_to_csr
    real = sm[sm >= 0]
    assert sorted(real.tolist()) == list(range(len(prob["col"])))
    assert P.sizes.num_tiles > 10
    assert P.num_slots % 4 == 0


def _status_of(rows, n):
    try:
        solver.plan(workloads.single_rows_problem(rows, n, np.zeros(n)))
    except _lib.DgError as e:
        return e.status
    return 0


def test_status_codes():
    assert _status_of([(np.array([0, 1]), np.array([2, 2]), 2, 1)], 2) == _lib.DG_EINFEASIBLE
    assert _status_of([(np.array([0, 1]), np.array([1, 1]), 1, 2)], 2) == _lib.DG_EFORCED
    # more than 4096 variables in a row
    assert _status_of([(np.arange(4097), np.ones(4097, np.int64), 0, 1)], 4097) == _lib.DG_EINVAL
    bad = workloads.single_rows_problem([(np.array([0, 1]), np.array([1, 1]), 0, 1)], 2, np.zeros(2))
    bad["col"] = bad["col"][::-1].copy()
    with pytest.raises(_lib.DgError) as e:
        solver.plan(bad)
    assert e.value.status == _lib.DG_EINVAL
    empty = dict(n=2, row_ptr=np.array([0, 0]), col=np.zeros(0, np.int32), coef=np.zeros(0, np.int32),
                 sense=np.zeros(1, np.int8), rhs=np.zeros(1, np.int32), c=np.zeros(2))
    with pytest.raises(_lib.DgError) as e:
        solver.plan(empty)
    assert e.value.status == _lib.DG_EINVAL
    # lanes per narrow long BDD: 0 or a power of two up to 32
    ok = workloads.single_rows_problem([(np.array([0, 1]), np.array([1, 1]), 0, 1)], 2, np.zeros(2))
    for lanes in (3, 64, -2):
        with pytest.raises(_lib.DgError) as e:
            solver.plan(ok, long_lanes=lanes)
        assert e.value.status == _lib.DG_EINVAL and "long_lanes" in str(e.value)
    for lanes in (0, 1, 8, 32):
        solver.plan(ok, long_lanes=lanes).validate()


def _bit_exact(prob):
    P = solver.plan(prob)
    O = oracle.Oracle(prob)
    assert P.sizes.num_nodes == O.num_nodes
    for j in range(P.m):
        for a, b in zip(P.bdd(j), O.bdd(j)):
            np.testing.assert_array_equal(a, b)
    P.validate()
    return P


def test_bdd_size_limits_route_rows_to_the_long_layout():
    """A BDD of exactly 254 nodes (x_0 + ... + x_29 <= 14) fits a tile lane;
    one more node, or a level of more than 128 nodes, makes the row a long
    BDD (one warp per BDD) instead of an error.  Either way the structure is
    the oracle's, bit for bit, and the arena passes the validator."""
    ok = workloads.single_rows_problem([(np.arange(30), np.ones(30, np.int64), 0, 14)], 30, np.zeros(30))
    P = _bit_exact(ok)
    assert len(P.bdd(0)[1]) == 254 and P.sizes.num_long_bdds == 0
    big = workloads.single_rows_problem([(np.arange(60), np.ones(60, np.int64), 0, 30)], 60, np.zeros(60))
    P = _bit_exact(big)
    assert P.sizes.num_long_bdds == 1 and P.sizes.num_long_nodes == P.sizes.num_nodes > 254
    assert P.sizes.num_tiles == 0
    # a knapsack row with a level of 112 nodes and more than 254 in all
    a = np.array([28, 31, 45, 57, 3, 9, 49, 56, 15, 19, 52, 25, 17, 49, 16, 25])
    P = _bit_exact(workloads.single_rows_problem([(np.arange(16), a, 0, 248)], 16, np.zeros(16)))
    assert P.sizes.num_long_bdds == 1


def test_long_and_tile_rows_mixed_in_one_arena():
    """Cardinality rows over 500 variables, a knapsack row with a level wider
    than 128 nodes and ordinary short rows in one arena: every row keeps the
    oracle's BDD; the long BDDs' slots follow the tiles' and the slot map is
    a permutation of the CSR positions."""
    prob = workloads.long_rows_mix(seed=3)
    P = _bit_exact(prob)
    assert P.sizes.num_long_bdds >= 3 and P.sizes.max_width > 128
    sm = P.slot_to_csr
    real = sm[sm >= 0]
    assert sorted(real.tolist()) == list(range(len(prob["col"])))


def test_problem_without_rows_plans_empty_arena():
    """Zero rows: no tiles, no slots, no launch groups; every variable is
    uncovered (its bound term is min(0, c_i))."""
    prob = dict(n=5, row_ptr=np.zeros(1, np.int64), col=np.zeros(0, np.int32), coef=np.zeros(0, np.int32),
                sense=np.zeros(0, np.int8), rhs=np.zeros(0, np.int32), c=np.array([1.0, -2, 3, -0.5, 0]))
    P = solver.plan(prob)
    assert (P.sizes.num_tiles, P.sizes.num_slots, P.sizes.num_launch_groups) == (0, 0, 0)
    P.validate()


def test_tile_budgets_respected():
    prob = workloads.tracking(frames=6, dets=60, seed=2)
    for tn, ts in [(256, 128), (1024, 512), (4096, 2048)]:
        P = solver.plan(prob, tile_nodes=tn, tile_slots=ts)
        assert P.sizes.smem_bytes <= 227 * 1024
        assert P.sizes.num_nodes_padded >= P.sizes.num_nodes


def test_host_memory_budget_fails_with_enomem():
    """Allocator-failure injection on the host: a budget below the arena
    image makes dg_plan fail with DG_ENOMEM, before anything is allocated."""
    prob = workloads.independent_set(n=20_000, seed=3)
    with pytest.raises(_lib.DgError) as e:
        solver.plan(prob, host_mb_limit=1)
    assert e.value.status == _lib.DG_ENOMEM
    solver.plan(prob, host_mb_limit=512)  # a sufficient budget passes


def test_calls_on_missing_arena_fail_cleanly():
    """Null arena / null state: status codes, no crash, no CUDA call needed."""
    lib = _lib.load()
    assert lib.dg_iterate(None, None, None, None, None, None, 0, 1, None, None) == _lib.DG_ESTATE
    assert lib.dg_lower_bound(None, None, None, None, None, None) == _lib.DG_ESTATE
    assert lib.dg_backward(None, None, None, None, None, None, 0, 1, 1, None, None, None, None, None, None,
                           None, 0, None) == _lib.DG_ESTATE
    assert lib.dg_iterate_checkpointed(None, None, None, None, None, None, 0, 1, 1, None, 0, None,
                                       None) == _lib.DG_ESTATE
    assert lib.dg_backward_checkpointed(None, None, None, None, 0, 1, 1, None, None, None, None, None, None,
                                        None, 0, None) == _lib.DG_ESTATE
    assert lib.dg_graph_replay(None, None) == _lib.DG_EINVAL
    assert b"null" in lib.dg_last_error()


@pytest.mark.parametrize("make", [lambda: workloads.set_cover(), lambda: workloads.independent_set(n=1500, seed=4),
                                  lambda: workloads.matching_quadratic(L=30, R=30, pairs=900, seed=5),
                                  lambda: workloads.tracking(frames=6, dets=200, seed=6),
                                  lambda: workloads.batched_mix(num=6, scale=0.03)[0],
                                  lambda: workloads.independent_set(n=800, avg_deg=48.0, seed=7),
                                  lambda: workloads.assignment(L=60, R=300, cand=260, seed=8)])
def test_plans_pass_the_validator(make):
    """Every plan the builder makes satisfies the arena invariants the kernels
    rely on (dg_plan_validate), also under non-default layout options."""
    rows = make()
    solver.plan(rows).validate()
    solver.plan(rows, chunk_rows=64, group_ratio_pct=50).validate()


def test_validator_catches_each_corruption(tmp_path):
    """The validator is not vacuous: a host harness builds a plan with the
    library's builder, breaks one invariant at a time and every broken copy
    is rejected while the intact one passes."""
    from paper_2205_11638_gb300 import build as B
    csrc = os.path.join(ROOT, "paper_2205_11638_gb300", "csrc")
    exe = tmp_path / "validate_harness"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-pthread", f"-I{os.path.join(B.CUDA_HOME, 'include')}",
                           f"-I{os.path.join(ROOT, 'include')}", f"-I{csrc}",
                           os.path.join(ROOT, "tests", "validate_harness.cpp"), os.path.join(csrc, "builder.cpp"),
                           "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).strip().splitlines()
    res = {ln.split("|")[0]: (int(ln.split("|")[1]), ln.split("|", 2)[2]) for ln in out}
    assert res.pop("intact") == (0, "")
    assert len(res) == 12
    for name, (st, msg) in res.items():
        assert st == _lib.DG_EINVAL and msg.startswith("dg_plan_validate:"), (name, st, msg)


def test_plan_is_deterministic():
    """The arena is rebuilt from the rows alone (solver resume saves only
    lambda and M): two plans of the same rows, built with several host
    threads, have the same layout."""
    rows = workloads.tracking(frames=6, dets=200, seed=9)
    P1 = solver.plan(rows, num_threads=4)
    P2 = solver.plan(rows, num_threads=3)
    assert np.array_equal(P1.slot_to_csr, P2.slot_to_csr)
    assert P1.launch_groups() == P2.launch_groups()
    for j in (0, 7, len(rows["row_ptr"]) - 2):
        for a, b in zip(P1.bdd(j), P2.bdd(j)):
            assert np.array_equal(a, b)
