"""FP64 CPU oracle of the BDD Lagrange-dual solver (DOGE-Train, arXiv 2205.11638).

TEST INFRASTRUCTURE ONLY: this package is imported by ``tests/``, by the smoke
check of ``__graft_entry__`` and by the CPU-baseline leg of ``bench.py``, and
by nothing else.  It shares no code with the CUDA path.

The arithmetic lives in ``dg_oracle.cpp`` (plain single-threaded C++, FP64);
this module only marshals numpy arrays through ctypes.  Every function cites
the passage of the paper it follows in the C++ source.  The pins that tie it
to the paper and to brute force are in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
# The same source built with -fopenmp: its sweeps run the (independent) BDDs
# of a sweep on all host cores.  Used only to time the oracle on every core;
# the checker is the single-threaded build.
_SO_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")
_lib = None
_lib_omp = None


def build(force: bool = False, openmp: bool = False) -> str:
    """Compiles the oracle with g++ (plain -O2, no architecture flags)."""
    src = os.path.join(_HERE, "dg_oracle.cpp")
    so = _SO_OMP if openmp else _SO
    os.makedirs(os.path.dirname(so), exist_ok=True)
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".tmp{os.getpid()}"
        extra = ["-fopenmp"] if openmp else []
        subprocess.check_call(["g++", "-O2", "-std=c++17", *extra, "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, so)
    return so


def _load(openmp: bool = False):
    global _lib, _lib_omp
    if openmp and _lib_omp is not None:
        return _lib_omp
    if not openmp and _lib is not None:
        return _lib
    lib = ctypes.CDLL(build(openmp=openmp))
    P = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    lib.orc_create.restype = ctypes.c_int
    lib.orc_create.argtypes = [ctypes.c_int, i64, P, P, P, P, P, P, ctypes.c_int, P, P,
                               ctypes.POINTER(ctypes.c_void_p)]
    lib.orc_destroy.argtypes = [P]
    lib.orc_num_slots.restype = i64
    lib.orc_num_slots.argtypes = [P]
    lib.orc_num_nodes.restype = i64
    lib.orc_num_nodes.argtypes = [P]
    lib.orc_bdd_size.restype = ctypes.c_int
    lib.orc_bdd_size.argtypes = [P, i64]
    lib.orc_bdd_export.argtypes = [P, i64, P, P, P]
    lib.orc_init_lambda.argtypes = [P, P, P]
    lib.orc_iterate.argtypes = [P, P, P, P, P, ctypes.c_int, P]
    lib.orc_sweep.argtypes = [P, ctypes.c_int, P, P, P, P]
    lib.orc_min_marginals.argtypes = [P, P, P, P]
    lib.orc_lower_bound.restype = ctypes.c_double
    lib.orc_lower_bound.argtypes = [P, P, P, P, P]
    lib.orc_lb_seed.argtypes = [P, P, P, P, P]
    lib.orc_minimiser.argtypes = [P, i64, P, ctypes.c_int, ctypes.c_int, P]
    lib.orc_backward.argtypes = [P, P, P, P, P, ctypes.c_int, P, P, P, P, P, P]
    lib.orc_nonparam_update.argtypes = [P, P, P]
    lib.orc_param_transform.argtypes = [P, P, P, P, P, P, P]
    lib.orc_param_transform_backward.argtypes = [P, P, P, P, P, P, P, P, P]
    lib.orc_smoothed.argtypes = [P, P, ctypes.c_double, P, P]
    lib.orc_last_error.restype = ctypes.c_char_p
    if openmp:
        _lib_omp = lib
    else:
        _lib = lib
    del dp
    return lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


class OracleError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"oracle status {status}: {msg}")
        self.status = status


class Oracle:
    """One binary program (Def. 1) with its BDDs, built by the oracle's own builder.

    ``rows`` is a dict of CSR arrays as produced by :mod:`workloads`
    (``n, row_ptr, col, coef, sense, rhs, c`` and optionally ``inst_row_ptr``,
    ``inst_var_ptr``).  State vectors are float64 arrays in CSR slot order.
    """

    def __init__(self, rows: dict, openmp: bool = False):
        lib = _load(openmp)
        self._lib = lib
        self._keep = {
            "row_ptr": np.ascontiguousarray(rows["row_ptr"], dtype=np.int64),
            "col": np.ascontiguousarray(rows["col"], dtype=np.int32),
            "coef": np.ascontiguousarray(rows["coef"], dtype=np.int32),
            "sense": np.ascontiguousarray(rows["sense"], dtype=np.int8),
            "rhs": np.ascontiguousarray(rows["rhs"], dtype=np.int32),
            "c": np.ascontiguousarray(rows["c"], dtype=np.float64),
        }
        self.n = int(rows["n"])
        self.m = len(self._keep["row_ptr"]) - 1
        irp = rows.get("inst_row_ptr")
        ivp = rows.get("inst_var_ptr")
        self.num_inst = 1 if irp is None else len(irp) - 1
        if irp is not None:
            self._keep["irp"] = np.ascontiguousarray(irp, dtype=np.int64)
            self._keep["ivp"] = np.ascontiguousarray(ivp, dtype=np.int32)
        k = self._keep
        h = ctypes.c_void_p()
        st = lib.orc_create(self.n, self.m, _p(k["row_ptr"]), _p(k["col"]), _p(k["coef"]), _p(k["sense"]),
                            _p(k["rhs"]), _p(k["c"]), self.num_inst,
                            _p(k.get("irp")), _p(k.get("ivp")), ctypes.byref(h))
        if st != 0:
            raise OracleError(st, lib.orc_last_error().decode())
        self._h = h
        self.num_slots = int(lib.orc_num_slots(h))
        self.num_nodes = int(lib.orc_num_nodes(h))
        self.col = k["col"]
        self.row_ptr = k["row_ptr"]
        self.c = k["c"]
        self.deg = np.bincount(self.col, minlength=self.n)

    def __del__(self):
        if getattr(self, "_h", None) is not None and getattr(self, "_lib", None) is not None:
            self._lib.orc_destroy(self._h)
            self._h = None

    # -- structure -------------------------------------------------------
    def bdd(self, j: int):
        """(level_start, lo, hi) of row j; children are ranks on the next level, -2 bottom, -1 top."""
        nn = self._lib.orc_bdd_size(self._h, j)
        k = int(self.row_ptr[j + 1] - self.row_ptr[j])
        ls = np.zeros(k + 1, np.int32)
        lo = np.zeros(nn, np.int32)
        hi = np.zeros(nn, np.int32)
        self._lib.orc_bdd_export(self._h, j, _p(ls), _p(lo), _p(hi))
        return ls, lo, hi

    # -- method ----------------------------------------------------------
    def init_lambda(self):
        lam = np.zeros(self.num_slots)
        M = np.zeros(self.num_slots)
        self._lib.orc_init_lambda(self._h, _p(lam), _p(M))
        return lam, M

    def _params(self, omega, alpha):
        if np.isscalar(omega):
            omega = np.full(self.num_slots, float(omega))
        if alpha is None:
            alpha = 1.0 / self.deg[self.col]
        return (np.ascontiguousarray(omega, dtype=np.float64),
                np.ascontiguousarray(alpha, dtype=np.float64))

    def iterate(self, lam, M, omega=0.5, alpha=None, iters=1, trace=False):
        """Runs Alg. 1 for ``iters`` iterations on copies of (lam, M)."""
        lam = np.array(lam, dtype=np.float64)
        M = np.array(M, dtype=np.float64)
        omega, alpha = self._params(omega, alpha)
        tr = np.zeros(max(iters, 1)) if trace else None
        self._lib.orc_iterate(self._h, _p(lam), _p(M), _p(omega), _p(alpha), int(iters), _p(tr))
        return (lam, M, tr[:iters]) if trace else (lam, M)

    def sweep(self, lam, M, forward: bool, omega=0.5, alpha=None):
        lam = np.array(lam, dtype=np.float64)
        M = np.array(M, dtype=np.float64)
        omega, alpha = self._params(omega, alpha)
        self._lib.orc_sweep(self._h, 1 if forward else 0, _p(lam), _p(M), _p(omega), _p(alpha))
        return lam, M

    def min_marginals(self, lam):
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        m0 = np.zeros(self.num_slots)
        m1 = np.zeros(self.num_slots)
        self._lib.orc_min_marginals(self._h, _p(lam), _p(m0), _p(m1))
        return m0, m1

    def lower_bound(self, lam, M, per_instance=False, energies=False):
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        M = np.ascontiguousarray(M, dtype=np.float64)
        pi = np.zeros(self.num_inst)
        E = np.zeros(self.m) if energies else None
        tot = self._lib.orc_lower_bound(self._h, _p(lam), _p(M), _p(pi), _p(E))
        out = [tot]
        if per_instance:
            out.append(pi)
        if energies:
            out.append(E)
        return tot if len(out) == 1 else tuple(out)

    def lb_seed(self, lam, M):
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        M = np.ascontiguousarray(M, dtype=np.float64)
        gl = np.zeros(self.num_slots)
        gM = np.zeros(self.num_slots)
        self._lib.orc_lb_seed(self._h, _p(lam), _p(M), _p(gl), _p(gM))
        return gl, gM

    def minimiser(self, j: int, lam_row, h: int, beta: int):
        lam_row = np.ascontiguousarray(lam_row, dtype=np.float64)
        x = np.zeros(len(lam_row), np.int32)
        self._lib.orc_minimiser(self._h, int(j), _p(lam_row), int(h), int(beta), _p(x))
        return x

    def nonparam_update(self, lam, theta):
        """eq. 2 on a copy of lam."""
        lam = np.array(lam, dtype=np.float64)
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        self._lib.orc_nonparam_update(self._h, _p(lam), _p(theta))
        return lam

    def param_transform(self, alpha_hat, omega_hat, theta_hat):
        """Alg. 3 output transforms; returns (alpha, omega, theta)."""
        ins = [np.ascontiguousarray(x, dtype=np.float64) for x in (alpha_hat, omega_hat, theta_hat)]
        outs = [np.zeros(self.num_slots) for _ in range(3)]
        self._lib.orc_param_transform(self._h, *[_p(x) for x in ins], *[_p(o) for o in outs])
        return tuple(outs)

    def param_transform_backward(self, alpha, omega, g_alpha, g_omega, g_theta):
        ins = [np.ascontiguousarray(x, dtype=np.float64) for x in (alpha, omega, g_alpha, g_omega, g_theta)]
        outs = [np.zeros(self.num_slots) for _ in range(3)]
        self._lib.orc_param_transform_backward(self._h, *[_p(x) for x in ins], *[_p(o) for o in outs])
        return tuple(outs)

    def smoothed(self, lam, a):
        """Smoothed subproblems (soft-min reading): (E_a per row, marginals per slot)."""
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        E = np.zeros(self.m)
        mg = np.zeros(self.num_slots)
        self._lib.orc_smoothed(self._h, _p(lam), float(a), _p(E), _p(mg))
        return E, mg

    def backward(self, lam0, M0, omega, alpha, iters, g_lamT, g_MT):
        """Alg. 2 through ``iters`` iterations; returns (g_lam0, g_M0, g_omega, g_alpha)."""
        omega, alpha = self._params(omega, alpha)
        lam0 = np.ascontiguousarray(lam0, dtype=np.float64)
        M0 = np.ascontiguousarray(M0, dtype=np.float64)
        g_lamT = np.ascontiguousarray(g_lamT, dtype=np.float64)
        g_MT = np.ascontiguousarray(g_MT, dtype=np.float64)
        outs = [np.zeros(self.num_slots) for _ in range(4)]
        self._lib.orc_backward(self._h, _p(lam0), _p(M0), _p(omega), _p(alpha), int(iters), _p(g_lamT), _p(g_MT),
                          *[_p(o) for o in outs])
        return tuple(outs)
