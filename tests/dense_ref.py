"""Dense plain-PyTorch restatement of Alg. 1 for tiny instances, used as an
autograd reference for the adjoint (Alg. 2).

Min-marginals are computed by enumerating each subproblem's feasible
assignments (no BDD, no shortest paths); the update follows Alg. 1 with the
sweep-start snapshot of sum_k M_ik.  Gradients come from torch.autograd, so
this shares nothing with the oracle's or the CUDA path's hand-written
backpropagation.  Only for inputs without ties (torch.min routes a tie's
gradient to one element, the rules of the other implementations may pick
another)."""
from __future__ import annotations

import numpy as np
import torch

from tests import brute


def feasible_sets(prob):
    out = []
    for j in range(len(prob["row_ptr"]) - 1):
        b, e = prob["row_ptr"][j], prob["row_ptr"][j + 1]
        X = brute.row_feasible(prob["coef"][b:e], int(prob["sense"][j]), int(prob["rhs"][j]))
        out.append(torch.as_tensor(X, dtype=torch.float64))
    return out


def iterate(prob, lam0, M0, omega, alpha, iters, X=None):
    """lam0, M0, omega, alpha: float64 tensors in CSR slot order (may require
    grad).  Returns (lam_T, M_T)."""
    X = X if X is not None else feasible_sets(prob)
    rp = prob["row_ptr"]
    col = torch.as_tensor(prob["col"], dtype=torch.int64)
    n = int(prob["n"])
    lam = list(lam0.unbind())
    M = list(M0.unbind())
    for _ in range(iters):
        for forward in (True, False):
            S = torch.zeros(n, dtype=torch.float64).index_add(0, col, torch.stack(M))
            for j in range(len(rp) - 1):
                b, e = int(rp[j]), int(rp[j + 1])
                k = e - b
                order = range(k) if forward else range(k - 1, -1, -1)
                for h in order:
                    lj = torch.stack(lam[b:e])
                    vals = X[j] @ lj
                    sel = X[j][:, h] > 0.5
                    m1 = vals[sel].min()
                    m0 = vals[~sel].min()
                    s = b + h
                    Mn = omega[s] * (m1 - m0)
                    lam[s] = lam[s] - Mn + alpha[s] * S[col[s]]
                    M[s] = Mn
    return torch.stack(lam), torch.stack(M)


def lower_bound(prob, lam, M, X=None):
    """Sum_j E^j(lambda) + sum_i min(0, S_i) (+ min(0, c_i) for uncovered i)."""
    X = X if X is not None else feasible_sets(prob)
    rp = prob["row_ptr"]
    col = torch.as_tensor(prob["col"], dtype=torch.int64)
    n = int(prob["n"])
    tot = lam.new_zeros(())
    for j in range(len(rp) - 1):
        b, e = int(rp[j]), int(rp[j + 1])
        tot = tot + (X[j] @ lam[b:e]).min()
    S = torch.zeros(n, dtype=torch.float64).index_add(0, col, M)
    deg = np.bincount(prob["col"], minlength=n)
    c = torch.as_tensor(prob["c"], dtype=torch.float64)
    cov = torch.as_tensor(deg > 0)
    return tot + torch.where(cov, torch.clamp(S, max=0.0), torch.clamp(c, max=0.0)).sum()
