"""Unregularised optimal transport by linear programming (test infrastructure only).

Solves the primal of Eqs. 2-3 (minimise sum Gamma C subject to Gamma >= 0 and the two
marginal constraints) on tiny grids with scipy's HiGHS solver, to bound the entropic
iterate of oracle.fot from the unregularised optimum.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import linprog


def ot_lp(a, b):
    """Return (optimal cost, optimal plan [Na, Nb]) for masses a, b on an n_r x n_c grid with
    C = ((j-L)^2 + (k-M)^2)/2 (pixel units)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n_r, n_c = a.shape
    jj, kk = np.meshgrid(np.arange(n_r), np.arange(n_c), indexing="ij")
    P = np.stack([jj.ravel(), kk.ravel()], axis=1).astype(np.float64)
    C = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1) / 2.0
    Na = Nb = n_r * n_c
    A_eq = np.zeros((Na + Nb, Na * Nb))
    for i in range(Na):
        A_eq[i, i * Nb:(i + 1) * Nb] = 1.0
    for j in range(Nb):
        A_eq[Na + j, j::Nb] = 1.0
    b_eq = np.concatenate([a.ravel(), b.ravel()])
    res = linprog(C.ravel(), A_eq=A_eq, b_eq=b_eq, bounds=(0, None), method="highs")
    assert res.status == 0, res.message
    return float(res.fun), res.x.reshape(Na, Nb), C
