"""1-D entropic Sinkhorn in FP64 (test infrastructure only).

When the input and target intensities are products, a = a1 (x) a2 and b = b1 (x) b2,
the cost of Eq. 3 splits into two 1-D costs and the kernel into Lambda (x) Lambda
(Sec. 2, H_jK decomposition), so every iterate of Algorithm 1 from V = 1/n^2 is a
product, u = u1 (x) u2, V = V1 (x) V2, i.e. f = f1 (+) f2 and psi = psi1 (+) psi2.
This module computes f1, psi1 (one axis) by the plain 1-D recursion, written
independently of oracle.fot, so the 2-D oracle and the 2-D CUDA path can both be
checked element by element at any grid size.
"""
from __future__ import annotations

import math

import numpy as np


def _lse_1d(z, eps):
    """out[o] = log sum_m exp(z[m] - (o-m)^2/(2 eps)) with an exact max per output."""
    n = z.shape[0]
    m = np.arange(n, dtype=np.float64)
    out = np.empty(n)
    for o in range(n):
        e = z - (o - m) ** 2 / (2.0 * eps)
        mx = e.max()
        out[o] = -np.inf if mx == -np.inf else mx + math.log(np.exp(e - mx).sum())
    return out


def sinkhorn_1d(p, q, eps, iters):
    """1-D log-domain Sinkhorn between masses p, q (unnormalised in, normalised here).

    Initial V1 = 1/n (the 1-D factor of Algorithm 1's V = 1/n^2).  eps is a scalar or a
    per-iteration array (px^2).  Returns the potentials after the last iteration and the
    log kernel sum of the last u-update.
    """
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    p = p / p.sum()
    q = q / q.sum()
    with np.errstate(divide="ignore"):
        lp, lq = np.log(p), np.log(q)
    eps_arr = np.atleast_1d(np.asarray(eps, dtype=np.float64))
    if len(eps_arr) == 1:
        eps_arr = np.full(iters, eps_arr[0])
    psi = np.full(q.shape[0], eps_arr[0] * math.log(1.0 / q.shape[0]))
    f = S = None
    for t in range(iters):
        e = float(eps_arr[t])
        S = _lse_1d(psi / e, e)
        f = e * (lp - S)
        T = _lse_1d(f / e, e)
        psi = e * (lq - T)
    return f, psi, S
