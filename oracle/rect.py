"""FP64 CPU oracle of Algorithm 1 between an input grid and an output grid of different sizes.

TEST INFRASTRUCTURE ONLY (the same rule as oracle/fot.py: only tests/, smoke() and bench.py's
CPU legs may import it).

Sec. 2 remarks that square, equal arrays are not essential to the method.  Here the input
plane has n_in_r x n_in_c pixels (indices j, k) and the target plane n_out_r x n_out_c pixels
(indices L, M), both with unit pixel spacing and centre-aligned: the pixel coordinates are
    x_j = j - (n_in_r - 1)/2,  X_L = L - (n_out_r - 1)/2   (and y_k, Y_M likewise),
so equal sizes give the cost of oracle/fot.py exactly.  The cost C_jkLM = ((x_j - X_L)^2 +
(y_k - Y_M)^2) / 2 (Eq. 3 with eps in px^2) still separates, Lambda becomes the rectangular
matrix Lambda_jL = exp(-(x_j - X_L)^2 / (2 eps)), and Eqs. 7-8 read, in the log domain,
    f   = eps (log a - log(Lambda_r V Lambda_c^T)),   on the input grid,
    psi = eps (log b - log(Lambda_r^T u Lambda_c)),   on the output grid,
with the marginals a = g^2 / sum g^2 (input grid) and b = G^2 / sum G^2 (output grid)."""
from __future__ import annotations

import math

import numpy as np
import torch

from oracle.fot import log0, marginal


def axis_lse_rect(Z, eps, n_out):
    """Y[r, o] = log sum_m exp(Z[r, m] - (X_o - x_m)^2 / (2 eps)), o = 0..n_out-1, with the
    centre-aligned coordinates x_m = m - (n_in - 1)/2 of Z's axis (n_in = Z.shape[1]) and
    X_o = o - (n_out - 1)/2 of the output axis.  Z is in natural-log units."""
    Z = np.asarray(Z, dtype=np.float64)
    n_in = Z.shape[1]
    x = torch.arange(n_in, dtype=torch.float64) - (n_in - 1) / 2.0
    X = torch.arange(n_out, dtype=torch.float64) - (n_out - 1) / 2.0
    D = (X[:, None] - x[None, :]) ** 2 / (2.0 * eps)                 # D[o, m]
    E = torch.from_numpy(Z)[:, None, :] - D[None, :, :]
    return torch.logsumexp(E, dim=-1).numpy()


def log_kernel_apply_rect(pot, eps, out_shape):
    """S_jk = log sum_LM exp(pot_LM/eps - C_jkLM/eps) for a potential on one grid and outputs
    on a grid of shape out_shape: a pass over pot's second axis, then over its first."""
    R = axis_lse_rect(np.asarray(pot, dtype=np.float64) / eps, eps, out_shape[1])   # [L, k]
    return axis_lse_rect(R.T, eps, out_shape[0]).T                                    # [j, k]


def log_kernel_apply_rect_dense(pot, eps, out_shape):
    """The same sum from the full four-index cost (tiny grids only; pins the separable form)."""
    pot = np.asarray(pot, dtype=np.float64)
    (pr, pc), (qr, qc) = pot.shape, out_shape
    X = np.arange(pr) - (pr - 1) / 2.0
    Y = np.arange(pc) - (pc - 1) / 2.0
    x = np.arange(qr) - (qr - 1) / 2.0
    y = np.arange(qc) - (qc - 1) / 2.0
    C = ((x[:, None, None, None] - X[None, None, :, None]) ** 2
         + (y[None, :, None, None] - Y[None, None, None, :]) ** 2) / 2.0             # [j,k,L,M]
    E = torch.from_numpy(pot[None, None, :, :] / eps - C / eps).reshape(qr, qc, -1)
    return torch.logsumexp(E, dim=-1).numpy()


def fot_iterate_rect(g, G, eps, iters=None, dense=False):
    """Algorithm 1 in the log domain between the grid of g (input) and the grid of G (output).
    eps: scalar or per-iteration array (px^2).  Start V = 1/(n_out_r n_out_c), i.e.
    psi0 = eps_0 log(1 / (n_out_r n_out_c)).  Returns f (input grid), psi (output grid),
    S_last, a, b, eps_last."""
    a, b = marginal(g), marginal(G)
    la, lb = log0(a), log0(b)
    eps_arr = np.atleast_1d(np.asarray(eps, dtype=np.float64))
    if iters is None:
        iters = len(eps_arr)
    if len(eps_arr) == 1:
        eps_arr = np.full(iters, eps_arr[0])
    apply = log_kernel_apply_rect_dense if dense else log_kernel_apply_rect
    psi = np.full(b.shape, eps_arr[0] * math.log(1.0 / b.size))
    f = S = None
    for t in range(iters):
        e = float(eps_arr[t])
        S = apply(psi, e, a.shape)                                   # Eq. 7
        f = e * (la - S)
        T = apply(f, e, b.shape)                                     # Eq. 8
        psi = e * (lb - T)
    return {"f": f, "psi": psi, "S_last": S, "a": a, "b": b, "eps_last": float(eps_arr[iters - 1])}


def marginals_rect(f, psi, eps):
    """Row sums (input grid) and column sums (output grid) of Gamma = exp((f + psi - C)/eps)."""
    S = log_kernel_apply_rect(psi, eps, f.shape)
    T = log_kernel_apply_rect(f, eps, psi.shape)
    with np.errstate(invalid="ignore"):
        rows = np.where(np.isfinite(f), np.exp(f / eps + S), 0.0)
        cols = np.where(np.isfinite(psi), np.exp(psi / eps + T), 0.0)
    return rows, cols
