"""Dense FP64 reference for gradients of a phase loss through unrolled FOT iterations
(test infrastructure only).

Loss (the backward workload): L = sum_jk w_jk phi_jk + sum_jk (phi_jk - phi*_jk)^2, with phi
the phase of Algorithm 1 (Eqs. 7-10 and trapezoid integration) after T iterations, as a
function of the input and target amplitudes g and G.  This module writes the whole chain
with dense torch.float64 tensors (the full N x N cost, so only tiny grids) and lets
torch.autograd differentiate it; it shares no code with oracle.fot (a second, independent
implementation) and none with the CUDA path.  Pinned against central finite differences
in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import math

import torch

T64 = torch.float64


def _cost(n_r, n_c):
    j = torch.arange(n_r, dtype=T64)
    k = torch.arange(n_c, dtype=T64)
    jj, kk = torch.meshgrid(j, k, indexing="ij")
    P = torch.stack([jj.reshape(-1), kk.reshape(-1)], 1)
    return ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1) / 2.0      # [N, N], pixel units


def _trapezoid_operator(n_r, n_c, dx):
    """phi = Op @ concat(Dx.ravel(), Dy.ravel()): the trapezoid integration of Algorithm 1
    (phi = 0 at the centre, centre column with Dx, then each row with Dy) as a matrix."""
    N = n_r * n_c
    Op = torch.zeros(N, 2 * N, dtype=T64)
    cr, cc = n_r // 2, n_c // 2

    def ix(j, k):
        return j * n_c + k

    col = {cr: torch.zeros(2 * N, dtype=T64)}
    for j in range(cr + 1, n_r):
        v = col[j - 1].clone()
        v[ix(j - 1, cc)] += 0.5 * dx
        v[ix(j, cc)] += 0.5 * dx
        col[j] = v
    for j in range(cr - 1, -1, -1):
        v = col[j + 1].clone()
        v[ix(j, cc)] -= 0.5 * dx
        v[ix(j + 1, cc)] -= 0.5 * dx
        col[j] = v
    for j in range(n_r):
        Op[ix(j, cc)] = col[j]
        v = col[j]
        for k in range(cc + 1, n_c):
            v = v.clone()
            v[N + ix(j, k - 1)] += 0.5 * dx
            v[N + ix(j, k)] += 0.5 * dx
            Op[ix(j, k)] = v
        v = col[j]
        for k in range(cc - 1, -1, -1):
            v = v.clone()
            v[N + ix(j, k)] -= 0.5 * dx
            v[N + ix(j, k + 1)] -= 0.5 * dx
            Op[ix(j, k)] = v
    return Op


def _log_mass(m):
    """log m with log 0 = -inf and no gradient through zero-mass pixels: the loss sees such a
    pixel only through exp(f/eps) = m exp(-S), which is linear in m = amp^2 / sum amp^2, so
    its derivative with respect to the amplitude is 0 there."""
    pos = m > 0
    safe = torch.where(pos, m, torch.ones_like(m))
    return torch.where(pos, torch.log(safe), torch.full_like(m, -math.inf))


def phase_loss(g, G, eps, iters, w, phi_target, dx):
    """L(g, G) for torch float64 tensors g, G (n_r x n_c, requires_grad allowed)."""
    n_r, n_c = g.shape
    C = _cost(n_r, n_c)
    a = (g * g) / (g * g).sum()
    b = (G * G) / (G * G).sum()
    la = _log_mass(a).reshape(-1)
    lb = _log_mass(b).reshape(-1)
    psi = torch.full((n_r * n_c,), eps * math.log(1.0 / (n_r * n_c)), dtype=T64)
    S = None
    for _ in range(iters):
        S = torch.logsumexp(psi[None, :] / eps - C / eps, dim=1)           # log(Lambda V Lambda)
        f = eps * (la - S)                                                  # Eq. 7
        Tt = torch.logsumexp(f[:, None] / eps - C / eps, dim=0)            # log(Lambda u Lambda)
        psi = eps * (lb - Tt)                                               # Eq. 8
    X = (torch.arange(n_r, dtype=T64) - n_r // 2) / (n_r * dx)
    Y = (torch.arange(n_c, dtype=T64) - n_c // 2) / (n_c * dx)
    XL = X[:, None].expand(n_r, n_c).reshape(-1)
    YM = Y[None, :].expand(n_r, n_c).reshape(-1)
    Wp = torch.exp(psi[None, :] / eps - C / eps - S[:, None])               # u/g^2 * Gamma
    Dx = Wp @ XL                                                            # Eq. 9
    Dy = Wp @ YM                                                            # Eq. 10
    phi = _trapezoid_operator(n_r, n_c, dx) @ torch.cat([Dx, Dy])
    phi = phi.reshape(n_r, n_c)
    return (w * phi).sum() + ((phi - phi_target) ** 2).sum(), phi


def gradients(g, G, eps, iters, w, phi_target, dx):
    """(L, dL/dg, dL/dG) by torch.autograd on the dense float64 chain."""
    gt = torch.tensor(g, dtype=T64, requires_grad=True)
    Gt = torch.tensor(G, dtype=T64, requires_grad=True)
    L, _ = phase_loss(gt, Gt, eps, iters, torch.as_tensor(w, dtype=T64),
                      torch.as_tensor(phi_target, dtype=T64), dx)
    L.backward()
    return float(L), gt.grad.numpy(), Gt.grad.numpy()


def loss_value(g, G, eps, iters, w, phi_target, dx):
    with torch.no_grad():
        L, _ = phase_loss(torch.as_tensor(g, dtype=T64), torch.as_tensor(G, dtype=T64), eps, iters,
                          torch.as_tensor(w, dtype=T64), torch.as_tensor(phi_target, dtype=T64), dx)
    return float(L)
