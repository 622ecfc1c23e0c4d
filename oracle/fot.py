"""FP64 CPU oracle of the FOT dual-potential iteration (Torchylo, Swan, Tellez, Hogan,
"A fast, large-scale optimal transport algorithm for holographic beam shaping").

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import this package; the CUDA product path never
does, and this file shares no code with it.

Everything here is plain float64 (numpy, and torch CPU tensors for the bulk
log-sum-exp), written for readability, not speed.

Units and notation (pixel units throughout):
  * grid indices j,k on the input plane, L,M on the target plane, each 0..n-1
    (Sec. 2); a square grid is the paper's case, rectangular n_r x n_c is allowed.
  * cost C_jkLM = ((j-L)^2 + (k-M)^2) / 2.  Eq. 3 divides by n^2 as well; that factor
    is moved into eps, eps_px = n^2 eps_paper, so Lambda_jK = exp(-(j-K)^2 / (2 eps_px))
    (Sec. 3, definition of Lambda below Eq. 6).
  * the entropic plan is Gamma = u exp(-C/eps) V (Eq. 6); the oracle works with the
    log-domain potentials f = eps log u, psi = eps log V, which is the same iteration
    as Eqs. 7-8 written without exponent overflow.  Zero-mass pixels carry -inf.
  * marginals a = g^2 / sum g^2 and b = G^2 / sum G^2 (marginal constraints of Eq. 2,
    normalised to equal, unit mass).

Parity status: every function below is pinned by a -m "not gpu" test
(tests/test_oracle_pins.py); none is "parity unpinned".  The unequal-grid form is in
oracle/rect.py (pins in tests/test_oracle_rect.py).
"""
from __future__ import annotations

import math

import numpy as np
import torch

_CHUNK_BYTES = 1 << 28


# ----------------------------------------------------------------------------------------
# marginals and logs
# ----------------------------------------------------------------------------------------
def marginal(amp):
    """a = g^2 / sum g^2: the mass constraint of Eq. 2 from an amplitude image, unit total."""
    amp = np.asarray(amp, dtype=np.float64)
    p = amp * amp
    return p / p.sum()


def log0(a):
    """Natural log with log 0 = -inf (zero-mass pixels)."""
    with np.errstate(divide="ignore"):
        return np.log(np.asarray(a, dtype=np.float64))


# ----------------------------------------------------------------------------------------
# one 1-D contraction of the separable kernel (Sec. 3, Lambda_jK, and the Toeplitz form of
# Sec. 3.1), in the log domain with an exact per-output maximum
# ----------------------------------------------------------------------------------------
def axis_lse(Z, eps):
    """Y[r, o] = log sum_m exp(Z[r, m] - (o - m)^2 / (2 eps)),  o = 0..len-1.

    Z is in natural-log units (already divided by eps).  torch.logsumexp subtracts the
    exact maximum of every output before exponentiating, and returns -inf when every
    term is -inf.
    """
    Z = np.asarray(Z, dtype=np.float64)
    n_rows, n = Z.shape
    idx = torch.arange(n, dtype=torch.float64)
    D = (idx[:, None] - idx[None, :]) ** 2 / (2.0 * eps)          # D[o, m]
    Zt = torch.from_numpy(Z)
    out = torch.empty((n_rows, n), dtype=torch.float64)
    step = max(1, _CHUNK_BYTES // (8 * n * n))
    for r0 in range(0, n_rows, step):
        E = Zt[r0:r0 + step, None, :] - D[None, :, :]
        out[r0:r0 + step] = torch.logsumexp(E, dim=-1)
    return out.numpy()


def axis_max(Z):
    """Y[r, o] = max_m (Z[r, m] - (o - m)^2 / 2): the eps -> 0 limit of axis_lse (times eps),
    i.e. one 1-D c-transform.  Brute force over m."""
    Z = np.asarray(Z, dtype=np.float64)
    n_rows, n = Z.shape
    idx = torch.arange(n, dtype=torch.float64)
    D = (idx[:, None] - idx[None, :]) ** 2 / 2.0
    Zt = torch.from_numpy(Z)
    out = torch.empty((n_rows, n), dtype=torch.float64)
    step = max(1, _CHUNK_BYTES // (8 * n * n))
    for r0 in range(0, n_rows, step):
        out[r0:r0 + step] = (Zt[r0:r0 + step, None, :] - D[None, :, :]).amax(dim=-1)
    return out.numpy()


# ----------------------------------------------------------------------------------------
# the log of the separable kernel application  log(Lambda . V . Lambda)  (Eqs. 7-8)
# ----------------------------------------------------------------------------------------
def log_kernel_apply(pot, eps):
    """S_jk = log sum_LM exp(pot_LM/eps - C_jkLM/eps) = log[Lambda . exp(pot/eps) . Lambda]_jk.

    Separable form (Sec. 2, H_jK decomposition): a pass over the second (contiguous) axis,
    R[L, k] = log sum_M exp(pot_LM/eps - (k-M)^2/(2 eps)), then a pass over the first axis,
    S[j, k] = log sum_L exp(R[L, k] - (j-L)^2/(2 eps)).
    """
    R = axis_lse(np.asarray(pot, dtype=np.float64) / eps, eps)     # [L, k]
    S = axis_lse(R.T, eps).T                                        # [j, k]
    return S


def log_kernel_apply_dense(pot, eps):
    """Same quantity from the full N x N cost C_jkLM (tiny grids only, pin P1)."""
    pot = np.asarray(pot, dtype=np.float64)
    n_r, n_c = pot.shape
    j = np.arange(n_r, dtype=np.float64)
    k = np.arange(n_c, dtype=np.float64)
    C = (((j[:, None, None, None] - j[None, None, :, None]) ** 2)
         + ((k[None, :, None, None] - k[None, None, None, :]) ** 2)) / 2.0   # C[j,k,L,M]
    E = torch.from_numpy(pot[None, None, :, :] / eps - C / eps).reshape(n_r, n_c, -1)
    return torch.logsumexp(E, dim=-1).numpy()


# ----------------------------------------------------------------------------------------
# Algorithm 1 in the log domain
# ----------------------------------------------------------------------------------------
def u_update(psi, la, eps, dense=False):
    """Eq. 7 in log form: u = g^2 / (Lambda V Lambda)  <=>  f = eps (log a - S)."""
    S = (log_kernel_apply_dense if dense else log_kernel_apply)(psi, eps)
    return eps * (la - S), S


def v_update(f, lb, eps, dense=False):
    """Eq. 8 in log form: V = G^2 / (Lambda u Lambda)  <=>  psi = eps (log b - T)."""
    T = (log_kernel_apply_dense if dense else log_kernel_apply)(f, eps)
    return eps * (lb - T), T


def fot_iterate(g, G, eps, iters=None, dense=False, psi0=None, record=None):
    """Algorithm 1 (initialisation and Sinkhorn loop) restated in the log domain.

    eps: scalar or array of per-iteration values (px^2); both half-steps of iteration t
    use eps[t].  Potentials keep px^2 units across eps changes.
    Initial V = 1/n^2 (Algorithm 1 initialisation)  ->  psi0 = eps_0 log(1/(n_r n_c)); the
    initial u is overwritten by the first u-update and never read.
    Returns dict with f, psi (final), S_last (the log kernel sum of the last u-update,
    i.e. log(Lambda V_prev Lambda), needed by Eqs. 9-10), a, b.
    record: optional callable(t, stage, f, psi, eps) after every half-step.
    """
    a, b = marginal(g), marginal(G)
    la, lb = log0(a), log0(b)
    eps_arr = np.atleast_1d(np.asarray(eps, dtype=np.float64))
    if iters is None:
        iters = len(eps_arr)
    if len(eps_arr) == 1:
        eps_arr = np.full(iters, eps_arr[0])
    n_r, n_c = a.shape
    psi = (np.full((n_r, n_c), eps_arr[0] * math.log(1.0 / (n_r * n_c)))
           if psi0 is None else np.array(psi0, dtype=np.float64))
    f = None
    S = None
    for t in range(iters):
        e = float(eps_arr[t])
        f, S = u_update(psi, la, e, dense)
        if record is not None:
            record(t, "u", f, psi, e)
        psi, _ = v_update(f, lb, e, dense)
        if record is not None:
            record(t, "v", f, psi, e)
    return {"f": f, "psi": psi, "S_last": S, "a": a, "b": b, "eps_last": float(eps_arr[iters - 1])}


def fot_iterate_expdomain(g, G, eps, iters):
    """Algorithm 1 exactly as printed, in the exponential domain with explicit n x n
    Lambda matrices and matrix products (Algorithm 1 loop, Eqs. 7-8).  Only valid while u and V
    stay inside the float64 range (large eps); used to pin the log-domain restatement."""
    a, b = marginal(g), marginal(G)
    n_r, n_c = a.shape
    jr = np.arange(n_r, dtype=np.float64)
    jc = np.arange(n_c, dtype=np.float64)
    Lam_r = np.exp(-(jr[:, None] - jr[None, :]) ** 2 / (2.0 * eps))
    Lam_c = np.exp(-(jc[:, None] - jc[None, :]) ** 2 / (2.0 * eps))
    u = np.full((n_r, n_c), 1.0 / (n_r * n_c))
    V = np.full((n_r, n_c), 1.0 / (n_r * n_c))
    for _ in range(iters):
        u = a / (Lam_r @ V @ Lam_c)
        V = b / (Lam_r @ u @ Lam_c)
    return u, V, Lam_r, Lam_c


def cfot_iterate(g, G, eps, iters):
    """cFOT (Sec. 3.1): Algorithm 1 in the exponential domain with every product by the Toeplitz
    matrix Lambda replaced by a linear convolution with lambda_j = exp(-j^2 / (2 eps)),
    j = -(n-1) .. n-1 (eps in px^2):
        u = a / (lambda * V * lambda),   V = b / (lambda * u * lambda),
    the convolutions along the columns and along the rows, V0 = 1/(n_r n_c).  Each convolution
    is np.convolve over one line, keeping the n outputs aligned with the input grid.
    Returns u, V and S_last = log(lambda * V_prev * lambda) of the last u-update."""
    a, b = marginal(g), marginal(G)
    n_r, n_c = a.shape
    lam_r = np.exp(-np.arange(-(n_r - 1), n_r, dtype=np.float64) ** 2 / (2.0 * eps))
    lam_c = np.exp(-np.arange(-(n_c - 1), n_c, dtype=np.float64) ** 2 / (2.0 * eps))

    def kernel_apply(X):
        # rows: (X * lambda)[j, k] = sum_M X[j, M] lambda_{k - M}; then the columns likewise
        Y = np.stack([np.convolve(X[j], lam_c)[n_c - 1:2 * n_c - 1] for j in range(n_r)])
        return np.stack([np.convolve(Y[:, k], lam_r)[n_r - 1:2 * n_r - 1] for k in range(n_c)], 1)

    V = np.full((n_r, n_c), 1.0 / (n_r * n_c))
    u = S = None
    for _ in range(iters):
        KV = kernel_apply(V)
        u = a / KV
        S = np.log(KV)
        V = b / kernel_apply(u)
    return u, V, S


# ----------------------------------------------------------------------------------------
# phase recovery: Eqs. 9-10 and the trapezoid integration step of Algorithm 1
# ----------------------------------------------------------------------------------------
def target_coords(n, dx):
    """X_L = (L - floor(n/2)) dX with dX = 1/(n dx): the Fourier-plane grid of Sec. 2
    (x_j = (j - floor(n/2))/sqrt(n) gives dx = dX = 1/sqrt(n))."""
    return (np.arange(n, dtype=np.float64) - n // 2) / (n * dx)


def moments(psi, S_last, eps, dx):
    """Eqs. 9-10 with u/g^2 = exp(-S_last) (exact: u = a / (Lambda V_prev Lambda)):

      Dx_jk = sum_LM X_L exp(psi_LM/eps - C_jkLM/eps - S_last_jk)
      Dy_jk = sum_LM Y_M exp(psi_LM/eps - C_jkLM/eps - S_last_jk)

    psi is the final target potential (V after the last V-update of Algorithm 1).
    Separable evaluation with signed weights:
      R[L,k]  = log sum_M exp(psi_LM/eps - (k-M)^2/2eps)
      RY[L,k] = sum_M Y_M exp(psi_LM/eps - (k-M)^2/2eps - R[L,k])
      Dx[j,k] = sum_L X_L      exp(R[L,k] - (j-L)^2/2eps - S_last[j,k])
      Dy[j,k] = sum_L RY[L,k]  exp(R[L,k] - (j-L)^2/2eps - S_last[j,k])
    """
    psi = np.asarray(psi, dtype=np.float64)
    n_r, n_c = psi.shape
    X = target_coords(n_r, dx)
    Y = target_coords(n_c, dx)
    Z = psi / eps
    R = axis_lse(Z, eps)                                             # [L, k]
    ic = np.arange(n_c, dtype=np.float64)
    Dc = (ic[:, None] - ic[None, :]) ** 2 / (2.0 * eps)              # [k, M]
    RY = np.empty_like(R)
    for L in range(n_r):
        with np.errstate(invalid="ignore"):
            w = np.exp(Z[L][None, :] - Dc - R[L][:, None])           # [k, M]
        w = np.where(np.isfinite(R[L])[:, None], w, 0.0)
        RY[L] = w @ Y
    ir = np.arange(n_r, dtype=np.float64)
    Dr = (ir[:, None] - ir[None, :]) ** 2 / (2.0 * eps)              # [j, L]
    Dx = np.empty((n_r, n_c))
    Dy = np.empty((n_r, n_c))
    for k in range(n_c):
        with np.errstate(invalid="ignore"):
            w = np.exp(R[:, k][None, :] - Dr - S_last[:, k][:, None])  # [j, L]
        w = np.where(np.isfinite(R[:, k])[None, :], w, 0.0)
        Dx[:, k] = w @ X
        Dy[:, k] = w @ RY[:, k]
    return Dx, Dy


def moments_dense(f, psi, a, eps, dx):
    """Eqs. 4-5 literally on a tiny grid: form the plan Gamma_jkLM = u_jk exp(-C_jkLM/eps) V_LM
    (Eq. 6, u = exp(f/eps), V = exp(psi/eps)) and take its first moments over (L, M) divided
    by g^2 = a.  Defined where a > 0 (NaN elsewhere).  Pins moments()."""
    f = np.asarray(f, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    n_r, n_c = psi.shape
    X = target_coords(n_r, dx)
    Y = target_coords(n_c, dx)
    j = np.arange(n_r, dtype=np.float64)
    k = np.arange(n_c, dtype=np.float64)
    C = (((j[:, None, None, None] - j[None, None, :, None]) ** 2)
         + ((k[None, :, None, None] - k[None, None, None, :]) ** 2)) / 2.0
    u = np.exp(f / eps)
    V = np.exp(psi / eps)
    Gamma = u[:, :, None, None] * np.exp(-C / eps) * V[None, None, :, :]
    with np.errstate(invalid="ignore", divide="ignore"):
        Dx = (Gamma * X[None, None, :, None]).sum(axis=(2, 3)) / a
        Dy = (Gamma * Y[None, None, None, :]).sum(axis=(2, 3)) / a
    return np.where(a > 0, Dx, np.nan), np.where(a > 0, Dy, np.nan)


def integrate_trapezoid(Dx, Dy, dx):
    """Algorithm 1 "Integrate" step (Sec. 2: trapezoid rule): integrate from the grid centre (phi = 0 there),
    first along the centre column k = c_k over j with Dx, then along every row over k with
    Dy, outward in both directions.  Phase in cycles (Sec. 2)."""
    Dx = np.asarray(Dx, dtype=np.float64)
    Dy = np.asarray(Dy, dtype=np.float64)
    n_r, n_c = Dx.shape
    cr, cc = n_r // 2, n_c // 2
    phi = np.zeros((n_r, n_c))
    col = np.zeros(n_r)
    for j in range(cr + 1, n_r):
        col[j] = col[j - 1] + dx * 0.5 * (Dx[j - 1, cc] + Dx[j, cc])
    for j in range(cr - 1, -1, -1):
        col[j] = col[j + 1] - dx * 0.5 * (Dx[j, cc] + Dx[j + 1, cc])
    phi[:, cc] = col
    for k in range(cc + 1, n_c):
        phi[:, k] = phi[:, k - 1] + dx * 0.5 * (Dy[:, k - 1] + Dy[:, k])
    for k in range(cc - 1, -1, -1):
        phi[:, k] = phi[:, k + 1] - dx * 0.5 * (Dy[:, k] + Dy[:, k + 1])
    return phi


def phase(psi, S_last, eps, dx):
    """Algorithm 1 phase step: moments (Eqs. 9-10) then trapezoid integration."""
    Dx, Dy = moments(psi, S_last, eps, dx)
    return integrate_trapezoid(Dx, Dy, dx), Dx, Dy


# ----------------------------------------------------------------------------------------
# convergence measures (Sec. 3: total variation of the marginal violation) and duality
# ----------------------------------------------------------------------------------------
def plan_marginals(f, psi, eps):
    """Row and column sums of Gamma = exp((f + psi - C)/eps), via the separable kernel."""
    S = log_kernel_apply(psi, eps)
    T = log_kernel_apply(f, eps)
    with np.errstate(invalid="ignore"):
        row = np.exp(f / eps + S)
        col = np.exp(psi / eps + T)
    row = np.where(np.isneginf(f), 0.0, row)
    col = np.where(np.isneginf(psi), 0.0, col)
    return row, col


def marginal_l1(f, psi, a, b, eps):
    """||Gamma 1 - a||_1 + ||Gamma^T 1 - b||_1 (total variation of the marginal violation,
    times two), evaluated with the exact kernel."""
    row, col = plan_marginals(f, psi, eps)
    return float(np.abs(row - a).sum() + np.abs(col - b).sum())


def source_violation(f, psi, a, eps):
    """||Gamma 1 - a||_1: the source half of the total variation of the marginal violation
    (the convergence measure Sec. 3 names).  Right after a V-half the target half is zero up to
    rounding (psi makes the column sums equal b), so it is the whole measure there."""
    row, _ = plan_marginals(f, psi, eps)
    return float(np.abs(row - a).sum())


def fot_iterate_tol(g, G, eps, max_iters, tol, check_every):
    """Algorithm 1's loop with a convergence stop (Sec. 3): after every check_every iterations
    (and after the last allowed one) measure the marginal violation of the current iterate
    (f_t, psi_t) at eps_t and stop at the first check where it is <= tol.

    eps: scalar or max_iters per-iteration values.  Returns fot_iterate's dict plus "iters"
    (iterations done) and "tv" (the last measured violation)."""
    a, b = marginal(g), marginal(G)
    la, lb = log0(a), log0(b)
    eps_arr = np.atleast_1d(np.asarray(eps, dtype=np.float64))
    if len(eps_arr) == 1:
        eps_arr = np.full(max_iters, eps_arr[0])
    n_r, n_c = a.shape
    psi = np.full((n_r, n_c), eps_arr[0] * math.log(1.0 / (n_r * n_c)))
    f = S = None
    t, tv = 0, math.inf
    while t < max_iters:
        for _ in range(min(check_every, max_iters - t)):
            e = float(eps_arr[t])
            f, S = u_update(psi, la, e)
            psi, _ = v_update(f, lb, e)
            t += 1
        tv = source_violation(f, psi, a, float(eps_arr[t - 1]))
        if tv <= tol:
            break
    return {"f": f, "psi": psi, "S_last": S, "a": a, "b": b, "eps_last": float(eps_arr[t - 1]),
            "iters": t, "tv": tv}


def dual_objective(f, psi, a, b, eps):
    """D(f, psi) = <f, a> + <psi, b> - eps sum Gamma + eps (entropic dual; zero-mass pixels
    contribute 0 to the inner products)."""
    with np.errstate(invalid="ignore"):
        fa = np.where(a > 0, f * a, 0.0).sum()
        pb = np.where(b > 0, psi * b, 0.0).sum()
    row, _ = plan_marginals(f, psi, eps)
    return float(fa + pb - eps * row.sum() + eps)


# ----------------------------------------------------------------------------------------
# L1 intensity loss of a phase solution (Sec. 5)
# ----------------------------------------------------------------------------------------
def intensity_loss(g, phi, G):
    """|| I - b ||_1 with I = |F[g e^{2 pi i phi}]|^2 and b = G^2, both normalised to unit total
    power (Sec. 5, the loss of the eps sweep), phi in cycles.  F is the 2-D DFT between the
    centred grids of Sec. 2: x_j = (j - floor(n/2)) dx on the input plane and
    X_L = (L - floor(n/2)) dX on the target plane with dx dX = 1/n, i.e.
        F[h]_LM = sum_jk h_jk exp(-2 pi i ((j - c_r)(L - c_r)/n_r + (k - c_c)(M - c_c)/n_c)).
    Written with the two DFT matrices (tiny and mid-size grids).  Returns (loss, I)."""
    g = np.asarray(g, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    n_r, n_c = g.shape
    jr = np.arange(n_r, dtype=np.float64) - n_r // 2
    jc = np.arange(n_c, dtype=np.float64) - n_c // 2
    Fr = np.exp(-2j * np.pi * np.outer(jr, jr) / n_r)     # [L, j]
    Fc = np.exp(-2j * np.pi * np.outer(jc, jc) / n_c)     # [M, k]
    field = g * np.exp(2j * np.pi * phi)
    X = Fr @ field @ Fc.T
    inten = np.abs(X) ** 2
    inten = inten / inten.sum()
    b = marginal(G)
    return float(np.abs(inten - b).sum()), inten


# ----------------------------------------------------------------------------------------
# c-transform (eps -> 0 limit of a half-step)
# ----------------------------------------------------------------------------------------
def c_transform(pot):
    """pot^c_jk = min_LM (C_jkLM - pot_LM) = -max_LM (pot_LM - C_jkLM), separably:
    max over M along rows, then over L along columns.  -inf entries of pot are excluded;
    an all -inf input gives +inf."""
    pot = np.asarray(pot, dtype=np.float64)
    R = axis_max(pot)              # [L, k]
    Mx = axis_max(R.T).T           # [j, k]
    return -Mx


def c_transform_dense(pot):
    """Brute force over all (L, M) pairs (tiny grids)."""
    pot = np.asarray(pot, dtype=np.float64)
    n_r, n_c = pot.shape
    j = np.arange(n_r, dtype=np.float64)
    k = np.arange(n_c, dtype=np.float64)
    C = (((j[:, None, None, None] - j[None, None, :, None]) ** 2)
         + ((k[None, :, None, None] - k[None, None, None, :]) ** 2)) / 2.0
    return (C - pot[None, None]).reshape(n_r, n_c, -1).min(axis=-1)
