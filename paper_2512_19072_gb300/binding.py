"""Thin ctypes binding of libfot.so (include/fot.h): argument marshalling only.

Every function here has the name of the C entry point it calls and takes torch CUDA
tensors (float32, contiguous, rows x cols) where the C call takes device pointers; the
stream is the current torch stream.  All arithmetic of the method runs in the library's
CUDA kernels.  Importing this module raises if libfot.so has not been built: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfot.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2512_19072_gb300.build` "
                      "(the FOT path has no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

FOT_FP32, FOT_MIXED, FOT_FP32_DENSE, FOT_AUTO, FOT_BF16 = 0, 1, 2, 3, 4
FOT_EPS_PX2, FOT_EPS_PAPER = 0, 1
FOT_KERNEL_PLAN, FOT_KERNEL_BAND, FOT_KERNEL_TENSOR, FOT_KERNEL_DENSE = 0, 1, 2, 3
FOT_KERNEL_CLASSES = 4
KERNEL_CLASS_NAMES = ("band_plan_kernel", "band_pass_kernel", "tc_pass_kernel", "axis_pass_kernel")
STATUS = {0: "FOT_OK", 1: "FOT_EINVAL", 2: "FOT_ENOMEM", 3: "FOT_ECUDA", 4: "FOT_ENONFINITE",
          5: "FOT_ETIMEOUT", 6: "FOT_EMASS", 7: "FOT_EUNSUPPORTED", 8: "FOT_ESTATE"}

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_DP = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "fot_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I, _P]),
    "fot_destroy": (None, [_P]),
    "fot_set_stream": (_I, [_P, _P]),
    "fot_set_problem": (_I, [_P, _P, _P]),
    "fot_solve": (_I, [_P, _P, _P, _D, _DP, _I, _I, _I]),
    "fot_resume": (_I, [_P, _DP, _I, _I, _I]),
    "fot_cfot_solve": (_I, [_P, _P, _P, _D, _DP, _I, _I, _I]),
    "fot_solve_tol": (_I, [_P, _P, _P, _D, _DP, _I, _I, _I, _D, _I, ctypes.POINTER(_I), _DP]),
    "fot_select_eps": (_I, [_P, _P, _P, _D, _DP, _I, _I, _I, _I, _D, _I, ctypes.POINTER(_I), _DP]),
    "fot_solve_rect": (_I, [_P, _I, _I, _P, _I, _I, _DP, _I, _I, _P, _P, _P]),
    "fot_solve_rect_fp64": (_I, [_P, _I, _I, _P, _I, _I, _DP, _I, _I, _P, _P, _P]),
    "fot_sync": (_I, [_P]),
    "fot_potentials": (_I, [_P, _P, _P]),
    "fot_set_potentials": (_I, [_P, _P, _P]),
    "fot_phase": (_I, [_P, _P, _P, _P]),
    "fot_marginal_error": (_I, [_P, _DP, _DP]),
    "fot_intensity_loss": (_I, [_P, _P, _DP, _P]),
    "fot_moments": (_I, [_P, _P, _P, _D, _D, _P, _P, _P]),
    "fot_u_update": (_I, [_P, _P, _D, _P, _P]),
    "fot_v_update": (_I, [_P, _P, _D, _P, _P]),
    "fot_c_transform": (_I, [_P, _P, _P]),
    "fot_u_update_noalloc": (_I, [_P, _P, _I, _I, _D, _P, _P, _P]),
    "fot_solve_phase_host": (_I, [_P, _P, _P, _D, _DP, _I, _I, _I, _P]),
    "fot_launch_count": (ctypes.c_int64, [_P]),
    "fot_loop_time": (_I, [_P, _DP, ctypes.POINTER(ctypes.c_int64)]),
    "fot_work_count": (_I, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "fot_work_split": (_I, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "fot_set_kernel_timing": (_I, [_P, _I]),
    "fot_kernel_times": (_I, [_P, _DP, ctypes.POINTER(ctypes.c_int64)]),
    "fot_status_string": (ctypes.c_char_p, [_I]),
    "fot_backward": (_I, [_P, _P, _P, _P, _P, _P, _I, _P, _P]),
    "fot_batch_create": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_I), ctypes.POINTER(_I), _I, _I, _P]),
    "fot_batch_destroy": (None, [_P]),
    "fot_batch_context": (_P, [_P, _I]),
    "fot_batch_solve": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _DP, _I, _I, _I]),
    "fot_batch_info": (_I, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_I)]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


class FotError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.fot_status_string(status).decode()
        super().__init__(f"{where}: {STATUS.get(status, status)} ({msg})")


def _check(status, where):
    if status != 0:
        raise FotError(status, where)


def _ptr(t):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _eps_arr(eps):
    e = np.ascontiguousarray(np.atleast_1d(np.asarray(eps, dtype=np.float64)))
    return e, e.ctypes.data_as(_DP), len(e)


class Context:
    """Owns one fot_ctx (rows x cols) and the device scratch it allocates."""

    def __init__(self, rows, cols, precision=FOT_FP32, device=None):
        if device is None:
            device = torch.cuda.current_device()
        self.rows, self.cols, self.device = rows, cols, device
        h = _P()
        with torch.cuda.device(device):
            _check(_lib.fot_create(ctypes.byref(h), rows, cols, precision, device, _stream()),
                   "fot_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.fot_destroy(self._h)
            self._h = None

    __del__ = close

    def _sync_stream(self):
        _lib.fot_set_stream(self._h, _stream())

    def empty(self):
        return torch.empty((self.rows, self.cols), dtype=torch.float32, device=f"cuda:{self.device}")


def fot_create(rows, cols, precision=FOT_FP32, device=None):
    return Context(rows, cols, precision, device)


def fot_destroy(ctx):
    ctx.close()


def fot_set_problem(ctx, g, G):
    ctx._sync_stream()
    _check(_lib.fot_set_problem(ctx._h, _ptr(g), _ptr(G)), "fot_set_problem")


def fot_solve(ctx, g, G, eps, iters=None, dx=0.0, eps_units=FOT_EPS_PX2):
    e, ep, ne = _eps_arr(eps)
    if iters is None:
        iters = ne
    ctx._sync_stream()
    _check(_lib.fot_solve(ctx._h, _ptr(g), _ptr(G), float(dx), ep, ne, eps_units, int(iters)),
           "fot_solve")


def fot_cfot_solve(ctx, g, G, eps, iters=None, dx=0.0, eps_units=FOT_EPS_PX2):
    e, ep, ne = _eps_arr(eps)
    if iters is None:
        iters = ne
    ctx._sync_stream()
    _check(_lib.fot_cfot_solve(ctx._h, _ptr(g), _ptr(G), float(dx), ep, ne, eps_units, int(iters)),
           "fot_cfot_solve")


def fot_solve_tol(ctx, g, G, eps, max_iters, tol, check_every, dx=0.0, eps_units=FOT_EPS_PX2):
    """Returns (iterations done, last measured marginal violation)."""
    e, ep, ne = _eps_arr(eps)
    ctx._sync_stream()
    it = ctypes.c_int(0)
    tv = ctypes.c_double(0.0)
    _check(_lib.fot_solve_tol(ctx._h, _ptr(g), _ptr(G), float(dx), ep, ne, eps_units, int(max_iters),
                              float(tol), int(check_every), ctypes.byref(it), ctypes.byref(tv)),
           "fot_solve_tol")
    return it.value, tv.value


def fot_select_eps(ctx, g, G, candidates, probe_iters, check_every, min_decrease=0.1, use_cfot=False,
                   dx=0.0, eps_units=FOT_EPS_PX2):
    """Smallest stable eps among the candidates: returns (index into candidates or -1, tv)."""
    c = np.ascontiguousarray(np.asarray(candidates, dtype=np.float64).ravel())
    idx = ctypes.c_int(-1)
    tv = ctypes.c_double(0.0)
    ctx._sync_stream()
    _check(_lib.fot_select_eps(ctx._h, _ptr(g), _ptr(G), float(dx), c.ctypes.data_as(_DP), len(c), eps_units,
                               int(probe_iters), int(check_every), float(min_decrease), int(bool(use_cfot)),
                               ctypes.byref(idx), ctypes.byref(tv)), "fot_select_eps")
    return idx.value, tv.value


def fot_solve_rect(g, G, eps, iters=None):
    """Algorithm 1 between the grid of g (input) and the grid of G (output), both float32 CUDA
    tensors; returns (f on the input grid, psi on the output grid)."""
    e, ep, ne = _eps_arr(eps)
    if iters is None:
        iters = ne
    f = torch.empty_like(g)
    psi = torch.empty_like(G)
    (ri, ci), (ro, co) = g.shape, G.shape
    _check(_lib.fot_solve_rect(_ptr(g), ri, ci, _ptr(G), ro, co, ep, ne, int(iters), _ptr(f), _ptr(psi),
                               _stream()), "fot_solve_rect")
    return f, psi


def _ptr64(t):
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def fot_solve_rect_fp64(g, G, eps, iters=None):
    """FP64 form of fot_solve_rect (float64 CUDA tensors in and out)."""
    e, ep, ne = _eps_arr(eps)
    if iters is None:
        iters = ne
    f = torch.empty_like(g)
    psi = torch.empty_like(G)
    (ri, ci), (ro, co) = g.shape, G.shape
    _check(_lib.fot_solve_rect_fp64(_ptr64(g), ri, ci, _ptr64(G), ro, co, ep, ne, int(iters), _ptr64(f),
                                    _ptr64(psi), _stream()), "fot_solve_rect_fp64")
    return f, psi


def fot_resume(ctx, eps, iters=None, eps_units=FOT_EPS_PX2):
    e, ep, ne = _eps_arr(eps)
    if iters is None:
        iters = ne
    ctx._sync_stream()
    _check(_lib.fot_resume(ctx._h, ep, ne, eps_units, int(iters)), "fot_resume")


def fot_sync(ctx):
    _check(_lib.fot_sync(ctx._h), "fot_sync")


def fot_potentials(ctx):
    f, psi = ctx.empty(), ctx.empty()
    ctx._sync_stream()
    _check(_lib.fot_potentials(ctx._h, _ptr(f), _ptr(psi)), "fot_potentials")
    return f, psi


def fot_set_potentials(ctx, f, psi):
    ctx._sync_stream()
    _check(_lib.fot_set_potentials(ctx._h, _ptr(f), _ptr(psi)), "fot_set_potentials")


def fot_phase(ctx):
    phi, dx, dy = ctx.empty(), ctx.empty(), ctx.empty()
    ctx._sync_stream()
    _check(_lib.fot_phase(ctx._h, _ptr(phi), _ptr(dx), _ptr(dy)), "fot_phase")
    return phi, dx, dy


def fot_moments(ctx, psi, logsum_u, eps, dx=0.0):
    phi, Dx, Dy = ctx.empty(), ctx.empty(), ctx.empty()
    ctx._sync_stream()
    _check(_lib.fot_moments(ctx._h, _ptr(psi), _ptr(logsum_u), float(eps), float(dx), _ptr(phi),
                            _ptr(Dx), _ptr(Dy)), "fot_moments")
    return phi, Dx, Dy


def fot_marginal_error(ctx):
    l1, dual = ctypes.c_double(), ctypes.c_double()
    ctx._sync_stream()
    _check(_lib.fot_marginal_error(ctx._h, ctypes.byref(l1), ctypes.byref(dual)),
           "fot_marginal_error")
    return l1.value, dual.value


def fot_intensity_loss(ctx, phi, with_intensity=False):
    """L1 intensity loss of the phase phi (cycles) for the loaded problem; with_intensity also
    returns the normalised far-field intensity."""
    out = ctypes.c_double()
    inten = ctx.empty() if with_intensity else None
    ctx._sync_stream()
    _check(_lib.fot_intensity_loss(ctx._h, _ptr(phi), ctypes.byref(out), _ptr(inten)),
           "fot_intensity_loss")
    return (out.value, inten) if with_intensity else out.value


def fot_u_update(ctx, psi, eps, with_logsum=False):
    f = ctx.empty()
    S = ctx.empty() if with_logsum else None
    ctx._sync_stream()
    _check(_lib.fot_u_update(ctx._h, _ptr(psi), float(eps), _ptr(f), _ptr(S)), "fot_u_update")
    return (f, S) if with_logsum else f


def fot_v_update(ctx, f, eps, with_logsum=False):
    psi = ctx.empty()
    T = ctx.empty() if with_logsum else None
    ctx._sync_stream()
    _check(_lib.fot_v_update(ctx._h, _ptr(f), float(eps), _ptr(psi), _ptr(T)), "fot_v_update")
    return (psi, T) if with_logsum else psi


def fot_u_update_noalloc(psi, log_a, eps, f_out=None, logsum_out=None):
    """Allocation-free u-update on the current device and stream (no context): the caller
    supplies psi, log_a and the outputs (torch tensors, rows x cols float32)."""
    rows, cols = psi.shape
    if f_out is None:
        f_out = torch.empty_like(psi)
    _check(_lib.fot_u_update_noalloc(_ptr(psi), _ptr(log_a), rows, cols, float(eps), _ptr(f_out),
                                     _ptr(logsum_out), _stream()), "fot_u_update_noalloc")
    return f_out


def fot_c_transform(ctx, pot):
    out = ctx.empty()
    ctx._sync_stream()
    _check(_lib.fot_c_transform(ctx._h, _ptr(pot), _ptr(out)), "fot_c_transform")
    return out


def fot_solve_phase_host(ctx, g_host, G_host, eps, iters=None, dx=0.0, eps_units=FOT_EPS_PX2,
                         phi_host=None):
    """g_host, G_host: pinned (or pageable) CPU float32 tensors; returns phi on the host."""
    e, ep, ne = _eps_arr(eps)
    if iters is None:
        iters = ne
    if phi_host is None:
        phi_host = torch.empty((ctx.rows, ctx.cols), dtype=torch.float32, pin_memory=True)
    for t in (g_host, G_host, phi_host):
        if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError("expected contiguous float32 host tensors")
    ctx._sync_stream()
    _check(_lib.fot_solve_phase_host(ctx._h, ctypes.c_void_p(g_host.data_ptr()),
                                     ctypes.c_void_p(G_host.data_ptr()), float(dx), ep, ne,
                                     eps_units, int(iters), ctypes.c_void_p(phi_host.data_ptr())),
           "fot_solve_phase_host")
    return phi_host


def fot_launch_count(ctx):
    return int(_lib.fot_launch_count(ctx._h))


def fot_loop_time(ctx):
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(_lib.fot_loop_time(ctx._h, ctypes.byref(ms), ctypes.byref(n)), "fot_loop_time")
    return ms.value, n.value


def fot_work_count(ctx, tensor=False):
    n, t = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.fot_work_count(ctx._h, ctypes.byref(n), ctypes.byref(t)), "fot_work_count")
    return (n.value, t.value) if tensor else n.value


def fot_work_split(ctx):
    """(banded GEMM, exact-window, tensor-core, dense) terms since creation."""
    out = (ctypes.c_int64 * 4)()
    _check(_lib.fot_work_split(ctx._h, out), "fot_work_split")
    return tuple(int(v) for v in out)


def fot_set_kernel_timing(ctx, on):
    _check(_lib.fot_set_kernel_timing(ctx._h, 1 if on else 0), "fot_set_kernel_timing")


def fot_kernel_times(ctx):
    """{class name: (ms, launches)} over the loops since timing was switched on / last read."""
    ms = (ctypes.c_double * FOT_KERNEL_CLASSES)()
    n = (ctypes.c_int64 * FOT_KERNEL_CLASSES)()
    _check(_lib.fot_kernel_times(ctx._h, ms, n), "fot_kernel_times")
    return {KERNEL_CLASS_NAMES[k]: (float(ms[k]), int(n[k])) for k in range(FOT_KERNEL_CLASSES)}


class _View(Context):
    """A context owned by a batch (not destroyed on its own)."""

    def __init__(self, handle, rows, cols, device):
        self._h = ctypes.c_void_p(handle)
        self.rows, self.cols, self.device = rows, cols, device

    def close(self):
        self._h = None

    __del__ = close


class Batch:
    """fot_batch: many problems of their own sizes solved together (one graph launch)."""

    def __init__(self, sizes, precision=FOT_FP32, device=None):
        if device is None:
            device = torch.cuda.current_device()
        self.sizes = [tuple(s) for s in sizes]
        self.device = device
        n = len(self.sizes)
        rows = (_I * n)(*[s[0] for s in self.sizes])
        cols = (_I * n)(*[s[1] for s in self.sizes])
        h = _P()
        with torch.cuda.device(device):
            _check(_lib.fot_batch_create(ctypes.byref(h), n, rows, cols, precision, device, _stream()),
                   "fot_batch_create")
        self._h = h
        self.contexts = [_View(_lib.fot_batch_context(h, q), *self.sizes[q], device) for q in range(n)]

    def close(self):
        if getattr(self, "_h", None):
            for c in self.contexts:
                c.close()
            _lib.fot_batch_destroy(self._h)
            self._h = None

    __del__ = close


def fot_batch_create(sizes, precision=FOT_FP32, device=None):
    return Batch(sizes, precision, device)


def fot_batch_destroy(batch):
    batch.close()


def fot_batch_context(batch, index):
    return batch.contexts[index]


def fot_batch_solve(batch, gs, Gs, eps, iters, dx=0.0, eps_units=FOT_EPS_PX2):
    """gs, Gs: lists of CUDA tensors; eps: array [count] or [count, n_eps] of px^2 values."""
    n = len(gs)
    e = np.ascontiguousarray(np.asarray(eps, dtype=np.float64).reshape(n, -1))
    ep = e.ctypes.data_as(_DP)
    gp = (_P * n)(*[_ptr(t) for t in gs])
    Gp = (_P * n)(*[_ptr(t) for t in Gs])
    _check(_lib.fot_batch_solve(batch._h, gp, Gp, float(dx), ep, e.shape[1], eps_units, int(iters)),
           "fot_batch_solve")
    batch._keep = (e, gs, Gs)


def fot_batch_info(batch):
    k, t = ctypes.c_int64(), _I()
    _check(_lib.fot_batch_info(batch._h, ctypes.byref(k), ctypes.byref(t)), "fot_batch_info")
    return k.value, bool(t.value)


def fot_backward(ctx, g, G, dL_dphi=None, dL_df=None, dL_dpsi=None, checkpoint_every=10):
    dg, dG = torch.empty_like(g), torch.empty_like(G)
    ctx._sync_stream()
    _check(_lib.fot_backward(ctx._h, _ptr(g), _ptr(G), _ptr(dL_dphi), _ptr(dL_df), _ptr(dL_dpsi),
                             int(checkpoint_every), _ptr(dg), _ptr(dG)), "fot_backward")
    return dg, dG


class FOTPhase(torch.autograd.Function):
    """phi (and the final potentials f, psi) of Algorithm 1 as a differentiable function of the
    amplitudes g, G: forward = fot_solve + fot_phase, backward = fot_backward (hand-written
    adjoint kernels through the unrolled iterations, checkpointed)."""

    @staticmethod
    def forward(fctx, g, G, eps, iters, dx, precision, checkpoint_every):
        g = g.detach().contiguous().float()
        G = G.detach().contiguous().float()
        ctx = fot_create(g.shape[0], g.shape[1], precision, g.device.index)
        fot_solve(ctx, g, G, eps, iters, dx)
        phi, _, _ = fot_phase(ctx)
        f, psi = fot_potentials(ctx)
        fctx.fot = ctx
        fctx.k = checkpoint_every
        fctx.save_for_backward(g, G)
        return phi, f, psi

    @staticmethod
    def backward(fctx, dphi, df, dpsi):
        g, G = fctx.saved_tensors
        c = lambda t: None if t is None else t.contiguous().float()
        dg, dG = fot_backward(fctx.fot, g, G, c(dphi), c(df), c(dpsi), fctx.k)
        fctx.fot.close()
        return dg, dG, None, None, None, None, None


def fot_phase_fn(g, G, eps, iters, dx=0.0, precision=FOT_FP32, checkpoint_every=10):
    return FOTPhase.apply(g, G, eps, iters, dx, precision, checkpoint_every)


def exported_symbols():
    return list(_SIGS)
