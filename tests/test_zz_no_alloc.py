"""The allocation-free u-update (fot_u_update_noalloc) against the context-based
fot_u_update, through the C ABI.

fot_u_update_noalloc is for callers that must not allocate device memory while they
run (a real-time loop that reserved its memory at start-up, a plug-in whose host owns
all device allocations); it keeps its intermediate in a static device array instead.
This file sorts last so that a run stopping at the first failure has run every other
test first.
"""
import gc

import numpy as np
import pytest
import torch

from paper_2512_19072_gb300 import inputs
from fot_testutil import POT_RTOL, assert_pot_close, f32, normwise, to_dev, to_np

pytestmark = pytest.mark.gpu


def _log_marginal(g):
    g = torch.as_tensor(g, dtype=torch.float64)
    la = 2.0 * torch.log(g) - torch.log((g * g).sum())
    return la.float().cuda().contiguous()


@pytest.mark.parametrize("shape,eps", [((96, 130), 2.5), ((1024, 1024), 209.7)])
def test_noalloc_matches_context_entry_point(fot_lib, shape, eps):
    B = fot_lib
    rng = np.random.default_rng(17)
    g = f32(rng.uniform(0.05, 1.0, size=shape))
    g[rng.uniform(size=shape) < 0.1] = 0.0
    G = f32(rng.uniform(0.05, 1.0, size=shape))
    n = max(shape)
    ctx = B.fot_create(*shape)
    B.fot_set_problem(ctx, to_dev(g), to_dev(G))
    la = _log_marginal(g)
    for call, seed in enumerate((31, 32)):          # two calls in a row share the scratch
        psi = to_dev(f32(inputs.random_potential(*shape, scale=0.3 * n * n, seed=seed, zero_frac=0.1)))
        f_ref, S_ref = B.fot_u_update(ctx, psi, eps * (1 + call), with_logsum=True)
        f = torch.full(shape, float("nan"), device="cuda")
        S = torch.full(shape, float("nan"), device="cuda")
        B.fot_u_update_noalloc(psi, la, eps * (1 + call), f_out=f, logsum_out=S)
        torch.cuda.synchronize()
        assert_pot_close(to_np(f), to_np(f_ref), rtol=POT_RTOL, what=f"f (call {call})")
        assert normwise(to_np(S), to_np(S_ref)) <= POT_RTOL
    ctx.close()


def test_noalloc_rejects_oversize(fot_lib):
    B = fot_lib
    big = torch.zeros(1, 1, device="cuda")
    with pytest.raises(B.FotError) as e:
        B._check(B._lib.fot_u_update_noalloc(B._ptr(big), B._ptr(big), 1025, 1024, 1.0,
                                             B._ptr(big), None, B._stream()), "noalloc")
    assert e.value.status == 1                      # FOT_EINVAL, nothing launched


def test_noalloc_allocates_nothing(fot_lib):
    """The entry point's contract: after a first call (the one-time set-up and the lazy
    loading of its kernels), further calls change neither the device's free memory nor
    torch's allocator state."""
    B = fot_lib
    shape, eps = (1024, 1024), 209.7
    rng = np.random.default_rng(23)
    g = f32(rng.uniform(0.05, 1.0, size=shape))
    la = _log_marginal(g)
    psi = to_dev(f32(inputs.random_potential(*shape, scale=0.3 * 1024 * 1024, seed=41, zero_frac=0.1)))
    f = torch.empty(shape, device="cuda")
    S = torch.empty(shape, device="cuda")
    B.fot_u_update_noalloc(psi, la, eps, f_out=f, logsum_out=S)     # warm-up
    torch.cuda.synchronize()
    # tensors left by earlier tests must not be collected (freed) inside the measured window
    gc.collect()
    gc.disable()
    try:
        free0, _ = torch.cuda.mem_get_info()
        alloc0 = torch.cuda.memory_allocated()
        for _ in range(3):
            B.fot_u_update_noalloc(psi, la, eps, f_out=f, logsum_out=S)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        alloc1 = torch.cuda.memory_allocated()
    finally:
        gc.enable()
    assert alloc1 == alloc0
    assert free1 == free0, (free0, free1)
    assert torch.isfinite(f[torch.isfinite(la)]).all()
