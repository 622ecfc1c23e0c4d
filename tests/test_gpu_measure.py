"""Measurement entry points on the GPU: per-kernel-class loop timing and the work split
(what the benchmark's roofline is computed from)."""
import numpy as np
import pytest

from paper_2512_19072_gb300 import inputs
from fot_testutil import f32, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "mixed", "dense"])
def test_kernel_times_cover_the_loop(fot_lib, prec):
    B = fot_lib
    P = {"fp32": B.FOT_FP32, "mixed": B.FOT_MIXED, "dense": B.FOT_FP32_DENSE}[prec]
    w = inputs.config3(256, iters=20)
    g, G = to_dev(f32(w.g)), to_dev(f32(w.G))
    ctx = B.fot_create(256, 256, P)
    with pytest.raises(B.FotError):
        B.fot_kernel_times(ctx)                    # timing off: FOT_ESTATE
    B.fot_set_kernel_timing(ctx, True)
    B.fot_solve(ctx, g, G, w.eps, w.iters)
    times = B.fot_kernel_times(ctx)
    loop_ms, loop_launches = B.fot_loop_time(ctx)
    launches = sum(n for _, n in times.values())
    ms = sum(t for t, _ in times.values())
    assert launches == loop_launches, (times, loop_launches)
    assert 0.0 < ms <= loop_ms * 1.001 + 1e-3, (ms, loop_ms)
    if prec == "dense":
        assert times["axis_pass_kernel"][1] == 4 * w.iters
    elif prec == "fp32":
        assert times["band_plan_kernel"][1] == 4 * w.iters
    else:
        # the plan class also holds the B-operand table writes: one whenever eps changes
        n_eps = len(set(np.asarray(w.eps, dtype=float).tolist()))
        assert 4 * w.iters < times["band_plan_kernel"][1] <= 4 * w.iters + n_eps
    # the sums reset on reading; a second solve is timed alone
    assert sum(n for _, n in B.fot_kernel_times(ctx).values()) == 0
    B.fot_solve(ctx, g, G, w.eps, w.iters)
    assert sum(n for _, n in B.fot_kernel_times(ctx).values()) == loop_launches
    B.fot_set_kernel_timing(ctx, False)
    ctx.close()


def test_work_split_adds_up(fot_lib):
    B = fot_lib
    w = inputs.config3(256, iters=10)
    for P in (B.FOT_FP32, B.FOT_MIXED, B.FOT_FP32_DENSE):
        ctx = B.fot_create(256, 256, P)
        B.fot_solve(ctx, to_dev(f32(w.g)), to_dev(f32(w.G)), w.eps, w.iters)
        split = B.fot_work_split(ctx)
        total, tensor = B.fot_work_count(ctx, tensor=True)
        assert sum(split) == total and split[2] == tensor
        assert all(v >= 0 for v in split)
        if P == B.FOT_FP32_DENSE:
            assert split[:3] == (0, 0, 0) and split[3] == 4 * w.iters * 256 ** 3
        else:
            assert split[3] == 0 and split[0] + split[1] > 0
        ctx.close()
