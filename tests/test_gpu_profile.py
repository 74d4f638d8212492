"""The per-kernel profiler (xrdvi_profile_kernels): its timings and the
evaluation counts the bench's roofline divides by.

Counts are checked against what they must satisfy by construction: on the
all-direct path every (sample, peak, tile point) is one side-uniform or mixed
evaluation; the backward's Gaussian terms (evaluated on 64-point blocks within
a peak's reach) are whole blocks and never exceed the evaluations they are
drawn from."""
import numpy as np
import pytest

from paper_2501_09308_gb300 import synth, xrdvi

pytestmark = pytest.mark.gpu

KTILE = 256


def _profile(inst, S, flags=0, steps=3):
    ctx = xrdvi.Context.from_instance(inst, S=S, flags=flags)
    ctx.fit(2, trace=False)
    km, work = ctx.profile_kernels(steps)
    ctx.close()
    return km, work


def _common(work):
    assert set(work) == set(xrdvi.WORK_COUNTS)
    assert all(v >= 0 for v in work.values())
    assert work["mixed_gauss_bwd"] % 64 == 0 and work["gauss_reach_bwd"] % 64 == 0
    assert work["mixed_gauss_bwd"] <= work["mixed"]
    assert work["gauss_reach_bwd"] <= work["gauss_reach"]


def test_dense_path_counts_every_peak_at_every_tile_point():
    inst = synth.small_problem(K=4, M=12, N=1200, S=4, seed=31, x_step=0.03)
    km, work = _profile(inst, 4, xrdvi.FLAG_DENSE)
    _common(work)
    T = -(-inst.N // KTILE)
    assert work["uniform"] + work["mixed"] == 4 * int(inst.offsets[-1]) * T * KTILE
    assert work["far_nodes"] == 0
    for slot in ("sample", "ranges", "direct", "lik", "bwd_uniform", "bwd_near", "grad_adam", "elbo"):
        assert km[slot] > 0.0, slot


def test_far_field_path_counts():
    inst = synth.small_problem(K=20, M=40, N=4500, S=4, seed=32, x_lo=10.0, x_step=0.02)
    km, work = _profile(inst, 4)
    _common(work)
    T = -(-inst.N // KTILE)
    assert work["far_nodes"] > 0
    # the direct part is a small fraction of the dense sum, and the mixed
    # range's Gaussian blocks a fraction of the mixed evaluations
    assert work["uniform"] + work["mixed"] < 4 * int(inst.offsets[-1]) * T * KTILE // 3
    assert 0 < work["mixed_gauss_bwd"] < work["mixed"]
    for slot in ("sample", "ranges", "direct", "lik", "bwd_uniform", "grad_adam", "elbo"):
        assert km[slot] > 0.0, slot
