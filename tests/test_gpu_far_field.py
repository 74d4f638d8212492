"""The far-field evaluation (Lorentzian tails of peaks beyond half a tile
width of a 256-point tile summed at 32 Chebyshev nodes and interpolated)
against the FP64 oracle's dense sum, and against the library's own
all-direct path (XRDVI_FLAG_DENSE).

Tolerances against the oracle are the plain path's (profile, LL, ELBO 1e-5
relative; gradient blocks 1e-4 of their max-norm).  Between the two GPU
paths the interpolation error (below 1e-8 of the tails) and FP32 rounding
in a different order remain: profile 2e-6 relative, gradient blocks 2e-5."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2501_09308_gb300 import synth, xrdvi

pytestmark = pytest.mark.gpu

F_TOL = 1e-5
G_TOL = 1e-4


def _params(ctx, seed):
    loc, raw = ctx.params()
    rng = np.random.default_rng(seed)
    loc = loc + rng.normal(0, 0.05, loc.shape).astype(np.float32)
    raw = raw + rng.normal(0, 0.1, raw.shape).astype(np.float32)
    ctx.set_params(loc, raw)
    return loc, raw


def _gpu(inst, S, seed, flags=0):
    ctx = xrdvi.Context.from_instance(inst, S=S, flags=flags)
    loc, raw = _params(ctx, seed)
    eps = synth.normals(5000 + seed, S, inst.K)
    g = ctx.elbo_grad(eps, want_f=True)
    ctx.close()
    return g, loc, raw, eps


def _against_oracle(inst, S, seed, flags=0, **okw):
    g, loc, raw, eps = _gpu(inst, S, seed, flags)
    o = oracle.Problem.from_instance(inst, **okw).elbo_grad(
        loc.astype(np.float64), raw.astype(np.float64), eps.astype(np.float64), want_f=True)
    rel = np.abs(g["f"] - o["f"]) / np.abs(o["f"])
    gerr = [float(np.max(np.abs(g["grad"][:, b] - o["grad"][:, b])) / np.max(np.abs(o["grad"][:, b])))
            for b in range(10)]
    print(f"\n{inst.name}: max rel f error {rel.max():.2e}, max gradient block error {max(gerr):.2e}")
    assert rel.max() <= F_TOL
    np.testing.assert_allclose(g["ll"], o["ll"], rtol=F_TOL)
    assert abs(g["elbo"] - o["elbo"]) <= F_TOL * abs(o["elbo"])
    assert max(gerr) <= G_TOL


@pytest.mark.parametrize("K,M,N,S,seed", [(20, 40, 4500, 4, 1), (6, 60, 2600, 6, 2), (12, 30, 9000, 2, 3)])
def test_far_field_parity_many_tiles(K, M, N, S, seed):
    inst = synth.small_problem(K=K, M=M, N=N, S=S, seed=seed, x_lo=10.0, x_step=90.0 / N)
    _against_oracle(inst, S, seed)


def test_far_field_matches_the_dense_path():
    inst = synth.small_problem(K=20, M=40, N=4500, S=4, seed=4, x_lo=10.0, x_step=0.02)
    a = _gpu(inst, 4, 4)[0]
    b = _gpu(inst, 4, 4, xrdvi.FLAG_DENSE)[0]
    assert np.max(np.abs(a["f"] - b["f"]) / b["f"]) <= 2e-6
    for blk in range(10):
        ref = np.max(np.abs(b["grad"][:, blk]))
        assert np.max(np.abs(a["grad"][:, blk] - b["grad"][:, blk])) <= 2e-5 * ref, blk


def test_far_field_with_angle_dependent_width():
    inst = synth.small_problem(K=8, M=30, N=3000, S=4, seed=5, x_lo=40.0, x_step=0.035)
    _against_oracle(inst, 4, 5, xrdvi.FLAG_SEC_WIDTH, width="sec")


def test_far_field_on_a_non_uniform_grid_with_a_one_point_tile():
    """Grid spacing varying by a factor of three, and N = 2305 = 9 tiles + 1:
    the last tile's span is a single point."""
    inst = synth.small_problem(K=10, M=30, N=2305, S=3, seed=6, x_lo=15.0, x_step=0.03)
    u = np.linspace(0.0, 1.0, inst.N)
    x = (15.0 + 70.0 * (u + 0.25 * np.sin(2 * np.pi * u) / (2 * np.pi) * 2.0)).astype(np.float32)
    assert np.all(np.diff(x) > 0)
    inst = dataclasses.replace(inst, x=x, name="nonuniform_N2305")
    _against_oracle(inst, 3, 6)


def test_far_field_fit_steps_match_the_oracle():
    inst = synth.small_problem(K=6, M=30, N=3000, S=8, seed=7, x_lo=10.0, x_step=0.03)
    ctx = xrdvi.Context.from_instance(inst, S=8, seed=4245)
    loc0, raw0 = ctx.params()
    trace = ctx.fit(3)
    loc1, raw1 = ctx.params()
    ctx.close()
    ref = oracle.Problem.from_instance(inst).fit(8, 3, 4245, loc=loc0.astype(np.float64),
                                                 raw=raw0.astype(np.float64))
    np.testing.assert_allclose(trace, ref["trace"], rtol=F_TOL)
    np.testing.assert_allclose(loc1, ref["loc"], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(raw1, ref["raw"], rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("K,M,N,S,seed,flags,okw", [
    (3, 6, 300, 4, 11, 0, {}),
    (8, 20, 2600, 8, 12, 0, {}),
    (1, 1, 1, 1, 13, 0, {}),
    (6, 30, 3000, 4, 14, xrdvi.FLAG_SEC_WIDTH, {"width": "sec"}),
    (5, 12, 1500, 4, 15, xrdvi.FLAG_NAIVE_SUM, {}),
])
def test_dense_path_parity(K, M, N, S, seed, flags, okw):
    """XRDVI_FLAG_DENSE (every peak at every point: k_forward, k_bwd_uniform,
    k_bwd_near) against the oracle."""
    inst = synth.small_problem(K=K, M=M, N=N, S=S, seed=seed, x_lo=40.0 if flags & xrdvi.FLAG_SEC_WIDTH else 10.0,
                               x_step=max(0.02, 40.0 / N))
    _against_oracle(inst, S, seed, xrdvi.FLAG_DENSE | flags, **okw)


def test_dense_path_fit_steps_match_the_oracle():
    inst = synth.small_problem(K=4, M=12, N=1200, S=8, seed=16, x_lo=10.0, x_step=0.03)
    ctx = xrdvi.Context.from_instance(inst, S=8, seed=4246, flags=xrdvi.FLAG_DENSE)
    loc0, raw0 = ctx.params()
    trace = ctx.fit(3)
    loc1, raw1 = ctx.params()
    ctx.close()
    ref = oracle.Problem.from_instance(inst).fit(8, 3, 4246, loc=loc0.astype(np.float64),
                                                 raw=raw0.astype(np.float64))
    np.testing.assert_allclose(trace, ref["trace"], rtol=F_TOL)
    np.testing.assert_allclose(loc1, ref["loc"], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(raw1, ref["raw"], rtol=1e-5, atol=1e-5)
