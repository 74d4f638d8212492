"""Shared-shape variant on the GPU (one shape draw per step, profiles as
phase-profile contractions on the tensor cores) against the FP64 oracle fed
the same tied noise: profile, likelihood, ELBO and gradient at the plain
path's tolerances, fit steps, the K=50 workload at full K and N, recovery."""
import numpy as np
import pytest

import oracle
from paper_2501_09308_gb300 import synth, xrdvi

pytestmark = pytest.mark.gpu

F_TOL = 1e-5
G_TOL = 1e-4


def _compare(inst, S, seed):
    ctx = xrdvi.Context.from_instance(inst, S=S, flags=xrdvi.FLAG_SHARED_SHAPES)
    loc, raw = ctx.params()
    rng = np.random.default_rng(seed)
    loc = loc + rng.normal(0, 0.05, loc.shape).astype(np.float32)
    raw = raw + rng.normal(0, 0.1, raw.shape).astype(np.float32)
    ctx.set_params(loc, raw)
    eps = synth.normals(3000 + seed, S, inst.K)
    g = ctx.elbo_grad(eps, want_f=True)
    ctx.close()
    P = oracle.Problem.from_instance(inst, shapes="shared")
    o = P.elbo_grad(loc.astype(np.float64), raw.astype(np.float64), eps.astype(np.float64), want_f=True)
    return g, o


def _check(g, o):
    rf = float(np.max(np.abs(g["f"] - o["f"]) / np.abs(o["f"])))
    np.testing.assert_allclose(g["ll"], o["ll"], rtol=F_TOL)
    assert abs(g["elbo"] - o["elbo"]) <= F_TOL * abs(o["elbo"])
    gerr = 0.0
    for b in range(10):
        ref = np.max(np.abs(o["grad"][:, b]))
        err = np.max(np.abs(g["grad"][:, b] - o["grad"][:, b]))
        gerr = max(gerr, err / ref)
        assert err <= G_TOL * ref, (b, err, ref)
    assert rf <= F_TOL, rf
    return rf, gerr


@pytest.mark.parametrize("K,M,N,S,seed", [
    (3, 6, 300, 4, 1),       # ragged tail, one row tile of the GEMMs
    (8, 20, 1000, 8, 2),
    (1, 1, 1, 1, 3),         # a single point, peak and sample
    (5, 12, 512, 130, 4),    # two row tiles (S > 128), ragged
    (40, 30, 2000, 64, 5),   # 400 backward GEMM columns (7 tiles), split-K
])
def test_shared_shape_parity(K, M, N, S, seed):
    inst = synth.small_problem(K=K, M=M, N=N, S=S, seed=seed, x_step=max(0.02, 15.0 / N))
    rf, gerr = _check(*_compare(inst, S, seed))
    print(f"\nshared K={K} N={N} S={S}: f {rf:.2e}, grad {gerr:.2e}")


def test_shared_shape_parity_k50_full_size():
    """The K=50, N=4500 workload (all 2194 peaks, all points) at S = 16."""
    inst = synth.config(1)
    rf, gerr = _check(*_compare(inst, 16, 9))
    print(f"\nshared K=50 N=4500 S=16: f {rf:.2e}, grad {gerr:.2e}")


def test_shared_shape_fit_steps_match_oracle():
    inst = synth.small_problem(K=3, M=6, N=300, S=8, seed=14)
    ctx = xrdvi.Context.from_instance(inst, S=8, seed=4242, flags=xrdvi.FLAG_SHARED_SHAPES)
    loc0, raw0 = ctx.params()
    trace = ctx.fit(3)
    loc1, raw1 = ctx.params()
    ctx.close()
    ref = oracle.Problem.from_instance(inst, shapes="shared").fit(8, 3, 4242, loc=loc0.astype(np.float64),
                                                                   raw=raw0.astype(np.float64))
    np.testing.assert_allclose(trace, ref["trace"], rtol=F_TOL)
    np.testing.assert_allclose(loc1, ref["loc"], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(raw1, ref["raw"], rtol=1e-5, atol=1e-5)


def test_shared_shape_fit_recovers_planted_phases():
    inst = synth.config(1)
    c = xrdvi.Context.from_instance(inst, S=inst.S, seed=3, flags=xrdvi.FLAG_SHARED_SHAPES)
    c.fit(inst.iters)
    post = c.posterior(4096, 77, top_m=1)
    c.close()
    print(f"\nshared-shape K=50 fit: top combination {np.flatnonzero(post['combos'][0]).tolist()}, "
          f"planted {inst.planted.tolist()}")
    assert set(np.flatnonzero(post["combos"][0]).tolist()) == set(inst.planted.tolist())
