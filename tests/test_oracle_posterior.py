"""Pins of the oracle's posterior over phase combinations and of planted-phase
recovery by the oracle's own SVI fit (no GPU)."""
import itertools
import math

import numpy as np
import pytest
from scipy import special

import oracle
from oracle import posterior as post
from paper_2501_09308_gb300 import synth


def test_logsumexp_against_library():
    rng = np.random.default_rng(1)
    a = rng.normal(scale=300, size=1000)
    assert post.logsumexp(a) == pytest.approx(special.logsumexp(a), rel=1e-14)


@pytest.mark.parametrize("K", [1, 5, 10])
def test_product_form_normalises_over_all_combinations(K):
    """The mean-field combination probabilities sum to one over all 2^K sets."""
    rng = np.random.default_rng(K)
    pi = rng.uniform(0.001, 0.999, size=K)
    assert abs(post.logsumexp(post.all_combination_logp(pi))) < 1e-12


@pytest.mark.parametrize("K,M", [(6, 64), (10, 40), (12, 25)])
def test_top_combinations_against_brute_force(K, M):
    rng = np.random.default_rng(100 + K)
    pi = rng.uniform(0.01, 0.99, size=K)
    pi[0] = 0.5  # a tie in cost between including and excluding phase 0
    combos, lp = post.top_combinations(pi, M)
    allp = post.all_combination_logp(pi)
    want = np.sort(allp)[::-1][:M]
    np.testing.assert_allclose(lp, want, rtol=0, atol=1e-12)
    assert np.all(np.diff(lp) <= 1e-12)
    # each reported set is a valid, distinct combination with the stated probability
    codes = set()
    for c, l in zip(combos, lp):
        code = int(np.sum(c.astype(np.int64) << np.arange(K)))
        codes.add(code)
        assert allp[code] == pytest.approx(l, abs=1e-12)
    assert len(codes) == len(lp)


def test_area_ratio_bits_and_marginals():
    """Area-ratio identification (1 % threshold) and the smoothed marginals."""
    areas = np.array([[10.0, 0.05, 5.0], [10.0, 0.2, 0.0]])
    bits = post.inclusion_bits(areas)
    np.testing.assert_array_equal(bits, [[True, False, True], [True, True, False]])
    np.testing.assert_allclose(post.marginal_pi(bits), [(2.5) / 3, 1.5 / 3, 1.5 / 3])


@pytest.mark.slow
def test_oracle_fit_recovers_planted_phases():
    """Synthetic analogue of the paper's identification result: the planted
    phases end above the 1 % area ratio in most posterior samples, every
    decoy below it (sparse prior shrinks non-present phases)."""
    inst = synth.make_problem(K=4, m_lo=8, m_hi=12, x_lo=20.0, x_step=0.04, N=800,
                              n_planted=2, S=8, iters=300, seed=11, name="t")
    P = oracle.Problem.from_instance(inst)
    fit = P.fit(8, 300, seed=3)
    assert fit["trace"][-1] > fit["trace"][0]
    res = post.posterior(P, fit["loc"], fit["raw"], 256, seed=9, top_m=4)
    planted = set(inst.planted.tolist())
    for k in range(P.K):
        if k in planted:
            assert res["pi"][k] > 0.9
        else:
            assert res["pi"][k] < 0.1
    top = res["combos"][0]
    assert set(np.flatnonzero(top).tolist()) == planted


@pytest.mark.slow
def test_exhaustive_enumeration_small_K():
    """For small K every sub-model is fitted; the evidence-ranked top
    combination is the planted one and agrees with the sparse fit's mode."""
    inst = synth.make_problem(K=3, m_lo=6, m_hi=8, x_lo=20.0, x_step=0.05, N=500,
                              n_planted=2, S=4, iters=200, seed=21, name="e")
    arrays = (inst.offsets, inst.pos, inst.inten, inst.x, inst.y, inst.bg)
    masks, elbos, p = post.enumerate_submodels(arrays, S=8, iters=1000, seed=5)
    assert abs(post.logsumexp(elbos - post.logsumexp(elbos))) < 1e-12
    best = masks[int(np.argmax(p))]
    assert set(np.flatnonzero(best).tolist()) == set(inst.planted.tolist())
    P = oracle.Problem.from_instance(inst)
    fit = P.fit(8, 1000, seed=5)
    res = post.posterior(P, fit["loc"], fit["raw"], 128, seed=2, top_m=1)
    np.testing.assert_array_equal(res["combos"][0], best)
