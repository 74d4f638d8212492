"""Pins of the oracle's estimator and likelihood variants (no GPU): the
Gaussian likelihood against scipy's normal density and central differences;
the importance-weighted bound (Burda et al., ICLR 2016) against its
definition written with scipy, its one-draw reduction, central differences,
the posterior module's importance-sampled evidence and the gamma-Poisson
closed form."""
import math

import numpy as np
import pytest
from scipy import special, stats

import oracle
from oracle import posterior as post
from paper_2501_09308_gb300 import synth

from test_oracle_elbo import _conjugate_setup


def _fd_grad(P, loc, raw, eps, h=1e-6):
    num = np.zeros((P.K, 10))
    for k in range(P.K):
        for j in range(5):
            for which in (0, 1):
                L, R = loc.copy(), raw.copy()
                A = L if which == 0 else R
                A[k, j] += h
                ep = P.elbo_grad(L, R, eps)["elbo"]
                A[k, j] -= 2 * h
                em = P.elbo_grad(L, R, eps)["elbo"]
                num[k, j + 5 * which] = (ep - em) / (2 * h)
    return num


def _perturbed(P, seed):
    loc, raw = P.init_params()
    rng = np.random.default_rng(seed)
    return loc + rng.normal(0, 0.05, loc.shape), raw + rng.normal(0, 0.1, raw.shape)


def _problem(**kw):
    inst = synth.small_problem(K=3, M=6, N=240, seed=4)
    return inst, oracle.Problem.from_instance(inst, **kw)


def test_gaussian_loglik_is_the_normal_density_with_variance_max_y_1():
    inst, P = _problem(likelihood="gauss")
    rng = np.random.default_rng(1)
    f = P.y + rng.normal(0, 30.0, P.N) + 5.0
    ref = stats.norm.logpdf(P.y, loc=f, scale=np.sqrt(np.maximum(P.y, 1.0))).sum()
    assert P.loglik(f, "gauss") == pytest.approx(ref, rel=1e-12)


def test_gaussian_likelihood_terms_and_gradient():
    """The per-draw LL is the Gaussian log density at the draw's profile, and
    the analytic gradient matches FP64 central differences (h = 1e-6)."""
    inst, P = _problem(likelihood="gauss")
    loc, raw = _perturbed(P, 2)
    eps = synth.normals(7, 2, P.K).astype(np.float64)
    r = P.elbo_grad(loc, raw, eps, want_f=True)
    for s in range(2):
        assert r["ll"][s] == pytest.approx(P.loglik(r["f"][s], "gauss"), rel=1e-12)
    num = _fd_grad(P, loc, raw, eps)
    rel = np.max(np.abs(num - r["grad"]), axis=0) / np.max(np.abs(r["grad"]), axis=0)
    assert np.all(rel < 1e-5), rel


def test_iw_bound_is_its_definition():
    """L_S = logsumexp_s(ln p(Y, theta_s) + ln|J_s| - ln q(u_s)) - ln S, with
    ln q written as scipy normal log densities of u = loc + sigma eps."""
    inst, P = _problem(objective="iw")
    loc, raw = _perturbed(P, 3)
    eps = synth.normals(8, 6, P.K).astype(np.float64)
    r = P.elbo_grad(loc, raw, eps)
    sig = np.logaddexp(0.0, raw)
    u = loc[None] + sig[None] * eps
    lq = stats.norm.logpdf(u, loc=loc[None], scale=sig[None]).sum(axis=(1, 2))
    lw = r["ll"] + r["lpj"] - lq
    assert r["elbo"] == pytest.approx(special.logsumexp(lw) - math.log(6), rel=1e-12)
    # Jensen: the bound is above the mean log weight
    assert r["elbo"] >= np.mean(lw)


def test_iw_gradient_at_one_draw_is_the_elbo_gradient():
    """With one draw the weight is 1 and -ln q differs from the analytic
    entropy by a constant in loc and by the same 1/sigma in raw, so the two
    objectives have the same gradient."""
    inst, P_iw = _problem(objective="iw")
    P_e = oracle.Problem.from_instance(inst)
    loc, raw = _perturbed(P_e, 4)
    eps = synth.normals(9, 1, P_e.K).astype(np.float64)
    np.testing.assert_allclose(P_iw.elbo_grad(loc, raw, eps)["grad"], P_e.elbo_grad(loc, raw, eps)["grad"],
                               rtol=1e-12, atol=1e-12)


def test_iw_gradient_against_central_differences():
    inst, P = _problem(objective="iw")
    loc, raw = _perturbed(P, 5)
    eps = synth.normals(10, 4, P.K).astype(np.float64)
    g = P.elbo_grad(loc, raw, eps)["grad"]
    num = _fd_grad(P, loc, raw, eps)
    rel = np.max(np.abs(num - g), axis=0) / np.max(np.abs(g), axis=0)
    assert np.all(rel < 1e-5), rel


def test_iw_bound_between_elbo_and_evidence_in_the_conjugate_case():
    """Gamma-Poisson case with q shifted 1.5 posterior standard deviations off:
    the ELBO is well below the closed-form ln p(Y), the importance-weighted
    bound with 2048 draws is within a few hundredths of it, and it equals the
    posterior module's importance-sampled evidence for the same draws."""
    P, loc, raw, lnZ, fixed_lpj, fixed_H, sig0 = _conjugate_setup()
    loc = loc.copy()
    loc[0, 0] += 1.5 / math.sqrt(P.y.sum())
    rng = np.random.default_rng(12)
    S = 2048
    eps = np.zeros((S, 1, 5))
    eps[:, 0, 0] = rng.standard_normal(S)
    P_iw = oracle.Problem(P.off, P.pos, P.inten, P.x, P.y, P.bg, objective="iw")
    lq_fixed = 4 * (-math.log(sig0) - 0.5 * math.log(2 * math.pi))
    l_iw = P_iw.elbo_grad(loc, raw, eps)["elbo"] - fixed_lpj + lq_fixed
    l_elbo = P.elbo_grad(loc, raw, eps)["elbo"] - fixed_lpj - fixed_H
    assert lnZ - l_elbo > 0.5
    assert abs(lnZ - l_iw) < 0.05
    res = post.posterior(P, loc, raw, S, eps=eps, top_m=1)
    assert P_iw.elbo_grad(loc, raw, eps)["elbo"] == pytest.approx(res["log_evidence"], rel=1e-12)


def test_shared_shape_noise_ties_the_shape_columns_to_sample_zero():
    """The shared-shape estimator is the plain one on noise whose shape
    columns (mu, w, r, alpha) are sample 0's and whose intensity column is
    each sample's own; with one sample nothing changes."""
    inst, P = _problem()
    P_sh = oracle.Problem.from_instance(inst, shapes="shared")
    loc, raw = _perturbed(P, 6)
    eps = synth.normals(11, 5, P.K).astype(np.float64)
    tied = eps.copy()
    tied[1:, :, 1:] = eps[0, :, 1:]
    a, b = P_sh.elbo_grad(loc, raw, eps), P.elbo_grad(loc, raw, tied)
    assert a["elbo"] == b["elbo"]
    np.testing.assert_array_equal(a["grad"], b["grad"])
    one = eps[:1]
    assert P_sh.elbo_grad(loc, raw, one)["elbo"] == P.elbo_grad(loc, raw, one)["elbo"]


def test_shared_shape_estimator_is_unbiased():
    """Averaged over independent noise, the shared-shape estimate of the
    ELBO and of its gradient agrees with the plain estimator's average (both
    estimate the same expectation) within four standard errors."""
    inst, P = _problem()
    P_sh = oracle.Problem.from_instance(inst, shapes="shared")
    loc, raw = _perturbed(P, 7)
    rng = np.random.default_rng(13)
    R, S = 300, 4
    vals = {"plain": [], "shared": []}
    grads = {"plain": [], "shared": []}
    for _ in range(R):
        eps = rng.standard_normal((S, P.K, 5))
        for name, Q in (("plain", P), ("shared", P_sh)):
            r = Q.elbo_grad(loc, raw, eps)
            vals[name].append(r["elbo"])
            grads[name].append(r["grad"])
    for name in ("plain", "shared"):
        vals[name] = np.array(vals[name])
        grads[name] = np.array(grads[name])
    se = math.sqrt(np.var(vals["plain"]) / R + np.var(vals["shared"]) / R)
    assert abs(vals["plain"].mean() - vals["shared"].mean()) <= 4 * se
    gse = np.sqrt(np.var(grads["plain"], axis=0) / R + np.var(grads["shared"], axis=0) / R)
    z = np.abs(grads["plain"].mean(axis=0) - grads["shared"].mean(axis=0)) / np.maximum(gse, 1e-300)
    assert np.mean(z <= 4) >= 0.97, np.sort(z.ravel())[-5:]


def test_sec_width_factor_is_secant_of_half_two_theta():
    """theta is half the diffraction angle 2-theta (given in degrees): at
    2-theta = 120 deg the width doubles, at 90 deg it grows by sqrt(2)."""
    lib = oracle.lib()
    assert lib.orc_sec(120.0) == pytest.approx(2.0, rel=1e-14)
    assert lib.orc_sec(90.0) == pytest.approx(math.sqrt(2.0), rel=1e-14)
    assert lib.orc_sec(1e-6) == pytest.approx(1.0, abs=1e-12)


def test_sec_width_profile_against_library_densities():
    """One asymmetric peak near 2-theta = 110 deg: at every point the profile
    is scipy's normal and Cauchy densities (scaled to unit height) with the
    side's FWHM times sec(x / 2) of that point."""
    x = np.linspace(108.0, 112.0, 401)
    P = oracle.Problem([0, 1], [110.0], [0.8], x, np.ones_like(x), np.zeros_like(x), width="sec")
    h, mu, w, r, al = 3.0, 0.02, 0.3, 0.4, 1.7
    f = P.profile(np.array([[[h, mu, w, r, al]]]))[0]
    d = x - (110.0 + mu)
    fwhm = np.where(d >= 0, al * w, w) / np.cos(np.radians(x / 2.0))
    sd = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    G = stats.norm.pdf(d, scale=sd) / stats.norm.pdf(0.0, scale=sd)
    L = stats.cauchy.pdf(d, scale=fwhm / 2.0) / stats.cauchy.pdf(0.0, scale=fwhm / 2.0)
    np.testing.assert_allclose(f, h * 0.8 * ((1 - r) * G + r * L), rtol=1e-12, atol=1e-14)


def test_sec_width_gradient_against_central_differences():
    inst = synth.small_problem(K=3, M=6, N=240, seed=4, x_lo=70.0, x_step=0.1)
    P = oracle.Problem.from_instance(inst, width="sec")
    loc, raw = _perturbed(P, 8)
    eps = synth.normals(12, 2, P.K).astype(np.float64)
    g = P.elbo_grad(loc, raw, eps)["grad"]
    num = _fd_grad(P, loc, raw, eps)
    rel = np.max(np.abs(num - g), axis=0) / np.max(np.abs(g), axis=0)
    assert np.all(rel < 1e-5), rel


def test_fitted_background_curve_is_a_chebyshev_exponential():
    """B(beta) = B exp(sum_j beta_j T_j(z)) with numpy's Chebyshev series and z
    the grid mapped onto [-1, 1]."""
    inst, P = _problem(background="fitted")
    beta = np.array([0.08, -0.05, 0.02])
    z = 2.0 * (P.x - P.x[0]) / (P.x[-1] - P.x[0]) - 1.0
    ref = P.bg * np.exp(np.polynomial.chebyshev.chebval(z, beta))
    np.testing.assert_allclose(P.background(beta), ref, rtol=1e-13)


def test_fitted_background_at_zero_is_the_fixed_model_plus_its_prior():
    inst, P_fit = _problem(background="fitted", bg_sd=0.1)
    P = oracle.Problem.from_instance(inst)
    loc, raw = _perturbed(P, 9)
    eps = synth.normals(13, 3, P.K).astype(np.float64)
    a, b = P_fit.elbo_grad(loc, raw, eps), P.elbo_grad(loc, raw, eps)
    lpb = 3 * stats.norm.logpdf(0.0, scale=0.1)
    assert a["elbo"] == pytest.approx(b["elbo"] + lpb, rel=1e-13)
    np.testing.assert_allclose(a["grad"], b["grad"], rtol=1e-12, atol=1e-12)


def test_fitted_background_gradient_against_central_differences():
    inst, P = _problem(background="fitted", bg_sd=0.1)
    loc, raw = _perturbed(P, 10)
    eps = synth.normals(14, 3, P.K).astype(np.float64)
    P.beta[:] = [0.03, -0.02, 0.01]
    g = P.elbo_grad(loc, raw, eps)["grad_beta"]
    num = np.zeros(3)
    for j in range(3):
        b0 = P.beta[j]
        P.beta[j] = b0 + 1e-6
        ep = P.elbo_grad(loc, raw, eps)["elbo"]
        P.beta[j] = b0 - 1e-6
        em = P.elbo_grad(loc, raw, eps)["elbo"]
        P.beta[j] = b0
        num[j] = (ep - em) / 2e-6
    np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-6 * np.max(np.abs(num)))


def test_fixed_r_and_alpha_equal_the_free_model_at_zero_width_minus_their_terms():
    """Holding r = 0.5 and alpha = 1.2 fixed equals the free model with those
    parameters' sigma -> 0 at the same values, minus exactly the removed terms
    per phase and draw: the Jacobian ln r(1 - r) of r, the normal prior of
    alpha, and their two entropy terms ln sigma + (1 + ln 2 pi)/2."""
    inst, P = _problem()
    Pf = oracle.Problem.from_instance(inst, fix_r=0.5, fix_alpha=1.2)
    loc, raw = _perturbed(P, 11)
    loc[:, 3], loc[:, 4] = 0.0, 1.2          # logit(0.5) = 0
    raw[:, 3] = raw[:, 4] = -60.0             # sigma = softplus(-60) ~ 8.8e-27
    eps = synth.normals(15, 3, P.K).astype(np.float64)
    a, b = Pf.elbo_grad(loc, raw, eps), P.elbo_grad(loc, raw, eps)
    sig0 = math.log1p(math.exp(-60.0))
    per_phase = (math.log(0.25) + stats.norm.logpdf(1.2, 1.0, 0.2)
                 + 2 * (math.log(sig0) + 0.5 * (1 + math.log(2 * math.pi))))
    assert a["elbo"] == pytest.approx(b["elbo"] - P.K * per_phase, rel=1e-12, abs=1e-9)
    np.testing.assert_array_equal(a["grad"][:, [3, 4, 8, 9]], 0.0)
    np.testing.assert_allclose(a["grad"][:, [0, 1, 2, 5, 6, 7]], b["grad"][:, [0, 1, 2, 5, 6, 7]], rtol=1e-9,
                               atol=1e-9 * np.max(np.abs(b["grad"])))


def test_fixed_r_and_alpha_gradient_against_central_differences():
    inst, _ = _problem()
    P = oracle.Problem.from_instance(inst, fix_r=0.3, fix_alpha=0.9)
    loc, raw = _perturbed(P, 12)
    eps = synth.normals(16, 2, P.K).astype(np.float64)
    g = P.elbo_grad(loc, raw, eps)["grad"]
    num = _fd_grad(P, loc, raw, eps)
    np.testing.assert_array_equal(num[:, [3, 4, 8, 9]], 0.0)   # the objective does not depend on them
    free = [0, 1, 2, 5, 6, 7]
    rel = np.max(np.abs(num[:, free] - g[:, free]), axis=0) / np.max(np.abs(g[:, free]), axis=0)
    assert np.all(rel < 1e-5), rel


@pytest.mark.parametrize("w,alpha,r", [(0.1, 1.0, 0.5), (0.05, 2.5, 0.2), (0.3, 0.4, 0.9)])
def test_area_factor_against_quadrature(w, alpha, r):
    """orc_area_factor equals the integral of the unit-height split
    pseudo-Voigt (FWHM w left of the peak, alpha w right of it)."""
    from scipy import integrate
    lib = oracle.lib()

    def v(d):
        side = alpha * w if d >= 0 else w
        t = d / side
        return (1 - r) * math.exp(-4 * math.log(2) * t * t) + r / (1 + 4 * t * t)

    left = integrate.quad(v, -np.inf, 0.0, epsabs=0, epsrel=1e-11, limit=500)[0]
    right = integrate.quad(v, 0.0, np.inf, epsabs=0, epsrel=1e-11, limit=500)[0]
    assert lib.orc_area_factor(w, alpha, r) == pytest.approx(left + right, rel=1e-8)


def test_area_normalised_peak_integrates_to_its_intensity():
    """One area-normalised peak (Gaussian-leaning, so the truncated tails are
    small) integrates over a wide grid to h I."""
    x = np.linspace(20.0, 80.0, 300001)
    P = oracle.Problem([0, 1], [50.0], [0.7], x, np.ones_like(x), np.zeros_like(x), normalisation="area")
    h = 123.0
    f = P.profile(np.array([[[h, 0.01, 0.08, 0.05, 1.6]]]))[0]
    area = np.trapezoid(f, x) if hasattr(np, "trapezoid") else np.trapz(f, x)
    assert area == pytest.approx(h * 0.7, rel=2e-4)


def test_area_normalised_gradient_against_central_differences():
    inst, _ = _problem()
    P = oracle.Problem.from_instance(inst, normalisation="area")
    loc, raw = _perturbed(P, 13)
    eps = synth.normals(17, 2, P.K).astype(np.float64)
    g = P.elbo_grad(loc, raw, eps)["grad"]
    num = _fd_grad(P, loc, raw, eps)
    rel = np.max(np.abs(num - g), axis=0) / np.max(np.abs(g), axis=0)
    assert np.all(rel < 1e-5), rel


@pytest.mark.parametrize("a,L,tau,a0", [(0.3, -1.2, 2 / 3, 0.0), (-2.0, 0.7, 0.5, math.log(0.1 / 0.9)),
                                        (4.0, 3.0, 1.0, 1.0)])
def test_gate_terms_against_logistic_densities(a, L, tau, a0):
    """y = (a + L)/tau with L standard logistic is logistic with location a/tau
    and scale 1/tau: ln q(y) and ln p(y) are scipy's logistic log-densities."""
    z, v, dp = oracle.gate_terms(a, L, tau, a0)
    y = (a + L) / tau
    assert z == pytest.approx(special.expit(y), rel=1e-14)
    ref = stats.logistic.logpdf(y, loc=a0 / tau, scale=1 / tau) - stats.logistic.logpdf(y, loc=a / tau, scale=1 / tau)
    assert v == pytest.approx(ref, rel=1e-12, abs=1e-12)
    h = 1e-6
    num = (stats.logistic.logpdf(y + h, loc=a0 / tau, scale=1 / tau)
           - stats.logistic.logpdf(y - h, loc=a0 / tau, scale=1 / tau)) / (2 * h)
    assert dp == pytest.approx(num, rel=1e-6, abs=1e-8)


def test_gate_noise_is_logistic_and_counter_keyed():
    L = oracle.gate_noise(7, 0, 3, 400, 25).ravel()
    assert stats.kstest(L, "logistic").pvalue > 1e-3
    assert not np.array_equal(oracle.gate_noise(7, 0, 4, 4, 3), oracle.gate_noise(7, 0, 3, 4, 3))


def test_gated_gradient_against_central_differences():
    inst, _ = _problem()
    P = oracle.Problem.from_instance(inst, gates=True, gate_prior=0.3)
    loc, raw = _perturbed(P, 14)
    P.gate_a[:] = [0.5, -0.3, 1.1]
    eps = synth.normals(18, 3, P.K).astype(np.float64)
    L = oracle.gate_noise(9, 0, 0, 3, P.K)
    r = P.elbo_grad(loc, raw, eps, gate_noise=L)
    num = np.zeros((P.K, 10))
    for k in range(P.K):
        for j in range(5):
            for which in (0, 1):
                Lc, R = loc.copy(), raw.copy()
                A = Lc if which == 0 else R
                A[k, j] += 1e-6
                ep = P.elbo_grad(Lc, R, eps, gate_noise=L)["elbo"]
                A[k, j] -= 2e-6
                em = P.elbo_grad(Lc, R, eps, gate_noise=L)["elbo"]
                num[k, j + 5 * which] = (ep - em) / 2e-6
    rel = np.max(np.abs(num - r["grad"]), axis=0) / np.max(np.abs(r["grad"]), axis=0)
    assert np.all(rel < 1e-5), rel
    ga = np.zeros(P.K)
    for k in range(P.K):
        a0 = P.gate_a[k]
        P.gate_a[k] = a0 + 1e-6
        ep = P.elbo_grad(loc, raw, eps, gate_noise=L)["elbo"]
        P.gate_a[k] = a0 - 1e-6
        em = P.elbo_grad(loc, raw, eps, gate_noise=L)["elbo"]
        P.gate_a[k] = a0
        ga[k] = (ep - em) / 2e-6
    np.testing.assert_allclose(r["grad_gate"], ga, rtol=1e-5, atol=1e-6 * np.max(np.abs(ga)))


def test_open_gates_give_the_ungated_profile():
    inst, P = _problem()
    Pg = oracle.Problem.from_instance(inst, gates=True)
    Pg.gate_a[:] = 60.0                      # z = sigmoid(90 + L/tau) = 1 to double precision
    loc, raw = _perturbed(P, 15)
    eps = synth.normals(19, 2, P.K).astype(np.float64)
    a = Pg.elbo_grad(loc, raw, eps, want_f=True, gate_noise=np.zeros((2, P.K)))
    b = P.elbo_grad(loc, raw, eps, want_f=True)
    np.testing.assert_allclose(a["f"], b["f"], rtol=1e-14)
    np.testing.assert_allclose(a["ll"], b["ll"], rtol=1e-14)
