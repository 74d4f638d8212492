"""Pins of the FP64 oracle's model, likelihood and priors against closed forms
and library routines (no GPU).  Each pin is chosen so that a plausible slip in
the oracle (a dropped term, a wrong sign, an inverted width convention) fails."""
import math

import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle
from oracle import posterior as post
from paper_2501_09308_gb300 import synth

LN2 = math.log(2.0)


def gauss_shape(d, fwhm):
    sig = fwhm / (2.0 * math.sqrt(2.0 * LN2))
    return stats.norm.pdf(d, scale=sig) / stats.norm.pdf(0.0, scale=sig)


def cauchy_shape(d, fwhm):
    return stats.cauchy.pdf(d, scale=fwhm / 2.0) / stats.cauchy.pdf(0.0, scale=fwhm / 2.0)


@pytest.mark.parametrize("w", [0.05, 0.1, 0.13])
@pytest.mark.parametrize("alpha", [1.0, 0.7, 1.4])
def test_pseudo_voigt_endpoints_are_gauss_and_lorentz(w, alpha):
    """Appendix A.2: V = (1-r) G + r L, so r = 0 is the Gaussian and r = 1 the
    Lorentzian; on the x >= rho side the width is alpha * w (split width)."""
    for d in np.linspace(-0.4, 0.4, 33):
        side = alpha * w if d >= 0 else w
        assert oracle.pvoigt(d, w, 0.0, alpha) == pytest.approx(gauss_shape(d, side), rel=1e-12, abs=1e-300)
        assert oracle.pvoigt(d, w, 1.0, alpha) == pytest.approx(cauchy_shape(d, side), rel=1e-12)


@pytest.mark.parametrize("r", [0.0, 0.3, 0.5, 1.0])
def test_fwhm_and_height(r):
    """Height-normalised: V(0) = 1; half maximum at -w/2 and at +alpha w/2."""
    w, alpha = 0.08, 1.3
    assert oracle.pvoigt(0.0, w, r, alpha) == pytest.approx(1.0, rel=1e-15)
    assert oracle.pvoigt(-w / 2, w, r, alpha) == pytest.approx(0.5, rel=1e-13)
    assert oracle.pvoigt(alpha * w / 2, w, r, alpha) == pytest.approx(0.5, rel=1e-13)


def test_alpha_one_is_symmetric_and_sign_form():
    """A(x; alpha) = alpha for x >= rho else 1 equals the sign form
    sign(x - rho)(alpha - 1)/2 + (alpha + 1)/2; alpha = 1 gives a symmetric peak."""
    for d in np.linspace(0.001, 0.5, 20):
        assert oracle.pvoigt(d, 0.1, 0.4, 1.0) == oracle.pvoigt(-d, 0.1, 0.4, 1.0)
        al = 1.7
        a_sign = np.sign(d) * (al - 1) / 2 + (al + 1) / 2
        assert oracle.pvoigt(d, 0.1, 0.4, al) == pytest.approx(oracle.pvoigt(d, 0.1 * a_sign, 0.4, 1.0), rel=1e-14)


@pytest.mark.parametrize("w,r,alpha", [(0.05, 0.0, 1.0), (0.1, 1.0, 1.0), (0.08, 0.4, 1.3), (0.12, 0.75, 0.6)])
def test_closed_form_area_matches_quadrature(w, r, alpha):
    """Closed-form area of the split pseudo-Voigt (used for the 1 % area-ratio
    identification rule) against adaptive quadrature."""
    f = lambda d: oracle.pvoigt(d, w, r, alpha)
    left, _ = integrate.quad(f, -np.inf, 0.0, epsabs=0, epsrel=1e-12, limit=500)
    right, _ = integrate.quad(f, 0.0, np.inf, epsabs=0, epsrel=1e-12, limit=500)
    assert left + right == pytest.approx(post.peak_area(w, r, alpha), rel=1e-8)


def test_profile_single_peak_and_superposition():
    """f = B + sum_k h_k sum_m I_m V: one peak against library densities, and
    the superposition of two phases equals the sum of each alone."""
    x = np.linspace(20, 30, 401)
    bg = 5.0 + 0.1 * x
    # one phase, one peak
    P1 = oracle.Problem([0, 1], [24.3], [0.7], x, np.ones_like(x), bg)
    th = np.array([[[1500.0, 0.02, 0.09, 0.35, 1.2]]])
    f = P1.profile(th)[0]
    d = x - (24.3 + 0.02)
    side = np.where(d >= 0, 1.2 * 0.09, 0.09)
    want = bg + 1500.0 * 0.7 * ((1 - 0.35) * gauss_shape(d, side) + 0.35 * cauchy_shape(d, side))
    np.testing.assert_allclose(f, want, rtol=1e-12)
    # two phases
    off = [0, 2, 5]
    pos = [21.0, 25.5, 22.2, 26.0, 28.9]
    inten = [1.0, 0.3, 0.5, 1.0, 0.2]
    P2 = oracle.Problem(off, pos, inten, x, np.ones_like(x), bg)
    th2 = np.array([[[900.0, -0.01, 0.07, 0.6, 0.9], [400.0, 0.03, 0.11, 0.2, 1.1]]])
    fa = oracle.Problem([0, 2], pos[:2], inten[:2], x, np.ones_like(x), bg).profile(th2[:, :1])[0]
    fb = oracle.Problem([0, 3], pos[2:], inten[2:], x, np.ones_like(x), bg).profile(th2[:, 1:])[0]
    np.testing.assert_allclose(P2.profile(th2)[0] - bg, (fa - bg) + (fb - bg), rtol=1e-12)


def test_poisson_loglik_direct_and_deviance():
    """Appendix A.2: -ln p(Y|Phi) = -sum [y ln f - f - ln y!] against the
    library Poisson log-pmf; the deviance split equals the direct form."""
    rng = np.random.default_rng(3)
    f = rng.uniform(0.5, 2e4, size=3000)
    y = rng.poisson(f).astype(np.float64)
    y[:7] = 0.0
    P = oracle.Problem([0, 1], [50.0], [1.0], np.arange(3000.0), y, np.zeros(3000))
    want = stats.poisson.logpmf(y, f).sum()
    assert P.loglik(f, "direct") == pytest.approx(want, rel=1e-11)
    assert P.loglik(f, "deviance") == pytest.approx(want, rel=1e-11)
    c = P.data_constant()
    yy = y[y > 0]
    assert c == pytest.approx(np.sum(special.xlogy(yy, yy) - yy - special.gammaln(yy + 1)), rel=1e-12)


def test_log_prior_against_library_densities():
    """Sec. 2.2 and Appendix B.2: h ~ Exp(lambda) = Gam(1, lambda) with lambda =
    1/max(Y-B); mu ~ N(0, 0.03); alpha ~ N(1, 0.2); r ~ U(0, 1); w ~ Gam(3, 100)."""
    x = np.linspace(10, 20, 50)
    y = np.full(50, 300.0)
    bg = np.full(50, 50.0)
    P = oracle.Problem([0, 1], [15.0], [1.0], x, y, bg)
    assert P.eta == pytest.approx(250.0)
    lam = 1.0 / 250.0
    for th in ([120.0, 0.013, 0.041, 0.3, 1.22], [3.0, -0.05, 0.15, 0.9, 0.8]):
        want = (stats.expon.logpdf(th[0], scale=1 / lam) + stats.norm.logpdf(th[1], 0, 0.03)
                + stats.gamma.logpdf(th[2], 3.0, scale=1 / 100.0) + stats.uniform.logpdf(th[3])
                + stats.norm.logpdf(th[4], 1.0, 0.2))
        assert P.log_prior(np.array(th)) == pytest.approx(want, rel=1e-13)


def test_gamma_moments_fix_the_rate_reading():
    """Sec. 2.2 gives E = alpha/lambda and V = alpha/lambda^2; with shape 3 and
    100 read as the rate, the width prior has mean 0.03 deg and variance 3e-4."""
    g = stats.gamma(3.0, scale=1 / 100.0)
    assert g.mean() == pytest.approx(3.0 / 100.0)
    assert g.var() == pytest.approx(3.0 / 100.0 ** 2)
    # and the oracle's w-part integrates to one with that mean
    P = oracle.Problem([0, 1], [15.0], [1.0], np.linspace(10, 20, 5), np.full(5, 10.0), np.ones(5))
    base = np.array([1.0, 0.0, 0.03, 0.5, 1.0])

    def pw(w):
        th = base.copy()
        th[2] = w
        return math.exp(P.log_prior(th) - P.log_prior(base)) * stats.gamma.pdf(0.03, 3.0, scale=0.01)

    z, _ = integrate.quad(pw, 0, 1, limit=200)
    m1, _ = integrate.quad(lambda w: w * pw(w), 0, 1, limit=200)
    assert z == pytest.approx(1.0, rel=1e-9)
    assert m1 == pytest.approx(0.03, rel=1e-9)


def test_log_jacobian_matches_numerical_derivative():
    P = oracle.Problem([0, 1], [15.0], [1.0], np.linspace(10, 20, 5), np.full(5, 10.0), np.ones(5))
    u0 = np.array([[3.1, 0.02, -2.9, 0.7, 1.1]])
    lib = oracle.lib()
    lj = lib.orc_log_jac(oracle._pd(oracle.f64(u0[0])))
    h = 1e-6
    jac = 0.0
    for j in range(5):
        up, um = u0.copy(), u0.copy()
        up[0, j] += h
        um[0, j] -= h
        _, tp = P.theta(up, np.full((1, 5), -80.0), np.zeros((1, 1, 5)))
        _, tm = P.theta(um, np.full((1, 5), -80.0), np.zeros((1, 1, 5)))
        jac += math.log(abs((tp[0, 0, j] - tm[0, 0, j]) / (2 * h)))
    assert lj == pytest.approx(jac, abs=1e-8)


def test_entropy_and_transforms():
    raw = np.array([[-2.2, 0.3, -5.0, 1.7, 0.0]])
    sig = np.logaddexp(0.0, raw)
    assert oracle.entropy(raw) == pytest.approx(np.sum(stats.norm(scale=sig).entropy()), rel=1e-13)
    for v in (-50.0, -3.0, 0.0, 2.5, 40.0):
        assert oracle.softplus(v) == pytest.approx(np.logaddexp(0.0, v), rel=1e-15)
        assert oracle.sigmoid(v) == pytest.approx(special.expit(v), rel=1e-15)


def test_theta_transform_reparameterisation():
    P = oracle.Problem.from_instance(synth.small_problem(K=3))
    loc, raw = P.init_params()
    eps = synth.normals(4, 2, P.K).astype(np.float64)
    u, th = P.theta(loc, raw, eps)
    sig = np.logaddexp(0.0, raw)
    np.testing.assert_allclose(u, loc[None] + sig[None] * eps, rtol=1e-15)
    np.testing.assert_allclose(th[..., 0], np.exp(u[..., 0]), rtol=1e-15)
    np.testing.assert_allclose(th[..., 2], np.exp(u[..., 2]), rtol=1e-15)
    np.testing.assert_allclose(th[..., 3], special.expit(u[..., 3]), rtol=1e-15)
    np.testing.assert_array_equal(th[..., 1], u[..., 1])
    np.testing.assert_array_equal(th[..., 4], u[..., 4])
