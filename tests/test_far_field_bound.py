"""The far field's approximation bound, checked in FP64 on the CPU.

The profile kernels sum the Lorentzian tails of peaks more than half a
half-width beyond a tile (and beyond their Gaussian reach) at 32 Chebyshev
nodes of the first kind of the tile's span and interpolate them with
barycentric Lagrange weights (Berrut & Trefethen, SIAM Review 2004); the
backward weights the same node values with W_p = sum_i g_i lam_p(x_i).  Both
are exact for the degree-31 interpolant, so their error is the interpolation
error of L = 1/(1 + t^2), L^2 t and L^2 with t = s (x - rho) on the span.
For poles at least 1.5 half-widths from the span's centre that error is below
1e-8 of the function's value at every point of the span (6e-9 at worst, for
the narrowest peaks), for every width: the scan below covers s h (width
scale times half-width) from 1e-2 to 5e3."""
import numpy as np

NODES = 32
GAP = 0.5   # far peaks: beyond the span by this many half-widths


def cheb_nodes(n):
    p = np.arange(n)
    return np.cos((2 * p + 1) * np.pi / (2 * n)), (-1.0) ** p * np.sin((2 * p + 1) * np.pi / (2 * n))


def interpolate(xn, wb, fn, x):
    """Barycentric interpolation of node values fn at points x (second form)."""
    d = x[:, None] - xn[None, :]
    exact = np.isclose(d, 0.0, atol=0.0)
    d[exact] = 1.0
    c = wb[None, :] / d
    out = (c @ fn) / c.sum(axis=1)
    hit = exact.any(axis=1)
    out[hit] = fn[np.argmax(exact[hit], axis=1)]
    return out


def worst_error(s, rho, x, xn, wb):
    errs = []
    for f in (lambda z: 1.0 / (1.0 + (s * (z - rho)) ** 2),
              lambda z: (s * (z - rho)) / (1.0 + (s * (z - rho)) ** 2) ** 2,
              lambda z: 1.0 / (1.0 + (s * (z - rho)) ** 2) ** 2):
        ex = f(x)   # no zero on the span: rho lies outside it
        errs.append(np.max(np.abs(interpolate(xn, wb, f(xn), x) - ex) / np.abs(ex)))
    return max(errs)


def test_nodes_reproduce_a_degree_31_polynomial():
    """The interpolation (hence the node weighting of the backward) is exact
    for polynomials of degree < 32: a dropped node or a wrong weight sign
    fails this."""
    xn, wb = cheb_nodes(NODES)
    rng = np.random.default_rng(1)
    coef = rng.normal(size=NODES)
    x = np.linspace(-1, 1, 257)
    poly = np.polynomial.chebyshev.Chebyshev(coef)
    assert np.max(np.abs(interpolate(xn, wb, poly(xn), x) - poly(x))) < 1e-12 * np.max(np.abs(poly(x)))


def test_far_lorentzian_tails_interpolate_below_1e8():
    xn, wb = cheb_nodes(NODES)
    x = np.linspace(-1.0, 1.0, 513)   # span in half-width units (a 256-point tile, finer)
    worst = 0.0
    for s in np.geomspace(1e-2, 5e3, 60):
        for dist in (1.0 + GAP, 1.0 + GAP * 1.5, 3.0, 10.0):
            for rho in (dist, -dist):
                worst = max(worst, worst_error(s, rho, x, xn, wb))
    assert worst < 1e-8, worst


def test_nearer_poles_would_not_meet_the_bound():
    """The gap matters: with the pole a tenth of a half-width beyond the span
    the same 32 nodes miss the bound by orders of magnitude (so the far/near
    split, not the node count alone, carries the accuracy)."""
    xn, wb = cheb_nodes(NODES)
    x = np.linspace(-1.0, 1.0, 513)
    worst = max(worst_error(s, 1.1, x, xn, wb) for s in np.geomspace(1.0, 1e3, 20))
    assert worst > 1e-6
