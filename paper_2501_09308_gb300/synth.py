"""Seeded synthetic diffractograms and candidate-phase tables.

This module is the one piece of input generation shared by the CUDA path, the
FP64 oracle, the tests and the benchmark.  It holds none of the inference
arithmetic (no likelihood, prior, variational transform, gradient or
posterior): it only draws candidate peak lists, planted phases, a background
and Poisson counts, and standard-normal noise arrays that either side can take
as injected Monte-Carlo noise.

The planted signal is simulated with library densities (``scipy.stats.norm``
and ``scipy.stats.cauchy``, each scaled to unit height and mixed 50/50), i.e.
a symmetric pseudo-Voigt data-generating process as the workload description
asks for; this simulator is independent of both implementations under test.

Problem setting (Appendix A.1 of the paper): a pattern D = {(x_i, y_i)} of N
2-theta points with integer counts, and K candidate phases, each a list of M_k
(position p_m in degrees, relative intensity I_m in [0, 1]) pairs.  The paper's
own data (a TiO2 mixture against 50 database candidates, Sec. 3.1) is not
available; these seeded instances have the same shape: tens to hundreds of
candidates, a few planted phases, a 2-theta grid of thousands of points and
peak counts of order 1e4.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 20250116
H0 = 1.0e4  # planted peak height scale in counts


@dataclasses.dataclass
class Instance:
    """One phase-search problem: candidate table + observed pattern (+ truth)."""

    name: str
    offsets: np.ndarray      # int32 [K+1], CSR offsets into pos/inten
    pos: np.ndarray          # float32 [sum M_k], degrees 2-theta
    inten: np.ndarray        # float32 [sum M_k], relative intensity in [0, 1]
    x: np.ndarray            # float32 [N], strictly increasing 2-theta grid
    y: np.ndarray            # float32 [N], integer-valued counts
    bg: np.ndarray           # float32 [N], fixed background B(x_i) > 0
    S: int                   # Monte-Carlo samples per step
    iters: int               # optimisation steps for a fit
    planted: np.ndarray      # int32 [n_planted], indices of the planted phases
    truth: dict              # planted h, mu, w, r per planted phase

    @property
    def K(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def N(self) -> int:
        return int(self.x.shape[0])

    @property
    def M(self) -> np.ndarray:
        return np.diff(self.offsets)

    @property
    def evals_per_iter(self) -> int:
        """Dense profile evaluations per Monte-Carlo step: S * sum(M_k) * N."""
        return int(self.S) * int(self.offsets[-1]) * int(self.N)


def _phase_peaks(rng, m, lo, hi):
    p = rng.uniform(lo, hi, size=m)
    inten = np.minimum(rng.exponential(0.2, size=m), 1.0)
    inten[np.argmax(inten)] = 1.0
    return p, inten


def _height_pv(d, fwhm, mix):
    """Unit-height 50/50 normal+Cauchy peak from library densities (simulator)."""
    from scipy import stats

    sig = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    g = stats.norm.pdf(d, scale=sig) / stats.norm.pdf(0.0, scale=sig)
    l = stats.cauchy.pdf(d, scale=fwhm / 2.0) / stats.cauchy.pdf(0.0, scale=fwhm / 2.0)
    return (1.0 - mix) * g + mix * l


def _simulate_counts(rng, x, bg, phases, planted, hs, mus, ws):
    f = bg.astype(np.float64).copy()
    for k, h, mu, w in zip(planted, hs, mus, ws):
        p, inten = phases[k]
        for pm, im in zip(p, inten):
            f += h * im * _height_pv(x - (pm + mu), w, 0.5)
    y = rng.poisson(f).astype(np.float64)
    return y


def make_problem(*, K, m_lo, m_hi, x_lo, x_step, N, n_planted, S, iters, seed,
                 background="linear", overlap=False, name="custom", true_bg_factor=None):
    """Generic seeded instance.  M_k ~ U{m_lo..m_hi} (m_lo == m_hi: fixed).
    true_bg_factor: optional array [N] multiplying the background the counts
    are simulated with (the instance still reports the unmultiplied one), for
    problems whose background is mis-specified."""
    rng = np.random.default_rng(seed)
    x = x_lo + x_step * np.arange(N, dtype=np.float64)
    x_hi = float(x[-1])
    span_lo, span_hi = x_lo, x_hi
    Ms = rng.integers(m_lo, m_hi + 1, size=K)
    phases = [_phase_peaks(rng, int(m), span_lo, span_hi) for m in Ms]
    planted = np.sort(rng.choice(K, size=n_planted, replace=False)).astype(np.int32)
    if overlap and n_planted >= 2:
        # overlapping peaks: copy >= 3 peaks of one planted phase into another at
        # offsets within +-0.1 deg, and give decoys peaks near planted ones.
        src, dst = int(planted[0]), int(planted[1])
        ps, is_ = phases[src]
        pd, id_ = phases[dst]
        ncopy = min(3, len(ps), len(pd))
        pick = rng.choice(len(ps), size=ncopy, replace=False)
        pd = pd.copy()
        pd[:ncopy] = ps[pick] + rng.uniform(-0.1, 0.1, size=ncopy)
        phases[dst] = (pd, id_)
        decoys = [k for k in range(K) if k not in set(planted.tolist())]
        for k in decoys[: max(1, len(decoys) // 4)]:
            pk, ik = phases[k]
            pk = pk.copy()
            srcp = phases[int(rng.choice(planted))][0]
            pk[0] = srcp[rng.integers(len(srcp))] + rng.uniform(-0.1, 0.1)
            phases[k] = (pk, ik)
    # keep every position inside (0, 180) and sort each phase by position
    for k in range(K):
        p, i = phases[k]
        p = np.clip(p, span_lo, span_hi)
        o = np.argsort(p, kind="stable")
        phases[k] = (p[o], i[o])
    hs = rng.uniform(0.2, 1.0, size=n_planted) * H0
    mus = rng.normal(0.0, 0.02, size=n_planted)
    ws = rng.uniform(0.05, 0.15, size=n_planted)
    xr = x - x_lo
    if background == "linear":
        bg = 50.0 + 1.0 * xr
    else:
        bg = 40.0 + 0.8 * xr + 0.01 * xr * xr
    bg_true = bg if true_bg_factor is None else bg * np.asarray(true_bg_factor, dtype=np.float64)
    y = _simulate_counts(rng, x, bg_true, phases, planted, hs, mus, ws)
    offsets = np.zeros(K + 1, dtype=np.int32)
    offsets[1:] = np.cumsum([len(p) for p, _ in phases])
    pos = np.concatenate([p for p, _ in phases]).astype(np.float32)
    inten = np.concatenate([i for _, i in phases]).astype(np.float32)
    return Instance(
        name=name, offsets=offsets, pos=pos, inten=inten,
        x=x.astype(np.float32), y=y.astype(np.float32), bg=bg.astype(np.float32),
        S=int(S), iters=int(iters), planted=planted,
        truth={"h": hs, "mu": mus, "w": ws, "r": np.full(n_planted, 0.5)},
    )


def config(idx: int, instance: int = 0) -> Instance:
    """The five workload configurations (tiny, K=50, differentiation,
    precision sweep, serving request).  Seed = base + 1000*config + instance."""
    seed = SEED_BASE + 1000 * idx + instance
    if idx == 0:
        return make_problem(K=8, m_lo=20, m_hi=20, x_lo=10.0, x_step=0.035, N=2000,
                            n_planted=3, S=16, iters=300, seed=seed,
                            background="linear", name="tiny_K8_N2000_S16")
    if idx == 1:
        return make_problem(K=50, m_lo=5, m_hi=80, x_lo=10.0, x_step=0.02, N=4500,
                            n_planted=4, S=256, iters=2000, seed=seed,
                            background="quadratic", overlap=True,
                            name="fit_K50_N4500_S256")
    if idx == 2:
        # finite-difference sub-instance of the K=50 setup
        return make_problem(K=6, m_lo=5, m_hi=80, x_lo=30.0, x_step=0.05, N=600,
                            n_planted=2, S=8, iters=100, seed=seed,
                            background="quadratic", overlap=True,
                            name="fd_K6_N600")
    if idx == 3:
        return make_problem(K=200, m_lo=5, m_hi=120, x_lo=10.0, x_step=0.01, N=9000,
                            n_planted=5, S=1024, iters=100, seed=seed,
                            background="quadratic", overlap=True,
                            name="precision_K200_N9000_S1024")
    if idx == 4:
        rng = np.random.default_rng(seed)
        K = int(rng.integers(10, 201))
        N = int(rng.integers(2000, 9001))
        step = 90.0 / N
        return make_problem(K=K, m_lo=5, m_hi=100, x_lo=10.0, x_step=step, N=N,
                            n_planted=3, S=256, iters=1000, seed=seed + 7,
                            background="linear", name=f"serve_K{K}_N{N}")
    raise ValueError(f"unknown configuration {idx}")


def small_problem(K=3, M=6, N=300, S=4, seed=1, x_lo=20.0, x_step=0.05, n_planted=2):
    """Small instance for parity tests: several point tiles and a ragged tail."""
    return make_problem(K=K, m_lo=max(1, M - 3), m_hi=M, x_lo=x_lo, x_step=x_step, N=N,
                        n_planted=min(n_planted, K), S=S, iters=10, seed=seed,
                        background="linear", name=f"small_K{K}_N{N}")


def normals(seed: int, S: int, K: int) -> np.ndarray:
    """Injected Monte-Carlo noise: float32 [S, K, 5] standard normals."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((S, K, 5)).astype(np.float32)


def arrival_times(n: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Poisson arrivals: cumulative sums of seeded exponential gaps (seconds)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
