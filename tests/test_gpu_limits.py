"""Parity with the FP64 oracle at the input limits the library accepts: the
largest peak table (K = 1024 phases, 24000 peaks in all; the compact
shared-memory layout at one resident block per SM) and the largest sample
count (S = 65536 draws in one step).  Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

import oracle
from paper_2501_09308_gb300 import synth, xrdvi

pytestmark = pytest.mark.gpu

F_TOL = 1e-5
G_TOL = 1e-4
MAX_K, MAX_PEAKS, MAX_S = 1024, 24000, 65536


def _max_table_problem(N=1200, S=2, seed=61):
    """K = 1024 phases of 24 peaks, then the last peak of the last 576 phases
    dropped: 448 * 24 + 576 * 23 = 24000 peaks."""
    inst = synth.make_problem(K=MAX_K, m_lo=24, m_hi=24, x_lo=20.0, x_step=0.05, N=N, n_planted=4, S=S,
                              iters=10, seed=seed)
    counts = np.diff(inst.offsets)
    keep = np.ones(int(inst.offsets[-1]), dtype=bool)
    for k in range(MAX_K - 576, MAX_K):
        keep[inst.offsets[k + 1] - 1] = False
        counts[k] -= 1
    offsets = np.zeros(MAX_K + 1, dtype=np.int32)
    offsets[1:] = np.cumsum(counts)
    out = synth.Instance(**{**inst.__dict__, "offsets": offsets, "pos": inst.pos[keep], "inten": inst.inten[keep]})
    assert int(out.offsets[-1]) == MAX_PEAKS and out.K == MAX_K
    return out


def _parity(inst, S, seed, want_f=True, rows=None):
    ctx = xrdvi.Context.from_instance(inst, S=S)
    loc, raw = ctx.params()
    rng = np.random.default_rng(seed)
    loc = loc + rng.normal(0, 0.05, loc.shape).astype(np.float32)
    raw = raw + rng.normal(0, 0.1, raw.shape).astype(np.float32)
    ctx.set_params(loc, raw)
    eps = synth.normals(seed, S, inst.K)
    g = ctx.elbo_grad(eps, want_f=want_f)
    ctx.close()
    o = oracle.Problem.from_instance(inst).elbo_grad(loc.astype(np.float64), raw.astype(np.float64),
                                                      eps.astype(np.float64), want_f=want_f)
    if want_f:
        sel = slice(None) if rows is None else rows
        rel = np.abs(g["f"][sel] - o["f"][sel]) / np.abs(o["f"][sel])
        assert rel.max() <= F_TOL, rel.max()
    np.testing.assert_allclose(g["ll"], o["ll"], rtol=F_TOL)
    assert np.max(np.abs(g["lpj"] - o["lpj"]) / np.maximum(1.0, np.abs(o["lpj"]))) <= F_TOL
    assert abs(g["elbo"] - o["elbo"]) <= F_TOL * abs(o["elbo"])
    for b in range(10):
        ref = np.max(np.abs(o["grad"][:, b]))
        err = np.max(np.abs(g["grad"][:, b] - o["grad"][:, b]))
        assert err <= G_TOL * ref, (b, err, ref)


def test_largest_peak_table_matches_the_oracle():
    """1024 phases and 24000 peaks over a 60-degree pattern: every profile
    value, log-likelihood, ELBO and gradient block within tolerance."""
    _parity(_max_table_problem(), 2, 61)


def test_largest_sample_count_matches_the_oracle():
    """S = 65536 draws of a three-phase problem: per-draw log-likelihoods and
    log joints of every draw, the ELBO and the gradient (FP64 reductions over
    all draws), and the profile rows of the first, middle and last draws."""
    inst = synth.small_problem(K=3, M=5, N=300, S=MAX_S, seed=62)
    _parity(inst, MAX_S, 62, rows=[0, 1, MAX_S // 2, MAX_S - 1])

