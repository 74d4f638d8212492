"""Oracle posterior over phase combinations (FP64, numpy + the C oracle).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

What the paper fixes and what is read here:

* Phase identification (Sec. 4, the area-ratio figure): a phase counts as
  present when its share of the total integrated peak area is at least 1 %.
* The paper's output is a probability for each subset of candidate phases
  given the data, obtained by an approximate search over all subsets
  (Abstract, Sec. 1).  Reading: draw S_post samples from the fitted mean-field q; each sample gives
  the inclusion bit b_sk = [area ratio_sk >= 0.01]; the marginal inclusion
  probability is pi_k = (sum_s b_sk + 1/2) / (S_post + 1) (the +1/2 keeps
  logs finite); the probability of a combination c in {0,1}^K is the
  mean-field product prod_k pi_k^c_k (1 - pi_k)^(1 - c_k).  The top-M
  combinations are the M most probable ones, listed by an exact best-first
  search over flip sets of the mode; their total mass is an FP64 log-sum-exp.
* Closed-form peak area (Reading of the height-normalised split pseudo-Voigt):
  area_k = h_k sum_m I_m ((1 + alpha_k) w_k / 2) [(1 - r_k) sqrt(pi / ln 2) / 2 + r_k pi / 2].
* Evidence (Sec. 3.2, the marginal likelihood p(Y)): importance sampling with
  q as proposal, log w_s = ln p(Y|theta_s) + ln p(theta_s) + ln|J_s| - ln q(u_s),
  ln Z = LSE_s(log w_s) - ln S_post, ESS = exp(2 LSE(log w) - LSE(2 log w)).
* Exhaustive enumeration for small K: every sub-model c (phases outside c
  removed) is fitted by the same SVI; p_enum(c) proportional to exp(ELBO_c) under a uniform
  prior over combinations, normalised by an FP64 log-sum-exp.  This is exact
  over combinations with each evidence replaced by its ELBO.

Pins: the area closed form against quadrature, LSE normalisation against
brute force over all 2^K products, top-M order against brute-force sorting,
the IS evidence against the conjugate closed form (tests/test_oracle_*).
Parity unpinned: the absolute combination probabilities at large K (no exact
reference exists; only the invariants above and planted-phase recovery apply).
"""
from __future__ import annotations

import heapq
import math

import numpy as np

from . import Problem, _pd, f64, lib, normals, softplus

LN2 = math.log(2.0)
AREA_G = 0.5 * math.sqrt(math.pi / LN2)   # integral of exp(-4 ln2 t^2) over the real line
AREA_L = 0.5 * math.pi


def peak_area(w, r, alpha_c):
    """Area of one unit-intensity, unit-height split pseudo-Voigt."""
    return ((1.0 + alpha_c) * w / 2.0) * ((1.0 - r) * AREA_G + r * AREA_L)


def phase_areas(prob: Problem, theta):
    """a[s, k] = h_k sum_m I_m peak_area(w_k, r_k, max(alpha_k, alpha_min))."""
    theta = f64(theta)
    Isum = np.add.reduceat(prob.inten, prob.off[:-1]) if prob.K > 0 else np.zeros(0)
    # empty phases are rejected at create time, so reduceat is safe
    h, w, r, al = theta[..., 0], theta[..., 2], theta[..., 3], theta[..., 4]
    if getattr(prob, "area_norm", False):   # h is already the area per unit intensity
        return h * Isum[None, :]
    ac = np.maximum(al, prob.prior.alpha_min)
    return h * Isum[None, :] * peak_area(w, r, ac)


def inclusion_bits(areas, threshold=0.01):
    tot = areas.sum(axis=1, keepdims=True)
    return (areas / tot) >= threshold


def marginal_pi(bits):
    S = bits.shape[0]
    return (bits.sum(axis=0) + 0.5) / (S + 1.0)


def logsumexp(a):
    a = np.asarray(a, dtype=np.float64)
    if a.size == 0:
        return -math.inf
    m = float(np.max(a))
    if not math.isfinite(m):
        return m
    return m + math.log(float(np.sum(np.exp(a - m))))


def top_combinations(pi, top_m):
    """The top_m most probable combinations under prod_k pi^c (1-pi)^(1-c),
    by best-first search over flip sets of the mode (exact: every set's cost
    is a sum of non-negative flip costs, and each set has one parent).
    Returns (bool [top_m, K], logp [top_m])."""
    pi = f64(pi)
    K = pi.shape[0]
    lp1, lp0 = np.log(pi), np.log1p(-pi)
    mode = pi > 0.5
    lmode = float(np.sum(np.where(mode, lp1, lp0)))
    cost = np.abs(lp1 - lp0)
    order = np.argsort(cost, kind="stable")
    c = cost[order]
    out_sets, out_lp = [], []
    # heap entries: (cost, tie-break id, last index used, tuple of indices)
    heap = [(0.0, 0, -1, ())]
    uid = 1
    while heap and len(out_sets) < top_m:
        cst, _, last, idx = heapq.heappop(heap)
        out_sets.append(idx)
        out_lp.append(lmode - cst)
        j = last + 1
        if j < K:
            # child 1: append j; child 2: replace last with j
            heapq.heappush(heap, (cst + c[j], uid, j, idx + (j,)))
            uid += 1
            if last >= 0:
                heapq.heappush(heap, (cst - c[last] + c[j], uid, j, idx[:-1] + (j,)))
                uid += 1
    combos = np.zeros((len(out_sets), K), dtype=bool)
    for r_, idx in enumerate(out_sets):
        row = mode.copy()
        for j in idx:
            row[order[j]] = ~row[order[j]]
        combos[r_] = row
    return combos, np.asarray(out_lp)


def all_combination_logp(pi):
    """log prob of every combination (K <= 20), bit k of the index = phase k."""
    pi = f64(pi)
    K = pi.shape[0]
    idx = np.arange(1 << K, dtype=np.int64)
    bits = ((idx[:, None] >> np.arange(K)) & 1).astype(bool)
    return np.where(bits, np.log(pi)[None, :], np.log1p(-pi)[None, :]).sum(axis=1)


def log_q(raw, eps, free=None):
    """ln q(u) of the mean-field normal at u = loc + sigma * eps, per sample
    (free[5]: which parameters are part of q; default all)."""
    sig = np.vectorize(softplus)(f64(raw))
    e = f64(eps)
    terms = -0.5 * e * e - np.log(sig)[None] - 0.5 * math.log(2 * math.pi)
    if free is not None:
        terms = terms * np.asarray(free, dtype=np.float64)[None, None, :]
    return np.sum(terms, axis=(1, 2))


def posterior(prob: Problem, loc, raw, S_post, seed=None, eps=None, top_m=8, threshold=0.01, gate_noise=None):
    """Posterior summary of a fitted q.  Noise: eps[S_post, K, 5] if given,
    else the oracle's Philox stream with tag 1 (posterior) at step 0 (gates:
    gate_noise[S_post, K], else the gate stream with tag 1)."""
    if eps is None:
        eps = normals(seed, 1, 0, S_post, prob.K)
    eps = f64(eps)
    u, th = prob.theta(loc, raw, eps)
    glp = np.zeros(S_post)
    th_eff = th
    if getattr(prob, "gates", False):   # the gate z scales the phase's profile and its area
        from . import gate_noise as _gn, gate_terms
        L = _gn(seed, 1, 0, S_post, prob.K) if gate_noise is None else f64(gate_noise)
        th_eff = th.copy()
        for s in range(S_post):
            for k in range(prob.K):
                z, v, _ = gate_terms(prob.gate_a[k], L[s, k], prob.gate_tau, prob.variant.gate_prior_logit)
                th_eff[s, k, 0] *= z
                glp[s] += v
    f = prob.profile(th_eff)
    ll = np.array([prob.loglik(f[s]) for s in range(S_post)])
    lpj = np.zeros(S_post)
    for s in range(S_post):
        for k in range(prob.K):
            lpj[s] += prob.log_prior_jac(u[s, k], th[s, k])
    lpj += glp
    lq = log_q(raw, eps, [prob.free(j) for j in range(5)])
    logw = ll + lpj - lq
    areas = phase_areas(prob, th_eff)
    bits = inclusion_bits(areas, threshold)
    pi = marginal_pi(bits)
    combos, clp = top_combinations(pi, top_m)
    lse_w = logsumexp(logw)
    return {
        "pi": pi, "bits": bits, "areas": areas, "combos": combos, "combo_logp": clp,
        "coverage_log": logsumexp(clp), "log_evidence": lse_w - math.log(S_post),
        "ess": math.exp(2 * lse_w - logsumexp(2 * logw)), "logw": logw, "ll": ll,
        "lpj": lpj, "lq": lq,
    }


def enumerate_submodels(inst_arrays, S, iters, seed, lr=0.01):
    """Fit every sub-model (non-empty subsets of phases) and return
    (masks [2^K - 1, K], elbo_c, p_enum).  ELBO_c is the mean of the last
    quarter of the trace.  inst_arrays = (offsets, pos, inten, x, y, bg)."""
    offsets, pos, inten, x, y, bg = inst_arrays
    offsets = np.asarray(offsets)
    K = len(offsets) - 1
    lam = 1.0 / float(np.max(np.asarray(y, np.float64) - np.asarray(bg, np.float64)))
    masks, elbos = [], []
    for code in range(1, 1 << K):
        keep = [k for k in range(K) if (code >> k) & 1]
        offs = [0]
        ps, is_ = [], []
        for k in keep:
            ps.append(np.asarray(pos)[offsets[k]:offsets[k + 1]])
            is_.append(np.asarray(inten)[offsets[k]:offsets[k + 1]])
            offs.append(offs[-1] + offsets[k + 1] - offsets[k])
        sub = Problem(np.array(offs), np.concatenate(ps), np.concatenate(is_), x, y, bg, lam=lam)
        res = sub.fit(S, iters, seed, lr=lr)
        tail = res["trace"][-max(1, iters // 4):]
        masks.append([(code >> k) & 1 for k in range(K)])
        elbos.append(float(np.mean(tail)))
    elbos = np.asarray(elbos)
    logp = elbos - logsumexp(elbos)
    return np.asarray(masks, dtype=bool), elbos, np.exp(logp)
