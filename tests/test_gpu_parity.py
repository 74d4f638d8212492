"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs and injected noise.

Tolerances (relative, FP32 kernels against the FP64 oracle):
  profile f[s, i]             max |df| / |f|                 <= 1e-5
  log-likelihood per sample   |dLL_s| / |LL_s|               <= 1e-5
  log prior + Jacobian        |d| / max(1, |lpj_s|)          <= 1e-5
  ELBO                        |dL| / |L|                     <= 1e-5
  gradient, per block         ||dg||_inf / ||g||_inf          <= 1e-4
(blocks: loc and raw of each of h, mu, w, r, alpha, over all phases).
"""
import numpy as np
import pytest

import oracle
from oracle import posterior as opost
from paper_2501_09308_gb300 import synth, xrdvi

pytestmark = pytest.mark.gpu

F_TOL = 1e-5
G_TOL = 1e-4


def perturbed_params(ctx, seed=0, scale=0.05):
    loc, raw = ctx.params()
    rng = np.random.default_rng(seed)
    loc = loc + rng.normal(0, scale, loc.shape).astype(np.float32)
    raw = raw + rng.normal(0, 2 * scale, raw.shape).astype(np.float32)
    ctx.set_params(loc, raw)
    return loc, raw


def compare(inst, S, *, seed=0, eps=None, want_f=True, params=None, **cfg):
    ctx = xrdvi.Context.from_instance(inst, S=S, **cfg)
    if params is None:
        loc, raw = perturbed_params(ctx, seed)
    else:
        loc, raw = params
        ctx.set_params(loc, raw)
    if eps is None:
        eps = synth.normals(1000 + seed, S, inst.K)
    g = ctx.elbo_grad(eps, want_f=want_f)
    P = oracle.Problem.from_instance(inst)
    o = P.elbo_grad(loc.astype(np.float64), raw.astype(np.float64), eps.astype(np.float64), want_f=want_f)
    ctx.close()
    return g, o


def assert_parity(g, o, check_f=True):
    if check_f:
        rel = np.abs(g["f"] - o["f"]) / np.abs(o["f"])
        assert rel.max() <= F_TOL, rel.max()
    np.testing.assert_allclose(g["ll"], o["ll"], rtol=F_TOL)
    assert np.max(np.abs(g["lpj"] - o["lpj"]) / np.maximum(1.0, np.abs(o["lpj"]))) <= F_TOL
    assert abs(g["elbo"] - o["elbo"]) <= F_TOL * abs(o["elbo"])
    for b in range(10):
        ref = np.max(np.abs(o["grad"][:, b]))
        err = np.max(np.abs(g["grad"][:, b] - o["grad"][:, b]))
        assert err <= G_TOL * ref, (b, err, ref)


@pytest.mark.parametrize("K,M,N,S,seed", [
    (3, 6, 300, 4, 1),      # three tiles, ragged tail of 44 points
    (8, 20, 1000, 8, 2),    # several phases, 8 tiles, ragged tail
    (1, 1, 1, 1, 3),        # a single point, a single peak, a single sample
    (2, 5, 128, 3, 4),      # exactly one tile
    (5, 12, 512, 16, 5),    # exactly four tiles
])
def test_elbo_grad_parity_small(K, M, N, S, seed):
    inst = synth.small_problem(K=K, M=M, N=N, S=S, seed=seed, x_step=max(0.02, 15.0 / N))
    g, o = compare(inst, S, seed=seed)
    assert_parity(g, o)


def test_parity_fd_sub_instance():
    inst = synth.config(2)
    g, o = compare(inst, 8, seed=7)
    assert_parity(g, o)


def test_parity_bf16_intensity_table_against_rounded_oracle():
    """With the bfloat16 intensity table the kernels match the oracle fed the
    same bf16-rounded intensities."""
    import torch
    inst = synth.small_problem(K=4, M=10, N=700, S=4, seed=9)
    rounded = torch.tensor(inst.inten).to(torch.bfloat16).to(torch.float32).numpy()
    inst_r = synth.Instance(**{**inst.__dict__, "inten": rounded})
    ctx = xrdvi.Context.from_instance(inst, S=4, flags=xrdvi.FLAG_BF16_INT)
    loc, raw = perturbed_params(ctx, 9)
    eps = synth.normals(9, 4, inst.K)
    g = ctx.elbo_grad(eps, want_f=True)
    o = oracle.Problem.from_instance(inst_r).elbo_grad(loc, raw, eps.astype(np.float64), want_f=True)
    assert_parity(g, o)


def test_peaks_outside_grid_and_zero_counts():
    inst = synth.small_problem(K=3, M=6, N=400, S=4, seed=11)
    pos = inst.pos.copy()
    pos[0] = 5.0      # far left of the grid
    pos[-1] = 170.0   # far right of the grid
    y = inst.y.copy()
    y[::7] = 0.0
    inst2 = synth.Instance(**{**inst.__dict__, "pos": pos, "y": y})
    g, o = compare(inst2, 4, seed=11)
    assert_parity(g, o)


def _shuffled_within_phases(inst, seed):
    rng = np.random.default_rng(seed)
    pos, inten = inst.pos.copy(), inst.inten.copy()
    for k in range(inst.K):
        a, b = inst.offsets[k], inst.offsets[k + 1]
        perm = rng.permutation(b - a) + a
        pos[a:b], inten[a:b] = inst.pos[perm], inst.inten[perm]
    # equal positions inside a phase exercise the stable order of the sort
    pos[inst.offsets[0] + 1] = pos[inst.offsets[0]]
    assert np.any(np.diff(pos) < 0)
    return synth.Instance(**{**inst.__dict__, "pos": pos, "inten": inten})


@pytest.mark.parametrize("device_arrays", [False, True])
def test_unsorted_peak_tables_match_the_oracle(device_arrays):
    """The candidate list of a phase is an unordered set of (p_m, I_m) pairs
    (App. A.1): xrdvi_create sorts each phase itself, from host arrays and from
    device arrays (XRDVI_FLAG_DEVICE_PTRS), and the result matches the oracle
    (whose direct sums do not depend on the order) element by element."""
    import torch
    inst = _shuffled_within_phases(synth.small_problem(K=6, M=15, N=1100, S=6, seed=21), 21)
    if device_arrays:
        d = [torch.tensor(a, device="cuda") for a in (inst.offsets, inst.pos, inst.inten, inst.x, inst.y, inst.bg)]
        ctx = xrdvi.Context.from_device(inst.K, inst.N, *[t.data_ptr() for t in d], S=6)
    else:
        ctx = xrdvi.Context.from_instance(inst, S=6)
    loc, raw = perturbed_params(ctx, 21)
    eps = synth.normals(1021, 6, inst.K)
    g = ctx.elbo_grad(eps, want_f=True)
    ctx.close()
    o = oracle.Problem.from_instance(inst).elbo_grad(loc.astype(np.float64), raw.astype(np.float64),
                                                    eps.astype(np.float64), want_f=True)
    assert_parity(g, o)


def test_non_finite_fit_is_reported_and_cleared():
    """A state whose intensity overflows FP32 (h = e^200) makes the profile,
    the ELBO and the gradient non-finite: the fit returns ENONFINITE (the
    gradient reduction flags a NaN or infinite entry on the device, the host
    checks it with the last ELBO).  The flag is cleared when read, so the fit
    resumes normally from a checkpoint taken before."""
    inst = synth.small_problem(K=3, M=6, N=300, S=4, seed=17)
    ctx = xrdvi.Context.from_instance(inst, S=4)
    loc0, raw0 = ctx.params()
    good = ctx.state()
    loc = loc0.copy()
    loc[:, 0] = 200.0
    ctx.set_params(loc, raw0)
    with pytest.raises(xrdvi.XrdviError) as e:
        ctx.fit(3)
    assert e.value.status == 5
    with pytest.raises(xrdvi.XrdviError) as e:
        ctx.elbo_grad(synth.normals(3, 4, inst.K))
    assert e.value.status == 5
    ctx.set_state(good)   # parameters and Adam moments from before the overflow
    tr = ctx.fit(3)
    ctx.close()
    assert np.all(np.isfinite(tr))


def test_alpha_below_clamp():
    inst = synth.small_problem(K=2, M=5, N=300, S=4, seed=12)
    ctx = xrdvi.Context.from_instance(inst, S=4)
    loc, raw = ctx.params()
    loc[:, 4] = -0.3
    raw[:, 4] = -30.0
    ctx.close()
    g, o = compare(inst, 4, params=(loc, raw))
    assert_parity(g, o)
    np.testing.assert_allclose(g["grad"][:, 4], o["grad"][:, 4], rtol=1e-5)


def test_naive_sum_flag_still_within_tolerance_on_small_case():
    inst = synth.small_problem(K=3, M=6, N=300, S=4, seed=1)
    g, o = compare(inst, 4, seed=1, flags=xrdvi.FLAG_NAIVE_SUM)
    assert_parity(g, o)


def test_philox_noise_matches_oracle_stream():
    """eps = NULL draws the fit stream (Philox4x32-10 + Box-Muller, step 0);
    the oracle's independent generator with the same key and counters gives
    the same normals, hence the same ELBO and gradient."""
    inst = synth.small_problem(K=4, M=8, N=500, S=8, seed=13)
    ctx = xrdvi.Context.from_instance(inst, S=8, seed=987654321)
    loc, raw = perturbed_params(ctx, 13)
    g_rng = ctx.elbo_grad(None, want_f=True)
    eps = oracle.normals(987654321, 0, 0, 8, inst.K).astype(np.float32)
    g_inj = ctx.elbo_grad(eps, want_f=True)
    ctx.close()
    assert abs(g_rng["elbo"] - g_inj["elbo"]) <= 1e-6 * abs(g_inj["elbo"])
    np.testing.assert_allclose(g_rng["f"], g_inj["f"], rtol=1e-5)
    for b in range(10):
        ref = np.max(np.abs(g_inj["grad"][:, b]))
        assert np.max(np.abs(g_rng["grad"][:, b] - g_inj["grad"][:, b])) <= 1e-4 * ref


def test_gpu_philox_matches_published_known_answers():
    """The device generator that draws the fit's noise reproduces the
    published Philox4x32-10 known-answer vectors (Salmon et al., SC'11;
    tests/golden/philox4x32_10_kat.json), bit for bit, and agrees with the
    oracle's generator on a spread of counters and keys."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.json")
    vecs = json.load(open(path))["vectors"]
    h = lambda ws: [int(w, 16) for w in ws]
    ctr = np.array([h(v["counter"]) for v in vecs], dtype=np.uint32)
    key = np.array([h(v["key"]) for v in vecs], dtype=np.uint32)
    out = xrdvi.xrdvi_philox4x32_10(ctr, key)
    np.testing.assert_array_equal(out, np.array([h(v["output"]) for v in vecs], dtype=np.uint32))
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 2 ** 32, size=(300, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(300, 2), dtype=np.uint64).astype(np.uint32)
    out = xrdvi.xrdvi_philox4x32_10(ctr, key)
    ref = np.array([oracle.philox(c.tolist(), k.tolist()) for c, k in zip(ctr, key)], dtype=np.uint32)
    np.testing.assert_array_equal(out, ref)


def test_adam_steps_match_oracle():
    """A few fused SVI steps (sample, profile, backward, Adam) against the
    oracle's fit loop on the same noise stream."""
    inst = synth.small_problem(K=3, M=6, N=300, S=4, seed=14)
    ctx = xrdvi.Context.from_instance(inst, S=4, seed=4242)
    loc0, raw0 = ctx.params()
    trace = ctx.fit(3)
    loc1, raw1 = ctx.params()
    ctx.close()
    P = oracle.Problem.from_instance(inst)
    ref = P.fit(4, 3, 4242, loc=loc0.astype(np.float64), raw=raw0.astype(np.float64))
    np.testing.assert_allclose(trace, ref["trace"], rtol=F_TOL)
    np.testing.assert_allclose(loc1, ref["loc"], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(raw1, ref["raw"], rtol=1e-5, atol=1e-5)


def test_fit_trace_equals_single_step_elbo_and_is_deterministic():
    inst = synth.small_problem(K=3, M=6, N=300, S=4, seed=15)
    c1 = xrdvi.Context.from_instance(inst, S=4, seed=77)
    e0 = c1.elbo_grad(None)["elbo"]
    tr = c1.fit(40)
    assert tr[0] == e0
    p1 = c1.params()
    c2 = xrdvi.Context.from_instance(inst, S=4, seed=77)
    tr2 = np.concatenate([c2.fit(17), c2.fit(23)])
    p2 = c2.params()
    np.testing.assert_array_equal(tr, tr2)
    np.testing.assert_array_equal(p1[0], p2[0])
    np.testing.assert_array_equal(p1[1], p2[1])


def test_checkpoint_resume_is_bit_identical():
    inst = synth.small_problem(K=4, M=8, N=500, S=8, seed=16)
    a = xrdvi.Context.from_instance(inst, S=8, seed=5)
    a.fit(25)
    st = a.state()
    ta = a.fit(30)
    pa = a.params()
    b = xrdvi.Context.from_instance(inst, S=8, seed=999)   # seed restored from the state
    b.set_state(st)
    tb = b.fit(30)
    pb = b.params()
    np.testing.assert_array_equal(ta, tb)
    np.testing.assert_array_equal(pa[0], pb[0])
    np.testing.assert_array_equal(pa[1], pb[1])
    assert b.info.step == 55


@pytest.mark.slow
def test_full_size_k50_parity_sampled_and_gradient():
    """K=50, N=4500, S=256 in the benchmark's launch configuration: profile
    rows and log-likelihoods of sampled draws against the oracle, and the
    full gradient and ELBO against the oracle's (OpenMP) evaluation."""
    inst = synth.config(1)
    S = inst.S
    ctx = xrdvi.Context.from_instance(inst, S=S)
    loc, raw = perturbed_params(ctx, 21, scale=0.02)
    eps = synth.normals(2100, S, inst.K)
    g = ctx.elbo_grad(eps, want_f=True)
    ctx.close()
    P = oracle.Problem.from_instance(inst)
    rows = [0, 1, 97, 255]
    u, th = P.theta(loc.astype(np.float64), raw.astype(np.float64), eps[rows].astype(np.float64))
    f = P.profile(th)
    rel = np.abs(g["f"][rows] - f) / f
    assert rel.max() <= F_TOL
    for r, s in enumerate(rows):
        assert abs(g["ll"][s] - P.loglik(f[r])) <= F_TOL * abs(P.loglik(f[r]))
    o = P.elbo_grad(loc.astype(np.float64), raw.astype(np.float64), eps.astype(np.float64))
    assert abs(g["elbo"] - o["elbo"]) <= F_TOL * abs(o["elbo"])
    for b in range(10):
        ref = np.max(np.abs(o["grad"][:, b]))
        assert np.max(np.abs(g["grad"][:, b] - o["grad"][:, b])) <= G_TOL * ref, b


def test_posterior_parity_with_oracle():
    """Same fitted q, same Philox posterior stream (tag 1): marginal
    inclusion probabilities, top-M combinations and IS evidence."""
    inst = synth.make_problem(K=6, m_lo=6, m_hi=10, x_lo=20.0, x_step=0.04, N=700,
                              n_planted=2, S=8, iters=300, seed=31, name="post")
    ctx = xrdvi.Context.from_instance(inst, S=8, seed=3)
    ctx.fit(600)
    loc, raw = ctx.params()
    Sp, seed = 512, 99
    g = ctx.posterior(Sp, seed, top_m=12)
    ctx.close()
    P = oracle.Problem.from_instance(inst)
    o = opost.posterior(P, loc.astype(np.float64), raw.astype(np.float64), Sp, seed=seed, top_m=12)
    assert np.max(np.abs(g["pi"] - o["pi"])) <= 2.0 / (Sp + 1)
    np.testing.assert_allclose(g["combo_logp"], o["combo_logp"], atol=1e-3)
    assert abs(g["log_evidence"] - o["log_evidence"]) <= F_TOL * abs(o["log_evidence"])
    assert g["coverage_log"] <= 1e-12
    top = set(np.flatnonzero(g["combos"][0]).tolist())
    assert top == set(inst.planted.tolist())


def test_recovery_tiny_config():
    """K=8, N=2000, S=16, 300 steps: the planted phases are identified."""
    inst = synth.config(0)
    ctx = xrdvi.Context.from_instance(inst, S=inst.S, seed=1)
    tr = ctx.fit(inst.iters)
    assert np.all(np.isfinite(tr)) and tr[-1] > tr[0]
    # more steps: the sparse prior needs time to shrink decoys from the start value
    ctx.fit(1500)
    res = ctx.posterior(1024, 5, top_m=4)
    ctx.close()
    top = set(np.flatnonzero(res["combos"][0]).tolist())
    assert top == set(inst.planted.tolist()), (res["pi"], inst.planted)


def test_contexts_with_different_table_sizes_coexist():
    """A context with a large peak table keeps working after a context with a
    small table is created (the kernels' shared-memory limit is global)."""
    big = synth.small_problem(K=40, M=60, N=500, S=4, seed=41)
    small = synth.small_problem(K=2, M=3, N=200, S=4, seed=42)
    cb = xrdvi.Context.from_instance(big, S=4)
    e1 = cb.elbo_grad(synth.normals(1, 4, big.K))["elbo"]
    cs = xrdvi.Context.from_instance(small, S=4)
    cs.elbo_grad(synth.normals(2, 4, small.K))
    e2 = cb.elbo_grad(synth.normals(1, 4, big.K))["elbo"]
    cb.close()
    cs.close()
    assert e1 == e2


def test_create_from_device_arrays_equals_host_create():
    import torch
    inst = synth.small_problem(K=4, M=8, N=600, S=4, seed=23, x_step=0.03)
    eps = synth.normals(23, 4, inst.K)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in
         (inst.offsets.astype(np.int32), inst.pos, inst.inten, inst.x, inst.y, inst.bg)]
    torch.cuda.synchronize()
    cd = xrdvi.Context.from_device(inst.K, inst.N, *[t.data_ptr() for t in d], S=4)
    ch = xrdvi.Context.from_instance(inst, S=4)
    a, b = cd.elbo_grad(eps, want_f=True), ch.elbo_grad(eps, want_f=True)
    cd.close()
    ch.close()
    assert a["elbo"] == b["elbo"]
    np.testing.assert_array_equal(a["grad"], b["grad"])
    np.testing.assert_array_equal(a["f"], b["f"])


def test_posterior_parity_area_normalised():
    """Posterior of the area-normalised model against the oracle's (area of a
    phase = h sum I) on the same fitted q and draws."""
    inst = synth.small_problem(K=5, M=10, N=600, S=8, seed=26, x_step=0.04)
    c = xrdvi.Context.from_instance(inst, S=8, seed=3, flags=xrdvi.FLAG_AREA_NORM)
    c.fit(200)
    loc, raw = c.params()
    post = c.posterior(256, 11, top_m=4)
    c.close()
    P = oracle.Problem.from_instance(inst, normalisation="area")
    ref = opost.posterior(P, loc.astype(np.float64), raw.astype(np.float64), 256, seed=11, top_m=4)
    assert np.max(np.abs(post["pi"] - ref["pi"])) <= 2.0 / 257
    assert abs(post["log_evidence"] - ref["log_evidence"]) <= F_TOL * abs(ref["log_evidence"])
