"""Binary-Concrete phase gates (model variant) on the GPU against the FP64
oracle on the same inputs, injected normals and injected logistic gate noise.

Tolerances as for the plain path: profile, LL and ELBO 1e-5 relative;
gradient blocks and the gate-logit gradient 1e-4 of their max-norm.  Gate
logits away from 0 are set through the checkpoint blob, whose last 3K floats
are the logits and their two Adam moments."""
import numpy as np
import pytest

import oracle
import oracle.posterior as opost
from paper_2501_09308_gb300 import synth, xrdvi

pytestmark = pytest.mark.gpu

F_TOL = 1e-5
G_TOL = 1e-4


def _set_logits(ctx, a):
    s = bytearray(ctx.state())
    K = a.size
    s[len(s) - 12 * K:len(s) - 8 * K] = np.asarray(a, dtype=np.float32).tobytes()
    ctx.set_state(bytes(s))


def _logistic(seed, S, K):
    u = np.random.default_rng(seed).uniform(1e-6, 1 - 1e-6, (S, K))
    return (np.log(u) - np.log1p(-u)).astype(np.float32)


def _run(inst, S, seed, flags=0, logits=None, tau=2.0 / 3.0, prior=0.5, **okw):
    ctx = xrdvi.Context.from_instance(inst, S=S, flags=xrdvi.FLAG_GATES | flags, gate_tau=tau, gate_prior=prior)
    loc, raw = ctx.params()
    rng = np.random.default_rng(seed)
    loc = loc + rng.normal(0, 0.05, loc.shape).astype(np.float32)
    raw = raw + rng.normal(0, 0.1, raw.shape).astype(np.float32)
    ctx.set_params(loc, raw)
    a = (rng.normal(0, 1.5, inst.K) if logits is None else np.asarray(logits)).astype(np.float32)
    _set_logits(ctx, a)
    eps = synth.normals(3000 + seed, S, inst.K)
    L = _logistic(4000 + seed, S, inst.K)
    g = ctx.elbo_grad(eps, want_f=True, gate_noise=L)
    g["grad_gate"] = ctx.gates()["grad"]
    np.testing.assert_array_equal(ctx.gates()["logits"], a)
    ctx.close()
    P = oracle.Problem.from_instance(inst, gates=True, gate_tau=tau, gate_prior=prior, **okw)
    P.gate_a[:] = a.astype(np.float64)
    o = P.elbo_grad(loc.astype(np.float64), raw.astype(np.float64), eps.astype(np.float64), want_f=True,
                    gate_noise=L.astype(np.float64))
    return g, o


def _check(g, o):
    assert np.max(np.abs(g["f"] - o["f"]) / np.maximum(np.abs(o["f"]), 1e-3 * np.max(np.abs(o["f"])))) <= F_TOL
    np.testing.assert_allclose(g["ll"], o["ll"], rtol=F_TOL)
    assert abs(g["elbo"] - o["elbo"]) <= F_TOL * abs(o["elbo"])
    for b in range(10):
        ref = np.max(np.abs(o["grad"][:, b]))
        err = np.max(np.abs(g["grad"][:, b] - o["grad"][:, b]))
        assert err <= G_TOL * ref, (b, err, ref)
    ref = np.max(np.abs(o["grad_gate"]))
    assert np.max(np.abs(g["grad_gate"] - o["grad_gate"])) <= G_TOL * ref


@pytest.mark.parametrize("K,M,N,S,seed", [(3, 6, 300, 4, 1), (8, 20, 1000, 8, 2), (1, 1, 1, 1, 3),
                                          (12, 30, 2100, 5, 4)])
def test_gated_parity(K, M, N, S, seed):
    inst = synth.small_problem(K=K, M=M, N=N, S=S, seed=seed, x_step=max(0.02, 15.0 / N))
    g, o = _run(inst, S, seed)
    _check(g, o)


def test_gated_parity_other_temperature_and_prior():
    inst = synth.small_problem(K=6, M=12, N=800, S=6, seed=5, x_step=0.03)
    g, o = _run(inst, 6, 5, tau=0.3, prior=0.1)
    _check(g, o)


@pytest.mark.parametrize("extra,okw", [(xrdvi.FLAG_AREA_NORM, {"normalisation": "area"}),
                                       (xrdvi.FLAG_SHARED_SHAPES, {"shapes": "shared"})])
def test_gated_parity_with_other_options(extra, okw):
    inst = synth.small_problem(K=5, M=10, N=700, S=6, seed=6, x_step=0.03)
    g, o = _run(inst, 6, 6, flags=extra, **okw)
    _check(g, o)


def test_wide_open_gates_give_the_ungated_profile():
    """Logits far above the noise: every z rounds to 1 in FP32 and the profile
    is the ungated one bit for bit."""
    inst = synth.small_problem(K=4, M=8, N=500, S=4, seed=7)
    eps = synth.normals(7, 4, inst.K)
    c0 = xrdvi.Context.from_instance(inst, S=4)
    f0 = c0.elbo_grad(eps, want_f=True)["f"]
    c0.close()
    c1 = xrdvi.Context.from_instance(inst, S=4, flags=xrdvi.FLAG_GATES)
    _set_logits(c1, np.full(inst.K, 60.0))
    f1 = c1.elbo_grad(eps, want_f=True, gate_noise=np.zeros((4, inst.K), np.float32))["f"]
    c1.close()
    np.testing.assert_array_equal(f1, f0)


def test_gated_fit_steps_match_oracle():
    """Three fused SVI steps (Philox normals and gate noise, Adam on the
    variational parameters and the gate logits) against the oracle's loop."""
    inst = synth.small_problem(K=3, M=6, N=300, S=8, seed=14)
    ctx = xrdvi.Context.from_instance(inst, S=8, seed=4244, flags=xrdvi.FLAG_GATES)
    loc0, raw0 = ctx.params()
    trace = ctx.fit(3)
    loc1, raw1 = ctx.params()
    a1 = ctx.gates()["logits"]
    ctx.close()
    ref = oracle.Problem.from_instance(inst, gates=True).fit(8, 3, 4244, loc=loc0.astype(np.float64),
                                                             raw=raw0.astype(np.float64))
    np.testing.assert_allclose(trace, ref["trace"], rtol=F_TOL)
    np.testing.assert_allclose(loc1, ref["loc"], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(raw1, ref["raw"], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(a1, ref["gate_a"], rtol=1e-5, atol=1e-5)


def test_gated_checkpoint_resume_is_bit_identical():
    inst = synth.small_problem(K=4, M=8, N=400, S=8, seed=15)
    a = xrdvi.Context.from_instance(inst, S=8, seed=9, flags=xrdvi.FLAG_GATES)
    a.fit(30)
    st = a.state()
    ta = a.fit(20)
    ga = a.gates()["logits"]
    b = xrdvi.Context.from_instance(inst, S=8, seed=1, flags=xrdvi.FLAG_GATES)
    b.set_state(st)
    tb = b.fit(20)
    gb = b.gates()["logits"]
    a.close()
    b.close()
    np.testing.assert_array_equal(ta, tb)
    np.testing.assert_array_equal(ga, gb)


def test_gated_posterior_parity():
    """Posterior with the gates: the area of a phase in a draw is z h sum I,
    and ln p - ln q of the gate logits joins each draw's log weight."""
    inst = synth.small_problem(K=5, M=10, N=600, S=8, seed=26, x_step=0.04)
    c = xrdvi.Context.from_instance(inst, S=8, seed=3, flags=xrdvi.FLAG_GATES)
    c.fit(200)
    loc, raw = c.params()
    a = c.gates()["logits"]
    post = c.posterior(256, 11, top_m=4)
    c.close()
    P = oracle.Problem.from_instance(inst, gates=True)
    P.gate_a[:] = a.astype(np.float64)
    ref = opost.posterior(P, loc.astype(np.float64), raw.astype(np.float64), 256, seed=11, top_m=4)
    assert np.max(np.abs(post["pi"] - ref["pi"])) <= 2.0 / 257
    assert abs(post["log_evidence"] - ref["log_evidence"]) <= F_TOL * abs(ref["log_evidence"])


def test_gated_fit_recovers_planted_phases_and_closes_decoy_gates():
    """The tiny workload fitted with gates: the planted phases carry the area,
    and their gate logits end above every decoy's."""
    inst = synth.config(0)
    c = xrdvi.Context.from_instance(inst, S=inst.S, flags=xrdvi.FLAG_GATES)
    c.fit(1000)
    a = c.gates()["logits"]
    post = c.posterior(512, 3, top_m=1)
    c.close()
    assert set(np.flatnonzero(post["combos"][0]).tolist()) == set(inst.planted.tolist())
    decoys = np.setdiff1d(np.arange(inst.K), inst.planted)
    assert np.min(a[inst.planted]) > np.max(a[decoys])
