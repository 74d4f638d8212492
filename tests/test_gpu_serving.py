"""Continuous-batching fit server: results equal to standalone fits (fits of
different K and N share every step's kernel launches, and a variant fit runs
its own kernels between them), admission by device-memory footprint,
continuous admission while fits run, device-side overlap, cancellation."""
import time

import numpy as np
import pytest

from paper_2501_09308_gb300 import serving, synth, xrdvi

pytestmark = pytest.mark.gpu

ITERS = 150


def _problems():
    return [synth.small_problem(K=3, M=6, N=300, S=8, seed=71),
            synth.small_problem(K=6, M=10, N=900, S=8, seed=72, x_step=0.03),
            synth.small_problem(K=9, M=14, N=1500, S=8, seed=73, x_step=0.02)]


def _alone(inst, seed):
    c = xrdvi.Context.from_instance(inst, S=inst.S, seed=seed)
    tr = c.fit(ITERS)
    post = c.posterior(256, 5, top_m=4)
    loc, raw = c.params()
    c.close()
    return tr[-1], post, loc, raw


def test_served_results_equal_standalone_results():
    """Each fit in the mix (three at once on three slots) equals the same fit
    run alone: identical kernels, fixed reduction orders, no shared state."""
    probs = _problems()
    srv = serving.Server(hbm_budget=8 << 30, max_slots=3)
    ids = [srv.submit(p, iters=ITERS, S_post=256, post_seed=5, top_m=4, seed=100 + i) for i, p in enumerate(probs)]
    served = [srv.wait(i) for i in ids]
    srv.close()
    spans = [(r["t_admit"], r["t_done"]) for r in served]
    overlap = any(a[0] < b[1] and b[0] < a[1] for i, a in enumerate(spans) for b in spans[i + 1:])
    assert overlap, spans
    for i, (p, r) in enumerate(zip(probs, served)):
        assert r["status"] == 0
        e, post, loc, raw = _alone(p, 100 + i)
        np.testing.assert_array_equal(r["loc"], loc)
        np.testing.assert_array_equal(r["raw"], raw)
        assert r["final_elbo"] == e
        np.testing.assert_array_equal(r["pi"], post["pi"])
        np.testing.assert_array_equal(r["combo_logp"], post["combo_logp"])


def test_batched_and_variant_fits_in_one_mix_equal_their_standalone_fits():
    """Five fits of different K, N and peak counts, one of them with the
    angle-dependent width (outside the batched step: its own kernels), one
    with the Gaussian likelihood and fixed r (inside it): each result equals
    the standalone fit bit for bit."""
    probs = _problems() + [synth.small_problem(K=5, M=9, N=1100, S=8, seed=77, x_step=0.04),
                           synth.small_problem(K=4, M=7, N=700, S=8, seed=78)]
    extra = [{}, {}, {}, {"flags": xrdvi.FLAG_SEC_WIDTH},
             {"flags": xrdvi.FLAG_GAUSS_LIK | xrdvi.FLAG_FIX_R, "fix_r_value": 0.4}]
    srv = serving.Server(hbm_budget=8 << 30, max_slots=5)
    ids = [srv.submit(p, iters=ITERS, S_post=128, post_seed=6, top_m=4, seed=200 + i, **extra[i])
           for i, p in enumerate(probs)]
    served = [srv.wait(i) for i in ids]
    srv.close()
    for i, (p, r) in enumerate(zip(probs, served)):
        assert r["status"] == 0, r
        c = xrdvi.Context.from_instance(p, S=p.S, seed=200 + i, **extra[i])
        tr = c.fit(ITERS)
        post = c.posterior(128, 6, top_m=4)
        loc, raw = c.params()
        c.close()
        np.testing.assert_array_equal(r["loc"], loc)
        np.testing.assert_array_equal(r["raw"], raw)
        assert r["final_elbo"] == tr[-1]
        np.testing.assert_array_equal(r["pi"], post["pi"])


def test_fit_batch_equals_standalone_fits():
    """xrdvi_fit_batch: five contexts of different K, N and S (gates, bf16
    intensities and area normalisation inside the batched step, the
    angle-dependent width with its own kernels) advanced together end exactly
    where xrdvi_fit leaves each of them, also when the steps are split over
    several calls; a context listed twice is rejected."""
    probs = _problems() + [synth.small_problem(K=5, M=9, N=1100, S=32, seed=77, x_step=0.04),
                           synth.small_problem(K=4, M=7, N=700, S=3, seed=78)]
    extra = [{}, {"flags": xrdvi.FLAG_GATES}, {"flags": xrdvi.FLAG_BF16_INT}, {"flags": xrdvi.FLAG_SEC_WIDTH},
             {"flags": xrdvi.FLAG_AREA_NORM}]
    ref = []
    for i, p in enumerate(probs):
        c = xrdvi.Context.from_instance(p, S=p.S, seed=300 + i, **extra[i])
        tr = c.fit(ITERS)
        ref.append((c.params(), tr[-1]))
        c.close()
    cs = [xrdvi.Context.from_instance(p, S=p.S, seed=300 + i, **extra[i]) for i, p in enumerate(probs)]
    last = xrdvi.xrdvi_fit_batch([c.h for c in cs], 37)
    last = xrdvi.xrdvi_fit_batch([c.h for c in cs], ITERS - 37)
    for c, (params, e), le in zip(cs, ref, last):
        np.testing.assert_array_equal(c.params()[0], params[0])
        np.testing.assert_array_equal(c.params()[1], params[1])
        assert le == e
        assert c.info.step == ITERS
    with pytest.raises(xrdvi.XrdviError) as err:
        xrdvi.xrdvi_fit_batch([cs[0].h, cs[0].h], 1)
    assert err.value.status == 1
    for c in cs:
        c.close()


def test_fit_batch_reuses_graphs_only_for_the_same_members():
    """xrdvi_fit_batch keeps the graphs it captured for a member set: repeated
    calls on the same set, a member restored from a saved state (new captured
    arguments), the set in another order and a subset each end exactly where
    xrdvi_fit leaves the same contexts."""
    probs = _problems()
    cs = [xrdvi.Context.from_instance(p, S=p.S, seed=500 + i) for i, p in enumerate(probs)]
    rs = [xrdvi.Context.from_instance(p, S=p.S, seed=500 + i) for i, p in enumerate(probs)]
    h = [c.h for c in cs]
    xrdvi.xrdvi_fit_batch(h, 20)
    xrdvi.xrdvi_fit_batch(h, 20)
    saved = cs[1].state()
    xrdvi.xrdvi_fit_batch(h, 5)
    cs[1].set_state(saved)
    xrdvi.xrdvi_fit_batch(h[::-1], 17)
    xrdvi.xrdvi_fit_batch(h[:2], 16)
    last = xrdvi.xrdvi_fit_batch(h, 3)
    for r, n in zip(rs, (81, 76, 65)):
        tr = r.fit(n)
    for c, r, le, n in zip(cs, rs, last, (81, 76, 65)):
        np.testing.assert_array_equal(c.params()[0], r.params()[0])
        np.testing.assert_array_equal(c.params()[1], r.params()[1])
        assert c.info.step == n
    assert last[2] == tr[-1]
    # a member closed and a new context in its place (possibly at the same
    # address): the kept graphs must not be replayed
    cs[2].close()
    rs[2].close()
    cs[2] = xrdvi.Context.from_instance(probs[2], S=probs[2].S, seed=600)
    rs[2] = xrdvi.Context.from_instance(probs[2], S=probs[2].S, seed=600)
    xrdvi.xrdvi_fit_batch([c.h for c in cs], 16)
    for r in rs:
        r.fit(16)
    for c, r in zip(cs, rs):
        np.testing.assert_array_equal(c.params()[0], r.params()[0])
        np.testing.assert_array_equal(c.params()[1], r.params()[1])
    for c in cs + rs:
        c.close()


def test_fit_batch_with_large_peak_tables_equals_standalone_fits():
    """Two fits whose peak tables (over 3500 peaks) take the compact layout
    share the multi-fit profile launches, beside a small fit with the wide
    layout; a fit with twice as many peaks sits alone in its occupancy group.
    Each ends bit-identical to its standalone fit."""
    probs = [synth.small_problem(K=60, M=70, N=900, S=8, seed=95, x_step=0.03),
             synth.small_problem(K=64, M=70, N=1300, S=8, seed=96, x_step=0.02),
             synth.small_problem(K=4, M=8, N=700, S=8, seed=97),
             synth.small_problem(K=150, M=100, N=600, S=4, seed=98, x_step=0.05)]
    assert int(probs[0].offsets[-1]) > 3500 and int(probs[1].offsets[-1]) > 3500
    ref = []
    for i, p in enumerate(probs):
        c = xrdvi.Context.from_instance(p, S=p.S, seed=400 + i)
        c.fit(40)
        ref.append(c.params())
        c.close()
    cs = [xrdvi.Context.from_instance(p, S=p.S, seed=400 + i) for i, p in enumerate(probs)]
    xrdvi.xrdvi_fit_batch([c.h for c in cs], 40)
    for c, (loc, raw) in zip(cs, ref):
        np.testing.assert_array_equal(c.params()[0], loc)
        np.testing.assert_array_equal(c.params()[1], raw)
        c.close()


def test_fit_batch_with_fits_that_fill_the_gpu_equals_standalone_fits():
    """Two full-size fits (the K=50 workload and a K=77 serving request, S=256:
    enough work items to fill the GPU alone, so each runs its own profile and
    likelihood kernels inside the batched step) beside a small fit that takes
    the shared multi-fit launches: each ends bit-identical to its standalone
    fit, across two calls."""
    probs = [synth.config(1), synth.config(4, instance=1), synth.small_problem(K=5, M=9, N=900, S=8, seed=81)]
    ref = []
    for i, p in enumerate(probs):
        c = xrdvi.Context.from_instance(p, S=p.S, seed=700 + i)
        tr = c.fit(24)
        ref.append((c.params(), tr[-1]))
        c.close()
    cs = [xrdvi.Context.from_instance(p, S=p.S, seed=700 + i) for i, p in enumerate(probs)]
    xrdvi.xrdvi_fit_batch([c.h for c in cs], 16)
    last = xrdvi.xrdvi_fit_batch([c.h for c in cs], 8)
    for c, (params, e), le in zip(cs, ref, last):
        np.testing.assert_array_equal(c.params()[0], params[0])
        np.testing.assert_array_equal(c.params()[1], params[1])
        assert le == e
        c.close()


def test_batched_fits_overlap_on_the_device():
    """Eight small fits served together finish in much less time than the
    same fits run one after another: their steps share kernel launches
    instead of taking turns on the GPU."""
    probs = [synth.small_problem(K=4 + i % 5, M=8, N=600 + 150 * i, S=16, seed=90 + i) for i in range(8)]
    iters = 300
    for p in probs[:2]:   # warm-up (module loading, pool growth)
        c = xrdvi.Context.from_instance(p, S=p.S)
        c.fit(20)
        c.close()
    t0 = time.perf_counter()
    for p in probs:
        c = xrdvi.Context.from_instance(p, S=p.S)
        c.fit(iters)
        c.close()
    t_seq = time.perf_counter() - t0
    srv = serving.Server(hbm_budget=8 << 30, max_slots=8)
    t0 = time.perf_counter()
    ids = [srv.submit(p, iters=iters, S_post=0) for p in probs]
    res = [srv.wait(i) for i in ids]
    t_mix = time.perf_counter() - t0
    srv.close()
    assert all(r["status"] == 0 for r in res)
    print(f"\n8 fits x {iters} steps: one after another {t_seq:.3f} s, served together {t_mix:.3f} s")
    assert t_mix < 0.6 * t_seq, (t_mix, t_seq)


def test_admission_by_footprint_serialises_when_only_one_fits():
    """Three same-size requests, three free slots, but a budget of 1.5
    footprints: they must run one after another."""
    probs = [synth.small_problem(K=6, M=10, N=900, S=8, seed=80 + i, x_step=0.03) for i in range(3)]
    fp = [xrdvi.xrdvi_footprint_bytes(p.K, p.N, int(p.offsets[-1]), p.S, 256, 4) for p in probs]
    assert len(set(fp)) == 1
    srv = serving.Server(hbm_budget=int(fp[0] * 1.5), max_slots=3)
    ids = [srv.submit(p, iters=ITERS, S_post=256, post_seed=5, top_m=4) for p in probs]
    res = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    spans = sorted((r["t_admit"], r["t_done"]) for r in res)
    for a, b in zip(spans, spans[1:]):
        assert a[1] <= b[0] + 1e-6, spans
    assert st["peak_bytes"] <= int(fp[0] * 1.5)
    assert [r["footprint_bytes"] for r in res] == fp


def test_requests_arriving_during_a_fit_are_admitted_before_it_ends():
    long = synth.small_problem(K=9, M=14, N=1500, S=8, seed=74, x_step=0.02)
    short = synth.small_problem(K=3, M=6, N=300, S=8, seed=75)
    srv = serving.Server(hbm_budget=8 << 30, max_slots=2)
    a = srv.submit(long, iters=3000, S_post=64, top_m=2)
    while srv.stats()["running"] == 0:
        time.sleep(0.005)
    b = srv.submit(short, iters=50, S_post=64, top_m=2)
    rb = srv.wait(b)
    ra = srv.wait(a)
    srv.close()
    assert rb["t_admit"] < ra["t_done"] and rb["t_done"] < ra["t_done"]


def test_invalid_request_completes_with_its_error_and_the_others_run():
    """A problem that fails validation (a negative count) is rejected when its
    context is created: its result carries EINVAL, and a valid request served
    beside it completes normally."""
    good = _problems()[0]
    y = good.y.copy()
    y[5] = -1.0
    bad = synth.Instance(**{**good.__dict__, "y": y})
    srv = serving.Server(hbm_budget=8 << 30, max_slots=2)
    rb = srv.submit(bad, iters=20, S_post=0)
    rg = srv.submit(good, iters=20, S_post=0)
    out_b, out_g = srv.wait(rb), srv.wait(rg)
    srv.close()
    assert out_b["status"] == 1
    assert out_g["status"] == 0 and np.isfinite(out_g["final_elbo"])


def test_zero_step_request_returns_the_posterior_of_the_initial_q():
    """iters = 0: the server skips the fit and draws the posterior of the
    standard initial q, as a standalone context does."""
    p = _problems()[1]
    srv = serving.Server(hbm_budget=8 << 30, max_slots=2)
    r = srv.wait(srv.submit(p, iters=0, S_post=128, post_seed=3, top_m=2, seed=5))
    srv.close()
    c = xrdvi.Context.from_instance(p, S=p.S, seed=5)
    post = c.posterior(128, 3, top_m=2)
    c.close()
    assert r["status"] == 0
    np.testing.assert_array_equal(r["pi"], post["pi"])


def test_replay_writes_one_jsonl_record_per_request(tmp_path):
    """The request loop's log: one JSON line per request with its arrival,
    admission and completion times, footprint and status."""
    import json
    probs = _problems()[:2]
    srv = serving.Server(hbm_budget=8 << 30, max_slots=2)
    path = tmp_path / "requests.jsonl"
    res = serving.replay_arrivals(srv, probs, [0.0, 0.01], jsonl=str(path), iters=30, S_post=0)
    srv.close()
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert len(lines) == 2
    for rec, p, r in zip(lines, probs, res):
        assert rec["K"] == p.K and rec["N"] == p.N and rec["status"] == 0
        assert rec["t_submit"] <= rec["t_admit"] <= rec["t_done"]
        assert rec["latency_s"] == pytest.approx(r["latency"])


def test_request_over_budget_is_rejected():
    p = _problems()[2]
    srv = serving.Server(hbm_budget=1 << 20, max_slots=1)
    with pytest.raises(xrdvi.XrdviError) as e:
        srv.submit(p, iters=10)
    srv.close()
    assert e.value.status == 2


def test_cancel_a_queued_request():
    long = synth.small_problem(K=9, M=14, N=1500, S=8, seed=76, x_step=0.02)
    srv = serving.Server(hbm_budget=8 << 30, max_slots=1)
    a = srv.submit(long, iters=2000, S_post=64, top_m=2)
    b = srv.submit(long, iters=2000, S_post=64, top_m=2)
    srv.cancel(b)
    rb = srv.wait(b)
    ra = srv.wait(a)
    srv.close()
    assert rb["status"] == 7 and ra["status"] == 0


def test_footprint_bound_covers_the_context_allocation():
    for p in _problems() + [synth.config(1)]:
        c = xrdvi.Context.from_instance(p, S=p.S)
        c.posterior(512, 1, top_m=8)
        used = c.info.device_bytes
        c.close()
        bound = xrdvi.xrdvi_footprint_bytes(p.K, p.N, int(p.offsets[-1]), p.S, 512, 8)
        assert used <= bound <= 2 * used + (8 << 20), (used, bound)
