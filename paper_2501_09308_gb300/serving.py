"""Continuous-batching request loop over the library's fit server.

``Server`` wraps ``xrdvi_server_*`` (the admission, slots, streams and memory
pool are native); ``replay_arrivals`` drives it with a timed request stream
(Poisson arrivals from ``synth.arrival_times``) and collects per-request
time-to-posterior (completion minus arrival).
"""
from __future__ import annotations

import time

import numpy as np

from . import xrdvi


class Server:
    def __init__(self, hbm_budget: int, max_slots: int):
        self.h = xrdvi.xrdvi_server_create(hbm_budget, max_slots)
        self._meta = {}

    def submit(self, inst, *, iters=None, S_post=4096, post_seed=1, top_m=8, **cfg):
        cfg.setdefault("S", inst.S)
        c = xrdvi.xrdvi_config_default(**cfg)
        rid = xrdvi.xrdvi_server_submit(self.h, inst.offsets, inst.pos, inst.inten, inst.x, inst.y, inst.bg, c,
                                        inst.iters if iters is None else iters, S_post, post_seed, top_m)
        self._meta[rid] = (inst.K, top_m)
        return rid

    def poll(self, rid, timeout_ms=0):
        K, top_m = self._meta[rid]
        r = xrdvi.xrdvi_server_poll(self.h, rid, timeout_ms, K, top_m)
        if r is not None:
            del self._meta[rid]
        return r

    def wait(self, rid, timeout_s=3600.0):
        t_end = time.monotonic() + timeout_s
        while True:
            r = self.poll(rid, 200)
            if r is not None:
                return r
            if time.monotonic() > t_end:
                raise TimeoutError(f"request {rid} not done after {timeout_s} s")

    def cancel(self, rid):
        xrdvi.xrdvi_server_cancel(self.h, rid)

    def stats(self):
        st = xrdvi.xrdvi_server_get_stats(self.h)
        return {f: getattr(st, f) for f, _ in st._fields_}

    def close(self):
        if self.h:
            xrdvi.xrdvi_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def enumerate_combinations(inst, *, iters=None, hbm_budget=16 << 30, **cfg):
    """Exact posterior over the 2^K - 1 non-empty phase combinations of a
    small-K problem (K <= 16): every sub-model fitted by the same SVI in
    sub-model batches on the GPU, scored by its tail-mean ELBO, normalised by
    an FP64 log-sum-exp on the GPU.  Returns (masks, elbo_c, p_c)."""
    cfg.setdefault("S", inst.S)
    c = xrdvi.xrdvi_config_default(**cfg)
    masks, elbo, logp = xrdvi.xrdvi_enumerate(inst.offsets, inst.pos, inst.inten, inst.x, inst.y, inst.bg, c,
                                              inst.iters if iters is None else iters, hbm_budget)
    return masks, elbo, np.exp(logp)


def replay_arrivals(server: Server, requests, arrivals_s, jsonl=None, **submit_kw):
    """Submit requests[i] at arrivals_s[i] seconds after the start, then wait
    for all.  Returns per-request dicts with 'latency' = done - submit and
    'queue_wait' = admit - submit.  jsonl (a path, optional): one JSON record
    per request (id, K, N, peaks, footprint, submit/admit/done times, latency,
    queue wait, status, final ELBO), in submission order."""
    import json
    t0 = time.monotonic()
    ids = []
    for inst, ta in zip(requests, arrivals_s):
        delay = ta - (time.monotonic() - t0)
        if delay > 0:
            time.sleep(delay)
        ids.append(server.submit(inst, **submit_kw))
    out = []
    for rid in ids:
        r = server.wait(rid)
        r["latency"] = r["t_done"] - r["t_submit"]
        r["queue_wait"] = r["t_admit"] - r["t_submit"]
        out.append(r)
    if jsonl:
        with open(jsonl, "w") as fh:
            for rid, inst, r in zip(ids, requests, out):
                fh.write(json.dumps({
                    "id": int(rid), "K": int(inst.K), "N": int(inst.N), "peaks": int(inst.offsets[-1]),
                    "footprint_bytes": int(r["footprint_bytes"]), "t_submit": r["t_submit"],
                    "t_admit": r["t_admit"], "t_done": r["t_done"], "latency_s": r["latency"],
                    "queue_wait_s": r["queue_wait"], "status": int(r["status"]),
                    "final_elbo": float(r["final_elbo"])}) + "\n")
    return out


def summarize(results, evals_per_fit):
    lat = np.array([r["latency"] for r in results])
    t_first = min(r["t_submit"] for r in results)
    t_last = max(r["t_done"] for r in results)
    span = t_last - t_first
    return {"requests": len(results), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
            "fits_per_s": len(results) / span, "makespan_s": span,
            "evals_per_s": float(np.sum(evals_per_fit)) / span}
