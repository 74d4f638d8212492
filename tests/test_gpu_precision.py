"""Precision variants on the K=200, N=9000 precision workload: FP32 peak table
with compensated sums (default), a bfloat16 intensity table, and naive FP32
sums, each measured against the FP64 oracle.  Run with -s to print the table.

Profile, likelihood and gradient use S=16 draws at the full K and N (the
oracle evaluates 2e9 profile terms in seconds); the marginal phase
probabilities come from a short S=1024 fit and compare the bf16 table with
the FP32 table on the same fitted q."""
import numpy as np
import pytest

import oracle
from paper_2501_09308_gb300 import synth, xrdvi

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _errors(g, o):
    rf = float(np.max(np.abs(g["f"] - o["f"]) / o["f"]))
    rll = float(np.max(np.abs(g["ll"] - o["ll"]) / np.abs(o["ll"])))
    re = abs(g["elbo"] - o["elbo"]) / abs(o["elbo"])
    rg = max(float(np.max(np.abs(g["grad"][:, b] - o["grad"][:, b])) / float(np.max(np.abs(o["grad"][:, b]))))
             for b in range(10))
    return {"f": rf, "ll": rll, "elbo": re, "grad": rg}


def test_precision_sweep_K200_N9000():
    import torch
    inst = synth.config(3)
    S = 16
    eps = synth.normals(3000, S, inst.K)
    base = xrdvi.Context.from_instance(inst, S=S)
    loc, raw = base.params()
    rng = np.random.default_rng(3)
    loc = loc + rng.normal(0, 0.03, loc.shape).astype(np.float32)
    raw = raw + rng.normal(0, 0.05, raw.shape).astype(np.float32)
    base.close()
    P = oracle.Problem.from_instance(inst)
    o = P.elbo_grad(loc.astype(np.float64), raw.astype(np.float64), eps.astype(np.float64), want_f=True)
    rounded = torch.tensor(inst.inten).to(torch.bfloat16).to(torch.float32).numpy()
    inst_r = synth.Instance(**{**inst.__dict__, "inten": rounded})
    o_r = oracle.Problem.from_instance(inst_r).elbo_grad(loc.astype(np.float64), raw.astype(np.float64),
                                                         eps.astype(np.float64), want_f=True)
    rows = {}
    for name, flags in (("fp32 table, compensated", 0), ("bf16 intensities, compensated", xrdvi.FLAG_BF16_INT),
                        ("fp32 table, naive sums", xrdvi.FLAG_NAIVE_SUM)):
        c = xrdvi.Context.from_instance(inst, S=S, flags=flags)
        c.set_params(loc, raw)
        g = c.elbo_grad(eps, want_f=True)
        c.close()
        rows[name] = (_errors(g, o), _errors(g, o_r) if flags == xrdvi.FLAG_BF16_INT else None)
    print("\nvariant                          | vs FP64 oracle (exact table): f, LL, ELBO, grad")
    for name, (e, er) in rows.items():
        line = f"{name:32s} | {e['f']:.2e} {e['ll']:.2e} {e['elbo']:.2e} {e['grad']:.2e}"
        if er:
            line += f" | vs bf16-rounded oracle: {er['f']:.2e} {er['ll']:.2e} {er['elbo']:.2e} {er['grad']:.2e}"
        print(line)
    e = rows["fp32 table, compensated"][0]
    assert e["f"] <= 1e-5 and e["ll"] <= 1e-5 and e["elbo"] <= 1e-5 and e["grad"] <= 1e-4
    er = rows["bf16 intensities, compensated"][1]
    assert er["f"] <= 1e-5 and er["ll"] <= 1e-5 and er["elbo"] <= 1e-5 and er["grad"] <= 1e-4
    eb = rows["bf16 intensities, compensated"][0]
    assert eb["f"] <= 4e-3          # bfloat16 keeps 8 significant bits of each intensity
    en = rows["fp32 table, naive sums"][0]
    assert en["elbo"] <= 1e-5 and en["grad"] <= 1e-4


def test_marginal_probabilities_fp32_vs_bf16_table():
    """Same fitted q (150 steps at S=1024, FP32 table), posterior drawn with
    the FP32 and with the bf16 intensity table: the marginal inclusion
    probabilities differ only where the area-ratio test sits on the edge."""
    inst = synth.config(3)
    c = xrdvi.Context.from_instance(inst, S=inst.S, seed=9)
    c.fit(150)
    loc, raw = c.params()
    p32 = c.posterior(1024, 3, top_m=4)
    c.close()
    c = xrdvi.Context.from_instance(inst, S=inst.S, seed=9, flags=xrdvi.FLAG_BF16_INT)
    c.set_params(loc, raw)
    p16 = c.posterior(1024, 3, top_m=4)
    c.close()
    d = float(np.max(np.abs(p32["pi"] - p16["pi"])))
    print(f"\nmax |pi_fp32 - pi_bf16| over K=200 phases (same q, 1024 draws): {d:.3e}; "
          f"log evidence {p32['log_evidence']:.6e} vs {p16['log_evidence']:.6e}")
    assert d <= 0.02
