"""The bounds-check build (XRDVI_DEBUG): its kernels clamp every peak-table
index and every decoded peak range into bounds and record the first violated
check in a device word, with no trap or early exit.  On a valid problem it
computes what the regular build computes and records nothing; a lookup past
the end of a one-entry table (the self-test, whose access the check keeps in
bounds) sets the word to that check's number.  The debug library is built on
first use (in a child process, which loads it through XRDVI_DEBUG=1)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2501_09308_gb300 import synth, xrdvi

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, {root!r})
import numpy as np
from paper_2501_09308_gb300 import synth, xrdvi
inst = synth.small_problem(K=5, M=12, N=1300, S=8, seed=41)
ctx = xrdvi.Context.from_instance(inst, S=8, seed=3)
g = ctx.elbo_grad(synth.normals(41, 8, inst.K), want_f=True)
tr = ctx.fit(25)
loc, raw = ctx.params()
ctx.close()
w0 = xrdvi.xrdvi_debug_word()
xrdvi.xrdvi_debug_selftest()
w1 = xrdvi.xrdvi_debug_word(reset=True)
w2 = xrdvi.xrdvi_debug_word()
print(json.dumps({{"elbo": g["elbo"], "grad": g["grad"].tolist(), "f": g["f"][:, ::97].tolist(),
                  "trace": tr.tolist(), "loc": loc.tolist(), "w": [w0, w1, w2]}}))
"""


def _regular():
    inst = synth.small_problem(K=5, M=12, N=1300, S=8, seed=41)
    ctx = xrdvi.Context.from_instance(inst, S=8, seed=3)
    g = ctx.elbo_grad(synth.normals(41, 8, inst.K), want_f=True)
    tr = ctx.fit(25)
    loc, _ = ctx.params()
    ctx.close()
    return g, tr, loc


def test_debug_build_matches_regular_build_and_reports_a_violation():
    env = dict(os.environ, XRDVI_DEBUG="1")
    out = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True,
                         text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["w"] == [0, 3, 0], d["w"]   # nothing on the valid problem; the self-test's table check (3)
    g, tr, loc = _regular()
    assert abs(d["elbo"] - g["elbo"]) <= 1e-9 * abs(g["elbo"])
    np.testing.assert_allclose(np.array(d["grad"]), g["grad"], rtol=1e-5, atol=1e-6 * np.abs(g["grad"]).max())
    np.testing.assert_allclose(np.array(d["f"]), g["f"][:, ::97], rtol=1e-6)
    np.testing.assert_allclose(np.array(d["trace"]), tr, rtol=1e-6)
    np.testing.assert_allclose(np.array(d["loc"]), loc, rtol=1e-4, atol=1e-5)


def test_regular_build_has_no_debug_word():
    with pytest.raises(xrdvi.XrdviError) as e:
        xrdvi.xrdvi_debug_word()
    assert e.value.status == 1
