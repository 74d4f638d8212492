"""The allocation-free ELBO + gradient entry point (xrdvi_elbo_grad_static).

It serves callers that may not allocate device memory themselves (their
memory belongs to a framework's allocator or to a fixed budget), so it takes
caller-owned device buffers and uses the library's static scratch array.
Here its results are checked against the regular entry point, which allocates
its own workspace, on two calls in a row with different inputs (the second
call runs on the scratch the first one left behind).  This file is collected
last so that a stop-at-first-failure run has run every other test first.
"""
import numpy as np
import pytest

from paper_2501_09308_gb300 import synth, xrdvi

pytestmark = pytest.mark.gpu

F_TOL = 1e-5   # relative, ELBO
G_TOL = 1e-4   # per-block max-norm relative, gradient


def _dev(a, dtype):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def test_static_scratch_entry_matches_regular_entry_on_two_calls():
    import torch
    inst = synth.small_problem(K=5, M=12, N=700, S=8, seed=61)
    ctx = xrdvi.Context.from_instance(inst, S=8)
    info = ctx.info
    cfg = ctx.cfg
    rng = np.random.default_rng(61)
    loc0, raw0 = ctx.params()
    d_off = _dev(inst.offsets, torch.int32)
    d_pos = _dev(inst.pos, torch.float32)
    d_int = _dev(inst.inten, torch.float32)
    d_x = _dev(inst.x, torch.float32)
    d_y = _dev(inst.y, torch.float32)
    d_bg = _dev(inst.bg, torch.float32)
    elbo = torch.empty(1, dtype=torch.float64, device="cuda")
    grad = torch.empty(inst.K * 10, dtype=torch.float32, device="cuda")
    for call in range(2):
        loc = (loc0 + rng.normal(0, 0.05, loc0.shape)).astype(np.float32)
        raw = (raw0 + rng.normal(0, 0.1, raw0.shape)).astype(np.float32)
        eps = synth.normals(100 + call, 8, inst.K)
        ctx.set_params(loc, raw)
        ref = ctx.elbo_grad(eps)
        d_loc, d_raw, d_eps = _dev(loc, torch.float32), _dev(raw, torch.float32), _dev(eps, torch.float32)
        elbo.fill_(float("nan"))
        grad.fill_(float("nan"))
        xrdvi.xrdvi_elbo_grad_static(inst.K, int(inst.offsets[-1]), d_off.data_ptr(), d_pos.data_ptr(),
                                     d_int.data_ptr(), inst.N, d_x.data_ptr(), d_y.data_ptr(),
                                     d_bg.data_ptr(), info.data_const, info.lambda_, cfg,
                                     d_loc.data_ptr(), d_raw.data_ptr(), d_eps.data_ptr(),
                                     elbo.data_ptr(), grad.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        e = float(elbo.item())
        g = grad.cpu().numpy().reshape(inst.K, 10)
        assert abs(e - ref["elbo"]) <= F_TOL * abs(ref["elbo"]), (call, e, ref["elbo"])
        for b in range(10):
            scale = np.max(np.abs(ref["grad"][:, b]))
            assert np.max(np.abs(g[:, b] - ref["grad"][:, b])) <= G_TOL * scale, (call, b)
    ctx.close()


def test_static_scratch_entry_rejects_problems_above_the_limit():
    import torch
    inst = synth.small_problem(K=5, M=12, N=700, S=8, seed=61)
    cfg = xrdvi.xrdvi_config_default(S=60000)   # needs far more than 32 MiB of scratch
    z = torch.zeros(8, device="cuda")
    with pytest.raises(xrdvi.XrdviError) as err:
        xrdvi.xrdvi_elbo_grad_static(inst.K, int(inst.offsets[-1]), z.data_ptr(), z.data_ptr(),
                                     z.data_ptr(), inst.N, z.data_ptr(), z.data_ptr(), z.data_ptr(),
                                     0.0, 1e-3, cfg, z.data_ptr(), z.data_ptr(), z.data_ptr(),
                                     z.data_ptr(), z.data_ptr(), 0)
    assert err.value.status == 1 and "scratch" in str(err.value)
