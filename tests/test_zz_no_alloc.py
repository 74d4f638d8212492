"""The allocation-free ELBO + gradient entry point (xrdvi_elbo_grad_static).

It serves callers that may not allocate device memory themselves (their
memory belongs to a framework's allocator or to a fixed budget), so it takes
caller-owned device buffers and uses the library's static scratch array.
Here its results are checked against the regular entry point, which allocates
its own workspace, on two calls in a row with different inputs (the second
call runs on the scratch the first one left behind); against the FP64 oracle
on a table whose peaks are shuffled within each phase (the entry sorts them on
the device); with the bfloat16 intensity flag; and on inputs the device check
must reject.  This file is collected last so that a stop-at-first-failure run
has run every other test first.
"""
import numpy as np
import pytest

import oracle
from paper_2501_09308_gb300 import synth, xrdvi

pytestmark = pytest.mark.gpu

F_TOL = 1e-5   # relative, ELBO
G_TOL = 1e-4   # per-block max-norm relative, gradient


def _dev(a, dtype):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


class _Static:
    """Device copies of one problem and the output buffers of the entry."""

    def __init__(self, inst):
        import torch
        self.inst = inst
        self.off = _dev(inst.offsets, torch.int32)
        self.pos = _dev(inst.pos, torch.float32)
        self.inten = _dev(inst.inten, torch.float32)
        self.x = _dev(inst.x, torch.float32)
        self.y = _dev(inst.y, torch.float32)
        self.bg = _dev(inst.bg, torch.float32)
        self.elbo = torch.empty(1, dtype=torch.float64, device="cuda")
        self.grad = torch.empty(inst.K * 10, dtype=torch.float32, device="cuda")

    def call(self, cfg, info, loc, raw, eps):
        import torch
        d_loc, d_raw, d_eps = _dev(loc, torch.float32), _dev(raw, torch.float32), _dev(eps, torch.float32)
        self.elbo.fill_(float("nan"))
        self.grad.fill_(float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        xrdvi.xrdvi_elbo_grad_static(self.inst.K, int(self.inst.offsets[-1]), self.off.data_ptr(),
                                     self.pos.data_ptr(), self.inten.data_ptr(), self.inst.N,
                                     self.x.data_ptr(), self.y.data_ptr(), self.bg.data_ptr(),
                                     info.data_const, info.lambda_, cfg, d_loc.data_ptr(), d_raw.data_ptr(),
                                     d_eps.data_ptr(), self.elbo.data_ptr(), self.grad.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        return float(self.elbo.item()), self.grad.cpu().numpy().reshape(self.inst.K, 10), free0 - free1


def _assert_close(e, g, ref_elbo, ref_grad):
    assert abs(e - ref_elbo) <= F_TOL * abs(ref_elbo), (e, ref_elbo)
    for b in range(10):
        scale = np.max(np.abs(ref_grad[:, b]))
        assert np.max(np.abs(g[:, b] - ref_grad[:, b])) <= G_TOL * scale, b


def test_static_scratch_entry_matches_regular_entry_on_two_calls():
    inst = synth.small_problem(K=5, M=12, N=700, S=8, seed=61)
    ctx = xrdvi.Context.from_instance(inst, S=8)
    info, cfg = ctx.info, ctx.cfg
    rng = np.random.default_rng(61)
    loc0, raw0 = ctx.params()
    st = _Static(inst)
    for call in range(2):
        loc = (loc0 + rng.normal(0, 0.05, loc0.shape)).astype(np.float32)
        raw = (raw0 + rng.normal(0, 0.1, raw0.shape)).astype(np.float32)
        eps = synth.normals(100 + call, 8, inst.K)
        ctx.set_params(loc, raw)
        ref = ctx.elbo_grad(eps)
        e, g, used = st.call(cfg, info, loc, raw, eps)
        _assert_close(e, g, ref["elbo"], ref["grad"])
        if call == 1:
            # the property the entry exists for: no device memory is taken
            assert used <= 0, used
    ctx.close()


def test_static_entry_sorts_shuffled_peaks_and_matches_the_oracle():
    """Peaks in random order within each phase (the candidate set of App. A.1
    is an unordered list): the entry sorts them on the device, and its ELBO
    and gradient match the FP64 oracle, whose direct sums do not depend on
    the order."""
    base = synth.small_problem(K=6, M=14, N=900, S=8, seed=62)
    rng = np.random.default_rng(62)
    pos, inten = base.pos.copy(), base.inten.copy()
    for k in range(base.K):
        a, b = base.offsets[k], base.offsets[k + 1]
        perm = rng.permutation(b - a) + a
        pos[a:b], inten[a:b] = base.pos[perm], base.inten[perm]
    assert np.any(np.diff(pos) < 0)
    inst = synth.Instance(**{**base.__dict__, "pos": pos, "inten": inten})
    ctx = xrdvi.Context.from_instance(base, S=8)
    info, cfg = ctx.info, ctx.cfg
    loc, raw = ctx.params()
    ctx.close()
    loc = (loc + rng.normal(0, 0.05, loc.shape)).astype(np.float32)
    raw = (raw + rng.normal(0, 0.1, raw.shape)).astype(np.float32)
    eps = synth.normals(162, 8, inst.K)
    e, g, _ = _Static(inst).call(cfg, info, loc, raw, eps)
    o = oracle.Problem.from_instance(inst).elbo_grad(loc.astype(np.float64), raw.astype(np.float64),
                                                     eps.astype(np.float64))
    _assert_close(e, g, o["elbo"], o["grad"])


def test_static_entry_bf16_flag_matches_regular_entry():
    """With XRDVI_FLAG_BF16_INT the entry rounds the intensities on the
    device, as xrdvi_create does on the host: both entries agree."""
    inst = synth.small_problem(K=4, M=10, N=600, S=4, seed=63)
    ctx = xrdvi.Context.from_instance(inst, S=4, flags=xrdvi.FLAG_BF16_INT)
    loc, raw = ctx.params()
    eps = synth.normals(63, 4, inst.K)
    ref = ctx.elbo_grad(eps)
    e, g, _ = _Static(inst).call(ctx.cfg, ctx.info, loc, raw, eps)
    ctx.close()
    _assert_close(e, g, ref["elbo"], ref["grad"])


def test_static_entry_turns_invalid_device_input_into_nan():
    """The device check rejects what xrdvi_create rejects on the host (x not
    increasing, an empty phase); the call cannot return a status for it, so
    the ELBO and gradient come back NaN.  A valid call right after is exact
    again."""
    inst = synth.small_problem(K=3, M=6, N=400, S=4, seed=64)
    ctx = xrdvi.Context.from_instance(inst, S=4)
    loc, raw = ctx.params()
    eps = synth.normals(64, 4, inst.K)
    ref = ctx.elbo_grad(eps)
    info, cfg = ctx.info, ctx.cfg
    ctx.close()
    x = inst.x.copy()
    x[7] = x[6]
    bad_x = synth.Instance(**{**inst.__dict__, "x": x})
    off = inst.offsets.copy()
    off[1] = off[0]
    bad_off = synth.Instance(**{**inst.__dict__, "offsets": off})
    for bad in (bad_x, bad_off):
        e, g, _ = _Static(bad).call(cfg, info, loc, raw, eps)
        assert np.isnan(e) and np.all(np.isnan(g))
    e, g, _ = _Static(inst).call(cfg, info, loc, raw, eps)
    _assert_close(e, g, ref["elbo"], ref["grad"])


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
    cfg = xrdvi.xrdvi_config_default(S=8, flags=xrdvi.FLAG_GATES)
    with pytest.raises(xrdvi.XrdviError) as err:
        xrdvi.xrdvi_elbo_grad_static(inst.K, int(inst.offsets[-1]), z.data_ptr(), z.data_ptr(),
                                     z.data_ptr(), inst.N, z.data_ptr(), z.data_ptr(), z.data_ptr(),
                                     0.0, 1e-3, cfg, z.data_ptr(), z.data_ptr(), z.data_ptr(),
                                     z.data_ptr(), z.data_ptr(), 0)
    assert err.value.status == 1
