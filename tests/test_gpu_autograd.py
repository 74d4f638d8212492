"""torch.autograd.Function wrapper over the CUDA forward/backward kernels."""
import numpy as np
import pytest

import oracle
from paper_2501_09308_gb300 import synth

pytestmark = pytest.mark.gpu


def test_autograd_gradients_match_oracle():
    """Differentiation workload: K=6, N=600 sub-instance; gradients of every
    variational parameter against the oracle's analytic gradient (itself
    pinned to FP64 central differences)."""
    import torch
    from paper_2501_09308_gb300.autograd import PhaseSearch
    inst = synth.config(2)
    S = 8
    mod = PhaseSearch(inst, S=S)
    with torch.no_grad():
        g = torch.Generator(device="cpu").manual_seed(0)
        mod.loc.add_((0.05 * torch.randn(mod.loc.shape, generator=g)).cuda())
        mod.raw.add_((0.1 * torch.randn(mod.raw.shape, generator=g)).cuda())
    eps_np = synth.normals(31, S, inst.K)
    eps = torch.tensor(eps_np, device="cuda")
    loss = mod(eps)
    loss.backward()
    P = oracle.Problem.from_instance(inst)
    o = P.elbo_grad(mod.loc.detach().cpu().numpy().astype(np.float64),
                    mod.raw.detach().cpu().numpy().astype(np.float64), eps_np.astype(np.float64))
    assert abs(-loss.item() - o["elbo"]) <= 1e-5 * abs(o["elbo"])
    gl = -mod.loc.grad.cpu().numpy()
    gr = -mod.raw.grad.cpu().numpy()
    for j in range(5):
        for mine, ref in ((gl[:, j], o["grad"][:, j]), (gr[:, j], o["grad"][:, 5 + j])):
            assert np.max(np.abs(mine - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_autograd_directional_derivative():
    """Loss differences along a random direction against the backward's
    directional derivative (FP32 profile: a loose, second check)."""
    import torch
    from paper_2501_09308_gb300.autograd import NegELBO, PhaseSearch
    inst = synth.config(2)
    mod = PhaseSearch(inst, S=8)
    eps = torch.tensor(synth.normals(3, 8, inst.K), device="cuda")
    loss = mod(eps)
    loss.backward()
    g = torch.Generator(device="cpu").manual_seed(1)
    dl = torch.randn(mod.loc.shape, generator=g).cuda()
    dr = torch.randn(mod.raw.shape, generator=g).cuda()
    dd = float((mod.loc.grad * dl).sum() + (mod.raw.grad * dr).sum())
    h = 1e-3
    with torch.no_grad():
        lp = NegELBO.apply(mod.loc + h * dl, mod.raw + h * dr, eps, mod.ctx).item()
        lm = NegELBO.apply(mod.loc - h * dl, mod.raw - h * dr, eps, mod.ctx).item()
    fd = (lp - lm) / (2 * h)
    assert abs(fd - dd) <= 1e-2 * abs(dd)


def test_torch_adam_on_autograd_matches_fused_fit():
    """Three torch.optim.Adam steps on the autograd loss, fed the fit stream's
    noise, reproduce three fused SVI steps of xrdvi_fit."""
    import torch
    from paper_2501_09308_gb300 import xrdvi
    from paper_2501_09308_gb300.autograd import PhaseSearch
    inst = synth.small_problem(K=3, M=6, N=300, S=4, seed=14)
    mod = PhaseSearch(inst, S=4, seed=4242)
    opt = torch.optim.Adam([mod.loc, mod.raw], lr=0.01, betas=(0.9, 0.999), eps=1e-8)
    for t in range(3):
        eps = torch.tensor(oracle.normals(4242, 0, t, 4, inst.K).astype(np.float32), device="cuda")
        opt.zero_grad()
        mod(eps).backward()
        opt.step()
    fused = xrdvi.Context.from_instance(inst, S=4, seed=4242)
    fused.fit(3)
    loc, raw = fused.params()
    np.testing.assert_allclose(mod.loc.detach().cpu().numpy(), loc, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(mod.raw.detach().cpu().numpy(), raw, rtol=1e-5, atol=1e-5)


def test_nothing_of_size_S_K_N_is_kept():
    """Profiles are recomputed in backward: the context holds far less than
    one S*K*N float array at the K=50, N=4500, S=256 size (its largest buffers
    are the phase-chunk partials of the profile, C <= 8 arrays of S*N)."""
    from paper_2501_09308_gb300 import xrdvi
    inst = synth.config(1)
    c = xrdvi.Context.from_instance(inst, S=inst.S)
    info = c.info
    c.close()
    assert info.device_bytes < 0.3 * inst.S * inst.K * inst.N * 4


@pytest.mark.slow
def test_autograd_full_size_k50_against_the_oracle():
    """The differentiation workload at its full size (K=50, N=4500, S=256)
    through torch.autograd: the loss and the gradients of every variational
    parameter against the oracle's evaluation (OpenMP, a few seconds)."""
    import torch
    from paper_2501_09308_gb300.autograd import PhaseSearch
    inst = synth.config(1)
    S = inst.S
    mod = PhaseSearch(inst, S=S)
    with torch.no_grad():
        g = torch.Generator(device="cpu").manual_seed(7)
        mod.loc.add_((0.02 * torch.randn(mod.loc.shape, generator=g)).cuda())
        mod.raw.add_((0.05 * torch.randn(mod.raw.shape, generator=g)).cuda())
    eps_np = synth.normals(77, S, inst.K)
    loss = mod(torch.tensor(eps_np, device="cuda"))
    loss.backward()
    o = oracle.Problem.from_instance(inst).elbo_grad(mod.loc.detach().cpu().numpy().astype(np.float64),
                                                    mod.raw.detach().cpu().numpy().astype(np.float64),
                                                    eps_np.astype(np.float64))
    assert abs(-loss.item() - o["elbo"]) <= 1e-5 * abs(o["elbo"])
    gl = -mod.loc.grad.cpu().numpy()
    gr = -mod.raw.grad.cpu().numpy()
    for j in range(5):
        for mine, ref in ((gl[:, j], o["grad"][:, j]), (gr[:, j], o["grad"][:, 5 + j])):
            assert np.max(np.abs(mine - ref)) <= 1e-4 * np.max(np.abs(ref)), j
