"""C ABI: the library loads and exports every function include/xrdvi.h
declares, and host-side validation rejects malformed inputs before any device
work (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2501_09308_gb300 import synth, xrdvi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(xrdvi_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported_and_bound():
    L = xrdvi.lib()
    names = declared_functions()
    assert len(names) >= 15
    for n in sorted(names):
        assert hasattr(L, n), n
        assert n in xrdvi.SIGNATURES, n


def test_config_default_is_papers_priors():
    cfg = xrdvi.xrdvi_config_default()
    assert cfg.size == ctypes.sizeof(xrdvi.Config)
    assert cfg.prior_mu_sd == pytest.approx(0.03)
    assert cfg.prior_alpha_mean == 1.0
    assert cfg.prior_alpha_sd == pytest.approx(0.2)
    assert cfg.prior_w_shape == 3.0
    assert cfg.prior_w_rate == 100.0


def _base():
    inst = synth.small_problem(K=2, M=4, N=64)
    return dict(offsets=inst.offsets.copy(), pos=inst.pos.copy(), inten=inst.inten.copy(),
                x=inst.x.copy(), y=inst.y.copy(), bg=inst.bg.copy())


def _bad(mod, **cfg):
    a = _base()
    mod(a)
    with pytest.raises(xrdvi.XrdviError) as e:
        xrdvi.xrdvi_create(a["offsets"], a["pos"], a["inten"], a["x"], a["y"], a["bg"],
                           xrdvi.xrdvi_config_default(**cfg))
    return e.value


@pytest.mark.parametrize("name,mod", [
    ("x not increasing", lambda a: a["x"].__setitem__(5, a["x"][4])),
    ("negative count", lambda a: a["y"].__setitem__(3, -1.0)),
    ("non-integer count", lambda a: a["y"].__setitem__(3, 2.5)),
    ("nan count", lambda a: a["y"].__setitem__(3, np.nan)),
    ("negative background", lambda a: a["bg"].__setitem__(0, -0.1)),
    ("position out of range", lambda a: a["pos"].__setitem__(0, 190.0)),
    ("intensity above one", lambda a: a["inten"].__setitem__(0, 1.5)),
    ("empty phase", lambda a: a["offsets"].__setitem__(1, 0)),
    ("offsets not from zero", lambda a: a["offsets"].__setitem__(0, 1)),
    ("no signal above background", lambda a: a["bg"].__setitem__(slice(None), 1e6)),
])
def test_invalid_inputs_are_rejected(name, mod):
    err = _bad(mod)
    assert err.status == 1, (name, err)


def test_invalid_config_is_rejected():
    assert _bad(lambda a: None, S=0).status == 1
    assert _bad(lambda a: None, prior_w_rate=-1.0).status == 1
    assert _bad(lambda a: None, beta1=1.0).status == 1
    cfg = xrdvi.xrdvi_config_default()
    cfg.size = 3
    a = _base()
    with pytest.raises(xrdvi.XrdviError) as e:
        xrdvi.xrdvi_create(a["offsets"], a["pos"], a["inten"], a["x"], a["y"], a["bg"], cfg)
    assert e.value.status == 1


def test_footprint_bound_is_monotone_and_rejects_bad_sizes():
    f = xrdvi.xrdvi_footprint_bytes
    base = f(50, 4500, 2194, 256, 4096, 16)
    assert base > 0
    assert f(50, 9000, 2194, 256, 4096, 16) > base
    assert f(50, 4500, 4000, 256, 4096, 16) > base
    assert f(50, 4500, 2194, 512, 4096, 16) > base
    assert f(50, 4500, 2194, 256, 0, 16) < base
    assert f(0, 4500, 2194, 256, 4096, 16) == 0
    assert f(50, 0, 2194, 256, 4096, 16) == 0


def test_enumerate_rejects_bad_sizes_before_device_work():
    a = _base()
    cfg = xrdvi.xrdvi_config_default()
    with pytest.raises(xrdvi.XrdviError) as e:
        xrdvi.xrdvi_enumerate(a["offsets"], a["pos"], a["inten"], a["x"], a["y"], a["bg"], cfg, 0, 1 << 30)
    assert e.value.status == 1
    big = synth.small_problem(K=17, M=3, N=64)
    with pytest.raises(xrdvi.XrdviError) as e:
        xrdvi.xrdvi_enumerate(big.offsets, big.pos, big.inten, big.x, big.y, big.bg, cfg, 10, 1 << 30)
    assert e.value.status == 1
    a["y"][3] = -1.0
    with pytest.raises(xrdvi.XrdviError) as e:
        xrdvi.xrdvi_enumerate(a["offsets"], a["pos"], a["inten"], a["x"], a["y"], a["bg"], cfg, 10, 1 << 30)
    assert e.value.status == 1


def test_angle_dependent_width_needs_angles_below_174_degrees():
    a = _base()
    a["x"] = np.linspace(170.0, 178.0, len(a["x"])).astype(np.float32)
    a["pos"][:] = 175.0
    with pytest.raises(xrdvi.XrdviError) as e:
        xrdvi.xrdvi_create(a["offsets"], a["pos"], a["inten"], a["x"], a["y"], a["bg"],
                           xrdvi.xrdvi_config_default(flags=xrdvi.FLAG_SEC_WIDTH))
    assert e.value.status == 1


def header_macros():
    """Integer macros of include/*.h (literals, shifts and products only)."""
    out = {}
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            for name, body in re.findall(r"^#define\s+(XRDVI_\w+)\s+([^/\n]*)", text, flags=re.M):
                expr = re.sub(r"(\d+)[uUlL]+", r"\1", body.strip())
                if expr and re.fullmatch(r"[0-9()<* ]+", expr):
                    out[name] = eval(expr, {"__builtins__": {}})
    return out


def test_binding_constants_match_the_header():
    """Flags and the profiler's array sizes are the header's values: a
    mismatch would pass wrong options or under-sized buffers across the ABI."""
    m = header_macros()
    flags = {k[len("XRDVI_"):]: v for k, v in m.items() if k.startswith("XRDVI_FLAG_")}
    assert len(flags) >= 13
    for name, v in flags.items():
        assert getattr(xrdvi, name) == v, name
    assert m["XRDVI_PROFILE_KERNELS"] == len(xrdvi.PROFILE_KERNELS)
    assert m["XRDVI_PROFILE_WORK"] == len(xrdvi.WORK_COUNTS)
    assert m["XRDVI_STATIC_SCRATCH_BYTES"] == 32 << 20


def _static_formula(S, K, T, M):
    """Scratch bytes of xrdvi_elbo_grad_static as include/xrdvi.h states them
    (before the alignment of its 18 arrays)."""
    return 48 * S * K * T + 2056 * S * T + 104 * S * K + 16 * S + 1416 * K + 8 * M + 32


def test_static_entry_rejects_every_size_the_header_formula_puts_above_the_limit():
    """The allocation-free entry checks its scratch size on the host before it
    touches a device pointer: every problem whose stated need exceeds the
    32 MiB array is refused with EINVAL (so the formula never overstates what
    the code needs).  The pointers passed are never dereferenced."""
    limit = 32 << 20
    m = header_macros()
    assert m["XRDVI_STATIC_SCRATCH_BYTES"] == limit
    K, N, M = 5, 700, 60
    T = (N + 255) // 256
    S = 1
    while _static_formula(S, K, T, M) <= limit:
        S += 1
    dummy = 1 << 20   # a non-null address the call must not use
    for s_try in (S, S + 1, S + 7):
        assert _static_formula(s_try, K, T, M) > limit
        cfg = xrdvi.xrdvi_config_default(S=s_try)
        with pytest.raises(xrdvi.XrdviError) as e:
            xrdvi.xrdvi_elbo_grad_static(K, M, dummy, dummy, dummy, N, dummy, dummy, dummy, 0.0, 1e-3, cfg,
                                         dummy, dummy, dummy, dummy, dummy, 0)
        assert e.value.status == 1 and "scratch" in str(e.value), (s_try, e.value)


def test_one_past_each_size_limit_is_rejected():
    """K = 1025 phases, 24001 peaks and S = 65537 draws give EINVAL before any
    device work (the largest accepted sizes run in test_gpu_limits)."""
    base = synth.small_problem(K=3, M=5, N=300, S=2, seed=63)
    with pytest.raises(xrdvi.XrdviError) as e:
        xrdvi.Context.from_instance(base, S=65537)
    assert e.value.status == 1
    big = synth.make_problem(K=1000, m_lo=24, m_hi=24, x_lo=20.0, x_step=0.05, N=300, n_planted=2, S=2,
                             iters=1, seed=63)
    assert int(big.offsets[-1]) == 24000
    over = synth.Instance(**{**big.__dict__, "offsets": np.concatenate([big.offsets[:-1], [24001]]).astype(np.int32),
                             "pos": np.concatenate([big.pos, big.pos[-1:]]),
                             "inten": np.concatenate([big.inten, big.inten[-1:]])})
    with pytest.raises(xrdvi.XrdviError) as e:
        xrdvi.Context.from_instance(over, S=2)
    assert e.value.status == 1 and "24000" in str(e.value)
    n = 1025
    many = synth.Instance(**{**base.__dict__, "offsets": np.arange(n + 1, dtype=np.int32),
                             "pos": np.full(n, 30.0, np.float32), "inten": np.full(n, 0.5, np.float32)})
    with pytest.raises(xrdvi.XrdviError) as e:
        xrdvi.Context.from_instance(many, S=2)
    assert e.value.status == 1 and "1024" in str(e.value)
