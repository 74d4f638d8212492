"""Thin ctypes binding of the xrdvi C ABI (``include/xrdvi.h``).

Argument marshalling only: every step of the fit, the profile and the
posterior runs in the CUDA library.  Functions carry the C names; ``Context``
is a small owner object around the opaque handle.  If the library is missing
and cannot be built, importing anything that needs it raises: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENONFINITE", 6: "EBUSY",
          7: "ECANCELED"}
FLAG_BF16_INT = 1 << 0
FLAG_NAIVE_SUM = 1 << 1
FLAG_GAUSS_LIK = 1 << 2   # Gaussian likelihood, variance max(y, 1)
FLAG_IW_ELBO = 1 << 3     # importance-weighted objective
FLAG_SHARED_SHAPES = 1 << 4   # one shape draw per step, tensor-core contractions
FLAG_SEC_WIDTH = 1 << 5       # side widths times sec(2theta / 2)
FLAG_FIT_BACKGROUND = 1 << 6  # background correction exp(sum beta_j T_j(z)) fitted in-model
FLAG_FIX_R = 1 << 7           # r held at fix_r_value
FLAG_FIX_ALPHA = 1 << 8       # alpha held at fix_alpha_value
FLAG_DEVICE_PTRS = 1 << 9     # xrdvi_create reads device arrays
FLAG_AREA_NORM = 1 << 10      # area-normalised profiles (h = integrated intensity)
FLAG_GATES = 1 << 11          # binary-Concrete phase gates
FLAG_DENSE = 1 << 12          # every peak evaluated directly (no far-field interpolation)


class XrdviError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"xrdvi {STATUS.get(status, status)}: {msg}")
        self.status = status


class Peaks(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("offsets", ctypes.POINTER(ctypes.c_int32)),
                ("pos_deg", ctypes.POINTER(ctypes.c_float)), ("rel_int", ctypes.POINTER(ctypes.c_float))]


class Pattern(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("x_deg", ctypes.POINTER(ctypes.c_float)),
                ("y_counts", ctypes.POINTER(ctypes.c_float)), ("bg", ctypes.POINTER(ctypes.c_float))]


class Config(ctypes.Structure):
    _fields_ = [("size", ctypes.c_uint32), ("S", ctypes.c_int32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("adam_eps", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("prior_mu_sd", ctypes.c_float),
                ("prior_alpha_mean", ctypes.c_float), ("prior_alpha_sd", ctypes.c_float),
                ("prior_w_shape", ctypes.c_float), ("prior_w_rate", ctypes.c_float),
                ("alpha_min", ctypes.c_float), ("init_h_frac", ctypes.c_float),
                ("init_sigma", ctypes.c_float), ("flags", ctypes.c_uint32), ("bg_prior_sd", ctypes.c_float),
                ("fix_r_value", ctypes.c_float), ("fix_alpha_value", ctypes.c_float),
                ("gate_tau", ctypes.c_float), ("gate_prior", ctypes.c_float)]


class Info(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("N", ctypes.c_int32), ("S", ctypes.c_int32),
                ("M_total", ctypes.c_int32), ("step", ctypes.c_int64), ("eta", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("data_const", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("point_tiles", ctypes.c_int32)]


class RequestOpts(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("S_post", ctypes.c_int32), ("post_seed", ctypes.c_uint64),
                ("top_m", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("K", ctypes.c_int32), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double), ("final_elbo", ctypes.c_double),
                ("log_evidence", ctypes.c_double), ("ess", ctypes.c_double), ("coverage_log", ctypes.c_double),
                ("elbo_tail_mean", ctypes.c_double),
                ("footprint_bytes", ctypes.c_size_t), ("pi", ctypes.POINTER(ctypes.c_double)),
                ("combos", ctypes.POINTER(ctypes.c_uint64)), ("combo_logp", ctypes.POINTER(ctypes.c_double)),
                ("loc", ctypes.POINTER(ctypes.c_float)), ("raw", ctypes.POINTER(ctypes.c_float))]


class ServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("running", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t), ("budget", ctypes.c_size_t),
                ("slots", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None

P = ctypes.POINTER
_f, _d, _i32, _u64 = ctypes.c_float, ctypes.c_double, ctypes.c_int32, ctypes.c_uint64
_vp = ctypes.c_void_p

# name -> (restype, argtypes); every function declared in include/xrdvi.h
SIGNATURES = {
    "xrdvi_config_default": (None, [P(Config)]),
    "xrdvi_create": (ctypes.c_int, [P(Peaks), P(Pattern), P(Config), P(_vp)]),
    "xrdvi_destroy": (None, [_vp]),
    "xrdvi_set_stream": (ctypes.c_int, [_vp, _vp]),
    "xrdvi_fit": (ctypes.c_int, [_vp, _i32, P(_d)]),
    "xrdvi_fit_batch": (ctypes.c_int, [P(_vp), _i32, _i32, P(_d)]),
    "xrdvi_elbo_grad": (ctypes.c_int, [_vp, P(_f), P(_d), P(_f), P(_f), P(_d), P(_d)]),
    "xrdvi_posterior": (ctypes.c_int, [_vp, _i32, _u64, _i32, P(_d), P(_u64), P(_d), P(_d), P(_d), P(_d)]),
    "xrdvi_get_params": (ctypes.c_int, [_vp, P(_f), P(_f)]),
    "xrdvi_set_params": (ctypes.c_int, [_vp, P(_f), P(_f)]),
    "xrdvi_get_state": (ctypes.c_int, [_vp, _vp, P(ctypes.c_size_t)]),
    "xrdvi_set_state": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "xrdvi_get_info": (ctypes.c_int, [_vp, P(Info)]),
    "xrdvi_forward_dev": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "xrdvi_backward_dev": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "xrdvi_profile_steps": (ctypes.c_int, [_vp, _i32, P(_f)]),
    "xrdvi_profile_kernels": (ctypes.c_int, [_vp, _i32, P(_f), P(ctypes.c_int64)]),
    "xrdvi_elbo_grad_static": (ctypes.c_int, [_i32, _i32, _vp, _vp, _vp, _i32, _vp, _vp, _vp, _d, _d,
                                              P(Config), _vp, _vp, _vp, _vp, _vp, _vp]),
    "xrdvi_footprint_bytes": (ctypes.c_size_t, [_i32, _i32, _i32, _i32, _i32, _i32]),
    "xrdvi_server_create": (ctypes.c_int, [ctypes.c_size_t, _i32, P(_vp)]),
    "xrdvi_server_submit": (ctypes.c_int, [_vp, P(Peaks), P(Pattern), P(Config), P(RequestOpts), P(_u64)]),
    "xrdvi_server_poll": (ctypes.c_int, [_vp, _u64, _i32, P(Result)]),
    "xrdvi_server_cancel": (ctypes.c_int, [_vp, _u64]),
    "xrdvi_server_get_stats": (ctypes.c_int, [_vp, P(ServerStats)]),
    "xrdvi_server_destroy": (None, [_vp]),
    "xrdvi_enumerate": (ctypes.c_int, [P(Peaks), P(Pattern), P(Config), _i32, ctypes.c_size_t, P(_d), P(_d)]),
    "xrdvi_enumerate_footprint_bytes": (ctypes.c_size_t, [_i32, _i32, _i32, _i32, _i32]),
    "xrdvi_gemm_nt_tf32x3": (ctypes.c_int, [_i32, _i32, _i32, _vp, _i32, _vp, _i32, _vp, _i32, _vp]),
    "xrdvi_get_background": (ctypes.c_int, [_vp, P(_f), P(_f), P(_f)]),
    "xrdvi_get_gates": (ctypes.c_int, [_vp, P(_f), P(_f)]),
    "xrdvi_philox4x32_10": (ctypes.c_int, [_i32, P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]),
    "xrdvi_debug_word": (ctypes.c_int, [P(_i32), _i32]),
    "xrdvi_debug_selftest": (ctypes.c_int, []),
    "xrdvi_last_error": (ctypes.c_char_p, []),
    "xrdvi_version": (ctypes.c_char_p, []),
}


def lib():
    """Load (building first if needed) the CUDA library."""
    global _lib
    with _lock:
        if _lib is None:
            # XRDVI_DEBUG=1: the bounds-check build (kernels clamp and record out-of-range indices)
            path = _build.build(debug=os.environ.get("XRDVI_DEBUG") == "1")
            if not os.path.exists(path):
                raise RuntimeError("xrdvi CUDA library is missing and could not be built")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status):
    if status != 0:
        msg = lib().xrdvi_last_error().decode(errors="replace")
        raise XrdviError(status, msg)


def _ptr(a, ct):
    return a.ctypes.data_as(P(ct))


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def xrdvi_config_default(**overrides) -> Config:
    cfg = Config()
    lib().xrdvi_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def xrdvi_create(offsets, pos, inten, x, y, bg, cfg: Config):
    offsets = np.ascontiguousarray(offsets, dtype=np.int32)
    pos, inten, x, y, bg = map(_f32, (pos, inten, x, y, bg))
    pk = Peaks(len(offsets) - 1, _ptr(offsets, ctypes.c_int32), _ptr(pos, _f), _ptr(inten, _f))
    pt = Pattern(len(x), _ptr(x, _f), _ptr(y, _f), _ptr(bg, _f))
    h = _vp()
    _check(lib().xrdvi_create(ctypes.byref(pk), ctypes.byref(pt), ctypes.byref(cfg), ctypes.byref(h)))
    return h


def xrdvi_create_device(K, N, d_offsets, d_pos, d_inten, d_x, d_y, d_bg, cfg: Config):
    """xrdvi_create from DEVICE arrays (integer addresses, e.g. tensor.data_ptr());
    sets XRDVI_FLAG_DEVICE_PTRS."""
    cfg.flags |= FLAG_DEVICE_PTRS
    pk = Peaks(int(K), ctypes.cast(_vp(d_offsets), ctypes.POINTER(ctypes.c_int32)),
               ctypes.cast(_vp(d_pos), ctypes.POINTER(_f)), ctypes.cast(_vp(d_inten), ctypes.POINTER(_f)))
    pt = Pattern(int(N), ctypes.cast(_vp(d_x), ctypes.POINTER(_f)), ctypes.cast(_vp(d_y), ctypes.POINTER(_f)),
                 ctypes.cast(_vp(d_bg), ctypes.POINTER(_f)))
    h = _vp()
    _check(lib().xrdvi_create(ctypes.byref(pk), ctypes.byref(pt), ctypes.byref(cfg), ctypes.byref(h)))
    return h


def xrdvi_destroy(h):
    if h:
        lib().xrdvi_destroy(h)


CUDA_STREAM_LEGACY = 0x1


def xrdvi_set_stream(h, stream_handle):
    """stream_handle: a cudaStream_t as an int.  0 (the legacy default
    stream, e.g. torch's default stream) maps to cudaStreamLegacy; None selects
    the context's own stream."""
    if stream_handle is None:
        _check(lib().xrdvi_set_stream(h, None))
    else:
        _check(lib().xrdvi_set_stream(h, _vp(stream_handle or CUDA_STREAM_LEGACY)))


def xrdvi_fit(h, iters, trace=True):
    tr = np.zeros(max(iters, 1), dtype=np.float64) if trace else None
    _check(lib().xrdvi_fit(h, int(iters), _ptr(tr, _d) if trace else None))
    return tr[:iters] if trace else None


def xrdvi_fit_batch(handles, iters):
    """Advances several contexts together (shared kernel launches per step);
    returns each fit's last ELBO estimate."""
    arr = (_vp * len(handles))(*[h.value if isinstance(h, _vp) else h for h in handles])
    last = np.zeros(len(handles))
    _check(lib().xrdvi_fit_batch(arr, len(handles), int(iters), _ptr(last, _d)))
    return last


def xrdvi_get_info(h) -> Info:
    info = Info()
    _check(lib().xrdvi_get_info(h, ctypes.byref(info)))
    return info


def xrdvi_elbo_grad(h, eps=None, want_f=False, want_grad=True, gate_noise=None):
    """One step without an update.  eps [S, K, 5] injected normals (None: the
    step's own draws); with the gate variant gate_noise [S, K] holds the
    logistic gate noise and is passed after eps."""
    info = xrdvi_get_info(h)
    S, K, N = info.S, info.K, info.N
    e = None if eps is None else _f32(eps).reshape(S * K * 5)
    if e is not None and gate_noise is not None:
        e = np.ascontiguousarray(np.concatenate([e, _f32(gate_noise).reshape(S * K)]))
    elbo = ctypes.c_double(0.0)
    grad = np.zeros((K, 10), dtype=np.float32)
    f = np.zeros((S, N), dtype=np.float32) if want_f else None
    ll = np.zeros(S)
    lpj = np.zeros(S)
    _check(lib().xrdvi_elbo_grad(h, _ptr(e, _f) if e is not None else None, ctypes.byref(elbo),
                                 _ptr(grad, _f) if want_grad else None,
                                 _ptr(f, _f) if want_f else None, _ptr(ll, _d), _ptr(lpj, _d)))
    out = {"elbo": elbo.value, "grad": grad, "ll": ll, "lpj": lpj}
    if want_f:
        out["f"] = f
    return out


def xrdvi_posterior(h, S_post, seed, top_m=8):
    info = xrdvi_get_info(h)
    K = info.K
    W = (K + 63) // 64
    pi = np.zeros(K)
    combos = np.zeros((top_m, W), dtype=np.uint64)
    clp = np.zeros(top_m)
    le, ess, cov = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().xrdvi_posterior(h, int(S_post), int(seed), int(top_m), _ptr(pi, _d),
                                 _ptr(combos, ctypes.c_uint64), _ptr(clp, _d), ctypes.byref(le),
                                 ctypes.byref(ess), ctypes.byref(cov)))
    bits = np.zeros((top_m, K), dtype=bool)
    for k in range(K):
        bits[:, k] = (combos[:, k // 64] >> np.uint64(k % 64)) & np.uint64(1)
    return {"pi": pi, "combos": bits, "combo_words": combos, "combo_logp": clp,
            "log_evidence": le.value, "ess": ess.value, "coverage_log": cov.value}


def xrdvi_get_params(h):
    K = xrdvi_get_info(h).K
    loc = np.zeros((K, 5), dtype=np.float32)
    raw = np.zeros((K, 5), dtype=np.float32)
    _check(lib().xrdvi_get_params(h, _ptr(loc, _f), _ptr(raw, _f)))
    return loc, raw


def xrdvi_set_params(h, loc, raw):
    loc, raw = _f32(loc), _f32(raw)
    _check(lib().xrdvi_set_params(h, _ptr(loc, _f), _ptr(raw, _f)))


def xrdvi_get_state(h) -> bytes:
    n = ctypes.c_size_t(0)
    _check(lib().xrdvi_get_state(h, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().xrdvi_get_state(h, buf, ctypes.byref(n)))
    return buf.raw[: n.value]


def xrdvi_set_state(h, state: bytes):
    buf = ctypes.create_string_buffer(state, len(state))
    _check(lib().xrdvi_set_state(h, buf, len(state)))


def xrdvi_forward_dev(h, loc_ptr, raw_ptr, eps_ptr, elbo_ptr):
    _check(lib().xrdvi_forward_dev(h, _vp(loc_ptr), _vp(raw_ptr), _vp(eps_ptr), _vp(elbo_ptr)))


def xrdvi_backward_dev(h, loc_ptr, raw_ptr, eps_ptr, grad_ptr):
    _check(lib().xrdvi_backward_dev(h, _vp(loc_ptr), _vp(raw_ptr), _vp(eps_ptr), _vp(grad_ptr)))


def xrdvi_elbo_grad_static(K, M_total, offsets_ptr, pos_ptr, inten_ptr, N, x_ptr, y_ptr, bg_ptr,
                           data_const, lambda_, cfg: Config, loc_ptr, raw_ptr, eps_ptr, elbo_ptr,
                           grad_ptr, stream_handle=0):
    """Allocation-free ELBO + gradient: every pointer is a device address
    (int) owned by the caller; scratch comes from the library's static array.
    Asynchronous on stream_handle (0: the legacy default stream)."""
    _check(lib().xrdvi_elbo_grad_static(int(K), int(M_total), _vp(offsets_ptr), _vp(pos_ptr),
                                        _vp(inten_ptr), int(N), _vp(x_ptr), _vp(y_ptr), _vp(bg_ptr),
                                        float(data_const), float(lambda_), ctypes.byref(cfg),
                                        _vp(loc_ptr), _vp(raw_ptr), _vp(eps_ptr), _vp(elbo_ptr),
                                        _vp(grad_ptr), _vp(stream_handle) if stream_handle else None))


KERNELS = ("sample", "forward", "backward", "grad_adam", "elbo")


def xrdvi_profile_steps(h, steps):
    ms = np.zeros(5, dtype=np.float32)
    _check(lib().xrdvi_profile_steps(h, int(steps), _ptr(ms, _f)))
    return dict(zip(KERNELS, ms.astype(float)))


def xrdvi_philox4x32_10(ctr, key):
    """Philox4x32-10 blocks computed on the GPU: ctr [n, 4], key [n, 2] (uint32)
    -> [n, 4] uint32."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(-1, 2))
    if len(c) != len(k):
        raise ValueError("one key per counter")
    out = np.zeros_like(c)
    u32 = ctypes.c_uint32
    _check(lib().xrdvi_philox4x32_10(len(c), _ptr(c, u32), _ptr(k, u32), _ptr(out, u32)))
    return out


def xrdvi_debug_word(reset=False):
    """First violated bounds check of the XRDVI_DEBUG build (0: none)."""
    w = ctypes.c_int32(0)
    _check(lib().xrdvi_debug_word(ctypes.byref(w), 1 if reset else 0))
    return int(w.value)


def xrdvi_debug_selftest():
    _check(lib().xrdvi_debug_selftest())


def xrdvi_version() -> str:
    return lib().xrdvi_version().decode()


class Context:
    """Owner of one fit (a problem, its device state and its q)."""

    def __init__(self, offsets, pos, inten, x, y, bg, cfg: Config | None = None, **cfg_overrides):
        if cfg is None:
            cfg = xrdvi_config_default(**cfg_overrides)
        self.cfg = cfg
        self.h = xrdvi_create(offsets, pos, inten, x, y, bg, cfg)

    @classmethod
    def from_instance(cls, inst, **cfg_overrides):
        cfg_overrides.setdefault("S", inst.S)
        return cls(inst.offsets, inst.pos, inst.inten, inst.x, inst.y, inst.bg, **cfg_overrides)

    @classmethod
    def from_device(cls, K, N, d_offsets, d_pos, d_inten, d_x, d_y, d_bg, **cfg_overrides):
        """Context from DEVICE arrays (integer addresses)."""
        self = cls.__new__(cls)
        self.cfg = xrdvi_config_default(**cfg_overrides)
        self.h = xrdvi_create_device(K, N, d_offsets, d_pos, d_inten, d_x, d_y, d_bg, self.cfg)
        return self

    def close(self):
        if getattr(self, "h", None):
            xrdvi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def info(self) -> Info:
        return xrdvi_get_info(self.h)

    def fit(self, iters, trace=True):
        return xrdvi_fit(self.h, iters, trace)

    def elbo_grad(self, eps=None, want_f=False, gate_noise=None):
        return xrdvi_elbo_grad(self.h, eps, want_f, gate_noise=gate_noise)

    def posterior(self, S_post, seed, top_m=8):
        return xrdvi_posterior(self.h, S_post, seed, top_m)

    def params(self):
        return xrdvi_get_params(self.h)

    def set_params(self, loc, raw):
        xrdvi_set_params(self.h, loc, raw)

    def state(self) -> bytes:
        return xrdvi_get_state(self.h)

    def set_state(self, s: bytes):
        xrdvi_set_state(self.h, s)

    def profile_steps(self, steps):
        return xrdvi_profile_steps(self.h, steps)

    def profile_kernels(self, steps):
        return xrdvi_profile_kernels(self.h, steps)

    def background(self):
        return xrdvi_get_background(self.h)

    def gates(self):
        return xrdvi_get_gates(self.h)

    def set_stream(self, stream_handle):
        xrdvi_set_stream(self.h, stream_handle)


# ---------------------------------------------------------------------------
# Serving
# ---------------------------------------------------------------------------
def xrdvi_footprint_bytes(K, N, M_total, S, S_post, top_m):
    return int(lib().xrdvi_footprint_bytes(int(K), int(N), int(M_total), int(S), int(S_post), int(top_m)))


def xrdvi_server_create(hbm_budget, max_slots):
    h = _vp()
    _check(lib().xrdvi_server_create(int(hbm_budget), int(max_slots), ctypes.byref(h)))
    return h


def xrdvi_server_submit(srv, offsets, pos, inten, x, y, bg, cfg: Config, iters, S_post=4096, post_seed=1,
                        top_m=8):
    offsets = np.ascontiguousarray(offsets, dtype=np.int32)
    pos, inten, x, y, bg = map(_f32, (pos, inten, x, y, bg))
    pk = Peaks(len(offsets) - 1, _ptr(offsets, ctypes.c_int32), _ptr(pos, _f), _ptr(inten, _f))
    pt = Pattern(len(x), _ptr(x, _f), _ptr(y, _f), _ptr(bg, _f))
    opts = RequestOpts(int(iters), int(S_post), int(post_seed), int(top_m))
    rid = ctypes.c_uint64(0)
    _check(lib().xrdvi_server_submit(srv, ctypes.byref(pk), ctypes.byref(pt), ctypes.byref(cfg),
                                     ctypes.byref(opts), ctypes.byref(rid)))
    return int(rid.value)


def xrdvi_server_poll(srv, req_id, timeout_ms, K, top_m):
    """Returns a dict, or None while the request is still queued / running."""
    W = (K + 63) // 64
    pi = np.zeros(K)
    combos = np.zeros((top_m, W), dtype=np.uint64)
    clp = np.zeros(top_m)
    loc = np.zeros((K, 5), dtype=np.float32)
    raw = np.zeros((K, 5), dtype=np.float32)
    res = Result()
    res.pi, res.combos, res.combo_logp = _ptr(pi, _d), _ptr(combos, ctypes.c_uint64), _ptr(clp, _d)
    res.loc, res.raw = _ptr(loc, _f), _ptr(raw, _f)
    st = lib().xrdvi_server_poll(srv, int(req_id), int(timeout_ms), ctypes.byref(res))
    if st == 4:
        return None
    _check(st)
    bits = np.zeros((top_m, K), dtype=bool)
    for k in range(K):
        bits[:, k] = (combos[:, k // 64] >> np.uint64(k % 64)) & np.uint64(1)
    return {"status": res.status, "t_submit": res.t_submit, "t_admit": res.t_admit, "t_done": res.t_done,
            "final_elbo": res.final_elbo, "log_evidence": res.log_evidence, "ess": res.ess,
            "coverage_log": res.coverage_log, "elbo_tail_mean": res.elbo_tail_mean,
            "footprint_bytes": res.footprint_bytes, "pi": pi,
            "combos": bits, "combo_logp": clp, "loc": loc, "raw": raw}


def xrdvi_server_cancel(srv, req_id):
    _check(lib().xrdvi_server_cancel(srv, int(req_id)))


def xrdvi_server_get_stats(srv) -> ServerStats:
    st = ServerStats()
    _check(lib().xrdvi_server_get_stats(srv, ctypes.byref(st)))
    return st


def xrdvi_server_destroy(srv):
    if srv:
        lib().xrdvi_server_destroy(srv)


def xrdvi_enumerate_footprint_bytes(K, N, M_total, S, nsub):
    return int(lib().xrdvi_enumerate_footprint_bytes(int(K), int(N), int(M_total), int(S), int(nsub)))


def xrdvi_enumerate(offsets, pos, inten, x, y, bg, cfg: Config, iters, hbm_budget):
    """Fits all 2^K - 1 non-empty sub-models in sub-model batches; returns
    (masks [2^K - 1, K] bool, elbo_c, logp_c), row c - 1 = combination c."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int32)
    pos, inten, x, y, bg = map(_f32, (pos, inten, x, y, bg))
    K = len(offsets) - 1
    n = max((1 << K) - 1, 0) if 0 < K <= 16 else 0
    pk = Peaks(K, _ptr(offsets, ctypes.c_int32), _ptr(pos, _f), _ptr(inten, _f))
    pt = Pattern(len(x), _ptr(x, _f), _ptr(y, _f), _ptr(bg, _f))
    elbo = np.zeros(max(n, 1))
    logp = np.zeros(max(n, 1))
    _check(lib().xrdvi_enumerate(ctypes.byref(pk), ctypes.byref(pt), ctypes.byref(cfg), int(iters),
                                 int(hbm_budget), _ptr(elbo, _d), _ptr(logp, _d)))
    codes = np.arange(1, n + 1)
    masks = ((codes[:, None] >> np.arange(K)[None, :]) & 1).astype(bool)
    return masks, elbo[:n], logp[:n]


def xrdvi_gemm_nt_tf32x3(M, N, K, d_A, lda, d_B, ldb, d_C, ldc, stream=None):
    """Device-pointer GEMM C = A . B^T on the tensor cores (3xTF32)."""
    _check(lib().xrdvi_gemm_nt_tf32x3(int(M), int(N), int(K), _vp(d_A), int(lda), _vp(d_B), int(ldb), _vp(d_C),
                                      int(ldc), _vp(stream or CUDA_STREAM_LEGACY)))


def xrdvi_get_background(h):
    """Fitted-background variant: {"beta": [3], "curve": [N], "grad_beta": [3]}."""
    info = xrdvi_get_info(h)
    beta = np.zeros(3, dtype=np.float32)
    curve = np.zeros(info.N, dtype=np.float32)
    gb = np.zeros(3, dtype=np.float32)
    _check(lib().xrdvi_get_background(h, _ptr(beta, _f), _ptr(curve, _f), _ptr(gb, _f)))
    return {"beta": beta, "curve": curve, "grad_beta": gb}


def xrdvi_get_gates(h):
    """Gate variant: {"logits": [K], "grad": [K]}."""
    K = xrdvi_get_info(h).K
    a = np.zeros(K, dtype=np.float32)
    g = np.zeros(K, dtype=np.float32)
    _check(lib().xrdvi_get_gates(h, _ptr(a, _f), _ptr(g, _f)))
    return {"logits": a, "grad": g}


PROFILE_KERNELS = ("sample", "ranges", "direct", "far_fwd", "lik", "bwd_uniform", "bwd_near", "far_bwd",
                   "grad_adam", "elbo")
WORK_COUNTS = ("uniform", "mixed", "gauss_reach", "far_nodes", "mixed_gauss_bwd", "gauss_reach_bwd")


def xrdvi_profile_kernels(h, steps):
    """Per-kernel mean ms per step over `steps` fit steps, and the last step's
    evaluation counts: ({name: ms}, {name: count})."""
    ms = np.zeros(len(PROFILE_KERNELS), dtype=np.float32)
    work = np.zeros(len(WORK_COUNTS), dtype=np.int64)
    _check(lib().xrdvi_profile_kernels(h, steps, _ptr(ms, _f), _ptr(work, ctypes.c_int64)))
    return ({k: float(v) for k, v in zip(PROFILE_KERNELS, ms)}, {k: int(v) for k, v in zip(WORK_COUNTS, work)})
