"""FP64 CPU oracle for the Monte-Carlo ELBO step (arXiv 2501.09308).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_2501_09308_gb300``) and neither imports the other;
the only shared module is the seeded input generator
``paper_2501_09308_gb300.synth``, which holds no inference arithmetic.

``xrdvi_oracle.c`` holds the model, likelihood, priors, Monte-Carlo ELBO,
analytic gradient, Adam and the fit loop in plain double-precision loops;
``posterior.py`` holds the posterior over phase combinations.  Every function
cites the passage of the paper it follows.

Parity pins: see ``tests/test_oracle_*.py``.  Unpinned parts are listed in
``posterior.py``'s header ("parity unpinned").
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xrdvi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Prior hyper-parameters (Appendix B.2): mu ~ Norm(0, 0.03), alpha ~ Norm(1, 0.2),
# r ~ Uni(0, 1), w ~ Gam(3, 100) read with 100 as a rate (mean 0.03 deg).
PRIOR_MU_SD = 0.03
PRIOR_ALPHA_MEAN = 1.0
PRIOR_ALPHA_SD = 0.2
PRIOR_W_SHAPE = 3.0
PRIOR_W_RATE = 100.0
ALPHA_MIN = 1e-3


class Prior(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("mu_sd", ctypes.c_double),
                ("alpha_mean", ctypes.c_double), ("alpha_sd", ctypes.c_double),
                ("w_shape", ctypes.c_double), ("w_rate", ctypes.c_double),
                ("alpha_min", ctypes.c_double)]


class Variant(ctypes.Structure):
    """orc_variant: likelihood, objective, shared shapes, angle-dependent width,
    fitted background (coefficients, their gradient and Adam moments)."""
    _PD = ctypes.POINTER(ctypes.c_double)
    _fields_ = [("lik", ctypes.c_int), ("iw", ctypes.c_int), ("shared", ctypes.c_int), ("sec", ctypes.c_int),
                ("bgfit", ctypes.c_int), ("bg_sd", ctypes.c_double), ("beta", _PD), ("grad_beta", _PD),
                ("m_beta", _PD), ("v_beta", _PD), ("fix_r", ctypes.c_int), ("fix_alpha", ctypes.c_int),
                ("r_value", ctypes.c_double), ("alpha_value", ctypes.c_double), ("area_norm", ctypes.c_int),
                ("gates", ctypes.c_int), ("gate_tau", ctypes.c_double), ("gate_prior_logit", ctypes.c_double),
                ("gate_a", _PD), ("grad_gate", _PD), ("m_gate", _PD), ("v_gate", _PD), ("gate_noise", _PD)]


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (no fast-math, no FMA
    contraction, so x86 and Arm builds round alike)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.POINTER
            d, i32, u32, u64 = ctypes.c_double, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
            pd, pi = P(d), P(i32)
            L.orc_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
            L.orc_normals.argtypes = [u64, u32, u32, i32, i32, pd]
            L.orc_softplus.restype = d
            L.orc_softplus.argtypes = [d]
            L.orc_sigmoid.restype = d
            L.orc_sigmoid.argtypes = [d]
            L.orc_theta.argtypes = [i32, i32, pd, pd, pd, pd, pd]
            L.orc_components.argtypes = [d, d, d, pd, pd]
            L.orc_pvoigt.restype = d
            L.orc_pvoigt.argtypes = [d, d, d, d]
            L.orc_profile.argtypes = [i32, pi, pd, pd, i32, pd, pd, i32, pd, d, pd]
            L.orc_loglik_direct.restype = d
            L.orc_loglik_direct.argtypes = [i32, pd, pd]
            L.orc_loglik_deviance.restype = d
            L.orc_loglik_deviance.argtypes = [i32, pd, pd, pd]
            L.orc_log_prior.restype = d
            L.orc_log_prior.argtypes = [P(Prior), pd]
            L.orc_log_jac.restype = d
            L.orc_log_jac.argtypes = [pd]
            L.orc_entropy.restype = d
            L.orc_entropy.argtypes = [i32, pd]
            L.orc_elbo_grad.argtypes = [i32, pi, pd, pd, i32, pd, pd, pd, P(Prior), i32,
                                        pd, pd, pd, pd, pd, pd, pd, pd]
            L.orc_elbo_grad_ex.argtypes = [i32, pi, pd, pd, i32, pd, pd, pd, P(Prior), P(Variant), i32,
                                           pd, pd, pd, pd, pd, pd, pd, pd]
            L.orc_fit_ex.argtypes = [i32, pi, pd, pd, i32, pd, pd, pd, P(Prior), P(Variant), i32, u64, i32, i32,
                                     d, d, d, d, pd, pd, pd, pd, pd]
            L.orc_profile_ex.argtypes = [i32, pi, pd, pd, i32, pd, pd, i32, pd, d, i32, i32, pd]
            L.orc_area_factor.restype = d
            L.orc_area_factor.argtypes = [d, d, d]
            L.orc_gate_noise.argtypes = [u64, ctypes.c_uint32, ctypes.c_uint32, i32, i32, pd]
            L.orc_gate_terms.restype = d
            L.orc_gate_terms.argtypes = [d, d, d, d, pd, pd]
            L.orc_sec.restype = d
            L.orc_sec.argtypes = [d]
            L.orc_background.argtypes = [i32, pd, pd, pd, pd, pd]
            L.orc_background_prior.restype = d
            L.orc_background_prior.argtypes = [pd, d]
            L.orc_tie_shapes.argtypes = [i32, i32, pd]
            L.orc_loglik_gauss.restype = d
            L.orc_loglik_gauss.argtypes = [i32, pd, pd]
            L.orc_iw_weights.restype = d
            L.orc_iw_weights.argtypes = [i32, i32, pd, pd, pd, pd, P(Variant), pd]
            L.orc_fixed_lpj.restype = d
            L.orc_fixed_lpj.argtypes = [P(Prior), P(Variant), pd, pd]
            L.orc_adam_step.argtypes = [i32, pd, pd, pd, pd, i32, d, d, d, d]
            L.orc_fit.argtypes = [i32, pi, pd, pd, i32, pd, pd, pd, P(Prior), i32, u64, i32, i32,
                                  d, d, d, d, pd, pd, pd, pd, pd]
            L.orc_max_threads.restype = i32
            _lib = L
    return _lib


def _pd(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pi(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Problem:
    """Double-precision copy of one instance (peak table + pattern + priors)."""

    def __init__(self, offsets, pos, inten, x, y, bg, *, lam=None,
                 mu_sd=PRIOR_MU_SD, alpha_mean=PRIOR_ALPHA_MEAN, alpha_sd=PRIOR_ALPHA_SD,
                 w_shape=PRIOR_W_SHAPE, w_rate=PRIOR_W_RATE, alpha_min=ALPHA_MIN,
                 likelihood="poisson", objective="elbo", shapes="independent", width="constant",
                 background="fixed", bg_sd=0.1, fix_r=None, fix_alpha=None, normalisation="height",
                 gates=False, gate_tau=2.0 / 3.0, gate_prior=0.5):
        # variants: likelihood "poisson" (the paper's) or "gauss" (variance
        # max(y, 1)); objective "elbo" or "iw" (importance-weighted bound);
        # shapes "independent" or "shared" (one shape draw per step); width
        # "constant" or "sec" (side widths times sec(2theta / 2) at each point)
        assert likelihood in ("poisson", "gauss") and objective in ("elbo", "iw")
        assert shapes in ("independent", "shared") and width in ("constant", "sec")
        assert background in ("fixed", "fitted")
        self.lik = 1 if likelihood == "gauss" else 0
        self.iw = 1 if objective == "iw" else 0
        self.shared = 1 if shapes == "shared" else 0
        self.sec = 1 if width == "sec" else 0
        self.bgfit = 1 if background == "fitted" else 0
        # fitted background: correction coefficients beta[3] (point estimate)
        self.beta = np.zeros(3)
        self._gb = np.zeros(3)
        # fix_r / fix_alpha: r / alpha held at that value (a model constant, not in q)
        self.fix_r, self.fix_alpha = fix_r, fix_alpha
        self.variant = Variant(self.lik, self.iw, self.shared, self.sec, self.bgfit, float(bg_sd),
                               _pd(self.beta), _pd(self._gb), None, None,
                               0 if fix_r is None else 1, 0 if fix_alpha is None else 1,
                               0.0 if fix_r is None else float(fix_r), 0.0 if fix_alpha is None else float(fix_alpha),
                               1 if normalisation == "area" else 0)
        # normalisation "height" (peak height h) or "area" (h = integrated intensity)
        assert normalisation in ("height", "area")
        self.area_norm = normalisation == "area"
        # gates: binary-Concrete phase gates with temperature gate_tau and prior
        # inclusion probability gate_prior; gate logits a[K] start at 0
        self.gates = bool(gates)
        self.gate_tau = float(gate_tau)
        self.gate_a = None
        self._ggate = None
        self.variant.gates = 1 if gates else 0
        self.variant.gate_tau = float(gate_tau)
        self.variant.gate_prior_logit = math.log(gate_prior / (1.0 - gate_prior))
        self.off = np.ascontiguousarray(offsets, dtype=np.int32)
        self.pos, self.inten = f64(pos), f64(inten)
        self.x, self.y, self.bg = f64(x), f64(y), f64(bg)
        self.K, self.N = len(self.off) - 1, len(self.x)
        if lam is None:
            # lambda = 1 / eta with eta = max(Y - B)  (Sec. 2.2)
            lam = 1.0 / float(np.max(self.y - self.bg))
        self.prior = Prior(lam, mu_sd, alpha_mean, alpha_sd, w_shape, w_rate, alpha_min)
        if self.gates:
            self.gate_a = np.zeros(self.K)
            self._ggate = np.zeros(self.K)
            self.variant.gate_a, self.variant.grad_gate = _pd(self.gate_a), _pd(self._ggate)

    def free(self, j):
        """Is parameter j (h, mu, w, r, alpha) part of q?"""
        return not ((j == 3 and self.fix_r is not None) or (j == 4 and self.fix_alpha is not None))

    @classmethod
    def from_instance(cls, inst, **kw):
        return cls(inst.offsets, inst.pos, inst.inten, inst.x, inst.y, inst.bg, **kw)

    @property
    def eta(self):
        return 1.0 / self.prior.lambda_

    def _args(self):
        return (self.K, _pi(self.off), _pd(self.pos), _pd(self.inten), self.N,
                _pd(self.x), _pd(self.y), _pd(self.bg))

    # ---- model -----------------------------------------------------------
    def profile(self, theta):
        """f[S, N] for physical parameters theta[S, K, 5]."""
        theta = f64(theta)
        S = theta.shape[0]
        f = np.zeros((S, self.N))
        lib().orc_profile_ex(self.K, _pi(self.off), _pd(self.pos), _pd(self.inten), self.N,
                             _pd(self.x), _pd(self.bg), S, _pd(theta), self.prior.alpha_min, self.sec,
                             1 if self.area_norm else 0, _pd(f))
        return f

    def loglik(self, f, form="direct"):
        f = f64(f)
        if form == "gauss":
            return lib().orc_loglik_gauss(self.N, _pd(self.y), _pd(f))
        if form == "direct":
            return lib().orc_loglik_direct(self.N, _pd(self.y), _pd(f))
        return lib().orc_loglik_deviance(self.N, _pd(self.y), _pd(f), None)

    def data_constant(self):
        """sum_i [y ln y - y - ln y!] (the data part of the deviance split)."""
        c = ctypes.c_double(0.0)
        lib().orc_loglik_deviance(self.N, _pd(self.y), _pd(self.bg), ctypes.byref(c))
        return c.value

    def theta(self, loc, raw, eps):
        eps = f64(eps)
        S = eps.shape[0]
        u = np.zeros((S, self.K, 5))
        th = np.zeros((S, self.K, 5))
        lib().orc_theta(S, self.K, _pd(f64(loc)), _pd(f64(raw)), _pd(eps), _pd(u), _pd(th))
        if self.fix_r is not None:
            th[:, :, 3] = self.fix_r
        if self.fix_alpha is not None:
            th[:, :, 4] = self.fix_alpha
        return u, th

    def log_prior(self, th_k):
        return lib().orc_log_prior(ctypes.byref(self.prior), _pd(f64(th_k)))

    def log_prior_jac(self, u_k, th_k):
        """ln p(theta) + ln|J| of one phase of one draw, without the terms of
        parameters held fixed."""
        u_k, th_k = f64(u_k), f64(th_k)
        return (lib().orc_log_prior(ctypes.byref(self.prior), _pd(th_k)) + lib().orc_log_jac(_pd(u_k))
                - lib().orc_fixed_lpj(ctypes.byref(self.prior), ctypes.byref(self.variant), _pd(u_k), _pd(th_k)))

    def elbo_grad(self, loc, raw, eps, want_f=False, gate_noise=None):
        """ELBO estimate + per-sample LL, log prior+Jacobian and the gradient
        [K, 10] (loc grads then raw grads) for injected noise eps[S, K, 5]."""
        eps = f64(eps).copy()
        S = eps.shape[0]
        if self.shared:
            lib().orc_tie_shapes(S, self.K, _pd(eps))
        if self.gates:   # logistic gate noise [S, K] (zeros: the gate at its location)
            gn = np.zeros((S, self.K)) if gate_noise is None else f64(gate_noise).copy()
            self.variant.gate_noise = _pd(gn)
        elbo = ctypes.c_double(0.0)
        ll = np.zeros(S)
        lpj = np.zeros(S)
        grad = np.zeros((self.K, 10))
        f = np.zeros((S, self.N)) if want_f else None
        lib().orc_elbo_grad_ex(*self._args(), ctypes.byref(self.prior), ctypes.byref(self.variant), S, _pd(f64(loc)),
                               _pd(f64(raw)), _pd(eps), ctypes.byref(elbo), _pd(ll), _pd(lpj),
                               _pd(grad), _pd(f) if want_f else None)
        out = {"elbo": elbo.value, "ll": ll, "lpj": lpj, "grad": grad}
        if self.bgfit:
            out["grad_beta"] = self._gb.copy()
        if self.gates:
            out["grad_gate"] = self._ggate.copy()
        if want_f:
            out["f"] = f
        return out

    def init_params(self, h_frac=0.1, sigma0=0.1):
        """Initial variational state.  Reading: loc at h = h_frac * eta, mu = 0,
        w = prior mean shape/rate, r = 1/2, alpha = prior mean; every sigma = sigma0."""
        loc = np.zeros((self.K, 5))
        loc[:, 0] = math.log(h_frac * self.eta)
        if self.area_norm:   # same starting curve: the height times the area of the initial shape
            loc[:, 0] += math.log(lib().orc_area_factor(self.prior.w_shape / self.prior.w_rate,
                                                        max(self.prior.alpha_mean, self.prior.alpha_min), 0.5))
        loc[:, 1] = 0.0
        loc[:, 2] = math.log(self.prior.w_shape / self.prior.w_rate)
        loc[:, 3] = 0.0
        loc[:, 4] = self.prior.alpha_mean
        raw = np.full((self.K, 5), math.log(math.expm1(sigma0)))
        return loc, raw

    def background(self, beta=None):
        """B(beta) [N] of the fitted-background variant (the current beta by default)."""
        b = self.beta if beta is None else f64(beta)
        out = np.zeros(self.N)
        lib().orc_background(self.N, _pd(self.x), _pd(self.bg), _pd(b), _pd(out), None)
        return out

    def fit(self, S, iters, seed, loc=None, raw=None, m=None, v=None, t0=0,
            lr=0.01, b1=0.9, b2=0.999, adam_eps=1e-8, m_beta=None, v_beta=None):
        if loc is None:
            loc, raw = self.init_params()
        loc, raw = f64(loc).copy(), f64(raw).copy()
        m = np.zeros((self.K, 10)) if m is None else f64(m).copy()
        v = np.zeros((self.K, 10)) if v is None else f64(v).copy()
        trace = np.zeros(iters)
        mb = np.zeros(3) if m_beta is None else f64(m_beta).copy()
        vb = np.zeros(3) if v_beta is None else f64(v_beta).copy()
        self.variant.m_beta, self.variant.v_beta = _pd(mb), _pd(vb)
        mg = np.zeros(self.K)
        vg = np.zeros(self.K)
        if self.gates:
            self.variant.m_gate, self.variant.v_gate = _pd(mg), _pd(vg)
        lib().orc_fit_ex(*self._args(), ctypes.byref(self.prior), ctypes.byref(self.variant), S, seed, t0, iters,
                         lr, b1, b2, adam_eps, _pd(loc), _pd(raw), _pd(m), _pd(v), _pd(trace))
        out = {"loc": loc, "raw": raw, "m": m, "v": v, "trace": trace}
        if self.bgfit:
            out.update({"beta": self.beta.copy(), "m_beta": mb, "v_beta": vb})
        if self.gates:
            out.update({"gate_a": self.gate_a.copy(), "m_gate": mg, "v_gate": vg})
        return out


def iw_weights(raw, eps, ll, lpj):
    """(L_S, normalised weights[S]) of the importance-weighted bound."""
    eps = f64(eps)
    S, K = eps.shape[0], eps.shape[1]
    wt = np.zeros(S)
    L = lib().orc_iw_weights(K, S, _pd(f64(raw)), _pd(eps), _pd(f64(ll)), _pd(f64(lpj)), None, _pd(wt))
    return L, wt


def gate_noise(seed, tag, it, S, K):
    """Logistic gate noise [S, K] of the oracle's stream."""
    L = np.zeros((S, K))
    lib().orc_gate_noise(seed, tag, it, S, K, _pd(L))
    return L


def gate_terms(a, L, tau, a0):
    """(z, ln p(y) - ln q(y), d ln p / dy) of one binary-Concrete gate."""
    z, dp = ctypes.c_double(0.0), ctypes.c_double(0.0)
    v = lib().orc_gate_terms(float(a), float(L), float(tau), float(a0), ctypes.byref(z), ctypes.byref(dp))
    return z.value, v, dp.value


def philox(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return list(o)


def normals(seed, tag, it, S, K):
    eps = np.zeros((S, K, 5))
    lib().orc_normals(seed, tag, it, S, K, _pd(eps))
    return eps


def softplus(x):
    return lib().orc_softplus(float(x))


def sigmoid(x):
    return lib().orc_sigmoid(float(x))


def components(d, w, alpha_c):
    G, L = ctypes.c_double(), ctypes.c_double()
    lib().orc_components(float(d), float(w), float(alpha_c), ctypes.byref(G), ctypes.byref(L))
    return G.value, L.value


def pvoigt(d, w, r, alpha_c):
    return lib().orc_pvoigt(float(d), float(w), float(r), float(alpha_c))


def entropy(raw):
    raw = f64(raw)
    return lib().orc_entropy(raw.shape[0], _pd(raw))


def adam_step(params, grad, m, v, t, lr=0.01, b1=0.9, b2=0.999, eps=1e-8):
    params, m, v = f64(params).copy(), f64(m).copy(), f64(v).copy()
    lib().orc_adam_step(params.size, _pd(params), _pd(f64(grad)), _pd(m), _pd(v), t, lr, b1, b2, eps)
    return params, m, v


def max_threads():
    return lib().orc_max_threads()
