"""FP64 CPU oracle for the muon-tomography log-posterior (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline``
and ``--impl reference`` legs may import this package.  The product path (the
CUDA library and its binding) never imports, links or runs it, and it never
imports the product: the two share nothing but the seeded input generator in
``paper_2603_28907_gb300.workloads``, which holds none of the method's
arithmetic.

The arithmetic lives in ``oracle.c`` (plain C, FP64, compiled without FMA
contraction).  This module compiles it on first use and exposes thin ctypes
wrappers that take numpy arrays.

Parity status of every routine is stated in ``oracle.c``; all are pinned by
``tests/test_oracle_*.py`` except where that file says "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
             "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class Problem(C.Structure):
    _fields_ = [
        ("L", C.c_int), ("R", C.c_int), ("Q", C.c_int),
        ("box", C.c_double * 3),
        ("rho", C.POINTER(C.c_double)),
        ("S", C.c_int), ("P", C.c_int),
        ("sensor", C.POINTER(C.c_double)),
        ("dir", C.POINTER(C.c_double)),
        ("counts", C.POINTER(C.c_int32)),
        ("G", C.c_int),
        ("gamma", C.c_double), ("I0", C.c_double), ("Lambda", C.c_double),
        ("tau", C.c_double), ("car_r", C.c_double), ("delta", C.c_double),
        ("mu", C.POINTER(C.c_double)),
    ]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_up = C.POINTER(C.c_uint32)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER(Problem)
            sig = {
                "or_philox": (None, [_up, _up, _up]),
                "or_u01": (C.c_double, [C.c_uint32, C.c_uint32]),
                "or_normals": (None, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int, _dp]),
                "or_t_exit": (C.c_double, [_dp, _dp, _dp]),
                "or_surface": (C.c_double, [C.c_int, C.c_int, _dp, _dp, C.c_double, C.c_double]),
                "or_sigma": (C.c_double, [C.c_double, C.c_double]),
                "or_ray_opacity": (C.c_double, [P, _dp, C.c_int, C.c_int, _dp]),
                "or_lambda": (C.c_double, [C.c_double, C.c_double, C.c_double]),
                "or_poisson_logpmf": (C.c_double, [C.c_int32, C.c_double]),
                "or_poisson_logpmf_centred": (C.c_double, [C.c_int32, C.c_double, C.c_double, C.c_double]),
                "or_loglik": (C.c_double, [P, _dp]),
                "or_loglik_terms": (None, [P, _dp, _dp, _dp]),
                "or_logprior": (C.c_double, [P, _dp]),
                "or_poisson_draw": (C.c_int32, [C.c_double, C.c_uint64, C.c_uint32, C.POINTER(C.c_int)]),
                "or_poisson_mean_attempts": (C.c_double, [C.c_double, C.c_uint64, C.c_int]),
                "or_generate_counts": (C.c_int, [P, _dp, C.c_uint64, C.c_int, _ip, _dp]),
                "or_rw_propose": (None, [P, _dp, C.c_double, C.c_uint64, C.c_uint32, C.c_uint32, _dp]),
                "or_accept_logu": (C.c_double, [C.c_uint64, C.c_uint32, C.c_uint32]),
                "or_mh_decide": (C.c_int, [C.c_double] * 5),
                "or_rw_chain": (C.c_int, [P, _dp, C.c_double, C.c_uint64, C.c_uint32, C.c_uint32,
                                          C.c_int, C.c_int, _dp, _dp, _dp]),
                "or_grad_loglik": (None, [P, _dp, _dp]),
                "or_grad_logprior": (None, [P, _dp, _dp]),
                "or_mala_propose": (None, [P, _dp, _dp, C.c_double, C.c_uint64, C.c_uint32,
                                           C.c_uint32, _dp]),
                "or_mala_logq": (C.c_double, [C.c_int, _dp, _dp, _dp, C.c_double]),
                "or_loglik_batch": (None, [P, C.c_int, _dp, _dp, C.c_int]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray, t=_dp):
    return a.ctypes.data_as(t)


class OracleProblem:
    """A problem (grid, units, sensors, pixels, counts, prior) in oracle form.

    ``prob`` is a dict as produced by ``paper_2603_28907_gb300.workloads``.
    Arrays are copied to contiguous FP64 / int32 and kept alive here.
    """

    def __init__(self, prob: dict, counts=None):
        self.lib = _load()
        self.L, self.R, self.Q = int(prob["L"]), int(prob["R"]), int(prob["Q"])
        self.box = _d(prob["box"])
        self.rho = _d(prob["rho"])
        self.sensors = _d(prob["sensors"]).reshape(-1, 3)
        self.dirs = _d(prob["dirs"]).reshape(-1, 3)
        self.S, self.P = self.sensors.shape[0], self.dirs.shape[0]
        c = counts if counts is not None else prob.get("counts")
        if c is None:
            c = np.zeros((self.S, self.P), np.int32)
        self.counts = np.ascontiguousarray(c, dtype=np.int32).reshape(self.S, self.P)
        self.mu = _d(prob["mu"]).reshape(self.L, self.R, self.Q)
        self.G = int(prob["G"])
        self.params = dict(gamma=float(prob["gamma"]), I0=float(prob["I0"]),
                           Lambda=float(prob["Lambda"]), tau=float(prob["tau"]),
                           car_r=float(prob["car_r"]), delta=float(prob["delta"]))
        self._mk()

    def _mk(self):
        s = Problem()
        s.L, s.R, s.Q = self.L, self.R, self.Q
        for i in range(3):
            s.box[i] = self.box[i]
        s.rho = _ptr(self.rho)
        s.S, s.P = self.S, self.P
        s.sensor = _ptr(self.sensors)
        s.dir = _ptr(self.dirs)
        s.counts = _ptr(self.counts, _ip)
        s.G = self.G
        for k, v in self.params.items():
            setattr(s, k, v)
        s.mu = _ptr(self.mu)
        self.s = s

    def with_counts(self, counts):
        self.counts = np.ascontiguousarray(counts, dtype=np.int32).reshape(self.S, self.P)
        self._mk()
        return self

    def set(self, **kw):
        """Override gamma / I0 / Lambda / tau / car_r / delta / G."""
        for k, v in kw.items():
            if k == "G":
                self.G = int(v)
            else:
                self.params[k] = float(v)
        self._mk()
        return self

    @property
    def n(self):
        return self.L * self.R * self.Q

    # --- forward model -------------------------------------------------
    def ray_opacity(self, H, s, p, with_units=False):
        H = _d(H)
        ul = np.zeros(self.L + 1)
        O = self.lib.or_ray_opacity(C.byref(self.s), _ptr(H), s, p, _ptr(ul))
        return (O, ul) if with_units else O

    def opacities(self, H):
        H = _d(H)
        out = np.zeros((self.S, self.P))
        self.lib.or_loglik_terms(C.byref(self.s), _ptr(H), None, _ptr(out))
        return out

    def loglik_terms(self, H):
        H = _d(H)
        out = np.zeros((self.S, self.P))
        self.lib.or_loglik_terms(C.byref(self.s), _ptr(H), _ptr(out), None)
        return out

    def loglik(self, H):
        return self.lib.or_loglik(C.byref(self.s), _ptr(_d(H)))

    def loglik_batch(self, Hs, n_threads=1):
        Hs = _d(Hs).reshape(-1, self.n)
        out = np.zeros(Hs.shape[0])
        self.lib.or_loglik_batch(C.byref(self.s), Hs.shape[0], _ptr(Hs), _ptr(out), n_threads)
        return out

    def logprior(self, H):
        return self.lib.or_logprior(C.byref(self.s), _ptr(_d(H)))

    def generate_counts(self, H_true, seed, count_mode=0):
        H = _d(H_true)
        counts = np.zeros((self.S, self.P), np.int32)
        lam = np.zeros((self.S, self.P))
        bad = self.lib.or_generate_counts(C.byref(self.s), _ptr(H), seed, count_mode,
                                          _ptr(counts, _ip), _ptr(lam))
        return counts, lam, bad

    # --- MCMC ------------------------------------------------------------
    def rw_propose(self, H, sigma, seed, chain, step):
        H = _d(H)
        out = np.zeros_like(H)
        self.lib.or_rw_propose(C.byref(self.s), _ptr(H), sigma, seed, chain, step, _ptr(out))
        return out

    def rw_chain(self, H, sigma, seed, chain, step0, n_steps, use_lik=True, trace=False):
        H = _d(H).copy()
        lp, ll = C.c_double(), C.c_double()
        tr = np.zeros((n_steps, self.n)) if trace else None
        acc = self.lib.or_rw_chain(C.byref(self.s), _ptr(H), sigma, seed, chain, step0, n_steps,
                                   int(use_lik), C.byref(lp), C.byref(ll),
                                   _ptr(tr) if trace else None)
        return H, acc, lp.value, ll.value, tr

    def grad_loglik(self, H):
        H = _d(H)
        g = np.zeros_like(H)
        self.lib.or_grad_loglik(C.byref(self.s), _ptr(H), _ptr(g))
        return g

    def grad_logprior(self, H):
        H = _d(H)
        g = np.zeros_like(H)
        self.lib.or_grad_logprior(C.byref(self.s), _ptr(H), _ptr(g))
        return g

    def mala_propose(self, H, grad, eps, seed, chain, step):
        H, grad = _d(H), _d(grad)
        out = np.zeros_like(H)
        self.lib.or_mala_propose(C.byref(self.s), _ptr(H), _ptr(grad), eps, seed, chain, step,
                                 _ptr(out))
        return out

    def mala_logq(self, b, a, grad_a, eps):
        b, a, g = _d(b), _d(a), _d(grad_a)
        return self.lib.or_mala_logq(b.size, _ptr(b), _ptr(a), _ptr(g), eps)


# --- free functions ------------------------------------------------------
def philox(ctr, key):
    lib = _load()
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib.or_philox(c, k, o)
    return [int(x) for x in o]


def u01(lo, hi):
    return _load().or_u01(lo, hi)


def normals(seed, stream, chain, step, n):
    z = np.zeros(n)
    _load().or_normals(seed, stream, chain, step, n, _ptr(z))
    return z


def t_exit(o, d, box):
    o, d, box = _d(o), _d(d), _d(box)
    return _load().or_t_exit(_ptr(o), _ptr(d), _ptr(box))


def surface(R, Q, box, h, x, y):
    box, h = _d(box), _d(h)
    return _load().or_surface(R, Q, _ptr(box), _ptr(h), x, y)


def sigma(u, gamma):
    return _load().or_sigma(u, gamma)


def poisson_logpmf(C_, lam):
    return _load().or_poisson_logpmf(int(C_), float(lam))


def poisson_logpmf_centred(C_, O, I0, Lambda):
    return _load().or_poisson_logpmf_centred(int(C_), float(O), float(I0), float(Lambda))


def poisson_draw(lam, seed, ray):
    st = C.c_int(0)
    k = _load().or_poisson_draw(float(lam), seed, ray, C.byref(st))
    return int(k), int(st.value)


def poisson_mean_attempts(lam, seed, n):
    """Mean number of attempts of the count sampler over rays 0 .. n-1 (test instrumentation)."""
    return _load().or_poisson_mean_attempts(float(lam), seed, int(n))


def accept_logu(seed, chain, step):
    return _load().or_accept_logu(seed, chain, step)


def mh_decide(lp_new, ll_new, lp_old, ll_old, logu):
    return bool(_load().or_mh_decide(lp_new, ll_new, lp_old, ll_old, logu))


STREAM = dict(GEOM=0, DATA=1, INIT=2, PROP=3, ACC=4, MALA=5)
