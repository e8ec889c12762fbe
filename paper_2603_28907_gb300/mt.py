"""ctypes binding of libmt.so (include/mt.h): argument marshalling only.

Every function here forwards to the C ABI of the same name; all arithmetic of
the path runs in the library's CUDA kernels.  Arrays may be torch tensors
(device or host) or numpy arrays (host).  There is no fallback: if the
library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# MT_CHECKED=1 loads the bounds-checked build (libmt_checked.so, built by
# build.build(checked=True)); it has the same ABI
LIB_PATH = os.path.join(HERE, "libmt_checked.so" if os.environ.get("MT_CHECKED") == "1" else "libmt.so")

PREC_F64, PREC_F32, PREC_F32C, PREC_BF16, PREC_F32A = 0, 1, 2, 3, 4
PRIOR_CAR, PRIOR_COPULA = 0, 1
FORWARD_MARCH, FORWARD_LINEAR = 0, 1
KERNEL_RW, KERNEL_MALA, KERNEL_HMC, KERNEL_NUTS = 0, 1, 2, 3
COUNTS_POISSON, COUNTS_ROUND = 0, 1

STATUS = {0: "MT_OK", -1: "MT_EINVAL", -2: "MT_ENOMEM", -3: "MT_ESTATE", -4: "MT_ECUDA",
          -5: "MT_ETIMEDOUT", -6: "MT_EDEVFLAG", -7: "MT_ECANCELED"}


class MtError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__(f"{fn}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(C.Structure):
    _fields_ = [("precision", C.c_int), ("n_grid", C.c_int), ("gamma", C.c_double),
                ("I0", C.c_double), ("atten", C.c_double), ("tau", C.c_double),
                ("car_r", C.c_double), ("min_thick", C.c_double)]


class Request(C.Structure):
    _fields_ = [("cfg", Config), ("n_layers", C.c_int), ("n_rows", C.c_int), ("n_cols", C.c_int),
                ("box", C.c_void_p), ("unit_density", C.c_void_p), ("prior_mean", C.c_void_p),
                ("n_sensors", C.c_int), ("sensors", C.c_void_p), ("n_pixels", C.c_int),
                ("dirs", C.c_void_p), ("counts", C.c_void_p), ("h_true", C.c_void_p),
                ("data_seed", C.c_uint64), ("n_chains", C.c_int), ("heights0", C.c_void_p),
                ("seed", C.c_uint64), ("kernel", C.c_int), ("step", C.c_double),
                ("n_super", C.c_int), ("n_within", C.c_int)]


class RequestInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("n_supersteps", C.c_int), ("submit_s", C.c_double),
                ("admit_s", C.c_double), ("done_s", C.c_double),
                ("superstep_ms_p50", C.c_double), ("superstep_ms_p99", C.c_double),
                ("gpu_start_ms", C.c_double), ("gpu_end_ms", C.c_double), ("gpu_busy_ms", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("n_done", C.c_int64), ("n_pending", C.c_int64), ("n_active", C.c_int64),
                ("superstep_ms_p50", C.c_double), ("superstep_ms_p99", C.c_double),
                ("ttp_s_p50", C.c_double), ("ttp_s_p99", C.c_double),
                ("chain_ray_evals_per_s", C.c_double), ("bytes_in_use", C.c_size_t),
                ("pool_bytes_at_start", C.c_size_t), ("pool_bytes_now", C.c_size_t)]


_lib = None
_vp, _dp, _ip, _lp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_int64)

SIGNATURES = {
    "mt_create": [C.POINTER(C.c_void_p), C.c_int, C.POINTER(Config), _vp],
    "mt_destroy": [_vp],
    "mt_set_grid": [_vp, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp],
    "mt_set_sensors": [_vp, C.c_int, _vp],
    "mt_set_pixels": [_vp, C.c_int, _vp],
    "mt_set_counts": [_vp, _vp],
    "mt_generate_data": [_vp, _vp, C.c_uint64, C.c_int, _vp, _vp],
    "mt_logpost": [_vp, C.c_int, _vp, _vp, _vp],
    "mt_ray_terms": [_vp, C.c_int, _vp, _vp, _vp],
    "mt_logpost_noalloc": [_vp, C.c_int, _vp, _vp, _vp],
    "mt_grad": [_vp, C.c_int, _vp, _vp, _vp],
    "mt_init_chains": [_vp, C.c_int, _vp, C.c_uint64],
    "mt_run": [_vp, C.c_int, C.c_double, C.c_int, C.c_int],
    "mt_get_state": [_vp, _vp, _vp, _vp, _vp, _lp],
    "mt_get_last_step": [_vp, _vp, _vp, _vp, _vp, _vp],
    "mt_set_state": [_vp, _vp, C.c_int64],
    "mt_sync": [_vp, C.c_double],
    "mt_set_timing": [_vp, C.c_int],
    "mt_get_timing": [_vp, C.c_int, _dp, _lp, C.c_int],
    "mt_get_work": [_vp, _dp, _dp, C.c_int],
    "mt_get_sizes": [_vp, _ip, _ip, _ip, _ip, _ip, _ip],
    "mt_set_prior": [_vp, C.c_int],
    "mt_set_hmc": [_vp, C.c_int],
    "mt_set_nuts": [_vp, C.c_int],
    "mt_set_adapt": [_vp, C.c_double, C.c_int],
    "mt_get_adapt": [_vp, _vp, _vp],
    "mt_set_metric_adapt": [_vp, C.c_int, C.c_double],
    "mt_get_metric": [_vp, _vp],
    "mt_set_forward": [_vp, C.c_int, C.c_int, _vp],
    "mt_copula_heights": [_vp, C.c_int, _vp, _vp],
    "mt_nested_rhat": [_vp, C.c_int, C.c_int, _vp, C.c_int, _vp, _dp],
    "mt_interface_std": [_vp, C.c_int, _vp, C.c_int, _vp],
    "mt_server_create": [C.POINTER(C.c_void_p), C.c_int, C.c_size_t, C.c_int],
    "mt_server_submit": [_vp, C.POINTER(Request), C.POINTER(C.c_int64)],
    "mt_server_wait": [_vp, C.c_int64, C.c_double, _vp, _vp, _vp, _vp, C.POINTER(RequestInfo)],
    "mt_server_stats": [_vp, C.POINTER(ServerStats)],
    "mt_server_cancel": [_vp, C.c_int64],
    "mt_server_destroy": [_vp],
}


def load():
    """Load libmt.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2603_28907_gb300.build` (needs nvcc)")
        lib = C.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = C.c_int
        lib.mt_last_error.argtypes = [_vp]
        lib.mt_last_error.restype = C.c_char_p
        lib.mt_server_last_error.argtypes = [_vp]
        lib.mt_server_last_error.restype = C.c_char_p
        _lib = lib
    return _lib


def _ptr(a):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


class Context:
    """One mt_ctx: a problem (grid, sensors, pixels, counts) and its chains."""

    def __init__(self, device: int = 0, precision: int = PREC_F32, n_grid: int = 64,
                 gamma: float = 1.0, I0: float = 1e4, atten: float = 150.0, tau: float = 0.01,
                 car_r: float = 0.99, min_thick: float = 0.1, stream=None):
        self.lib = load()
        self.cfg = Config(precision, n_grid, gamma, I0, atten, tau, car_r, min_thick)
        h = C.c_void_p()
        st = self.lib.mt_create(C.byref(h), device, C.byref(self.cfg),
                                None if stream is None else C.c_void_p(int(stream)))
        if st != 0:
            raise MtError("mt_create", st, self.lib.mt_last_error(None).decode())
        self.h = h
        self.device = device
        self.precision = precision
        self._keep = []

    # -- plumbing
    def _ck(self, name, st):
        if st != 0:
            raise MtError(name, st, self.lib.mt_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.mt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def height_dtype(self):
        return np.float64 if self.precision == PREC_F64 else np.float32

    # -- problem set-up
    def set_grid(self, n_layers, n_rows, n_cols, box, unit_density, prior_mean=None):
        box = np.ascontiguousarray(box, np.float64)
        rho = np.ascontiguousarray(unit_density, np.float64)
        mu = None if prior_mean is None else np.ascontiguousarray(prior_mean, np.float64)
        self._ck("mt_set_grid", self.lib.mt_set_grid(self.h, n_layers, n_rows, n_cols, _ptr(box),
                                                     _ptr(rho), _ptr(mu)))

    def set_sensors(self, pos):
        pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
        self._ck("mt_set_sensors", self.lib.mt_set_sensors(self.h, pos.shape[0], _ptr(pos)))

    def set_pixels(self, dirs):
        dirs = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
        self._ck("mt_set_pixels", self.lib.mt_set_pixels(self.h, dirs.shape[0], _ptr(dirs)))

    def set_counts(self, counts):
        if not hasattr(counts, "data_ptr"):
            counts = np.ascontiguousarray(counts, np.int32)
        self._ck("mt_set_counts", self.lib.mt_set_counts(self.h, _ptr(counts)))

    def generate_data(self, h_true, seed, count_mode=COUNTS_POISSON, counts_out=None,
                      lambda_out=None):
        h = np.ascontiguousarray(h_true, np.float64)
        self._ck("mt_generate_data", self.lib.mt_generate_data(
            self.h, _ptr(h), seed, count_mode, _ptr(counts_out), _ptr(lambda_out)))

    def sizes(self):
        v = [C.c_int() for _ in range(6)]
        self._ck("mt_get_sizes", self.lib.mt_get_sizes(self.h, *[C.byref(x) for x in v]))
        return dict(zip(["L", "R", "Q", "S", "P", "C"], [x.value for x in v]))

    # -- evaluation
    def _check_batch(self, name, heights, outs, device_only=False):
        """Reject arrays the library would read or write out of bounds: heights
        [n][L][R][Q] of the precision's dtype (FP64 / FP32), outputs of at least
        n doubles, torch tensors on the context's device."""
        want = np.dtype(self.height_dtype)
        sz = self.sizes()
        lrq = (sz["L"], sz["R"], sz["Q"])
        arrs = [("heights", heights)] + [(k, v) for k, v in outs if v is not None]
        for label, a in arrs:
            if hasattr(a, "data_ptr"):
                dt = np.dtype(str(a.dtype).replace("torch.", ""))
                dev = a.device.index if a.device.type == "cuda" else None
                if device_only and a.device.type != "cuda":
                    raise ValueError(f"{name}: {label} must be a CUDA tensor")
                if a.device.type == "cuda" and dev != self.device:
                    raise ValueError(f"{name}: {label} is on cuda:{dev}, the context on cuda:{self.device}")
            elif isinstance(a, np.ndarray):
                if device_only:
                    raise ValueError(f"{name}: {label} must be device memory")
                dt = a.dtype
            else:
                raise TypeError(f"{name}: {label}: unsupported array type {type(a)}")
            if label == "heights":
                if dt != want:
                    raise ValueError(f"{name}: heights must be {want} for this precision, got {dt}")
                if tuple(a.shape[1:]) != lrq:
                    raise ValueError(f"{name}: heights must be [n][{lrq[0]}][{lrq[1]}][{lrq[2]}], "
                                     f"got {tuple(a.shape)}")
            else:
                if dt != np.dtype(np.float64):
                    raise ValueError(f"{name}: {label} must be float64, got {dt}")
                size = a.numel() if hasattr(a, "numel") else a.size
                if size < heights.shape[0]:
                    raise ValueError(f"{name}: {label} holds {size} values, need {heights.shape[0]}")

    def logpost(self, heights, loglik_out=None, logprior_out=None):
        self._check_batch("mt_logpost", heights, [("loglik_out", loglik_out), ("logprior_out", logprior_out)])
        n = heights.shape[0]
        self._ck("mt_logpost", self.lib.mt_logpost(self.h, n, _ptr(heights), _ptr(loglik_out),
                                                   _ptr(logprior_out)))

    def logpost_noalloc(self, heights, loglik_out, logprior_out=None):
        """mt_logpost_noalloc: device arrays only; allocates nothing."""
        self._check_batch("mt_logpost_noalloc", heights,
                          [("loglik_out", loglik_out), ("logprior_out", logprior_out)], device_only=True)
        n = heights.shape[0]
        self._ck("mt_logpost_noalloc", self.lib.mt_logpost_noalloc(
            self.h, n, _ptr(heights), _ptr(loglik_out), _ptr(logprior_out)))

    def ray_terms(self, heights, opacity_out=None, term_out=None):
        n = heights.shape[0]
        self._ck("mt_ray_terms", self.lib.mt_ray_terms(self.h, n, _ptr(heights),
                                                       _ptr(opacity_out), _ptr(term_out)))

    def grad(self, heights, grad_out, logpost_out=None):
        n = heights.shape[0]
        self._ck("mt_grad", self.lib.mt_grad(self.h, n, _ptr(heights), _ptr(grad_out),
                                             _ptr(logpost_out)))

    # -- chains
    def init_chains(self, heights0, seed):
        self._ck("mt_init_chains", self.lib.mt_init_chains(self.h, heights0.shape[0],
                                                           _ptr(heights0), seed))

    def run(self, kernel, step, n_super, n_within):
        self._ck("mt_run", self.lib.mt_run(self.h, kernel, float(step), n_super, n_within))

    def get_state(self, heights_out=None, loglik_out=None, logprior_out=None, accepts_out=None):
        stp = C.c_int64()
        self._ck("mt_get_state", self.lib.mt_get_state(self.h, _ptr(heights_out), _ptr(loglik_out),
                                                       _ptr(logprior_out), _ptr(accepts_out),
                                                       C.byref(stp)))
        return stp.value

    def run_traced(self, kernel, step, n_super, n_within, loglik_trace, logprior_trace,
                   accepts_trace=None):
        """mt_run one super-step at a time, reading each chain's log-likelihood
        and log-prior (and accept count) after every super-step into row k of
        the [n_super][C] traces (device or host; one mt_get_state, which
        synchronises, per super-step)."""
        for k in range(n_super):
            self.run(kernel, step, 1, n_within)
            self.get_state(None, loglik_trace[k], logprior_trace[k],
                           None if accepts_trace is None else accepts_trace[k])

    def get_last_step(self, proposal_out=None, loglik_out=None, logprior_out=None,
                      accepted_out=None, logu_out=None):
        self._ck("mt_get_last_step", self.lib.mt_get_last_step(
            self.h, _ptr(proposal_out), _ptr(loglik_out), _ptr(logprior_out), _ptr(accepted_out),
            _ptr(logu_out)))

    def set_state(self, heights, step):
        self._ck("mt_set_state", self.lib.mt_set_state(self.h, _ptr(heights), step))

    def sync(self, timeout_s=0.0):
        self._ck("mt_sync", self.lib.mt_sync(self.h, float(timeout_s)))

    def set_timing(self, on):
        self._ck("mt_set_timing", self.lib.mt_set_timing(self.h, int(on)))

    def get_work(self, reset=False):
        ev, tot = C.c_double(), C.c_double()
        self._ck("mt_get_work", self.lib.mt_get_work(self.h, C.byref(ev), C.byref(tot), int(reset)))
        return ev.value, tot.value

    def set_forward(self, kind, n_z=0, h_ref=None):
        h = None if h_ref is None else np.ascontiguousarray(h_ref, np.float64)
        self._ck("mt_set_forward", self.lib.mt_set_forward(self.h, int(kind), int(n_z), _ptr(h)))

    def set_hmc(self, n_leapfrog):
        self._ck("mt_set_hmc", self.lib.mt_set_hmc(self.h, int(n_leapfrog)))

    def set_adapt(self, target_accept, n_adapt):
        self._ck("mt_set_adapt", self.lib.mt_set_adapt(self.h, float(target_accept), int(n_adapt)))

    def get_adapt(self, eps_out=None, accept_prob_out=None):
        self._ck("mt_get_adapt", self.lib.mt_get_adapt(self.h, _ptr(eps_out), _ptr(accept_prob_out)))

    def set_nuts(self, max_depth):
        self._ck("mt_set_nuts", self.lib.mt_set_nuts(self.h, int(max_depth)))

    def set_metric_adapt(self, on, shrink=1e-3):
        self._ck("mt_set_metric_adapt", self.lib.mt_set_metric_adapt(self.h, int(on), float(shrink)))

    def get_metric(self, inv_metric_out):
        self._ck("mt_get_metric", self.lib.mt_get_metric(self.h, _ptr(inv_metric_out)))

    def set_prior(self, kind):
        self._ck("mt_set_prior", self.lib.mt_set_prior(self.h, int(kind)))

    def copula_heights(self, latent, heights_out):
        self._ck("mt_copula_heights", self.lib.mt_copula_heights(
            self.h, latent.shape[0], _ptr(latent), _ptr(heights_out)))

    def nested_rhat(self, draws, n_super, rhat_out=None):
        """mt_nested_rhat on draws [n_draws][n_chains][L][R][Q]; returns the maximum."""
        mx = C.c_double()
        self._ck("mt_nested_rhat", self.lib.mt_nested_rhat(
            self.h, draws.shape[0], draws.shape[1], _ptr(draws), int(n_super), _ptr(rhat_out),
            C.byref(mx)))
        return mx.value

    def interface_std(self, samples, n_z, std_out):
        """mt_interface_std on samples [n_samples][L][R][Q] into std_out [L][n_z][R][Q]."""
        self._ck("mt_interface_std", self.lib.mt_interface_std(
            self.h, samples.shape[0], _ptr(samples), int(n_z), _ptr(std_out)))

    def get_timing(self, kernel_id, reset=False):
        ms, n = C.c_double(), C.c_int64()
        self._ck("mt_get_timing", self.lib.mt_get_timing(self.h, kernel_id, C.byref(ms),
                                                         C.byref(n), int(reset)))
        return ms.value, n.value


def from_workload(prob: dict, precision=PREC_F32, device=0, stream=None, **over) -> Context:
    """Context for a problem dict from workloads.problem() (grid, sensors, pixels; no counts)."""
    kw = dict(n_grid=int(prob["G"]), gamma=float(prob["gamma"]), I0=float(prob["I0"]),
              atten=float(prob["Lambda"]), tau=float(prob["tau"]), car_r=float(prob["car_r"]),
              min_thick=float(prob["delta"]))
    kw.update(over)
    ctx = Context(device=device, precision=precision, stream=stream, **kw)
    ctx.set_grid(int(prob["L"]), int(prob["R"]), int(prob["Q"]), prob["box"], prob["rho"],
                 prob["mu"])
    ctx.set_sensors(prob["sensors"])
    ctx.set_pixels(prob["dirs"])
    return ctx


class Server:
    """mt_server: continuous batching of whole inversions on one GPU."""

    def __init__(self, device=0, hbm_budget_bytes=64 << 30, max_active=8):
        self.lib = load()
        h = C.c_void_p()
        st = self.lib.mt_server_create(C.byref(h), device, int(hbm_budget_bytes), int(max_active))
        if st != 0:
            raise MtError("mt_server_create", st, self.lib.mt_server_last_error(None).decode())
        self.h = h
        self._keep = {}

    def _ck(self, name, st):
        if st != 0:
            raise MtError(name, st, self.lib.mt_server_last_error(self.h).decode())

    def submit(self, prob, heights0, precision=PREC_F32, counts=None, data_seed=2, seed=4,
               kernel=KERNEL_RW, step=0.01, n_super=1, n_within=1, **cfg_over):
        """Queue one inversion of a workloads.problem() dict; returns its id."""
        cfg = dict(n_grid=int(prob["G"]), gamma=float(prob["gamma"]), I0=float(prob["I0"]),
                   atten=float(prob["Lambda"]), tau=float(prob["tau"]),
                   car_r=float(prob["car_r"]), min_thick=float(prob["delta"]))
        cfg.update(cfg_over)
        arrs = dict(box=np.ascontiguousarray(prob["box"], np.float64),
                    rho=np.ascontiguousarray(prob["rho"], np.float64),
                    mu=np.ascontiguousarray(prob["mu"], np.float64),
                    sensors=np.ascontiguousarray(prob["sensors"], np.float64),
                    dirs=np.ascontiguousarray(prob["dirs"], np.float64),
                    h0=np.ascontiguousarray(heights0, np.float64 if precision == PREC_F64 else np.float32))
        if counts is not None:
            arrs["counts"] = np.ascontiguousarray(counts, np.int32)
        else:
            arrs["h_true"] = np.ascontiguousarray(prob["H_true"], np.float64)
        r = Request()
        r.cfg = Config(precision, cfg["n_grid"], cfg["gamma"], cfg["I0"], cfg["atten"], cfg["tau"],
                       cfg["car_r"], cfg["min_thick"])
        r.n_layers, r.n_rows, r.n_cols = int(prob["L"]), int(prob["R"]), int(prob["Q"])
        r.box, r.unit_density, r.prior_mean = _ptr(arrs["box"]), _ptr(arrs["rho"]), _ptr(arrs["mu"])
        r.n_sensors, r.sensors = arrs["sensors"].shape[0], _ptr(arrs["sensors"])
        r.n_pixels, r.dirs = arrs["dirs"].shape[0], _ptr(arrs["dirs"])
        r.counts = _ptr(arrs.get("counts"))
        r.h_true = _ptr(arrs.get("h_true"))
        r.data_seed = data_seed
        r.n_chains, r.heights0 = arrs["h0"].shape[0], _ptr(arrs["h0"])
        r.seed, r.kernel, r.step = seed, kernel, float(step)
        r.n_super, r.n_within = int(n_super), int(n_within)
        rid = C.c_int64()
        self._ck("mt_server_submit", self.lib.mt_server_submit(self.h, C.byref(r), C.byref(rid)))
        self._keep[rid.value] = (prob, arrs["h0"].shape, arrs["h0"].dtype)
        return rid.value

    def wait(self, rid, timeout_s=0.0):
        prob, shape, dtype = self._keep[rid]
        H = np.zeros(shape, dtype)
        ll = np.zeros(shape[0])
        lp = np.zeros(shape[0])
        acc = np.zeros(shape[0], np.int64)
        info = RequestInfo()
        self._ck("mt_server_wait", self.lib.mt_server_wait(self.h, rid, float(timeout_s), _ptr(H),
                                                           _ptr(ll), _ptr(lp), _ptr(acc),
                                                           C.byref(info)))
        return dict(heights=H, loglik=ll, logprior=lp, accepts=acc,
                    info={k: getattr(info, k) for k, _ in RequestInfo._fields_})

    def cancel(self, rid):
        self._ck("mt_server_cancel", self.lib.mt_server_cancel(self.h, int(rid)))

    def stats(self):
        st = ServerStats()
        self._ck("mt_server_stats", self.lib.mt_server_stats(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.lib.mt_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
