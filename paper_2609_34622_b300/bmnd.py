"""Thin ctypes binding of the C ABI in include/bmnd.h.

Argument marshalling only: every step of the denoiser runs in the CUDA kernels
of ``libbmnd.so``.  Tensors are torch CUDA tensors (float32, contiguous); the
stream defaults to torch's current stream.  There is no CPU fallback: if the
library is missing, importing functions from here raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbmnd.so")
MAX_NDIM = 8

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = range(6)
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EUNSUPPORTED"}

SCHEDULES = {"generated": 0, "off": 1, "sparse": 2, "balanced": 3}
POWER_MODES = {"classic": 0, "noise_floor": 1, "variance_scaled": 2}
GROUP_TRANSFORMS = {"haar": 0, "dct": 1}
WEIGHT_MODELS = {"classic": 0, "variance": 1, "risk": 2}
WEIGHT_SCOPES = {"patch": 0, "group": 1}
MATCH_METRICS = {"ssd": 0, "poisson_deviance": 1, "pearson": 2, "anscombe_ssd": 3}
MATCH_POLICIES = {"fixed": 0, "reference_finite_count": 1, "candidate_standardized": 2}
MOMENT_NMAX = 4096
HT_RULES = {"hard": 0, "soft": 1}
WEIGHT_DOMAINS = {"coefficient": 0, "windowed_synthesis": 1}
SPATIAL_TRANSFORMS = {"dct": 0, "bior1.5": 1}


class BmndError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class bmnd_noise(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("sigma", ctypes.c_double), ("poisson_scale", ctypes.c_double)]


class bmnd_params(ctypes.Structure):
    _fields_ = [("lambda_ht", ctypes.c_double), ("gamma_ht", ctypes.c_double),
                ("gamma_wie", ctypes.c_double), ("tau_ht", ctypes.c_double),
                ("tau_wie", ctypes.c_double), ("s_v", ctypes.c_double),
                ("kaiser_beta", ctypes.c_double), ("shift_density", ctypes.c_double),
                ("passes", ctypes.c_int), ("schedule", ctypes.c_int), ("power_mode", ctypes.c_int),
                ("group_transform", ctypes.c_int), ("min_group", ctypes.c_int),
                ("weight_model", ctypes.c_int), ("weight_scope", ctypes.c_int),
                ("match_metric", ctypes.c_int), ("match_policy", ctypes.c_int),
                ("match_t", ctypes.c_double), ("beta_s", ctypes.c_double), ("kappa_s", ctypes.c_double),
                ("ht_rule", ctypes.c_int), ("weight_domain", ctypes.c_int), ("cov_planes", ctypes.c_int),
                ("spatial_transform", ctypes.c_int)]


class bmnd_job(ctypes.Structure):
    _fields_ = [("y", ctypes.c_void_p), ("out", ctypes.c_void_p), ("ndim", ctypes.c_int),
                ("shape", ctypes.c_int64 * MAX_NDIM), ("noise", bmnd_noise),
                ("patch", ctypes.c_int * MAX_NDIM), ("step", ctypes.c_int * MAX_NDIM),
                ("search", ctypes.c_int * MAX_NDIM), ("group_size", ctypes.c_int * 2),
                ("stages", ctypes.c_int), ("mass_conserve", ctypes.c_int)]


class bmnd_server_config(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int)]


class bmnd_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("voxels_per_s", ctypes.c_double), ("steps", ctypes.c_int64),
                ("mean_jobs_per_step", ctypes.c_double)]


EXPORTS = ["bmnd_default_params", "bmnd_create", "bmnd_destroy", "bmnd_last_error", "bmnd_denoise",
           "bmnd_denoise_ex", "bmnd_stage", "bmnd_schedule", "bmnd_match", "bmnd_denoise_batch",
           "bmnd_set_profiling", "bmnd_kernel_stats", "bmnd_denoise_noalloc", "bmnd_server_create",
           "bmnd_server_submit", "bmnd_server_wait", "bmnd_server_get_stats", "bmnd_server_destroy",
           "bmnd_graph_create", "bmnd_graph_launch", "bmnd_graph_destroy", "bmnd_autotune", "bmnd_autotune_batch",
           "bmnd_match_moments", "bmnd_coverage", "bmnd_decision_stats", "bmnd_denoise_batch_host",
           "bmnd_plan_info", "bmnd_fp32_fma_peak"]
KERNEL_KINDS = {"schedule": 0, "stage1": 1, "stage2": 2, "reduce": 3, "mc_sweep": 4, "match": 5}

_lib = None


def load(path: str = LIB_PATH):
    """Load libbmnd.so and declare the exported signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libbmnd.so not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    vp, i64p, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)
    P = ctypes.POINTER
    lib.bmnd_default_params.argtypes = [P(bmnd_params)]
    lib.bmnd_default_params.restype = None
    lib.bmnd_create.argtypes = [P(vp), ctypes.c_int, ctypes.c_size_t]
    lib.bmnd_destroy.argtypes = [vp]
    lib.bmnd_last_error.argtypes = [vp]
    lib.bmnd_last_error.restype = ctypes.c_char_p
    common = [vp, vp, ctypes.c_int, i64p, bmnd_noise, ip, ip, ip]
    lib.bmnd_denoise.argtypes = common + [ip, ctypes.c_int, ctypes.c_int, vp, vp]
    lib.bmnd_denoise_ex.argtypes = common + [ip, ctypes.c_int, ctypes.c_int, P(bmnd_params), vp, vp]
    lib.bmnd_stage.argtypes = [vp, vp, vp, ctypes.c_int, i64p, bmnd_noise, ip, ip, ip, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, P(bmnd_params), vp, vp]
    lib.bmnd_schedule.argtypes = [vp, ctypes.c_int, i64p, ip, ip, P(bmnd_params), vp, ctypes.c_int64,
                                  i64p, vp]
    lib.bmnd_match.argtypes = [vp, vp, ctypes.c_int, i64p, bmnd_noise, ip, ip, ip, ctypes.c_int,
                               ctypes.c_int, P(bmnd_params), vp, vp, vp, ctypes.c_int64, i64p, vp]
    lib.bmnd_denoise_batch.argtypes = [vp, ctypes.c_int, P(bmnd_job), P(bmnd_params), vp]
    lib.bmnd_autotune_batch.argtypes = [vp, ctypes.c_int, P(bmnd_job), P(bmnd_params), vp, ip]
    lib.bmnd_set_profiling.argtypes = [vp, ctypes.c_int]
    lib.bmnd_server_create.argtypes = [P(vp), ctypes.c_int, P(bmnd_server_config)]
    lib.bmnd_server_submit.argtypes = [vp, P(bmnd_job), i64p]
    lib.bmnd_server_wait.argtypes = [vp, ctypes.c_int64, ctypes.c_int, P(ctypes.c_double)]
    lib.bmnd_server_get_stats.argtypes = [vp, P(bmnd_server_stats)]
    lib.bmnd_server_destroy.argtypes = [vp]
    lib.bmnd_denoise_noalloc.argtypes = [vp, ctypes.c_int, i64p, bmnd_noise, ip, ip, ip, ip, ctypes.c_int,
                                         ctypes.c_int, vp, vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.bmnd_kernel_stats.argtypes = [vp, ctypes.c_int, ctypes.c_int, i64p, ctypes.POINTER(ctypes.c_double)]
    lib.bmnd_graph_create.argtypes = common + [ip, ctypes.c_int, ctypes.c_int, P(bmnd_params), vp, P(vp)]
    lib.bmnd_graph_launch.argtypes = [vp, vp]
    lib.bmnd_autotune.argtypes = common + [ip, ctypes.c_int, ctypes.c_int, P(bmnd_params), vp, vp, ip]
    lib.bmnd_graph_destroy.argtypes = [vp]
    lib.bmnd_decision_stats.argtypes = [vp, ctypes.c_int, P(ctypes.c_uint64)]
    lib.bmnd_denoise_batch_host.argtypes = [vp, ctypes.c_int, P(bmnd_job), P(bmnd_params), vp]
    lib.bmnd_plan_info.argtypes = [vp, ctypes.c_int, i64p, ip, ip, ip, ip, ctypes.c_int, ctypes.c_int,
                                   P(bmnd_params), i64p]
    lib.bmnd_fp32_fma_peak.argtypes = [ctypes.c_int, P(ctypes.c_double)]
    fp = ctypes.POINTER(ctypes.c_float)
    lib.bmnd_match_moments.argtypes = [ctypes.c_int, ctypes.c_int, fp, fp]
    lib.bmnd_coverage.argtypes = [vp, ctypes.c_int, i64p, ip, ip, P(bmnd_params), vp, i64p,
                                  ctypes.POINTER(ctypes.c_double), vp]
    for name in EXPORTS[1:]:
        if name != "bmnd_last_error":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def params(**kw) -> bmnd_params:
    """Profile with App. A defaults; keyword overrides by field name (string
    options accept the names used by the oracle)."""
    p = bmnd_params()
    load().bmnd_default_params(ctypes.byref(p))
    maps = dict(schedule=SCHEDULES, power_mode=POWER_MODES, group_transform=GROUP_TRANSFORMS,
                weight_model=WEIGHT_MODELS, weight_scope=WEIGHT_SCOPES, match_metric=MATCH_METRICS,
                match_policy=MATCH_POLICIES, ht_rule=HT_RULES, weight_domain=WEIGHT_DOMAINS,
                spatial_transform=SPATIAL_TRANSFORMS)
    for k, v in kw.items():
        if k in maps and isinstance(v, str):
            v = maps[k][v]
        setattr(p, k, v)
    return p


def bmnd_match_moments(metric, count: int = MOMENT_NMAX + 1):
    """Host-computed finite-count moment tables (mu, v), n = 0..count-1, of a
    Poisson matching distance (name or BMND_METRIC_* value), as float32."""
    import numpy as np
    m = MATCH_METRICS[metric] if isinstance(metric, str) else int(metric)
    mu = np.zeros(count, np.float32)
    v = np.zeros(count, np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    rc = load().bmnd_match_moments(m, int(count), mu.ctypes.data_as(fp), v.ctypes.data_as(fp))
    if rc != 0:
        raise BmndError(rc, "bmnd_match_moments(%r, %d)" % (metric, count))
    return mu, v


def noise(spec) -> bmnd_noise:
    kind, val = spec
    if kind == "gaussian":
        return bmnd_noise(0, float(val), 1.0)
    if kind == "poisson":
        return bmnd_noise(1, 0.0, float(val))
    raise ValueError(kind)


def _ints(vals, ctype=ctypes.c_int):
    return (ctype * max(len(vals), 1))(*[int(v) for v in vals])


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(t.data_ptr())


def _check_tensor(t, name):
    import torch
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError("%s must be a contiguous float32 CUDA tensor" % name)


class Context:
    """Owns a bmnd_ctx on one device."""

    def __init__(self, device: int = 0, scratch_budget: int = 0):
        lib = load()
        self._lib = lib
        self.handle = ctypes.c_void_p()
        st = lib.bmnd_create(ctypes.byref(self.handle), int(device), int(scratch_budget))
        if st != OK:
            raise BmndError(st, "bmnd_create failed")
        self.device = device

    def close(self):
        if self.handle:
            self._lib.bmnd_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != OK:
            raise BmndError(st, self._lib.bmnd_last_error(self.handle).decode())

    # -- entry points ------------------------------------------------------

    def bmnd_denoise(self, y, out, noise_spec, patch, step, search, group_size=(16, 32), stages=2,
                     mass_conserve=0, prm: bmnd_params | None = None, stream=None, raw_shape=None):
        """Both stages; y/out are CUDA tensors (or raw device pointers with raw_shape)."""
        shape = raw_shape if raw_shape is not None else tuple(y.shape)
        if raw_shape is None:
            _check_tensor(y, "y")
            _check_tensor(out, "out")
        D = len(shape)
        st = self._lib.bmnd_denoise_ex(self.handle, _ptr(y), D, _ints(shape, ctypes.c_int64), noise(noise_spec),
                                       _ints(patch), _ints(step), _ints(search), _ints(group_size), int(stages),
                                       int(mass_conserve), ctypes.byref(prm) if prm is not None else None,
                                       _ptr(out), _stream(stream))
        self._check(st)
        return out

    def bmnd_autotune(self, y, out, noise_spec, patch, step, search, group_size=(16, 32), stages=2,
                      mass_conserve=0, prm: bmnd_params | None = None, stream=None):
        """Time several tile cores on y and keep the fastest for this problem in
        the context; returns the chosen core (one entry per axis)."""
        _check_tensor(y, "y")
        _check_tensor(out, "out")
        shape = tuple(y.shape)
        core = (ctypes.c_int * len(shape))()
        st = self._lib.bmnd_autotune(self.handle, _ptr(y), len(shape), _ints(shape, ctypes.c_int64),
                                     noise(noise_spec), _ints(patch), _ints(step), _ints(search),
                                     _ints(group_size), int(stages), int(mass_conserve),
                                     ctypes.byref(prm) if prm is not None else None, _ptr(out), _stream(stream),
                                     core)
        self._check(st)
        return tuple(core)

    def bmnd_graph_create(self, y, out, noise_spec, patch, step, search, group_size=(16, 32), stages=2,
                          mass_conserve=0, prm: bmnd_params | None = None):
        """Record both stages on the bound CUDA tensors y / out as a replayable
        graph (refill y, then Graph.bmnd_graph_launch)."""
        _check_tensor(y, "y")
        _check_tensor(out, "out")
        shape = tuple(y.shape)
        h = ctypes.c_void_p()
        st = self._lib.bmnd_graph_create(self.handle, _ptr(y), len(shape), _ints(shape, ctypes.c_int64),
                                         noise(noise_spec), _ints(patch), _ints(step), _ints(search),
                                         _ints(group_size), int(stages), int(mass_conserve),
                                         ctypes.byref(prm) if prm is not None else None, _ptr(out), ctypes.byref(h))
        self._check(st)
        return Graph(self._lib, h, y, out)

    def bmnd_stage(self, y, pilot, out, noise_spec, patch, step, search, group_max, stage, mass_conserve=0,
                   prm: bmnd_params | None = None, stream=None):
        _check_tensor(y, "y")
        _check_tensor(out, "out")
        if pilot is not None:
            _check_tensor(pilot, "pilot")
        shape = tuple(y.shape)
        st = self._lib.bmnd_stage(self.handle, _ptr(y), _ptr(pilot), len(shape), _ints(shape, ctypes.c_int64),
                                  noise(noise_spec), _ints(patch), _ints(step), _ints(search), int(group_max),
                                  int(stage), int(mass_conserve), ctypes.byref(prm) if prm is not None else None,
                                  _ptr(out), _stream(stream))
        self._check(st)
        return out

    def bmnd_schedule(self, shape, patch, step, prm: bmnd_params | None = None, stream=None):
        import torch
        cap = 1
        for s in shape:
            cap *= int(s)
        origins = torch.empty(cap, dtype=torch.int64, device="cuda:%d" % self.device)
        n = ctypes.c_int64()
        st = self._lib.bmnd_schedule(self.handle, len(shape), _ints(shape, ctypes.c_int64), _ints(patch),
                                     _ints(step), ctypes.byref(prm) if prm is not None else None,
                                     _ptr(origins), cap, ctypes.byref(n), _stream(stream))
        self._check(st)
        return origins[: n.value]

    def bmnd_coverage(self, shape, patch, step, prm: bmnd_params | None = None, coverage=None, stream=None):
        """Reference coverage of a schedule (Sec. 9.3): fills the int32 CUDA
        tensor `coverage` (if given) with C(x) and returns (|R|, CV(C))."""
        if coverage is not None:
            import torch
            if not (coverage.is_cuda and coverage.dtype == torch.int32 and coverage.is_contiguous()
                    and coverage.numel() == int(np.prod(shape))):
                raise ValueError("coverage must be a contiguous int32 CUDA tensor of prod(shape) elements")
        n = ctypes.c_int64()
        cv = ctypes.c_double()
        st = self._lib.bmnd_coverage(self.handle, len(shape), _ints(shape, ctypes.c_int64), _ints(patch),
                                     _ints(step), ctypes.byref(prm) if prm is not None else None,
                                     _ptr(coverage) if coverage is not None else None, ctypes.byref(n),
                                     ctypes.byref(cv), _stream(stream))
        self._check(st)
        return n.value, cv.value

    def bmnd_match(self, guide, noise_spec, patch, step, search, group_max, stage,
                   prm: bmnd_params | None = None, stream=None):
        """Returns (origins [R], groups [R, group_max] with -1 padding, counts [R])."""
        import torch
        _check_tensor(guide, "guide")
        shape = tuple(guide.shape)
        cap = guide.numel()
        dev = guide.device
        origins = torch.empty(cap, dtype=torch.int64, device=dev)
        groups = torch.empty(cap * group_max, dtype=torch.int64, device=dev)
        counts = torch.empty(cap, dtype=torch.int32, device=dev)
        n = ctypes.c_int64()
        st = self._lib.bmnd_match(self.handle, _ptr(guide), len(shape), _ints(shape, ctypes.c_int64),
                                  noise(noise_spec), _ints(patch), _ints(step), _ints(search), int(group_max),
                                  int(stage), ctypes.byref(prm) if prm is not None else None, _ptr(origins),
                                  _ptr(groups), _ptr(counts), cap, ctypes.byref(n), _stream(stream))
        self._check(st)
        R = n.value
        return origins[:R], groups[: R * group_max].view(R, group_max), counts[:R]

    def _device_jobs(self, ys, outs, cfgs):
        n = len(ys)
        arr = (bmnd_job * n)()
        for i, (y, o, c) in enumerate(zip(ys, outs, cfgs)):
            _check_tensor(y, "y[%d]" % i)
            _check_tensor(o, "out[%d]" % i)
            j = arr[i]
            j.y, j.out = y.data_ptr(), o.data_ptr()
            j.ndim = y.dim()
            for a, s in enumerate(y.shape):
                j.shape[a] = int(s)
                j.patch[a] = int(c["patch"][a])
                j.step[a] = int(c["step"][a])
                j.search[a] = int(c["search"][a])
            j.noise = noise(c["noise"])
            gs = c.get("group_size", (16, 32))
            j.group_size[0], j.group_size[1] = int(gs[0]), int(gs[1])
            j.stages = int(c.get("stages", 2))
            j.mass_conserve = int(c.get("mass_conserve", 0))
        return arr

    def bmnd_denoise_batch(self, ys, outs, cfgs, prm: bmnd_params | None = None, stream=None):
        """ys/outs: lists of CUDA tensors; cfgs: list of dicts with keys noise,
        patch, step, search, group_size, stages, mass_conserve."""
        arr = self._device_jobs(ys, outs, cfgs)
        st = self._lib.bmnd_denoise_batch(self.handle, len(ys), arr, ctypes.byref(prm) if prm is not None else None,
                                          _stream(stream))
        self._check(st)
        return outs

    def bmnd_autotune_batch(self, ys, outs, cfgs, prm: bmnd_params | None = None, stream=None):
        """Time several tile cores on the whole batch (as bmnd_denoise_batch
        runs it) and keep the fastest for the first job's problem key;
        returns the chosen core of the first job."""
        arr = self._device_jobs(ys, outs, cfgs)
        core = (ctypes.c_int * ys[0].dim())()
        st = self._lib.bmnd_autotune_batch(self.handle, len(ys), arr,
                                           ctypes.byref(prm) if prm is not None else None, _stream(stream), core)
        self._check(st)
        return tuple(core)

    def bmnd_denoise_batch_host(self, ys, outs, cfgs, prm: bmnd_params | None = None, stream=None):
        """ys/outs: lists of C-contiguous float32 numpy arrays (host memory;
        pinned tensors' numpy views work too); returns when outs hold the
        results."""
        n = len(ys)
        arr = (bmnd_job * n)()
        for i, (y, o, c) in enumerate(zip(ys, outs, cfgs)):
            if not (y.dtype == np.float32 and o.dtype == np.float32 and y.flags.c_contiguous
                    and o.flags.c_contiguous and y.shape == o.shape):
                raise ValueError("y[%d] / out[%d] must be C-contiguous float32 arrays of one shape" % (i, i))
            j = arr[i]
            j.y, j.out = y.ctypes.data, o.ctypes.data
            j.ndim = y.ndim
            for a, sz in enumerate(y.shape):
                j.shape[a] = int(sz)
                j.patch[a] = int(c["patch"][a])
                j.step[a] = int(c["step"][a])
                j.search[a] = int(c["search"][a])
            j.noise = noise(c["noise"])
            gs = c.get("group_size", (16, 32))
            j.group_size[0], j.group_size[1] = int(gs[0]), int(gs[1])
            j.stages = int(c.get("stages", 2))
            j.mass_conserve = int(c.get("mass_conserve", 0))
        st = self._lib.bmnd_denoise_batch_host(self.handle, n, arr, ctypes.byref(prm) if prm is not None else None,
                                               _stream(stream))
        self._check(st)
        return outs

    def bmnd_plan_info(self, shape, patch, step, search, group_size=(16, 32), stages=2, mass_conserve=0,
                       prm: bmnd_params | None = None) -> dict:
        info = (ctypes.c_int64 * 8)()
        st = self._lib.bmnd_plan_info(self.handle, len(shape), _ints(shape, ctypes.c_int64), _ints(patch),
                                      _ints(step), _ints(search), _ints(group_size), int(stages), int(mass_conserve),
                                      ctypes.byref(prm) if prm is not None else None, info)
        self._check(st)
        D = int(info[3])
        return {"tiles": int(info[0]), "region": int(info[1]), "capacity": int(info[2]), "axes": D,
                "core": tuple(int(info[4 + a]) for a in range(D))}

    def bmnd_set_profiling(self, enable: bool):
        self._check(self._lib.bmnd_set_profiling(self.handle, int(bool(enable))))

    def bmnd_decision_stats(self, reset: bool = False) -> dict:
        """Counts of the decisions taken in double precision since the last reset:
        rescored candidates, windows scored entirely in double precision, and
        coefficients decided in double precision at the hard threshold."""
        c = (ctypes.c_uint64 * 3)()
        self._check(self._lib.bmnd_decision_stats(self.handle, int(reset), c))
        return {"rescored": int(c[0]), "full_windows": int(c[1]), "ht_coefficients": int(c[2])}

    def bmnd_kernel_stats(self, reset: bool = False) -> dict:
        """{kind: (launches, total_ms)} for every kernel kind; reset clears after reading."""
        res = {}
        kinds = list(KERNEL_KINDS.items())
        for i, (name, k) in enumerate(kinds):
            n = ctypes.c_int64()
            ms = ctypes.c_double()
            last = i == len(kinds) - 1
            self._check(self._lib.bmnd_kernel_stats(self.handle, k, int(reset and last), ctypes.byref(n),
                                                    ctypes.byref(ms)))
            res[name] = (n.value, ms.value)
        return res


class Graph:
    """A recorded bmnd_denoise_ex call on bound device tensors (bmnd_graph_*).
    Refill the bound input tensor, then launch again."""

    def __init__(self, lib, handle, y, out):
        self._lib, self.handle, self.y, self.out = lib, handle, y, out

    def bmnd_graph_launch(self, stream=None):
        st = self._lib.bmnd_graph_launch(self.handle, _stream(stream))
        if st != OK:
            raise BmndError(st, "graph launch failed")
        return self.out

    def close(self):
        if self.handle:
            self._lib.bmnd_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _fill_job(j, y_ptr, out_ptr, shape, c):
    j.y, j.out = y_ptr, out_ptr
    j.ndim = len(shape)
    for a, sz in enumerate(shape):
        j.shape[a] = int(sz)
        j.patch[a] = int(c["patch"][a])
        j.step[a] = int(c["step"][a])
        j.search[a] = int(c["search"][a])
    j.noise = noise(c["noise"])
    gs = c.get("group_size", (16, 32))
    j.group_size[0], j.group_size[1] = int(gs[0]), int(gs[1])
    j.stages = int(c.get("stages", 2))
    j.mass_conserve = int(c.get("mass_conserve", 0))


class Server:
    """Request server of the C ABI (bmnd_server_*): host numpy arrays in,
    host numpy arrays out; admission by device-memory budget and continuous
    batching happen in the library's worker thread."""

    def __init__(self, device: int = 0, mem_budget: int = 0, max_slots: int = 0):
        lib = load()
        self._lib = lib
        self.handle = ctypes.c_void_p()
        cfg = bmnd_server_config(int(mem_budget), int(max_slots))
        st = lib.bmnd_server_create(ctypes.byref(self.handle), int(device), ctypes.byref(cfg))
        if st != OK:
            raise BmndError(st, "bmnd_server_create failed")
        self._keep = {}

    def bmnd_server_submit(self, y: np.ndarray, cfg: dict, out: np.ndarray | None = None) -> int:
        y = np.ascontiguousarray(y, dtype=np.float32)
        if out is None:
            out = np.empty_like(y)
        j = bmnd_job()
        _fill_job(j, y.ctypes.data, out.ctypes.data, y.shape, cfg)
        t = ctypes.c_int64()
        st = self._lib.bmnd_server_submit(self.handle, ctypes.byref(j), ctypes.byref(t))
        if st != OK:
            raise BmndError(st, "submit rejected")
        self._keep[t.value] = (y, out)
        return t.value

    def bmnd_server_wait(self, ticket: int, timeout_ms: int = -1):
        """Returns (output array, latency in ms)."""
        lat = ctypes.c_double()
        st = self._lib.bmnd_server_wait(self.handle, int(ticket), int(timeout_ms), ctypes.byref(lat))
        y, out = self._keep.pop(ticket)
        if st != OK:
            raise BmndError(st, "job failed")
        return out, lat.value

    def bmnd_server_get_stats(self) -> dict:
        s = bmnd_server_stats()
        st = self._lib.bmnd_server_get_stats(self.handle, ctypes.byref(s))
        if st != OK:
            raise BmndError(st, "stats")
        return {f: getattr(s, f) for f, _ in bmnd_server_stats._fields_}

    def close(self):
        if self.handle:
            self._lib.bmnd_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bmnd_denoise_noalloc(y, out, noise_spec, patch, step, search, group_size=(16, 32), stages=2,
                         mass_conserve=0, stream=None):
    """Allocation-free denoising on the current device (no context): the
    library's scratch is a fixed 64 MiB device array; see include/bmnd.h."""
    _check_tensor(y, "y")
    _check_tensor(out, "out")
    shape = tuple(y.shape)
    err = ctypes.create_string_buffer(256)
    st = load().bmnd_denoise_noalloc(_ptr(y), len(shape), _ints(shape, ctypes.c_int64), noise(noise_spec),
                                     _ints(patch), _ints(step), _ints(search), _ints(group_size), int(stages),
                                     int(mass_conserve), _ptr(out), _stream(stream), err, len(err))
    if st != OK:
        raise BmndError(st, err.value.decode())
    return out


def denoise(y, cfg: dict, ctx: Context | None = None, prm=None, stream=None):
    """Convenience: allocate the output and denoise a CUDA tensor y."""
    import torch
    ctx = ctx or Context(y.device.index or 0)
    out = torch.empty_like(y)
    ctx.bmnd_denoise(y, out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                     cfg.get("group_size", (16, 32)), cfg.get("stages", 2), cfg.get("mass_conserve", 0),
                     prm, stream)
    return out


def exported_symbols(path: str = LIB_PATH) -> list[str]:
    """Names of include/bmnd.h entry points present in the library (no GPU needed)."""
    lib = ctypes.CDLL(path)
    return [n for n in EXPORTS if hasattr(lib, n)]


def bmnd_fp32_fma_peak(device: int = 0) -> float:
    """Measured FP32 FMA throughput of a device, TFLOP/s."""
    lib = load()
    v = ctypes.c_double()
    st = lib.bmnd_fp32_fma_peak(int(device), ctypes.byref(v))
    if st != OK:
        raise BmndError(st, "bmnd_fp32_fma_peak failed")
    return v.value
