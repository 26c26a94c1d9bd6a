"""FP64 CPU oracle for the BMND two-stage denoiser (ctypes binding).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path; the library it loads is compiled from ``bmnd_oracle.c`` in
this folder (see :func:`build`).

Every function follows the paper's definitions in double precision; the C file
names the definition, equation or proposition each step follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bmnd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
MAXD = 8


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (OpenMP, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"])
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("shape", ctypes.c_int64 * MAXD),
        ("patch", ctypes.c_int * MAXD),
        ("step", ctypes.c_int * MAXD),
        ("search", ctypes.c_int * MAXD),
        ("noise_kind", ctypes.c_int),
        ("sigma", ctypes.c_double),
        ("s_p", ctypes.c_double),
        ("group_max", ctypes.c_int * 2),
        ("stages", ctypes.c_int),
        ("mass_conserve", ctypes.c_int),
        ("lambda_ht", ctypes.c_double),
        ("gamma_ht", ctypes.c_double),
        ("gamma_wie", ctypes.c_double),
        ("tau_ht", ctypes.c_double),
        ("tau_wie", ctypes.c_double),
        ("s_v", ctypes.c_double),
        ("kaiser_beta", ctypes.c_double),
        ("shift_density", ctypes.c_double),
        ("passes", ctypes.c_int),
        ("schedule", ctypes.c_int),
        ("power_mode", ctypes.c_int),
        ("group_transform", ctypes.c_int),
        ("min_group", ctypes.c_int),
        ("weight_model", ctypes.c_int),
        ("weight_scope", ctypes.c_int),
        ("match_metric", ctypes.c_int),
        ("match_policy", ctypes.c_int),
        ("match_t", ctypes.c_double),
        ("beta_s", ctypes.c_double),
        ("kappa_s", ctypes.c_double),
        ("ht_rule", ctypes.c_int),
        ("weight_domain", ctypes.c_int),
        ("cov_planes", ctypes.c_int),
        ("spatial_ht", ctypes.c_int),
    ]


SCHEDULES = {"generated": 0, "off": 1, "sparse": 2, "balanced": 3}
POWER_MODES = {"classic": 0, "noise_floor": 1, "variance_scaled": 2}
GROUP_TRANSFORMS = {"haar": 0, "dct": 1}
WEIGHT_MODELS = {"classic": 0, "variance": 1, "risk": 2}
WEIGHT_SCOPES = {"patch": 0, "group": 1}
METRICS = {"ssd": 0, "poisson_deviance": 1, "pearson": 2, "anscombe_ssd": 3}
POLICIES = {"fixed": 0, "reference_finite_count": 1, "candidate_standardized": 2}
HT_RULES = {"hard": 0, "soft": 1}
WEIGHT_DOMAINS = {"coefficient": 0, "windowed_synthesis": 1}
SPATIAL_TRANSFORMS = {"dct": 0, "bior1.5": 1}
NMAX = 4096  # moment tables cover pooled counts 0..NMAX (larger counts use NMAX)

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, i64 = P(ctypes.c_double), P(ctypes.c_int64)
        _lib.or_schedule.argtypes = [P(_Params), i64, ctypes.c_int64]
        _lib.or_schedule.restype = ctypes.c_int64
        _lib.or_match_ref.argtypes = [P(_Params), d, ctypes.c_int, ctypes.c_int64, ctypes.c_int, i64, d]
        _lib.or_match_ref.restype = ctypes.c_int
        _lib.or_stage.argtypes = [P(_Params), d, d, ctypes.c_int, d, d, i64, P(ctypes.c_int), ctypes.c_int]
        _lib.or_stage.restype = ctypes.c_int64
        _lib.or_denoise.argtypes = [P(_Params), d, d, d]
        _lib.or_stage_points.argtypes = [P(_Params), d, d, ctypes.c_int, ctypes.c_int64, i64, d]
        _lib.or_filter_group.argtypes = [P(_Params), ctypes.c_int, d, d, ctypes.c_int, i64, d, d, d, d, d]
        _lib.or_group_transform.argtypes = [P(_Params), ctypes.c_int, ctypes.c_int, d, ctypes.c_int]
        _lib.or_bior15_matrix.argtypes = [ctypes.c_int, d]
        _lib.or_bior15_synthesis.argtypes = [ctypes.c_int, d]
        _lib.or_dct_matrix.argtypes = [ctypes.c_int, d]
        _lib.or_haar_matrix.argtypes = [ctypes.c_int, d]
        _lib.or_kaiser.argtypes = [ctypes.c_int, ctypes.c_double, d]
        _lib.or_bessel_i0.argtypes = [ctypes.c_double]
        _lib.or_bessel_i0.restype = ctypes.c_double
        _lib.or_num_threads.restype = ctypes.c_int
        _lib.or_coverage.argtypes = [P(_Params), P(ctypes.c_int32), d]
        _lib.or_coverage.restype = ctypes.c_int64
        _lib.or_anscombe.argtypes = [ctypes.c_double]
        _lib.or_anscombe.restype = ctypes.c_double
        _lib.or_phi.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        _lib.or_phi.restype = ctypes.c_double
        _lib.or_moments.argtypes = [ctypes.c_int, ctypes.c_int, d, d]
        _lib.or_raw_count_of.argtypes = [P(_Params), ctypes.c_double]
        _lib.or_raw_count_of.restype = ctypes.c_double
        _lib.or_exact_sum.argtypes = [d, ctypes.c_int64]
        _lib.or_exact_sum.restype = ctypes.c_double
        _lib.or_moment_table_f32.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_float), P(ctypes.c_float)]
    return _lib


def params(shape, patch, step, search, noise=("poisson", 1.0), group_size=(16, 32), stages=2,
           mass_conserve=0, **kw) -> _Params:
    """Build the parameter block.  Defaults are the standard configuration of
    App. A (generated schedule with shift density 2 and 2 passes, lambda_HT = 3,
    gamma_HT = 3, s_v = 0.4, Kaiser beta = 2, minimum group 2, variance
    weights in patch scope, Haar along the group axis, DCT on the patch axes)."""
    D = len(shape)
    if D > MAXD:
        raise ValueError("oracle supports up to %d axes" % MAXD)
    p = _Params()
    p.ndim = D
    for a in range(D):
        p.shape[a] = int(shape[a])
        p.patch[a] = int(patch[a])
        p.step[a] = int(step[a])
        p.search[a] = int(search[a])
    kind, val = noise
    if kind == "gaussian":
        p.noise_kind, p.sigma, p.s_p = 0, float(val), 1.0
    elif kind == "poisson":
        p.noise_kind, p.sigma, p.s_p = 1, 0.0, float(val)
    else:
        raise ValueError(kind)
    p.group_max[0], p.group_max[1] = int(group_size[0]), int(group_size[1])
    p.stages = int(stages)
    p.mass_conserve = int(mass_conserve)
    p.lambda_ht = kw.pop("lambda_ht", 3.0)
    p.gamma_ht = kw.pop("gamma_ht", 3.0)
    p.gamma_wie = kw.pop("gamma_wie", 0.0)
    p.tau_ht = kw.pop("tau_ht", 0.0)
    p.tau_wie = kw.pop("tau_wie", 0.0)
    p.s_v = kw.pop("s_v", 0.4)
    p.kaiser_beta = kw.pop("kaiser_beta", 2.0)
    p.shift_density = kw.pop("shift_density", 2.0)
    p.passes = kw.pop("passes", 2)
    p.schedule = SCHEDULES[kw.pop("schedule", "generated")]
    p.power_mode = POWER_MODES[kw.pop("power_mode", "classic")]
    p.group_transform = GROUP_TRANSFORMS[kw.pop("group_transform", "haar")]
    p.min_group = kw.pop("min_group", 2)
    p.weight_model = WEIGHT_MODELS[kw.pop("weight_model", "variance")]
    p.weight_scope = WEIGHT_SCOPES[kw.pop("weight_scope", "patch")]
    # stage-1 matching distance and acceptance policy (Secs. 4.2-4.3); the
    # defaults are App. A's SSD, beta_s = 0.1 and kappa_s = 1 (Sec. 9.4), t = 3
    p.match_metric = METRICS[kw.pop("match_metric", "ssd")]
    p.match_policy = POLICIES[kw.pop("match_policy", "fixed")]
    p.match_t = kw.pop("match_t", 3.0)
    p.beta_s = kw.pop("beta_s", 0.1)
    p.kappa_s = kw.pop("kappa_s", 1.0)
    # stage-1 thresholding rule (Def. "Coefficient thresholding"; hard in App. A)
    p.ht_rule = HT_RULES[kw.pop("ht_rule", "hard")]
    # aggregation-weight domain (Sec. 7; coefficient domain in App. A)
    p.weight_domain = WEIGHT_DOMAINS[kw.pop("weight_domain", "coefficient")]
    # leading group-axis planes with the shared-source variance (Sec. 5;
    # App. A lists 4, the CUDA path implements 0 = the diagonal model)
    p.cov_planes = int(kw.pop("cov_planes", 0))
    # spatial transform of the hard-threshold stage (App. A: bior1.5; the
    # DCT is the default here; stage 2 always uses the DCT)
    p.spatial_ht = SPATIAL_TRANSFORMS[kw.pop("spatial_transform", "dct")]
    if kw:
        raise TypeError("unknown oracle parameters: %s" % sorted(kw))
    return p


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def schedule(p: _Params) -> np.ndarray:
    lib = _load()
    n = lib.or_schedule(ctypes.byref(p), None, 0)
    out = np.empty(n, np.int64)
    lib.or_schedule(ctypes.byref(p), _iptr(out), n)
    return out


def coverage(p: _Params):
    """Reference coverage C(x) (Sec. 9.3) of the schedule p selects: returns
    (C as an int32 array of the shape, number of references, CV(C))."""
    shape = tuple(p.shape[a] for a in range(p.ndim))
    cov = np.zeros(shape, np.int32)
    cv = ctypes.c_double()
    n = _load().or_coverage(ctypes.byref(p), cov.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(cv))
    return cov, int(n), cv.value


def match_ref(p: _Params, guide, stage: int, ref_lin: int):
    lib = _load()
    g = _f64(guide).ravel()
    M = p.group_max[stage - 1]
    mem = np.empty(64, np.int64)
    sc = np.empty(64, np.float64)
    n = lib.or_match_ref(ctypes.byref(p), _dptr(g), stage, int(ref_lin), M, _iptr(mem), _dptr(sc))
    return mem[:n].copy(), sc[:n].copy()


def stage(p: _Params, y, pilot, stage: int, want_den=False, want_groups=False):
    lib = _load()
    yy = _f64(y).ravel()
    pl = _f64(pilot).ravel() if pilot is not None else None
    out = np.empty_like(yy)
    den = np.empty_like(yy) if want_den else None
    R = lib.or_schedule(ctypes.byref(p), None, 0)
    gmax = p.group_max[stage - 1]
    groups = np.empty((R, gmax), np.int64) if want_groups else None
    counts = np.empty(R, np.int32) if want_groups else None
    lib.or_stage(ctypes.byref(p), _dptr(yy), _dptr(pl) if pl is not None else None, stage, _dptr(out),
                 _dptr(den) if den is not None else None,
                 _iptr(groups) if groups is not None else None,
                 counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if counts is not None else None,
                 gmax)
    shape = np.asarray(y).shape
    res = [out.reshape(shape)]
    if want_den:
        res.append(den.reshape(shape))
    if want_groups:
        res += [groups, counts]
    return res[0] if len(res) == 1 else tuple(res)


def denoise(p: _Params, y):
    """Both stages; returns (estimate, stage-1 pilot)."""
    lib = _load()
    yy = _f64(y).ravel()
    out = np.empty_like(yy)
    pilot = np.empty_like(yy)
    lib.or_denoise(ctypes.byref(p), _dptr(yy), _dptr(out), _dptr(pilot))
    shape = np.asarray(y).shape
    return out.reshape(shape), pilot.reshape(shape)


def stage_points(p: _Params, y, pilot, stage: int, points_lin):
    lib = _load()
    yy = _f64(y).ravel()
    pl = _f64(pilot).ravel() if pilot is not None else None
    pts = np.ascontiguousarray(points_lin, dtype=np.int64)
    out = np.empty(len(pts), np.float64)
    lib.or_stage_points(ctypes.byref(p), _dptr(yy), _dptr(pl) if pl is not None else None, stage,
                        len(pts), _iptr(pts), _dptr(out))
    return out


def filter_group(p: _Params, stage: int, y, pilot, members):
    lib = _load()
    yy = _f64(y).ravel()
    pl = _f64(pilot).ravel() if pilot is not None else None
    mem = np.ascontiguousarray(members, dtype=np.int64)
    n = len(mem)
    P = int(np.prod([p.patch[a] for a in range(p.ndim)]))
    Y, var, C, pt = (np.empty(n * P) for _ in range(4))
    w = np.empty(n)
    lib.or_filter_group(ctypes.byref(p), stage, _dptr(yy), _dptr(pl) if pl is not None else None, n,
                        _iptr(mem), _dptr(Y), _dptr(var), _dptr(C), _dptr(pt), _dptr(w))
    sh = (n, P)
    return dict(Y=Y.reshape(sh), var=var.reshape(sh), C=C.reshape(sh), p=pt.reshape(sh), w=w)


def group_transform(p: _Params, x, mode: int = 0, stage: int = 1):
    """The group transform of stage `stage` on a group tensor x of shape
    (count, *patch): mode 0: T x, 1: U x with U = T^{-1} the synthesis,
    2: (T.^2) x, 3: U^T x."""
    lib = _load()
    a = _f64(x).copy()
    lib.or_group_transform(ctypes.byref(p), stage, a.shape[0], _dptr(a), mode)
    return a


def bior15_matrix(n: int) -> np.ndarray:
    """bior1.5 analysis matrix of a periodic length-n axis (n a power of
    two), full depth, coefficients coarsest first."""
    a = np.empty(n * n)
    _load().or_bior15_matrix(n, _dptr(a))
    return a.reshape(n, n)


def bior15_synthesis(n: int) -> np.ndarray:
    """bior1.5 synthesis matrix (columns: patches synthesized from unit
    coefficients), built from the synthesis filters."""
    a = np.empty(n * n)
    _load().or_bior15_synthesis(n, _dptr(a))
    return a.reshape(n, n)


def dct_matrix(n: int) -> np.ndarray:
    a = np.empty(n * n)
    _load().or_dct_matrix(n, _dptr(a))
    return a.reshape(n, n)


def haar_matrix(n: int) -> np.ndarray:
    a = np.empty(n * n)
    _load().or_haar_matrix(n, _dptr(a))
    return a.reshape(n, n)


def kaiser(n: int, beta: float) -> np.ndarray:
    a = np.empty(n)
    _load().or_kaiser(n, beta, _dptr(a))
    return a


def bessel_i0(x: float) -> float:
    return _load().or_bessel_i0(x)


def num_threads() -> int:
    return _load().or_num_threads()


# ---- Poisson-aware matching (Secs. 4.2-4.3) ----

def anscombe(n: float) -> float:
    """A(n) = 2 sqrt(n + 3/8)."""
    return _load().or_anscombe(float(n))


def phi(metric: str, r: float, c: float) -> float:
    """FP64 per-entry contribution phi_m(r, c) of Eq. (varphi)."""
    return _load().or_phi(METRICS[metric], float(r), float(c))


def moments(metric: str, n: int):
    """FP64 finite-count moments (mu_m(n), v_m(n)) (Prop. "Universal finite-count moments")."""
    mu, v = ctypes.c_double(), ctypes.c_double()
    _load().or_moments(METRICS[metric], int(n), ctypes.byref(mu), ctypes.byref(v))
    return mu.value, v.value


def moment_table_f32(metric: str, count: int = NMAX + 1):
    """The FP64 moments (mu, v) for n = 0..count-1 rounded to float32."""
    mu = np.zeros(count, np.float32)
    v = np.zeros(count, np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    _load().or_moment_table_f32(METRICS[metric], int(count), mu.ctypes.data_as(fp), v.ctypes.data_as(fp))
    return mu, v


def exact_sum(x) -> float:
    """The oracle's exact summation (Shewchuk expansions, rounded once)."""
    a = _f64(x).ravel()
    return _load().or_exact_sum(_dptr(a), len(a))


def raw_count(p: _Params, v: float) -> float:
    """Eq. (raw-counts) with the integer reading: the nearest integer when
    y / s_P lies within a relative 2^-20 of it, else [y / s_P]_+."""
    return _load().or_raw_count_of(ctypes.byref(p), float(v))
