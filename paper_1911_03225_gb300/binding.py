"""Thin ctypes binding of the C ABI in ``include/fdm.h`` (argument marshalling only).

Every step of the FDM time loop runs in the CUDA library ``libfdm_gb300.so``; this module
converts numpy arrays and parameters, and turns status codes into exceptions.  There is no
CPU fallback: if the library is missing or cannot be loaded, ``load()`` raises.
"""
import ctypes as C
import os
import warnings
from dataclasses import dataclass, asdict, field
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfdm_gb300.so")

FDM_OK = 0
FDM_ERR_INVALID_ARG = 1
FDM_ERR_OOM = 2
FDM_ERR_NET_BURGERS = 3
FDM_WARN_NOT_DIV_FREE = 4
FDM_ERR_NONFINITE = 5
FDM_ERR_TIMEOUT = 6
FDM_ERR_DEVICE = 7
FDM_ERR_STATE = 8
FDM_ERR_TOO_LARGE = 9

V_PRESCRIBED, V_STRESS = 0, 1
LOAD_STRESS, LOAD_STRAIN_RAMP, LOAD_ZERO_MEAN_STRESS, LOAD_STRAIN_RATE = 0, 1, 2, 3
FP64, MIXED, DF64 = 0, 1, 2
# stress components in Voigt order (FDM_S11 .. FDM_S12)
STRESS_COMPONENTS = ("11", "22", "33", "23", "13", "12")
T_MIDPOINT, T_LITERAL = 0, 1

FIELD_UP13, FIELD_ALPHA11, FIELD_ALPHA12, FIELD_TAU13, FIELD_V1, FIELD_V2 = 1, 2, 4, 8, 16, 32
FIELDS = {"up13": FIELD_UP13, "alpha11": FIELD_ALPHA11, "alpha12": FIELD_ALPHA12,
          "tau13": FIELD_TAU13, "v1": FIELD_V1, "v2": FIELD_V2}

# every entry point declared in include/fdm.h
EXPORTS = ["fdm_default_params", "fdm_device_bytes", "fdm_create", "fdm_set_density",
           "fdm_set_plastic_distortion", "fdm_set_clock", "fdm_static_solve", "fdm_step",
           "fdm_read_fields", "fdm_get_info", "fdm_kernels_per_step", "fdm_destroy",
           "fdm_status_str", "fdm_enqueue_steps", "fdm_enqueue_phase", "fdm_sync",
           "fdm_static_solve_noalloc", "fdm_batch_create", "fdm_batch_device_bytes",
           "fdm_batch_set_plastic_distortion", "fdm_batch_set_budget", "fdm_batch_enqueue_steps",
           "fdm_batch_sync", "fdm_batch_get_info", "fdm_batch_read_fields", "fdm_batch_launches_per_step",
           "fdm_batch_destroy", "fdm_get_launch_config", "fdm_batch_get_launch_config",
           "fdm_set_launch_config", "fdm_launch_candidates", "fdm_set_mobility_field", "fdm_set_loading",
           "fdm_read_stress13_planes", "fdm_read_stress_planes", "fdm_batch_sync_status",
           "fdm_debug_fail_allocation", "fdm_static_solve_heterogeneous", "fdm_set_shear_modulus_field",
           "fdm_measure_arith_rate", "fdm_batch_enqueue_steps_persistent", "fdm_debug_barrier",
           "fdm_debug_fp64_math",
           "fdm_static_solve_heterogeneous_layer", "fdm_equilibrate"]


class CParams(C.Structure):
    _fields_ = [("n1", C.c_int32), ("n2", C.c_int32), ("nz", C.c_int32), ("nh", C.c_int32),
                ("dx", C.c_double), ("E", C.c_double), ("nu", C.c_double),
                ("velocity_mode", C.c_int32),
                ("v0", C.c_double), ("mobility", C.c_double), ("tau_y", C.c_double),
                ("beta", C.c_double), ("theta", C.c_double), ("cfl", C.c_double),
                ("dt_max", C.c_double),
                ("loading_mode", C.c_int32),
                ("sigma_bar13", C.c_double), ("eps_bar13_0", C.c_double),
                ("eps_bar13_rate", C.c_double),
                ("time_level", C.c_int32), ("precision", C.c_int32), ("autotune", C.c_int32)]


class CLaunchConfig(C.Structure):
    _fields_ = [("rows_per_block", C.c_int32), ("cols_per_block", C.c_int32),
                ("stencil_block_rows", C.c_int32), ("stencil_nodes", C.c_int32),
                ("stencil_min_blocks", C.c_int32), ("tuned", C.c_int32),
                ("kernel_us", C.c_double * 4)]


def _launch_config(c: CLaunchConfig) -> dict:
    d = {f: getattr(c, f) for f, _ in CLaunchConfig._fields_ if f != "kernel_us"}
    d["kernel_us"] = [float(x) for x in c.kernel_us]
    return d


class CStepInfo(C.Structure):
    _fields_ = [("step", C.c_int64), ("t", C.c_double), ("dt", C.c_double),
                ("max_abs_v0", C.c_double), ("mean_up13", C.c_double),
                ("eps_bar13", C.c_double), ("sigma_bar13", C.c_double),
                ("sum_a12_pos", C.c_double), ("sum_a12_neg", C.c_double),
                ("sum_a11_pos", C.c_double), ("sum_a11_neg", C.c_double),
                ("sum_abs_alpha", C.c_double), ("status", C.c_int32)]


@dataclass
class Params:
    """Mirror of ``fdm_params`` (dimensionless units of Sec. 3.2.1)."""
    n1: int
    n2: int
    nz: int = 0
    nh: int = 4
    dx: float = 1.0
    E: float = 1.0
    nu: float = 0.3
    velocity_mode: int = V_PRESCRIBED
    v0: float = 1.0
    mobility: float = 1.0
    tau_y: float = 0.0
    beta: float = 1.0
    theta: float = 1.0
    cfl: float = 0.5
    dt_max: float = 0.0
    loading_mode: int = LOAD_STRESS
    sigma_bar13: float = 0.0
    eps_bar13_0: float = 0.0
    eps_bar13_rate: float = 0.0
    time_level: int = T_MIDPOINT
    precision: int = FP64
    autotune: int = 1

    def to_c(self) -> CParams:
        return CParams(**asdict(self))


@dataclass
class StepInfo:
    step: int
    t: float
    dt: float
    max_abs_v0: float
    mean_up13: float
    eps_bar13: float
    sigma_bar13: float
    sum_a12_pos: float
    sum_a12_neg: float
    sum_a11_pos: float
    sum_a11_neg: float
    sum_abs_alpha: float
    status: int


class FDMError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, status_str(status), status))


_lib = None


def load():
    """Load the CUDA library (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libfdm_gb300.so is not built; run paper_1911_03225_gb300/build.py "
                          "(or __graft_entry__.build())")
    lib = C.CDLL(LIB_PATH)
    d = C.POINTER(C.c_double)
    H = C.c_void_p
    lib.fdm_default_params.argtypes = [C.POINTER(CParams)]
    lib.fdm_default_params.restype = None
    lib.fdm_device_bytes.argtypes = [C.POINTER(CParams)]
    lib.fdm_device_bytes.restype = C.c_size_t
    lib.fdm_create.argtypes = [C.POINTER(CParams), C.c_void_p, C.POINTER(H)]
    lib.fdm_set_density.argtypes = [H, d, d, C.c_double, d]
    lib.fdm_set_plastic_distortion.argtypes = [H, d]
    lib.fdm_set_clock.argtypes = [H, C.c_int64, C.c_double]
    lib.fdm_static_solve.argtypes = [H]
    lib.fdm_step.argtypes = [H, C.c_int32, C.POINTER(CStepInfo)]
    lib.fdm_read_fields.argtypes = [H, C.c_uint32, d, d, d, d, d, d]
    lib.fdm_enqueue_steps.argtypes = [H, C.c_int32]
    lib.fdm_enqueue_phase.argtypes = [H, C.c_int32]
    lib.fdm_sync.argtypes = [H]
    lib.fdm_static_solve_noalloc.argtypes = [C.POINTER(CParams), C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.fdm_static_solve_noalloc.restype = C.c_int
    lib.fdm_batch_enqueue_steps_persistent.argtypes = [C.c_void_p, C.c_int32]
    lib.fdm_batch_enqueue_steps_persistent.restype = C.c_int
    lib.fdm_debug_barrier.argtypes = [C.c_int32, C.c_double]
    lib.fdm_debug_barrier.restype = None
    lib.fdm_measure_arith_rate.argtypes = [C.c_int32, C.c_void_p, d]
    lib.fdm_measure_arith_rate.restype = C.c_int
    lib.fdm_debug_fp64_math.argtypes = [C.c_int32, d, d, C.c_int64]
    lib.fdm_debug_fp64_math.restype = C.c_int
    PP = C.POINTER(CParams)
    lib.fdm_batch_create.argtypes = [C.c_int32, PP, C.c_void_p, C.POINTER(H)]
    lib.fdm_batch_device_bytes.argtypes = [C.c_int32, PP]
    lib.fdm_batch_device_bytes.restype = C.c_size_t
    lib.fdm_batch_set_plastic_distortion.argtypes = [H, C.c_int32, d]
    lib.fdm_batch_set_budget.argtypes = [H, C.c_int32, C.c_int64]
    lib.fdm_batch_enqueue_steps.argtypes = [H, C.c_int32]
    lib.fdm_batch_sync.argtypes = [H, C.POINTER(C.c_int64)]
    lib.fdm_batch_sync_status.argtypes = [H, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]
    lib.fdm_batch_sync_status.restype = C.c_int
    lib.fdm_static_solve_heterogeneous.argtypes = [H, d, C.c_double, C.c_int32, d, d, C.POINTER(C.c_int32),
                                                   C.POINTER(C.c_double)]
    lib.fdm_static_solve_heterogeneous.restype = C.c_int
    lib.fdm_static_solve_heterogeneous_layer.argtypes = [H, d, C.c_double, C.c_int32, d, C.c_int32,
                                                         C.POINTER(C.c_int32), d, C.POINTER(C.c_int32),
                                                         C.POINTER(C.c_double)]
    lib.fdm_static_solve_heterogeneous_layer.restype = C.c_int
    lib.fdm_equilibrate.argtypes = [H, C.c_double, C.c_int32, C.c_int64, C.POINTER(C.c_int64),
                                    C.POINTER(C.c_double)]
    lib.fdm_equilibrate.restype = C.c_int
    lib.fdm_set_shear_modulus_field.argtypes = [H, d, C.c_double, C.c_int32]
    lib.fdm_set_shear_modulus_field.restype = C.c_int
    lib.fdm_debug_fail_allocation.argtypes = [C.c_int32]
    lib.fdm_debug_fail_allocation.restype = None
    lib.fdm_batch_get_info.argtypes = [H, C.c_int32, C.POINTER(CStepInfo)]
    lib.fdm_batch_read_fields.argtypes = [H, C.c_int32, C.c_uint32, d, d]
    lib.fdm_batch_launches_per_step.argtypes = [H]
    lib.fdm_batch_launches_per_step.restype = C.c_int32
    lib.fdm_batch_destroy.argtypes = [H]
    lib.fdm_batch_destroy.restype = None
    lib.fdm_get_launch_config.argtypes = [H, C.POINTER(CLaunchConfig)]
    lib.fdm_get_launch_config.restype = C.c_int
    lib.fdm_batch_get_launch_config.argtypes = [H, C.c_int32, C.POINTER(CLaunchConfig)]
    lib.fdm_batch_get_launch_config.restype = C.c_int
    lib.fdm_set_launch_config.argtypes = [H, C.POINTER(CLaunchConfig)]
    lib.fdm_set_launch_config.restype = C.c_int
    lib.fdm_set_mobility_field.argtypes = [H, d]
    lib.fdm_set_mobility_field.restype = C.c_int
    lib.fdm_set_loading.argtypes = [H, C.c_int32, C.c_double, C.c_double, C.c_double]
    lib.fdm_set_loading.restype = C.c_int
    lib.fdm_read_stress13_planes.argtypes = [H, C.c_int32, C.POINTER(C.c_int32), d]
    lib.fdm_read_stress13_planes.restype = C.c_int
    lib.fdm_read_stress_planes.argtypes = [H, C.c_int32, C.c_int32, C.POINTER(C.c_int32), d]
    lib.fdm_read_stress_planes.restype = C.c_int
    lib.fdm_launch_candidates.argtypes = [C.POINTER(CParams), C.POINTER(CLaunchConfig), C.c_int32]
    lib.fdm_launch_candidates.restype = C.c_int32
    for name in ("fdm_batch_create", "fdm_batch_set_plastic_distortion", "fdm_batch_set_budget",
                 "fdm_batch_enqueue_steps", "fdm_batch_sync", "fdm_batch_get_info", "fdm_batch_read_fields"):
        getattr(lib, name).restype = C.c_int
    lib.fdm_get_info.argtypes = [H, C.POINTER(CStepInfo)]
    lib.fdm_kernels_per_step.argtypes = [H]
    lib.fdm_kernels_per_step.restype = C.c_int32
    lib.fdm_destroy.argtypes = [H]
    lib.fdm_destroy.restype = None
    lib.fdm_status_str.argtypes = [C.c_int]
    lib.fdm_status_str.restype = C.c_char_p
    for name in ("fdm_create", "fdm_set_density", "fdm_set_plastic_distortion", "fdm_set_clock",
                 "fdm_static_solve", "fdm_step", "fdm_read_fields", "fdm_get_info",
                 "fdm_enqueue_steps", "fdm_enqueue_phase", "fdm_sync"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def debug_barrier(extra_arrivals: int, limit_seconds: float = 0.0):
    """Test hook: barriers of the persistent batched step wait for extra_arrivals more blocks
    than the grid holds (> 0: none completes) and give up after limit_seconds (<= 0: 1 s)."""
    load().fdm_debug_barrier(int(extra_arrivals), float(limit_seconds))


def debug_fail_allocation(n: int):
    """Test hook: the n-th device or pinned allocation from now on fails once (n < 0: off)."""
    load().fdm_debug_fail_allocation(int(n))


def status_str(s: int) -> str:
    return load().fdm_status_str(int(s)).decode()


def default_params(n1: int, n2: int) -> Params:
    cp = CParams()
    load().fdm_default_params(C.byref(cp))
    d = {f: getattr(cp, f) for f, _ in CParams._fields_}
    d["n1"], d["n2"] = n1, n2
    return Params(**d)


def device_bytes(p: Params) -> int:
    return int(load().fdm_device_bytes(C.byref(p.to_c())))


def debug_fp64_math(op: int, x) -> np.ndarray:
    """1/sqrt(x) (op 0) or 1/x (op 1) elementwise as the FP64 stencil computes them (a test
    hook)."""
    xs = np.ascontiguousarray(x, dtype=np.float64).ravel()
    y = np.empty_like(xs)
    _check(load().fdm_debug_fp64_math(int(op), _dptr(xs), _dptr(y), int(xs.size)), "fdm_debug_fp64_math")
    return y


def measure_arith_rate(precision: int, stream: Optional[int] = None) -> float:
    """Measured multiply-add rate of the current GPU in GFLOP/s (multiply-add = 2 flops):
    FP64, FP32 (``MIXED``) or double-word (``DF64``, two FP64-equivalent flops per
    double-word multiply-add).  About 0.2 s of GPU time."""
    out = C.c_double(0.0)
    _check(load().fdm_measure_arith_rate(int(precision), C.c_void_p(stream or 0), C.byref(out)),
           "fdm_measure_arith_rate")
    return float(out.value)


def static_solve_noalloc(params: Params, sigma_bar13: float, d_up13: int, d_tau13: int,
                        stream: Optional[int] = None):
    """tau13 for a caller-owned device array, without any device allocation.

    For callers that cannot allocate device memory (their HBM is already committed, or only
    their own pool may allocate).  ``d_up13`` and ``d_tau13`` are device addresses of
    [n2][n1] float64 arrays (e.g. ``tensor.data_ptr()``); work is enqueued on ``stream``.
    The library's fixed scratch limits the grid to n1, n2 <= 256; overlapping calls race.
    """
    _check(load().fdm_static_solve_noalloc(C.byref(params.to_c()), float(sigma_bar13), C.c_void_p(d_up13),
                                            C.c_void_p(d_tau13), C.c_void_p(stream or 0)),
           "fdm_static_solve_noalloc")


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _field(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        raise ValueError("expected array of shape %s, got %s" % (shape, a.shape))
    return a


def _check(st, what):
    if st != FDM_OK:
        raise FDMError(st, what)


class FDM:
    """One FDM layer simulation resident on the GPU (handle of the C ABI)."""

    def __init__(self, params: Params, stream: Optional[int] = None):
        self.lib = load()
        self.params = params
        self.shape = (params.n2, params.n1)
        h = C.c_void_p()
        _check(self.lib.fdm_create(C.byref(params.to_c()), C.c_void_p(stream or 0), C.byref(h)), "fdm_create")
        self.h = h

    # -- state
    def set_density(self, alpha11, alpha12, mean_up13: float = 0.0) -> float:
        a11, a12 = _field(alpha11, self.shape), _field(alpha12, self.shape)
        res = C.c_double(0.0)
        st = self.lib.fdm_set_density(self.h, _dptr(a11), _dptr(a12), float(mean_up13), C.byref(res))
        if st == FDM_WARN_NOT_DIV_FREE:
            warnings.warn("Nye field is not divergence-free (residual %.3e); its divergence-free "
                          "part was used" % res.value)
        else:
            _check(st, "fdm_set_density")
        return res.value

    def set_mobility_field(self, factor=None):
        """Per-cell mobility factor m(x) >= 0 multiplying the celerity (heterogeneous drag,
        m = 0 in impenetrable precipitates, Sec. 5.3); None restores m = 1."""
        if factor is None:
            _check(self.lib.fdm_set_mobility_field(self.h, None), "fdm_set_mobility_field")
            return
        f = _field(factor, self.shape)
        _check(self.lib.fdm_set_mobility_field(self.h, _dptr(f)), "fdm_set_mobility_field")

    def set_plastic_distortion(self, up13):
        u = _field(up13, self.shape)
        _check(self.lib.fdm_set_plastic_distortion(self.h, _dptr(u)), "fdm_set_plastic_distortion")

    def set_clock(self, step: int, t: float):
        _check(self.lib.fdm_set_clock(self.h, int(step), float(t)), "fdm_set_clock")

    # -- compute
    def static_solve(self):
        _check(self.lib.fdm_static_solve(self.h), "fdm_static_solve")

    def read_stress13_planes(self, planes) -> np.ndarray:
        """sigma13 of the current state on the given planes x3 of the 3-D cell (the layer is
        planes 0 .. nh-1); returns [len(planes)][n2][n1]."""
        pl = np.ascontiguousarray(planes, dtype=np.int32)
        out = np.empty((len(pl),) + self.shape, dtype=np.float64)
        _check(self.lib.fdm_read_stress13_planes(self.h, len(pl), pl.ctypes.data_as(C.POINTER(C.c_int32)),
                                                 _dptr(out)), "fdm_read_stress13_planes")
        return out

    def static_solve_heterogeneous(self, mu_factor, tol: float = 1e-12, max_iter: int = 200):
        """Antiplane static problem with the shear modulus mu * mu_factor(x) (heterogeneous
        medium, Sec. 3.1.2; needs nh == nz).  Returns (sigma13, sigma23, iterations, residual);
        sigma13 also becomes the handle's tau13."""
        f = _field(mu_factor, self.shape)
        s13, s23 = np.empty(self.shape), np.empty(self.shape)
        it, r = C.c_int32(0), C.c_double(0.0)
        _check(self.lib.fdm_static_solve_heterogeneous(self.h, _dptr(f), float(tol), int(max_iter), _dptr(s13),
                                                       _dptr(s23), C.byref(it), C.byref(r)),
               "fdm_static_solve_heterogeneous")
        return s13, s23, it.value, r.value

    def static_solve_heterogeneous_layer(self, mu_factor, tol: float = 1e-12, max_iter: int = 200, planes=()):
        """Static problem of a plastic layer thinner than the cell in a medium whose moduli
        are scaled by mu_factor(x1, x2), uniform through the depth (FP64 handles, nz even):
        returns (tau13 = layer average of sigma13, sigma13 on the planes or None, iterations,
        residual)."""
        p = self.params
        f = _field(mu_factor, (p.n2, p.n1))
        tau = np.zeros((p.n2, p.n1))
        pl = np.ascontiguousarray(planes, dtype=np.int32)
        out = np.zeros((len(pl), p.n2, p.n1)) if len(pl) else None
        it, res = C.c_int32(0), C.c_double(0.0)
        _check(self.lib.fdm_static_solve_heterogeneous_layer(
            self.h, _dptr(f), float(tol), int(max_iter), _dptr(tau), len(pl),
            pl.ctypes.data_as(C.POINTER(C.c_int32)) if len(pl) else None,
            _dptr(out) if out is not None else None, C.byref(it), C.byref(res)),
            "fdm_static_solve_heterogeneous_layer")
        return tau, out, it.value, res.value

    def set_shear_modulus_field(self, mu_factor=None, tol: float = 1e-12, max_iter: int = 200):
        """Heterogeneous elasticity in every later static solve and step: shear modulus
        mu * mu_factor(x) (needs nh == nz); None returns to the layer solve."""
        if mu_factor is None:
            _check(self.lib.fdm_set_shear_modulus_field(self.h, None, 0.0, 1), "fdm_set_shear_modulus_field")
            return
        f = _field(mu_factor, self.shape)
        _check(self.lib.fdm_set_shear_modulus_field(self.h, _dptr(f), float(tol), int(max_iter)),
               "fdm_set_shear_modulus_field")

    def read_stress_planes(self, comp, planes) -> np.ndarray:
        """Stress component ``comp`` ("11", "22", "33", "23", "13", "12" or its Voigt index) of
        the current state on the given planes x3 of the 3-D cell; returns
        [len(planes)][n2][n1]."""
        c = STRESS_COMPONENTS.index(comp) if isinstance(comp, str) else int(comp)
        pl = np.ascontiguousarray(planes, dtype=np.int32)
        out = np.empty((len(pl),) + self.shape, dtype=np.float64)
        _check(self.lib.fdm_read_stress_planes(self.h, c, len(pl), pl.ctypes.data_as(C.POINTER(C.c_int32)),
                                               _dptr(out)), "fdm_read_stress_planes")
        return out

    def set_loading(self, mode: int, sigma_bar13: float = 0.0, eps_bar13_0: float = 0.0,
                    eps_bar13_rate: float = 0.0):
        """Switch the macroscopic loading for the following steps (stages of Sec. 5.1)."""
        _check(self.lib.fdm_set_loading(self.h, int(mode), float(sigma_bar13), float(eps_bar13_0),
                                        float(eps_bar13_rate)), "fdm_set_loading")

    def equilibrate(self, tol: float = 1e-6, chunk: int = 50, max_steps: int = 100000):
        """Equilibration stage of Sec. 5.1 (``fdm_equilibrate``): zero mean stress until a chunk
        of steps changes U13 by less than ``tol`` (relative L2, reduced on the device) or
        ``max_steps`` are taken.  Returns (steps taken, last relative change); the loading
        stays at zero mean stress (switch it with ``set_loading`` for the next stage)."""
        taken, change = C.c_int64(0), C.c_double(0.0)
        _check(self.lib.fdm_equilibrate(self.h, float(tol), int(chunk), int(max_steps), C.byref(taken),
                                        C.byref(change)), "fdm_equilibrate")
        return int(taken.value), float(change.value)

    def step(self, nsteps: int = 1, info: bool = True) -> Optional[StepInfo]:
        if info:
            ci = CStepInfo()
            _check(self.lib.fdm_step(self.h, int(nsteps), C.byref(ci)), "fdm_step")
            return StepInfo(**{f: getattr(ci, f) for f, _ in CStepInfo._fields_})
        _check(self.lib.fdm_step(self.h, int(nsteps), None), "fdm_step")
        return None

    def enqueue_steps(self, nsteps: int = 1):
        """Enqueue steps on the handle's stream without waiting."""
        _check(self.lib.fdm_enqueue_steps(self.h, int(nsteps)), "fdm_enqueue_steps")

    def enqueue_phase(self, phase: int):
        """Enqueue kernel ``phase`` of the current step (phases run in order 0..k-1)."""
        _check(self.lib.fdm_enqueue_phase(self.h, int(phase)), "fdm_enqueue_phase")

    def sync(self):
        """Wait for the stream; raise on a device-side error."""
        _check(self.lib.fdm_sync(self.h), "fdm_sync")

    def info(self) -> StepInfo:
        ci = CStepInfo()
        _check(self.lib.fdm_get_info(self.h, C.byref(ci)), "fdm_get_info")
        return StepInfo(**{f: getattr(ci, f) for f, _ in CStepInfo._fields_})

    def read_fields(self, *names, out=None):
        """Returns {name: array [n2][n1] float64} for names in up13, alpha11, alpha12,
        tau13, v1, v2 (``out`` may supply preallocated host arrays by name)."""
        mask = 0
        arrs = {}
        ptrs = []
        for nm in ("up13", "alpha11", "alpha12", "tau13", "v1", "v2"):
            if nm in names:
                mask |= FIELDS[nm]
                a = out[nm] if out and nm in out else np.empty(self.shape, dtype=np.float64)
                arrs[nm] = a
                ptrs.append(_dptr(a))
            else:
                ptrs.append(None)
        unknown = set(names) - set(FIELDS)
        if unknown:
            raise ValueError("unknown fields %s" % sorted(unknown))
        _check(self.lib.fdm_read_fields(self.h, mask, *ptrs), "fdm_read_fields")
        return arrs

    def kernels_per_step(self) -> int:
        return int(self.lib.fdm_kernels_per_step(self.h))

    def launch_config(self) -> dict:
        """Launch shapes of the step kernels (autotuned or heuristic)."""
        c = CLaunchConfig()
        _check(self.lib.fdm_get_launch_config(self.h, C.byref(c)), "fdm_get_launch_config")
        return _launch_config(c)

    def set_launch_config(self, cfg: dict):
        """Pin the launch shapes (keys as returned by ``launch_config``)."""
        c = CLaunchConfig()
        for f, _ in CLaunchConfig._fields_:
            if f in cfg and f not in ("kernel_us", "tuned"):
                setattr(c, f, int(cfg[f]))
        _check(self.lib.fdm_set_launch_config(self.h, C.byref(c)), "fdm_set_launch_config")

    def close(self):
        if getattr(self, "h", None):
            self.lib.fdm_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _params_array(params):
    arr = (CParams * len(params))()
    for i, p in enumerate(params):
        arr[i] = p.to_c()
    return arr


def launch_candidates(params: "Params") -> list:
    """The launch configurations the autotuner times for these parameters (no GPU needed)."""
    lib = load()
    cp = params.to_c()
    n = int(lib.fdm_launch_candidates(C.byref(cp), None, 0))
    arr = (CLaunchConfig * max(n, 1))()
    lib.fdm_launch_candidates(C.byref(cp), arr, n)
    return [_launch_config(arr[i]) for i in range(n)]


def batch_device_bytes(params) -> int:
    return int(load().fdm_batch_device_bytes(len(params), _params_array(params)))


class Batch:
    """Many independent FDM instances stepped together on the GPU (``fdm_batch_*``).

    Instances with identical parameters share each kernel launch; every instance has a step
    budget and only instances with budget left advance, so uneven run lengths share launches.
    """

    def __init__(self, params, stream: Optional[int] = None):
        self.lib = load()
        self.params = list(params)
        self.count = len(self.params)
        h = C.c_void_p()
        _check(self.lib.fdm_batch_create(self.count, _params_array(self.params), C.c_void_p(stream or 0),
                                         C.byref(h)), "fdm_batch_create")
        self.h = h

    def set_plastic_distortion(self, i: int, up13):
        p = self.params[i]
        u = _field(up13, (p.n2, p.n1))
        _check(self.lib.fdm_batch_set_plastic_distortion(self.h, int(i), _dptr(u)),
               "fdm_batch_set_plastic_distortion")

    def set_budget(self, i: int, steps: int):
        _check(self.lib.fdm_batch_set_budget(self.h, int(i), int(steps)), "fdm_batch_set_budget")

    def enqueue_steps(self, nsteps: int):
        _check(self.lib.fdm_batch_enqueue_steps(self.h, int(nsteps)), "fdm_batch_enqueue_steps")

    def enqueue_steps_persistent(self, nsteps: int):
        """The same steps as ``enqueue_steps`` in one persistent launch (mixed precision)."""
        _check(self.lib.fdm_batch_enqueue_steps_persistent(self.h, int(nsteps)),
               "fdm_batch_enqueue_steps_persistent")

    def sync(self) -> np.ndarray:
        """Wait; return every instance's remaining step budget (raises on device errors)."""
        left = np.zeros(self.count, dtype=np.int64)
        _check(self.lib.fdm_batch_sync(self.h, left.ctypes.data_as(C.POINTER(C.c_int64))), "fdm_batch_sync")
        return left

    def sync_status(self):
        """Wait; return (remaining step budgets, device-side status of every instance) without
        raising on instance errors."""
        left = np.zeros(self.count, dtype=np.int64)
        status = np.zeros(self.count, dtype=np.int32)
        _check(self.lib.fdm_batch_sync_status(self.h, left.ctypes.data_as(C.POINTER(C.c_int64)),
                                              status.ctypes.data_as(C.POINTER(C.c_int32))), "fdm_batch_sync_status")
        return left, status

    def info(self, i: int) -> StepInfo:
        ci = CStepInfo()
        _check(self.lib.fdm_batch_get_info(self.h, int(i), C.byref(ci)), "fdm_batch_get_info")
        return StepInfo(**{f: getattr(ci, f) for f, _ in CStepInfo._fields_})

    def read_fields(self, i: int, *names):
        p = self.params[i]
        out = {}
        up = np.empty((p.n2, p.n1)) if "up13" in names else None
        tau = np.empty((p.n2, p.n1)) if "tau13" in names else None
        mask = (FIELD_UP13 if up is not None else 0) | (FIELD_TAU13 if tau is not None else 0)
        _check(self.lib.fdm_batch_read_fields(self.h, int(i), mask, _dptr(up) if up is not None else None,
                                              _dptr(tau) if tau is not None else None), "fdm_batch_read_fields")
        if up is not None:
            out["up13"] = up
        if tau is not None:
            out["tau13"] = tau
        return out

    def launches_per_step(self) -> int:
        return int(self.lib.fdm_batch_launches_per_step(self.h))

    def launch_config(self, i: int) -> dict:
        """Launch shapes of the group holding instance i."""
        c = CLaunchConfig()
        _check(self.lib.fdm_batch_get_launch_config(self.h, i, C.byref(c)), "fdm_batch_get_launch_config")
        return _launch_config(c)

    def close(self):
        if getattr(self, "h", None):
            self.lib.fdm_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
