"""FP64 CPU oracle for the FDM layer-case time step (arXiv 1911.03225).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by
the CPU-baseline leg of ``bench.py``; never by the product path.  The arithmetic lives in
``fdm_oracle.c`` (plain C, FP64); this module only marshals numpy arrays through ctypes.
It shares no code with the CUDA library and never loads it.
"""
import ctypes as C
from dataclasses import dataclass, field, asdict

import numpy as np

from .build import build_oracle

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build_oracle())
        d = C.POINTER(C.c_double)
        _lib.oracle_fft1d.argtypes = [C.c_int, d, d, C.c_int]
        _lib.oracle_fft2d.argtypes = [C.c_int, C.c_int, d, d, C.c_int]
        _lib.oracle_layer_symbol.argtypes = [C.c_double] * 5
        _lib.oracle_layer_symbol.restype = C.c_double
        _lib.oracle_kernel_table.argtypes = [C.c_int] * 4 + [C.c_double, C.c_double, d]
        _lib.oracle_static_tau.argtypes = [C.c_int, C.c_int, d, d, C.c_double, d]
        _lib.oracle_curl_inverse.argtypes = [C.c_int, C.c_int, C.c_double, d, d, C.c_double, d, d]
        _lib.oracle_curl_inverse.restype = C.c_double
        _lib.oracle_alpha_from_up.argtypes = [C.c_int, C.c_int, C.c_double, d, d, d]
        _lib.oracle_knp1d_step.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, d, d, d]
        _lib.oracle_knp2d_step.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, d, d, d]
        _lib.oracle_sum.argtypes = [C.c_size_t, d]
        _lib.oracle_sum.restype = C.c_double
        _lib.oracle_alpha_sums.argtypes = [C.c_int, C.c_int, C.c_double, d, d]
        _lib.oracle_run.argtypes = [C.c_void_p, d, d, C.c_void_p, C.c_int, d, d, d]
        _lib.oracle_stress13_planes.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, d,
                                                C.c_double, C.c_int, C.POINTER(C.c_int), d]
        _lib.oracle_stress_planes.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, d,
                                              C.c_double, C.c_int, C.c_int, C.POINTER(C.c_int), d]
        _lib.oracle_stress_symbol.argtypes = [C.c_int] + [C.c_double] * 5
        _lib.oracle_stress_symbol.restype = C.c_double
        _lib.oracle_hetero_antiplane.argtypes = [C.c_int, C.c_int, d, d, C.c_int, C.c_double, C.c_double, C.c_int,
                                                 d, d, d]
        _lib.oracle_hetero_antiplane.restype = C.c_int
        _lib.oracle_run.restype = C.c_int
        _lib.oracle_run_hetero.argtypes = [C.c_void_p, d, d, C.c_void_p, C.c_int, d, d, d, d, C.c_double, C.c_int]
        _lib.oracle_run_hetero.restype = C.c_int
        _lib.oracle_hetero_layer.argtypes = [C.c_int] * 4 + [C.c_double, C.c_double, d, d, C.c_int, C.c_double,
                                                              C.c_double, C.c_int, d, d, d]
        _lib.oracle_hetero_layer.restype = C.c_int
        _lib.oracle_set_threads.argtypes = [C.c_int]
        _lib.oracle_set_threads.restype = C.c_int
        _lib.oracle_threads.restype = C.c_int
    return _lib


def set_threads(n: int) -> int:
    """Threads of the oracle's parallel loops (independent rows, columns and nodes);
    n < 1 takes every core.  Results are identical for every count.  Returns the count in
    effect (1 when built without OpenMP).  The default is 1, the plain serial program."""
    return lib().oracle_set_threads(int(n))


def threads() -> int:
    return lib().oracle_threads()


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _Params(C.Structure):
    _fields_ = [("n1", C.c_int32), ("n2", C.c_int32), ("nz", C.c_int32), ("nh", C.c_int32),
                ("dx", C.c_double), ("E", C.c_double), ("nu", C.c_double),
                ("velocity_mode", C.c_int32),
                ("v0", C.c_double), ("mobility", C.c_double), ("tau_y", C.c_double),
                ("beta", C.c_double), ("theta", C.c_double), ("cfl", C.c_double),
                ("dt_max", C.c_double),
                ("loading_mode", C.c_int32),
                ("sigma_bar13", C.c_double), ("eps_bar13_0", C.c_double),
                ("eps_bar13_rate", C.c_double),
                ("time_level", C.c_int32)]


class _Scalars(C.Structure):
    _fields_ = [("step", C.c_int64), ("t", C.c_double), ("dt", C.c_double),
                ("max_abs_v0", C.c_double), ("mean_up13", C.c_double),
                ("eps_bar13", C.c_double), ("sigma_bar13", C.c_double)]


@dataclass
class Params:
    """Dimensionless problem parameters (Sec. 3.2.1 non-dimensionalisation)."""
    n1: int
    n2: int
    nz: int = 0            # 0 -> cubic cell, nz = n1
    nh: int = 4
    dx: float = 1.0
    E: float = 1.0
    nu: float = 0.3
    velocity_mode: int = 0  # 0 prescribed uniform v0, 1 stress driven
    v0: float = 1.0
    mobility: float = 1.0
    tau_y: float = 0.0
    beta: float = 1.0
    theta: float = 1.0
    cfl: float = 0.5
    dt_max: float = 0.0
    loading_mode: int = 0   # 0 stress, 1 strain ramp, 2 zero mean stress
    sigma_bar13: float = 0.0
    eps_bar13_0: float = 0.0
    eps_bar13_rate: float = 0.0
    time_level: int = 0     # 0 midpoint, 1 literal

    @property
    def mu(self):
        return self.E / (2.0 * (1.0 + self.nu))

    def _c(self):
        d = asdict(self)
        if d["nz"] == 0:
            d["nz"] = d["n1"]
        return _Params(**d)


def fft1d(x, sign=-1):
    x = np.asarray(x, dtype=np.complex128)
    re, im = _f64(x.real.copy()), _f64(x.imag.copy())
    lib().oracle_fft1d(len(x), _p(re), _p(im), sign)
    return re + 1j * im


def fft2d(x, sign=-1):
    x = np.asarray(x, dtype=np.complex128)
    n2, n1 = x.shape
    re, im = _f64(x.real.copy()), _f64(x.imag.copy())
    lib().oracle_fft2d(n1, n2, _p(re), _p(im), sign)
    return re + 1j * im


def layer_symbol(n1, n2, n3, mu, nu):
    return lib().oracle_layer_symbol(n1, n2, n3, mu, nu)


def kernel_table(n1, n2, nz, nh, mu, nu):
    K = np.zeros((n2, n1))
    lib().oracle_kernel_table(n1, n2, nz, nh, mu, nu, _p(K))
    return K


def static_tau(up13, K, sigma_bar13=0.0):
    up13, K = _f64(up13), _f64(K)
    out = np.zeros_like(up13)
    n2, n1 = up13.shape
    lib().oracle_static_tau(n1, n2, _p(up13), _p(K), sigma_bar13, _p(out))
    return out


def curl_inverse(a11, a12, mean_up13=0.0, dx=1.0):
    """Returns (U13, relative divergence residual, mean alpha (2,))."""
    a11, a12 = _f64(a11), _f64(a12)
    n2, n1 = a11.shape
    out = np.zeros_like(a11)
    ma = np.zeros(2)
    r = lib().oracle_curl_inverse(n1, n2, dx, _p(a11), _p(a12), mean_up13, _p(out), _p(ma))
    return out, r, ma


def alpha_from_up(up13, dx=1.0):
    up13 = _f64(up13)
    n2, n1 = up13.shape
    a11, a12 = np.zeros_like(up13), np.zeros_like(up13)
    lib().oracle_alpha_from_up(n1, n2, dx, _p(up13), _p(a11), _p(a12))
    return a11, a12


def knp1d_step(phi, v0, dt, theta=1.0, h=1.0, time_level=0):
    phi = _f64(phi)
    v0 = _f64(np.broadcast_to(v0, phi.shape))
    out = np.zeros_like(phi)
    lib().oracle_knp1d_step(len(phi), h, theta, dt, time_level, _p(phi), _p(v0), _p(out))
    return out


def knp2d_step(phi, v0, dt, theta=1.0, h=1.0, time_level=0):
    phi = _f64(phi)
    v0 = _f64(np.broadcast_to(v0, phi.shape))
    n2, n1 = phi.shape
    out = np.zeros_like(phi)
    lib().oracle_knp2d_step(n1, n2, h, theta, dt, time_level, _p(phi), _p(v0), _p(out))
    return out


def compensated_sum(x):
    x = _f64(np.ravel(x))
    return lib().oracle_sum(x.size, _p(x))


def alpha_sums(up13, h=1.0):
    up13 = _f64(up13)
    n2, n1 = up13.shape
    out = np.zeros(5)
    lib().oracle_alpha_sums(n1, n2, h, _p(up13), _p(out))
    return out


@dataclass
class State:
    up13: np.ndarray
    step: int = 0
    t: float = 0.0
    dt: float = 0.0
    max_abs_v0: float = 0.0
    mean_up13: float = 0.0
    eps_bar13: float = 0.0
    sigma_bar13: float = 0.0
    tau13: np.ndarray = field(default=None, repr=False)
    v0: np.ndarray = field(default=None, repr=False)


def stress13_planes(up13, nz, nh, mu, nu, sigma_bar13, planes):
    """sigma13 on the planes x3 in ``planes`` of the 3-D cell of nz voxels whose planes
    0 .. nh-1 carry U13 (Sec. 3.1.2, Sec. 3.2.1).  Returns [len(planes)][n2][n1]."""
    u = _f64(up13)
    n2, n1 = u.shape
    pl = np.ascontiguousarray(planes, dtype=np.int32)
    out = np.zeros((len(pl), n2, n1))
    lib().oracle_stress13_planes(n1, n2, int(nz), int(nh), float(mu), float(nu), _p(u), float(sigma_bar13),
                                 len(pl), pl.ctypes.data_as(C.POINTER(C.c_int)), _p(out))
    return out


# Voigt order of the stress components (11, 22, 33, 23, 13, 12)
STRESS_COMPONENTS = ("11", "22", "33", "23", "13", "12")


def stress_symbol(comp, n1, n2, n3, mu, nu):
    """sigma-hat_comp / U13-hat for the direction n (Sec. 3.1.2 Green operator)."""
    return lib().oracle_stress_symbol(STRESS_COMPONENTS.index(comp), n1, n2, n3, mu, nu)


def stress_planes(up13, nz, nh, mu, nu, sigma_bar13, comp, planes):
    """Stress component ``comp`` ("11", "22", "33", "23", "13" or "12") on the planes x3 in
    ``planes`` of the 3-D cell of nz voxels whose planes 0 .. nh-1 carry U13 (Sec. 3.1.2,
    Sec. 3.2.1).  Returns [len(planes)][n2][n1]."""
    u = _f64(up13)
    n2, n1 = u.shape
    pl = np.ascontiguousarray(planes, dtype=np.int32)
    out = np.zeros((len(pl), n2, n1))
    lib().oracle_stress_planes(n1, n2, int(nz), int(nh), float(mu), float(nu), _p(u), float(sigma_bar13),
                               STRESS_COMPONENTS.index(comp), len(pl), pl.ctypes.data_as(C.POINTER(C.c_int)),
                               _p(out))
    return out


def hetero_antiplane(mu, up13, stress_control, load, tol=0.0, max_iter=50):
    """Antiplane static problem with a shear modulus field mu(x) (Sec. 3.1.2, heterogeneous
    medium; plastic layer filling the cell): returns (sigma13, sigma23, iterations, residual).
    ``load``: sigma_bar13 under stress control, else eps_bar13 (strain control)."""
    m, u = _f64(mu), _f64(up13)
    n2, n1 = u.shape
    s13, s23, r = np.zeros((n2, n1)), np.zeros((n2, n1)), C.c_double(0.0)
    it = lib().oracle_hetero_antiplane(n1, n2, _p(m), _p(u), int(bool(stress_control)), float(load), float(tol),
                                       int(max_iter), _p(s13), _p(s23), C.byref(r))
    return s13, s23, it, r.value


def hetero_layer(factor, up13, nz, nh, mu, nu, stress_control, load, tol=0.0, max_iter=50, planes=False):
    """Static problem of a plastic layer of nh planes in a cell of nz with a modulus field
    f(x1, x2) uniform through the depth (Sec. 3.1.2 heterogeneous medium, layer of Sec. 3.2.1):
    returns (tau13 = layer average of sigma13, sigma13 of every plane or None, iterations,
    residual).  ``load``: sigma_bar13 under stress control, else eps_bar13."""
    fa, u = _f64(factor), _f64(up13)
    n2, n1 = u.shape
    tau = np.zeros((n2, n1))
    s13 = np.zeros((int(nz), n2, n1)) if planes else None
    r = C.c_double(0.0)
    it = lib().oracle_hetero_layer(n1, n2, int(nz), int(nh), float(mu), float(nu), _p(fa), _p(u),
                                   int(bool(stress_control)), float(load), float(tol), int(max_iter), _p(tau),
                                   None if s13 is None else _p(s13), C.byref(r))
    return tau, s13, it, r.value


def run(params: Params, up13, nsteps, K=None, state: State = None, mobility_factor=None, shear_modulus=None,
        hetero_tol=0.0, hetero_max_iter=50):
    """Advance ``nsteps`` FDM steps (Sec. 3.1.1) from ``up13`` (or ``state``).
    ``mobility_factor``: optional per-node m(x) >= 0 multiplying the celerity
    (heterogeneous drag, m = 0 in impenetrable precipitates; Sec. 5.3).
    ``shear_modulus``: optional field mu(x) (heterogeneous elasticity, layer filling the
    cell): each step's static problem is then ``hetero_antiplane`` with ``hetero_tol`` and
    ``hetero_max_iter``."""
    p = params._c()
    if K is None:
        K = kernel_table(p.n1, p.n2, p.nz, p.nh, params.mu, params.nu)
    if state is None:
        state = State(up13=_f64(up13).copy())
    sc = _Scalars(step=state.step, t=state.t, dt=state.dt, max_abs_v0=state.max_abs_v0,
                  mean_up13=state.mean_up13, eps_bar13=state.eps_bar13,
                  sigma_bar13=state.sigma_bar13)
    u = _f64(state.up13).copy()
    tau = np.zeros_like(u)
    v0 = np.zeros_like(u)
    mf = None if mobility_factor is None else _f64(mobility_factor)
    if mf is not None and mf.shape != u.shape:
        raise ValueError("mobility factor must have the field's shape")
    mu = None if shear_modulus is None else _f64(shear_modulus)
    if mu is not None and mu.shape != u.shape:
        raise ValueError("shear modulus must have the field's shape")
    rc = lib().oracle_run_hetero(C.byref(p), _p(_f64(K)), _p(u), C.byref(sc), int(nsteps), _p(tau), _p(v0),
                                 None if mf is None else _p(mf), None if mu is None else _p(mu), float(hetero_tol),
                                 int(hetero_max_iter))
    return State(up13=u, step=sc.step, t=sc.t, dt=sc.dt, max_abs_v0=sc.max_abs_v0,
                 mean_up13=sc.mean_up13, eps_bar13=sc.eps_bar13, sigma_bar13=sc.sigma_bar13,
                 tau13=tau, v0=v0), rc
