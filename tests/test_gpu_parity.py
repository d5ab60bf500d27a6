"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element
on the same seeded inputs.  Tolerances: FP64 path 1e-11 relative L2; mixed precision
(FP32 fields, FFT and stencil; FP64 scalars) 1e-5 relative L2 unless stated."""
import numpy as np
import pytest

import oracle
from paper_1911_03225_gb300 import FDM, FDMError, Params, inputs
from paper_1911_03225_gb300 import binding as B

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
TOL_MIXED = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def oparams(p: Params) -> oracle.Params:
    d = {k: getattr(p, k) for k in oracle.Params.__dataclass_fields__}
    return oracle.Params(**d)


def run_both(p: Params, up0=None, alpha=None, mean=0.0, steps=10):
    with FDM(p) as sim:
        if alpha is not None:
            sim.set_density(alpha[0], alpha[1], mean)
            start = sim.read_fields("up13")["up13"]
        else:
            sim.set_plastic_distortion(up0)
            start = up0
        info = sim.step(steps)
        got = sim.read_fields("up13", "tau13")
    if alpha is not None:
        up_o, _, _ = oracle.curl_inverse(alpha[0], alpha[1], mean, p.dx)
    else:
        up_o = up0
    ref, rc = oracle.run(oparams(p), up_o, steps)
    assert rc == 0
    return got, info, ref, start


# ------------------------------------------------------------------ static problem
@pytest.mark.parametrize("shape", [(32, 64), (64, 64), (128, 32), (256, 256)])
@pytest.mark.parametrize("nh", [1, 4])
@pytest.mark.parametrize("precision", [B.FP64, B.DF64])
def test_static_solve_matches_oracle(shape, nh, precision):
    n2, n1 = shape
    up = np.random.default_rng(n1 + n2).standard_normal(shape)
    p = Params(n1=n1, n2=n2, nh=nh, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_STRESS, sigma_bar13=0.013,
               precision=precision)
    with FDM(p) as sim:
        sim.set_plastic_distortion(up)
        sim.static_solve()
        tau = sim.read_fields("tau13")["tau13"]
    K = oracle.kernel_table(n1, n2, n1, nh, p.E / (2 * (1 + p.nu)), p.nu)
    ref = oracle.static_tau(up, K, 0.013)
    assert rel(tau, ref) < 1e-12


def test_static_solve_strain_control_and_zero_alpha():
    n = 64
    up = np.full((n, n), 0.37)
    p = Params(n1=n, n2=n, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_STRAIN_RAMP, eps_bar13_0=2e-3)
    with FDM(p) as sim:
        sim.set_plastic_distortion(up)
        sim.static_solve()
        tau = sim.read_fields("tau13")["tau13"]
    mu = 1 / 2.6
    np.testing.assert_allclose(tau, 2 * mu * 2e-3 - mu * (4 / 64) * 0.37, rtol=0, atol=1e-15)


# ------------------------------------------------------------------ curl inverse and readout
@pytest.mark.parametrize("precision,tol", [(B.FP64, 1e-12), (B.DF64, 1e-12), (B.MIXED, 1e-5)])
def test_set_density_matches_oracle(precision, tol):
    n = 128
    a11, a12 = inputs.ring_alpha(n, r0=30.0, sigma=2.0)
    p = Params(n1=n, n2=n, precision=precision)
    with FDM(p) as sim:
        res = sim.set_density(a11, a12, 0.25)
        up = sim.read_fields("up13")["up13"]
    ref, res_o, _ = oracle.curl_inverse(a11, a12, 0.25)
    assert rel(up, ref) < tol
    assert abs(res - res_o) < 1e-6


def test_set_density_non_square_and_residual():
    n1, n2 = 64, 32
    u = np.random.default_rng(5).standard_normal((n2, n1))
    a11, a12 = oracle.alpha_from_up(u)
    # add a gradient (non-divergence-free) part
    g1, g2 = np.gradient(np.random.default_rng(6).standard_normal((n2, n1)))
    b11, b12 = a11 + g2 - g2.mean(), a12 + g1 - g1.mean()
    with FDM(Params(n1=n1, n2=n2)) as sim:
        with pytest.warns(UserWarning):
            res = sim.set_density(b11, b12, -0.5)
        up = sim.read_fields("up13")["up13"]
    ref, res_o, _ = oracle.curl_inverse(b11, b12, -0.5)
    assert rel(up, ref) < 1e-12
    assert res == pytest.approx(res_o, rel=1e-9)


def test_net_burgers_vector_rejected():
    n = 32
    a11 = np.full((n, n), 0.1)
    with FDM(Params(n1=n, n2=n)) as sim:
        with pytest.raises(FDMError) as e:
            sim.set_density(a11, np.zeros((n, n)))
        assert e.value.status == B.FDM_ERR_NET_BURGERS


@pytest.mark.parametrize("precision,tol", [(B.FP64, 1e-12), (B.DF64, 1e-12), (B.MIXED, 2e-5)])
def test_alpha_and_velocity_readout(precision, tol):
    n1, n2 = 128, 64
    u = inputs.random_up(128, seed=2, ell=5.0)[:n2, :]
    u = oracle.curl_inverse(*oracle.alpha_from_up(u))[0]   # periodic, band-limited
    p = Params(n1=n1, n2=n2, velocity_mode=B.V_STRESS, precision=precision, mobility=1.5)
    with FDM(p) as sim:
        sim.set_plastic_distortion(u)
        sim.static_solve()
        f = sim.read_fields("alpha11", "alpha12", "v1", "v2", "tau13")
    a11, a12 = oracle.alpha_from_up(u)
    assert rel(f["alpha11"], a11) < tol and rel(f["alpha12"], a12) < tol
    K = oracle.kernel_table(n1, n2, n1, 4, 1 / 2.6, 0.3)
    v0 = -1.5 * oracle.static_tau(u, K, 0.0)
    m = np.hypot(a11, a12)
    assert rel(f["v1"], v0 * a12 / m) < 10 * tol and rel(f["v2"], -v0 * a11 / m) < 10 * tol


@pytest.mark.parametrize("precision,tol", [(B.FP64, TOL64), (B.DF64, TOL64), (B.MIXED, TOL_MIXED)])
def test_stress13_planes_of_the_3d_cell_match_oracle(precision, tol):
    """sigma13 through the 3-D cell (Sec. 3.1.2 on the nz-voxel cell; the layer is planes
    0 .. nh-1): planes inside, at the edge of and far from the layer against the oracle's
    term-by-term 3-D transform; the layer average of the planes is the step's tau13."""
    n1, n2, nz, nh = 64, 32, 32, 4
    up0 = inputs.random_up(64, seed=14, ell=4.0)[:n2, :n1].copy()
    p = Params(n1=n1, n2=n2, nz=nz, nh=nh, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_STRESS,
               sigma_bar13=0.02, precision=precision)
    planes = [0, 1, 2, 3, 4, 9, 16, 31]
    with FDM(p) as sim:
        sim.set_plastic_distortion(up0)
        sim.static_solve()
        tau = sim.read_fields("tau13")["tau13"]
        got = sim.read_stress13_planes(planes)
        assert sim.info().step == 0
    ref = oracle.stress13_planes(up0, nz, nh, 1 / 2.6, 0.3, 0.02, planes)
    for g, r in zip(got, ref):
        assert rel(g, r) < tol
    assert rel(got[:nh].mean(axis=0), tau) < (1e-13 if precision != B.MIXED else 1e-6)


def test_stress13_planes_at_scale_reproduce_the_layer_reduction():
    """The K(xi1, xi2) reduction validated at scale: on a 1024^2 x 1024 cell the average of
    the four layer planes equals tau13 of the reduced static solve."""
    n, nz, nh = 1024, 1024, 4
    up0 = inputs.random_up(n, seed=15, ell=16.0)
    p = Params(n1=n, n2=n, nz=nz, nh=nh, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_STRESS, sigma_bar13=0.01)
    with FDM(p) as sim:
        sim.set_plastic_distortion(up0)
        sim.static_solve()
        tau = sim.read_fields("tau13")["tau13"]
        planes = sim.read_stress13_planes([0, 1, 2, 3, 512])
    assert rel(planes[:4].mean(axis=0), tau) < 1e-12
    # far from the layer the stress is the macroscopic stress plus a decayed image field
    assert abs(planes[4].mean() - 0.01) < 1e-12
    assert np.abs(planes[4] - 0.01).max() < np.abs(tau - 0.01).max()


@pytest.mark.parametrize("precision,tol", [(B.FP64, TOL64), (B.DF64, TOL64), (B.MIXED, TOL_MIXED)])
@pytest.mark.parametrize("nh", [3, 4])
def test_stress_planes_all_components_match_oracle(precision, tol, nh):
    """Every stress component through the 3-D cell (Sec. 3.1.2 on the nz-voxel cell) against
    the oracle's term-by-term transform of the Green-operator vector form: planes in, at the
    edge of and far from the layer, a non-square grid, input with Nyquist content; the GPU
    folds the sum over xi3 into cos or i sin weights and the closed-form symbols."""
    n1, n2, nz = 64, 32, 32
    up0 = inputs.random_up(64, seed=16, ell=4.0)[:n2, :n1].copy()
    p = Params(n1=n1, n2=n2, nz=nz, nh=nh, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_STRESS,
               sigma_bar13=0.02, precision=precision)
    planes = [0, 1, 2, 3, 4, 9, 16, 31]
    with FDM(p) as sim:
        sim.set_plastic_distortion(up0)
        sim.static_solve()
        got = {c: sim.read_stress_planes(c, planes) for c in B.STRESS_COMPONENTS}
        s13 = sim.read_stress13_planes(planes)
        assert sim.info().step == 0
    for c in B.STRESS_COMPONENTS:
        ref = oracle.stress_planes(up0, nz, nh, 1 / 2.6, 0.3, 0.02, c, planes)
        assert rel(got[c], ref) < tol, c
        for g in got[c]:
            assert abs(g.mean() - (0.02 if c == "13" else 0.0)) < 1e-6
    np.testing.assert_array_equal(got["13"], s13)


def test_stress_planes_at_scale_reflection_symmetry():
    """At 1024^2 x 1024 (three-plane layer, mid-plane x3 = 1): reflecting x3 about the
    layer's mid-plane maps U13 e1 (x) e3 to minus itself, so 13 and 23 are even and 11, 22,
    33 and 12 odd about it, at every distance."""
    n, nz, nh = 1024, 1024, 3
    up0 = inputs.random_up(n, seed=17, ell=16.0)
    p = Params(n1=n, n2=n, nz=nz, nh=nh, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_STRESS, sigma_bar13=0.0)
    with FDM(p) as sim:
        sim.set_plastic_distortion(up0)
        for c in B.STRESS_COMPONENTS:
            sign = 1.0 if c in ("13", "23") else -1.0
            s = sim.read_stress_planes(c, [2, 0, 5, nz - 3, 300, nz - 298])
            scale = np.abs(s[:2]).max()
            assert scale > 1e-4, c
            for a, b in ((0, 1), (2, 3), (4, 5)):
                assert np.abs(s[a] - sign * s[b]).max() < 1e-12 * scale, (c, a)


# ------------------------------------------------------------------ time stepping
@pytest.mark.parametrize("precision", [B.FP64, B.DF64])
def test_config0_lines_annihilation(precision):
    """128x128, two opposite edge walls 32 apart, v0 = +1, minmod, CFL 0.5, 200 steps,
    static solve every step, E = 1, nu = 0.3, no load."""
    n = 128
    a11, a12 = inputs.lines_alpha(n)
    p = Params(n1=n, n2=n, velocity_mode=B.V_PRESCRIBED, v0=1.0, theta=1.0, cfl=0.5, precision=precision)
    got, info, ref, start = run_both(p, alpha=(a11, a12), mean=0.0, steps=200)
    assert rel(got["up13"], ref.up13) < TOL64
    # the walls have annihilated by t = 100: tau13 is zero up to rounding, so compare it on
    # the scale of the initial stress
    K = oracle.kernel_table(n, n, n, 4, 1 / 2.6, 0.3)
    scale = np.linalg.norm(oracle.static_tau(start, K, 0.0))
    assert np.linalg.norm(got["tau13"] - ref.tau13) < TOL64 * scale
    assert info.step == 200 and info.t == pytest.approx(ref.t, rel=1e-14)
    assert info.dt == pytest.approx(0.5, rel=1e-15)
    s = oracle.alpha_sums(ref.up13)
    assert info.sum_abs_alpha == pytest.approx(s[4], rel=1e-11, abs=1e-12)
    assert abs(info.sum_a12_pos + info.sum_a12_neg) < 1e-9   # total Burgers vector


@pytest.mark.parametrize("precision,tol", [(B.FP64, TOL64), (B.DF64, TOL64), (B.MIXED, TOL_MIXED)])
def test_ring_expansion_short(precision, tol):
    """Config-1 shape at reduced size: ring, MC limiter (theta = 2), CFL 0.4, v0 = -1."""
    n = 256
    a11, a12 = inputs.ring_alpha(n, r0=50.0, sigma=2.0)
    p = Params(n1=n, n2=n, v0=-1.0, theta=2.0, cfl=0.4, precision=precision)
    got, info, ref, _ = run_both(p, alpha=(a11, a12), mean=0.0, steps=5)
    assert rel(got["up13"], ref.up13) < tol
    assert rel(got["tau13"], ref.tau13) < tol


# FP64 and mixed: one rounding unit of the path (stricter than needed, and they pass it);
# double-word: its unit 2^-48 accumulated over the 100 steps, because its per-step rounding
# is 30x that of FP64 and the MC-limited scheme amplifies every step's share.
@pytest.mark.parametrize("precision,eps", [(B.FP64, 1e-16), (B.DF64, 100 * 2.0 ** -48), (B.MIXED, 6e-8)])
def test_ring_expansion_long_within_rounding_envelope(precision, eps):
    """With the MC limiter the scheme amplifies rounding differences (about 1e-16 -> 1e-11
    in 10 steps, saturating near 1e-8): over 100 steps the GPU must stay within the
    oracle's own spread under a perturbation of the size of the path's rounding."""
    n, steps = 256, 100
    a11, a12 = inputs.ring_alpha(n, r0=50.0, sigma=2.0)
    p = Params(n1=n, n2=n, v0=-1.0, theta=2.0, cfl=0.4, precision=precision)
    got, info, ref, _ = run_both(p, alpha=(a11, a12), mean=0.0, steps=steps)
    up0, _, _ = oracle.curl_inverse(a11, a12, 0.0)
    pert = up0 * (1 + eps * np.random.default_rng(0).standard_normal(up0.shape))
    ref2, _ = oracle.run(oparams(p), pert, steps)
    envelope = rel(ref2.up13, ref.up13)
    assert rel(got["up13"], ref.up13) < 10 * envelope + 1e-14
    # physics: the loop radius grows as r0 + t and the total Burgers vector stays zero
    assert abs(info.sum_a12_pos + info.sum_a12_neg) < 1e-9 * info.sum_abs_alpha
    assert info.t == pytest.approx(40.0, rel=1e-12)


@pytest.mark.parametrize("v0", [-1.0, 1.0])
@pytest.mark.parametrize("precision,eps", [(B.FP64, 1e-16), (B.DF64, 100 * 2.0 ** -48), (B.MIXED, 6e-8)])
def test_square_loop_expansion_and_shrinkage(v0, precision, eps):
    """Polygonal loop (Sec. 4.4.2): square of half side ~40 cells, Gaussian section sigma 2,
    MC limiter, CFL 0.4, expansion (v0 = -1) and shrinkage (v0 = +1), 20 steps.  The MC
    limiter amplifies rounding differences, and more so at the square's corners than on the
    smooth ring, so the GPU must stay within the oracle's own spread under a perturbation
    of the size of the path's rounding (as for the long ring run); the full-size run is
    checked against the exact solution in test_gpu_full_configs.py.  The square sits off
    the grid's symmetry: on a symmetric square the limiter meets exact ties along the
    diagonals, and rounding order alone would pick the branch."""
    n, steps = 128, 20
    up0 = inputs.square_up(n, half_side=40.3, sigma=2.0, centre=(64.31, 63.77))
    p = Params(n1=n, n2=n, v0=v0, theta=2.0, cfl=0.4, precision=precision)
    got, info, ref, _ = run_both(p, up0=up0, steps=steps)
    pert = up0 * (1 + eps * np.random.default_rng(1).standard_normal(up0.shape))
    ref2, _ = oracle.run(oparams(p), pert, steps)
    envelope = rel(ref2.up13, ref.up13)
    assert rel(got["up13"], ref.up13) < 10 * envelope + 1e-14
    assert info.t == pytest.approx(ref.t, rel=1e-12)


def _precipitates(n, centres, radius):
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    m = np.ones((n, n))
    for cx, cy in centres:
        m[np.hypot(x - cx, y - cy) <= radius] = 0.0
    return m


@pytest.mark.parametrize("precision,eps", [(B.FP64, 1e-16), (B.DF64, 100 * 2.0 ** -48), (B.MIXED, 6e-8)])
def test_orowan_precipitates_match_oracle(precision, eps):
    """Heterogeneous drag (Sec. 5.3): edge walls driven by an applied stress through a field
    of impenetrable precipitates (m = 0) and a softer zone (m = 0.5), stress-driven velocity,
    minmod, 40 steps.  The driven wall pair amplifies rounding differences by ~1.3 per step
    (it does so without precipitates too: exact after one step, 1e-8 after five), so the GPU
    must stay within the oracle's own spread under a perturbation of the size of the path's
    rounding.  Exactly: nodes inside precipitates never change, their velocity is zero."""
    n, steps = 128, 40
    up0 = inputs.lines_up(n, sep=32.0, sigma=3.0)
    m = _precipitates(n, [(64, 30), (64, 90), (40, 64)], 6.0)
    m[:, 100:110] *= 0.5
    p = Params(n1=n, n2=n, velocity_mode=B.V_STRESS, mobility=1.0, loading_mode=B.LOAD_STRESS,
               sigma_bar13=0.05, cfl=0.4, theta=1.0, precision=precision)
    with FDM(p) as sim:
        sim.set_mobility_field(m)
        sim.set_plastic_distortion(up0)
        first = sim.step(1)
        f1 = sim.read_fields("up13")["up13"]
        sim.set_plastic_distortion(up0)
        info = sim.step(steps)
        got = sim.read_fields("up13", "tau13", "v1")
    ref1, _ = oracle.run(oparams(p), up0, 1, mobility_factor=m)
    ref, rc = oracle.run(oparams(p), up0, steps, mobility_factor=m)
    assert rc == 0
    tol1 = TOL64 if precision != B.MIXED else TOL_MIXED
    assert rel(f1, ref1.up13) < tol1 and first.dt == pytest.approx(ref1.dt, rel=tol1)
    pert = up0 * (1 + eps * np.random.default_rng(2).standard_normal(up0.shape))
    ref2, _ = oracle.run(oparams(p), pert, steps, mobility_factor=m)
    envelope = rel(ref2.up13, ref.up13)
    assert rel(got["up13"], ref.up13) < 10 * envelope + 1e-14
    inside = m == 0.0
    if precision == B.FP64:
        np.testing.assert_array_equal(got["up13"][inside], up0[inside])
    else:
        assert np.abs(got["up13"][inside] - up0[inside]).max() < 1e-6 * np.abs(up0).max()
    assert np.all(got["v1"][inside] == 0.0)


@pytest.mark.parametrize("precision,tol", [(B.FP64, TOL64), (B.DF64, TOL64), (B.MIXED, TOL_MIXED)])
def test_staged_loading_equilibration_then_strain_rate(precision, tol):
    """Sec. 5.1: lattice friction (tau_y = 0.02, beta = 0.05), a zero-mean-stress stage of 30
    steps, then a strain rate in time for 30 more steps, switched on the live handle; the
    oracle runs the same two stages with its state carried over."""
    n = 64
    up0 = inputs.random_up(n, seed=12, ell=6.0, rms_alpha=0.1)
    p = Params(n1=n, n2=n, velocity_mode=B.V_STRESS, mobility=1.0, tau_y=0.02, beta=0.05,
               loading_mode=B.LOAD_ZERO_MEAN_STRESS, cfl=0.4, theta=1.0, precision=precision)
    with FDM(p) as sim:
        sim.set_plastic_distortion(up0)
        i1 = sim.step(30)
        f1 = sim.read_fields("up13", "tau13")
        sim.set_loading(B.LOAD_STRAIN_RATE, eps_bar13_0=1e-4, eps_bar13_rate=2e-4)
        i2 = sim.step(30)
        f2 = sim.read_fields("up13", "tau13")
    r1, _ = oracle.run(oparams(p), up0, 30)
    p2 = oparams(Params(**{**p.__dict__, "loading_mode": B.LOAD_STRAIN_RATE, "eps_bar13_0": 1e-4,
                           "eps_bar13_rate": 2e-4}))
    r2, _ = oracle.run(p2, None, 30, state=r1)
    assert abs(f1["tau13"].mean()) < 1e-12 * np.abs(f1["tau13"]).max() + (0 if precision != B.MIXED else 1e-7)
    assert i1.sigma_bar13 == 0.0
    assert rel(f1["up13"], r1.up13) < tol and rel(f1["tau13"], r1.tau13) < tol
    assert rel(f2["up13"], r2.up13) < tol and rel(f2["tau13"], r2.tau13) < tol
    assert i2.step == 60 and i2.t == pytest.approx(r2.t, rel=tol)
    assert i2.eps_bar13 == pytest.approx(1e-4 + 2e-4 * i2.t, rel=1e-14)


def test_lattice_friction_at_the_paper_parameters():
    """Sec. 5.1 parameters of the lattice friction, FP64: beta = 1e-8 and tau_y = 1 MPa over
    mu = 26.1 GPa (aluminium, Sec. 4), with U13 of order 1, so that the phase U13 / beta of
    cos(U13 / beta) is of order 1e8 and the term is meaningful only with U13 kept to FP64.
    One step is compared strictly (the friction term enters v0 at every node).  Over longer
    runs this velocity law is chaotic at the rounding level: the oracle's own response to a
    1e-16 perturbation of its input grows to ~1e-10 in two steps and ~1e-4 in twenty (the
    phase of cos(U13 / beta) decorrelates once U13 moves by ~beta), so the two-stage run
    (20 steps at zero mean stress, then 20 steps of strain rate) is checked against ten
    times that spread, plus the exact invariants of both stages."""
    n = 128
    up0 = inputs.random_up(n, seed=12, ell=6.0, rms_alpha=0.1)
    assert np.abs(up0).max() > 1.0
    tau_y = 1e6 / 26.1e9
    p = Params(n1=n, n2=n, velocity_mode=B.V_STRESS, mobility=1.0, tau_y=tau_y, beta=1e-8,
               loading_mode=B.LOAD_ZERO_MEAN_STRESS, cfl=0.4, theta=1.0, precision=B.FP64)
    p2 = Params(**{**p.__dict__, "loading_mode": B.LOAD_STRAIN_RATE, "eps_bar13_0": 1e-4, "eps_bar13_rate": 2e-4})
    with FDM(p) as sim:
        sim.set_plastic_distortion(up0)
        first = sim.step(1)
        f1 = sim.read_fields("up13", "tau13")
        sim.set_plastic_distortion(up0)
        ia = sim.step(20)
        fa = sim.read_fields("up13", "tau13")
        sim.set_loading(B.LOAD_STRAIN_RATE, eps_bar13_0=1e-4, eps_bar13_rate=2e-4)
        ib = sim.step(20)
        fb = sim.read_fields("up13", "tau13")
    r1, rc = oracle.run(oparams(p), up0, 1)
    assert rc == 0
    assert rel(f1["up13"], r1.up13) < TOL64 and rel(f1["tau13"], r1.tau13) < TOL64
    assert first.dt == pytest.approx(r1.dt, rel=TOL64)
    ra, _ = oracle.run(oparams(p), up0, 20)
    rb, _ = oracle.run(oparams(p2), None, 20, state=ra)
    pert = up0 + 1e-16 * np.abs(up0).max() * np.random.default_rng(3).standard_normal(up0.shape)
    qa, _ = oracle.run(oparams(p), pert, 20)
    qb, _ = oracle.run(oparams(p2), None, 20, state=qa)
    env_a, env_b = rel(qa.up13, ra.up13), rel(qb.up13, rb.up13)
    assert env_a > 1e-8          # strict parity is out of reach after a few steps
    assert rel(fa["up13"], ra.up13) < 10 * env_a and rel(fb["up13"], rb.up13) < 10 * env_b
    # zero mean stress through the first stage; strain rate in time in the second
    assert ia.sigma_bar13 == 0.0 and abs(fa["tau13"].mean()) < 1e-13 * np.abs(fa["tau13"]).max()
    assert ib.step == 40 and ib.eps_bar13 == pytest.approx(1e-4 + 2e-4 * ib.t, rel=1e-14)
    for i in (ia, ib):
        assert abs(i.sum_a12_pos + i.sum_a12_neg) < 1e-9 * i.sum_abs_alpha
        assert abs(i.sum_a11_pos + i.sum_a11_neg) < 1e-9 * i.sum_abs_alpha


@pytest.mark.parametrize("precision", [B.FP64, B.MIXED])
def test_equilibration_driver_stops_when_the_field_settles(precision):
    """The zero-mean-stress stage (Sec. 5.1) run by the library in chunks, its stopping test
    reduced on the device, stops where a host-side loop over the same chunks (reading the
    field back after each) stops, with the same relative change."""
    n = 64
    up0 = inputs.random_up(n, seed=13, ell=6.0, rms_alpha=0.1)
    p = Params(n1=n, n2=n, velocity_mode=B.V_STRESS, tau_y=0.05, beta=0.05, loading_mode=B.LOAD_STRESS,
               sigma_bar13=0.3, cfl=0.4, theta=1.0, precision=precision)
    with FDM(p) as sim:
        sim.set_plastic_distortion(up0)
        taken, change = sim.equilibrate(tol=1e-4, chunk=20, max_steps=4000)
        info = sim.info()
    assert taken < 4000 and change < 1e-4
    assert info.sigma_bar13 == 0.0 and info.step == taken
    with FDM(p) as sim:
        sim.set_plastic_distortion(up0)
        sim.set_loading(B.LOAD_ZERO_MEAN_STRESS)
        prev, k, ch = sim.read_fields("up13")["up13"], 0, np.inf
        while k < 4000:
            sim.step(20, info=False)
            k += 20
            cur = sim.read_fields("up13")["up13"]
            ch = np.linalg.norm(cur - prev) / np.linalg.norm(prev)
            if ch < 1e-4:
                break
            prev = cur
    assert k == taken and ch == pytest.approx(change, rel=1e-9)


def test_mobility_field_cleared_and_uniform_factor_rescales_time():
    n = 64
    up0 = inputs.random_up(n, seed=8, ell=6.0)
    p = Params(n1=n, n2=n, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_STRESS, sigma_bar13=0.02, cfl=0.4)
    with FDM(p) as sim:
        sim.set_plastic_distortion(up0)
        a = sim.step(10)
        ua = sim.read_fields("up13")["up13"]
        sim.set_mobility_field(np.full((n, n), 4.0))
        sim.set_plastic_distortion(up0)
        b = sim.step(10)
        ub = sim.read_fields("up13")["up13"]
        sim.set_mobility_field(None)
        sim.set_plastic_distortion(up0)
        c = sim.step(10)
        uc = sim.read_fields("up13")["up13"]
        with pytest.raises(FDMError):
            sim.set_mobility_field(np.full((n, n), -1.0))
    assert np.abs(ub - ua).max() < 1e-12 * np.abs(ua).max()
    assert b.t == pytest.approx(a.t / 4.0, rel=1e-13)
    np.testing.assert_array_equal(uc, ua)
    assert c.t == a.t


@pytest.mark.parametrize("shape", [(128, 128), (64, 256)])
@pytest.mark.parametrize("precision,tol", [(B.FP64, TOL64), (B.DF64, TOL64), (B.MIXED, TOL_MIXED)])
def test_coupled_random_field(shape, precision, tol):
    """Config-2 shape at reduced size: random field, stress-driven velocity M = 1, strain
    ramp 1e-4 per step, CFL 0.4 adaptive, minmod."""
    n2, n1 = shape
    up0 = inputs.random_up(max(shape), seed=0, ell=16.0)[:n2, :n1]
    up0 = up0 - up0.mean()
    p = Params(n1=n1, n2=n2, velocity_mode=B.V_STRESS, mobility=1.0, loading_mode=B.LOAD_STRAIN_RAMP,
               eps_bar13_rate=1e-4, cfl=0.4, theta=1.0, precision=precision)
    got, info, ref, _ = run_both(p, up0=up0, steps=60)
    assert rel(got["up13"], ref.up13) < tol
    assert rel(got["tau13"], ref.tau13) < tol
    assert info.t == pytest.approx(ref.t, rel=tol)
    assert info.eps_bar13 == pytest.approx(ref.eps_bar13, rel=1e-15)
    assert info.sigma_bar13 == pytest.approx(ref.sigma_bar13, rel=tol, abs=1e-14)
    assert info.mean_up13 == pytest.approx(ref.mean_up13, rel=tol, abs=1e-13)


@pytest.mark.parametrize("time_level", [B.T_MIDPOINT, B.T_LITERAL])
@pytest.mark.parametrize("theta", [1.0, 1.5, 2.0])
@pytest.mark.parametrize("precision", [B.FP64, B.DF64])
def test_scheme_variants(time_level, theta, precision):
    """Both time levels of Sec. 3.2.2 Step 3 (reading G3) and three limiter parameters over 25
    stress-driven steps at 1e-11.  The literal time level with theta > 1 amplifies rounding
    differences (the oracle's response to a single 2^-48 perturbation of its input grows
    ~200-fold in 25 steps), so the double words, which round at 2^-48 every step, are held
    there to ten times the oracle's own spread under a perturbation of that size."""
    n = 64
    up0 = inputs.random_up(n, seed=4, ell=5.0)
    p = Params(n1=n, n2=n, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_STRESS, sigma_bar13=0.02,
               mobility=2.0, cfl=0.7, theta=theta, time_level=time_level, precision=precision)
    got, _, ref, _ = run_both(p, up0=up0, steps=25)
    tol = TOL64
    if precision == B.DF64 and time_level == B.T_LITERAL and theta > 1.0:
        pert = up0 + 100 * 2.0 ** -48 * np.abs(up0).max() * np.random.default_rng(4).standard_normal(up0.shape)
        ref2, _ = oracle.run(oparams(p), pert, 25)
        tol = max(TOL64, 10 * rel(ref2.up13, ref.up13))
    assert rel(got["up13"], ref.up13) < tol


def test_zero_mean_stress_and_friction():
    n = 64
    up0 = inputs.random_up(n, seed=8, ell=6.0) + 0.3
    p = Params(n1=n, n2=n, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_ZERO_MEAN_STRESS,
               tau_y=0.01, beta=0.05, cfl=0.4, nh=2, nz=32)
    got, info, ref, _ = run_both(p, up0=up0, steps=20)
    assert rel(got["up13"], ref.up13) < TOL64
    assert info.sigma_bar13 == 0.0
    assert info.eps_bar13 == pytest.approx(ref.eps_bar13, rel=1e-12)


def test_uniform_state_and_zero_steps():
    n = 32
    p = Params(n1=n, n2=n, velocity_mode=B.V_STRESS, dt_max=0.5)
    with FDM(p) as sim:
        sim.set_plastic_distortion(np.full((n, n), 1.25))
        i0 = sim.step(0)
        assert i0.step == 0 and i0.t == 0.0
        i = sim.step(3)
        u = sim.read_fields("up13")["up13"]
    assert (u == 1.25).all()
    assert i.t == pytest.approx(1.5) and i.max_abs_v0 == 0.0


def test_restart_equals_uninterrupted_run():
    n = 64
    up0 = inputs.random_up(n, seed=12, ell=6.0)
    p = Params(n1=n, n2=n, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_STRAIN_RAMP, eps_bar13_rate=1e-3, cfl=0.4)
    with FDM(p) as a:
        a.set_plastic_distortion(up0)
        i30 = a.step(30)
        mid = a.read_fields("up13")["up13"]
        i60 = a.step(30)
        full = a.read_fields("up13")["up13"]
    with FDM(p) as b:
        b.set_plastic_distortion(mid)
        b.set_clock(30, i30.t)   # the strain ramp is driven by the step counter
        j60 = b.step(30)
        again = b.read_fields("up13")["up13"]
    np.testing.assert_array_equal(again, full)
    assert j60.t == i60.t and j60.step == 60


def test_step_before_state_is_an_error():
    with FDM(Params(n1=32, n2=32)) as sim:
        with pytest.raises(FDMError) as e:
            sim.step(1)
        assert e.value.status == B.FDM_ERR_STATE


def test_nonfinite_state_reported():
    n = 32
    up = np.zeros((n, n))
    up[3, 4] = 1e308
    p = Params(n1=n, n2=n, velocity_mode=B.V_STRESS)
    with FDM(p) as sim:
        sim.set_plastic_distortion(up)
        with pytest.raises(FDMError) as e:
            sim.step(2)
        assert e.value.status == B.FDM_ERR_NONFINITE


@pytest.mark.parametrize("precision", [B.FP64, B.DF64, B.MIXED])
def test_nonfinite_input_rejected_and_state_kept(precision):
    """A field with a NaN or an infinity is refused (invalid argument) and the state, step
    and time of the handle stay as they were."""
    n = 32
    up0 = inputs.random_up(n, seed=18, ell=4.0)
    p = Params(n1=n, n2=n, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_STRAIN_RAMP, eps_bar13_rate=1e-3,
               cfl=0.4, precision=precision)
    with FDM(p) as sim:
        sim.set_plastic_distortion(up0)
        i0 = sim.step(3)
        before = sim.read_fields("up13")["up13"]
        for bad in (np.nan, np.inf, -np.inf):
            u = up0.copy()
            u[5, 7] = bad
            with pytest.raises(FDMError) as e:
                sim.set_plastic_distortion(u)
            assert e.value.status == B.FDM_ERR_INVALID_ARG
            np.testing.assert_array_equal(sim.read_fields("up13")["up13"], before)
            i = sim.info()
            assert i.step == i0.step == 3 and i.t == i0.t
        assert sim.step(1).step == 4


def test_largest_grid_runs_and_conserves():
    """Maximum size 4096^2 FP64: one coupled step; the total Burgers vector stays 0 and the
    mean stress equals the macroscopic stress."""
    n = 4096
    up0 = inputs.random_up(n, seed=1, ell=16.0)
    p = Params(n1=n, n2=n, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_STRAIN_RAMP, eps_bar13_rate=1e-4, cfl=0.4)
    with FDM(p) as sim:
        sim.set_plastic_distortion(up0)
        info = sim.step(1)
        f = sim.read_fields("tau13", "up13")
    assert np.isfinite(f["tau13"]).all() and np.isfinite(f["up13"]).all()
    assert abs(info.sum_a12_pos + info.sum_a12_neg) < 1e-8 * info.sum_abs_alpha
    # the static solve of step 0 had sigma_bar13 = -mu (nh/nz) <U13^0>
    sig0 = -(1 / 2.6) * (4 / n) * up0.mean()
    assert abs(f["tau13"].mean() - sig0) < 1e-12 * np.abs(f["tau13"]).max()
