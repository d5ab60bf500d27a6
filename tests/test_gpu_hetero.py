"""Heterogeneous elasticity (Sec. 3.1.2, heterogeneous medium) for a plastic layer filling the
cell: the GPU fixed-point iteration against the oracle's, iterate for iterate, in every
precision and loading mode; the homogeneous limit against the layer solve; convergence and
equilibrium at 1024^2."""
import numpy as np
import pytest

import oracle
from paper_1911_03225_gb300 import FDM, FDMError, Params, inputs
from paper_1911_03225_gb300 import binding as B

pytestmark = pytest.mark.gpu

MU = 1 / 2.6   # E = 1, nu = 0.3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def modulus_factor(n2, n1, seed, lo=0.25, hi=1.0, ell=3.0):
    rng = np.random.default_rng(seed)
    F = np.fft.fft2(rng.standard_normal((n2, n1)))
    k2 = np.fft.fftfreq(n2)[:, None] * 2 * np.pi
    k1 = np.fft.fftfreq(n1)[None, :] * 2 * np.pi
    f = np.real(np.fft.ifft2(F * np.exp(-(k1 ** 2 + k2 ** 2) * ell ** 2 / 4)))
    f = (f - f.min()) / (f.max() - f.min())
    return lo + (hi - lo) * f


def params(n1, n2, precision, stress):
    if stress:
        return Params(n1=n1, n2=n2, nz=8, nh=8, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_STRESS,
                      sigma_bar13=0.02, precision=precision)
    return Params(n1=n1, n2=n2, nz=8, nh=8, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_STRAIN_RAMP,
                  eps_bar13_0=1e-3, eps_bar13_rate=1e-4, precision=precision)


@pytest.mark.parametrize("precision,tol", [(B.FP64, 1e-11), (B.DF64, 1e-11), (B.MIXED, 1e-5)])
@pytest.mark.parametrize("stress", [True, False])
def test_hetero_iterates_match_oracle(precision, tol, stress):
    """25 iterations exactly (tolerance 0) on a 64 x 32 grid, modulus contrast 4, random
    plastic field with Nyquist content."""
    n1, n2 = 64, 32
    up0 = inputs.random_up(64, seed=19, ell=4.0)[:n2, :n1].copy()
    f = modulus_factor(n2, n1, 20)
    with FDM(params(n1, n2, precision, stress)) as sim:
        sim.set_plastic_distortion(up0)
        s13, s23, it, r = sim.static_solve_heterogeneous(f, tol=0.0, max_iter=25)
        tau = sim.read_fields("tau13")["tau13"]
        assert sim.info().step == 0
    load = 0.02 if stress else 1e-3
    o13, o23, oit, orr = oracle.hetero_antiplane(MU * f, up0, stress, load, tol=0.0, max_iter=25)
    assert it == oit == 25
    assert rel(s13, o13) < tol and rel(s23, o23) < tol
    if precision == B.MIXED:
        assert r < 1e-5   # the last increment is below FP32 rounding of the field
    else:
        assert r == pytest.approx(orr, rel=1e-8)
    np.testing.assert_array_equal(tau, s13)


def test_hetero_homogeneous_modulus_is_the_layer_solve():
    n = 64
    up0 = inputs.random_up(n, seed=21, ell=4.0)
    with FDM(params(n, n, B.FP64, True)) as sim:
        sim.set_plastic_distortion(up0)
        sim.static_solve()
        tau = sim.read_fields("tau13")["tau13"]
        s13, s23, it, r = sim.static_solve_heterogeneous(np.ones((n, n)), tol=1e-14, max_iter=5)
    assert it <= 2 and r <= 1e-14
    assert rel(s13, tau) < 1e-13


def test_hetero_converges_at_scale_and_is_in_equilibrium():
    """1024^2, contrast 4, stress control: converged to 1e-12 within the basic scheme's rate
    ((kappa - 1)/(kappa + 1) = 0.6 per iteration); the returned stress is divergence free off
    the Nyquist indices and its mean is the prescribed stress."""
    n = 1024
    up0 = inputs.random_up(n, seed=22, ell=16.0)
    f = modulus_factor(n, n, 23, ell=24.0)
    with FDM(params(n, n, B.FP64, True)) as sim:
        sim.set_plastic_distortion(up0)
        s13, s23, it, r = sim.static_solve_heterogeneous(f, tol=1e-12, max_iter=200)
    assert r <= 1e-12 and it <= 80
    assert s13.mean() == pytest.approx(0.02, abs=1e-12)
    k1 = 2 * np.pi * np.fft.fftfreq(n)[None, :]
    k2 = 2 * np.pi * np.fft.fftfreq(n)[:, None]
    inner = (np.abs(k1) < np.pi - 1e-9) & (np.abs(k2) < np.pi - 1e-9)
    S13 = np.fft.fft2(s13)
    div = k1 * S13 + k2 * np.fft.fft2(s23)
    assert np.abs(div[inner]).max() < 1e-9 * np.abs(S13).max()


def test_hetero_invalid_arguments():
    n = 32
    with FDM(Params(n1=n, n2=n, nz=32, nh=4)) as sim:   # layer thinner than the cell
        sim.set_plastic_distortion(np.zeros((n, n)))
        with pytest.raises(FDMError) as e:
            sim.static_solve_heterogeneous(np.ones((n, n)))
        assert e.value.status == B.FDM_ERR_INVALID_ARG
    with FDM(params(n, n, B.FP64, True)) as sim:
        sim.set_plastic_distortion(np.zeros((n, n)))
        bad = np.ones((n, n))
        bad[3, 3] = 0.0
        with pytest.raises(FDMError) as e:
            sim.static_solve_heterogeneous(bad)
        assert e.value.status == B.FDM_ERR_INVALID_ARG


def coupled_hetero(n1, n2, precision, loading=B.LOAD_STRAIN_RAMP):
    return Params(n1=n1, n2=n2, nz=8, nh=8, velocity_mode=B.V_STRESS, loading_mode=loading, eps_bar13_rate=1e-4,
                  sigma_bar13=0.0, cfl=0.4, theta=1.0, precision=precision)


@pytest.mark.parametrize("precision,tol", [(B.FP64, 1e-11), (B.DF64, 1e-11), (B.MIXED, 1e-5)])
def test_hetero_steps_match_oracle(precision, tol):
    """Eight coupled steps (stress-driven, strain ramp, CFL 0.4) with the heterogeneous static
    problem in every step, 20 iterations each, against the oracle's time loop."""
    n1, n2 = 64, 32
    up0 = inputs.random_up(64, seed=24, ell=4.0)[:n2, :n1].copy()
    f = modulus_factor(n2, n1, 25)
    p = coupled_hetero(n1, n2, precision)
    with FDM(p) as sim:
        sim.set_plastic_distortion(up0)
        sim.set_shear_modulus_field(f, tol=0.0, max_iter=20)
        info = sim.step(8)
        got = sim.read_fields("up13", "tau13")
    op = oracle.Params(n1=n1, n2=n2, nz=8, nh=8, velocity_mode=1, loading_mode=1, eps_bar13_rate=1e-4, cfl=0.4,
                       theta=1.0)
    ref, rc = oracle.run(op, up0, 8, shear_modulus=MU * f, hetero_tol=0.0, hetero_max_iter=20)
    assert rc == 0 and info.step == 8
    assert rel(got["up13"], ref.up13) < tol
    assert rel(got["tau13"], ref.tau13) < (tol if precision != B.MIXED else 1e-4)
    assert info.t == pytest.approx(ref.t, rel=tol)


def test_hetero_uniform_modulus_steps_equal_layer_steps():
    n = 64
    up0 = inputs.random_up(n, seed=26, ell=4.0)
    p = coupled_hetero(n, n, B.FP64)
    with FDM(p) as a, FDM(p) as b:
        a.set_plastic_distortion(up0)
        b.set_plastic_distortion(up0)
        b.set_shear_modulus_field(np.ones((n, n)), tol=1e-14, max_iter=5)
        ia, ib = a.step(10), b.step(10)
        ua, ub = a.read_fields("up13")["up13"], b.read_fields("up13")["up13"]
        with pytest.raises(FDMError) as e:
            b.enqueue_phase(0)
        assert e.value.status == B.FDM_ERR_STATE
        b.set_shear_modulus_field(None)
        b.enqueue_phase(0)
    assert rel(ub, ua) < 1e-11
    assert ib.t == pytest.approx(ia.t, rel=1e-11)


def test_hetero_steps_at_scale_never_increase_the_energy():
    """512^2, contrast 4, zero macroscopic stress, stress-driven motion: the stored energy
    1/2 sum (sigma13^2 + sigma23^2) / mu falls between checkpoints."""
    n = 512
    up0 = inputs.random_up(n, seed=27, ell=16.0)
    f = modulus_factor(n, n, 28, ell=24.0)
    p = coupled_hetero(n, n, B.FP64, loading=B.LOAD_STRESS)
    w = []
    with FDM(p) as sim:
        sim.set_plastic_distortion(up0)
        sim.set_shear_modulus_field(f, tol=1e-12, max_iter=200)
        for _ in range(5):
            s13, s23, it, r = sim.static_solve_heterogeneous(f, tol=1e-12, max_iter=200)
            w.append(0.5 * float(np.sum((s13 ** 2 + s23 ** 2) / (MU * f))))
            sim.step(10)
    w = np.array(w)
    assert (np.diff(w) < 0).all(), w


# ------------------------------------------------------------------ layer thinner than the cell
def layer_params(n1, n2, nz, nh, stress):
    common = dict(n1=n1, n2=n2, nz=nz, nh=nh, velocity_mode=B.V_STRESS, precision=B.FP64)
    if stress:
        return Params(loading_mode=B.LOAD_STRESS, sigma_bar13=0.02, **common)
    return Params(loading_mode=B.LOAD_STRAIN_RAMP, eps_bar13_0=1e-3, eps_bar13_rate=1e-4, **common)


@pytest.mark.parametrize("stress", [True, False])
def test_hetero_layer_iterates_match_oracle(stress):
    """A layer of 3 planes in a cell of 16 (Sec. 3.1.2 heterogeneous medium, Sec. 3.2.1 layer),
    modulus contrast 4 uniform through the depth, 25 iterations exactly: the GPU iterates the
    independent x3 modes, the oracle the full 3-D strain field; the layer average of sigma13
    and sigma13 on planes in, at the edge of and far from the layer agree."""
    n1, n2, nz, nh = 64, 32, 16, 3
    up0 = inputs.random_up(64, seed=21, ell=4.0)[:n2, :n1].copy()
    f = modulus_factor(n2, n1, 22)
    planes = [0, 1, 2, 3, 8, 15]
    p = layer_params(n1, n2, nz, nh, stress)
    with FDM(p) as sim:
        sim.set_plastic_distortion(up0)
        tau, got_planes, it, r = sim.static_solve_heterogeneous_layer(f, tol=0.0, max_iter=25, planes=planes)
        assert sim.info().step == 0
    load = 0.02 if stress else 1e-3
    ref, ref_planes, it_o, r_o = oracle.hetero_layer(f, up0, nz, nh, MU, 0.3, stress, load, tol=0.0, max_iter=25,
                                                     planes=True)
    assert it == it_o == 25 and r == pytest.approx(r_o, rel=1e-9)
    assert rel(tau, ref) < 1e-11
    assert rel(got_planes, ref_planes[planes]) < 1e-11


def test_hetero_layer_homogeneous_limit_and_filled_cell():
    """A uniform modulus gives the layer solve's tau13 (one iteration is exact); a layer filling
    the cell gives the antiplane solver's sigma13 iterate for iterate."""
    n1, n2 = 64, 64
    up0 = inputs.random_up(64, seed=23, ell=5.0)
    with FDM(layer_params(n1, n2, 32, 4, True)) as sim:
        sim.set_plastic_distortion(up0)
        sim.static_solve()
        ref = sim.read_fields("tau13")["tau13"]
        tau, _, it, _ = sim.static_solve_heterogeneous_layer(np.ones((n2, n1)), tol=0.0, max_iter=2)
    assert rel(tau, ref) < 1e-12
    f = modulus_factor(n2, n1, 24)
    with FDM(layer_params(n1, n2, 8, 8, True)) as sim:
        sim.set_plastic_distortion(up0)
        s13, _, it_a, r_a = sim.static_solve_heterogeneous(f, tol=0.0, max_iter=20)
        tau, planes, it, r = sim.static_solve_heterogeneous_layer(f, tol=0.0, max_iter=20, planes=[0, 5])
    assert it == it_a == 20 and r == pytest.approx(r_a, rel=1e-9)
    assert rel(tau, s13) < 1e-12 and rel(planes[1], s13) < 1e-12


def test_hetero_layer_at_scale_converges_symmetric_about_the_layer():
    """512^2 cell 16 deep, layer of 4 planes, contrast 4: converges to 1e-10; sigma13 is even about
    the layer's mid-plane (x3 = 1.5), and differs from the homogeneous layer solve."""
    n, nz, nh = 512, 16, 4
    up0 = inputs.random_up(n, seed=25, ell=16.0)
    f = modulus_factor(n, n, 26, ell=12.0)
    with FDM(layer_params(n, n, nz, nh, True)) as sim:
        sim.set_plastic_distortion(up0)
        tau, planes, it, r = sim.static_solve_heterogeneous_layer(f, tol=1e-10, max_iter=300,
                                                                  planes=[0, 3, 1, 2, 6, 13])
        sim.static_solve()
        homog = sim.read_fields("tau13")["tau13"]
    assert it < 300 and r <= 1e-10
    scale = np.abs(planes).max()
    assert np.abs(planes[0] - planes[1]).max() < 1e-9 * scale
    assert np.abs(planes[2] - planes[3]).max() < 1e-9 * scale
    assert np.abs(planes[4] - planes[5]).max() < 1e-9 * scale   # x3 = 6 and 13 -> 1.5 +- 4.5
    assert rel(tau, homog) > 1e-2


def test_hetero_layer_rejects_other_precisions_and_odd_depth():
    n = 32
    up0 = inputs.random_up(n, seed=27, ell=4.0)
    for p in (Params(n1=n, n2=n, nz=8, nh=2, precision=B.MIXED), Params(n1=n, n2=n, nz=9, nh=2)):
        with FDM(p) as sim:
            sim.set_plastic_distortion(up0)
            with pytest.raises(FDMError) as e:
                sim.static_solve_heterogeneous_layer(np.ones((n, n)), max_iter=2)
            assert e.value.status == B.FDM_ERR_INVALID_ARG
