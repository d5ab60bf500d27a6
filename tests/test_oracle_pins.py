"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each checks it against a closed
form, a textbook routine, a brute-force construction, a symmetry of the continuous
problem, or a number printed in the paper.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1911_03225_gb300 import inputs, units

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- FFT
@pytest.mark.parametrize("n", [2, 4, 8, 16])
def test_fft_equals_direct_dft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    j = np.arange(n)
    dft = np.array([np.sum(x * np.exp(-2j * np.pi * k * j / n)) for k in range(n)])
    np.testing.assert_allclose(oracle.fft1d(x, -1), dft, atol=1e-12)
    idft = np.array([np.sum(x * np.exp(2j * np.pi * k * j / n)) for k in range(n)])
    np.testing.assert_allclose(oracle.fft1d(x, +1), idft, atol=1e-12)


def test_fft2d_equals_numpy():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((16, 64)) + 1j * rng.standard_normal((16, 64))
    np.testing.assert_allclose(oracle.fft2d(x, -1), np.fft.fft2(x), atol=1e-11)
    np.testing.assert_allclose(oracle.fft2d(x, +1), np.fft.ifft2(x) * x.size, atol=1e-11)


# --------------------------------------------------------------------------- static problem
def test_layer_symbol_special_directions():
    # shear eigenstrain e1(x)e3 varying along e1 or e3 is compatible -> no stress;
    # varying along e2 it is fully constrained -> sigma13 = -mu U13.
    mu, nu = 0.4, 0.3
    assert oracle.layer_symbol(1, 0, 0, mu, nu) == 0.0
    assert oracle.layer_symbol(0, 0, 1, mu, nu) == 0.0
    assert oracle.layer_symbol(0, 1, 0, mu, nu) == pytest.approx(-mu, abs=1e-15)


def _isotropic_C(lam, mu):
    d = np.eye(3)
    return (lam * np.einsum("ij,kl->ijkl", d, d)
            + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))


def _tensor_green_layer_tau(phi, nz, nh, lam, mu, sigma_bar13):
    """Layer-averaged sigma13 from the general Green-operator formula (see below)."""
    return _tensor_green_sigma13(phi, nz, nh, lam, mu, sigma_bar13)[:nh].mean(axis=0)


def _tensor_green_sigma13(phi, nz, nh, lam, mu, sigma_bar13):
    """sigma13 on every plane of the 3-D cell from the general Green-operator formula of
    Sec. 3.1.2, sigma-hat = (C0:Gamma0-hat - I):C0:U^p-hat, Gamma0-hat =
    [xi (x) (xi.C0.xi)^-1 (x) xi]^(s), evaluated with full 3x3x3x3 tensors."""
    n2, n1 = phi.shape
    C0 = _isotropic_C(lam, mu)
    I4 = 0.5 * (np.einsum("ik,jl->ijkl", np.eye(3), np.eye(3)) + np.einsum("il,jk->ijkl", np.eye(3), np.eye(3)))
    U = np.zeros((nz, n2, n1))
    U[:nh] = phi[None]
    Uh = np.fft.fftn(U)                      # axes (x3, x2, x1)
    f3, f2, f1 = (np.fft.fftfreq(m) * m for m in (nz, n2, n1))
    s13 = np.zeros_like(Uh)
    for a, b, c in itertools.product(range(nz), range(n2), range(n1)):
        xi = np.array([f1[c] / n1, f2[b] / n2, f3[a] / nz])
        if not xi.any():
            continue
        A = np.einsum("j,ijkl,l->ik", xi, C0, xi)
        Ai = np.linalg.inv(A)
        G = np.einsum("i,jk,l->ijkl", xi, Ai, xi)
        # minor and major symmetrisation
        G = 0.25 * (G + G.transpose(1, 0, 2, 3) + G.transpose(0, 1, 3, 2) + G.transpose(1, 0, 3, 2))
        G = 0.5 * (G + G.transpose(2, 3, 0, 1))
        Up = np.zeros((3, 3), dtype=complex)
        Up[0, 2] = Uh[a, b, c]
        op = np.einsum("ijmn,mnkl->ijkl", C0, G) - I4
        s = np.einsum("ijkl,klpq,pq->ij", op, C0, Up)
        s13[a, b, c] = s[0, 2]
    s13[0, 0, 0] = sigma_bar13 * U.size
    return np.real(np.fft.ifftn(s13))


def test_static_layer_matches_tensor_green_operator():
    n, nz, nh = 8, 8, 4
    E, nu = 1.0, 0.3
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    phi = np.random.default_rng(3).standard_normal((n, n))
    K = oracle.kernel_table(n, n, nz, nh, mu, nu)
    tau = oracle.static_tau(phi, K, 0.123)
    ref = _tensor_green_layer_tau(phi, nz, nh, lam, mu, 0.123)
    np.testing.assert_allclose(tau, ref, atol=1e-13, rtol=0)


def test_stress13_planes_match_tensor_green_operator():
    """sigma13 through the whole 3-D cell (inside and outside the layer) against the general
    tensor formula on an 8 x 8 x 8 cell, and its average over the layer planes equals the
    layer-reduced tau13 (the reduction K(xi1, xi2) of Sec. 3.2.1)."""
    n, nz, nh = 8, 8, 3
    E, nu = 1.0, 0.3
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    phi = np.random.default_rng(4).standard_normal((n, n))
    ref = _tensor_green_sigma13(phi, nz, nh, lam, mu, 0.07)
    got = oracle.stress13_planes(phi, nz, nh, mu, nu, 0.07, list(range(nz)))
    np.testing.assert_allclose(got, ref, atol=1e-13, rtol=0)
    K = oracle.kernel_table(n, n, nz, nh, mu, nu)
    np.testing.assert_allclose(got[:nh].mean(axis=0), oracle.static_tau(phi, K, 0.07), atol=1e-13, rtol=0)


def test_stress13_planes_of_a_full_layer_are_the_plane_problem():
    """nh = nz: the plastic distortion fills the cell, sigma13 no longer varies in x3 and every
    plane carries the layer result."""
    n = 16
    mu, nu = 1 / 2.6, 0.3
    phi = np.random.default_rng(5).standard_normal((n, n))
    got = oracle.stress13_planes(phi, 8, 8, mu, nu, 0.0, [0, 3, 7])
    tau = oracle.static_tau(phi, oracle.kernel_table(n, n, 8, 8, mu, nu), 0.0)
    for g in got:
        np.testing.assert_allclose(g, tau, atol=1e-12, rtol=0)


def _tensor_green_stress(phi, nz, nh, lam, mu, sigma_bar13):
    """All six stress components on every plane of the 3-D cell from the general tensor
    formula of Sec. 3.1.2 (as _tensor_green_sigma13), keyed by Voigt name."""
    n2, n1 = phi.shape
    C0 = _isotropic_C(lam, mu)
    I4 = 0.5 * (np.einsum("ik,jl->ijkl", np.eye(3), np.eye(3)) + np.einsum("il,jk->ijkl", np.eye(3), np.eye(3)))
    U = np.zeros((nz, n2, n1))
    U[:nh] = phi[None]
    Uh = np.fft.fftn(U)
    f3, f2, f1 = (np.fft.fftfreq(m) * m for m in (nz, n2, n1))
    S = np.zeros((3, 3) + Uh.shape, dtype=complex)
    for a, b, c in itertools.product(range(nz), range(n2), range(n1)):
        xi = np.array([f1[c] / n1, f2[b] / n2, f3[a] / nz])
        if not xi.any():
            continue
        Ai = np.linalg.inv(np.einsum("j,ijkl,l->ik", xi, C0, xi))
        G = np.einsum("i,jk,l->ijkl", xi, Ai, xi)
        G = 0.25 * (G + G.transpose(1, 0, 2, 3) + G.transpose(0, 1, 3, 2) + G.transpose(1, 0, 3, 2))
        G = 0.5 * (G + G.transpose(2, 3, 0, 1))
        Up = np.zeros((3, 3), dtype=complex)
        Up[0, 2] = Uh[a, b, c]
        op = np.einsum("ijmn,mnkl->ijkl", C0, G) - I4
        S[:, :, a, b, c] = np.einsum("ijkl,klpq,pq->ij", op, C0, Up)
    S[0, 2, 0, 0, 0] = S[2, 0, 0, 0, 0] = sigma_bar13 * U.size
    real = np.real(np.fft.ifftn(S, axes=(2, 3, 4)))
    idx = {"11": (0, 0), "22": (1, 1), "33": (2, 2), "23": (1, 2), "13": (0, 2), "12": (0, 1)}
    return {k: real[i, j] for k, (i, j) in idx.items()}


def _band_limited(phi):
    """Drops the Nyquist row and column of the 2-D spectrum (no mode whose odd symbols the
    Nyquist reading zeroes)."""
    F = np.fft.fft2(phi)
    n2, n1 = phi.shape
    F[n2 // 2, :] = 0.0
    F[:, n1 // 2] = 0.0
    return np.real(np.fft.ifft2(F))


def test_stress_planes_all_components_match_tensor_green_operator():
    """Every stress component through the 3-D cell against the general tensor formula on an
    8 x 4 x 8 cell.  The input has no Nyquist content in x1, x2 and the layer is 4 planes
    deep (chi-hat vanishes at the x3 Nyquist index), so the reading for odd symbols at
    Nyquist indices plays no part; the 13 component is the sigma13 routine's."""
    n1, n2, nz, nh = 8, 4, 8, 4
    E, nu = 1.0, 0.3
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    phi = _band_limited(np.random.default_rng(6).standard_normal((n2, n1)))
    ref = _tensor_green_stress(phi, nz, nh, lam, mu, 0.05)
    for comp in oracle.STRESS_COMPONENTS:
        got = oracle.stress_planes(phi, nz, nh, mu, nu, 0.05, comp, list(range(nz)))
        assert np.abs(ref[comp]).max() > 1e-2
        np.testing.assert_allclose(got, ref[comp], atol=1e-13, rtol=0, err_msg=comp)
    np.testing.assert_allclose(oracle.stress_planes(phi, nz, 3, mu, nu, 0.05, "13", [0, 2, 5]),
                               oracle.stress13_planes(phi, nz, 3, mu, nu, 0.05, [0, 2, 5]), atol=1e-15, rtol=0)


def test_stress_planes_are_in_equilibrium():
    """div sigma = 0 (Sec. 3.1.2 equilibrium) for the assembled 3-D field: sum_j xi_j
    sigma-hat_ij vanishes at every mode off the Nyquist indices."""
    n1, n2, nz, nh = 8, 8, 8, 2
    mu, nu = 0.4, 0.25
    phi = _band_limited(np.random.default_rng(7).standard_normal((n2, n1)))
    sig = {c: oracle.stress_planes(phi, nz, nh, mu, nu, 0.0, c, list(range(nz))) for c in oracle.STRESS_COMPONENTS}
    T = np.empty((3, 3, nz, n2, n1))
    for c, (i, j) in zip(oracle.STRESS_COMPONENTS, [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]):
        T[i, j] = T[j, i] = sig[c]
    Th = np.fft.fftn(T, axes=(2, 3, 4))
    f3, f2, f1 = np.meshgrid(np.fft.fftfreq(nz), np.fft.fftfreq(n2), np.fft.fftfreq(n1), indexing="ij")
    div = np.einsum("jabc,ijabc->iabc", np.stack([f1, f2, f3]), Th)
    inner = (np.abs(f1) < 0.5) & (np.abs(f2) < 0.5) & (np.abs(f3) < 0.5)
    assert np.abs(div[:, inner]).max() < 1e-12 * np.abs(Th).max()
    assert np.abs(Th).max() > 1.0


def test_stress_planes_reflection_symmetry_about_the_layer():
    """Reflecting x3 about the layer's mid-plane maps the eigen-distortion U13 e1 (x) e3 to
    minus itself, so the stress obeys R sigma(x) R = -sigma(R x): 13 and 23 are even about
    the mid-plane, 11, 22, 33 and 12 odd.  Odd layer (mid-plane on a voxel plane), input
    with Nyquist content."""
    n, nz, nh = 8, 16, 3
    mu, nu = 1 / 2.6, 0.3
    phi = np.random.default_rng(8).standard_normal((n, n))
    c = (nh - 1) // 2
    for comp in oracle.STRESS_COMPONENTS:
        sign = 1.0 if comp in ("13", "23") else -1.0
        for d in (1, 2, 5):
            up, dn = oracle.stress_planes(phi, nz, nh, mu, nu, 0.0, comp, [(c + d) % nz, (c - d) % nz])
            np.testing.assert_allclose(up, sign * dn, atol=1e-13, rtol=0, err_msg=comp)
        if sign < 0:
            mid = oracle.stress_planes(phi, nz, nh, mu, nu, 0.0, comp, [c])[0]
            np.testing.assert_allclose(mid, 0.0, atol=1e-13)


def test_stress_planes_of_a_full_layer_are_antiplane_shear():
    """nh = nz: U13 no longer varies along x3 and the problem is antiplane shear (displacement
    u3 only): mu lap u3 = mu d1 U13, sigma13 = mu (d1 u3 - U13), sigma23 = mu d2 u3, the other
    components vanish.  u3 from a spectral Poisson solve."""
    n1, n2, nz = 16, 8, 4
    mu, nu = 0.35, 0.2
    phi = _band_limited(np.random.default_rng(9).standard_normal((n2, n1)))
    k1 = 2 * np.pi * np.fft.fftfreq(n1)[None, :]
    k2 = 2 * np.pi * np.fft.fftfreq(n2)[:, None]
    lap = -(k1 ** 2 + k2 ** 2)
    lap[0, 0] = 1.0
    rhs = 1j * k1 * np.fft.fft2(phi)
    u3h = rhs / lap
    u3h[0, 0] = 0.0
    d1 = np.real(np.fft.ifft2(1j * k1 * u3h))
    d2 = np.real(np.fft.ifft2(1j * k2 * u3h))
    # the mean of sigma13 is the macroscopic stress (the xi = 0 term)
    want = {"13": mu * (d1 - (phi - phi.mean())) + 0.01, "23": mu * d2}
    for comp in oracle.STRESS_COMPONENTS:
        got = oracle.stress_planes(phi, nz, nz, mu, nu, 0.01, comp, [0, 1, 3])
        for g in got:
            np.testing.assert_allclose(g, want.get(comp, 0.0), atol=1e-13, rtol=0, err_msg=comp)


def test_stress_planes_nyquist_reading():
    """Reading G8 for the cell: a field made of the x1 Nyquist mode gives no stress in the
    components whose symbol is odd in n1 (11, 22, 33, 23); 13 and 12 see it."""
    n1, n2, nz, nh = 8, 8, 8, 3
    x1 = np.arange(n1)[None, :]
    x2 = np.arange(n2)[:, None]
    phi = np.cos(np.pi * x1) * np.cos(2 * np.pi * x2 / n2)
    for comp in oracle.STRESS_COMPONENTS:
        got = oracle.stress_planes(phi, nz, nh, 0.4, 0.3, 0.0, comp, [0, 1, 4])
        if comp in ("11", "22", "33", "23"):
            assert np.abs(got).max() == 0.0, comp
        elif comp == "13":
            assert np.abs(got).max() > 0.05
    # 12 (odd in n2 and n3) sees the x1 Nyquist mode through its x2 and x3 variation
    assert np.abs(oracle.stress_planes(phi, nz, nh, 0.4, 0.3, 0.0, "12", [0, 1, 4])).max() > 1e-3


def _spectral_derivative_matrix(n):
    """Dense first-derivative matrix of the trigonometric interpolant on n periodic
    nodes (unit spacing), Nyquist mode dropped, built by direct trig sums."""
    j = np.arange(n)
    diff = j[:, None] - j[None, :]
    D = np.zeros((n, n))
    for k in range(-(n // 2) + 1, n // 2):
        w = 2 * np.pi * k / n
        # (1/n) sum_k i w exp(i w (j-l)) -> real part -w sin(w (j - l)) / n
        D += -w * np.sin(w * diff) / n
    return D


def test_static_layer_matches_dense_real_space_solve():
    """Brute force: assemble div(C0:(grad_s u - eps^p)) = 0 on an 8x8x8 periodic cell with
    dense spectral differentiation matrices, solve for u by least squares, average sigma13
    over the layer.  Independent of the Green operator and of the layer symbol."""
    n, nz, nh = 8, 8, 4
    E, nu = 1.0, 0.3
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    rng = np.random.default_rng(7)
    phi = rng.standard_normal((n, n))
    ph = np.fft.fft2(phi)
    ph[n // 2, :] = 0.0
    ph[:, n // 2] = 0.0              # no in-plane Nyquist content (odd symbols vanish there)
    phi = np.real(np.fft.ifft2(ph))
    D = _spectral_derivative_matrix(n)
    I = np.eye(n)
    d1 = np.kron(I, np.kron(I, D))   # flat index (x3, x2, x1), x1 fastest
    d2 = np.kron(I, np.kron(D, I))
    d3 = np.kron(D, np.kron(I, I))
    d = [d1, d2, d3]
    L = d1 @ d1 + d2 @ d2 + d3 @ d3
    m = n ** 3
    A = np.zeros((3 * m, 3 * m))
    for i in range(3):
        for k in range(3):
            blk = (lam + mu) * d[i] @ d[k]
            if i == k:
                blk = blk + mu * L
            A[i * m:(i + 1) * m, k * m:(k + 1) * m] = blk
    U = np.zeros((nz, n, n))
    U[:nh] = phi[None]
    u_flat = U.ravel()
    b = np.zeros(3 * m)
    b[0:m] = mu * (d3 @ u_flat)          # d_3 (2 mu eps^p_13)
    b[2 * m:3 * m] = mu * (d1 @ u_flat)  # d_1 (2 mu eps^p_31)
    sol = np.linalg.lstsq(A, b, rcond=1e-10)[0]
    u1, u3 = sol[0:m], sol[2 * m:3 * m]
    s13 = (mu * (d3 @ u1 + d1 @ u3) - mu * u_flat).reshape(nz, n, n)
    tau_dense = s13[:nh].mean(axis=0)
    # periodic u -> zero mean strain -> sigma_bar13 = -mu <U13>_cell (strain control, eps = 0)
    sig_bar = -mu * (nh / nz) * phi.mean()
    K = oracle.kernel_table(n, n, nz, nh, mu, nu)
    tau = oracle.static_tau(phi, K, sig_bar)
    np.testing.assert_allclose(tau, tau_dense, atol=1e-11, rtol=0)


def test_kernel_table_even_and_zero_at_origin():
    K = oracle.kernel_table(16, 16, 16, 4, 0.385, 0.3)
    assert K[0, 0] == 0.0
    np.testing.assert_array_equal(K, np.roll(K[::-1, :], 1, axis=0))
    np.testing.assert_array_equal(K, np.roll(K[:, ::-1], 1, axis=1))
    assert (K <= 0).all()


def test_uniform_up_gives_macroscopic_stress_only():
    K = oracle.kernel_table(16, 16, 16, 4, 0.385, 0.3)
    tau = oracle.static_tau(np.full((16, 16), 2.5), K, -0.07)
    np.testing.assert_allclose(tau, -0.07, atol=1e-15)


def test_thick_layer_limit_is_plane_problem():
    # nh = nz: the layer fills the cell, only xi3 = 0 survives, tau-hat = m(xi1,xi2,0) U-hat
    n = 16
    mu, nu = 0.385, 0.3
    K = oracle.kernel_table(n, n, n, n, mu, nu)
    k = np.fft.fftfreq(n) * n
    kx, ky = np.meshgrid(k, k)
    r2 = kx ** 2 + ky ** 2
    with np.errstate(invalid="ignore", divide="ignore"):
        ref = np.where(r2 > 0, -mu * ky ** 2 / r2, 0.0)   # m(n1, n2, 0) = -mu n2^2
    np.testing.assert_allclose(K, ref, atol=1e-14)


# --------------------------------------------------------------------------- curl inverse
def test_curl_inverse_single_mode_closed_form():
    n = 32
    x, y = np.meshgrid(np.arange(n), np.arange(n))
    k1, k2 = 3, 5
    w1, w2 = 2 * np.pi * k1 / n, 2 * np.pi * k2 / n
    phi = 0.7 * np.sin(w1 * x + w2 * y)
    a11 = -0.7 * w2 * np.cos(w1 * x + w2 * y)   # -d2 U13
    a12 = 0.7 * w1 * np.cos(w1 * x + w2 * y)    # d1 U13
    up, res, ma = oracle.curl_inverse(a11, a12, mean_up13=0.25)
    np.testing.assert_allclose(up, phi + 0.25, atol=1e-13)
    assert res < 1e-14
    np.testing.assert_allclose(ma, 0.0, atol=1e-15)
    b11, b12 = oracle.alpha_from_up(phi)
    np.testing.assert_allclose(b11, a11, atol=1e-13)
    np.testing.assert_allclose(b12, a12, atol=1e-13)


def test_curl_inverse_removes_gradient_part():
    # alpha = grad psi (curl-free, div != 0) carries no dislocation content -> U13 = 0
    n = 32
    x, y = np.meshgrid(np.arange(n), np.arange(n))
    w1, w2 = 2 * np.pi * 2 / n, 2 * np.pi * 1 / n
    a11 = w1 * np.cos(w1 * x + w2 * y)
    a12 = w2 * np.cos(w1 * x + w2 * y)
    up, res, _ = oracle.curl_inverse(a11, a12)
    np.testing.assert_allclose(up, 0.0, atol=1e-14)
    assert res == pytest.approx(1.0, abs=1e-12)


def test_curl_inverse_round_trip_random():
    u = inputs.random_up(64, seed=5, ell=6.0)
    a11, a12 = oracle.alpha_from_up(u)
    up, res, _ = oracle.curl_inverse(a11, a12, mean_up13=u.mean())
    assert res < 1e-13
    # spectral derivatives drop the Nyquist modes; compare band-limited parts
    uh = np.fft.fft2(u)
    uh[32, :] = 0
    uh[:, 32] = 0
    np.testing.assert_allclose(up, np.real(np.fft.ifft2(uh)), atol=1e-12)


# --------------------------------------------------------------------------- transport
def _rand(n2, n1, seed):
    return np.random.default_rng(seed).standard_normal((n2, n1))


def test_constant_state_is_stationary():
    phi = np.full((16, 16), 3.25)
    out = oracle.knp2d_step(phi, 1.0, 0.5, theta=2.0)
    np.testing.assert_array_equal(out, phi)


@pytest.mark.parametrize("v0", [1.0, -1.0])
@pytest.mark.parametrize("axis", [1, 0])
def test_cfl_one_shifts_monotone_data_exactly(v0, axis):
    """At |v0| dt/dx = 1 the exact solution shifts monotone data by one cell; with the
    midpoint rule (G3) the scheme reproduces it exactly at nodes whose 5-point stencil is
    strictly monotone (1-D reduction in x or in y)."""
    n = 64
    s = np.arange(n)
    prof = np.sin(2 * np.pi * s / n) + 0.3 * np.sin(4 * np.pi * s / n + 0.4)
    phi = np.tile(prof, (n, 1)) if axis == 1 else np.tile(prof[:, None], (1, n))
    out = oracle.knp2d_step(phi, v0, dt=1.0, theta=1.5, time_level=0)
    d = np.diff(prof, append=prof[0])
    checked = 0
    for j in range(n):
        win = [d[(j + o) % n] for o in (-2, -1, 0, 1)]
        if all(w > 1e-3 for w in win) or all(w < -1e-3 for w in win):
            inc = win[0] > 0
            src = (j - 1) % n if (inc == (v0 > 0)) else (j + 1) % n
            line = out[0, :] if axis == 1 else out[:, 0]
            assert line[j] == pytest.approx(prof[src], abs=1e-13)
            checked += 1
    assert checked > n // 2


def test_literal_time_level_is_not_exact_at_cfl_one():
    n = 64
    s = np.arange(n)
    prof = np.sin(2 * np.pi * s / n)
    phi = np.tile(prof, (n, 1))
    out = oracle.knp2d_step(phi, 1.0, dt=1.0, theta=1.0, time_level=1)
    assert np.abs(out[0] - np.roll(prof, 1))[5:12].max() > 1e-4


@pytest.mark.parametrize("theta", [1.0, 2.0])
@pytest.mark.parametrize("time_level", [0, 1])
def test_2d_scheme_on_x_only_data_equals_1d_scheme(theta, time_level):
    n = 64
    prof = inputs.lines_up(n)[0] + 0.1 * np.random.default_rng(2).standard_normal(n)
    v0 = np.linspace(-1, 1, n)
    out2 = oracle.knp2d_step(np.tile(prof, (8, 1)), np.tile(v0, (8, 1)), 0.4, theta, 1.0, time_level)
    out1 = oracle.knp1d_step(prof, v0, 0.4, theta, 1.0, time_level)
    for r in range(8):
        np.testing.assert_allclose(out2[r], out1, atol=1e-14, rtol=0)


@pytest.mark.parametrize("time_level", [0, 1])
def test_offset_equivariance(time_level):
    phi = _rand(32, 32, 11)
    v0 = _rand(32, 32, 12)
    a = oracle.knp2d_step(phi, v0, 0.2, 2.0, 1.0, time_level)
    b = oracle.knp2d_step(phi + 5.0, v0, 0.2, 2.0, 1.0, time_level)
    np.testing.assert_allclose(b - 5.0, a, atol=1e-12, rtol=0)


@pytest.mark.parametrize("time_level", [0, 1])
def test_symmetries(time_level):
    phi = _rand(32, 32, 21)
    v0 = _rand(32, 32, 22)
    f = lambda p, v: oracle.knp2d_step(p, v, 0.3, 1.0, 1.0, time_level)
    base = f(phi, v0)
    # periodic translation
    np.testing.assert_allclose(f(np.roll(phi, (3, -5), (0, 1)), np.roll(v0, (3, -5), (0, 1))),
                               np.roll(base, (3, -5), (0, 1)), atol=1e-13)
    # mirror x1 -> -x1 (node j -> -j)
    mx = lambda a: np.roll(a[:, ::-1], 1, axis=1)
    np.testing.assert_allclose(f(mx(phi), mx(v0)), mx(base), atol=1e-13)
    # mirror x2 -> -x2
    my = lambda a: np.roll(a[::-1, :], 1, axis=0)
    np.testing.assert_allclose(f(my(phi), my(v0)), my(base), atol=1e-13)
    # exchange x1 <-> x2
    np.testing.assert_allclose(f(phi.T.copy(), v0.T.copy()), base.T, atol=1e-13)
    # (U13, v0) -> (-U13, -v0) leaves phi_t + v0 |grad phi| = 0 invariant
    np.testing.assert_allclose(f(-phi, -v0), -base, atol=1e-13)


@pytest.mark.parametrize("v0", [0.8, -0.8])
def test_planar_faces_are_exact(v0):
    """On a pyramid U = A - a|x1-c| - b|x2-c| each face is a plane; away from the edges the
    interpolant is exact and the one-sided speeds select one corner, so the update is the
    exact solution U - dt v0 |grad U|."""
    n, c, a, b, dt = 64, 32, 0.7, 0.4, 0.3
    x, y = np.meshgrid(np.arange(n), np.arange(n))
    phi = 10.0 - a * np.abs(x - c) - b * np.abs(y - c)
    out = oracle.knp2d_step(phi, v0, dt, theta=2.0)
    inner = (np.abs(x - c) > 3) & (np.abs(y - c) > 3) & (np.abs(x - c) < 28) & (np.abs(y - c) < 28)
    np.testing.assert_allclose(out[inner], (phi - dt * v0 * math.hypot(a, b))[inner], atol=1e-13)


def test_no_new_extrema_random():
    phi = inputs.random_up(64, seed=3, ell=4.0)
    v0 = np.random.default_rng(4).uniform(-1, 1, (64, 64))
    for theta in (1.0, 2.0):
        out = oracle.knp2d_step(phi, v0, 0.4 / np.abs(v0).max(), theta)
        span = phi.max() - phi.min()
        assert out.max() <= phi.max() + 1e-3 * span
        assert out.min() >= phi.min() - 1e-3 * span


def _ring_error(n, L=64.0, r0=16.0, sig=2.0, T=4.0, cfl=0.4):
    h = L / n
    x = (np.arange(n) * h) - L / 2
    X, Y = np.meshgrid(x, x)
    R = np.hypot(X, Y)
    phi = inputs.ring_profile(R, r0, sig)
    dt = cfl * h
    steps = int(round(T / dt))
    for _ in range(steps):
        phi = oracle.knp2d_step(phi, -1.0, dt, theta=2.0, h=h)
    exact = inputs.ring_profile(np.maximum(R - steps * dt, 0.0), r0, sig)   # Hopf-Lax dilation
    band = np.abs(R - (r0 + steps * dt)) < 4 * sig
    return np.sqrt(np.mean((phi - exact)[band] ** 2))


def test_hopf_lax_ring_expansion_converges():
    """phi_t - |grad phi| = 0 (v0 = -1) has the Hopf-Lax solution phi(x,t) = max over the
    disc of radius t, i.e. phi0(max(r - t, 0)) for a decreasing radial profile: the loop
    radius grows as r0 + t (Sec. 4.4.1).  The error must shrink at least like h^1.5."""
    e1, e2, e3 = _ring_error(64), _ring_error(128), _ring_error(256)
    assert e2 < e1 and e3 < e2
    assert math.log2(e1 / e2) > 1.5 and math.log2(e2 / e3) > 1.5


def _square_setup(n, L=64.0, a=12.0, sig=1.5):
    """Square loop (half side a, Gaussian section sig) on an L x L periodic cell with n nodes
    per side: (U13, signed distance to the square, X, Y, h)."""
    h = L / n
    x = (np.arange(n) * h) - L / 2
    X, Y = np.meshgrid(x, x)
    sd = inputs.square_signed_distance(X, Y, a)
    return inputs.loop_profile(sd, sig), sd, X, Y, h


def _square_move(phi, v0, T, h, cfl=0.4):
    dt = cfl * h
    steps = int(round(T / dt))
    for _ in range(steps):
        phi = oracle.knp2d_step(phi, v0, dt, theta=2.0, h=h)
    return phi, steps * dt


def _rms(e, mask):
    return float(np.sqrt(np.mean(e[mask] ** 2)))


def test_square_loop_expansion_takes_the_fan_and_shrinkage_keeps_corners():
    """Sec. 4.4.2: a loop with corners admits several weak solutions; the scheme must pick the
    viscosity (Hopf-Lax) one.  With U13 = profile(signed distance to the square), profile
    decreasing, the dilation (v0 = -1) is profile(sd - t): the exterior distance turns each
    corner into an arc of radius t (expansion fan); the erosion (v0 = +1) is profile(sd + t):
    corners stay sharp.  The expanding loop must converge to the fan and stay far from the
    sharp-cornered alternative; the shrinking loop converges at order > 1.5, corners included."""
    T, sig = 6.0, 1.5
    fan, alt = {}, {}
    for n in (64, 128):
        phi0, sd, X, Y, h = _square_setup(n)
        phi, t = _square_move(phi0, -1.0, T, h)
        band = np.abs(sd - t) < 6.0
        fan[n] = _rms(phi - inputs.loop_profile(sd - t, sig), band)
        sharp = inputs.loop_profile(np.maximum(np.abs(X), np.abs(Y)) - 12.0 - t, sig)
        alt[n] = _rms(phi - sharp, band)
    assert fan[128] < fan[64]
    assert alt[128] > 0.25 and alt[128] > 3.5 * fan[128]
    shrink, corner = {}, {}
    for n in (64, 128, 256):
        phi0, sd, X, Y, h = _square_setup(n)
        phi, t = _square_move(phi0, 1.0, T, h)
        band = np.abs(sd + t) < 6.0
        err = phi - inputs.loop_profile(sd + t, sig)
        shrink[n] = _rms(err, band)
        corner[n] = _rms(err, band & (np.abs(np.abs(X) - np.abs(Y)) < 1.0))
    assert math.log2(shrink[64] / shrink[128]) > 1.5 and math.log2(shrink[128] / shrink[256]) > 1.5
    assert corner[256] < 2.5 * shrink[256]


def test_square_loop_expansion_then_shrinkage_returns_the_initial_loop():
    """Sec. 4.4.2: reversing the expanded polygonal loop brings back its initial shape: the
    closing (dilation then erosion by the same disc) of the convex sublevel sets returns
    them, so the exact solution returns U0.  The numerical round trip converges to U0,
    corners included."""
    rel, corner = {}, {}
    for n in (128, 256):
        phi0, sd, X, Y, h = _square_setup(n)
        phi, _ = _square_move(phi0, -1.0, 6.0, h)
        phi, _ = _square_move(phi, 1.0, 6.0, h)
        rel[n] = np.linalg.norm(phi - phi0) / np.linalg.norm(phi0)
        corner[n] = _rms(phi - phi0, (np.abs(sd) < 6.0) & (np.abs(np.abs(X) - np.abs(Y)) < 1.0))
    assert rel[128] < 2e-2 and rel[256] < 4e-3
    assert corner[256] < 0.5 * corner[128]


def _flat_top_ring(n, r_in, r_out, s):
    """U13 of a loop whose density is uniform across its width (Sec. 4.2: the density is
    spread uniformly over a surface of the dislocation's width), edges smoothed over s."""
    from scipy.special import erf
    c = n / 2
    x, y = np.meshgrid(np.arange(n) - c, np.arange(n) - c)
    r = np.hypot(x, y)
    rr = np.linspace(0, 4 * n, 400001)
    g = 0.5 * (erf((rr - r_in) / (math.sqrt(2) * s)) - erf((rr - r_out) / (math.sqrt(2) * s)))
    G = np.cumsum(g[::-1])[::-1] * (rr[1] - rr[0])
    return np.interp(r, rr, G), r


def _grad_mag(p):
    return np.hypot(np.roll(p, -1, 1) - p, np.roll(p, -1, 0) - p)


def test_ring_peak_density_preserved_and_radius_grows():
    """For uniform v0 the transport of |alpha| is conservative: no damping and no spreading
    (Sec. 4.1); the loop expands at unit speed (Sec. 4.4.1).  The midpoint reading (G3)
    keeps the peak; the literal one overshoots it."""
    n = 128
    phi0, r = _flat_top_ring(n, 20.0, 36.0, 1.5)
    peak0 = _grad_mag(phi0).max()
    w0 = np.sum(_grad_mag(phi0) > 0.5 * peak0)
    results = {}
    for tl in (0, 1):
        phi = phi0.copy()
        for _ in range(50):
            phi = oracle.knp2d_step(phi, -1.0, 0.4, theta=2.0, time_level=tl)
        results[tl] = phi
    mag = _grad_mag(results[0])
    assert abs(mag.max() / peak0 - 1.0) < 0.01
    assert _grad_mag(results[1]).max() / peak0 > 1.05
    # radius grows as r0 + t (t = 20): density-weighted mean radius of the band
    rmean = np.sum(mag * r) / np.sum(mag)
    rmean0 = np.sum(_grad_mag(phi0) * r) / np.sum(_grad_mag(phi0))
    assert rmean - rmean0 == pytest.approx(20.0, abs=0.5)
    # no spreading: the band area grows only with the circumference
    w = np.sum(mag > 0.5 * peak0)
    assert w / w0 == pytest.approx((28.0 + 20.0) / 28.0, rel=0.05)


def test_annihilation_matches_characteristics():
    """Two opposite edge walls moving toward each other (v0 = +1, erosion); the exact
    solution is the running minimum over [x - t, x + t] (Sec. 4.3)."""
    n = 128
    prof = inputs.lines_up(n)[0]
    phi = np.tile(prof, (4, 1))
    dt, steps = 0.5, 16
    for _ in range(steps):
        phi = oracle.knp2d_step(phi, 1.0, dt, theta=1.0)
    t = dt * steps
    xf = np.arange(n, dtype=float)
    ss = np.linspace(-t, t, 801)
    exact = np.array([np.min(np.interp(xi + ss, xf, prof, period=n)) for xi in xf])
    err = np.linalg.norm(phi[0] - exact) / np.linalg.norm(exact)
    assert err < 2e-2   # h = 1 on sigma = 3 edges; the exact solution has kinks
    # after the walls met (t > 16) the plateau and the density are gone
    for _ in range(40):
        phi = oracle.knp2d_step(phi, 1.0, dt, theta=1.0)
    assert phi.max() < 0.05 * prof.max()
    assert oracle.alpha_sums(phi)[4] < 0.05 * oracle.alpha_sums(np.tile(prof, (4, 1)))[4]


# --------------------------------------------------------------------------- reductions, loading
def test_compensated_sum_is_exact_on_hard_case():
    x = np.array([1e16, 1.0, -1e16, 3.0, 1e-3] * 1000)
    assert oracle.compensated_sum(x) == math.fsum(x)
    y = np.random.default_rng(0).standard_normal(100000) * 1e8
    assert oracle.compensated_sum(y) == pytest.approx(math.fsum(y), abs=1e-6)


def test_total_burgers_vector_vanishes_and_sums_match_numpy():
    u = inputs.random_up(32, seed=9, ell=3.0)
    s = oracle.alpha_sums(u)
    a12 = np.roll(u, -1, axis=1) - u
    a11 = -(np.roll(u, -1, axis=0) - u)
    assert abs(s[0] + s[1]) < 1e-13 and abs(s[2] + s[3]) < 1e-13
    assert s[0] == pytest.approx(a12[a12 > 0].sum(), rel=1e-13)
    assert s[4] == pytest.approx(np.hypot(a11, a12).sum(), rel=1e-13)


def test_loading_paths_on_dislocation_free_state():
    n = 16
    mu = 1.0 / 2.6
    up = np.full((n, n), 0.2)
    # strain ramp: sigma_bar = 2 mu eps - mu (nh/nz) <U13>; with uniform U13 tau = sigma_bar
    p = oracle.Params(n1=n, n2=n, velocity_mode=1, loading_mode=1, eps_bar13_rate=1e-2, cfl=0.4, dt_max=1.0)
    st, rc = oracle.run(p, up, 3)
    assert rc == 0
    eps = 1e-2 * 2
    np.testing.assert_allclose(st.tau13, 2 * mu * eps - mu * (4 / 16) * 0.2, atol=1e-15)
    assert st.eps_bar13 == pytest.approx(3e-2)
    # zero mean stress (Sec. 5.1): eps_bar = <U13>/2, tau = 0
    p = oracle.Params(n1=n, n2=n, velocity_mode=1, loading_mode=2, cfl=0.4, dt_max=1.0)
    st, rc = oracle.run(p, up, 2)
    np.testing.assert_allclose(st.tau13, 0.0, atol=1e-15)
    assert st.eps_bar13 == pytest.approx(0.5 * (4 / 16) * 0.2)
    assert st.t == pytest.approx(2.0)   # no motion -> dt = dt_max


def test_stress_driven_velocity_and_cfl_step():
    n = 32
    up = inputs.random_up(n, seed=1, ell=4.0)
    p = oracle.Params(n1=n, n2=n, velocity_mode=1, loading_mode=0, sigma_bar13=0.01, mobility=2.0, cfl=0.4)
    st, _ = oracle.run(p, up, 0)
    np.testing.assert_allclose(st.v0, -2.0 * st.tau13, atol=0)
    st1, _ = oracle.run(p, up, 1)
    assert st1.dt == pytest.approx(0.4 / np.abs(st.v0).max(), rel=1e-15)
    assert st1.tau13.mean() == pytest.approx(0.01, abs=1e-15)


@pytest.mark.parametrize("theta,tau_y", [(1.0, 0.0), (2.0, 0.0), (1.0, 0.02)])
def test_energy_never_increases_under_stress_driven_motion(theta, tau_y):
    """Sec. 3.2 (dissipation): with the linear mobility law the plastic rate is M (tau13 -
    tau_y cos(U13/beta)) |grad U13| and the dissipation (tau13 - tau_y cos) dU13/dt >= 0, so
    the stored energy -- elastic, -1/2 sum tau13 (U13 - <U13>) at zero macroscopic stress,
    plus the wiggly potential beta tau_y sin(U13/beta) -- never increases along the scheme's
    steps (a dropped term or a sign error in the static solve or the celerity law breaks it)."""
    n, beta = 32, 0.05
    up = inputs.random_up(n, seed=3, ell=4.0, rms_alpha=0.1)
    K = oracle.kernel_table(n, n, n, 4, 1 / 2.6, 0.3)
    p = oracle.Params(n1=n, n2=n, velocity_mode=1, loading_mode=0, sigma_bar13=0.0, cfl=0.4, theta=theta,
                      tau_y=tau_y, beta=beta)

    def energy(u):
        tau = oracle.static_tau(u, K, 0.0)
        return -0.5 * np.sum(tau * (u - u.mean())) + np.sum(beta * tau_y * np.sin(u / beta))

    st, _ = oracle.run(p, up, 0, K=K)
    w = [energy(up)]
    for _ in range(30):
        st, rc = oracle.run(p, up, 1, K=K, state=st)
        assert rc == 0
        w.append(energy(st.up13))
    w = np.array(w)
    assert (np.diff(w) < 0).all()
    assert w[-1] < 0.5 * w[0]


# ------------------------------------------------------------------ heterogeneous elasticity
def _smooth_field(n2, n1, seed, lo, hi, ell=3.0):
    """Seeded smooth field with values spread over [lo, hi] (a test input)."""
    rng = np.random.default_rng(seed)
    F = np.fft.fft2(rng.standard_normal((n2, n1)))
    k2 = np.fft.fftfreq(n2)[:, None] * 2 * np.pi
    k1 = np.fft.fftfreq(n1)[None, :] * 2 * np.pi
    f = np.real(np.fft.ifft2(F * np.exp(-(k1 ** 2 + k2 ** 2) * ell ** 2 / 4)))
    f = (f - f.min()) / (f.max() - f.min())
    return lo + (hi - lo) * f


@pytest.mark.parametrize("stress_control", [True, False])
def test_hetero_homogeneous_modulus_is_the_layer_solve(stress_control):
    """mu(x) = mu: the polarisation is -mu U13 alone, one iteration is exact, and the stress
    is the layer solve of a layer filling the cell (K with nh = nz) and, for 23, the 3-D
    cell's sigma23 on any plane."""
    n1, n2, nz = 16, 8, 4
    mu, nu = 0.37, 0.3
    up = np.random.default_rng(11).standard_normal((n2, n1))
    load = 0.02 if stress_control else 3e-3
    s13, s23, it, r = oracle.hetero_antiplane(np.full((n2, n1), mu), up, stress_control, load, tol=0.0, max_iter=2)
    sbar = load if stress_control else mu * (2 * load - up.mean())
    K = oracle.kernel_table(n1, n2, nz, nz, mu, nu)
    np.testing.assert_allclose(s13, oracle.static_tau(up, K, sbar), atol=1e-13, rtol=0)
    np.testing.assert_allclose(s23, oracle.stress_planes(up, nz, nz, mu, nu, sbar, "23", [1])[0], atol=1e-13, rtol=0)
    assert r < 1e-14


def test_hetero_laminates_have_closed_forms():
    """Fields depending on one coordinate only.  Along x1: equilibrium makes sigma13 uniform,
    g1 = U13 + Sigma / mu, and <g1> = 2 eps_bar13 gives Sigma = (2 eps_bar13 - <U13>) /
    <1/mu> (harmonic mean); sigma23 = 0.  Along x2: compatibility makes g1 uniform (= 2
    eps_bar13), so sigma13 = mu (2 eps_bar13 - U13) pointwise, and sigma23 = 0; under stress
    control g1 = (sigma_bar13 + <mu U13>) / <mu>."""
    n = 32
    x = np.arange(n)
    mu_line = 0.5 + 0.4 * np.sin(2 * np.pi * x / n) ** 2 + 0.1 * (x % 3)
    u_line = np.cos(2 * np.pi * 3 * x / n) + 0.3 * np.sin(2 * np.pi * x / n)
    eps = 2e-3
    mu1, u1 = np.tile(mu_line, (n, 1)), np.tile(u_line, (n, 1))
    s13, s23, it, r = oracle.hetero_antiplane(mu1, u1, False, eps, tol=1e-15, max_iter=400)
    sig = (2 * eps - u_line.mean()) / np.mean(1.0 / mu_line)
    np.testing.assert_allclose(s13, sig, atol=1e-12, rtol=0)
    np.testing.assert_allclose(s23, 0.0, atol=1e-12)
    s13, _, _, _ = oracle.hetero_antiplane(mu1, u1, True, 0.05, tol=1e-15, max_iter=400)
    np.testing.assert_allclose(s13, 0.05, atol=1e-12, rtol=0)
    mu2, u2 = mu1.T.copy(), u1.T.copy()
    s13, s23, it, r = oracle.hetero_antiplane(mu2, u2, False, eps, tol=1e-15, max_iter=400)
    np.testing.assert_allclose(s13, mu2 * (2 * eps - u2), atol=1e-12, rtol=0)
    np.testing.assert_allclose(s23, 0.0, atol=1e-12)
    s13, _, _, _ = oracle.hetero_antiplane(mu2, u2, True, 0.05, tol=1e-15, max_iter=400)
    g1 = (0.05 + np.mean(mu_line * u_line)) / np.mean(mu_line)
    np.testing.assert_allclose(s13, mu2 * (g1 - u2), atol=1e-12, rtol=0)


def test_hetero_solution_is_in_equilibrium_and_compatible():
    """Random modulus (contrast 4) and plastic field, iterated to convergence: the stress is
    divergence free and g = (sigma13 / mu + U13, sigma23 / mu) is a gradient (curl g = 0),
    at every mode off the Nyquist indices; <sigma13> is the prescribed stress."""
    n1, n2 = 32, 16
    mu = _smooth_field(n2, n1, 12, 0.25, 1.0)
    up = _smooth_field(n2, n1, 13, -1.0, 1.0, ell=2.0)
    s13, s23, it, r = oracle.hetero_antiplane(mu, up, True, 0.03, tol=1e-14, max_iter=500)
    assert r <= 1e-14 and it < 500
    assert s13.mean() == pytest.approx(0.03, abs=1e-14)
    k1 = 2 * np.pi * np.fft.fftfreq(n1)[None, :]
    k2 = 2 * np.pi * np.fft.fftfreq(n2)[:, None]
    inner = (np.abs(k1) < np.pi - 1e-9) & (np.abs(k2) < np.pi - 1e-9)
    div = k1 * np.fft.fft2(s13) + k2 * np.fft.fft2(s23)
    assert np.abs(div[inner]).max() < 1e-11 * np.abs(np.fft.fft2(s13)).max()
    g1, g2 = s13 / mu + up, s23 / mu
    curl = k1 * np.fft.fft2(g2) - k2 * np.fft.fft2(g1)
    assert np.abs(curl[inner]).max() < 1e-11 * np.abs(np.fft.fft2(g1)).max()
    assert np.abs(s23).max() > 1e-2


def test_hetero_iteration_contracts_at_the_basic_scheme_rate():
    """Successive increments of the fixed-point iteration shrink at least by the factor
    (kappa - 1) / (kappa + 1) of the reference medium mu0 = (min + max) / 2, kappa = max / min
    (a dropped or mis-signed polarisation term stalls or diverges)."""
    n = 32
    mu = _smooth_field(n, n, 14, 0.2, 1.0)
    up = _smooth_field(n, n, 15, -1.0, 1.0, ell=2.0)
    rho = (1.0 - 0.2) / (1.0 + 0.2)
    res = [oracle.hetero_antiplane(mu, up, False, 1e-3, tol=0.0, max_iter=k)[3] for k in range(2, 12)]
    for a, b in zip(res, res[1:]):
        assert b <= rho * a * (1 + 1e-9)
    assert res[-1] < 0.05 * res[0]


def test_hetero_steps_with_uniform_modulus_are_the_layer_steps():
    """A uniform modulus field in the time loop reproduces the layer solve with nh = nz."""
    n = 32
    up0 = inputs.random_up(n, seed=16, ell=4.0)
    p = oracle.Params(n1=n, n2=n, nz=8, nh=8, velocity_mode=1, loading_mode=1, eps_bar13_rate=1e-3, cfl=0.4)
    a, _ = oracle.run(p, up0, 6)
    b, _ = oracle.run(p, up0, 6, shear_modulus=np.full((n, n), p.mu), hetero_tol=1e-15, hetero_max_iter=5)
    assert np.abs(b.up13 - a.up13).max() < 1e-12 * np.abs(a.up13).max()
    assert b.t == pytest.approx(a.t, rel=1e-12)


def test_hetero_steps_never_increase_the_stored_energy():
    """Heterogeneous modulus, zero macroscopic stress, stress-driven motion: the stored energy
    1/2 sum (sigma13^2 + sigma23^2) / mu (the minimum over compatible g of the elastic energy,
    whose derivative in U13 is -sigma13) never increases along the steps."""
    n = 32
    up0 = inputs.random_up(n, seed=17, ell=4.0)
    mu = _smooth_field(n, n, 18, 0.1, 0.4)
    p = oracle.Params(n1=n, n2=n, nz=8, nh=8, velocity_mode=1, loading_mode=0, sigma_bar13=0.0, cfl=0.4)
    K = oracle.kernel_table(n, n, 8, 8, p.mu, p.nu)

    def energy(u):
        s13, s23, _, _ = oracle.hetero_antiplane(mu, u, True, 0.0, tol=1e-14, max_iter=500)
        return 0.5 * np.sum((s13 ** 2 + s23 ** 2) / mu)

    st, _ = oracle.run(p, up0, 0, K=K, shear_modulus=mu, hetero_tol=1e-14, hetero_max_iter=500)
    w = [energy(up0)]
    for _ in range(15):
        st, rc = oracle.run(p, up0, 1, K=K, state=st, shear_modulus=mu, hetero_tol=1e-14, hetero_max_iter=500)
        assert rc == 0
        w.append(energy(st.up13))
    assert (np.diff(w) < 0).all()
    assert w[-1] < 0.8 * w[0]


# --------------------------------------------------------------------------- paper's numbers
def test_nondimensional_numbers_printed_in_paper():
    g = json.load(open(os.path.join(GOLDEN, "paper_nondimensional.json")))
    al = units.Material(b=g["b_m"], mu=g["mu_Pa"], rho=g["rho_kg_per_m3"], eta=g["eta_Pa_s_per_m"])
    assert al.stress_scale() / 1e6 == pytest.approx(g["remote_tau13_MPa_approx"], rel=0.01)
    assert al.alpha_dimensionless(g["alpha0_per_m"]) == pytest.approx(g["alpha0_dimensionless"], rel=0.01)
    # alpha0 = b / S0 with S0 = 100 b^2
    assert 1.0 / (g["S0_b2"] * g["b_m"]) == pytest.approx(g["alpha0_per_m"], rel=0.01)
    dx1 = g["cell_b"] / g["grid_1d"]
    assert dx1 == pytest.approx(g["dx_1d_approx"], rel=0.03)
    dt1 = units.cfl_time_step(g["cfl"], dx1, g["v0_dimensionless"])
    assert dt1 == pytest.approx(g["dt_1d_approx"], rel=0.03)
    assert al.time_seconds(dt1) == pytest.approx(g["dt_1d_seconds_approx"], rel=0.03)
    dx2 = g["cell_b"] / g["grid_2d"]
    assert dx2 == pytest.approx(g["dx_2d"], rel=0.01)
    dt2 = units.cfl_time_step(g["cfl"], dx2, 1.0)
    assert dt2 == pytest.approx(g["dt_2d_approx"], rel=0.03)
    assert al.time_seconds(dt2) == pytest.approx(g["dt_2d_seconds_approx"], rel=0.03)


# ------------------------------------------------------------------ heterogeneous drag
def _obstacle_mask(n, centres, radius):
    """Mobility factor with impenetrable circular precipitates (m = 0 inside, 1 outside)."""
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    m = np.ones((n, n))
    for cx, cy in centres:
        m[np.hypot(x - cx, y - cy) <= radius] = 0.0
    return m


def test_mobility_factor_one_is_the_uniform_law():
    n = 32
    up0 = inputs.random_up(n, seed=5, ell=4.0)
    p = oracle.Params(n1=n, n2=n, velocity_mode=1, loading_mode=1, eps_bar13_rate=1e-3, cfl=0.4)
    a, _ = oracle.run(p, up0, 8)
    b, _ = oracle.run(p, up0, 8, mobility_factor=np.ones((n, n)))
    np.testing.assert_array_equal(a.up13, b.up13)
    assert a.t == b.t


def test_precipitates_never_change_and_the_rest_moves():
    """Sec. 5.3 (Orowan): inside a precipitate the drag is infinite, so v0 = 0 there; the
    update at a node with v0 = 0 returns the node's value exactly (both speeds vanish, the
    intermediate points coincide with the node, the weights are 1/2), so U13 inside the
    precipitates never changes while the walls around them move."""
    n = 64
    up0 = inputs.lines_up(n, sep=24.0, sigma=2.0)
    m = _obstacle_mask(n, [(32, 20), (32, 44)], 5.0)
    p = oracle.Params(n1=n, n2=n, velocity_mode=0, v0=1.0, cfl=0.5)
    st, rc = oracle.run(p, up0, 20, mobility_factor=m)
    assert rc == 0
    inside = m == 0.0
    np.testing.assert_array_equal(st.up13[inside], up0[inside])
    assert np.abs(st.up13 - up0)[~inside].max() > 0.5
    np.testing.assert_array_equal(st.v0[inside], 0.0)


def test_uniform_mobility_factor_rescales_time_only():
    """The update depends on v0 only through v0 dt and through ratios of speeds, and dt
    follows CFL / max |v0|: a uniform factor c gives the same field per step with time
    steps divided by c."""
    n = 32
    up0 = inputs.random_up(n, seed=6, ell=4.0)
    p = oracle.Params(n1=n, n2=n, velocity_mode=1, loading_mode=0, sigma_bar13=0.02, cfl=0.4)
    a, _ = oracle.run(p, up0, 10)
    b, _ = oracle.run(p, up0, 10, mobility_factor=np.full((n, n), 4.0))
    assert np.abs(b.up13 - a.up13).max() < 1e-13 * np.abs(a.up13).max()
    assert b.t == pytest.approx(a.t / 4.0, rel=1e-14)


# ------------------------------------------------------------------ staged loading (Sec. 5.1)
def test_strain_rate_loading_on_a_dislocation_free_state():
    """Without dislocations (U13 uniform) nothing moves, tau13 is the macroscopic stress, and
    the strain-rate mode gives sigma_bar13 = 2 mu (eps0 + rate t) - mu (nh/nz) <U13> at the
    start of every step."""
    n = 16
    u0 = np.full((n, n), 0.3)
    p = oracle.Params(n1=n, n2=n, velocity_mode=1, loading_mode=3, eps_bar13_0=1e-3, eps_bar13_rate=2e-4,
                      cfl=0.4, dt_max=0.5)
    st, rc = oracle.run(p, u0, 7)
    mu = 1.0 / 2.6
    assert rc == 0 and st.t == pytest.approx(3.5, rel=1e-15)
    np.testing.assert_array_equal(st.up13, u0)
    assert st.sigma_bar13 == pytest.approx(2 * mu * (1e-3 + 2e-4 * 3.5) - mu * (4 / 16) * 0.3, rel=1e-14)
    np.testing.assert_allclose(st.tau13, 2 * mu * (1e-3 + 2e-4 * 3.0) - mu * (4 / 16) * 0.3, rtol=1e-13)


def test_zero_mean_stress_stage_then_strain_rate_stage():
    """Two stages carried by the state: the zero-mean-stress stage keeps sigma_bar13 = 0 with
    eps_bar13 = (nh/nz) <U13> / 2, and the strain-rate stage that follows starts from the
    stage-one time (eps = eps0 + rate t, t carried on)."""
    n = 32
    up0 = inputs.random_up(n, seed=9, ell=4.0)
    p1 = oracle.Params(n1=n, n2=n, velocity_mode=1, loading_mode=2, cfl=0.4)
    st1, _ = oracle.run(p1, up0, 15)
    assert st1.sigma_bar13 == 0.0
    assert st1.eps_bar13 == pytest.approx(0.5 * (4 / 32) * st1.mean_up13, rel=1e-15)
    assert abs(st1.tau13.mean()) < 1e-14
    p2 = oracle.Params(n1=n, n2=n, velocity_mode=1, loading_mode=3, eps_bar13_rate=1e-3, cfl=0.4)
    st2, _ = oracle.run(p2, None, 10, state=st1)
    assert st2.step == 25 and st2.t > st1.t
    assert st2.eps_bar13 == pytest.approx(1e-3 * st2.t, rel=1e-14)


def test_thread_count_does_not_change_results():
    """The oracle's loops over independent rows, columns and nodes may run on several threads;
    every value is still formed by the same operations and every sum in its serial order, so
    the transform, the Green-kernel table and whole coupled and ring runs are bit-identical
    for every thread count."""
    prev = oracle.threads()
    n1, n2 = 64, 32
    up0 = inputs.random_up(64, seed=21, ell=5.0)[:n2, :n1].copy()
    a11, a12 = inputs.ring_alpha(64, r0=15.0, sigma=2.0)
    coupled = oracle.Params(n1=n1, n2=n2, velocity_mode=1, loading_mode=1, eps_bar13_rate=1e-3, cfl=0.4)
    ring = oracle.Params(n1=64, n2=64, v0=-1.0, theta=2.0, cfl=0.4)
    runs = []
    try:
        for threads in (1, 3, 0):
            oracle.set_threads(threads)
            u_ring, _, _ = oracle.curl_inverse(a11, a12, 0.1)
            st_c, rc_c = oracle.run(coupled, up0, 12)
            st_r, rc_r = oracle.run(ring, u_ring, 12)
            assert rc_c == rc_r == 0
            runs.append((oracle.fft2d(up0), oracle.kernel_table(n1, n2, 16, 3, 0.4, 0.25), st_c.up13, st_c.tau13,
                         st_c.t, st_r.up13, st_r.tau13))
    finally:
        oracle.set_threads(prev)
    for other in runs[1:]:
        for a, b in zip(runs[0], other):
            np.testing.assert_array_equal(a, b)


# ------------------------------------------------------------------ heterogeneous layer thinner than the cell
def _layer_case(seed=3):
    n1, n2 = 32, 16
    u = inputs.random_up(32, seed=seed, ell=4.0)[:n2, :n1].copy()
    f = inputs.modulus_factor(n1, n2, seed=1, lo=0.25, hi=1.0, ell=6.0)
    return u, f


@pytest.mark.parametrize("stress_control,load", [(1, 0.013), (0, 0.002)])
def test_hetero_layer_homogeneous_limit_is_the_layer_solve(stress_control, load):
    """Uniform modulus: the polarisation is -C0 : eps^p whatever the strain, so one iteration
    gives the exact solution, whose layer average is the layer solve's tau13 (Sec. 3.2.1 K
    table) and whose planes are the 3-D cell's sigma13 (both pinned above)."""
    u, _ = _layer_case()
    n2, n1 = u.shape
    nz, nh, mu, nu = 16, 3, 1 / 2.6, 0.3
    tau, planes, it, _ = oracle.hetero_layer(np.ones((n2, n1)), u, nz, nh, mu, nu, stress_control, load,
                                             tol=0.0, max_iter=2, planes=True)
    sig = load if stress_control else 2 * mu * load - mu * (nh / nz) * u.mean()
    ref = oracle.static_tau(u, oracle.kernel_table(n1, n2, nz, nh, mu, nu), sig)
    assert it == 2 and np.linalg.norm(tau - ref) / np.linalg.norm(ref) < 1e-13
    ps = oracle.stress13_planes(u, nz, nh, mu, nu, sig, list(range(nz)))
    assert np.linalg.norm(planes - ps) / np.linalg.norm(ps) < 1e-13


@pytest.mark.parametrize("stress_control,load", [(1, 0.013), (0, 0.002)])
def test_hetero_layer_filling_the_cell_is_the_antiplane_problem(stress_control, load):
    """Layer filling the cell (nh = nz): U^p is uniform along x3, only the x3-independent part
    of the strain is forced, and the iteration is the antiplane one iterate for iterate (same
    reference medium, same loading): sigma13 on every plane equals the antiplane solution."""
    u, f = _layer_case()
    mu, nu = 1 / 2.6, 0.3
    tau, planes, it, r = oracle.hetero_layer(f, u, 8, 8, mu, nu, stress_control, load, tol=0.0, max_iter=15,
                                             planes=True)
    s13, _, it2, r2 = oracle.hetero_antiplane(mu * f, u, stress_control, load, tol=0.0, max_iter=15)
    assert it == it2 == 15 and r == pytest.approx(r2, rel=1e-9)
    assert np.linalg.norm(tau - s13) / np.linalg.norm(s13) < 1e-13
    assert np.abs(planes - s13[None]).max() < 1e-13 * np.abs(s13).max()


def test_hetero_layer_thin_layer_converges_with_reflection_symmetry():
    """A layer of 3 planes in a cell of 16 with a contrast-4 modulus field: the iteration
    contracts at no more than (kappa - 1) / (kappa + 1) per step and converges; the converged
    sigma13 is even about the layer's mid-plane (the medium is uniform through the depth and
    the eigen-distortion symmetric about that plane), and its layer average differs from the
    homogeneous layer solve (the heterogeneity matters)."""
    u, f = _layer_case()
    mu, nu, nz, nh = 1 / 2.6, 0.3, 16, 3
    kappa = f.max() / f.min()
    rs = []
    for k in (30, 31):
        rs.append(oracle.hetero_layer(f, u, nz, nh, mu, nu, 1, 0.013, tol=0.0, max_iter=k)[3])
    assert rs[1] / rs[0] <= (kappa - 1) / (kappa + 1) + 1e-3
    tau, planes, it, r = oracle.hetero_layer(f, u, nz, nh, mu, nu, 1, 0.013, tol=1e-12, max_iter=400, planes=True)
    assert it < 400 and r <= 1e-12
    scale = np.abs(planes).max()
    for z in range(nz):
        zr = (nh - 1 - z) % nz
        assert np.abs(planes[z] - planes[zr]).max() < 1e-10 * scale
    assert np.isfinite(tau).all()
    ref = oracle.static_tau(u, oracle.kernel_table(32, 16, nz, nh, mu, nu), 0.013)
    assert np.linalg.norm(tau - ref) / np.linalg.norm(ref) > 1e-2
