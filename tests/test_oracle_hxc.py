"""Pins of the Hartree and LDA exchange-correlation oracle (oracle/hxc.py): closed forms,
finite-difference convergence of the Poisson equation, and derivative identities."""
import numpy as np
import pytest

from oracle import hxc

SKEWED = np.array([[9.0, 0.0, 0.0], [2.5, 8.0, 0.0], [1.5, -2.0, 10.0]])


def frac_grid(shape):
    return np.meshgrid(*[np.arange(n) / n for n in shape], indexing="ij")


@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, -1), (1, -1, 3)])
def test_plane_wave_density_has_the_closed_form_potential(m):
    """rho = rho0 + a cos(2 pi m . f): V_H = 4 pi a / |G|^2 cos(2 pi m . f), G = sum m_i b_i,
    and E_H = pi a^2 Omega / |G|^2 (the constant rho0 sits on the background)."""
    shape = (18, 16, 20)
    f = frac_grid(shape)
    phase = 2.0 * np.pi * (m[0] * f[0] + m[1] * f[1] + m[2] * f[2])
    rho0, a = 0.3, 0.17
    rho = rho0 + a * np.cos(phase)
    # |G|^2 from the reciprocal metric: G . G = 4 pi^2 m^T (A A^T)^-1 m (A: rows a_i)
    mv = np.array(m, dtype=np.float64)
    g2 = float(4.0 * np.pi ** 2 * mv @ np.linalg.inv(SKEWED @ SKEWED.T) @ mv)
    v, e = hxc.hartree(rho, SKEWED)
    np.testing.assert_allclose(v, 4.0 * np.pi * a / g2 * np.cos(phase), rtol=0, atol=1e-12 * 4.0 * np.pi * a / g2)
    omega = abs(np.linalg.det(SKEWED))
    assert e == pytest.approx(np.pi * a * a * omega / g2, rel=1e-12)


def test_potential_has_zero_mean_and_is_linear():
    rng = np.random.default_rng(5)
    r1, r2 = rng.random((12, 10, 14)), rng.random((12, 10, 14))
    v1, _ = hxc.hartree(r1, SKEWED)
    v2, _ = hxc.hartree(r2, SKEWED)
    v12, _ = hxc.hartree(2.0 * r1 - r2, SKEWED)
    assert abs(v1.mean()) < 1e-12 * np.abs(v1).max()
    np.testing.assert_allclose(v12, 2.0 * v1 - v2, atol=1e-12 * np.abs(v12).max())


def _fd_residual(n, L):
    """max |FD laplacian V_H + 4 pi (rho - mean rho)| / max |4 pi (rho - mean rho)| for a smooth
    periodic rho on an n^3 grid."""
    cell = np.diag(L)
    f = frac_grid((n, n, n))
    rho = np.exp(0.8 * np.cos(2 * np.pi * f[0])) * (1.0 + 0.3 * np.sin(2 * np.pi * 2 * f[1])) \
        * (1.2 + np.cos(2 * np.pi * (f[2] + 0.1)))
    v, _ = hxc.hartree(rho, cell)
    lap = np.zeros_like(v)
    for ax, length in enumerate(L):
        h = length / n
        lap += (np.roll(v, 1, ax) - 2.0 * v + np.roll(v, -1, ax)) / (h * h)
    src = 4.0 * np.pi * (rho - rho.mean())
    return np.max(np.abs(lap + src)) / np.max(np.abs(src))


def test_poisson_residual_falls_at_second_order():
    """A three-point Laplacian of V_H reproduces -4 pi (rho - mean): the residual falls 4x per halving of h."""
    L = (7.0, 8.0, 9.0)
    r1, r2, r3 = _fd_residual(24, L), _fd_residual(48, L), _fd_residual(96, L)
    assert 3.6 < r1 / r2 < 4.4 and 3.8 < r2 / r3 < 4.2
    assert r3 < 2e-3


def test_exchange_closed_forms():
    ex, vx = hxc.lda_exchange(np.array([1.0, 2.0]))
    # eps_x(rs = 1) = -(3/4) (9 / (4 pi^2))^(1/3) = -0.4581652932831... hartree
    assert ex[0] == pytest.approx(-0.45816529328314287, rel=1e-14)
    assert ex[1] == pytest.approx(ex[0] / 2.0, rel=1e-14)
    np.testing.assert_allclose(vx, 4.0 / 3.0 * ex, rtol=1e-15)
    # the same from rho: eps_x = -(3/4) (3/pi)^(1/3) rho^(1/3)
    rho = 0.05
    e, _ = hxc.lda_exchange(hxc.wigner_seitz_radius(np.array([rho])))
    assert e[0] == pytest.approx(-0.75 * (3.0 / np.pi) ** (1.0 / 3.0) * rho ** (1.0 / 3.0), rel=1e-14)


def test_pz81_values_and_continuity_at_rs_1():
    ec, _ = hxc.pz81_correlation(np.array([1.0, 1.0 - 1e-12]))
    assert ec[0] == pytest.approx(-0.1423 / (1.0 + 1.0529 + 0.3334), rel=1e-14)
    assert ec[1] == pytest.approx(-0.048 - 0.0116, abs=1e-10)
    # the fit's two branches meet at rs = 1 to within 5e-5 hartree (energy) and 5e-4 (potential)
    e, v = hxc.pz81_correlation(np.array([1.0 - 1e-9, 1.0 + 1e-9]))
    assert abs(e[0] - e[1]) < 5e-5 and abs(v[0] - v[1]) < 5e-4


@pytest.mark.parametrize("rho", [1e-3, 0.02, 0.3, 2.0, 50.0])
def test_potential_is_the_density_derivative_of_the_energy(rho):
    """v_xc = d(rho eps_xc)/d rho, by central differences (away from the rs = 1 branch point)."""
    h = 1e-5 * rho
    eps, v = hxc.lda_xc(np.array([rho - h, rho + h, rho]))
    fd = ((rho + h) * eps[1] - (rho - h) * eps[0]) / (2.0 * h)
    assert v[2] == pytest.approx(fd, rel=1e-8)


def test_non_positive_density_gives_zero():
    eps, v = hxc.lda_xc(np.array([0.0, -0.2, 0.1]))
    assert eps[0] == eps[1] == 0.0 and v[0] == v[1] == 0.0 and eps[2] < 0.0 and v[2] < 0.0
