"""Pins for Thom's wall vorticity (Sec. 3.1, Eq. (25)), the operator L(omega)
(Sec. 3, Eqs. (8) and (22)) and the RES monitors (Sec. 3.2, Eqs. (26)-(27)).

Thom's formula is exact when psi is quadratic in the wall-normal direction
with psi = 0 and d psi / dn equal to the wall speed; central differences are
exact on quadratics, so L must equal the continuum right-hand side of the
vorticity transport equation (Sec. 2, Eq. (4)) evaluated in closed form.
"""
import numpy as np
import pytest

import oracle


def grid(N):
    x = np.arange(N + 1) / N
    return np.meshgrid(x, x)


@pytest.mark.parametrize("N", [8, 16, 24])
def test_thom_exact_for_wall_normal_quadratics(N):
    X, Y = grid(N)
    a, U = 1.7, 0.8
    h = 1.0 / N
    sl = slice(1, N)  # non-corner wall nodes
    # bottom: psi = a y^2 -> omega_wall = -psi_yy = -2a
    w = oracle.thom(N, a * Y**2, np.zeros_like(X), U=U)
    assert np.allclose(w[0, sl], -2 * a, rtol=1e-12)
    # lid: psi = a (1-y)^2 - U (1-y): psi(1) = 0, psi_y(1) = U, -psi_yy = -2a
    w = oracle.thom(N, a * (1 - Y) ** 2 - U * (1 - Y), np.zeros_like(X), U=U)
    assert np.allclose(w[N, sl], -2 * a, rtol=1e-10)
    # left / right walls
    w = oracle.thom(N, a * X**2, np.zeros_like(X), U=U)
    assert np.allclose(w[sl, 0], -2 * a, rtol=1e-12)
    w = oracle.thom(N, a * (1 - X) ** 2, np.zeros_like(X), U=U)
    assert np.allclose(w[sl, N], -2 * a, rtol=1e-12)
    # corners are zero, interior untouched
    interior = np.full_like(X, 3.25)
    w = oracle.thom(N, np.zeros_like(X), interior, U=U)
    assert w[0, 0] == w[0, N] == w[N, 0] == w[N, N] == 0.0
    assert np.all(w[1:N, 1:N] == 3.25)
    assert np.allclose(w[N, sl], -2 * U / h, rtol=1e-14)


def test_thom_regularised_lid_profile():
    N = 16
    X, Y = grid(N)
    w = oracle.thom(N, np.zeros_like(X), np.zeros_like(X), U=1.0, profile=1)
    x = X[N, 1:N]
    assert np.allclose(w[N, 1:N], -2 * 16 * x**2 * (1 - x) ** 2 * N, rtol=1e-13)


def _poly(X, Y, c):
    """c0 + c1 x + c2 y + c3 x^2 + c4 x y + c5 y^2 and its derivatives."""
    f = c[0] + c[1] * X + c[2] * Y + c[3] * X**2 + c[4] * X * Y + c[5] * Y**2
    fx = c[1] + 2 * c[3] * X + c[4] * Y
    fy = c[2] + c[4] * X + 2 * c[5] * Y
    lap = 2 * c[3] + 2 * c[5]
    return f, fx, fy, lap


@pytest.mark.parametrize("N", [8, 32])
@pytest.mark.parametrize("advect", [1, 0])
def test_L_exact_on_quadratics(N, advect):
    X, Y = grid(N)
    rng = np.random.default_rng(N + advect)
    cp, cw = rng.standard_normal(6), rng.standard_normal(6)
    psi, psi_x, psi_y, _ = _poly(X, Y, cp)
    om, om_x, om_y, om_lap = _poly(X, Y, cw)
    Re = 250.0
    # Eq. (4): d omega / dt = -psi_y omega_x + psi_x omega_y + nu lap(omega)
    ref = (-psi_y * om_x + psi_x * om_y) * advect + om_lap / Re
    out = oracle.rhs_L(N, Re, psi, om, advect=advect)
    assert np.abs(out[1:N, 1:N] - ref[1:N, 1:N]).max() < 1e-10
    assert not out[0].any() and not out[N].any()


def test_velocity_sign_convention():
    """u = psi_y, v = -psi_x (Eq. (2)): with psi = y, u = 1 advects omega = x
    so d omega/dt = -u omega_x = -1; with psi = x, v = -1 advects omega = y so
    d omega/dt = -v omega_y = +1."""
    N = 8
    X, Y = grid(N)
    out = oracle.rhs_L(N, 1e30, Y, X)
    assert np.allclose(out[1:N, 1:N], -1.0, atol=1e-12)
    out = oracle.rhs_L(N, 1e30, X, Y)
    assert np.allclose(out[1:N, 1:N], 1.0, atol=1e-12)


def test_monitors_closed_form():
    N = 4
    z = np.zeros((N + 1, N + 1))
    om1 = z.copy()
    om1[2, 3] = -0.5
    om1[1, 1] = 0.25
    psi1 = z + 0.1
    out = oracle.monitors(N, 0.01, z, psi1, z, om1)
    assert out[0] == pytest.approx(0.5 / 0.01)
    assert out[1] == pytest.approx(0.1 * (N + 1) ** 2 / (N + 1))
    assert out[2] == pytest.approx(0.75 / (N + 1))
