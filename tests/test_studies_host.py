"""Host-side pieces of the studies (no GPU): the vortex census and the
centreline extraction, on fields whose answer is known by construction."""
import numpy as np

from tests.studies.precision_study import centrelines
from tests.studies.steady_study import vortex_census


def grid(N):
    x = np.arange(N + 1) / N
    return np.meshgrid(x, x)  # X[j, i] = x_i, Y[j, i] = y_j


def test_census_names_primary_and_corner_eddies():
    """A clockwise primary vortex (psi < 0) with positive eddies in the bottom
    corners and the top-left corner, and a negative eddy inside the
    bottom-right one: primary, BL1, BR1, BR2 (nested), TL1."""
    N = 128
    X, Y = grid(N)
    psi = -np.sin(np.pi * X) * np.sin(np.pi * Y)

    def bump(x0, y0, r, a):
        return a * np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / r**2)

    # carve positive corner regions, then a negative one inside bottom-right
    for x0, y0 in ((0.06, 0.06), (0.94, 0.06), (0.06, 0.94)):
        psi = np.where((X - x0) ** 2 + (Y - y0) ** 2 < 0.07**2, 0.01 + bump(x0, y0, 0.03, 0.02), psi)
    psi = np.where((X - 0.95) ** 2 + (Y - 0.05) ** 2 < 0.02**2, -0.001, psi)
    psi[0, :] = psi[-1, :] = psi[:, 0] = psi[:, -1] = 0.0
    c = vortex_census(psi)
    assert c["primary"]["sign"] == -1 and c["primary"]["area"] > 0.9
    assert abs(c["primary"]["x"] - 0.5) < 0.02 and abs(c["primary"]["y"] - 0.5) < 0.02
    assert {k for k in c if k != "primary"} == {"BL1", "BR1", "BR2", "TL1"}
    assert c["BL1"]["sign"] == 1 and c["BR2"]["sign"] == -1
    assert c["BR1"]["area"] > c["BR2"]["area"]


def test_census_ignores_rounding_noise():
    N = 64
    X, Y = grid(N)
    psi = -np.sin(np.pi * X) * np.sin(np.pi * Y)
    psi[1, 1] = 1e-16  # a single-node sign flip at rounding level
    c = vortex_census(psi)
    assert list(c) == ["primary"]


def test_centrelines_of_a_linear_shear():
    """psi = y^2 / 2 has u = y and v = 0 (Eq. (22)): the extracted centreline
    u(y) is y at interior nodes and the lid speed 1 at the top."""
    N = 32
    X, Y = grid(N)
    psi = 0.5 * Y**2
    u, v = centrelines(psi)
    y = np.arange(N + 1) / N
    assert np.allclose(u[1:N], y[1:N], atol=1e-14) and u[N] == 1.0 and u[0] == 0.0
    assert np.allclose(v, 0.0, atol=1e-14)
