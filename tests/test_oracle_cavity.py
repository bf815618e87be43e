"""Pins for the oracle's full cavity step (Secs. 2-3).

Invariants of the discrete method, independent of any implementation:
  * psi = 0 on every wall and the lid vorticity starts at -2U/h (Eq. (25));
  * reversing the lid mirrors the flow: the discrete scheme is equivariant under
    x -> 1 - x with (psi, omega, U) -> (-psi, -omega, -U); the oracle sums the
    paper's terms left to right, which is not mirror-paired, so this holds to
    rounding (an index or offset error breaks it at O(1));
  * with transport switched off (Stokes limit) the flow is mirror-symmetric;
  * the lid drives a clockwise primary vortex (psi < 0 inside) and the total
    circulation tends to -U (Stokes' theorem: the lid is the only moving wall);
  * with a smooth (regularised) lid the scheme converges at second order in
    space under grid refinement.
"""
import numpy as np
import pytest

import oracle
from oracle import OP_5PT, OP_COMPACT


def dt_rule(N, Re):
    h = 1.0 / N
    return 0.25 * min(h, Re * h * h / 4)


@pytest.mark.parametrize("op", [OP_5PT, OP_COMPACT])
def test_rest_state_and_walls(op):
    N, Re = 16, 100.0
    c = oracle.Cavity(N, Re, dt_rule(N, Re), op=op)
    w = c.omega()
    assert not c.psi().any()
    assert np.all(w[N, 1:N] == -2.0 * N) and not w[:N].any()
    assert c.step(3) == oracle.OK
    p, w = c.psi(), c.omega()
    assert not p[0].any() and not p[N].any() and not p[:, 0].any() and not p[:, N].any()
    assert w[0, 0] == w[0, N] == w[N, 0] == w[N, N] == 0.0
    assert len(c.cycle_log()) == 15  # five Poisson solves per step


@pytest.mark.parametrize("op", [OP_5PT, OP_COMPACT])
@pytest.mark.parametrize("N", [16, 24])
def test_lid_reversal_mirror_equivariance(op, N):
    Re = 400.0
    dt = dt_rule(N, Re)
    a = oracle.Cavity(N, Re, dt, op=op)
    b = oracle.Cavity(N, Re, dt, op=op, U=-1.0)
    a.step(6)
    b.step(6)
    pa, wa, pb, wb = a.psi(), a.omega(), b.psi(), b.omega()
    assert np.abs(pa).max() > 1e-4
    assert np.abs(pb + pa[:, ::-1]).max() <= 1e-13 * np.abs(pa).max()
    assert np.abs(wb + wa[:, ::-1]).max() <= 1e-13 * np.abs(wa).max()
    assert np.array_equal(a.cycle_log(), b.cycle_log())


@pytest.mark.parametrize("op", [OP_5PT, OP_COMPACT])
def test_stokes_limit_is_mirror_symmetric(op):
    N, Re = 24, 50.0
    c = oracle.Cavity(N, Re, dt_rule(N, Re), op=op, advect=0)
    c.step(8)
    p, w = c.psi(), c.omega()
    assert np.abs(p - p[:, ::-1]).max() <= 1e-13 * np.abs(p).max()
    assert np.abs(w - w[:, ::-1]).max() <= 1e-13 * np.abs(w).max()
    # with transport on, the symmetry is broken
    c2 = oracle.Cavity(N, Re, dt_rule(N, Re), op=op)
    c2.step(8)
    p2 = c2.psi()
    assert np.abs(p2 - p2[:, ::-1]).max() > 1e-6


def test_primary_vortex_sign_and_circulation():
    N, Re = 32, 100.0
    c = oracle.Cavity(N, Re, dt_rule(N, Re))
    c.step(200)
    p, w = c.psi(), c.omega()
    # clockwise primary vortex centred in the cavity; the counter-rotating
    # corner eddies (psi > 0) are orders of magnitude weaker
    assert p.min() < -0.05 and p.max() < 1e-3 * -p.min()
    j, i = np.unravel_index(np.argmin(p), p.shape)
    assert N // 4 < i < 3 * N // 4 and N // 2 < j < N
    # trapezoidal integral of omega over the square, walls included
    wt = np.ones(N + 1)
    wt[0] = wt[-1] = 0.5
    circ = np.sum(w * np.outer(wt, wt)) / N**2
    assert circ == pytest.approx(-1.0, abs=0.1)


def test_circulation_error_shrinks_with_h():
    errs = []
    for N in (16, 32):
        Re = 100.0
        dt = dt_rule(64, Re)
        c = oracle.Cavity(N, Re, dt)
        c.step(int(round(0.5 / dt)))
        wt = np.ones(N + 1)
        wt[0] = wt[-1] = 0.5
        errs.append(abs(np.sum(c.omega() * np.outer(wt, wt)) / N**2 + 1.0))
    assert errs[1] < 0.75 * errs[0]


@pytest.mark.slow
def test_second_order_self_convergence_regularised_lid():
    """Regularised lid U(x) = 16 x^2 (1-x)^2, Re = 100, same dt on every grid,
    run until nu t = (2 h_coarse)^2; differences between successive grids
    shrink by ~4 (second order in space)."""
    Re = 100.0
    Ns = (16, 32, 64)
    dt = dt_rule(Ns[-1], Re)
    T = (2.0 / Ns[0]) ** 2 * Re
    nsteps = int(round(T / dt))
    fields = []
    for N in Ns:
        c = oracle.Cavity(N, Re, dt, profile=1)
        assert c.step(nsteps) == oracle.OK
        s = N // Ns[0]
        fields.append(c.psi()[::s, ::s])
    d1 = np.abs(fields[0] - fields[1]).max()
    d2 = np.abs(fields[1] - fields[2]).max()
    assert 3.0 < d1 / d2 < 5.0, d1 / d2


def test_set_state_reapplies_thom_and_continues():
    N, Re = 16, 100.0
    dt = dt_rule(N, Re)
    a = oracle.Cavity(N, Re, dt)
    a.step(4)
    b = oracle.Cavity(N, Re, dt)
    w = a.omega()
    w_bad_walls = w.copy()
    w_bad_walls[0] = 123.0
    b.set_state(a.psi(), w_bad_walls)
    assert np.array_equal(b.omega(), w)
    a.step(2)
    b.step(2)
    assert np.array_equal(a.psi(), b.psi()) and np.array_equal(a.omega(), b.omega())


def test_rejects_bad_arguments():
    with pytest.raises(ValueError):
        oracle.Cavity(44, 100.0, 1e-3)       # 44 = 4 * 11 does not coarsen to 2, 3, 5 or 7
    with pytest.raises(ValueError):
        oracle.Cavity(16, -1.0, 1e-3)
    with pytest.raises(ValueError):
        oracle.Cavity(16, 100.0, 0.0)


def test_max_cycles_reports_noconv():
    N, Re = 16, 100.0
    c = oracle.Cavity(N, Re, dt_rule(N, Re), max_cycles=1)
    c.set_option("max_cycles", 1)
    assert c.step(2) == oracle.ERR_NOCONV
