"""Pins for the oracle's Poisson path (Sec. 3, Eqs. (14)-(21)).

Closed forms: sin(pi x) sin(pi y) is an exact eigenvector of both discrete
operators; manufactured continuum solutions converge at order 2 (5-point) and
4 (compact); an independent direct solver (a 2-D DST-I, which diagonalises
both operators with Dirichlet walls) gives the exact discrete solution; the
smoother leaves that solution fixed; full weighting is 1/4 the transpose of
bilinear prolongation.
"""
import numpy as np
import pytest
import scipy.fft

import oracle
from oracle import OP_5PT, OP_COMPACT

OPS = (OP_5PT, OP_COMPACT)


def grid(N):
    x = np.arange(N + 1) / N
    X, Y = np.meshgrid(x, x)  # X[j, i] = x_i, Y[j, i] = y_j
    return X, Y


def mu(N, k=1):
    """Eigenvalue of the 1-D second difference on sin(k pi x)."""
    h = 1.0 / N
    return -4.0 / h**2 * np.sin(k * np.pi * h / 2) ** 2


def interior(a):
    return a[1:-1, 1:-1]


@pytest.mark.parametrize("N", [8, 16, 24, 64])
@pytest.mark.parametrize("op", OPS)
def test_operator_eigenvector(N, op):
    X, Y = grid(N)
    S = np.sin(np.pi * X) * np.sin(np.pi * Y)
    h = 1.0 / N
    m = mu(N)
    lam = 2 * m if op == OP_5PT else 2 * m + h**2 / 6 * m * m
    out = oracle.apply_operator(N, op, S)
    assert np.abs(interior(out) - lam * interior(S)).max() < 1e-11 * abs(lam)
    assert np.all(out[0] == 0) and np.all(out[-1] == 0) and np.all(out[:, 0] == 0) and np.all(out[:, -1] == 0)


@pytest.mark.parametrize("N", [8, 32])
def test_compact_rhs_eigenvector(N):
    """B of Eq. (17) is (1 + h^2/12 (dxx + dyy)) omega, so on S it is (1 + h^2 mu / 6) S."""
    X, Y = grid(N)
    S = np.sin(np.pi * X) * np.sin(np.pi * Y)
    h = 1.0 / N
    f = oracle.poisson_rhs(N, OP_COMPACT, S)
    assert np.abs(interior(f) + (1 + h**2 * mu(N) / 6) * interior(S)).max() < 1e-14
    f5 = oracle.poisson_rhs(N, OP_5PT, S)
    assert np.array_equal(interior(f5), -interior(S))


@pytest.mark.parametrize("N", [16, 48, 80, 112, 128])
@pytest.mark.parametrize("op", OPS)
def test_solve_returns_discrete_eigenvector(N, op):
    X, Y = grid(N)
    S = np.sin(np.pi * X) * np.sin(np.pi * Y)
    h = 1.0 / N
    m = mu(N)
    lam = 2 * m if op == OP_5PT else 2 * m + h**2 / 6 * m * m
    f = lam * S
    f[0] = f[-1] = 0
    f[:, 0] = f[:, -1] = 0
    # the residual's round-off floor is ~3e-13 at N = 128, so ask for 1e-12
    psi, cycles, rel = oracle.poisson_solve(N, op, f, tol=1e-12)
    assert rel <= 1e-12 and cycles < 20
    assert np.abs(psi - S).max() < 1e-11


def _mms(X, Y):
    """psi = (1 + x) sin(pi x) sin(2 pi y) and omega = -lap psi, by hand."""
    p = np.pi
    sx, cx, s2y = np.sin(p * X), np.cos(p * X), np.sin(2 * p * Y)
    psi = (1 + X) * sx * s2y
    psi_xx = (2 * p * cx - p * p * (1 + X) * sx) * s2y
    psi_yy = -4 * p * p * psi
    return psi, -(psi_xx + psi_yy)


@pytest.mark.parametrize("op,order", [(OP_5PT, 2.0), (OP_COMPACT, 4.0)])
def test_manufactured_solution_order(op, order):
    errs = []
    Ns = (16, 32, 64, 128)
    for N in Ns:
        X, Y = grid(N)
        psi_ex, om = _mms(X, Y)
        f = oracle.poisson_rhs(N, op, om)
        psi, _, rel = oracle.poisson_solve(N, op, f, tol=1e-13)
        errs.append(np.abs(psi - psi_ex).max())
    obs = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(obs - order) < 0.15), obs


def dst_solve(N, op, f):
    """Exact discrete solution of L_h psi = f by the 2-D DST-I (independent of the oracle)."""
    h = 1.0 / N
    k = np.arange(1, N)
    mk = -4.0 / h**2 * np.sin(k * np.pi * h / 2) ** 2
    MX, MY = np.meshgrid(mk, mk)
    lam = MX + MY if op == OP_5PT else MX + MY + h**2 / 6 * MX * MY
    fh = scipy.fft.dstn(interior(f), type=1)
    psi = np.zeros_like(f)
    psi[1:-1, 1:-1] = scipy.fft.idstn(fh / lam, type=1)
    return psi


def random_rhs(N, seed):
    rng = np.random.default_rng(seed)
    f = np.zeros((N + 1, N + 1))
    f[1:-1, 1:-1] = rng.standard_normal((N - 1, N - 1))
    return f


@pytest.mark.parametrize("N", [16, 24, 40, 56, 96])
@pytest.mark.parametrize("op", OPS)
def test_solve_matches_direct_dst(N, op):
    f = random_rhs(N, seed=N + 7 * op)
    ref = dst_solve(N, op, f)
    psi, cycles, rel = oracle.poisson_solve(N, op, f, tol=1e-13)
    assert rel <= 1e-13
    assert np.abs(psi - ref).max() < 1e-12 * np.abs(ref).max()
    # and the oracle's operator agrees with the DST's symbol
    assert np.abs(interior(oracle.apply_operator(N, op, ref) - f)).max() < 1e-9 * np.abs(f).max()


@pytest.mark.parametrize("beta", [1.0, 0.6, 1.3])
@pytest.mark.parametrize("op", OPS)
def test_smoother_fixed_point(op, beta):
    N = 32
    f = random_rhs(N, seed=3)
    ref = dst_solve(N, op, f)
    out = oracle.smooth(N, op, ref, f, beta=beta, nsweeps=3)
    assert np.abs(out - ref).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("op", OPS)
def test_first_colour_of_first_sweep_is_pointwise_solve(op):
    """From psi = 0 the first colour's neighbours are all zero, so Eq. (15) at
    beta = 1 solves each of its nodes alone: psi_P = f_P / d, with d the
    diagonal of L_h (read off the already-pinned operator on a unit spike).
    The other colours must differ from that, since they see updated values."""
    N = 16
    f = random_rhs(N, seed=11)
    spike = np.zeros_like(f)
    spike[5, 7] = 1.0
    d = oracle.apply_operator(N, op, spike)[5, 7]
    out = oracle.smooth(N, op, np.zeros_like(f), f, nsweeps=1)
    J, I = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="ij")
    first = (I % 2 == 0) & (J % 2 == 0) if op == OP_COMPACT else ((I + J) % 2 == 0)
    first &= (I > 0) & (I < N) & (J > 0) & (J < N)
    assert np.allclose(out[first], f[first] / d, rtol=1e-15, atol=0)
    rest = ~first & (I > 0) & (I < N) & (J > 0) & (J < N)
    assert np.abs(out[rest] - f[rest] / d).max() > 1e-3
    # and repeated sweeps converge to the exact discrete solution
    ref = dst_solve(N, op, f)
    out = oracle.smooth(N, op, np.zeros_like(f), f, nsweeps=1500)
    assert np.abs(out - ref).max() < 1e-10 * np.abs(ref).max()


def test_restriction_is_quarter_transpose_of_prolongation():
    rng = np.random.default_rng(5)
    for Nf in (8, 16, 24):
        Nc = Nf // 2
        r = np.zeros((Nf + 1, Nf + 1))
        r[1:-1, 1:-1] = rng.standard_normal((Nf - 1, Nf - 1))
        e = np.zeros((Nc + 1, Nc + 1))
        e[1:-1, 1:-1] = rng.standard_normal((Nc - 1, Nc - 1))
        lhs = np.sum(oracle.restrict(Nf, r) * e)
        Pe = oracle.prolong_add(Nc, e, np.zeros((Nf + 1, Nf + 1)))
        rhs = 0.25 * np.sum(r * Pe)
        assert lhs == pytest.approx(rhs, rel=1e-13)


def test_prolongation_reproduces_bilinear_functions():
    Nc = 6
    Xc, Yc = grid(Nc)
    e = 1 + 2 * Xc + 3 * Yc + 4 * Xc * Yc
    Xf, Yf = grid(2 * Nc)
    out = oracle.prolong_add(Nc, e, np.zeros((2 * Nc + 1, 2 * Nc + 1)))
    ref = 1 + 2 * Xf + 3 * Yf + 4 * Xf * Yf
    assert np.abs(interior(out - ref)).max() < 1e-14


def test_restriction_of_constant_and_walls():
    Nf = 12
    r = np.zeros((Nf + 1, Nf + 1))
    r[1:-1, 1:-1] = 2.5
    fc = oracle.restrict(Nf, r)
    assert np.all(fc[0] == 0) and np.all(fc[:, -1] == 0)
    assert np.allclose(fc[1:-1, 1:-1], 2.5, rtol=0, atol=1e-15)


@pytest.mark.parametrize("direct", [1, 0])
@pytest.mark.parametrize("N", [128, 224, 320])
@pytest.mark.parametrize("op", OPS)
def test_multigrid_contraction(op, N, direct):
    """A V(2,2) cycle contracts the residual by at least 5x per cycle, with
    the exact coarse solve (R15) and with the smoothed coarsest grid (R12),
    also when that grid has 7 (224 = 7 * 32) or 5 (320 = 5 * 64) intervals."""
    f = random_rhs(N, seed=1)
    psi = np.zeros_like(f)
    prev = np.linalg.norm(f)
    for _ in range(4):
        psi, cycles, rel = oracle.poisson_solve(N, op, f, psi0=psi, tol=1e-300, max_cycles=1, direct=direct)
        r = np.linalg.norm(oracle.residual(N, op, psi, f))
        assert r < 0.2 * prev
        prev = r


def test_zero_rhs_gives_zero_in_one_cycle():
    N = 16
    psi, cycles, rel = oracle.poisson_solve(N, OP_COMPACT, np.zeros((N + 1, N + 1)), tol=1e-10)
    assert cycles == 1 and rel == 0.0 and not psi.any()


def test_rejects_unsupported_sizes():
    f = np.zeros((37, 37))
    psi, cycles, rel = oracle.poisson_solve(36, OP_5PT, f)   # 36 = 4 * 9
    assert cycles == oracle.ERR_ARG


@pytest.mark.parametrize("n", [2, 4, 5, 6, 7, 8, 10, 12, 14, 16])
@pytest.mark.parametrize("op", OPS)
def test_direct_coarse_solve_matches_dst(n, op):
    """The exact coarse solve of reading R15 (dense -L_h, Cholesky) against the
    independent DST-I solution, and on the discrete eigenvector."""
    f = random_rhs(n, seed=100 + n + op)
    ref = dst_solve(n, op, f)
    psi = oracle.direct_solve(n, op, f)
    assert np.abs(psi - ref).max() < 1e-13 * np.abs(ref).max()
    X, Y = grid(n)
    S = np.sin(np.pi * X) * np.sin(np.pi * Y)
    h = 1.0 / n
    m = mu(n)
    lam = 2 * m if op == OP_5PT else 2 * m + h**2 / 6 * m * m
    fe = lam * S
    fe[0] = fe[-1] = 0
    fe[:, 0] = fe[:, -1] = 0
    assert np.abs(oracle.direct_solve(n, op, fe) - S).max() < 1e-13


@pytest.mark.parametrize("N", [8, 16, 96, 224, 320])
@pytest.mark.parametrize("op", OPS)
def test_exact_coarse_level_keeps_the_solution_and_speeds_convergence(N, op):
    """Both coarsest-level treatments (R15 exact solve at <= 16 intervals,
    R12 smoothing of the 2/3/5/7-interval grid) reach the DST-I solution; the
    exact coarse solve never needs more cycles."""
    f = random_rhs(N, seed=N + 3 * op)
    ref = dst_solve(N, op, f)
    out = {}
    for direct in (1, 0):
        psi, cycles, rel = oracle.poisson_solve(N, op, f, tol=1e-12, nu1=2, nu2=1, direct=direct)
        assert rel <= 1e-12 and cycles > 0
        assert np.abs(psi - ref).max() < 1e-10 * np.abs(ref).max()
        out[direct] = cycles
    assert out[1] <= out[0], out
