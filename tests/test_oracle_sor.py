"""Pins for the oracle's paper-literal SOR solver (Sec. 3, Eq. (15)).

Eq. (15)'s superscripts say which neighbours are already new: (i-1, j-1),
(i-1, j), (i-1, j+1) and (i, j-1).  That is a lexicographic sweep with i the
outer loop.  A sweep in that order is, by the textbook definition of SOR, the
solve of the lower-triangular system (D + beta L) x' = beta f -
(beta U + (beta - 1) D) x for the splitting A = D + L + U of the operator's
matrix with the unknowns numbered in sweep order; for the 5-point operator,
which that order makes consistently ordered, Young's theory fixes the
convergence rate: cos^2(pi h) for Gauss-Seidel and exactly beta - 1 for every
beta above the optimum 2 / (1 + sin(pi h)).
"""
import numpy as np
import pytest

import oracle
from oracle import OP_5PT, OP_COMPACT

from test_oracle_poisson import dst_solve, random_rhs

OPS = (OP_5PT, OP_COMPACT)


def operator_matrix(N, op):
    """Matrix of L_h on the interior unknowns, numbered in sweep order
    k = (i - 1)(N - 1) + (j - 1), assembled column by column."""
    n = N - 1
    A = np.zeros((n * n, n * n))
    for i in range(1, N):
        for j in range(1, N):
            e = np.zeros((N + 1, N + 1))
            e[j, i] = 1.0
            col = oracle.apply_operator(N, op, e)
            A[:, (i - 1) * n + (j - 1)] = col[1:-1, 1:-1].T.reshape(-1)
    return A


def to_vec(a):
    return a[1:-1, 1:-1].T.reshape(-1)  # [j, i] -> sweep order (i outer)


@pytest.mark.parametrize("beta", [0.5, 1.0, 1.6])
@pytest.mark.parametrize("op", OPS)
def test_one_sweep_is_the_triangular_solve_of_sor(op, beta):
    N = 7
    A = operator_matrix(N, op)
    D = np.diag(np.diag(A))
    L = np.tril(A, -1)
    U = np.triu(A, 1)
    f = random_rhs(N, seed=3)
    rng = np.random.default_rng(4)
    psi0 = np.zeros((N + 1, N + 1))
    psi0[1:-1, 1:-1] = rng.standard_normal((N - 1, N - 1))
    x = to_vec(psi0)
    expect = np.linalg.solve(D + beta * L, beta * to_vec(f) - (beta * U + (beta - 1.0) * D) @ x)
    got = to_vec(oracle.sor_lex(N, op, psi0, f, beta, 1))
    assert np.abs(got - expect).max() < 1e-12 * np.abs(expect).max()
    # The transposed order (j outer) gives the same sweep for the 5-point
    # stencil (in both orders W and S are new, E and N old) but a different
    # one for the compact stencil, whose diagonals (i-1, j+1) and (i+1, j-1)
    # swap roles: the pin tells the two orders apart where they differ.
    perm = np.array([(k % (N - 1)) * (N - 1) + k // (N - 1) for k in range(A.shape[0])])
    At = A[np.ix_(perm, perm)]
    Dt, Lt, Ut = np.diag(np.diag(At)), np.tril(At, -1), np.triu(At, 1)
    other = np.linalg.solve(Dt + beta * Lt, beta * to_vec(f)[perm] - (beta * Ut + (beta - 1.0) * Dt) @ x[perm])
    if op == OP_COMPACT:
        assert np.abs(got[perm] - other).max() > 1e-6 * np.abs(other).max()
    else:
        assert np.abs(got[perm] - other).max() < 1e-12 * np.abs(other).max()


@pytest.mark.parametrize("beta", [0.8, 1.0, 1.3])
@pytest.mark.parametrize("op", OPS)
def test_exact_solution_is_a_fixed_point(op, beta):
    N = 16
    f = random_rhs(N, seed=11)
    ref = dst_solve(N, op, f)
    out = oracle.sor_lex(N, op, ref, f, beta, 3)
    assert np.abs(out - ref).max() < 1e-13 * np.abs(ref).max()


def test_gauss_seidel_rate_is_cos_squared():
    """Lexicographic Gauss-Seidel on the 5-point Laplacian: rho = cos^2(pi h)."""
    N = 16
    rng = np.random.default_rng(5)
    psi = np.zeros((N + 1, N + 1))
    psi[1:-1, 1:-1] = rng.standard_normal((N - 1, N - 1))
    f = np.zeros_like(psi)
    psi = oracle.sor_lex(N, OP_5PT, psi, f, 1.0, 400)
    a = np.linalg.norm(psi)
    b = np.linalg.norm(oracle.sor_lex(N, OP_5PT, psi, f, 1.0, 1))
    assert abs(b / a - np.cos(np.pi / N) ** 2) < 1e-6


def test_over_relaxed_rate_is_beta_minus_one():
    """For beta above 2 / (1 + sin(pi h)) every eigenvalue of the SOR
    iteration has modulus beta - 1 (5-point, consistently ordered)."""
    N = 16
    beta = 1.8
    assert beta > 2.0 / (1.0 + np.sin(np.pi / N))
    rng = np.random.default_rng(6)
    psi = np.zeros((N + 1, N + 1))
    psi[1:-1, 1:-1] = rng.standard_normal((N - 1, N - 1))
    f = np.zeros_like(psi)
    psi = oracle.sor_lex(N, OP_5PT, psi, f, beta, 50)
    a = np.linalg.norm(psi)
    b = np.linalg.norm(oracle.sor_lex(N, OP_5PT, psi, f, beta, 200))
    assert abs((b / a) ** (1.0 / 200) - (beta - 1.0)) < 2e-3


@pytest.mark.parametrize("op", OPS)
def test_sor_solve_reaches_the_direct_solution(op):
    N = 24
    f = random_rhs(N, seed=12)
    ref = dst_solve(N, op, f)
    psi, passes, rel = oracle.sor_solve(N, op, f, tol=1e-12, max_checks=2000, sweeps_per_check=8, beta=1.7)
    assert passes > 0 and rel <= 1e-12
    assert np.abs(psi - ref).max() < 1e-10 * np.abs(ref).max()
    # the stopping test ran after every pass: one pass fewer had not converged
    _, p2, rel2 = oracle.sor_solve(N, op, f, tol=1e-12, max_checks=passes - 1, sweeps_per_check=8, beta=1.7)
    assert p2 == oracle.ERR_NOCONV and rel2 > 1e-12


def test_cavity_with_sor_agrees_with_multigrid():
    """Both solvers stop at the same relative residual, so the time steps agree
    to that tolerance."""
    N, Re, dt = 16, 100.0, 1e-3
    a = oracle.Cavity(N, Re, dt, 1e-12)
    b = oracle.Cavity(N, Re, dt, 1e-12, solver=1, sor_sweeps=4, beta=1.6, max_cycles=5000)
    assert a.step(3) == oracle.OK and b.step(3) == oracle.OK
    assert np.abs(a.psi() - b.psi()).max() < 1e-9 * np.abs(a.psi()).max()
    assert np.abs(a.omega() - b.omega()).max() < 1e-9 * np.abs(a.omega()).max()
    assert len(b.cycle_log()) == 15 and b.cycle_log().min() >= 1
