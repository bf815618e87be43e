"""Pins for the oracle's SSPRK(5,4) integrator (Sec. 3, Eqs. (9)-(13)).

The coefficient table is checked against the digits the paper prints (a text
fixture), and the integrator is checked against the mathematics: the eight
fourth-order conditions of the equivalent Butcher tableau, the stability
polynomial on y' = lambda y, and the observed global order on a nonlinear ODE.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ssprk54_paper_coefficients.txt")


def _paper_table():
    alpha = np.zeros((6, 5))
    beta = np.zeros((6, 5))
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        kind, s, k, val = line.split()
        (alpha if kind == "alpha" else beta)[int(s), int(k)] = float(val)
    return alpha, beta


def _butcher(alpha, beta):
    """Butcher (A, b, c) of a Shu-Osher scheme: stage s is y_n + dt sum_k a[s,k] L(Y_k)."""
    a = np.zeros((6, 5))
    for s in range(1, 6):
        for k in range(s):
            a[s] += alpha[s, k] * a[k]
            a[s, k] += beta[s, k]
    A = a[:5]          # stage inputs Y_0..Y_4
    b = a[5]
    return A, b, A.sum(axis=1)


def _order_conditions(alpha, beta):
    A, b, c = _butcher(alpha, beta)
    return np.array([
        b.sum() - 1.0,
        b @ c - 1 / 2,
        b @ c**2 - 1 / 3,
        b @ (A @ c) - 1 / 6,
        b @ c**3 - 1 / 4,
        b @ (c * (A @ c)) - 1 / 8,
        b @ (A @ c**2) - 1 / 12,
        b @ (A @ (A @ c)) - 1 / 24,
    ])


def test_coefficients_match_paper_digits():
    alpha, beta = oracle.ssprk54_coefficients()
    pa, pb = _paper_table()
    for s in range(6):
        for k in range(5):
            for got, printed, kind in ((alpha[s, k], pa[s, k], "alpha"), (beta[s, k], pb[s, k], "beta")):
                if (kind, s, k) == ("alpha", 2, 1):
                    # reading: the printed 0.555626... breaks sum(alpha[2]) = 1
                    assert got == pytest.approx(1.0 - pa[2, 0], abs=1e-15)
                    assert abs(got - printed) == pytest.approx(3e-6, rel=1e-6)
                elif (kind, s, k) == ("beta", 1, 0):
                    assert abs(got - printed) < 1e-11
                else:
                    assert got == printed, (kind, s, k)


def test_stage_weights_sum_to_one():
    alpha, _ = oracle.ssprk54_coefficients()
    assert np.allclose(alpha[1:].sum(axis=1), 1.0, atol=2e-16)


def test_fourth_order_conditions():
    alpha, beta = oracle.ssprk54_coefficients()
    err = _order_conditions(alpha, beta)
    assert np.abs(err).max() < 1e-14, err


def test_printed_coefficient_breaks_order_conditions():
    """The reading of alpha[2][1] is forced: the printed digits miss order 1-4 at ~1e-7."""
    pa, pb = _paper_table()
    pb[1, 0] = 0.391752226571890
    err = _order_conditions(pa, pb)
    assert np.abs(err).max() > 1e-8


def test_stability_polynomial_is_taylor_to_fourth_order():
    """On y' = lam y one step multiplies by R(z), a degree-5 polynomial equal to
    exp(z) through z^4, so (R(z) - T4(z)) / z^5 is the same constant for every z."""
    ratios = []
    for z in (1.0, 0.5, -0.5, -1.0, 0.25):
        R = oracle.ssprk54_step(np.array([1.0]), 1.0, lambda s, y: z * y)[0]
        T4 = sum(z**k / math.factorial(k) for k in range(5))
        ratios.append((R - T4) / z**5)
    ratios = np.array(ratios)
    assert np.ptp(ratios) < 1e-10 * max(1.0, abs(ratios).max())
    assert 0 < ratios[0] < 1 / 120  # an SSP(5,4) method damps the z^5 term below exp's
    # and that constant is b^T A^4 e of the Butcher tableau of the paper's
    # printed table (with the reading of alpha[2][1]): R(z) = 1 + z b^T (I - zA)^-1 e
    pa, pb = _paper_table()
    pa[2, 1] = 1.0 - pa[2, 0]
    pb[1, 0] = 0.391752226571890
    A, b, _ = _butcher(pa, pb)
    c5 = b @ np.linalg.matrix_power(A, 4) @ np.ones(5)
    assert abs(ratios[0] - c5) < 1e-9 * c5


def test_global_order_four_on_nonlinear_ode():
    """y' = -y^2 + sin(t)-free autonomous form: y' = -y^2, y(0) = 1, y(t) = 1/(1+t)."""
    T = 2.0
    errs = []
    for n in (10, 20, 40, 80):
        dt = T / n
        y = np.array([1.0])
        for _ in range(n):
            y = oracle.ssprk54_step(y, dt, lambda s, v: -v * v)
        errs.append(abs(y[0] - 1.0 / (1.0 + T)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 3.7) and np.all(orders < 4.5), orders


def test_stage_inputs_are_passed_in_order():
    seen = []

    def L(stage, y):
        seen.append(stage)
        return -y

    oracle.ssprk54_step(np.ones(3), 0.1, L)
    assert seen == [0, 1, 2, 3, 4]
