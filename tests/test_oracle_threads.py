"""The oracle's OpenMP loops change no bit: every node is computed by the same
expression whatever the thread count, and the reductions (residual norms,
monitors) and the lexicographic SOR sweep stay serial.  A cavity stepped with
one thread and with several gives identical fields and cycle logs."""
import os

import numpy as np
import pytest

import oracle
from paper_0809_3098_gb300.workloads import dt_rule, smooth_random_state

THREADS = max(2, min(8, os.cpu_count() or 2))


def run(N, Re, steps, threads, **opts):
    oracle.set_threads(threads)
    try:
        c = oracle.Cavity(N, Re, dt_rule(N, Re), 1e-10, **opts)
        psi, omega = smooth_random_state(N, seed=11)
        c.set_state(psi, omega)
        assert c.step(steps) == oracle.OK
        out = (c.psi(), c.omega(), c.cycle_log())
        c.close()
        return out
    finally:
        oracle.set_threads(1)


@pytest.mark.parametrize("N,op", [(128, oracle.OP_COMPACT), (96, oracle.OP_5PT), (192, oracle.OP_COMPACT)])
def test_threads_bitwise_identical(N, op):
    a = run(N, 3000.0, 3, 1, op=op)
    b = run(N, 3000.0, 3, THREADS, op=op)
    assert np.array_equal(a[2], b[2])
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_threads_bitwise_identical_sor_solver():
    opts = dict(solver=1, sor_sweeps=16, beta=1.8, max_cycles=1000)
    a = run(96, 2000.0, 1, 1, **opts)
    b = run(96, 2000.0, 1, THREADS, **opts)
    assert np.array_equal(a[2], b[2])
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_thread_count_is_kept_and_clamped():
    oracle.set_threads(3)
    assert oracle.get_threads() == 3
    oracle.set_threads(0)
    assert oracle.get_threads() == 1
