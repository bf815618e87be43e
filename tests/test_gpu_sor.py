"""The paper-literal SOR solver on the GPU (solver = 1): Eq. (15) swept
lexicographically, in the order of its n / n+1 superscripts, by wavefronts in
one thread block.  The oracle sweeps the same order node by node, so both
make the same number of passes per solve and agree to rounding."""
import numpy as np
import pytest

import oracle
from paper_0809_3098_gb300 import lc
from paper_0809_3098_gb300.workloads import dt_rule, smooth_random_state

pytestmark = pytest.mark.gpu
OPS = {"5pt": lc.LC_OP_5PT, "compact": lc.LC_OP_COMPACT}


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def pair(N, Re, op, **opts):
    dt = dt_rule(N, Re)
    g = lc.Cavity(N, Re, dt, 1e-10, op=op, solver=1, **opts)
    r = oracle.Cavity(N, Re, dt, 1e-10, op=op, solver=1, **opts)
    return g, r


# 128 keeps the grid in shared memory; 160 does not and sweeps in global memory
@pytest.mark.parametrize("N", [8, 16, 20, 32, 64, 128, 160])
@pytest.mark.parametrize("opname", ["5pt", "compact"])
def test_sor_cavity_matches_oracle(N, opname):
    g, r = pair(N, 400.0, OPS[opname], sor_sweeps=8, beta=1.5, max_cycles=20000)
    g.step(2)
    assert r.step(2) == oracle.OK
    assert np.array_equal(g.cycle_log(), r.cycle_log())
    assert rel(g.psi(), r.psi()) < 1e-12 and rel(g.omega(), r.omega()) < 1e-12


@pytest.mark.parametrize("beta", [0.8, 1.0])
@pytest.mark.parametrize("sweeps", [1, 5])
def test_sor_relaxation_and_pass_length(beta, sweeps):
    g, r = pair(24, 1000.0, lc.LC_OP_COMPACT, sor_sweeps=sweeps, beta=beta, max_cycles=100000)
    g.step(1)
    assert r.step(1) == oracle.OK
    assert np.array_equal(g.cycle_log(), r.cycle_log())
    assert rel(g.psi(), r.psi()) < 1e-12 and rel(g.omega(), r.omega()) < 1e-12


@pytest.mark.parametrize("N,opname", [(1024, "compact"), (384, "5pt")])
def test_sor_fixed_passes_large_grid(N, opname):
    """One pass of 3 sweeps per solve (max_cycles = 1) from a non-trivial state:
    the wavefront schedule at full size, against the oracle's node-by-node
    sweeps.  Every solve stops at the cap, so the step reports NOCONV."""
    Re = 10000.0
    psi, om = smooth_random_state(N, seed=5)
    g, r = pair(N, Re, OPS[opname], sor_sweeps=3, beta=1.2, max_cycles=1)
    g.set_state(psi, om)
    r.set_state(psi, om)
    g.step(1)
    with pytest.raises(lc.LCError) as e:
        g.synchronize()
    assert e.value.code == lc.LC_ERR_NOCONV
    assert r.step(1) == oracle.ERR_NOCONV
    assert rel(g.psi(), r.psi()) < 1e-12 and rel(g.omega(), r.omega()) < 1e-12


def test_sor_graph_equals_eager_and_options():
    a = lc.Cavity(32, 500.0, solver=1, sor_sweeps=4, beta=1.4, max_cycles=20000)
    b = lc.Cavity(32, 500.0, solver=1, sor_sweeps=4, beta=1.4, max_cycles=20000, graph=0)
    a.step(2)
    b.step(2)
    assert np.array_equal(a.psi(), b.psi()) and np.array_equal(a.omega(), b.omega())
    assert np.array_equal(a.cycle_log(), b.cycle_log())
    m = lc.Cavity(32, 500.0, precision=lc.LC_PREC_MIXED)
    with pytest.raises(lc.LCError):
        m.set_option("solver", 1)
    with pytest.raises(lc.LCError):
        a.set_option("sor_sweeps", 0)


def test_sor_agrees_with_multigrid():
    """Both solvers stop at the same relative residual."""
    N, Re = 64, 1000.0
    s = lc.Cavity(N, Re, tol=1e-12, solver=1, sor_sweeps=16, beta=1.8, max_cycles=50000)
    m = lc.Cavity(N, Re, tol=1e-12)
    s.step(3)
    m.step(3)
    assert rel(s.psi(), m.psi()) < 1e-8 and rel(s.omega(), m.omega()) < 1e-8
