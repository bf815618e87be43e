"""Batched engine: many cavities of different N and Re in one graph launch
per step.  Each cavity keeps its own stopping rule, so it must give exactly
the bits of a single-cavity mixed-precision context with the same inputs."""
import numpy as np
import pytest

from paper_0809_3098_gb300 import lc
from paper_0809_3098_gb300.workloads import batch_cavities, smooth_random_state

pytestmark = pytest.mark.gpu
MIXED = lc.LC_PREC_MIXED


def singles(Ns, Res, steps, **opts):
    out = []
    for N, Re in zip(Ns, Res):
        c = lc.Cavity(N, Re, precision=MIXED, **opts)
        c.step(steps)
        out.append((c.psi(), c.omega(), c.cycle_log()))
        c.close()
    return out


@pytest.mark.parametrize("op", [lc.LC_OP_COMPACT, lc.LC_OP_5PT])
def test_batch_bitwise_equals_single_contexts(op):
    Ns, Res = [128, 192, 224, 256, 320, 384], [1000.0, 3000.0, 5000.0, 12000.0, 15000.0, 25000.0]
    b = lc.Batch(Ns, Res, op=op)
    b.step(3)
    ref = singles(Ns, Res, 3, op=op)
    for c, (p, w, cyc) in enumerate(ref):
        assert np.array_equal(b.cycle_log(c), cyc), c
        assert np.array_equal(b.psi(c), p) and np.array_equal(b.omega(c), w), c


def test_batch_eager_equals_graph_and_autotune_keeps_bits():
    Ns, Res = [256, 128, 512], [5000.0, 800.0, 20000.0]
    a = lc.Batch(Ns, Res)
    e = lc.Batch(Ns, Res, graph=0)
    t = lc.Batch(Ns, Res)
    a.step(2)
    e.step(2)
    t.step(1)
    shapes = t.autotune(reps=2)
    assert len(shapes) >= 1 and all(0 <= s <= 4 for s in shapes)
    t.step(1)
    for c in range(3):
        assert np.array_equal(a.psi(c), e.psi(c)) and np.array_equal(a.omega(c), e.omega(c))
        assert np.array_equal(a.psi(c), t.psi(c)) and np.array_equal(a.omega(c), t.omega(c))
        assert np.array_equal(a.cycle_log(c), t.cycle_log(c))


@pytest.mark.parametrize("graph", [0, 1])
def test_batch_pdl_bitwise_equals_plain_launches(graph):
    """Programmatic dependent launch (the default) against plain stream order,
    in the step graph and eagerly."""
    Ns, Res = [256, 128, 384], [5000.0, 800.0, 20000.0]
    a = lc.Batch(Ns, Res, graph=graph)
    b = lc.Batch(Ns, Res, graph=graph, pdl=0)
    a.step(2)
    b.step(2)
    for c in range(3):
        assert np.array_equal(a.cycle_log(c), b.cycle_log(c))
        assert np.array_equal(a.psi(c), b.psi(c)) and np.array_equal(a.omega(c), b.omega(c))


def test_schedule_autotuner_restores_state_and_sets_schedule():
    """After the schedule search the batch is back at its starting state and
    steps exactly like a fresh batch given the chosen (nu1, nu2)."""
    Ns, Res = [128, 256, 384], [1500.0, 8000.0, 25000.0]
    t = lc.Batch(Ns, Res)
    t.step(2)
    ref_state = [(t.psi(c), t.omega(c)) for c in range(3)]
    nu1, nu2 = t.autotune_schedule(steps=2)
    assert (nu1, nu2) in {(1, 1), (2, 1), (1, 2), (2, 2), (3, 1), (3, 2)}
    for c in range(3):
        assert np.array_equal(t.psi(c), ref_state[c][0]) and np.array_equal(t.omega(c), ref_state[c][1])
    assert t.info(0)["steps"] == 2
    t.step(2)
    f = lc.Batch(Ns, Res, nu1=nu1, nu2=nu2)
    for c in range(3):
        f.set_state(c, *ref_state[c])
    f.step(2)
    for c in range(3):
        assert np.array_equal(t.psi(c), f.psi(c)) and np.array_equal(t.omega(c), f.omega(c))


def test_batch_set_state_and_dt():
    Ns, Res = [128, 256], [2000.0, 6000.0]
    dts = [1e-3, 0.0]
    b = lc.Batch(Ns, Res, dts)
    assert b.info(0)["dt"] == 1e-3 and b.info(1)["dt"] == 0.25 * min(1 / 256, 6000 / 256**2 / 4)
    psi, om = smooth_random_state(128, seed=4)
    b.set_state(0, psi, om)
    b.step(2)
    c = lc.Cavity(128, 2000.0, 1e-3, precision=MIXED)
    c.set_state(psi, om)
    c.step(2)
    assert np.array_equal(b.psi(0), c.psi()) and np.array_equal(b.omega(0), c.omega())


def test_batch_of_32_uneven_cavities_matches_singles():
    """The benchmark's batch: 32 cavities, N from {256, 384, 512, 768, 1024},
    Re log-uniform in [1000, 30000] (seed 0); two cavities checked bitwise."""
    cav = batch_cavities(32, seed=0)
    Ns, Res = [n for n, _ in cav], [r for _, r in cav]
    b = lc.Batch(Ns, Res)
    b.step(2)
    for c in (0, int(np.argmax(Ns))):
        ref = singles([Ns[c]], [Res[c]], 2)[0]
        assert np.array_equal(b.cycle_log(c), ref[2])
        assert np.array_equal(b.psi(c), ref[0]) and np.array_equal(b.omega(c), ref[1])


def test_batch_rhs64_bitwise_equals_single_contexts():
    Ns, Res = [128, 320, 256], [2000.0, 15000.0, 30000.0]
    b = lc.Batch(Ns, Res, rhs64=1)
    b.step(3)
    ref = singles(Ns, Res, 3, rhs64=1)
    for c, (p, w, cyc) in enumerate(ref):
        assert np.array_equal(b.cycle_log(c), cyc), c
        assert np.array_equal(b.psi(c), p) and np.array_equal(b.omega(c), w), c


def test_batch_errors():
    with pytest.raises(lc.LCError):
        lc.Batch([100], [1000.0])
    with pytest.raises(lc.LCError):
        lc.Batch([64], [1000.0])  # below 128: no tile level
    b = lc.Batch([128, 256], [1000.0, 1000.0], max_cycles=1, tol=1e-14)
    b.step(1)
    with pytest.raises(lc.LCError) as e:
        b.synchronize()
    assert e.value.code == lc.LC_ERR_NOCONV


def test_batch_of_256_cavities_the_maximum():
    """The largest batch (256 cavities): the first and the last give the bits
    of single contexts."""
    Ns = [128] * 255 + [256]
    Res = [1000.0 + 100.0 * k for k in range(256)]
    b = lc.Batch(Ns, Res)
    b.step(1)
    for c in (0, 255):
        ref = singles([Ns[c]], [Res[c]], 1)[0]
        assert np.array_equal(b.psi(c), ref[0]) and np.array_equal(b.omega(c), ref[1])


@pytest.mark.parametrize("rhs64", [1, 0])
def test_batch_cavities_beside_the_oracle(rhs64):
    """A three-cavity batch (N = 128, 256, 384; Re 1000, 5000, 20000) after
    10 steps from rest, each cavity directly against the FP64 oracle."""
    import oracle
    from paper_0809_3098_gb300.workloads import dt_rule

    Ns, Res, steps = [128, 256, 384], [1000.0, 5000.0, 20000.0], 10
    b = lc.Batch(Ns, Res, rhs64=rhs64)
    b.step(steps)
    oracle.set_threads(8)
    try:
        for c, (N, Re) in enumerate(zip(Ns, Res)):
            r = oracle.Cavity(N, Re, dt_rule(N, Re), 1e-10)
            assert r.step(steps) == oracle.OK
            rp, rw = r.psi(), r.omega()
            ep = np.abs(b.psi(c) - rp).max() / np.abs(rp).max()
            ew = np.abs(b.omega(c) - rw).max() / np.abs(rw).max()
            assert ep < 1e-6 and ew < 1e-6, (c, ep, ew)
            r.close()
    finally:
        oracle.set_threads(1)


def test_batch_smoothed_coarsest_grid_bitwise_equals_single_contexts():
    """coarse_direct = 0 in the batch and in single contexts: the same bits."""
    Ns, Res = [128, 224, 320], [2000.0, 9000.0, 15000.0]
    b = lc.Batch(Ns, Res, coarse_direct=0)
    b.step(2)
    ref = singles(Ns, Res, 2, coarse_direct=0)
    for c, (p, w, cyc) in enumerate(ref):
        assert np.array_equal(b.cycle_log(c), cyc), c
        assert np.array_equal(b.psi(c), p) and np.array_equal(b.omega(c), w), c
