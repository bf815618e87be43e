"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle.

Both sides run the same algorithm (same operator, colour order, V-cycle and
stopping rule), so they agree to rounding and make the same number of V-cycles
per solve; the bar for the FP64 path is 1e-10 relative (max-norm over all
nodes, relative to the reference's max), and the cycle logs must be equal.
"""
import numpy as np
import pytest

import oracle
from paper_0809_3098_gb300 import lc
from paper_0809_3098_gb300.workloads import dt_rule, smooth_random_state

pytestmark = pytest.mark.gpu

OPS = {"5pt": lc.LC_OP_5PT, "compact": lc.LC_OP_COMPACT}


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def pair(N, Re, op, tol=1e-10, **opts):
    dt = dt_rule(N, Re)
    g = lc.Cavity(N, Re, dt, tol, op=op, **opts)
    opts.pop("monitor", None)  # the oracle computes monitors by a separate call
    r = oracle.Cavity(N, Re, dt, tol, op=op, **opts)
    return g, r


@pytest.mark.parametrize("N", [8, 10, 14, 16, 20, 24, 28, 32, 40, 48, 56, 96])
@pytest.mark.parametrize("opname", ["5pt", "compact"])
def test_small_grids_match_oracle(N, opname):
    g, r = pair(N, 400.0, OPS[opname])
    g.step(4)
    assert r.step(4) == oracle.OK
    assert rel(g.psi(), r.psi()) < 1e-12
    assert rel(g.omega(), r.omega()) < 1e-12
    assert np.array_equal(g.cycle_log(), r.cycle_log())


def test_rest_state():
    N = 64
    g = lc.Cavity(N, 1000.0)
    w = g.omega()
    assert not g.psi().any()
    assert np.all(w[N, 1:N] == -2.0 * N) and not w[:N].any() and w[N, 0] == 0 and w[N, N] == 0


def test_config_128_re1000_100_steps():
    """Lid-driven cavity, 128x128, Re 1000, dt rule, tol 1e-10, 100 steps, FP64."""
    N, Re, steps = 128, 1000.0, 100
    g, r = pair(N, Re, lc.LC_OP_COMPACT)
    g.step(steps)
    assert r.step(steps) == oracle.OK
    ep, ew = rel(g.psi(), r.psi()), rel(g.omega(), r.omega())
    assert ep <= 1e-10 and ew <= 1e-10, (ep, ew)
    gl, rl = g.cycle_log(), r.cycle_log()
    assert len(gl) == 5 * steps
    assert np.array_equal(gl, rl)
    assert g.residual() <= 1e-10


@pytest.mark.parametrize("opname", ["5pt", "compact"])
def test_options_match_oracle(opname):
    N = 64
    g, r = pair(N, 2000.0, OPS[opname], nu1=1, nu2=3, beta=1.15, nuc=8)
    g.step(3)
    r.step(3)
    assert rel(g.psi(), r.psi()) < 1e-12 and rel(g.omega(), r.omega()) < 1e-12
    assert np.array_equal(g.cycle_log(), r.cycle_log())


def test_regularised_lid_stokes_limit():
    N = 64
    g, r = pair(N, 50.0, lc.LC_OP_COMPACT, profile=1, advect=0)
    g.step(5)
    r.step(5)
    assert rel(g.psi(), r.psi()) < 1e-12 and rel(g.omega(), r.omega()) < 1e-12
    p = g.psi()
    assert np.array_equal(p, p[:, ::-1])  # Stokes limit: mirror-symmetric, bit for bit


@pytest.mark.parametrize("N", [64, 1024])
def test_lid_reversal_equivariance_bitwise(N):
    """Mirror-paired sums make the GPU scheme exactly equivariant under
    x -> 1 - x, (psi, omega, U) -> (-psi, -omega, -U), at any size."""
    Re = 10000.0
    a = lc.Cavity(N, Re)
    b = lc.Cavity(N, Re, U=-1.0)
    a.step(3)
    b.step(3)
    pa, pb = a.psi(), b.psi()
    assert np.abs(pa).max() > 0
    assert np.array_equal(pb, -pa[:, ::-1])
    assert np.array_equal(b.omega(), -a.omega()[:, ::-1])


def test_set_state_then_step_matches_oracle():
    N = 96
    psi, omega = smooth_random_state(N, seed=7)
    g, r = pair(N, 3000.0, lc.LC_OP_COMPACT)
    g.set_state(psi, omega)
    r.set_state(psi, omega)
    # Thom walls agree to rounding (-2 N^2 psi on the GPU, -2 psi / h^2 in the oracle)
    assert rel(g.omega(), r.omega()) < 1e-14
    g.step(2)
    r.step(2)
    assert rel(g.psi(), r.psi()) < 1e-12 and rel(g.omega(), r.omega()) < 1e-12
    assert np.array_equal(g.cycle_log(), r.cycle_log())


def test_monitors_match_oracle():
    N, Re = 64, 1000.0
    g, r = pair(N, Re, lc.LC_OP_COMPACT, monitor=1)
    g.step(3)
    r.step(2)
    p0, w0 = r.psi(), r.omega()
    r.step(1)
    ref = oracle.monitors(N, dt_rule(N, Re), p0, r.psi(), w0, r.omega())
    out = g.monitor()
    assert np.allclose(out[:3], ref, rtol=1e-9, atol=0)
    assert out[3] == r.cycle_log()[-1]


def test_checkpoint_roundtrip(tmp_path):
    N = 32
    a = lc.Cavity(N, 500.0)
    a.step(3)
    path = str(tmp_path / "ck.bin")
    a.save(path)
    b = lc.Cavity(N, 500.0)
    b.load(path)
    assert b.params["steps"] == 3
    assert np.array_equal(a.psi(), b.psi()) and np.array_equal(a.omega(), b.omega())
    a.step(2)
    b.step(2)
    assert np.array_equal(a.psi(), b.psi()) and np.array_equal(a.omega(), b.omega())


def test_library_workspace_and_own_stream():
    N = 32
    a = lc.Cavity(N, 500.0, workspace="library")
    b = lc.Cavity(N, 500.0)
    a.step(2)
    b.step(2)
    assert np.array_equal(a.psi(), b.psi())


def test_nonfinite_state_reports_error():
    N = 16
    g = lc.Cavity(N, 100.0)
    psi, omega = np.zeros((N + 1, N + 1)), np.zeros((N + 1, N + 1))
    omega[5, 5] = np.nan
    g.set_state(psi, omega)
    g.step(1)
    with pytest.raises(lc.LCError) as e:
        g.synchronize()
    assert e.value.code == lc.LC_ERR_NONFINITE


def test_max_cycles_reports_noconv():
    g = lc.Cavity(64, 1000.0, max_cycles=1, tol=1e-14)
    g.step(1)
    with pytest.raises(lc.LCError) as e:
        g.synchronize()
    assert e.value.code == lc.LC_ERR_NOCONV
    g.synchronize()  # the status is cleared once reported


def test_invalid_arguments():
    with pytest.raises(lc.LCError):
        lc.Cavity(44, 100.0)  # 44 = 4 * 11 does not coarsen to 2, 3, 5 or 7
    g = lc.Cavity(16, 100.0)
    with pytest.raises(lc.LCError):
        g.set_option("nu1", 0)
    with pytest.raises(lc.LCError):
        g.set_option("beta", 2.5)
    small = np.zeros(10)
    assert lc.lc_get_psi(g.handle, small) == lc.LC_ERR_SIZE
    g.step(1)
    with pytest.raises(lc.LCError):
        g.set_option("op", 0)  # layout options only before first use
    h = g.handle
    g.close()
    assert lc.lc_step(h, 1) == lc.LC_ERR_ARG


def test_runs_on_torch_stream_in_order():
    """Work is enqueued on torch's current stream, so torch events bracket it."""
    import torch

    g = lc.Cavity(256, 1000.0)
    g.step(1)
    g.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    g.step(3)
    e1.record(s)
    e1.synchronize()
    assert e0.elapsed_time(e1) > 0.05  # three steps of ~25 V-cycles cannot take < 50 us
    a = torch.zeros(1, device="cuda")
    with torch.cuda.stream(torch.cuda.Stream()):
        h = lc.Cavity(64, 100.0)  # binds the side stream
        h.step(2)
        h.synchronize()
    assert g.params["steps"] == 4


NOCL = dict(coarse_cluster=0)  # the one-block coarse V-cycle
MODES = {
    "phases": dict(blocked=0),
    "tiles": dict(blocked=1, fine_phases=0, coarse_max=2, **NOCL),
    "tiles+fine-phases": dict(blocked=1, fine_phases=1, coarse_max=4, **NOCL),
    "tiles+fine-phases-fused": dict(blocked=1, fine_phases=1, coarse_max=4, fused=1, **NOCL),
    "coarse-block": dict(blocked=1, fine_phases=0, coarse_max=64, **NOCL),
    "tiles110x54": dict(blocked=1, fine_phases=0, coarse_max=4, tile_shape=0, **NOCL),
    "tiles110x22": dict(blocked=1, fine_phases=0, coarse_max=4, tile_shape=1, **NOCL),
    "tiles16x16": dict(blocked=1, fine_phases=0, coarse_max=2, tile_shape=3, **NOCL),
    # coarse levels on a thread-block cluster: strips of 1..16 rows, uneven
    # splits (3 and 5 blocks), and the largest level the shared memory takes
    "cluster16": dict(blocked=1, fine_phases=1, coarse_cluster=16, cluster_max=256),
    "cluster3-split8": dict(blocked=1, fine_phases=0, coarse_cluster=3, cluster_max=64, cluster_split=8),
    "cluster5-split4": dict(blocked=1, fine_phases=1, coarse_cluster=5, cluster_max=512, cluster_split=4),
    "cluster8-split32": dict(blocked=1, fine_phases=1, coarse_cluster=8, cluster_split=32),
    # kernels launched one after another instead of with programmatic
    # dependent launch (the default): the same kernels and values
    "phases-2-levels": dict(fine_phases=2),
    "fused-coarser-levels": dict(fused=2),
    "fused-all-levels": dict(fused=3),
    "phases-3-levels-no-cluster": dict(fine_phases=3, **NOCL),
    "no-pdl": dict(pdl=0),
    "no-pdl-eager": dict(pdl=0, graph=0),
    "pdl-eager": dict(graph=0),
}


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("N", [16, 24, 48, 112, 128, 160])
@pytest.mark.parametrize("opname", ["5pt", "compact"])
def test_execution_modes_match_oracle(mode, N, opname):
    dt = dt_rule(N, 800.0)
    g = lc.Cavity(N, 800.0, dt, 1e-10, op=OPS[opname], **MODES[mode])
    r = oracle.Cavity(N, 800.0, dt, 1e-10, op=OPS[opname])
    g.step(3)
    r.step(3)
    assert rel(g.psi(), r.psi()) < 1e-12 and rel(g.omega(), r.omega()) < 1e-12
    assert np.array_equal(g.cycle_log(), r.cycle_log())


@pytest.mark.parametrize("N", [224, 256, 320, 384])
def test_execution_modes_are_bitwise_identical(N):
    """Tiles recompute halos with the same per-node expression, so every mode
    gives the same bits (a halo too small would show up here)."""
    out = {}
    for name, opts in MODES.items():
        g = lc.Cavity(N, 5000.0, nu1=3, nu2=1, **opts)
        g.step(2)
        out[name] = (g.psi(), g.omega(), g.cycle_log())
    ref = out["phases"]
    for name, (p, w, cyc) in out.items():
        assert np.array_equal(cyc, ref[2]), name
        assert np.array_equal(p, ref[0]) and np.array_equal(w, ref[1]), name


@pytest.mark.parametrize("fine_phases", [0, 1])
def test_1024_big_tiles_one_step_matches_oracle(fine_phases):
    N, Re = 1024, 10000.0
    dt = dt_rule(N, Re)
    g = lc.Cavity(N, Re, dt, 1e-10, fine_phases=fine_phases)
    r = oracle.Cavity(N, Re, dt, 1e-10)
    g.step(1)
    r.step(1)
    # the FP64 parity bar; after one step from rest psi is ~1e-5, so the
    # oracle's unfused arithmetic and the GPU's FMAs differ at ~1e-12 of it
    assert rel(g.psi(), r.psi()) < 1e-10 and rel(g.omega(), r.omega()) < 1e-10
    assert np.array_equal(g.cycle_log(), r.cycle_log())


def test_fused_smoother_equals_phase_launches_at_1024():
    """The cooperative fine-level smoother (colour phases separated by a grid
    barrier) gives the bits of one launch per colour phase."""
    a = lc.Cavity(1024, 10000.0, fused=1)
    b = lc.Cavity(1024, 10000.0, fused=0)
    a.step(2)
    b.step(2)
    assert np.array_equal(a.cycle_log(), b.cycle_log())
    assert np.array_equal(a.psi(), b.psi()) and np.array_equal(a.omega(), b.omega())


def test_fused_barrier_timeout_is_reported_and_context_recovers():
    """A barrier that waits for a block that never arrives gives up after its
    bound (about 0.2 s), the host reads LC_ERR_TIMEOUT, and the context steps
    on correctly afterwards."""
    N = 256
    g = lc.Cavity(N, 1000.0, nu1=1, fused=1)
    g.step(1)
    g.synchronize()
    g.set_option("barrier_extra", 1)  # only for the two stand-alone passes below, never inside a step
    lc.lc_bench_kernel(g.handle, 4, 1)  # one warm-up and one timed fused pass, each with 3 barriers
    with pytest.raises(lc.LCError) as e:
        g.synchronize()
    assert e.value.code == lc.LC_ERR_TIMEOUT
    g.set_option("barrier_extra", 0)
    ref = lc.Cavity(N, 1000.0, nu1=1, fused=1)
    psi, om = smooth_random_state(N, seed=9)
    g.set_state(psi, om)
    ref.set_state(psi, om)
    g.step(2)
    ref.step(2)
    assert np.array_equal(g.psi(), ref.psi()) and np.array_equal(g.omega(), ref.omega())


def test_maximum_grid_8192_mirror_equivariance():
    """The largest accepted grid, N = 8192 (8193^2 nodes, 537 MB per FP64
    field): one step with the lid moving each way gives mirror-image bits,
    which checks every index of every level at that size."""
    N = 8192
    a = lc.Cavity(N, 10000.0)
    a.step(1)
    pa, wa = a.psi(), a.omega()
    a.close()
    b = lc.Cavity(N, 10000.0, U=-1.0)
    b.step(1)
    assert np.array_equal(b.psi(), -pa[:, ::-1]) and np.array_equal(b.omega(), -wa[:, ::-1])
    assert np.abs(pa).max() > 0.0


@pytest.mark.parametrize("precision", [lc.LC_PREC_FP64, lc.LC_PREC_MIXED])
def test_lid_at_rest_keeps_the_fluid_at_rest(precision):
    """U = 0: the degenerate cavity has zero right-hand sides everywhere; every
    solve stops after its first cycle and the state stays exactly zero."""
    g = lc.Cavity(128, 1000.0, precision=precision, U=0.0)
    g.step(3)
    assert not g.psi().any() and not g.omega().any()
    assert (g.cycle_log() == 1).all()


@pytest.mark.parametrize("mode", ["phases", "coarse-block", "cluster16", "cluster3-split8", "tiles"])
@pytest.mark.parametrize("N", [48, 128, 224])
def test_smoothed_coarsest_grid_matches_oracle(mode, N):
    """coarse_direct = 0: the V-cycle goes down to the 2-, 3-, 5- or 7-interval
    grid and smooths it nuc times (instead of solving the first level of at
    most 16 intervals exactly); both sides switch together."""
    dt = dt_rule(N, 800.0)
    g = lc.Cavity(N, 800.0, dt, 1e-10, coarse_direct=0, **MODES[mode])
    r = oracle.Cavity(N, 800.0, dt, 1e-10, coarse_direct=0)
    g.step(3)
    r.step(3)
    assert rel(g.psi(), r.psi()) < 1e-12 and rel(g.omega(), r.omega()) < 1e-12
    assert np.array_equal(g.cycle_log(), r.cycle_log())


@pytest.mark.parametrize("N", [32, 96, 160])
def test_exact_coarse_level_sizes(N):
    """The exactly solved level is 16, 12 and 10 intervals here (the 2-D sine
    transform of 15, 11 and 9 unknowns per side); the GPU's transform and the
    oracle's Cholesky solve agree to rounding and give the same cycle counts."""
    g, r = pair(N, 1500.0, lc.LC_OP_COMPACT)
    g.step(3)
    assert r.step(3) == oracle.OK
    assert rel(g.psi(), r.psi()) < 1e-12 and rel(g.omega(), r.omega()) < 1e-12
    assert np.array_equal(g.cycle_log(), r.cycle_log())
    assert g.params["levels"] == {32: 2, 96: 4, 160: 5}[N]
