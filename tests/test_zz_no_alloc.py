"""lc_monitor_noalloc, the allocation-free monitor entry point.

It serves callers that cannot allocate device memory (a framework that owns
all device memory through its own pool, work issued during CUDA graph
capture, a fixed memory budget): it reduces two device states the caller
already holds, with its scratch in a fixed device array of the library.
Checked through the C ABI against lc_monitor of a context on the same pair of
states, on two calls in a row (the shared scratch must be reset between
calls).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_0809_3098_gb300 import lc

pytestmark = pytest.mark.gpu


def _dev(a, torch, pitch=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if pitch is not None and pitch > a.shape[1]:
        padded = np.full((a.shape[0], pitch), 7.0)  # junk in the padding must be ignored
        padded[:, : a.shape[1]] = a
        a = padded
    return torch.from_numpy(a).cuda()


def test_noalloc_monitor_matches_lc_monitor_on_two_calls():
    import torch

    N, Re = 96, 1000.0
    cav = lc.Cavity(N, Re, monitor=1)
    cav.step(2)
    states = [(cav.psi(), cav.omega())]
    refs = []
    for _ in range(2):
        cav.step(1)
        refs.append(cav.monitor()[:3].copy())
        states.append((cav.psi(), cav.omega()))
    dt = cav.params["dt"]
    stream = torch.cuda.current_stream()
    out = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
    for k, pitch in ((0, N + 1), (1, N + 9)):  # two calls in a row; the second with padded rows
        (p0, w0), (p1, w1) = states[k], states[k + 1]
        d = [_dev(a, torch, pitch) for a in (p0, p1, w0, w1)]
        rc = lc.lc_monitor_noalloc(N, d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), d[3].data_ptr(),
                                   pitch, dt, out.data_ptr(), stream.cuda_stream)
        assert rc == lc.LC_OK, lc.last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(refs[k] > 0)
        assert np.allclose(got, refs[k], rtol=1e-12, atol=0), (k, got, refs[k])


def test_noalloc_monitor_at_the_largest_size():
    """N = LC_NOALLOC_MAX_N, the size the fixed scratch holds, on device states
    with a known answer: psi1 - psi0 = 2^-10 everywhere, omega1 - omega0 =
    j / 8 on row j.  Every sum is exact in FP64, so the monitors are too."""
    import torch

    N = lc.LC_NOALLOC_MAX_N
    n = N + 1
    dt = 0.5
    psi0 = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    psi1 = torch.full((n, n), 2.0 ** -10, dtype=torch.float64, device="cuda")
    w0 = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    w1 = (torch.arange(n, dtype=torch.float64, device="cuda") / 8.0)[:, None].expand(n, n).contiguous()
    out = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):  # the shared counter and partials must be reset between calls
        rc = lc.lc_monitor_noalloc(N, psi0.data_ptr(), psi1.data_ptr(), w0.data_ptr(), w1.data_ptr(), n, dt,
                                   out.data_ptr(), stream.cuda_stream)
        assert rc == lc.LC_OK, lc.last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = [N / 8.0 / dt, n * 2.0 ** -10, n * (N * (N + 1) / 2) / 8.0 / n]
        assert got.tolist() == want, (got, want)
        out.fill_(-1.0)
