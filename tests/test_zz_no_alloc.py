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


def test_noalloc_monitor_rejects_bad_sizes():
    import torch

    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = x.data_ptr()
    assert lc.lc_monitor_noalloc(lc.LC_NOALLOC_MAX_N + 1, p, p, p, p, 10**5, 1.0, p) == lc.LC_ERR_SIZE
    assert "LC_NOALLOC_MAX_N" in lc.last_error()
    assert lc.lc_monitor_noalloc(8, p, p, p, p, 8, 1.0, p) == lc.LC_ERR_ARG  # pitch < N + 1
    assert lc.lc_monitor_noalloc(8, 0, p, p, p, 9, 1.0, p) == lc.LC_ERR_ARG
    assert lc.lc_monitor_noalloc(8, p, p, p, p, 9, 0.0, p) == lc.LC_ERR_ARG
