"""ctypes binding of the C ABI in ``include/lc.h`` (argument marshalling only).

Every step of the method runs in the CUDA library ``_lib/liblc.so``; this
module only converts Python arguments.  If the library is missing or cannot be
loaded, importing the binding's functions raises: there is no CPU fallback.

PyTorch is used only as plumbing: by default a context takes its device
workspace from a ``torch.empty(..., dtype=torch.uint8, device="cuda")`` tensor
and runs on torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblc.so")

LC_OK = 0
LC_ERR_ARG = -1
LC_ERR_CUDA = -2
LC_ERR_NOCONV = -3
LC_ERR_NONFINITE = -4
LC_ERR_TIMEOUT = -5
LC_ERR_SIZE = -6
LC_ERR_IO = -7

LC_OP_5PT = 0
LC_OP_COMPACT = 1
LC_PREC_FP64 = 0
LC_PREC_MIXED = 1

_ERRNAMES = {v: k for k, v in dict(globals()).items() if k.startswith("LC_ERR_")}

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


class LCError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {_ERRNAMES.get(code, code)}: {last_error()}")


def lib() -> ctypes.CDLL:
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built ({LIB_PATH} missing); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, ci, cd, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "lc_create": ([ci, cd, cd, cd], vp),
        "lc_destroy": ([vp], None),
        "lc_step": ([vp, ci], ci),
        "lc_get_psi": ([vp, _dp, sz], ci),
        "lc_get_omega": ([vp, _dp, sz], ci),
        "lc_residual": ([vp], cd),
        "lc_last_error": ([], ctypes.c_char_p),
        "lc_set_option": ([vp, ctypes.c_char_p, cd], ci),
        "lc_set_stream": ([vp, vp], ci),
        "lc_workspace_bytes": ([ci, ci], sz),
        "lc_bind_workspace": ([vp, vp, sz], ci),
        "lc_monitor": ([vp, _dp], ci),
        "lc_set_state": ([vp, _dp, _dp], ci),
        "lc_save": ([vp, ctypes.c_char_p], ci),
        "lc_load": ([vp, ctypes.c_char_p], ci),
        "lc_cycle_log": ([vp, ctypes.POINTER(ci), sz, ctypes.POINTER(sz)], ci),
        "lc_synchronize": ([vp], ci),
        "lc_get_params": ([vp, _dp], ci),
        "lc_launch_stats": ([vp, _dp], ci),
        "lc_bench_kernel": ([vp, ci, ci, _dp], ci),
        "lc_selftest_conversions": ([ctypes.c_longlong, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_longlong)], ci),
        "lc_monitor_noalloc": ([ci, vp, vp, vp, vp, sz, cd, vp, vp], ci),
        "lc_batch_create": ([ci, ctypes.POINTER(ci), _dp, _dp, cd, ci], vp),
        "lc_batch_destroy": ([vp], None),
        "lc_batch_set_option": ([vp, ctypes.c_char_p, cd], ci),
        "lc_batch_set_stream": ([vp, vp], ci),
        "lc_batch_workspace_bytes": ([ci, ctypes.POINTER(ci), ci], sz),
        "lc_batch_bind_workspace": ([vp, vp, sz], ci),
        "lc_batch_step": ([vp, ci], ci),
        "lc_batch_get": ([vp, ci, ci, _dp, sz], ci),
        "lc_batch_set_state": ([vp, ci, _dp, _dp], ci),
        "lc_batch_cycle_log": ([vp, ci, ctypes.POINTER(ci), sz, ctypes.POINTER(sz)], ci),
        "lc_batch_synchronize": ([vp], ci),
        "lc_batch_info": ([vp, ci, _dp], ci),
        "lc_batch_autotune": ([vp, ci, ctypes.POINTER(ci), ci], ci),
        "lc_batch_autotune_schedule": ([vp, ci, ctypes.POINTER(ci)], ci),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def last_error() -> str:
    return (lib().lc_last_error() or b"").decode()


def _check(rc: int, where: str) -> int:
    if rc != LC_OK:
        raise LCError(rc, where)
    return rc


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


# Thin same-name wrappers ----------------------------------------------------
def lc_create(N: int, Re: float, dt: float, tol: float) -> int:
    h = lib().lc_create(N, Re, dt, tol)
    if not h:
        raise LCError(LC_ERR_ARG, "lc_create")
    return h


def lc_destroy(ctx: int) -> None:
    lib().lc_destroy(ctx)


def lc_step(ctx: int, nsteps: int) -> int:
    return lib().lc_step(ctx, nsteps)


def lc_get_psi(ctx: int, out: np.ndarray) -> int:
    return lib().lc_get_psi(ctx, _p(out), out.size)


def lc_get_omega(ctx: int, out: np.ndarray) -> int:
    return lib().lc_get_omega(ctx, _p(out), out.size)


def lc_residual(ctx: int) -> float:
    return lib().lc_residual(ctx)


def lc_set_option(ctx: int, key: str, value: float) -> int:
    return lib().lc_set_option(ctx, key.encode(), float(value))


def lc_set_stream(ctx: int, stream_handle: int) -> int:
    """stream_handle 0 is the legacy default stream (torch's default stream)."""
    return lib().lc_set_stream(ctx, stream_handle)


def lc_workspace_bytes(N: int, precision: int = LC_PREC_FP64) -> int:
    return lib().lc_workspace_bytes(N, precision)


def lc_bind_workspace(ctx: int, dev_ptr: int, nbytes: int) -> int:
    return lib().lc_bind_workspace(ctx, dev_ptr, nbytes)


def lc_monitor(ctx: int) -> tuple[int, np.ndarray]:
    out = np.zeros(4)
    return lib().lc_monitor(ctx, _p(out)), out


def lc_set_state(ctx: int, psi: np.ndarray, omega: np.ndarray) -> int:
    return lib().lc_set_state(ctx, _p(psi), _p(omega))


def lc_save(ctx: int, path: str) -> int:
    return lib().lc_save(ctx, path.encode())


def lc_load(ctx: int, path: str) -> int:
    return lib().lc_load(ctx, path.encode())


def lc_synchronize(ctx: int) -> int:
    return lib().lc_synchronize(ctx)


def lc_cycle_log(ctx: int, max_n: int = 65536) -> tuple[int, np.ndarray]:
    out = np.zeros(max_n, dtype=np.int32)
    n = ctypes.c_size_t(0)
    rc = lib().lc_cycle_log(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), max_n, ctypes.byref(n))
    return rc, out[: n.value].copy()


def lc_get_params(ctx: int) -> np.ndarray:
    out = np.zeros(7)
    _check(lib().lc_get_params(ctx, _p(out)), "lc_get_params")
    return out


def lc_launch_stats(ctx: int) -> np.ndarray:
    out = np.zeros(2)
    _check(lib().lc_launch_stats(ctx, _p(out)), "lc_launch_stats")
    return out


def lc_bench_kernel(ctx: int, kernel: int, reps: int) -> np.ndarray:
    out = np.zeros(4)
    _check(lib().lc_bench_kernel(ctx, kernel, reps, _p(out)), "lc_bench_kernel")
    return out


def lc_selftest_conversions(n: int, seed: int = 0) -> tuple[int, int]:
    """Mismatches (FP64 -> FP32, FP32 -> FP64) of the library's integer
    conversions against the hardware's on n generated values."""
    out = (ctypes.c_longlong * 2)()
    _check(lib().lc_selftest_conversions(n, seed, out), "lc_selftest_conversions")
    return out[0], out[1]


LC_NOALLOC_MAX_N = 8192


def lc_monitor_noalloc(N: int, psi0_ptr: int, psi1_ptr: int, omega0_ptr: int, omega1_ptr: int, pitch: int,
                       dt: float, out_ptr: int, stream_handle: int = 0) -> int:
    """Monitors of two device states without any allocation (device pointers in and out)."""
    return lib().lc_monitor_noalloc(N, psi0_ptr, psi1_ptr, omega0_ptr, omega1_ptr, pitch, dt, out_ptr,
                                    stream_handle)


# Convenience object ---------------------------------------------------------
class Cavity:
    """One lid-driven cavity on the GPU (see ``include/lc.h``).

    ``workspace="torch"`` binds a torch CUDA tensor as the device workspace;
    ``"library"`` lets the library cudaMalloc its own.  ``stream`` is a
    ``torch.cuda.Stream`` (default: torch's current stream when torch is used).
    Options are ``lc_set_option`` keys.
    """

    def __init__(self, N: int, Re: float, dt: float = 0.0, tol: float = 1e-10, *, workspace: str = "torch",
                 stream=None, **options):
        self.N = N
        self._ws = None
        self._h = lc_create(N, Re, dt, tol)
        try:
            for key in ("op", "precision"):
                if key in options:
                    self.set_option(key, options.pop(key))
            for k, v in options.items():
                self.set_option(k, v)
            if workspace == "torch":
                import torch

                nbytes = lc_workspace_bytes(N, int(self.precision))
                self._ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
                _check(lc_bind_workspace(self._h, self._ws.data_ptr(), nbytes), "lc_bind_workspace")
                s = stream if stream is not None else torch.cuda.current_stream()
                _check(lc_set_stream(self._h, s.cuda_stream), "lc_set_stream")
            elif stream is not None:
                _check(lc_set_stream(self._h, stream.cuda_stream), "lc_set_stream")
        except Exception:
            self.close()
            raise

    precision = LC_PREC_FP64

    def set_option(self, key: str, value: float) -> None:
        _check(lc_set_option(self._h, key, value), f"lc_set_option({key})")
        if key == "precision":
            self.precision = int(value)

    @property
    def handle(self) -> int:
        return self._h

    @property
    def params(self) -> dict:
        p = lc_get_params(self._h)
        return dict(N=int(p[0]), Re=p[1], dt=p[2], tol=p[3], h=p[4], levels=int(p[5]), steps=int(p[6]))

    def step(self, n: int = 1) -> None:
        _check(lc_step(self._h, n), "lc_step")

    def synchronize(self) -> None:
        _check(lc_synchronize(self._h), "lc_synchronize")

    def psi(self) -> np.ndarray:
        out = np.empty((self.N + 1, self.N + 1))
        _check(lc_get_psi(self._h, out), "lc_get_psi")
        return out

    def omega(self) -> np.ndarray:
        out = np.empty((self.N + 1, self.N + 1))
        _check(lc_get_omega(self._h, out), "lc_get_omega")
        return out

    def set_state(self, psi: np.ndarray, omega: np.ndarray) -> None:
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        omega = np.ascontiguousarray(omega, dtype=np.float64)
        assert psi.shape == omega.shape == (self.N + 1, self.N + 1)
        _check(lc_set_state(self._h, psi, omega), "lc_set_state")

    def residual(self) -> float:
        return lc_residual(self._h)

    def monitor(self) -> np.ndarray:
        rc, out = lc_monitor(self._h)
        _check(rc, "lc_monitor")
        return out

    def cycle_log(self) -> np.ndarray:
        rc, out = lc_cycle_log(self._h)
        _check(rc, "lc_cycle_log")
        return out

    def save(self, path: str) -> None:
        _check(lc_save(self._h, path), "lc_save")

    def load(self, path: str) -> None:
        _check(lc_load(self._h, path), "lc_load")

    def close(self) -> None:
        if getattr(self, "_h", None):
            lc_destroy(self._h)
            self._h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many cavities advanced together (``lc_batch_*``; mixed precision).

    ``Ns`` / ``Res`` give each cavity's size and Reynolds number; ``dts``
    (optional) its time step (<= 0: the rule).  Workspace and stream as
    :class:`Cavity`.
    """

    def __init__(self, Ns, Res, dts=None, tol: float = 1e-10, *, workspace: str = "torch", stream=None,
                 **options):
        n = len(Ns)
        self.Ns = [int(x) for x in Ns]
        self._ws = None
        Na = (ctypes.c_int * n)(*self.Ns)
        Ra = np.ascontiguousarray(Res, dtype=np.float64)
        Da = np.ascontiguousarray(dts if dts is not None else np.zeros(n), dtype=np.float64)
        self._h = lib().lc_batch_create(n, Na, _p(Ra), _p(Da), tol, LC_PREC_MIXED)
        if not self._h:
            raise LCError(LC_ERR_ARG, "lc_batch_create")
        try:
            for key in ("op", "coarse_max"):
                if key in options:
                    self.set_option(key, options.pop(key))
            for k, v in options.items():
                self.set_option(k, v)
            if workspace == "torch":
                import torch

                nbytes = lib().lc_batch_workspace_bytes(n, Na, LC_PREC_MIXED)
                self._ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
                _check(lib().lc_batch_bind_workspace(self._h, self._ws.data_ptr(), nbytes), "lc_batch_bind_workspace")
                s = stream if stream is not None else torch.cuda.current_stream()
                _check(lib().lc_batch_set_stream(self._h, s.cuda_stream), "lc_batch_set_stream")
            elif stream is not None:
                _check(lib().lc_batch_set_stream(self._h, stream.cuda_stream), "lc_batch_set_stream")
        except Exception:
            self.close()
            raise

    @property
    def handle(self) -> int:
        return self._h

    @property
    def count(self) -> int:
        return len(self.Ns)

    def set_option(self, key: str, value: float) -> None:
        _check(lib().lc_batch_set_option(self._h, key.encode(), float(value)), f"lc_batch_set_option({key})")

    def step(self, n: int = 1) -> None:
        _check(lib().lc_batch_step(self._h, n), "lc_batch_step")

    def synchronize(self) -> None:
        _check(lib().lc_batch_synchronize(self._h), "lc_batch_synchronize")

    def _get(self, c: int, field: int) -> np.ndarray:
        N = self.Ns[c]
        out = np.empty((N + 1, N + 1))
        _check(lib().lc_batch_get(self._h, c, field, _p(out), out.size), "lc_batch_get")
        return out

    def psi(self, c: int) -> np.ndarray:
        return self._get(c, 0)

    def omega(self, c: int) -> np.ndarray:
        return self._get(c, 1)

    def set_state(self, c: int, psi, omega) -> None:
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        omega = np.ascontiguousarray(omega, dtype=np.float64)
        _check(lib().lc_batch_set_state(self._h, c, _p(psi), _p(omega)), "lc_batch_set_state")

    def cycle_log(self, c: int) -> np.ndarray:
        out = np.zeros(65536, dtype=np.int32)
        n = ctypes.c_size_t(0)
        _check(lib().lc_batch_cycle_log(self._h, c, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), out.size,
                                        ctypes.byref(n)), "lc_batch_cycle_log")
        return out[: n.value].copy()

    def info(self, c: int) -> dict:
        out = np.zeros(8)
        _check(lib().lc_batch_info(self._h, c, _p(out)), "lc_batch_info")
        return dict(N=int(out[0]), Re=out[1], dt=out[2], levels=int(out[3]), coarse_level=int(out[4]),
                    steps=int(out[5]), tile_shape0=int(out[6]), workspace_bytes=int(out[7]))

    def autotune(self, reps: int = 5) -> list:
        shapes = (ctypes.c_int * 16)()
        _check(lib().lc_batch_autotune(self._h, reps, shapes, 16), "lc_batch_autotune")
        return [s for s in shapes if s >= 0]

    def autotune_schedule(self, steps: int = 2) -> tuple:
        """Picks the fastest smoothing schedule (nu1, nu2); see lc.h."""
        nu = (ctypes.c_int * 2)()
        _check(lib().lc_batch_autotune_schedule(self._h, steps, nu), "lc_batch_autotune_schedule")
        return nu[0], nu[1]

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().lc_batch_destroy(self._h)
            self._h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
