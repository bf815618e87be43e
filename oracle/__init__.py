"""Plain FP64 CPU oracle for the lid-driven cavity step (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use this package to check and time the CUDA library.  The library
never imports it and shares no code with it.

The arithmetic lives in ``lc_oracle.c`` (plain C, ``-O2 -ffp-contract=off``,
OpenMP over loops whose iterations are independent, one thread unless
``set_threads`` says otherwise); this module compiles it with gcc and wraps it
with ctypes.  Arrays are numpy
``float64`` of shape ``(N+1, N+1)`` indexed ``[j, i]`` (row j = y index,
column i = x index), which is the C layout ``j*(N+1) + i``.

Every function cites the passage of Cardoso & Bicudo (arXiv:0809.3098) it
follows; see the header of ``lc_oracle.c`` for the equation map.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblc_oracle.so")

OP_5PT = 0
OP_COMPACT = 1

OK = 0
ERR_ARG = -1
ERR_NOCONV = -3
ERR_NONFINITE = -4

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
L_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, _dp, _dp)


def build(force: bool = False) -> str:
    """Compile lc_oracle.c into a shared library (plain IEEE FP64, no FMA)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-std=c11",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.or_ssprk54_coefficients.argtypes = [_dp, _dp]
        L.or_ssprk54_step.argtypes = [ci, _dp, cd, L_FN, vp, _dp]
        L.or_poisson_rhs.argtypes = [ci, ci, _dp, _dp]
        L.or_apply_operator.argtypes = [ci, ci, _dp, _dp]
        L.or_residual.argtypes = [ci, ci, _dp, _dp, _dp]
        L.or_smooth.argtypes = [ci, ci, _dp, _dp, cd, ci]
        L.or_sor_lex.argtypes = [ci, ci, _dp, _dp, cd, ci]
        L.or_sor_solve.argtypes = [ci, ci, _dp, _dp, cd, ci, ci, cd, _dp]
        L.or_sor_solve.restype = ci
        L.or_restrict.argtypes = [ci, _dp, _dp]
        L.or_prolong_add.argtypes = [ci, _dp, _dp]
        L.or_poisson_solve.argtypes = [ci, ci, _dp, _dp, cd, ci, ci, ci, cd, _dp]
        L.or_poisson_solve.restype = ci
        L.or_poisson_solve2.argtypes = [ci, ci, _dp, _dp, cd, ci, ci, ci, cd, ci, _dp]
        L.or_poisson_solve2.restype = ci
        L.or_direct_solve.argtypes = [ci, ci, _dp, _dp]
        L.or_direct_solve.restype = ci
        L.or_thom.argtypes = [ci, cd, ci, _dp, _dp]
        L.or_rhs_L.argtypes = [ci, cd, ci, _dp, _dp, _dp]
        L.or_monitors.argtypes = [ci, cd, _dp, _dp, _dp, _dp, _dp]
        L.or_create.argtypes = [ci, cd, cd, cd, ci]
        L.or_create.restype = vp
        L.or_destroy.argtypes = [vp]
        L.or_set_option.argtypes = [vp, ctypes.c_char_p, cd]
        L.or_set_option.restype = ci
        L.or_step.argtypes = [vp, ci]
        L.or_step.restype = ci
        L.or_get.argtypes = [vp, ci, _dp]
        L.or_get.restype = ci
        L.or_set_state.argtypes = [vp, _dp, _dp]
        L.or_set_state.restype = ci
        L.or_last_residual.argtypes = [vp]
        L.or_last_residual.restype = cd
        L.or_cycle_log.argtypes = [vp, ctypes.POINTER(ci), ctypes.c_longlong]
        L.or_cycle_log.restype = ctypes.c_longlong
        L.or_set_threads.argtypes = [ci]
        L.or_get_threads.restype = ci
        _lib = L
    return _lib


def set_threads(n: int) -> None:
    """Threads for the oracle's independent loops (colour phases, stencils,
    transfers, the Runge-Kutta combination); reductions and the lexicographic
    SOR sweep stay serial, so results are bit-identical for any count."""
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return int(lib().or_get_threads())


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _field(N: int) -> np.ndarray:
    return np.zeros((N + 1, N + 1), dtype=np.float64)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Components (each wraps the C function of the same name).

def ssprk54_coefficients():
    """Shu-Osher alpha, beta tables of SSPRK(5,4), Eqs. (9)-(13): shape (6, 5)."""
    a = np.zeros(30)
    b = np.zeros(30)
    lib().or_ssprk54_coefficients(_p(a), _p(b))
    return a.reshape(6, 5), b.reshape(6, 5)


def ssprk54_step(y: np.ndarray, dt: float, L) -> np.ndarray:
    """One SSPRK(5,4) step of y' = L(stage, y) (Eqs. (9)-(13)); returns y_{n+1}."""
    y = _f64(y).copy()
    n = y.size

    def cb(_user, stage, yp, outp):
        yy = np.ctypeslib.as_array(yp, shape=(n,))
        out = np.ctypeslib.as_array(outp, shape=(n,))
        out[:] = L(stage, yy.copy())

    fn = L_FN(cb)
    work = np.zeros(11 * n)
    lib().or_ssprk54_step(n, _p(y), dt, fn, None, _p(work))
    return y


def poisson_rhs(N: int, op: int, omega) -> np.ndarray:
    """f = -B (compact, Eq. (17)) or f = -omega (5-point) at interior nodes."""
    f = _field(N)
    lib().or_poisson_rhs(N, op, _p(_f64(omega)), _p(f))
    return f


def apply_operator(N: int, op: int, psi) -> np.ndarray:
    """L_h psi at interior nodes (compact: A + C - (5/3) a psi; 5-point: A - 2 a psi)."""
    out = _field(N)
    lib().or_apply_operator(N, op, _p(_f64(psi)), _p(out))
    return out


def residual(N: int, op: int, psi, f) -> np.ndarray:
    out = _field(N)
    lib().or_residual(N, op, _p(_f64(psi)), _p(_f64(f)), _p(out))
    return out


def smooth(N: int, op: int, psi, f, beta: float = 1.0, nsweeps: int = 1) -> np.ndarray:
    """Colour-ordered SOR sweeps of Eq. (15)."""
    psi = _f64(psi).copy()
    lib().or_smooth(N, op, _p(psi), _p(_f64(f)), beta, nsweeps)
    return psi


def sor_lex(N: int, op: int, psi, f, beta: float = 1.0, nsweeps: int = 1) -> np.ndarray:
    """SOR sweeps of Eq. (15) in the order of its superscripts (i outer, j inner)."""
    psi = _f64(psi).copy()
    lib().or_sor_lex(N, op, _p(psi), _p(_f64(f)), beta, nsweeps)
    return psi


def sor_solve(N: int, op: int, f, psi0=None, tol: float = 1e-10, max_checks: int = 1000,
              sweeps_per_check: int = 16, beta: float = 1.0):
    """Lexicographic SOR solve of L_h psi = f (reading R13): passes of
    sweeps_per_check sweeps until the stopping test of R7 holds.  Returns
    (psi, passes, rel); passes is negative (ERR_NOCONV) if max_checks ran out."""
    psi = _field(N) if psi0 is None else _f64(psi0).copy()
    rel = ctypes.c_double(0.0)
    n = lib().or_sor_solve(N, op, _p(_f64(f)), _p(psi), tol, max_checks, sweeps_per_check, beta,
                           ctypes.byref(rel))
    return psi, n, rel.value


def restrict(Nf: int, r) -> np.ndarray:
    out = _field(Nf // 2)
    lib().or_restrict(Nf, _p(_f64(r)), _p(out))
    return out


def prolong_add(Nc: int, e, psi) -> np.ndarray:
    psi = _f64(psi).copy()
    lib().or_prolong_add(Nc, _p(_f64(e)), _p(psi))
    return psi


def poisson_solve(N: int, op: int, f, psi0=None, tol: float = 1e-10, max_cycles: int = 100,
                  nu1: int = 2, nu2: int = 2, beta: float = 1.0, direct: int = 1):
    """Multigrid solve of L_h psi = f (reading R7).  direct = 1 solves the
    first level below the finest with at most 16 intervals exactly (R15),
    0 smooths the coarsest level (R12).  Returns (psi, cycles, rel)."""
    psi = _field(N) if psi0 is None else _f64(psi0).copy()
    rel = ctypes.c_double(0.0)
    cycles = lib().or_poisson_solve2(N, op, _p(_f64(f)), _p(psi), tol, max_cycles, nu1, nu2, beta, int(direct),
                                     ctypes.byref(rel))
    return psi, cycles, rel.value


def direct_solve(n: int, op: int, f) -> np.ndarray:
    """Exact solve of L_h psi = f on an n-interval grid (the coarse solve of
    reading R15): dense -L_h built from the operator, Cholesky, substitution."""
    psi = _field(n)
    rc = lib().or_direct_solve(n, op, _p(_f64(f)), _p(psi))
    if rc != OK:
        raise ValueError(f"or_direct_solve({n}) failed: {rc}")
    return psi


def thom(N: int, psi, omega, U: float = 1.0, profile: int = 0) -> np.ndarray:
    """Wall vorticity by Thom's formula, Eq. (25); returns omega with new walls."""
    omega = _f64(omega).copy()
    lib().or_thom(N, U, profile, _p(_f64(psi)), _p(omega))
    return omega


def rhs_L(N: int, Re: float, psi, omega, advect: int = 1) -> np.ndarray:
    """L(omega), Eq. (8), with u, v from Eq. (22)."""
    out = _field(N)
    lib().or_rhs_L(N, Re, advect, _p(_f64(psi)), _p(_f64(omega)), _p(out))
    return out


def monitors(N: int, dt: float, psi0, psi1, om0, om1) -> np.ndarray:
    """[max|d omega|/dt, RES_psi, RES_omega] between two states (Eqs. (26)-(27))."""
    out = np.zeros(3)
    lib().or_monitors(N, dt, _p(_f64(psi0)), _p(_f64(psi1)), _p(_f64(om0)), _p(_f64(om1)), _p(out))
    return out


# --------------------------------------------------------------------------
class Cavity:
    """The full time-stepper: psi = omega = 0 at rest, Thom walls, SSPRK(5,4)."""

    def __init__(self, N: int, Re: float, dt: float, tol: float = 1e-10, op: int = OP_COMPACT, **options):
        self.N = N
        self.dt = dt
        self._h = lib().or_create(N, Re, dt, tol, op)
        if not self._h:
            raise ValueError(f"oracle rejected N={N} Re={Re} dt={dt} tol={tol} op={op}")
        for k, v in options.items():
            self.set_option(k, v)

    def set_option(self, key: str, value: float) -> None:
        if lib().or_set_option(self._h, key.encode(), float(value)) != OK:
            raise ValueError(f"unknown oracle option {key}")

    def step(self, n: int = 1) -> int:
        return lib().or_step(self._h, n)

    def psi(self) -> np.ndarray:
        out = _field(self.N)
        lib().or_get(self._h, 0, _p(out))
        return out

    def omega(self) -> np.ndarray:
        out = _field(self.N)
        lib().or_get(self._h, 1, _p(out))
        return out

    def set_state(self, psi, omega) -> None:
        lib().or_set_state(self._h, _p(_f64(psi)), _p(_f64(omega)))

    def last_residual(self) -> float:
        return lib().or_last_residual(self._h)

    def cycle_log(self) -> np.ndarray:
        out = np.zeros(1_000_000, dtype=np.int32)
        n = lib().or_cycle_log(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), out.size)
        return out[:n].copy()

    def close(self) -> None:
        if self._h:
            lib().or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
