"""Workload definitions and seeded input generators.

Shared by the tests and the benchmark for both the CUDA library and the CPU
oracle; it holds none of the method's arithmetic.  The cavity itself starts
from rest and needs no random input; the seeded fields below only serve
parity tests that start from a non-trivial state.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def dt_rule(N: int, Re: float) -> float:
    """Time step of the benchmark workloads: 0.25 min(h, Re h^2 / 4), h = 1/N."""
    h = 1.0 / N
    return 0.25 * min(h, Re * h * h / 4.0)


@dataclass(frozen=True)
class Workload:
    name: str
    N: int
    Re: float
    steps: int
    tol: float = 1e-10
    precision: str = "fp64"
    op: str = "compact"
    extra: dict = field(default_factory=dict)

    @property
    def dt(self) -> float:
        return dt_rule(self.N, self.Re)

    @property
    def interior_nodes(self) -> int:
        return (self.N - 1) ** 2


# The five benchmark configurations (lid-driven cavity on the unit square,
# lid u = 1, no-slip elsewhere, psi = omega = 0 at t = 0).
CAVITY_128_RE1000 = Workload("cavity-128-Re1000-fp64", 128, 1000.0, 100)
CAVITY_1024_RE10000 = Workload("cavity-1024-Re10000-fp64", 1024, 10000.0, 20000, extra={"monitor_every": 1000})
PRECISION_1024 = tuple(Workload(f"cavity-1024-Re{int(r)}-mixed", 1024, r, 20000, precision="mixed")
                       for r in (5000.0, 10000.0, 20000.0, 30000.0))
STRESS_2048 = Workload("cavity-2048-Re30000-mixed", 2048, 30000.0, 200000, precision="mixed")


def batch_cavities(count: int = 32, seed: int = 0):
    """Batch workload: grids uniform over {256, 384, 512, 768, 1024} intervals and
    Re log-uniform in [1000, 30000], drawn in that order from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    Ns = rng.choice(np.array([256, 384, 512, 768, 1024]), size=count)
    Res = np.exp(rng.uniform(np.log(1000.0), np.log(30000.0), size=count))
    return [(int(n), float(r)) for n, r in zip(Ns, Res)]


def smooth_random_state(N: int, seed: int, modes: int = 6, amplitude: float = 1.0):
    """A seeded smooth (psi, omega) pair: psi is a random sum of sin(k pi x)
    sin(l pi y) modes (zero on the walls), omega a random sum of cos modes.
    Not a consistent state: the tests install it and let both sides step."""
    rng = np.random.default_rng(seed)
    x = np.arange(N + 1) / N
    X, Y = np.meshgrid(x, x)
    psi = np.zeros((N + 1, N + 1))
    omega = np.zeros((N + 1, N + 1))
    for k in range(1, modes + 1):
        for l in range(1, modes + 1):
            a, b = rng.standard_normal(2) * amplitude / (k * k + l * l)
            psi += a * np.sin(k * np.pi * X) * np.sin(l * np.pi * Y)
            omega += b * (k * k + l * l) * np.cos(k * np.pi * X) * np.cos(l * np.pi * Y)
    psi[0, :] = psi[-1, :] = 0.0
    psi[:, 0] = psi[:, -1] = 0.0
    return psi, omega


def random_interior(N: int, seed: int) -> np.ndarray:
    """Seeded standard-normal interior values, zero walls."""
    rng = np.random.default_rng(seed)
    a = np.zeros((N + 1, N + 1))
    a[1:-1, 1:-1] = rng.standard_normal((N - 1, N - 1))
    return a
