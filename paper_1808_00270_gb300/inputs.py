"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds no arithmetic of the method: it only draws initial states
and samples the model's input kernels from their closed-form expressions.
Both the CUDA library and the FP64 oracle receive exactly these arrays.

Workload recipe (a stand-in for the paper's nanocolloid suspension, whose
reconstructed kernels and MD data are not available):
  * positions uniform in a cubic periodic box of edge L = (N / density)^(1/3);
  * velocities Maxwell-distributed, N(0, kT/M) per component;
  * conservative soft repulsion U(r) = A (1 - r/r_c)^2, A = 25;
  * self kernel K^s(t) = 5 exp(-t/tau_s) cos(3 t) (+ 0.5 exp(-t/2) for the
    large suspension);
  * pair kernel K^p(r, t) = 2 (1 - r/r_c)^2 exp(-t/tau_p), passed as one
    separable term f(r) g(t): f tabulated on r = k dr, g sampled at t = m dt.
The self-kernel samples are continuous values K(m dt); the library converts
them to the discrete weights of the paper's delta-comb kernel.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n: int
    box: float
    m_max: int
    dt: float
    r_c: float
    tau_s: float
    tau_p: float
    steps: int
    tail: bool = False          # add 0.5 exp(-t/2) to K^s
    A_cons: float = 25.0
    kT: float = 1.0
    mass: float = 1.0
    seed: int = 1
    r_c_min: float = 0.0
    nr: int = 1024              # radial table points on [0, r_c]

    @property
    def density(self) -> float:
        return self.n / self.box ** 3

    def describe(self) -> dict:
        return {"workload": self.name, "n": self.n, "box": round(self.box, 4),
                "density": round(self.density, 5), "m_max": self.m_max, "dt": self.dt,
                "r_c": self.r_c, "tau_s": self.tau_s, "tau_p": self.tau_p,
                "slow_tail": self.tail}


def box_for_density(n: int, density: float) -> float:
    return (n / density) ** (1.0 / 3.0)


# The three single-system workloads: a 64-particle oracle-sized system, a
# 4096-particle system, and the 262144-particle suspension with m_max = 400.
SMALL = Workload("gld_n64_m32", n=64, box=8.0, m_max=32, dt=0.01, r_c=2.0,
                 tau_s=0.2, tau_p=0.1, steps=1000)
MEDIUM = Workload("gld_n4096_m200", n=4096, box=box_for_density(4096, 0.1), m_max=200,
                  dt=0.005, r_c=2.0, tau_s=0.5, tau_p=0.3, steps=10_000)
LARGE = Workload("gld_n262144_m400", n=262144, box=box_for_density(262144, 0.1), m_max=400,
                 dt=0.005, r_c=2.5, tau_s=0.5, tau_p=0.3, steps=1000, tail=True)

# A quarter-size copy of the suspension for profiler captures (its 0.31 GB
# history ring is still larger than L2).
LARGE_QUARTER = Workload("gld_n65536_m400", n=65536, box=box_for_density(65536, 0.1), m_max=400,
                         dt=0.005, r_c=2.5, tau_s=0.5, tau_p=0.3, steps=1000, tail=True)

WORKLOADS = {w.name: w for w in (SMALL, MEDIUM, LARGE, LARGE_QUARTER)}


def initial_state(w: Workload, seed: int | None = None):
    """Uniform positions in [0, L)^3 and Maxwell velocities, float64 [n, 3]."""
    rng = np.random.default_rng(w.seed if seed is None else seed)
    pos = rng.uniform(0.0, w.box, size=(w.n, 3))
    vel = rng.normal(0.0, math.sqrt(w.kT / w.mass), size=(w.n, 3))
    return pos, vel


def self_kernel_samples(w: Workload) -> np.ndarray:
    """K^s(m dt), m = 0 .. m_max-1."""
    t = np.arange(w.m_max) * w.dt
    ks = 5.0 * np.exp(-t / w.tau_s) * np.cos(3.0 * t)
    if w.tail:
        ks = ks + 0.5 * np.exp(-t / 2.0)
    return ks


def memory_modes(w: Workload):
    """The damped modes exp((-rate + i omega) t) the workload's kernels are
    made of: K^s (rate 1/tau_s, omega 3), its slow tail (rate 1/2), the pair
    kernel's time factor (rate 1/tau_p).  Returns (rates, omegas)."""
    rates, omegas = [1.0 / w.tau_s], [3.0]
    if w.tail:
        rates.append(0.5)
        omegas.append(0.0)
    rates.append(1.0 / w.tau_p)
    omegas.append(0.0)
    return np.array(rates), np.array(omegas)


def pair_kernel_tables(w: Workload):
    """Separable pair kernel: g[1, m_max] = exp(-m dt/tau_p), f[1, nr] = 2 (1 - r/r_c)^2."""
    t = np.arange(w.m_max) * w.dt
    g = np.exp(-t / w.tau_p)[None, :]
    dr = w.r_c / (w.nr - 1)
    r = np.arange(w.nr) * dr
    f = (2.0 * np.clip(1.0 - r / w.r_c, 0.0, None) ** 2)[None, :]
    return g, f, dr


def random_history(n: int, m_max: int, scale: float = 0.005, seed: int = 7) -> np.ndarray:
    """A random displacement history [m_max-1, n, 3] (index m-1 holds dR_{n-m})."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, size=(m_max - 1, n, 3))


def batch_systems(count: int = 512, seed: int = 4, n_range=(256, 16384), density_range=(0.02, 0.2),
                  m_choices=(100, 200, 400)) -> list:
    """Uneven independent systems: N = round(exp U(ln 256, ln 16384)), density
    exp U(ln 0.02, ln 0.2), m_max drawn from {100, 200, 400}; kernels as the
    4096-particle workload (tau_s = 0.5, tau_p = 0.3, dt = 0.005, r_c = 2);
    seed of system k is seed * 100000 + k."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        rho = math.exp(rng.uniform(math.log(density_range[0]), math.log(density_range[1])))
        m = int(rng.choice(m_choices))
        out.append(Workload(f"batch{k}_n{n}_m{m}", n=n, box=box_for_density(n, rho), m_max=m, dt=0.005,
                            r_c=2.0, tau_s=0.5, tau_p=0.3, steps=1, seed=seed * 100000 + k))
    return out


@dataclasses.dataclass(frozen=True)
class Request:
    arrival: float  # seconds after the start of the trace
    w: Workload
    steps: int


def serve_trace(count: int = 1000, rate: float = 50.0, seed: int = 5, n_range=(512, 65536),
                density_range=(0.02, 0.2), m_range=(64, 400), step_range=(2000, 20000)) -> list:
    """Poisson arrivals at `rate` per second of requests with N log-uniform in
    [512, 65536], density log-uniform in [0.02, 0.2], m_max uniform in
    [64, 400], steps uniform in [2000, 20000]; kernels as batch_systems."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for k in range(count):
        t += rng.exponential(1.0 / rate)
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        rho = math.exp(rng.uniform(math.log(density_range[0]), math.log(density_range[1])))
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        steps = int(rng.integers(step_range[0], step_range[1] + 1))
        w = Workload(f"req{k}_n{n}_m{m}", n=n, box=box_for_density(n, rho), m_max=m, dt=0.005, r_c=2.0,
                     tau_s=0.5, tau_p=0.3, steps=steps, seed=seed * 100000 + k)
        out.append(Request(t, w, steps))
    return out
