"""Seeded synthetic inputs for the StaRMAP workloads.

This module holds no arithmetic of the method itself: it only defines the
problem data (domain, grid size, boundary types, CFL number, material fields,
sources and initial conditions) as plain functions of the physical
coordinates (x, y).  Both the CUDA path and the FP64 oracle evaluate these
functions at the staggered grid points they compute on their own.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): a 64-bit Weyl sequence with
increment 0x9E3779B97F4A7C15 followed by the variant-13 mixing function; a
uniform double in [0, 1) takes the top 53 bits.

Workloads (the paper's own test problems stand in for any dataset; none is
needed):

* ``gaussian_p5``      -- 2D P_5, FP64, 64x64 periodic on [-1,1]^2, sigma_a=0,
                          sigma_s0=1, isotropic Gaussian R_0^0 (std 0.1),
                          CFL 0.5, 100 steps (section 6.2 style pulse).
* ``checkerboard_p13`` -- 2D P_13, FP32, 512x512 on [0,7]^2, extrapolation
                          boundaries, 7x7 unit blocks, 11 of the 48 outer
                          blocks absorbing (sigma_a=10), the rest scattering
                          (sigma_s0=1), unit isotropic source in [3,4]^2,
                          run to t=3.2 (section 6.3).
* ``random_p39``       -- 2D P_39, FP32 (and FP64), 1024x1024 periodic on
                          [-1,1]^2, sigma_a=0, log10 sigma_s0 uniform in
                          [-1,1] on a 32x32 periodic lattice, bilinearly
                          interpolated, Gaussian R_0^0 (std 0.1), 200 steps.
* ``batched``          -- 256 uneven instances (n in 64..512, N in 3..15),
                          piecewise-constant random media, Gaussian sources.
"""
from __future__ import annotations

import dataclasses
import json
import math
import os
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream (published definition, see module docstring)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def uniforms(self, count: int) -> np.ndarray:
        return np.array([self.uniform() for _ in range(count)], dtype=np.float64)

    def randint(self, hi: int) -> int:
        """Uniform integer in [0, hi) by rejection-free scaling (hi small)."""
        return min(int(self.uniform() * hi), hi - 1)


# A field is a function f(t, x, y) -> array, broadcasting over numpy arrays.
Field = Callable[[float, np.ndarray, np.ndarray], np.ndarray]


@dataclasses.dataclass
class Problem:
    """Problem data in the spirit of the paper's ``par`` struct (section 5.1)."""

    name: str
    N: int                                   # moment order
    ax: Tuple[float, float, float, float]    # xmin, xmax, ymin, ymax
    n: Tuple[int, int]                       # cells in x and y
    bc: Tuple[str, str]                      # 'periodic' | 'extrapolation' per axis
    cn: float = 0.5                          # CFL number
    precision: str = "fp64"                  # 'fp64' | 'fp32'
    system: str = "pn2d"                     # 'pn2d' | 'slab'
    sigma_a: Field = None
    sigma_s0: Field = None
    # Optional anisotropic scattering: sigma_sl(l) factor so that
    # Sigma_sl = sigma_s0 * sigma_sl_factor[l] for l >= 1 (None = isotropic).
    sigma_sl_factor: Optional[Sequence[float]] = None
    sources: List[Tuple[int, Field]] = dataclasses.field(default_factory=list)
    ic: List[Tuple[int, Field]] = dataclasses.field(default_factory=list)
    time_dependent: bool = False
    nsteps: Optional[int] = None
    t_final: Optional[float] = None


def _const(v: float) -> Field:
    return lambda t, x, y: np.full(np.broadcast(x, y).shape, float(v))


def gaussian_std(x0: float, y0: float, s: float, mass: float = 1.0) -> Field:
    """Isotropic 2D normal density with standard deviation s and given mass."""
    def f(t, x, y):
        r2 = (np.asarray(x) - x0) ** 2 + (np.asarray(y) - y0) ** 2
        return mass / (2.0 * math.pi * s * s) * np.exp(-r2 / (2.0 * s * s))
    return f


def gaussian_paper(sigma: float) -> Field:
    """The paper's Gaussian of section 6.4 with pseudo-time sigma (unit mass)."""
    def f(t, x, y):
        r2 = np.asarray(x) ** 2 + np.asarray(y) ** 2
        return 1.0 / (4.0 * math.pi * sigma) * np.exp(-r2 / (4.0 * sigma))
    return f


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------

def gaussian_p5(n: int = 64, nsteps: int = 100, N: int = 5,
                precision: str = "fp64") -> Problem:
    return Problem(
        name=f"gaussian_p{N}_{n}",
        N=N, ax=(-1.0, 1.0, -1.0, 1.0), n=(n, n),
        bc=("periodic", "periodic"), cn=0.5, precision=precision,
        sigma_a=_const(0.0), sigma_s0=_const(1.0),
        ic=[(0, gaussian_std(0.0, 0.0, 0.1))], nsteps=nsteps)


def checkerboard_layout(seed: int = 1211, n_absorbing: int = 11) -> np.ndarray:
    """7x7 block flags: 1 = absorbing, 0 = scattering, centre block = source.

    The paper's figure with the block layout is not available, so the
    n_absorbing absorbing blocks are drawn at random among the 48 outer blocks
    by a seeded partial Fisher-Yates shuffle."""
    rng = SplitMix64(seed)
    cells = [(bx, by) for by in range(7) for bx in range(7) if (bx, by) != (3, 3)]
    for i in range(n_absorbing):
        j = i + rng.randint(len(cells) - i)
        cells[i], cells[j] = cells[j], cells[i]
    flags = np.zeros((7, 7), dtype=np.int32)   # flags[by, bx]
    for bx, by in cells[:n_absorbing]:
        flags[by, bx] = 1
    return flags


def _block_index(v, lo, width, count):
    k = np.floor((np.asarray(v, dtype=np.float64) - lo) / width).astype(np.int64)
    return np.clip(k, 0, count - 1)


def checkerboard_p13(n: int = 512, N: int = 13, t_final: float = 3.2,
                     seed: int = 1211, precision: str = "fp32") -> Problem:
    flags = checkerboard_layout(seed)

    def absorbing(x, y):
        bx = _block_index(x, 0.0, 1.0, 7)
        by = _block_index(y, 0.0, 1.0, 7)
        return flags[by, bx] == 1

    def sigma_a(t, x, y):
        return np.where(absorbing(x, y), 10.0, 0.0)

    def sigma_s0(t, x, y):
        return np.where(absorbing(x, y), 0.0, 1.0)

    def source(t, x, y):
        bx = _block_index(x, 0.0, 1.0, 7)
        by = _block_index(y, 0.0, 1.0, 7)
        return np.where((bx == 3) & (by == 3), 1.0, 0.0)

    return Problem(
        name=f"checkerboard_p{N}_{n}", N=N, ax=(0.0, 7.0, 0.0, 7.0), n=(n, n),
        bc=("extrapolation", "extrapolation"), cn=0.5, precision=precision,
        sigma_a=sigma_a, sigma_s0=sigma_s0, sources=[(0, source)],
        ic=[], t_final=t_final)


def smooth_log_field(seed: int, lattice: int, lo: float, hi: float,
                     ax: Tuple[float, float, float, float]) -> Field:
    """10**v with v iid uniform in [lo, hi] on a periodic lattice x lattice
    grid of nodes over the domain, bilinearly interpolated (periodic)."""
    rng = SplitMix64(seed)
    v = lo + (hi - lo) * rng.uniforms(lattice * lattice).reshape(lattice, lattice)  # v[iy, ix]
    x0, x1, y0, y1 = ax

    def f(t, x, y):
        u = (np.asarray(x, dtype=np.float64) - x0) / (x1 - x0) * lattice
        w = (np.asarray(y, dtype=np.float64) - y0) / (y1 - y0) * lattice
        iu = np.floor(u)
        iw = np.floor(w)
        fu = u - iu
        fw = w - iw
        i0 = iu.astype(np.int64) % lattice
        j0 = iw.astype(np.int64) % lattice
        i1 = (i0 + 1) % lattice
        j1 = (j0 + 1) % lattice
        val = ((1 - fu) * (1 - fw) * v[j0, i0] + fu * (1 - fw) * v[j0, i1]
               + (1 - fu) * fw * v[j1, i0] + fu * fw * v[j1, i1])
        return 10.0 ** val
    return f


def random_p39(n: int = 1024, N: int = 39, nsteps: int = 200, seed: int = 2205,
               precision: str = "fp32") -> Problem:
    ax = (-1.0, 1.0, -1.0, 1.0)
    return Problem(
        name=f"random_p{N}_{n}", N=N, ax=ax, n=(n, n),
        bc=("periodic", "periodic"), cn=0.5, precision=precision,
        sigma_a=_const(0.0), sigma_s0=smooth_log_field(seed, 32, -1.0, 1.0, ax),
        ic=[(0, gaussian_std(0.0, 0.0, 0.1))], nsteps=nsteps)


def piecewise_blocks(rng: SplitMix64, blocks: int, lo: float, hi: float,
                     ax: Tuple[float, float, float, float], shift: float = 0.37) -> Field:
    """Field constant on a blocks x blocks periodic partition of the domain,
    values iid U[lo, hi].  The block lattice is shifted by `shift` block
    widths so that block edges do not fall on the staggered grid points of
    the grid sizes used (a point exactly on an edge would take either value
    depending on the last bit of its computed coordinate)."""
    vals = lo + (hi - lo) * rng.uniforms(blocks * blocks).reshape(blocks, blocks)
    x0, x1, y0, y1 = ax
    wx = (x1 - x0) / blocks
    wy = (y1 - y0) / blocks

    def f(t, x, y):
        bx = np.floor((np.asarray(x, dtype=np.float64) - x0) / wx - shift).astype(np.int64) % blocks
        by = np.floor((np.asarray(y, dtype=np.float64) - y0) / wy - shift).astype(np.int64) % blocks
        return vals[by, bx]
    return f


def closure_medium(seed: int, n: int = 512, N: int = 39, t_final: float = 0.5,
                   precision: str = "fp32") -> Problem:
    """Instance of the learned-closure workload (seed 2205000 + seed):
    periodic [-1, 1]^2 with n x n cells; sigma_a constant on 8 x 8 blocks,
    iid U[0, 0.5]; sigma_s0 = 10**v on another 8 x 8 block lattice, v iid
    U[-1, 1] (log-uniform in [0.1, 10]); initial R_0^0 the sum of three
    Gaussian pulses (centres U[-0.7, 0.7]^2, std U[0.04, 0.1], mass
    U[0.5, 1.5]); all other moments zero, no source."""
    rng = SplitMix64(2205000 + seed)
    ax = (-1.0, 1.0, -1.0, 1.0)
    sigma_a = piecewise_blocks(rng, 8, 0.0, 0.5, ax)
    log_s = piecewise_blocks(rng, 8, -1.0, 1.0, ax, shift=0.61)
    pulses = []
    for _ in range(3):
        u = rng.uniforms(4)
        pulses.append(gaussian_std(-0.7 + 1.4 * u[0], -0.7 + 1.4 * u[1], 0.04 + 0.06 * u[2], mass=0.5 + u[3]))

    def sigma_s0(t, x, y):
        return 10.0 ** log_s(t, x, y)

    def ic0(t, x, y):
        return sum(f(t, x, y) for f in pulses)
    return Problem(
        name=f"closure_medium_{seed}_p{N}_{n}", N=N, ax=ax, n=(n, n), bc=("periodic", "periodic"), cn=0.5,
        precision=precision, sigma_a=sigma_a, sigma_s0=sigma_s0, ic=[(0, ic0)], t_final=t_final)


def closure_c5(seed: int, n: int = 512, N: int = 39, t_final: float = 3.2, precision: str = "fp32") -> Problem:
    """Instance of the learned-closure workload in its source-driven form
    (seed 2205500 + seed): [0, 7]^2 with n x n cells and extrapolation
    boundaries, to t = 3.2 (the checkerboard's domain and time), the
    batched workload's media scaled to the domain: sigma_a iid U[0, 5] and
    sigma_s0 iid U[0, 10] on 8 x 8 blocks; an isotropic Gaussian source of
    R_0^0 (std 0.35, unit mass) centred uniformly in [1.75, 5.25]^2; zero
    initial state."""
    rng = SplitMix64(2205500 + seed)
    ax = (0.0, 7.0, 0.0, 7.0)
    sigma_a = piecewise_blocks(rng, 8, 0.0, 5.0, ax)
    sigma_s0 = piecewise_blocks(rng, 8, 0.0, 10.0, ax, shift=0.61)
    c = rng.uniforms(2)
    src = gaussian_std(1.75 + 3.5 * c[0], 1.75 + 3.5 * c[1], 0.35)
    return Problem(
        name=f"closure_c5_{seed}_p{N}_{n}", N=N, ax=ax, n=(n, n), bc=("extrapolation", "extrapolation"), cn=0.5,
        precision=precision, sigma_a=sigma_a, sigma_s0=sigma_s0, sources=[(0, src)], ic=[], t_final=t_final)


BEAM_ANGLE = math.pi / 6
BEAM_INTERFACE = 0.3


def beam(moments: Sequence[float], n: int = 150, t_final: float = 0.6, g: float = 0.85,
         precision: str = "fp32", interface: float = BEAM_INTERFACE) -> Problem:
    """The beam of section 6: a continuous source qbar(x) delta(Omega -
    Omega_0), Omega_0 in the plane at the angle pi/6 to the x axis, qbar the
    line source's Gaussian (pseudo-time 3.2e-4, unit mass) at the origin, on
    [-0.6, 0.6]^2 with extrapolation boundaries; void for x < 0.3, for
    x >= 0.3 no absorption and Henyey-Greenstein scattering
    Sigma_sl = 100 g^l.  `moments` are the beam direction's moments of the
    components (their real harmonics at Omega_0, one per component: the
    order N is len(moments) = (N+1)(N+2)/2).  `interface` moves the medium's
    edge (beyond 0.6: all void)."""
    ncomp = len(moments)
    N = int(round((math.sqrt(8 * ncomp + 1) - 3) / 2))
    if (N + 1) * (N + 2) // 2 != ncomp:
        raise ValueError("moments must hold one value per component of a 2D system")
    qbar = gaussian_paper(3.2e-4)

    def medium(x):
        return np.asarray(x) >= interface

    def sigma_a(t, x, y):
        return 0.0 * np.asarray(x) + 0.0 * np.asarray(y)

    def sigma_s0(t, x, y):
        return np.where(medium(x), 100.0, 0.0) + 0.0 * np.asarray(y)

    def scaled(c):
        return lambda t, x, y: c * qbar(t, x, y)

    sources = [(j, scaled(float(c))) for j, c in enumerate(moments) if abs(c) > 1e-14]
    return Problem(name=f"beam_p{N}_{n}" + ("" if interface == BEAM_INTERFACE else "_void"), N=N, ax=(-0.6, 0.6, -0.6, 0.6), n=(n, n),
                   bc=("extrapolation", "extrapolation"), cn=0.5, precision=precision,
                   sigma_a=sigma_a, sigma_s0=sigma_s0, sigma_sl_factor=[g ** l for l in range(N + 1)],
                   sources=sources, ic=[], t_final=t_final)


def batched_instance(k: int, nsteps: int = 100) -> Problem:
    """Instance k of the batched workload (seed 12112205 + k)."""
    rng = SplitMix64(12112205 + k)
    sizes = list(range(64, 513, 32))
    n = sizes[rng.randint(len(sizes))]
    N = [3, 5, 7, 9, 11, 13, 15][rng.randint(7)]
    bc = ["periodic", "extrapolation"][rng.randint(2)]
    ax = (0.0, 1.0, 0.0, 1.0)
    sigma_a = piecewise_blocks(rng, 8, 0.0, 5.0, ax)
    sigma_s0 = piecewise_blocks(rng, 8, 0.0, 10.0, ax)
    cx = 0.25 + 0.5 * rng.uniform()
    cy = 0.25 + 0.5 * rng.uniform()
    return Problem(
        name=f"batched_{k}", N=N, ax=ax, n=(n, n), bc=(bc, bc), cn=0.5,
        precision="fp32", sigma_a=sigma_a, sigma_s0=sigma_s0,
        sources=[(0, gaussian_std(cx, cy, 0.05))], ic=[], nsteps=nsteps)


def fourier_mode_ic(count: int, seed: int):
    """Random complex amplitudes for a Fourier-mode initial condition."""
    rng = SplitMix64(seed)
    re = rng.uniforms(count) * 2 - 1
    im = rng.uniforms(count) * 2 - 1
    return re + 1j * im


# ---------------------------------------------------------------- config files
CONFIG_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "configs")
_GENERATORS = {"gaussian_p5": gaussian_p5, "checkerboard_p13": checkerboard_p13, "random_p39": random_p39,
               "batched_instance": batched_instance, "closure_medium": closure_medium, "closure_c5": closure_c5}


def load_config(name_or_path: str):
    """A run described by a JSON file (configs/<name>.json, or a path): the
    generator of this module it names with its keyword arguments, called
    once, once per instance k ("instances": count, k passed as the first
    argument) or once per seed ("seeds").  Returns (problems, description)."""
    path = name_or_path if name_or_path.endswith(".json") else os.path.join(CONFIG_DIR, name_or_path + ".json")
    with open(path) as f:
        c = json.load(f)
    gen = _GENERATORS[c["generator"]]
    kw = dict(c.get("kwargs", {}))
    if "instances" in c:
        problems = [gen(k, **kw) for k in range(int(c["instances"]))]
    elif "seeds" in c:
        problems = [gen(int(s), **kw) for s in c["seeds"]]
    else:
        problems = [gen(**kw)]
    return problems, c.get("description", c.get("name", ""))
