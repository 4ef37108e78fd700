"""Seeded, synthetic problem definitions shared by the tests, the benchmark and the oracle runs.

This module holds no arithmetic of the method: only the problem parameters and the
counter-based random draws (splitmix64) that pick amplitudes and batch members. The
solver on each side (CUDA library, CPU oracle) computes everything else itself.

The paper (arXiv:1006.0663) prints no grid sizes or step counts; the five workloads
below are the benchmark configurations the library is measured on:

* ``c1``: FP64, a = 0.5, s = -2, m = 2, r* in [-50, 150] x 256, theta x 64, 1000 steps;
* ``c2``: double-double, a = 0.9, s = -2, m = 2, r* in [-100, 400] x 2048, theta x 128,
  40000 steps, waveform at r* = 300 every step;
* ``c3``: quad-double, a = 0.99, s = 0, m = 0, r* in [-100, 400] x 1024, theta x 64,
  40000 steps;
* ``c4``: 64 double-double instances of uneven size, 5000 steps each;
* ``c5``: FP64 and double-double, a = 0.9, s = -2, m = 2, r* in [-200, 1800] x 16384,
  theta x 512, 2000 steps;
* ``tails``: quad-double, a = 0.9, s = 0, m = 0, l' = 0 pulse, r* in [-760, 840] x 12801,
  theta x 32, 48000 steps (t = 1500 M), observer at r* = 50 (the Kerr-tails study).

Every instance has dt = 0.25 dr* as its outer (sampling) step, integrated with
``substeps`` Lax-Wendroff iterations of dt/substeps; ``substeps`` is fixed per workload
by the stability analysis of the discrete operator (``oracle/stability.py``).
"""
from __future__ import annotations

import dataclasses

MASK64 = (1 << 64) - 1


def splitmix64(state: int):
    """Steele, Lea & Flood (2014) SplittableRandom / splitmix64 output function.

    Returns (next_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


class Draws:
    """A counter-based stream of splitmix64 outputs from a seed."""

    def __init__(self, seed: int):
        self.state = int(seed) & MASK64

    def u64(self) -> int:
        self.state, z = splitmix64(self.state)
        return z

    def unit(self) -> float:
        """Exact double in [0, 1): (u64 >> 11) * 2^-53."""
        return (self.u64() >> 11) * (2.0 ** -53)

    def below(self, n: int) -> int:
        """Integer in [0, n) by multiply-shift of the top 53 bits (exact for n < 2^11)."""
        return (self.u64() >> 11) * n >> 53


def amplitudes(seed: int):
    """Complex pulse amplitude A = A_R + i A_I, each uniform in [0.5, 1), exact doubles."""
    d = Draws(seed)
    ar = 0.5 + 0.5 * d.unit()
    ai = 0.5 + 0.5 * d.unit()
    return ar, ai


def parity_of(m: int, s: int) -> int:
    """Sign of the axis reflection of a spin-weight-s, azimuthal-m field: (-1)^(m+s)."""
    return 1 if (m + s) % 2 == 0 else -1


@dataclasses.dataclass(frozen=True)
class Problem:
    name: str
    M: float
    a: float
    s: int
    m: int
    rstar_min: float
    rstar_max: float
    n_r: int
    n_theta: int
    steps: int            # outer steps of dt = 0.25 dr*
    substeps: int         # Lax-Wendroff iterations per outer step
    words: int            # 1 FP64, 2 double-double, 4 quad-double
    ell: int              # multipole of the initial angular profile
    seed: int
    center: float = 40.0
    width: float = 4.0
    rstar_obs: float = 300.0
    theta_order: int = 10
    ko_sigma: float = 0.0  # r* dissipation (not in the paper; 0 = the paper's scheme)
    ko_theta: float = 0.0  # theta dissipation (not in the paper; 0 = the paper's scheme)
    theta_filter: int = 0  # theta filter l_cut (not in the paper; 0 = the paper's scheme)
    theta_filter_period: int = 1  # outer steps between its projections

    @property
    def dr(self) -> float:
        return (self.rstar_max - self.rstar_min) / (self.n_r - 1)

    @property
    def dt(self) -> float:
        return 0.25 * self.dr

    @property
    def parity(self) -> int:
        return parity_of(self.m, self.s)

    @property
    def amps(self):
        return amplitudes(self.seed)

    @property
    def points(self) -> int:
        return self.n_r * self.n_theta

    def with_(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


# Substep counts k: the smallest k for which the excess (numerical over exact) growth of the
# most unstable discrete mode over the whole run stays below 10x; see oracle/stability.py.
# r* dissipation sigma = 2 (not in the paper): with it c1 stays bounded over its 1000 steps
# (without it a near-stationary short r* wave grows as e^{0.15 t} from t ~ 150 M on) and c5
# grows only as the physics does over its 2000; on c2 and c3 it does not stop the growth of
# trapped high-l modes that these r* grids do not resolve.
C1 = Problem("c1", 1.0, 0.5, -2, 2, -50.0, 150.0, 256, 64, 1000, 46, 1, 2, 1, rstar_obs=100.0, ko_sigma=2.0)
C2 = Problem("c2", 1.0, 0.9, -2, 2, -100.0, 400.0, 2048, 128, 40000, 88, 2, 2, 2, ko_sigma=2.0)
C3 = Problem("c3", 1.0, 0.99, 0, 0, -100.0, 400.0, 1024, 64, 40000, 20, 4, 0, 3, ko_sigma=2.0,
             theta_filter=7, theta_filter_period=8)
C5 = Problem("c5", 1.0, 0.9, -2, 2, -200.0, 1800.0, 16384, 512, 2000, 81, 1, 2, 5, rstar_obs=1000.0,
             ko_sigma=2.0)

# Kerr-tails study (Sec. 3.C, Fig. 1): a scalar field (s = 0, m = 0) started as a pure l' = 0
# Gaussian pulse on a = 0.9, observed at r* = 50 for t = 1500 M. The r* boundaries are far
# enough that what they reflect (from 15 pulse widths ahead of the pulse centre on) reaches
# the observer only after t = 1500 M, so the late-time field there is the boundary-free tail.
# Quad-double: the multipoles l = 0..8 of the late field are tens of orders of magnitude apart.
# dr* = 1/8 with 2 iterations per dt = 0.25 dr*: the scheme's own damping of short r*
# wavelengths then outweighs the growth of near-stationary short waves where the lower-order
# terms of the system amplify a frozen wave (with dr* = 1/2 and 9 iterations they grow as
# e^{0.2 t} from t ~ 150 M on).
TAILS = Problem("tails", 1.0, 0.9, 0, 0, -760.0, 840.0, 12801, 32, 48000, 2, 4, 0, 7, center=25.0,
                width=4.0, rstar_obs=50.0)

CONFIGS = {p.name: p for p in (C1, C2, C3, C5, TAILS)}

BATCH_SIZE = 64
BATCH_STEPS = 5000
BATCH_SEED_BASE = 1000
BATCH_THETA = (32, 64, 128, 256)
# Substep counts of the 64 batch members, from the same stability analysis.
BATCH_SUBSTEPS = (80, 6, 12, 3, 4, 2, 3, 1, 5, 3, 38, 10, 92, 24, 19, 5, 6, 12, 121, 4, 23, 46, 5,
                  24, 158, 12, 4, 10, 13, 7, 157, 132, 13, 72, 6, 155, 18, 30, 8, 14, 274, 71, 12,
                  142, 98, 9, 41, 10, 111, 64, 7, 12, 23, 6, 66, 11, 4, 88, 8, 16, 454, 43, 133, 65)


def batch_member(i: int, substeps: int | None = None) -> Problem:
    """Instance i of the 64-member double-double batch (seed 1000 + i).

    Draw order: n_r uniform in [512, 4096], n_theta in {32, 64, 128, 256}, m in [-4, 4],
    s in {0, -1, -2}, a uniform in [0, 0.99], then the amplitudes. ell = max(|m|, |s|),
    r* in [-100, 400]."""
    d = Draws(BATCH_SEED_BASE + i)
    n_r = 512 + d.below(4096 - 512 + 1)
    n_theta = BATCH_THETA[d.below(4)]
    m = -4 + d.below(9)
    s = -d.below(3)
    a = 0.99 * d.unit()
    seed = d.u64() & 0x7FFFFFFF
    ell = max(abs(m), abs(s))
    k = substeps if substeps is not None else BATCH_SUBSTEPS[i]
    return Problem(f"c4[{i}]", 1.0, a, s, m, -100.0, 400.0, n_r, n_theta, BATCH_STEPS, k, 2, ell,
                   seed)
