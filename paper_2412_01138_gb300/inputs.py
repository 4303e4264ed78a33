"""Seeded synthetic problem descriptors for the Parareal EIFE-linear solver.

This module only *describes* inputs: grid sizes, the box, D, the time
partition, the interpolation nodes of the two exponential Runge-Kutta
tableaux and the parameters of separable source terms and initial data.
It contains none of the method's arithmetic (no quadrature, no transform,
no phi-function, no time stepping); both the CUDA library and the CPU
oracle evaluate these descriptors with code of their own.

Random draws use SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): a 64-bit counter advanced by
0x9E3779B97F4A7C15 and finalised by two xor-shift-multiply rounds.  A draw is
mapped to a double in [0, 1) as (x >> 11) * 2^-53, and normals come from the
Box-Muller transform.  The CUDA library implements the same generator in C
for seeded random interpolation nodes, so both sides draw identical nodes.

Descriptor conventions (shared with ``include/pe.h``):

* spatial factor kinds (one per axis of a separable term)
    S_ONE   = 0 : 1
    S_SIN   = 1 : sin(p0*x + p1)
    S_GAUSS = 2 : exp(-(x - p0)^2 / (2 p1^2))
    S_POLY  = 3 : p0 + p1 x + p2 x^2 + p3 x^3
    S_MOVING_HAT = 4 : max(1 - |x - c(t)|/p3, 0), c(t) = p0 + p1 sin(2 pi p2 t)
                   (depends on t: only the general forcing path takes it)
* time factor kinds
    T_EXP   = 0 : exp(p0*t)            (p0 = 0 gives a constant)
    T_SIN   = 1 : sin(p0*t + p1)
* a separable term is  amp * time(t) * prod_a spatial_a(x_a).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence, Tuple

S_ONE, S_SIN, S_GAUSS, S_POLY, S_MOVING_HAT = 0, 1, 2, 3, 4
T_EXP, T_SIN = 0, 1

_MASK64 = (1 << 64) - 1

#: smallest admissible gap between two seeded random interpolation nodes
#: (the Lagrange basis needs distinct nodes; near-coincident nodes make the
#: Vandermonde system behind the weights ill-conditioned).
MIN_NODE_GAP = 1e-3


class SplitMix64:
    """SplitMix64 stream (published definition; see module docstring)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_range(self, a: float, b: float) -> float:
        return a + (b - a) * self.uniform()

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform on {lo, ..., hi} (inclusive)."""
        return lo + min(int(self.uniform() * (hi - lo + 1)), hi - lo)

    def normal(self) -> float:
        """Standard normal by Box-Muller (one of the pair is used)."""
        u1 = 1.0 - self.uniform()  # (0, 1]
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def draw_random_nodes(s: int, seed: int) -> Tuple[float, ...]:
    """s distinct interpolation nodes c_i ~ U(0,1), sorted ascending.

    The whole set is redrawn from the same stream while its smallest gap is
    below MIN_NODE_GAP.  The CUDA library's seeded-node option
    (``pe_tableau.random``) follows exactly this procedure.
    """
    rng = SplitMix64(seed)
    while True:
        c = sorted(rng.uniform() for _ in range(s))
        if s == 1 or min(b - a for a, b in zip(c, c[1:])) >= MIN_NODE_GAP:
            return tuple(c)


def uniform_nodes(s: int) -> Tuple[float, ...]:
    """The paper's "uniformly selected" nodes, read as c_i = (i-1)/s."""
    return tuple(i / s for i in range(s))


@dataclass(frozen=True)
class Factor:
    kind: int
    p: Tuple[float, ...] = ()

    def params4(self) -> Tuple[float, float, float, float]:
        q = tuple(self.p) + (0.0,) * (4 - len(self.p))
        return q[:4]


@dataclass(frozen=True)
class Term:
    """amp * time(t) * prod_a factors[a](x_a)."""

    amp: float
    factors: Tuple[Factor, ...]
    tkind: int = T_EXP
    tp: Tuple[float, float] = (0.0, 0.0)


@dataclass(frozen=True)
class Problem:
    d: int
    n: Tuple[int, ...]                       # interior nodes per axis
    box: Tuple[Tuple[float, float], ...]     # (lo, hi) per axis
    D: float
    t0: float
    T: float
    N: int                                   # Parareal slices
    M: int                                   # fine substeps per slice
    fine_nodes: Tuple[float, ...]            # c^F, q nodes in [0, 1]
    coarse_nodes: Tuple[float, ...]          # c^G, p nodes in [0, 1]
    u0: Tuple[Term, ...]                     # initial data (time factors ignored)
    forcing: Tuple[Term, ...]
    quad_pts: int = 3                        # Gauss points per axis per element
    tol: float = 1e-12
    exact: Optional[Tuple[Term, ...]] = None  # exact solution, when known
    label: str = ""
    boundary: Tuple[Term, ...] = ()          # Dirichlet data: separable terms on the closed box
    periodic: Tuple[bool, ...] = ()          # per-axis periodic flags (missing = Dirichlet)

    @property
    def ndof(self) -> int:
        out = 1
        for v in self.n:
            out *= v
        return out

    @property
    def q(self) -> int:
        return len(self.fine_nodes)

    @property
    def p(self) -> int:
        return len(self.coarse_nodes)

    @property
    def R(self) -> int:
        return len(self.forcing)


# ---------------------------------------------------------------------------
# building blocks
# ---------------------------------------------------------------------------

def sin_mode(d: int, box, D: float, rate: float = -1.0):
    """Manufactured u = e^{rate t} prod_a sin(pi (x_a - lo_a)/L_a) and its f.

    f = u_t - D Lap u = (rate + D pi^2 sum_a 1/L_a^2) u.
    """
    facs = tuple(Factor(S_SIN, (math.pi / (hi - lo), -math.pi * lo / (hi - lo))) for lo, hi in box)
    kappa = sum((math.pi / (hi - lo)) ** 2 for lo, hi in box)
    u0 = (Term(1.0, facs),)
    f = (Term(rate + D * kappa, facs, T_EXP, (rate, 0.0)),)
    exact = (Term(1.0, facs, T_EXP, (rate, 0.0)),)
    return u0, f, exact


def gaussian_bumps(rng: SplitMix64, d: int, count: int, omega=(1.0, 20.0),
                   width=(0.02, 0.1)) -> Tuple[Term, ...]:
    """Bumps a*exp(-|x-c|^2/(2w^2))*sin(w_t t + phi) on the unit box.

    Draw order per bump: c_1..c_d ~ U(0,1), w ~ U[width], a ~ N(0,1),
    omega ~ U[omega], phi ~ U[0, 2 pi).
    """
    out = []
    for _ in range(count):
        c = [rng.uniform() for _ in range(d)]
        w = rng.uniform_range(*width)
        a = rng.normal()
        om = rng.uniform_range(*omega)
        ph = rng.uniform_range(0.0, 2.0 * math.pi)
        out.append(Term(a, tuple(Factor(S_GAUSS, (ci, w)) for ci in c), T_SIN, (om, ph)))
    return tuple(out)


# ---------------------------------------------------------------------------
# the five benchmark workloads and the paper's examples
# ---------------------------------------------------------------------------

def config1() -> Problem:
    """1D, 63 interior nodes, D=1, manufactured e^{-t} sin(pi x); 8 x 16, RK2/RK2, FP64."""
    box = ((0.0, 1.0),)
    u0, f, ex = sin_mode(1, box, 1.0)
    return Problem(1, (63,), box, 1.0, 0.0, 1.0, 8, 16, uniform_nodes(2), uniform_nodes(2),
                   u0, f, 3, 1e-12, ex, "d1_n63_N8_M16")


def config2(seed: int = 2) -> Problem:
    """2D 255^2, D=0.1, manufactured + 8 bumps; 32 x 64, RK4 fine, random-node RK2 coarse."""
    box = ((0.0, 1.0), (0.0, 1.0))
    D = 0.1
    u0, f, _ = sin_mode(2, box, D)
    rng = SplitMix64(seed)
    coarse = draw_random_nodes(2, seed)
    bumps = gaussian_bumps(rng, 2, 8)
    return Problem(2, (255, 255), box, D, 0.0, 1.0, 32, 64, uniform_nodes(4), coarse,
                   u0, f + bumps, 3, 1e-6, None, "d2_n255_N32_M64_bumps8")


def config3(seed: int = 3, n: int = 127, N: int = 64) -> Problem:
    """3D 127^3, D=0.05, manufactured + 16 bumps; 64 x 32, RK4 fine, RK2 {0,1/2} coarse."""
    box = ((0.0, 1.0),) * 3
    D = 0.05
    u0, f, _ = sin_mode(3, box, D)
    rng = SplitMix64(seed)
    bumps = gaussian_bumps(rng, 3, 16)
    return Problem(3, (n, n, n), box, D, 0.0, 1.0, N, 32, uniform_nodes(4), uniform_nodes(2),
                   u0, f + bumps, 3, 1e-6, None, f"d3_n{n}_N{N}_M32_bumps16")


def config4_problem(index: int, base_seed: int = 4) -> Problem:
    """One of the 512 uneven 2D problems of the batched workload."""
    rng = SplitMix64((base_seed << 32) | index)
    lo, hi = math.log(31.0), math.log(511.0)
    nx = int(round(math.exp(rng.uniform_range(lo, hi))))
    ny = int(round(math.exp(rng.uniform_range(lo, hi))))
    D = math.exp(rng.uniform_range(math.log(0.01), math.log(1.0)))
    nb = rng.randint(4, 16)
    N = rng.randint(16, 64)
    box = ((0.0, 1.0), (0.0, 1.0))
    u0, f, _ = sin_mode(2, box, D)
    bumps = gaussian_bumps(rng, 2, nb)
    return Problem(2, (nx, ny), box, D, 0.0, 1.0, N, 32, uniform_nodes(4), uniform_nodes(2),
                   u0, f + bumps, 3, 1e-6, None, f"batch{index}_{nx}x{ny}_N{N}")


def config4(count: int = 512, base_seed: int = 4) -> List[Problem]:
    return [config4_problem(i, base_seed) for i in range(count)]


def config5(seed: int = 1, n: int = 511, N: int = 128) -> Problem:
    """2D 511^2, D=0.02, T=2, 12 bumps with omega ~ U[1,50]; 128 x 32, RK4/RK2."""
    box = ((0.0, 1.0), (0.0, 1.0))
    u0, _, _ = sin_mode(2, box, 0.02)
    rng = SplitMix64(seed)
    bumps = gaussian_bumps(rng, 2, 12, omega=(1.0, 50.0))
    return Problem(2, (n, n), box, 0.02, 0.0, 2.0, N, 32, uniform_nodes(4), uniform_nodes(2),
                   u0, bumps, 3, 1e-6, None, f"d2_n{n}_N{N}_M32_bumps12_seed{seed}")


def example1(Nx: int, N: int, M: int, q: int, p: int, quad_pts: int = 3) -> Problem:
    """Example 1 of the paper: u = x(1-x)e^t on [0,1], t in [0,1], D = 1."""
    box = ((0.0, 1.0),)
    poly = Factor(S_POLY, (0.0, 1.0, -1.0, 0.0))
    u0 = (Term(1.0, (poly,)),)
    f = (Term(1.0, (Factor(S_POLY, (2.0, 1.0, -1.0, 0.0)),), T_EXP, (1.0, 0.0)),)
    exact = (Term(1.0, (poly,), T_EXP, (1.0, 0.0)),)
    return Problem(1, (Nx - 1,), box, 1.0, 0.0, 1.0, N, M, uniform_nodes(q), uniform_nodes(p),
                   u0, f, quad_pts, 0.0, exact, f"ex1_Nx{Nx}_{N}x{M}")


def example2(Nx: int, Ny: int, N: int, M: int, q: int, p: int, quad_pts: int = 3) -> Problem:
    """Example 2: u = e^{-4 pi^2 t} sin(pi(x-1/4)) sin(2 pi(y-1/8)) on [1/4,5/4]x[1/8,5/8], T=0.6."""
    box = ((0.25, 1.25), (0.125, 0.625))
    fx = Factor(S_SIN, (math.pi, -math.pi * 0.25))
    fy = Factor(S_SIN, (2.0 * math.pi, -2.0 * math.pi * 0.125))
    r = -4.0 * math.pi ** 2
    u0 = (Term(1.0, (fx, fy)),)
    f = (Term(math.pi ** 2, (fx, fy), T_EXP, (r, 0.0)),)
    exact = (Term(1.0, (fx, fy), T_EXP, (r, 0.0)),)
    return Problem(2, (Nx - 1, Ny - 1), box, 1.0, 0.0, 0.6, N, M, uniform_nodes(q), uniform_nodes(p),
                   u0, f, quad_pts, 0.0, exact, f"ex2_{Nx}x{Ny}_{N}x{M}")


def example3(Nx: int, N: int, M: int, q: int, p: int, quad_pts: int = 3) -> Problem:
    """Example 3: D = 1/8 on [0,1/4]x[1/8,3/8]x[0,1/4], T = 0.4, single sine mode."""
    box = ((0.0, 0.25), (0.125, 0.375), (0.0, 0.25))
    fs = tuple(Factor(S_SIN, (4.0 * math.pi, -4.0 * math.pi * s)) for s in (0.25, 0.125, 0.5))
    r = -4.0 * math.pi ** 2
    u0 = (Term(1.0, fs),)
    f = (Term(2.0 * math.pi ** 2, fs, T_EXP, (r, 0.0)),)
    exact = (Term(1.0, fs, T_EXP, (r, 0.0)),)
    return Problem(3, (Nx - 1,) * 3, box, 0.125, 0.0, 0.4, N, M, uniform_nodes(q), uniform_nodes(p),
                   u0, f, quad_pts, 0.0, exact, f"ex3_{Nx}_{N}x{M}")


def example4(Nx: int, alpha: float, freq: float, N: int = 4, M: int = 16, q: int = 2, p: int = 2,
             quad_pts: int = 3) -> Problem:
    """Example 4: u_t = alpha u_xx + g on [0,1], T = 1, u0 = 4x(1-x), g a hat of half-width
    w = 0.05 and height 100 sqrt(alpha) centred at c(t) = 0.5 + (0.5 - w) sin(2 pi f t)."""
    w = 0.05
    box = ((0.0, 1.0),)
    u0 = (Term(1.0, (Factor(S_POLY, (0.0, 4.0, -4.0, 0.0)),)),)
    g = (Term(100.0 * math.sqrt(alpha), (Factor(S_MOVING_HAT, (0.5, 0.5 - w, freq, w)),)),)
    return Problem(1, (Nx - 1,), box, alpha, 0.0, 1.0, N, M, uniform_nodes(q), uniform_nodes(p),
                   u0, g, quad_pts, 0.0, None, f"ex4_Nx{Nx}_a{alpha}_f{freq}_{N}x{M}")


def moving_hat_2d(n=(63, 47), N=4, M=8, seed=21) -> Problem:
    """2D source: a hat moving along x times a fixed Gaussian along y, plus seeded bumps."""
    box = ((0.0, 1.0), (0.0, 1.0))
    rng = SplitMix64(seed)
    u0, f, _ = sin_mode(2, box, 0.05)
    hat = Term(3.0, (Factor(S_MOVING_HAT, (0.5, 0.35, 2.0, 0.1)), Factor(S_GAUSS, (0.5, 0.15))))
    return Problem(2, tuple(n), box, 0.05, 0.0, 1.0, N, M, uniform_nodes(4), uniform_nodes(2),
                   u0, f + (hat,) + gaussian_bumps(rng, 2, 3), 3, 1e-6, None, "moving_hat_2d")


def scaled(prob: Problem, n: Sequence[int], N: Optional[int] = None, M: Optional[int] = None) -> Problem:
    """Same problem on another grid / time partition (used for small parity cases)."""
    return replace(prob, n=tuple(n), N=prob.N if N is None else N, M=prob.M if M is None else M,
                   label=prob.label + f"_scaled{'x'.join(map(str, n))}")
