"""Seeded synthetic inputs for the fractional-diffusion workloads.

This module only *samples* problem data on the host (grids, diffusion
coefficients, initial values, source factors); it contains none of the
solver's arithmetic.  Both the CPU oracle and the CUDA path consume exactly
the arrays produced here, so they see identical bits.

Random draws use SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written here from its
published definition.

Problem family (Massei, Mazza, Robol, arXiv:1804.05522):
  * 1D: Eq. (system_FD) of §2.2.1 on [0,1], nodes x_i = i h, h = 1/(N+1).
  * 2D: the Sylvester step of Eq. (sylv-timestepping), §4.2, on [0,1]^2 with
    separable coefficients d_{1,±}(x), d_{2,±}(y) (Remark rem:diff, §4).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1804055220
_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (64-bit state, golden-gamma increment)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def normal(self) -> float:
        """Standard normal by Box-Muller (first variate only)."""
        u1 = self.uniform()
        u2 = self.uniform()
        u1 = max(u1, 1e-300)
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + int(self.uniform() * (hi - lo + 1))

    def normal_array(self, shape) -> np.ndarray:
        n = int(np.prod(shape))
        return np.array([self.normal() for _ in range(n)], dtype=np.float64).reshape(shape)


def grid(N: int) -> np.ndarray:
    """Interior nodes x_i = i h, i = 1..N, h = 1/(N+1) on [0,1] (§2.2.1, Eq. (part))."""
    h = 1.0 / (N + 1)
    return np.arange(1, N + 1, dtype=np.float64) * h


def coeff_power(alpha: float, x: np.ndarray, a: float, b: float):
    """d_+(x) = Γ(3-α)(a + x)^α and d_-(x) = Γ(3-α)(b - x)^α, sampled on the host."""
    gam = math.gamma(3.0 - alpha)
    return gam * (a + x) ** alpha, gam * (b - x) ** alpha


@dataclass
class OpSpec:
    """One 1D operator  shift*I + dt/h^α (D_+ T_α + D_- T_αᵀ)  (Eq. (system_FD))."""
    N: int
    alpha: float
    h: float
    dt: float
    shift: float
    d_plus: np.ndarray
    d_minus: np.ndarray
    leaf: int
    tol: float


@dataclass
class Workload:
    name: str
    dim: int
    steps: int
    dt: float
    ops: list                      # [OpSpec] (1D) or [OpSpec_x, OpSpec_y] (2D)
    u0: np.ndarray                 # (N,) or (N, N) column-major semantics X[i, j] = u(x_i, y_j)
    src_left: np.ndarray           # (N, r) source factors in x
    src_right: np.ndarray | None   # (N, r) source factors in y (2D) else None
    src_amp: np.ndarray            # (r,)  w_l(t) = amp_l + sin_amp_l * sin(omega_l t)
    src_sin_amp: np.ndarray
    src_omega: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.ops[0].N

    def source_weights(self, t: float) -> np.ndarray:
        return self.src_amp + self.src_sin_amp * np.sin(self.src_omega * t)

    def source(self, t: float) -> np.ndarray:
        """Dense sampling of f(., t) (host, for checks)."""
        w = self.source_weights(t)
        if self.dim == 1:
            return self.src_left @ w
        return (self.src_left * w) @ self.src_right.T


def u0_profile(x: np.ndarray) -> np.ndarray:
    return x * x * (1.0 - x) * (1.0 - x)


def fd1d(N=1024, alpha=1.5, steps=32, leaf=64, tol=1e-10, seed_index=0, coeff_scale=1.0) -> Workload:
    """1D workload: GL shifted FD, implicit Euler, seeded sum of 8 random sines as source."""
    x = grid(N)
    h = 1.0 / (N + 1)
    dt = 1.0 / steps
    dp, dm = coeff_power(alpha, x, 0.0, 1.0)
    dp, dm = dp * coeff_scale, dm * coeff_scale
    rng = SplitMix64(SEED_BASE + seed_index)
    f = np.zeros(N)
    for _ in range(8):
        a = rng.normal()
        om = rng.randint(1, 64)
        ph = 2.0 * math.pi * rng.uniform()
        f += a * np.sin(math.pi * om * x + ph)
    op = OpSpec(N, alpha, h, dt, 1.0, dp, dm, leaf, tol)
    return Workload(f"fd1d_n{N}_a{alpha}", 1, steps, dt, [op], u0_profile(x), f[:, None].copy(), None,
                    np.array([1.0]), np.array([0.0]), np.array([0.0]))


def fd2d(N=256, alpha=(1.3, 1.7), steps=50, leaf=64, tol=1e-10, coeff_scale=(1.0, 1.0)) -> Workload:
    """2D workload on [0,1]^2 with the paper's source (§5.1):
    f = 100 (sin 10πx cos πy + sin 10t sin πx · y(1-y)), rank <= 2 in (x, y).
    Coefficients: d_{1,±} = Γ(3-α1) x^α1, Γ(3-α1)(1-x)^α1 ; d_{2,±} = Γ(3-α2)(1+y)^α2, Γ(3-α2)(2-y)^α2.
    """
    x = grid(N)
    h = 1.0 / (N + 1)
    dt = 1.0 / steps
    a1, a2 = alpha
    dxp, dxm = coeff_power(a1, x, 0.0, 1.0)
    dyp, dym = coeff_power(a2, x, 1.0, 2.0)
    opx = OpSpec(N, a1, h, dt, 0.5, dxp * coeff_scale[0], dxm * coeff_scale[0], leaf, tol)
    opy = OpSpec(N, a2, h, dt, 0.5, dyp * coeff_scale[1], dym * coeff_scale[1], leaf, tol)
    u = u0_profile(x)
    U0 = np.outer(u, u)
    FL = np.stack([np.sin(10 * math.pi * x), np.sin(math.pi * x)], 1)
    FR = np.stack([np.cos(math.pi * x), x * (1.0 - x)], 1)
    return Workload(f"fd2d_n{N}_a{a1}_{a2}", 2, steps, dt, [opx, opy], U0, FL, FR,
                    np.array([100.0, 0.0]), np.array([0.0, 100.0]), np.array([0.0, 10.0]))


def fd2d_paper(N=4096, alpha=(1.3, 1.7), steps=8, leaf=256, tol=1e-8) -> Workload:
    """The shape of the paper's 2D experiment (§6.2): constant diffusion
    coefficients d_{1,±} = d_{2,±} = 1, Δt = 1, 8 implicit-Euler steps, the
    paper's source f (rank <= 2), on the grid x_i = i/(N+1) (the printed
    Δx = 1/(N+2) is read as the grid of §2.2.1), U0 = u0(x) u0(y)ᵀ."""
    w = fd2d(N=N, alpha=alpha, steps=steps, leaf=leaf, tol=tol)
    w.dt = 1.0
    for op in w.ops:
        op.dt = 1.0
        op.d_plus = np.ones(N)
        op.d_minus = np.ones(N)
    w.name = f"fd2d_paper_n{N}_a{alpha[0]}_{alpha[1]}"
    return w


def u0_factors(w: Workload):
    """Factors (W0, Z0) of the 2D initial value U0 = u0(x) u0(y)ᵀ (rank one),
    for the factored time loop."""
    x = grid(w.N)
    u = u0_profile(x)
    return u[:, None].copy(), u[:, None].copy()


def random_matrix(m: int, n: int, seed: int) -> np.ndarray:
    """Seeded dense test matrix (standard normal entries), column-major semantics."""
    rng = SplitMix64(SEED_BASE + 7919 * seed)
    return rng.normal_array((m, n))


def random_matrix_fast(m: int, n: int, seed: int) -> np.ndarray:
    """Seeded dense test matrix for large sizes: SplitMix64 seeds a numpy PCG64 stream."""
    rng = SplitMix64(SEED_BASE + 104729 * seed)
    g = np.random.Generator(np.random.PCG64(rng.next_u64()))
    return g.standard_normal((m, n))


def batch(count=64, steps=20, sizes_log2=(9, 14), seed_index=0, leaf=64):
    """Batch of independent instances (served together): even index -> 1D,
    odd -> 2D; N = 2^(lo + floor((hi - lo) u)) with u ~ U[0,1) (uneven mix of
    512 .. 8192 by default); alpha ~ U[1.1, 1.9] (independently per direction
    in 2D); diffusion coefficients scaled by s = 10^U[-1, 1] per direction;
    implicit Euler with dt = 1/steps.  `leaf` is the HODLR leaf used unless the
    batch autotunes it."""
    lo, hi = sizes_log2
    out = []
    for idx in range(count):
        rng = SplitMix64(SEED_BASE + 40000 + 1000 * seed_index + idx)
        N = 1 << (lo + int((hi - lo) * rng.uniform()))
        a1 = 1.1 + 0.8 * rng.uniform()
        a2 = 1.1 + 0.8 * rng.uniform()
        s1 = 10.0 ** (2.0 * rng.uniform() - 1.0)
        s2 = 10.0 ** (2.0 * rng.uniform() - 1.0)
        lf = min(leaf, max(8, N // 2))
        if idx % 2 == 0:
            out.append(fd1d(N=N, alpha=a1, steps=steps, leaf=lf, seed_index=idx, coeff_scale=s1))
        else:
            out.append(fd2d(N=N, alpha=(a1, a2), steps=steps, leaf=lf, coeff_scale=(s1, s2)))
    return out


def sample_points(N: int, count: int, seed: int):
    """Seeded (i, j) index pairs, uniform on [0, N)^2 (SplitMix64), at which
    stored expected values of an N x N field are compared."""
    rng = SplitMix64(SEED_BASE + 300007 * seed)
    ii = np.array([int(rng.uniform() * N) for _ in range(count)], dtype=np.int64)
    jj = np.array([int(rng.uniform() * N) for _ in range(count)], dtype=np.int64)
    return ii, jj


def projection_vectors(N: int, count: int, seed: int):
    """Seeded unit vectors u_k, v_k (columns of two N x count arrays) for the
    bilinear functionals u_kᵀ X v_k of an N x N field."""
    U = random_matrix_fast(N, count, 2 * seed + 1)
    V = random_matrix_fast(N, count, 2 * seed + 2)
    return U / np.linalg.norm(U, axis=0), V / np.linalg.norm(V, axis=0)


# Named workloads (sizes of the paper-shaped configurations).
WORKLOADS = {
    "fd1d_n1024": lambda: fd1d(N=1024, alpha=1.5, steps=32, leaf=64, tol=1e-10),
    "fd2d_n256": lambda: fd2d(N=256, alpha=(1.3, 1.7), steps=50, leaf=64, tol=1e-10),
    "fd2d_n1024": lambda: fd2d(N=1024, alpha=(1.5, 1.5), steps=100, leaf=128, tol=1e-10),
    "fd2d_n2048": lambda: fd2d(N=2048, alpha=(1.5, 1.5), steps=100, leaf=128, tol=1e-10),
    "fd2d_n4096": lambda: fd2d(N=4096, alpha=(1.5, 1.5), steps=100, leaf=128, tol=1e-10),
    "fd2d_n16384": lambda: fd2d(N=16384, alpha=(1.2, 1.8), steps=20, leaf=256, tol=1e-10),
}
