"""Seeded input generators (points, weights, problem data).

Everything here is drawn from numpy's PCG64 generator with an explicit seed, so
the same call returns the same arrays on any machine.  The arrays are FP64 and
C-contiguous: points are (N, d) point-major, the parameter vector theta stacks
each layer's augmented weight (W_l b_l) of shape h_l x (h_{l-1}+1) column by
column (first index fastest), the flattening convention of Sec. 2.

Problems (closed forms of Sec. 4, App. A):
  * poisson2d_sin   -Δu = 2π² sin(πx)sin(πy) on [0,1]², u = 0 on the boundary
                    (Eq. 11; App. A.2).
  * poisson5d_cos   -Δu = π² Σ cos(πx_i), u = Σ cos(πx_i) on the boundary
                    (App. A.3 / A.5).
  * poisson100d_norm -Δu = -2d, u = ‖x‖² on the boundary (App. A.5, Eq. 13).
  * heat4d_sin      ∂_t u - κ Δ_x u = 0 with κ = 1/4 on [0,1]×[0,1]⁴, initial
                    value Π sin(πx_i), zero spatial boundary; solution
                    exp(-κ d̃ π² t) Π sin(πx_i) (App. A.6).  The network input
                    is (t, x_1..x_4), so d = 5 and coordinate 0 is time.

Sampling readings (the paper does not state them): interior points are uniform
in the unit cube; a boundary point picks one of the 2d faces uniformly, pins
that coordinate to 0 or 1 and draws the rest uniformly.  For the heat problem
the boundary set is half initial points (t = 0) and half spatial-boundary
points (App. A.6).  Weights are Xavier-uniform with zero bias.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Dict, Sequence, Tuple

import numpy as np

PI = math.pi


# ---------------------------------------------------------------------------
# Problem data
# ---------------------------------------------------------------------------
@dataclass(frozen=True)
class Problem:
    name: str
    d: int                       # network input dimension (includes t for heat)
    op: str                      # "laplace" (residual -Δu - f) or "heat" (∂_t u - κΔ_x u - f)
    kappa: float
    f: Callable[[np.ndarray], np.ndarray]
    g: Callable[[np.ndarray], np.ndarray]
    u_star: Callable[[np.ndarray], np.ndarray]


def _sin2d_f(x):
    return 2.0 * PI * PI * np.sin(PI * x[:, 0]) * np.sin(PI * x[:, 1])


def _sin2d_u(x):
    return np.sin(PI * x[:, 0]) * np.sin(PI * x[:, 1])


def _cos_u(x):
    return np.cos(PI * x).sum(axis=1)


def _cos_f(x):
    return PI * PI * np.cos(PI * x).sum(axis=1)


def _norm2_u(x):
    return (x * x).sum(axis=1)


def _norm2_f_factory(d):
    return lambda x: np.full(x.shape[0], -2.0 * d)


def _heat_u_factory(dt, kappa):
    # exp(-κ d̃ π² t) Π_i sin(π x_i), with x = (t, x_1..x_d̃)
    def u(x):
        return np.exp(-kappa * dt * PI * PI * x[:, 0]) * np.prod(np.sin(PI * x[:, 1:]), axis=1)
    return u


PROBLEMS: Dict[str, Problem] = {
    "poisson2d_sin": Problem("poisson2d_sin", 2, "laplace", 0.0, _sin2d_f,
                             lambda x: np.zeros(x.shape[0]), _sin2d_u),
    "poisson5d_cos": Problem("poisson5d_cos", 5, "laplace", 0.0, _cos_f, _cos_u, _cos_u),
    "poisson100d_norm": Problem("poisson100d_norm", 100, "laplace", 0.0,
                                _norm2_f_factory(100), _norm2_u, _norm2_u),
    "heat4d_sin": Problem("heat4d_sin", 5, "heat", 0.25,
                          lambda x: np.zeros(x.shape[0]),
                          _heat_u_factory(4, 0.25), _heat_u_factory(4, 0.25)),
}


def poisson_norm_problem(d: int) -> Problem:
    """-Δu = -2d, u = ‖x‖² for any d (the d = 100 case of App. A.5)."""
    return Problem(f"poisson{d}d_norm", d, "laplace", 0.0, _norm2_f_factory(d), _norm2_u, _norm2_u)


def poisson_cos_problem(d: int) -> Problem:
    """-Δu = π² Σ cos(πx_i), u = Σ cos(πx_i) for any d (the d = 5 case of App. A.3)."""
    return Problem(f"poisson{d}d_cos", d, "laplace", 0.0, _cos_f, _cos_u, _cos_u)


# ---------------------------------------------------------------------------
# Network shapes and weights
# ---------------------------------------------------------------------------
def layer_shapes(d: int, widths: Sequence[int]) -> Tuple[Tuple[int, int], ...]:
    """(h_l, h_{l-1}+1) of each augmented weight W̃_l = (W_l b_l)."""
    dims = [d] + list(widths)
    return tuple((dims[l], dims[l - 1] + 1) for l in range(1, len(dims)))


def param_count(d: int, widths: Sequence[int]) -> int:
    """D = Σ_l h_l (h_{l-1} + 1): weights plus biases."""
    return sum(r * c for r, c in layer_shapes(d, widths))


def xavier_theta(d: int, widths: Sequence[int], seed: int) -> np.ndarray:
    """Xavier-uniform weights (gain 1), zero biases, packed column-stacked."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for rows, cols in layer_shapes(d, widths):
        fan_in, fan_out = cols - 1, rows
        a = math.sqrt(6.0 / (fan_in + fan_out))
        w = rng.uniform(-a, a, size=(rows, cols - 1))
        wt = np.concatenate([w, np.zeros((rows, 1))], axis=1)
        parts.append(wt.reshape(-1, order="F"))
    return np.ascontiguousarray(np.concatenate(parts))


# ---------------------------------------------------------------------------
# Collocation points
# ---------------------------------------------------------------------------
def sample_interior(n: int, d: int, rng: np.random.Generator) -> np.ndarray:
    return np.ascontiguousarray(rng.uniform(0.0, 1.0, size=(n, d)))


def sample_boundary(n: int, d: int, rng: np.random.Generator, first: int = 0) -> np.ndarray:
    """Uniform on the faces x_k ∈ {0, 1} of the unit cube, k >= first."""
    x = rng.uniform(0.0, 1.0, size=(n, d))
    faces = rng.integers(first, d, size=n)
    side = rng.integers(0, 2, size=n).astype(np.float64)
    x[np.arange(n), faces] = side
    return np.ascontiguousarray(x)


def sample_heat_conditions(n: int, d: int, rng: np.random.Generator) -> np.ndarray:
    """Half initial points (t = 0), half spatial-boundary points (App. A.6)."""
    n0 = n // 2
    x0 = rng.uniform(0.0, 1.0, size=(n0, d))
    x0[:, 0] = 0.0
    xb = sample_boundary(n - n0, d, rng, first=1)
    return np.ascontiguousarray(np.concatenate([x0, xb], axis=0))


# ---------------------------------------------------------------------------
# Workloads (the shapes of the paper's experiments)
# ---------------------------------------------------------------------------
@dataclass(frozen=True)
class Workload:
    name: str
    problem: str
    widths: Tuple[int, ...]
    n_int: int
    n_bdy: int
    seed: int = 0
    lam: float = 1e-3
    beta: float = 0.0
    lr: float = 0.1
    momentum: float = 0.0
    n_eval: int = 10000
    extra: Dict[str, object] = field(default_factory=dict)

    @property
    def prob(self) -> Problem:
        return PROBLEMS[self.problem]

    @property
    def d(self) -> int:
        return self.prob.d


WORKLOADS: Dict[str, Workload] = {
    # 2d Poisson, 2->32->32->1, fixed 900/120 points, one plain FP64 step.
    "poisson2d_small": Workload("poisson2d_small", "poisson2d_sin", (32, 32, 1), 900, 120),
    # 5d Poisson, 5->64->64->48->48->1, 3000/500 points, lr 0.1, λ = 1e-3.
    "poisson5d": Workload("poisson5d", "poisson5d_cos", (64, 64, 48, 48, 1), 3000, 500),
    # 100d Poisson, 100->768->768->512->512->1, 2048/512 points resampled each step.
    "poisson100d": Workload("poisson100d", "poisson100d_norm", (768, 768, 512, 512, 1), 2048, 512),
    # (4+1)d heat, 5->128->128->64->1, 4000/1000 points.
    "heat4d": Workload("heat4d", "heat4d_sin", (128, 128, 64, 1), 4000, 1000),
}


@dataclass(frozen=True)
class BatchMember:
    """One problem of the many-PINN serving workload."""
    d: int
    widths: Tuple[int, ...]
    n_int: int
    n_bdy: int

    @property
    def prob(self) -> Problem:
        return poisson_cos_problem(self.d)


def many_pinns(count: int = 64, seed: int = 0) -> Tuple[BatchMember, ...]:
    """Independent Poisson PINNs of uneven size: d uniform in {2, 5, 10, 20, 50},
    2 or 3 hidden tanh layers (3 or 4 linear layers) with widths uniform in
    {32, 64, 128, 256, 512}, N_Ω uniform in [500, 4000] and N_∂ = N_Ω / 4."""
    rng = np.random.Generator(np.random.PCG64([seed, 64]))
    out = []
    for _ in range(count):
        d = int(rng.choice([2, 5, 10, 20, 50]))
        depth = int(rng.integers(3, 5))
        widths = tuple(int(rng.choice([32, 64, 128, 256, 512])) for _ in range(depth - 1)) + (1,)
        n_int = int(rng.integers(500, 4001))
        out.append(BatchMember(d, widths, n_int, max(1, n_int // 4)))
    return tuple(out)


def make_batch(prob: Problem, n_int: int, n_bdy: int, seed: int, step: int = 0):
    """Interior points, f, boundary points, g for one step of a seeded stream."""
    rng = np.random.Generator(np.random.PCG64([seed, step]))
    x_int = sample_interior(n_int, prob.d, rng)
    if prob.op == "heat":
        x_bdy = sample_heat_conditions(n_bdy, prob.d, rng)
    else:
        x_bdy = sample_boundary(n_bdy, prob.d, rng)
    f = np.ascontiguousarray(prob.f(x_int), dtype=np.float64)
    g = np.ascontiguousarray(prob.g(x_bdy), dtype=np.float64)
    return x_int, f, x_bdy, g


def eval_points(prob: Problem, n: int, seed: int) -> np.ndarray:
    """Held-out points for the relative L2 error (uniform in the cube)."""
    rng = np.random.Generator(np.random.PCG64([seed, 1 << 30]))
    return sample_interior(n, prob.d, rng)
