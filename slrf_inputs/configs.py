"""Named synthetic workloads and the seeded start block.

Every workload is a shape-and-seed recipe; nothing here is computed by the eigensolver.

* ``bar1d_2000``      1D linear-FEM bar, n = 2000, Dirichlet; gamma = 4150.528 lies midway
                      between the 20th and 21st eigenvalue; block 32, m = 8 poles.
* ``q1_lap_41``       3D Q1 Laplacian on 41^3 nodes (40^3 elements, h = 1/40), Neumann,
                      A = K + 1e-3 B; gamma = 259.0666 lies midway between the 6-fold
                      cluster at 258.33 (eigenvalues 100..105) and the next value 259.80,
                      so the interval holds 105 eigenvalues; block 160, m = 8.
* ``q1_elast_64``     3D Q1 elasticity on 64x64x32 nodes, z = 0 clamped (n = 380,928),
                      E_e ~ lognormal(0, 0.5), nu = 0.3, rho = 1; block 480, m = 8.
* small variants (``bar1d``, ``q1_lap``, ``q1_elast``) with any size for tests.

The start block is a standard Gaussian drawn with numpy's PCG64 generator
``default_rng(seed)`` and laid out row-major n x L (L contiguous), the layout the
solver library takes.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import fem


@dataclass
class Workload:
    name: str
    pencil: fem.CsrPair
    gamma: float
    block: int  # L
    m: int  # upper-half-plane poles
    seed: int
    it_max: int
    n_expected: int | None = None  # eigenvalue count in (0, gamma] when known by construction
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.pencil.n


def start_block(n: int, L: int, seed: int) -> np.ndarray:
    """Gaussian start block V1, float64, C-contiguous (n, L)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal((n, L)))


def bar1d(n: int = 2000, gamma: float | None = None, block: int = 32, m: int = 8, seed: int = 1,
          it_max: int = 200) -> Workload:
    p = fem.bar1d(n)
    if gamma is None:
        if n != 2000:
            raise ValueError("give gamma for n != 2000")
        gamma = 4150.528
    return Workload(f"bar1d_{n}", p, gamma, block, m, seed, it_max, 20 if n == 2000 else None)


def q1_lap_interval(nodes: int, want: int, shift: float = 1e-3):
    """gamma for the Q1 Neumann Laplacian on nodes^3 nodes (unit cube): the midpoint of the
    spectral gap nearest to `want` eigenvalues, from the tensor-product spectrum
    lambda_abc = mu_a + mu_b + mu_c + shift with the 1D FEM values
    mu_k = 6 (1 - cos(k pi/(nodes-1))) / (h^2 (2 + cos(k pi/(nodes-1)))), h = 1/(nodes-1).
    Returns (gamma, count)."""
    h = 1.0 / (nodes - 1)
    c = np.cos(np.arange(nodes) * np.pi / (nodes - 1))
    mu = 6.0 * (1.0 - c) / (h * h * (2.0 + c))
    lam = np.sort((mu[:, None, None] + mu[None, :, None] + mu[None, None, :]).ravel()) + shift
    gaps = np.nonzero(np.diff(lam) > 1e-6 * lam[1:])[0]
    g = gaps[np.argmin(np.abs(gaps + 1 - want))]
    return 0.5 * (lam[g] + lam[g + 1]), int(g + 1)


def q1_lap(nodes: int = 41, gamma: float | None = None, block: int | None = None, m: int = 8, seed: int = 2,
           it_max: int = 40) -> Workload:
    p = fem.q1_scalar((nodes, nodes, nodes), shift=1e-3)
    count = None
    if gamma is None:
        if nodes == 41:
            gamma, count = 259.0666, 105
        else:
            gamma, count = q1_lap_interval(nodes, 100)
    if block is None:
        block = 160 if nodes == 41 else int(np.ceil(1.5 * (count or 100)))
    return Workload(f"q1_lap_{nodes}", p, gamma, block, m, seed, it_max, count)


def q1_elast(nodes=(64, 64, 32), gamma: float | None = None, block: int = 480, m: int = 8, seed: int = 3,
             it_max: int = 80, e_sigma: float = 0.5) -> Workload:
    nodes = tuple(nodes)
    ne = int(np.prod([s - 1 for s in nodes]))
    E = np.exp(np.random.default_rng(seed).normal(0.0, e_sigma, ne))
    p = fem.q1_elasticity(nodes, E=E, nu=0.3, rho=1.0, clamp_face=(2, 0))
    if gamma is None:
        raise ValueError("give gamma")
    return Workload("q1_elast_" + "x".join(map(str, nodes)), p, gamma, block, m, seed, it_max)
