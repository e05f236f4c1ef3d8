"""Seeded synthetic inputs for the RaNN domain-decomposition solver.

This module is shared by the CPU oracle, the tests and the benchmark. It holds
the *problem data* only -- PDE operator choice, coefficients, sources, the
manufactured exact solutions, subdomain-grid parameters and the fixed random
hidden-layer weights -- and none of the method's arithmetic (no window
functions, no features, no PCA, no Schwarz, no Krylov).

Random numbers: the hidden weights R_j and biases b_j of every subdomain
network are drawn uniformly (Sec. 5, Example 1: U(-1,1); Sec. 2, Eq. (net)),
here from SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used as a counter-based generator: draw i of stream
`seed` is mix64(seed + (i + 1) * 0x9E3779B97F4A7C15).  Order of draws: for each
subdomain j, the m*d entries of R_j in (neuron, dim) order, then its m biases.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
BASE_SEED = 2412192070


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Draws start..start+n-1 of the SplitMix64 stream `seed` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float, hi: float, start: int = 0) -> np.ndarray:
    """U[lo, hi) doubles: 53 high bits of each draw scaled to [0, 1)."""
    u = (splitmix64(seed, n, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


# Operator / coefficient / source kinds (integer codes match include/rann_dd.h).
OP_POISSON, OP_DIFFUSION, OP_HEAT = 0, 1, 2
COEF_CONST, COEF_MULTISCALE, COEF_PIECEWISE = 0, 1, 2
G_ZERO, G_SINPROD = 0, 1
LAYOUT_CELL, LAYOUT_PAPER = 0, 1
PCA_ABS, PCA_VARIANCE, PCA_NONE = 0, 1, 2


@dataclasses.dataclass
class Problem:
    """One RaNN-DD problem: the PDE of Eq. (1), the subdomain grid, the local
    networks and the solver settings.  Field names follow the C descriptor."""
    name: str
    dim: int                       # 2 or 3 (space-time problems count t)
    op: int                        # OP_*
    sub: Tuple[int, ...]           # subdomains per dim (l_i)
    pts: Tuple[int, ...]           # collocation points per subdomain cell per dim
    neurons: int                   # m
    w_range: float                 # R, b ~ U[-w_range, w_range]
    seed: int
    overlap: Tuple[float, ...] = (0.0, 0.0, 0.0)   # cell layout: absolute overlap per dim
    delta: float = 2.0             # paper layout: overlap ratio delta
    layout: int = LAYOUT_CELL
    c0: float = 0.0                # Poisson reaction term: -Lap u + c0 u
    nu: float = 1.0                # heat diffusivity: u_t - nu Lap_x u
    coef: int = COEF_CONST
    coef_value: float = 1.0        # COEF_CONST value of a
    eps: float = 1.0 / 16.0        # COEF_MULTISCALE period
    coef_grid: int = 0             # COEF_PIECEWISE g (g x g cells)
    coef_vals: Optional[np.ndarray] = None   # COEF_PIECEWISE values, [g*g] row-major (y major)
    rho: float = 0.5               # L = prod tanh(x_i/rho) tanh((1-x_i)/rho) [* tanh(t/rho)]
    g_kind: int = G_ZERO           # G = 0 or prod_{spatial} sin(pi x_i)
    f0: float = 0.0                # f = f0 + sum_k fc[k] prod_i sin(pi fa[k,i] x_i)
    fc: Optional[np.ndarray] = None
    fa: Optional[np.ndarray] = None  # [nterms, dim] integer frequencies (spatial dims)
    pca_mode: int = PCA_VARIANCE
    pca_thr: float = 1e-12
    solver: str = "cg_as"          # "cg_as" | "gmres_ras"
    precond: str = "as"            # "as" | "sas" | "ras" | "none"
    restart: int = 50
    rtol: float = 1e-10
    maxit: int = 2000
    exact: Optional[str] = None    # name of a manufactured exact solution

    @property
    def J(self) -> int:
        return int(np.prod(self.sub[: self.dim]))

    @property
    def spatial_dims(self) -> int:
        return self.dim - 1 if self.op == OP_HEAT else self.dim

    def grid_shape(self) -> Tuple[int, ...]:
        return tuple(int(self.sub[i] * self.pts[i]) for i in range(self.dim))

    def n_points(self) -> int:
        return int(np.prod(self.grid_shape()))


def weights(p: Problem) -> Tuple[np.ndarray, np.ndarray]:
    """Hidden weights R [J, m, dim] and biases b [J, m], U[-r, r] (Sec. 2 Eq. (net))."""
    J, m, d = p.J, p.neurons, p.dim
    per = m * d + m
    u = uniform(p.seed, J * per, -p.w_range, p.w_range)
    u = u.reshape(J, per)
    R = u[:, : m * d].reshape(J, m, d).copy()
    b = u[:, m * d:].copy()
    return R, b


def grid_points(p: Problem) -> np.ndarray:
    """Cell-centred global collocation grid, [N, dim], dim 0 fastest."""
    shp = p.grid_shape()
    axes = [(np.arange(n) + 0.5) / n for n in shp]
    mesh = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
    return np.stack([m.reshape(-1) for m in mesh], axis=1)


def test_points(p: Problem, per_dim: int) -> np.ndarray:
    """Uniformly spaced test points including the boundary, [M, dim]."""
    ax = np.linspace(0.0, 1.0, per_dim)
    mesh = np.meshgrid(*([ax] * p.dim), indexing="ij")[::-1]
    return np.stack([m.reshape(-1) for m in mesh], axis=1)


def boundary_points(p: Problem, per_edge: int) -> np.ndarray:
    """Points on the Dirichlet boundary (and on t=0 for space-time problems)."""
    rng = np.linspace(0.0, 1.0, per_edge)
    out = []
    ns = p.spatial_dims
    for i in range(ns):
        for side in (0.0, 1.0):
            mesh = np.meshgrid(*([rng] * p.dim), indexing="ij")
            pts = np.stack([m.reshape(-1) for m in mesh], axis=1)
            pts[:, i] = side
            out.append(pts)
    if p.op == OP_HEAT:
        mesh = np.meshgrid(*([rng] * p.dim), indexing="ij")
        pts = np.stack([m.reshape(-1) for m in mesh], axis=1)
        pts[:, p.dim - 1] = 0.0
        out.append(pts)
    return np.unique(np.concatenate(out, axis=0), axis=0)


def exact_solution(p: Problem, x: np.ndarray) -> Optional[np.ndarray]:
    """Manufactured exact solutions of the configured problems (closed forms)."""
    if p.exact is None:
        return None
    if p.exact == "sinprod":
        return np.prod(np.sin(np.pi * x[:, : p.spatial_dims]), axis=1)
    if p.exact == "heat":
        t = x[:, p.dim - 1]
        return np.exp(-2.0 * p.nu * np.pi ** 2 * t) * np.prod(np.sin(np.pi * x[:, :2]), axis=1)
    if p.exact == "multiscale_sin":
        # Example 1: u = (1/n) sum_{i=1}^n sin(2^i pi x) sin(2^i pi y), n = len(fc)
        n = len(p.fc)
        return sum(np.sin(2 ** i * np.pi * x[:, 0]) * np.sin(2 ** i * np.pi * x[:, 1])
                   for i in range(1, n + 1)) / n
    raise ValueError(p.exact)


def fourier_source(seed: int, nmodes: int = 8, maxfreq: int = 4) -> Tuple[np.ndarray, np.ndarray]:
    """Random Fourier source f = sum_k c_k sin(pi a_k x) sin(pi b_k y):
    (a_k, b_k) uniform on {1..maxfreq}^2 and c_k ~ N(0,1) (Box-Muller on
    SplitMix64 draws)."""
    u = uniform(seed, 4 * nmodes, 0.0, 1.0)
    freqs = 1 + np.floor(u[: 2 * nmodes] * maxfreq).astype(np.int64)
    u1 = np.maximum(u[2 * nmodes: 3 * nmodes], 2.0 ** -53)
    u2 = u[3 * nmodes:]
    c = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return c, freqs.reshape(nmodes, 2).astype(np.float64)


def piecewise_coef(seed: int, g: int = 4, lo: float = 0.5, hi: float = 2.0) -> np.ndarray:
    return uniform(seed, g * g, lo, hi)


# --------------------------------------------------------------------------
# The configured workloads.  Sizes follow the problem statements; "small"
# variants keep the dimension, operator and overlap but shrink the grid and the
# network so that the CPU oracle finishes in seconds.
# --------------------------------------------------------------------------

def _sin_term(dim_sp: int, coef: float) -> Tuple[np.ndarray, np.ndarray]:
    return np.array([coef]), np.ones((1, dim_sp))


def poisson2d_2x2(neurons=100, pts=20, seed=BASE_SEED + 1) -> Problem:
    """2D Poisson -Lap u = f, u = sin(pi x) sin(pi y), 2x2 subdomains, overlap 0.1."""
    fc, fa = _sin_term(2, 2.0 * np.pi ** 2)
    return Problem(name="poisson2d_2x2", dim=2, op=OP_POISSON, sub=(2, 2), pts=(pts, pts),
                   neurons=neurons, w_range=1.0, seed=seed, overlap=(0.1, 0.1),
                   rho=0.5, fc=fc, fa=fa, pca_mode=PCA_VARIANCE, pca_thr=1e-12,
                   solver="cg_as", precond="as", exact="sinprod")


def multiscale2d(sub=8, pts=40, neurons=300, seed=BASE_SEED + 2) -> Problem:
    """2D multiscale diffusion -div(a grad u) = 1, a = 2 + sin(2 pi x/eps) sin(2 pi y/eps)."""
    ov = 0.05 if sub == 8 else 0.4 / sub
    return Problem(name=f"multiscale2d_{sub}x{sub}", dim=2, op=OP_DIFFUSION, sub=(sub, sub),
                   pts=(pts, pts), neurons=neurons, w_range=2.0, seed=seed,
                   overlap=(ov, ov), coef=COEF_MULTISCALE, eps=1.0 / 16.0, rho=0.5,
                   f0=1.0, pca_mode=PCA_VARIANCE, pca_thr=1e-12,
                   solver="gmres_ras", precond="ras", restart=50)


def heat3d(sub=(8, 8, 4), pts=(16, 16, 8), neurons=400, seed=BASE_SEED + 3) -> Problem:
    """Space-time heat u_t = 0.1 Lap u, u(0) = sin(pi x) sin(pi y), exact solution known."""
    ov = tuple(0.4 / s for s in sub)
    return Problem(name="heat3d", dim=3, op=OP_HEAT, sub=tuple(sub), pts=tuple(pts),
                   neurons=neurons, w_range=1.0, seed=seed, overlap=ov, nu=0.1,
                   rho=1.0, g_kind=G_SINPROD, f0=0.0, pca_mode=PCA_VARIANCE,
                   pca_thr=1e-12, solver="gmres_ras", precond="ras", exact="heat")


def poisson3d(sub=4, pts=12, neurons=400, seed=BASE_SEED + 4) -> Problem:
    """3D Poisson -Lap u = 3 pi^2 u, u = sin sin sin, 4^3 subdomains, overlap 0.1."""
    fc, fa = _sin_term(3, 3.0 * np.pi ** 2)
    return Problem(name="poisson3d", dim=3, op=OP_POISSON, sub=(sub,) * 3, pts=(pts,) * 3,
                   neurons=neurons, w_range=1.0, seed=seed, overlap=(0.1,) * 3, rho=1.0,
                   fc=fc, fa=fa, pca_mode=PCA_VARIANCE, pca_thr=1e-12,
                   solver="cg_as", precond="as", exact="sinprod")


def piecewise2d(instance: int = 0, sub=None, pts=24, neurons=200) -> Problem:
    """Diffusion with a smoothed piecewise-constant 4x4 coefficient and a random
    8-mode Fourier source; instance i uses l = {4,6,...,16}[i mod 7]."""
    seed = BASE_SEED + 5 + 1000 * instance
    l = sub if sub is not None else (4, 6, 8, 10, 12, 14, 16)[instance % 7]
    fc, fa = fourier_source(seed ^ 0x5EED)
    vals = piecewise_coef(seed ^ 0xC0EF)
    return Problem(name=f"piecewise2d_{instance}", dim=2, op=OP_DIFFUSION, sub=(l, l),
                   pts=(pts, pts), neurons=neurons, w_range=1.0, seed=seed,
                   overlap=(0.4 / l, 0.4 / l), coef=COEF_PIECEWISE, coef_grid=4,
                   coef_vals=vals, rho=0.5, fc=fc, fa=fa, pca_mode=PCA_VARIANCE,
                   pca_thr=1e-12, solver="gmres_ras", precond="ras", restart=50)


def example1_paper(n: int = 2, sub: int = 4, pts: int = 10, neurons: int = 16,
                   delta: float = 2.0, seed: int = BASE_SEED + 10) -> Problem:
    """Example 1 of the paper: multi-scale Laplacian, node-centred subdomains
    with overlap ratio delta, rho = (1/2)^n.  f uses omega_i^2 (the derivative
    of the stated u; the printed f drops the square)."""
    fc = np.array([2.0 / n * (2 ** i) ** 2 * np.pi ** 2 for i in range(1, n + 1)])
    fa = np.array([[2.0 ** i, 2.0 ** i] for i in range(1, n + 1)])
    return Problem(name=f"example1_n{n}", dim=2, op=OP_POISSON, sub=(sub, sub),
                   pts=(pts, pts), neurons=neurons, w_range=1.0, seed=seed,
                   layout=LAYOUT_PAPER, delta=delta, rho=0.5 ** n, fc=fc, fa=fa,
                   pca_mode=PCA_ABS, pca_thr=1e-3, solver="gmres_ras", precond="as",
                   exact="multiscale_sin")


CONFIG_NAMES = ["poisson2d_2x2", "multiscale2d", "heat3d", "poisson3d", "piecewise2d"]


def config(name: str, small: bool = False) -> Problem:
    """Full-size configured workloads, or their small (oracle-sized) variants."""
    if name == "poisson2d_2x2":
        return poisson2d_2x2(neurons=40, pts=10) if small else poisson2d_2x2()
    if name == "multiscale2d":
        return multiscale2d(sub=4, pts=10, neurons=40) if small else multiscale2d()
    if name == "heat3d":
        return heat3d(sub=(2, 2, 2), pts=(6, 6, 4), neurons=40) if small else heat3d()
    if name == "poisson3d":
        return poisson3d(sub=2, pts=6, neurons=40) if small else poisson3d()
    if name == "piecewise2d":
        return piecewise2d(0, sub=4, pts=8, neurons=30) if small else piecewise2d(0)
    if name == "example1":
        return example1_paper()
    raise KeyError(name)
