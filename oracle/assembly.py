"""Oracle: subdomain geometry, window functions and collocation assembly.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline use this package; the product path never does.

Follows the paper step by step, in float64, with no blocking or fusion:
  * Sec. 5 Example 1: overlapping box subdomains Omega_j with centre mu_j and
    half-width sigma_j per dimension; window functions
    omega_hat_j = prod_i [1 + cos(pi (x_i - mu_i)/sigma_i)]^2 inside the box,
    zero outside, normalised omega_j = omega_hat_j / sum_k omega_hat_k
    (Sec. 2, partition of unity sum_j omega_j = 1).
  * Sec. 2 Eq. (net): Phi_j(x) = tanh(R_j x_hat + b_j) with inputs normalised
    to [-1, 1]^d per subdomain, x_hat = (x - mu_j) / sigma_j (Sec. 5).
  * Sec. 1 Eq. (operator): constraining operator C u = L u + G, with
    L = prod_i tanh(x_i/rho) tanh((1-x_i)/rho) (Eq. (cons1); times tanh(t/rho)
    for space-time problems, Eq. (cons2)).
  * Sec. 2 Eq. (sum)/(system): (H_j)_{ik} = A[L omega_j phi_j^k](x_i) and
    F_i = f(x_i) - A[G](x_i); Sec. 4: (Psi_j)_{ik} = omega_j phi_j^k(x_i).
Derivatives come from hyper-dual numbers applied to the whole product.

Layout readings (where the paper is silent or garbled):
  * cell layout: mu_k = (k + 1/2)/l, sigma = (1/l + overlap)/2 per dim;
    paper layout (Example 1): mu_k = k/(l-1), sigma = (delta/2)/(l-1).
  * collocation points: the cell-centred grid x_q = (q + 1/2)/(l n) per dim.
  * rows of block j: the grid points strictly inside box_j, dim 0 fastest.
"""
from __future__ import annotations

import numpy as np

import rann_inputs as ri
from . import hyperdual as hd


# ----------------------------------------------------------------- geometry --

def centres_halfwidths(p: ri.Problem):
    """Per-dim subdomain centres mu[i] (array over k) and half-widths sigma[i]."""
    mu, sig = [], []
    for i in range(p.dim):
        l = p.sub[i]
        if p.layout == ri.LAYOUT_PAPER:
            if l == 1:
                raise ValueError("paper layout needs at least 2 subdomains per dim")
            mu.append(np.arange(l) / (l - 1.0))
            sig.append(0.5 * p.delta / (l - 1.0))
        else:
            mu.append((np.arange(l) + 0.5) / l)
            sig.append(0.5 * (1.0 / l + p.overlap[i]))
    return mu, sig


def subdomain_multi_index(p: ri.Problem, j: int):
    """Subdomain j -> (k_0, k_1[, k_2]) with k_0 fastest."""
    ks = []
    for i in range(p.dim):
        ks.append(j % p.sub[i])
        j //= p.sub[i]
    return ks


def box_rows(p: ri.Problem, j: int) -> np.ndarray:
    """Global indices of the collocation points strictly inside box_j (dim 0 fastest)."""
    mu, sig = centres_halfwidths(p)
    ks = subdomain_multi_index(p, j)
    shp = p.grid_shape()
    ranges = []
    for i in range(p.dim):
        q = np.arange(shp[i])
        x = (q + 0.5) / shp[i]
        ranges.append(q[np.abs(x - mu[i][ks[i]]) < sig[i]])
    strides = np.cumprod([1] + list(shp[:-1]))
    # meshgrid over (last dim, ..., dim 0) in "ij" order makes dim 0 vary fastest
    grids = np.meshgrid(*[ranges[i] for i in reversed(range(p.dim))], indexing="ij")
    idx = sum(g.reshape(-1) * strides[p.dim - 1 - a] for a, g in enumerate(grids))
    return np.asarray(idx, dtype=np.int64)


def neighbours(p: ri.Problem, j: int) -> list:
    """Subdomains whose box shares at least one collocation point with box_j."""
    rows_j = set(box_rows(p, j).tolist())
    return [k for k in range(p.J) if rows_j.intersection(box_rows(p, k).tolist())]


# ---------------------------------------------------------- hyper-dual fields --

def _coords(X: np.ndarray, direction: int):
    return [hd.HD.var(X[:, i], seed=(i == direction)) for i in range(X.shape[1])]


def window_hat(p: ri.Problem, xs, k: int):
    """omega_hat_k at the points (hyper-dual), zero outside the open box."""
    mu, sig = centres_halfwidths(p)
    ks = subdomain_multi_index(p, k)
    val = hd.HD.const(np.ones_like(xs[0].a))
    inside = np.ones_like(xs[0].a, dtype=bool)
    for i in range(p.dim):
        u = (xs[i] - mu[i][ks[i]]) * (1.0 / sig[i])
        inside &= np.abs(u.a) < 1.0
        h = 1.0 + hd.cos(np.pi * u)
        val = val * (h * h)
    zero = hd.HD.const(np.zeros_like(xs[0].a))
    return hd.where(inside, val, zero)


def window(p: ri.Problem, xs, j: int):
    """omega_j = omega_hat_j / sum_k omega_hat_k (hyper-dual)."""
    total = None
    for k in range(p.J):
        w = window_hat(p, xs, k)
        total = w if total is None else total + w
    return window_hat(p, xs, j) / total


def constraint_L(p: ri.Problem, xs):
    rho = p.rho
    val = hd.HD.const(np.ones_like(xs[0].a))
    for i in range(p.spatial_dims):
        val = val * hd.tanh(xs[i] * (1.0 / rho)) * hd.tanh((1.0 - xs[i]) * (1.0 / rho))
    if p.op == ri.OP_HEAT:
        val = val * hd.tanh(xs[p.dim - 1] * (1.0 / rho))
    return val


def constraint_G(p: ri.Problem, xs):
    if p.g_kind == ri.G_ZERO:
        return hd.HD.const(np.zeros_like(xs[0].a))
    val = hd.HD.const(np.ones_like(xs[0].a))
    for i in range(p.spatial_dims):
        val = val * hd.sin(np.pi * xs[i])
    return val


def _smooth_box(x, i: int, g: int):
    """Smooth indicator of [i/g, (i+1)/g]: 1/2[tanh((x-i/g)/w) - tanh((x-(i+1)/g)/w)],
    w = 1/(8g); the outermost cells extend to +-infinity so the g indicators sum to 1."""
    w = 1.0 / (8.0 * g)
    left = hd.tanh((x - i / g) * (1.0 / w)) if i > 0 else hd.HD.const(np.ones_like(x.a))
    right = hd.tanh((x - (i + 1) / g) * (1.0 / w)) if i < g - 1 else -hd.HD.const(np.ones_like(x.a))
    return 0.5 * (left - right)


def coefficient(p: ri.Problem, xs):
    """Diffusion coefficient a(x) (hyper-dual)."""
    if p.coef == ri.COEF_CONST:
        return hd.HD.const(np.full_like(xs[0].a, p.coef_value))
    if p.coef == ri.COEF_MULTISCALE:
        e = p.eps
        return 2.0 + hd.sin(2.0 * np.pi / e * xs[0]) * hd.sin(2.0 * np.pi / e * xs[1])
    if p.coef == ri.COEF_PIECEWISE:
        g = p.coef_grid
        total = hd.HD.const(np.zeros_like(xs[0].a))
        sx = [_smooth_box(xs[0], c, g) for c in range(g)]
        sy = [_smooth_box(xs[1], c, g) for c in range(g)]
        for cy in range(g):
            for cx in range(g):
                total = total + float(p.coef_vals[cy * g + cx]) * (sx[cx] * sy[cy])
        return total
    raise ValueError(p.coef)


def source_f(p: ri.Problem, X: np.ndarray) -> np.ndarray:
    f = np.full(X.shape[0], p.f0, dtype=np.float64)
    if p.fc is not None:
        for c, a in zip(p.fc, p.fa):
            term = np.full(X.shape[0], float(c))
            for i in range(p.spatial_dims):
                term = term * np.sin(np.pi * a[i] * X[:, i])
            f = f + term
    return f


def apply_operator(p: ri.Problem, X: np.ndarray, field) -> np.ndarray:
    """A[v] at the points, where field(xs) builds v as a hyper-dual expression.

    Poisson: -Lap v + c0 v.  Diffusion: -div(a grad v) = -a Lap v - grad a . grad v.
    Heat (last coordinate t): v_t - nu Lap_x v."""
    d = p.dim
    ns = p.spatial_dims
    first, second, value = [], [], None
    acoef = []
    for i in range(d):
        xs = _coords(X, i)
        v = field(xs)
        value = v.a
        first.append(v.b)
        second.append(v.d)
        if p.op == ri.OP_DIFFUSION:
            a = coefficient(p, xs)
            acoef.append(a)
    lap = sum(second[i] for i in range(ns))
    if p.op == ri.OP_POISSON:
        return -lap + p.c0 * value
    if p.op == ri.OP_DIFFUSION:
        a0 = acoef[0].a
        a0 = a0[:, None] if value.ndim == 2 else a0
        out = -a0 * lap
        for i in range(ns):
            gi = acoef[i].b
            gi = gi[:, None] if value.ndim == 2 else gi
            out = out - gi * first[i]
        return out
    if p.op == ri.OP_HEAT:
        return first[d - 1] - p.nu * lap
    raise ValueError(p.op)


# ------------------------------------------------------------------ assembly --

def block(p: ri.Problem, R: np.ndarray, b: np.ndarray, j: int):
    """Rows, Psi_j and H_j of subdomain j (Sec. 2 Eq. (system), Sec. 4)."""
    rows = box_rows(p, j)
    X = ri.grid_points(p)[rows]
    mu, sig = centres_halfwidths(p)
    ks = subdomain_multi_index(p, j)
    Rj, bj = R[j], b[j]

    def features(xs):
        z = hd.HD.const(np.broadcast_to(bj[None, :], (X.shape[0], bj.shape[0])).copy())
        for i in range(p.dim):
            xh = (xs[i] - mu[i][ks[i]]) * (1.0 / sig[i])
            xh2 = hd.HD(xh.a[:, None], xh.b[:, None], xh.c[:, None], xh.d[:, None])
            z = z + xh2 * Rj[None, :, i]
        return hd.tanh(z)

    def basis(xs):
        w = window(p, xs, j)
        lw = constraint_L(p, xs) * w
        lw2 = hd.HD(lw.a[:, None], lw.b[:, None], lw.c[:, None], lw.d[:, None])
        return lw2 * features(xs)

    xs0 = _coords(X, -1)
    w0 = window(p, xs0, j).a
    phi0 = features(xs0).a
    Psi = w0[:, None] * phi0
    H = apply_operator(p, X, basis)
    return rows, Psi, H


def rhs(p: ri.Problem, X: np.ndarray = None) -> np.ndarray:
    """F_i = f(x_i) - A[G](x_i) on the global grid (Sec. 2 Eq. (system))."""
    if X is None:
        X = ri.grid_points(p)
    AG = apply_operator(p, X, lambda xs: constraint_G(p, xs))
    return source_f(p, X) - AG


def assemble(p: ri.Problem, R: np.ndarray, b: np.ndarray):
    """All blocks: list of (rows_j, Psi_j, H_j), and F."""
    blocks = [block(p, R, b, j) for j in range(p.J)]
    return blocks, rhs(p)
