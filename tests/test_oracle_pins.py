"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: a
published value, a closed form, an invariant, a special case that reduces to
exact arithmetic, or brute force.  The planted-mistake tests at the end show
that a plausible slip in the oracle trips at least one of these pins.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import rann_inputs as ri
from oracle import assembly as asm
from oracle import hyperdual as hd
from oracle import linalg as la
from oracle import solver as sv

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_pins.json")))
BANDS = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_bands.json")))
SMALL = ["poisson2d_2x2", "multiscale2d", "heat3d", "poisson3d", "piecewise2d"]


# ------------------------------------------------------------------ inputs --

def test_splitmix64_published_vector():
    got = ["%016x" % int(v) for v in ri.splitmix64(0, 4)]
    assert got == GOLDEN["splitmix64_seed0"]["value"]


def test_weights_range_and_order():
    p = ri.config("poisson2d_2x2", small=True)
    R, b = ri.weights(p)
    assert R.shape == (p.J, p.neurons, p.dim) and b.shape == (p.J, p.neurons)
    assert np.all(np.abs(R) <= p.w_range) and np.all(np.abs(b) <= p.w_range)
    # draw order: subdomain j, then R_j in (neuron, dim) order, then b_j
    u = ri.uniform(p.seed, p.neurons * p.dim + p.neurons, -1.0, 1.0)
    np.testing.assert_array_equal(R[0].reshape(-1), u[: p.neurons * p.dim])
    np.testing.assert_array_equal(b[0], u[p.neurons * p.dim:])


# ------------------------------------------------------------- hyper-dual --

def test_hyperdual_against_closed_form_derivatives():
    x = np.linspace(-1.3, 1.7, 41)
    X = hd.HD.var(x, seed=True)
    f = hd.tanh(3.0 * X) * hd.sin(X) / (2.0 + X * X)
    t, s, c = np.tanh(3 * x), np.sin(x), np.cos(x)
    q = 2.0 + x * x
    # f = T S / Q with T = tanh(3x), S = sin x, Q = 2 + x^2
    T1, T2 = 3 * (1 - t * t), -18 * t * (1 - t * t)
    S1, S2 = c, -s
    Q1, Q2 = 2 * x, 2.0 + 0 * x
    N, N1 = t * s, T1 * s + t * S1
    N2 = T2 * s + 2 * T1 * S1 + t * S2
    f0 = N / q
    f1 = (N1 * q - N * Q1) / q ** 2
    f2 = (N2 * q - N * Q2) / q ** 2 - 2 * Q1 * (N1 * q - N * Q1) / q ** 3
    np.testing.assert_allclose(f.a, f0, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(f.b, f1, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(f.c, f1, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(f.d, f2, rtol=1e-12, atol=1e-13)


def test_hyperdual_exp_cos():
    x = np.linspace(-2, 2, 17)
    f = hd.exp(hd.cos(hd.HD.var(x, True)))
    e = np.exp(np.cos(x))
    np.testing.assert_allclose(f.b, -np.sin(x) * e, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(f.d, (np.sin(x) ** 2 - np.cos(x)) * e, rtol=1e-13, atol=1e-15)


# ------------------------------------------------------------- geometry --

@pytest.mark.parametrize("name", SMALL + ["example1"])
def test_partition_of_unity(name):
    """Sec. 2: the normalised windows sum to one everywhere on Omega."""
    p = ri.config(name, small=True)
    rng = np.random.default_rng(7)
    X = rng.random((500, p.dim))
    X[:20] = np.round(X[:20])          # corners and faces of the cube
    xs = asm._coords(X, 0)
    ws = [asm.window(p, xs, j) for j in range(p.J)]
    total = sum(w.a for w in ws)
    np.testing.assert_allclose(total, GOLDEN["pou_sum"]["value"], rtol=0, atol=4e-16)
    # derivatives of the sum vanish as well
    np.testing.assert_allclose(sum(w.b for w in ws), 0.0, atol=1e-11)
    np.testing.assert_allclose(sum(w.d for w in ws), 0.0, atol=1e-9)
    assert all(np.all(w.a >= 0) for w in ws)


def test_window_support_is_the_box():
    p = ri.config("multiscale2d", small=True)
    mu, sig = asm.centres_halfwidths(p)
    X = np.random.default_rng(1).random((2000, 2))
    xs = asm._coords(X, -1)
    for j in (0, 5, 15):
        ks = asm.subdomain_multi_index(p, j)
        inside = np.all([np.abs(X[:, i] - mu[i][ks[i]]) < sig[i] for i in range(2)], axis=0)
        w = asm.window(p, xs, j).a
        assert np.all(w[~inside] == 0.0) and np.all(w[inside] > 0.0)


def test_box_rows_match_brute_force():
    for name in SMALL + ["example1"]:
        p = ri.config(name, small=True)
        X = ri.grid_points(p)
        mu, sig = asm.centres_halfwidths(p)
        for j in range(p.J):
            ks = asm.subdomain_multi_index(p, j)
            inside = np.all([np.abs(X[:, i] - mu[i][ks[i]]) < sig[i] for i in range(p.dim)], axis=0)
            np.testing.assert_array_equal(asm.box_rows(p, j), np.nonzero(inside)[0])


def test_overlap_ratio_reading():
    """Cell layout: delta = 1 + overlap * l (config 2: overlap 0.05, l = 8 -> 1.4)."""
    p = ri.multiscale2d()
    _, sig = asm.centres_halfwidths(p)
    assert abs(2 * sig[0] * p.sub[0] - 1.4) < 1e-14


# ----------------------------------------------------- operator and RHS --

def _field(fn):
    return lambda xs: fn(xs)


@pytest.mark.parametrize("name", ["poisson2d_2x2", "poisson3d", "heat3d"])
def test_operator_on_manufactured_solution(name):
    """A[u_exact] = f for the manufactured solutions (closed forms)."""
    p = ri.config(name, small=True)
    X = np.random.default_rng(3).random((300, p.dim))

    def u(xs):
        v = hd.HD.const(np.ones_like(xs[0].a))
        for i in range(p.spatial_dims):
            v = v * hd.sin(np.pi * xs[i])
        if p.op == ri.OP_HEAT:
            v = v * hd.exp(-2.0 * p.nu * np.pi ** 2 * xs[p.dim - 1])
        return v
    Au = asm.apply_operator(p, X, u)
    np.testing.assert_allclose(Au, asm.source_f(p, X), rtol=1e-12, atol=1e-11)


def test_diffusion_operator_closed_form():
    """-div(a grad u) for u = x^2 y and the multiscale a (Sec. 5 config 2)."""
    p = ri.config("multiscale2d", small=True)
    X = np.random.default_rng(4).random((200, 2))
    x, y = X[:, 0], X[:, 1]
    k = 2 * np.pi / p.eps
    a = 2 + np.sin(k * x) * np.sin(k * y)
    ax = k * np.cos(k * x) * np.sin(k * y)
    ay = k * np.sin(k * x) * np.cos(k * y)
    expect = -(ax * 2 * x * y + ay * x * x + a * 2 * y)
    got = asm.apply_operator(p, X, lambda xs: xs[0] * xs[0] * xs[1])
    np.testing.assert_allclose(got, expect, rtol=1e-12, atol=1e-10)


def test_piecewise_coefficient_indicators_sum_to_one():
    p = ri.config("piecewise2d", small=True)
    p.coef_vals = np.ones(16)
    X = np.random.default_rng(5).random((300, 2))
    xs = asm._coords(X, 0)
    a = asm.coefficient(p, xs)
    np.testing.assert_allclose(a.a, 1.0, atol=4e-15)
    np.testing.assert_allclose(a.b, 0.0, atol=1e-12)
    # and at a cell centre the coefficient is that cell's value up to the smoothing
    p.coef_vals = np.arange(1.0, 17.0)
    c = np.array([[(2 + 0.5) / 4, (1 + 0.5) / 4]])
    val = asm.coefficient(p, asm._coords(c, -1)).a[0]
    assert abs(val - p.coef_vals[1 * 4 + 2]) < 0.01


def test_rhs_heat_closed_form():
    """F = f - A[G] = -2 nu pi^2 sin(pi x) sin(pi y) for the heat problem."""
    p = ri.config("heat3d", small=True)
    X = ri.grid_points(p)
    F = asm.rhs(p, X)
    np.testing.assert_allclose(F, -2 * p.nu * np.pi ** 2 * np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]),
                               rtol=1e-12, atol=1e-12)


def test_block_entries_against_finite_differences():
    """(H_j)_{ik} = A[L omega_j phi_j^k](x_i): central differences of the
    value-only basis function agree to O(h^2)."""
    for name in ["multiscale2d", "heat3d"]:
        p = ri.config(name, small=True)
        R, b = ri.weights(p)
        j = 1
        rows, Psi, H = asm.block(p, R, b, j)
        X = ri.grid_points(p)[rows]
        mu, sig = asm.centres_halfwidths(p)
        ks = asm.subdomain_multi_index(p, j)

        def v(Y):   # plain float evaluation of L * omega_j * phi (all neurons)
            xs = asm._coords(Y, -1)
            lw = (asm.constraint_L(p, xs) * asm.window(p, xs, j)).a
            z = b[j][None, :] + sum(((Y[:, i] - mu[i][ks[i]]) / sig[i])[:, None] * R[j][None, :, i]
                                    for i in range(p.dim))
            return lw[:, None] * np.tanh(z)

        def a_of(Y):
            return asm.coefficient(p, asm._coords(Y, -1)).a

        sel = np.arange(0, X.shape[0], max(1, X.shape[0] // 7))
        Y = X[sel]
        h = 1e-4
        d1, d2 = [], []
        for i in range(p.dim):
            e = np.zeros(p.dim)
            e[i] = h
            vp, vm, v0 = v(Y + e), v(Y - e), v(Y)
            d1.append((vp - vm) / (2 * h))
            d2.append((vp - 2 * v0 + vm) / h ** 2)
        ns = p.spatial_dims
        lap = sum(d2[:ns])
        if p.op == ri.OP_DIFFUSION:
            a0 = a_of(Y)[:, None]
            ga = []
            for i in range(ns):
                e = np.zeros(p.dim)
                e[i] = h
                ga.append(((a_of(Y + e) - a_of(Y - e)) / (2 * h))[:, None])
            fd = -a0 * lap - sum(ga[i] * d1[i] for i in range(ns))
        else:
            fd = d1[p.dim - 1] - p.nu * lap
        scale = np.max(np.abs(H[sel]))
        np.testing.assert_allclose(H[sel], fd, rtol=0, atol=2e-4 * scale)


def test_constraint_gives_G_on_boundary():
    """Eq. (operator): u_hat = G exactly on the Dirichlet boundary for any W."""
    for name in ["poisson2d_2x2", "heat3d"]:
        p = ri.config(name, small=True)
        S = sv.build_system(p)
        W = np.random.default_rng(2).standard_normal(S.dof)
        Xb = ri.boundary_points(p, 9)
        u = sv.evaluate(S, W, Xb)
        xs = asm._coords(Xb, -1)
        np.testing.assert_array_equal(u, asm.constraint_G(p, xs).a)


# -------------------------------------------------------------------- PCA --

def test_pca_rank_rules_on_known_spectrum():
    rng = np.random.default_rng(11)
    n, m = 40, 12
    U, _ = np.linalg.qr(rng.standard_normal((n, m)))
    V, _ = np.linalg.qr(rng.standard_normal((m, m)))
    s = 10.0 ** -np.arange(m)          # 1, 0.1, ..., 1e-11
    Psi = U @ np.diag(s) @ V.T
    assert sv.pca(Psi, ri.PCA_ABS, 3e-4).rank == 4            # 1..1e-3 > 3e-4
    # variance: tail sum_{k>p} s_k^2 / total <= eps; total ~ 1.0101
    assert sv.pca(Psi, ri.PCA_VARIANCE, 1e-12).rank == 6     # tail at p=6: ~1e-12 * 1.0101 / 1.0101
    assert sv.pca(Psi, ri.PCA_VARIANCE, 1e-3).rank == 2
    assert sv.pca(Psi, ri.PCA_NONE, 0).rank == m


def test_pca_eckart_young():
    """||Psi - Psi V V^T||_F^2 = sum_{k > p} sigma_k^2 and V has orthonormal columns."""
    p = ri.config("multiscale2d", small=True)
    R, b = ri.weights(p)
    _, Psi, _ = asm.block(p, R, b, 5)
    pc = sv.pca(Psi, ri.PCA_ABS, 1e-2)
    resid = np.linalg.norm(Psi - Psi @ pc.V @ pc.V.T) ** 2
    tail = np.sum(pc.sigma[pc.rank:] ** 2)
    assert abs(resid - tail) <= 1e-8 * tail + 1e-24
    np.testing.assert_allclose(pc.V.T @ pc.V, np.eye(pc.rank), atol=1e-13)


def test_svd_brute_force_small():
    """Singular values of an 8x4 matrix equal sqrt(eig(A^T A)) computed by brute
    force on the characteristic polynomial's roots (exactly representable case)."""
    A = np.zeros((8, 4))
    A[0, 0], A[1, 1], A[2, 2], A[3, 3] = 5.0, 3.0, 2.0, 0.5
    Q, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((8, 8)))
    pc = sv.pca(Q @ A, ri.PCA_ABS, 1.0)
    np.testing.assert_allclose(pc.sigma, [5.0, 3.0, 2.0, 0.5], rtol=1e-14)
    assert pc.rank == 3


def test_jacobi_svd_2x2_closed_form():
    """A 2 x 2 matrix [[a, b], [c, d]] has singular values
    s1 = sqrt((S + sqrt(S^2 - 4 D^2)) / 2) and s2 = |D| / s1 with
    S = a^2 + b^2 + c^2 + d^2, D = ad - bc (s1 s2 = |det A|)."""
    for a, b, c, d in [(3.0, 1.0, -2.0, 4.0), (1.0, 2.0, 2.0, 4.0), (0.0, 5.0, 0.0, 0.0), (1e-3, 7.0, -2.0, 1e5)]:
        A = np.array([[a, b], [c, d]])
        S, D = a * a + b * b + c * c + d * d, a * d - b * c
        disc = np.sqrt(max(S * S - 4 * D * D, 0.0))
        s1 = np.sqrt((S + disc) / 2)
        want = np.array([s1, abs(D) / s1])
        s, Vt = la.jacobi_svd(A)
        np.testing.assert_allclose(s, want, rtol=1e-13, atol=4e-16 * want[0])
        np.testing.assert_allclose(Vt @ Vt.T, np.eye(2), atol=1e-15)
        # A^T A v_k = s_k^2 v_k
        for k in range(2):
            np.testing.assert_allclose(A.T @ (A @ Vt[k]), s[k] ** 2 * Vt[k], atol=1e-12 * want[0] ** 2)


@pytest.mark.parametrize("n,m", [(40, 12), (12, 12), (7, 30), (300, 41)])
def test_jacobi_svd_on_a_planted_spectrum(n, m):
    """A = U diag(s) V^T with orthonormal U, V and a known spectrum spanning 14
    orders of magnitude (tall, square and wide, odd m): the oracle's Jacobi SVD
    returns s to rounding of the largest value and the planted right singular
    vectors up to sign."""
    rng = np.random.default_rng(n * 131 + m)
    k = min(n, m)
    U, _ = np.linalg.qr(rng.standard_normal((n, k)))
    V, _ = np.linalg.qr(rng.standard_normal((m, k)))
    s = 10.0 ** -np.linspace(0, 14, k)
    A = U @ np.diag(s) @ V.T
    sg, Vt = la.jacobi_svd(A)
    assert sg.shape == (k,) and Vt.shape == (k, m)
    np.testing.assert_allclose(sg, s, rtol=0, atol=64 * max(n, m) * 2.2e-16)
    np.testing.assert_allclose(Vt @ Vt.T, np.eye(k), atol=1e-13)
    # vectors whose singular value is separated from the rest by a gap g are
    # fixed to an angle of about eps ||A|| / g (A itself carries rounding):
    # those with g > 1e-3 equal the planted ones up to sign
    for j in range(k):
        gap = min(abs(s[j] - s[i]) for i in range(k) if i != j) if k > 1 else 1.0
        if gap > 1e-3:
            assert abs(abs(Vt[j] @ V[:, j]) - 1.0) < 1e-12
    # reconstruction: A = (A V) V^T on the row space
    np.testing.assert_allclose((A @ Vt.T) @ Vt, A, atol=1e-13)


def test_jacobi_svd_rank_deficient_and_zero_columns():
    """Duplicate and zero columns: exactly zero singular values beyond the
    rank, and the kept vectors still orthonormal."""
    rng = np.random.default_rng(4)
    B = rng.standard_normal((20, 3))
    A = np.concatenate([B, B[:, :1], np.zeros((20, 2))], axis=1)     # rank 3 of 6 columns
    s, Vt = la.jacobi_svd(A)
    assert np.all(s[3:] <= 1e-14 * s[0])
    np.testing.assert_allclose(Vt @ Vt.T, np.eye(6), atol=1e-13)
    np.testing.assert_allclose(s[:3] ** 2, np.sort(np.linalg.eigvalsh(A.T @ A))[::-1][:3], rtol=1e-12)
    assert sv.pca(A, ri.PCA_ABS, 1e-8).rank == 3


def test_errors_closed_form():
    """Sec. 5 error measures on a case with known values: u = (1, -1, 1, -1)
    (mean 0, population std 1, ||u|| = 2) and u_hat = u + 1/2 give
    e_L2 = ||1/2||/||u|| = 1/2 and e_L1 = mean |1/2| / std(u) = 1/2; a sign or
    normalisation slip changes one of them."""
    u = np.array([1.0, -1.0, 1.0, -1.0])
    e2, e1 = sv.errors(u + 0.5, u)
    assert e2 == pytest.approx(0.5, rel=1e-15)
    assert e1 == pytest.approx(0.5, rel=1e-15)
    # u + 2 = (3, 1, 3, 1) has std 1 still; the error (-1, -2, -2, -2)
    e2, e1 = sv.errors(np.array([2.0, -1.0, 1.0, -1.0]), u + 2.0)
    assert e1 == pytest.approx(7.0 / 4.0, rel=1e-15)
    assert e2 == pytest.approx(np.sqrt(13.0 / 20.0), rel=1e-15)


# ---------------------------------------------------------- linear algebra --

def _exact_normal_solution(H, F):
    """Brute force: solve H^T H w = H^T F in rational arithmetic."""
    n = H.shape[1]
    A = [[sum(Fraction(int(H[r, i])) * int(H[r, j]) for r in range(H.shape[0])) for j in range(n)]
         for i in range(n)]
    y = [sum(Fraction(int(H[r, i])) * int(F[r]) for r in range(H.shape[0])) for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        y[c], y[piv] = y[piv], y[c]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c] / A[c][c]
                A[r] = [a - f * b for a, b in zip(A[r], A[c])]
                y[r] -= f * y[c]
    return np.array([float(y[i] / A[i][i]) for i in range(n)])


def test_householder_lstsq_exact_rational():
    rng = np.random.default_rng(5)
    H = rng.integers(-4, 5, size=(9, 4)).astype(float)
    F = rng.integers(-6, 7, size=9).astype(float)
    w = la.qr_lstsq(H, F)
    np.testing.assert_allclose(w, _exact_normal_solution(H, F), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(H.T @ (F - H @ w), 0.0, atol=1e-11)


def test_householder_qr_factors():
    A = np.random.default_rng(9).standard_normal((12, 7))
    V, beta, Rf = la.householder_qr(A)
    Q = np.eye(12)
    Q = np.stack([la.apply_qt(V, beta, Q[:, c]) for c in range(12)], axis=1).T   # Q = (Q^T)^T
    np.testing.assert_allclose(Q.T @ Q, np.eye(12), atol=1e-14)
    np.testing.assert_allclose((Q[:, :7] @ Rf), A, atol=1e-13)


def test_back_substitute_pseudo_inverse():
    P = np.array([[2.0, 1.0, 0.0], [0.0, 1e-20, 1.0], [0.0, 0.0, 4.0]])
    s = la.back_substitute(P, np.array([3.0, 5.0, 8.0]))
    assert s[1] == 0.0 and s[2] == 2.0 and s[0] == 1.5


def test_pcg_and_gmres_against_dense_solve():
    rng = np.random.default_rng(21)
    n = 30
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.linspace(1, 50, n)) @ Q.T
    b = rng.standard_normal(n)
    x, it, _ = la.pcg(lambda v: A @ v, b, None, 1e-12, 200)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9)
    Dinv = 1.0 / np.diag(A)
    x2, _, _ = la.pcg(lambda v: A @ v, b, lambda v: Dinv * v, 1e-12, 200)
    np.testing.assert_allclose(x2, np.linalg.solve(A, b), rtol=1e-9)
    N = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.3
    x3, it3, hist = la.gmres(lambda v: N @ v, b, None, 1e-12, 10, 500)
    np.testing.assert_allclose(x3, np.linalg.solve(N, b), rtol=1e-9)
    # within a restart cycle the GMRES residual estimate never increases
    h = np.array(hist[1:11])
    assert np.all(np.diff(h) <= 1e-15)
    # left preconditioning changes the iterates, not the solution
    x4, _, _ = la.gmres(lambda v: N @ v, b, lambda v: v / np.diag(N), 1e-12, 10, 500)
    np.testing.assert_allclose(x4, np.linalg.solve(N, b), rtol=1e-9)


def test_cg_exact_in_n_steps():
    """In exact arithmetic CG finishes in at most n steps; with 3 distinct
    eigenvalues it finishes in 3."""
    rng = np.random.default_rng(8)
    Q, _ = np.linalg.qr(rng.standard_normal((20, 20)))
    A = Q @ np.diag([1.0] * 7 + [3.0] * 7 + [10.0] * 6) @ Q.T
    b = rng.standard_normal(20)
    _, it, _ = la.pcg(lambda v: A @ v, b, None, 1e-12, 50)
    assert it == 3


def test_cgs_and_bicg_against_dense_solve():
    """The CG variants of Sec. 5 (Table 1b) reach the direct solution on an SPD
    system (with a Jacobi preconditioner) and on a nonsymmetric one."""
    rng = np.random.default_rng(31)
    n = 30
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.linspace(1, 50, n)) @ Q.T
    b = rng.standard_normal(n)
    Dinv = 1.0 / np.diag(A)
    xs = np.linalg.solve(A, b)
    x, it, _ = la.cgs(lambda v: A @ v, b, lambda v: Dinv * v, 1e-12, 200)
    np.testing.assert_allclose(x, xs, rtol=1e-9)
    x, it, _ = la.bicg(lambda v: A @ v, lambda v: A.T @ v, b, lambda v: Dinv * v, lambda v: Dinv * v, 1e-12, 200)
    np.testing.assert_allclose(x, xs, rtol=1e-9)
    N = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.3
    xn = np.linalg.solve(N, b)
    x, _, _ = la.cgs(lambda v: N @ v, b, None, 1e-12, 200)
    np.testing.assert_allclose(x, xn, rtol=1e-8)
    x, _, _ = la.bicg(lambda v: N @ v, lambda v: N.T @ v, b, None, None, 1e-12, 200)
    np.testing.assert_allclose(x, xn, rtol=1e-8)


def test_bicg_needs_the_transposed_preconditioner():
    """BiCG's shadow sequence uses M^T: with a nonsymmetric M it finishes in at
    most n steps (finite termination), and M in place of M^T breaks that."""
    rng = np.random.default_rng(32)
    n = 24
    N = np.eye(n) * 3 + rng.standard_normal((n, n)) * 0.4
    Mm = np.linalg.inv(np.tril(N))                       # nonsymmetric approximate inverse
    b = rng.standard_normal(n)
    _, it, hist = la.bicg(lambda v: N @ v, lambda v: N.T @ v, b, lambda v: Mm @ v, lambda v: Mm.T @ v, 1e-10, 3 * n)
    assert hist[-1] <= 1e-10 and it <= n + 2
    _, it2, hist2 = la.bicg(lambda v: N @ v, lambda v: N.T @ v, b, lambda v: Mm @ v, lambda v: Mm @ v, 1e-10, n + 2)
    assert hist2[-1] > 1e-10


def test_cgs_terminates_with_few_distinct_eigenvalues():
    """With 3 distinct eigenvalues the Krylov space closes after 3 steps; CGS,
    which squares the CG polynomial, reaches the solution in at most 3."""
    rng = np.random.default_rng(33)
    Q, _ = np.linalg.qr(rng.standard_normal((20, 20)))
    A = Q @ np.diag([1.0] * 7 + [3.0] * 7 + [10.0] * 6) @ Q.T
    b = rng.standard_normal(20)
    x, it, _ = la.cgs(lambda v: A @ v, b, None, 1e-11, 50)
    assert it <= 3
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9)


# ------------------------------------------------------------- Schwarz --

@pytest.mark.parametrize("kind", ["ras", "sas"])
def test_restricted_partition_of_identity(kind):
    """Sec. 3: sum_i R_i^T D_i R_i = I."""
    p = ri.config("multiscale2d", small=True)
    S = sv.build_system(p)
    M = sv.schwarz(S, kind)
    total = np.zeros(S.dof)
    for ix, D in zip(M.idx, M.D):
        np.add.at(total, ix, D)
    np.testing.assert_allclose(total, 1.0, rtol=1e-15)


@pytest.mark.parametrize("kind", ["as", "sas", "ras"])
def test_schwarz_transpose_is_the_adjoint(kind):
    """M^T = sum_i R_i^T A_i^{-1} D_i R_i: <M^T r, s> = <r, M s> (D_i moves to the input side)."""
    p = ri.config("multiscale2d", small=True)
    S = sv.build_system(p)
    M = sv.schwarz(S, kind)
    rng = np.random.default_rng(5)
    r, s = rng.standard_normal(S.dof), rng.standard_normal(S.dof)
    lhs, rhs = M.apply_t(r) @ s, r @ M.apply(s)
    assert abs(lhs - rhs) <= 1e-8 * np.linalg.norm(M.apply_t(r)) * np.linalg.norm(s)
    if kind != "as":   # not symmetric: M^T differs from M
        assert np.linalg.norm(M.apply_t(r) - M.apply(r)) > 1e-6 * np.linalg.norm(M.apply(r))


def test_local_matrix_is_restricted_normal_matrix():
    """A_i = R_i H^T H R_i^T against the dense normal matrix."""
    p = ri.config("multiscale2d", small=True)
    S = sv.build_system(p)
    Hd = S.dense()
    A = Hd.T @ Hd
    sets = sv.extended_sets(S)
    for i in (0, 5):
        ix = np.concatenate([np.arange(S.offsets[k], S.offsets[k + 1]) for k in sets[i]])
        np.testing.assert_allclose(sv.local_matrix(S, sets[i]), A[np.ix_(ix, ix)],
                                   rtol=1e-12, atol=1e-9 * np.abs(A).max())


def test_extended_sets_are_3x3_neighbourhoods():
    p = ri.config("multiscale2d", small=True)   # 4x4 subdomains, delta = 1.4
    S = sv.build_system(p)
    sets = sv.extended_sets(S)
    assert sets[0] == [0, 1, 4, 5]
    assert sets[5] == [0, 1, 2, 4, 5, 6, 8, 9, 10]


def test_as_one_iteration_on_2x2():
    """Table 2 (J = 2x2): AS-preconditioned CG stops after one iteration."""
    p = ri.config("poisson2d_2x2")
    S = sv.build_system(p)
    sol = sv.solve(S, "cg", sv.schwarz(S, "as"), 1e-10)
    assert sol.iters == GOLDEN["as_iters_2x2"]["value"]
    # M_AS^{-1} H^T H = J I on every vector
    # (exact up to rounding amplified by kappa(H^T H): the tolerance is kappa * eps)
    x = np.random.default_rng(0).standard_normal(S.dof)
    y = sv.schwarz(S, "as").apply(S.normal(x))
    Hd = S.dense()
    kappa = np.linalg.cond(Hd.T @ Hd)
    assert np.linalg.norm(y - p.J * x) <= 10 * kappa * 2.2e-16 * np.linalg.norm(p.J * x)


def test_as_cg_one_iteration_on_2x2x2():
    """Table 3 (J = 2x2x2): AS-preconditioned CG takes one iteration."""
    p = ri.config("poisson3d", small=True)
    S = sv.build_system(p)
    sol = sv.solve(S, "cg", sv.schwarz(S, "as"), 1e-10)
    assert sol.iters == GOLDEN["as_cg_iters_2x2x2"]["value"]


def test_krylov_matches_direct_least_squares():
    """The preconditioned solves reach the least-squares minimum of the QR solve."""
    p = ri.config("multiscale2d", small=True)
    S = sv.build_system(p)
    qr = sv.solve_qr(S)
    for kind, solver in [("as", "cg"), ("sas", "gmres"), ("as", "cgs"), ("sas", "cgs"), ("ras", "cgs"),
                         ("as", "bicg"), ("sas", "bicg")]:
        sol = sv.solve(S, solver, sv.schwarz(S, kind), 1e-10, 50, 3000)
        assert abs(sol.res_ls - qr.res_ls) <= 1e-8 * np.linalg.norm(S.F), (kind, solver)


@pytest.mark.parametrize("solver", ["cgs", "bicg"])
def test_cg_variants_one_iteration_on_2x2(solver):
    """With M_AS^{-1} H^T H = J I on J = 2x2 (Table 2), any Krylov method is done
    after one step; Table 1b's variants included."""
    p = ri.config("poisson2d_2x2")
    S = sv.build_system(p)
    sol = sv.solve(S, solver, sv.schwarz(S, "as"), 1e-8)
    assert sol.iters == 1


def test_manufactured_solution_accuracy():
    """Config 1 (2D Poisson, 2x2): e_L2 well below the paper's 1e-3..1e-5 band edge."""
    p = ri.config("poisson2d_2x2")
    S = sv.build_system(p)
    sol = sv.solve(S, "cg", sv.schwarz(S, "as"), 1e-10)
    X = ri.test_points(p, 50)
    e2, e1 = sv.errors(sv.evaluate(S, sol.W, X), ri.exact_solution(p, X))
    assert e2 < 1e-3 and e1 < 1e-3


def test_forced_ranks_reproduce_the_rule_and_extend_the_basis():
    """build_system(ranks=...): the rule's own ranks give the same system; one
    more column on a subdomain appends Psi_j's next right singular vector and
    cannot raise the least-squares minimum; ranks outside 1..min(N_j, m) are
    rejected."""
    p = ri.config("poisson2d_2x2", small=True)
    R, b = ri.weights(p)
    S = sv.build_system(p, R, b)
    ranks = [pc.rank for pc in S.pcas]
    S1 = sv.build_system(p, R, b, ranks=ranks)
    for B0, B1 in zip(S.B, S1.B):
        np.testing.assert_array_equal(B0, B1)
    j = next(j for j in range(p.J) if ranks[j] < min(S.B[j].shape[0], p.neurons))
    r2 = list(ranks)
    r2[j] += 1
    S2 = sv.build_system(p, R, b, ranks=r2)
    np.testing.assert_array_equal(S2.pcas[j].V[:, :ranks[j]], S.pcas[j].V)
    _, Psi, _ = asm.block(p, R, b, j)
    Vt = np.linalg.svd(Psi, full_matrices=False)[2]
    np.testing.assert_allclose(np.abs(S2.pcas[j].V[:, -1]), np.abs(Vt[ranks[j]]), atol=1e-12)
    assert S2.pcas[j].borderline == S.pcas[j].borderline

    def ls_min(Sx):
        return np.linalg.norm(Sx.F - Sx.H(np.linalg.lstsq(Sx.dense(), Sx.F, rcond=None)[0]))

    assert ls_min(S2) <= ls_min(S) * (1 + 1e-12)
    with pytest.raises(ValueError):
        sv.build_system(p, R, b, ranks=[0] * p.J)


# ------------------------------------------------------------- Table 1 --

def test_table1_largest_eigenvalues_of_the_preconditioned_normal_matrix():
    """Sec. 5, Example 1, Table 1 (4x4 subdomains, 40x40 points, delta = 2,
    m = 16, no PCA): the largest real part of the eigenvalues of
    M^{-1} H^T H for AS, SAS and RAS within the band of the paper's values
    (another random draw), and for AS at most 4^2 = 16, the bound the paper
    gives: a collocation point lies in at most 4 subdomains (checked here on
    the geometry), squared by the least-squares form."""
    import dataclasses
    p = dataclasses.replace(ri.example1_paper(), pca_mode=ri.PCA_NONE)
    counts = np.zeros(p.n_points(), dtype=int)
    for j in range(p.J):
        counts[asm.box_rows(p, j)] += 1
    assert counts.max() == 4
    S = sv.build_system(p)
    A = S.dense()
    A = A.T @ A
    n = A.shape[0]
    assert n == 256 and S.n_rows == 1600
    band = BANDS["table1_lambda_max"]
    for kind, ref in band["value"].items():
        M = sv.schwarz(S, kind)
        Minv = np.column_stack([M.apply(e) for e in np.eye(n)])
        lmax = float(np.linalg.eigvals(Minv @ A).real.max())
        assert abs(lmax - ref) <= band["rel_band"] * ref, (kind, lmax, ref)
        if kind == "as":
            assert lmax <= 16.0 * (1 + 1e-9)


def test_table1_error_of_the_as_preconditioned_gmres_solution():
    """Sec. 5, Example 1, Table 1: the relative L2 error of u_hat on 350 x 350
    test points after AS-preconditioned GMRES to 1e-5 (no PCA, m = 16),
    within the band of the paper's value."""
    import dataclasses
    p = dataclasses.replace(ri.example1_paper(), pca_mode=ri.PCA_NONE)
    S = sv.build_system(p)
    sol = sv.solve(S, "gmres", sv.schwarz(S, "as"), 1e-5, 50, 3000)
    X = ri.test_points(p, 350)
    e2, _ = sv.errors(sv.evaluate(S, sol.W, X), ri.exact_solution(p, X))
    band = BANDS["table1_eL2_as"]
    assert abs(e2 - band["value"]) <= band["rel_band"] * band["value"], e2


# ------------------------------------------------------- differentiation --

def _lstsq_and_adjoint(S, c):
    """W = H^+ F and lam = (H^T H)^{-1} c from one SVD of the dense H."""
    U, sg, Vt = np.linalg.svd(S.dense(), full_matrices=False)
    W = Vt.T @ ((U.T @ S.F) / sg)
    lam = Vt.T @ ((Vt @ c) / sg ** 2)
    return W, lam


@pytest.mark.parametrize("c0,loss_kind,g_kind", [(0.0, "linear", ri.G_ZERO), (0.7, "linear", ri.G_SINPROD),
                                                  (0.3, "quadratic", ri.G_SINPROD)])
def test_grad_c0_is_the_derivative_of_the_least_squares_solution(c0, loss_kind, g_kind):
    """grad_c0 against central differences of l(W(c0)) for a loss that depends
    on c0 only through the least-squares solution W(c0) of -Lap u + c0 u:
    l = c . W, or l = 1/2 ||W - w0||^2 (dl/dW = W - w0); with G = 0 and with
    G = prod sin(pi x_i) (so each of the formula's three terms is exercised).
    The PCA basis does not depend on c0, which the test checks."""
    import dataclasses
    p = dataclasses.replace(ri.config("poisson2d_2x2", small=True), c0=c0, g_kind=g_kind)
    R, b = ri.weights(p)
    S = sv.build_system(p, R, b)
    rng = np.random.default_rng(11)
    c = rng.standard_normal(S.dof)
    w0 = rng.standard_normal(S.dof)

    def loss_and_grad(W):
        if loss_kind == "linear":
            return float(c @ W), c
        return 0.5 * float(np.sum((W - w0) ** 2)), W - w0

    W, _ = _lstsq_and_adjoint(S, c)
    _, lam = _lstsq_and_adjoint(S, loss_and_grad(W)[1])
    grad = sv.grad_c0(S, W, lam)
    h = 1e-4

    def loss(c0v):
        S2 = sv.build_system(dataclasses.replace(p, c0=c0v), R, b)
        for pa, pb in zip(S.pcas, S2.pcas):
            np.testing.assert_array_equal(pa.V, pb.V)
        return loss_and_grad(_lstsq_and_adjoint(S2, c)[0])[0]

    fd = (loss(c0 + h) - loss(c0 - h)) / (2 * h)
    assert abs(grad - fd) <= 2e-5 * abs(fd)


@pytest.mark.parametrize("loss_kind,g_kind", [("linear", ri.G_ZERO), ("quadratic", ri.G_SINPROD)])
def test_grad_coef_is_the_derivative_of_the_least_squares_solution(loss_kind, g_kind):
    """grad_coef against central differences of l(W(a)) in three cell values
    a_c of the piecewise diffusion coefficient (a 2 x 2 grid of subdomains,
    4 x 4 coefficient cells); G = 0 and G = sin(pi x) sin(pi y) (then
    dF/da_c = -A_c[G] is not zero, so each term of the formula is exercised).
    The PCA basis does not depend on a, which the test checks."""
    import dataclasses
    p = dataclasses.replace(ri.piecewise2d(0, sub=2, pts=8, neurons=20), g_kind=g_kind)
    R, b = ri.weights(p)
    S = sv.build_system(p, R, b)
    rng = np.random.default_rng(5)
    c = rng.standard_normal(S.dof)
    w0 = rng.standard_normal(S.dof)

    def loss_and_grad(W):
        if loss_kind == "linear":
            return float(c @ W), c
        return 0.5 * float(np.sum((W - w0) ** 2)), W - w0

    W, _ = _lstsq_and_adjoint(S, c)
    _, lam = _lstsq_and_adjoint(S, loss_and_grad(W)[1])
    grad = sv.grad_coef(S, W, lam)
    assert grad.shape == (16,)
    h = 1e-5
    for cell in (0, 5, 14):
        def loss(delta):
            vals = p.coef_vals.copy()
            vals[cell] += delta
            S2 = sv.build_system(dataclasses.replace(p, coef_vals=vals), R, b)
            for pa, pb in zip(S.pcas, S2.pcas):
                np.testing.assert_array_equal(pa.V, pb.V)
            return loss_and_grad(_lstsq_and_adjoint(S2, c)[0])[0]
        fd = (loss(h) - loss(-h)) / (2 * h)
        assert abs(grad[cell] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(grad).max()), (cell, grad[cell], fd)


def test_eval_matrix_transpose_is_the_adjoint_of_u_hat():
    """E^T r equals the brute-force transpose of the evaluation matrix at the
    collocation points (columns from evaluate on unit coefficient vectors)."""
    p = ri.config("heat3d", small=True)
    S = sv.build_system(p)
    X = ri.grid_points(p)
    g0 = sv.evaluate(S, np.zeros(S.dof), X)
    E = np.stack([sv.evaluate(S, np.eye(S.dof)[c], X) - g0 for c in range(S.dof)], axis=1)
    r = np.random.default_rng(8).standard_normal(X.shape[0])
    np.testing.assert_allclose(sv.eval_matrix_t(S, r), E.T @ r, rtol=0, atol=1e-12 * np.abs(E.T @ r).max())


# ------------------------------------------------------ planted mistakes --

def test_planted_dropped_window_normalisation_is_caught(monkeypatch):
    monkeypatch.setattr(asm, "window", lambda p, xs, j: asm.window_hat(p, xs, j))
    with pytest.raises(AssertionError):
        test_partition_of_unity("multiscale2d")


def test_planted_diffusion_sign_is_caught(monkeypatch):
    orig = asm.apply_operator

    def wrong(p, X, field):
        if p.op != ri.OP_DIFFUSION:
            return orig(p, X, field)
        q = ri.Problem(**{**p.__dict__})
        q.op = ri.OP_POISSON
        return orig(q, X, field) * 2.0   # drops grad a . grad v, uses a = 2
    monkeypatch.setattr(asm, "apply_operator", wrong)
    with pytest.raises(AssertionError):
        test_diffusion_operator_closed_form()


def test_planted_wrong_restriction_is_caught(monkeypatch):
    orig = sv.extended_sets
    monkeypatch.setattr(sv, "extended_sets", lambda S, lvl=1: orig(S, 0))   # block Jacobi
    with pytest.raises(AssertionError):
        test_as_one_iteration_on_2x2()


def test_planted_transposed_weights_is_caught(monkeypatch):
    orig = ri.weights

    def swapped(p):
        R, b = orig(p)
        return R[:, :, ::-1].copy(), b
    monkeypatch.setattr(ri, "weights", swapped)
    with pytest.raises(AssertionError):
        test_weights_range_and_order()
