"""Oracle: textbook dense linear algebra and Krylov solvers in float64.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline use this package; the product path never does.

  * householder_qr / qr_solve: Householder QR (Golub & Van Loan, Alg. 5.2.1),
    used for the direct least-squares solve (Sec. 5, the QR baseline of
    Table 3) and for the local inverses A_i^{-1} = P_i^{-1} Q_i^T (Sec. 3);
    where P_i is singular, the pseudo-inverse reading zeroes the components
    whose pivot |P_kk| < 1e-14 max |P_kk|.
  * pcg: preconditioned conjugate gradients (Saad, Iterative Methods for
    Sparse Linear Systems, Alg. 9.1), stopping on ||b - A x|| / ||b||.
  * gmres: left-preconditioned restarted GMRES(k) with modified Gram-Schmidt
    and Givens rotations (Saad Alg. 9.4), stopping on
    ||M^{-1}(b - A x)|| / ||M^{-1} b|| (Sec. 5, Example 1 stopping rule).
  * cgs, bicg: the two CG variants of Sec. 5 (Table 1b) -- conjugate
    gradient squared (Sonneveld 1989) and biconjugate gradients (Fletcher
    1976), preconditioned as in Barrett et al., "Templates for the Solution of
    Linear Systems" (1994), Figs. 2.9 and 2.8; BiCG also applies A^T and M^T.
    Both stop on ||b - A x|| / ||b||.
  * jacobi_svd: the reduced SVD that the PCA of Sec. 4 (Eq. (pca)) needs --
    singular values and right singular vectors by one-sided Jacobi rotations
    (Hestenes 1958; Golub & Van Loan Sec. 8.6.3) applied to the triangular
    factor of a Householder QR (the QR-preconditioned form of Drmac and
    Veselic 2008), with the pairs of each sweep visited in round-robin order
    so that the m/2 rotations of one round touch disjoint columns.
No LAPACK: every factorisation here is written out (numpy supplies only
vector arithmetic, norms and products).
"""
from __future__ import annotations

import numpy as np


def householder_qr(A: np.ndarray):
    """A (n x k, n >= k) -> (V, beta, Rfac): reflectors I - beta v v^T and upper Rfac."""
    A = np.array(A, dtype=np.float64, copy=True)
    n, k = A.shape
    V = np.zeros((n, k))
    beta = np.zeros(k)
    for c in range(k):
        x = A[c:, c]
        normx = np.linalg.norm(x)
        if normx == 0.0:
            continue
        v = x.copy()
        alpha = -normx if x[0] >= 0 else normx
        v[0] -= alpha
        vnorm2 = v @ v
        if vnorm2 == 0.0:
            continue
        bt = 2.0 / vnorm2
        A[c:, c:] -= bt * np.outer(v, v @ A[c:, c:])
        V[c:, c] = v
        beta[c] = bt
    return V, beta, np.triu(A[:k, :k])


def apply_qt(V: np.ndarray, beta: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Q^T y for the reflectors of householder_qr."""
    y = np.array(y, dtype=np.float64, copy=True)
    for c in range(V.shape[1]):
        if beta[c] != 0.0:
            v = V[c:, c]
            y[c:] -= beta[c] * v * (v @ y[c:])
    return y


def back_substitute(Rf: np.ndarray, y: np.ndarray, rel_tol: float = 1e-14) -> np.ndarray:
    """Solve Rf s = y (upper triangular); components with |R_kk| below
    rel_tol * max |R_kk| are set to zero (pseudo-inverse reading, Sec. 3)."""
    k = Rf.shape[0]
    s = np.zeros(k)
    dmax = np.max(np.abs(np.diag(Rf))) if k else 0.0
    for i in range(k - 1, -1, -1):
        d = Rf[i, i]
        if abs(d) <= rel_tol * dmax:
            s[i] = 0.0
            continue
        s[i] = (y[i] - Rf[i, i + 1:] @ s[i + 1:]) / d
    return s


def qr_lstsq(H: np.ndarray, F: np.ndarray) -> np.ndarray:
    """min ||H W - F||_2 by Householder QR (the direct solver of Sec. 5)."""
    V, beta, Rf = householder_qr(H)
    y = apply_qt(V, beta, F)[: H.shape[1]]
    return back_substitute(Rf, y)


def pcg(apply_A, b: np.ndarray, apply_M=None, rtol=1e-10, maxit=1000):
    """Preconditioned CG from x0 = 0; returns (x, iters, history of ||r||/||b||)."""
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = np.linalg.norm(b)
    hist = [1.0]
    if bnorm == 0.0:
        return x, 0, hist
    z = apply_M(r) if apply_M else r.copy()
    pvec = z.copy()
    rz = r @ z
    it = 0
    while it < maxit:
        Ap = apply_A(pvec)
        pAp = pvec @ Ap
        if pAp <= 0.0:
            break
        alpha = rz / pAp
        x = x + alpha * pvec
        r = r - alpha * Ap
        it += 1
        rel = np.linalg.norm(r) / bnorm
        hist.append(rel)
        if rel <= rtol:
            break
        z = apply_M(r) if apply_M else r.copy()
        rz_new = r @ z
        pvec = z + (rz_new / rz) * pvec
        rz = rz_new
    return x, it, hist


def gmres(apply_A, b: np.ndarray, apply_M=None, rtol=1e-10, restart=50, maxit=1000):
    """Left-preconditioned GMRES(restart) from x0 = 0.

    Returns (x, iters, history of the preconditioned relative residual)."""
    M = apply_M if apply_M else (lambda v: v.copy())
    n = b.shape[0]
    x = np.zeros(n)
    Mb = M(b)
    mbnorm = np.linalg.norm(Mb)
    hist = [1.0]
    if mbnorm == 0.0:
        return x, 0, hist
    it = 0
    while it < maxit:
        r = M(b - apply_A(x))
        beta = np.linalg.norm(r)
        if beta / mbnorm <= rtol:
            break
        k = min(restart, maxit - it)
        V = np.zeros((k + 1, n))
        Hh = np.zeros((k + 1, k))
        cs = np.zeros(k)
        sn = np.zeros(k)
        g = np.zeros(k + 1)
        g[0] = beta
        V[0] = r / beta
        jdone = 0
        for j in range(k):
            w = M(apply_A(V[j]))
            for i in range(j + 1):
                Hh[i, j] = w @ V[i]
                w = w - Hh[i, j] * V[i]
            Hh[j + 1, j] = np.linalg.norm(w)
            if Hh[j + 1, j] != 0.0:
                V[j + 1] = w / Hh[j + 1, j]
            for i in range(j):
                t = cs[i] * Hh[i, j] + sn[i] * Hh[i + 1, j]
                Hh[i + 1, j] = -sn[i] * Hh[i, j] + cs[i] * Hh[i + 1, j]
                Hh[i, j] = t
            den = np.hypot(Hh[j, j], Hh[j + 1, j])
            cs[j], sn[j] = (1.0, 0.0) if den == 0.0 else (Hh[j, j] / den, Hh[j + 1, j] / den)
            Hh[j, j] = cs[j] * Hh[j, j] + sn[j] * Hh[j + 1, j]
            Hh[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            jdone = j + 1
            hist.append(abs(g[j + 1]) / mbnorm)
            if abs(g[j + 1]) / mbnorm <= rtol or Hh[j, j] == 0.0:
                break
        y = np.zeros(jdone)
        for i in range(jdone - 1, -1, -1):
            y[i] = (g[i] - Hh[i, i + 1:jdone] @ y[i + 1:]) / Hh[i, i] if Hh[i, i] != 0.0 else 0.0
        x = x + V[:jdone].T @ y
        if hist[-1] <= rtol:
            break
    return x, it, hist


def cgs(apply_A, b: np.ndarray, apply_M=None, rtol=1e-10, maxit=1000):
    """Preconditioned conjugate gradient squared from x0 = 0 (shadow residual
    r~ = r_0); returns (x, iters, history of ||r||/||b||)."""
    M = apply_M if apply_M else (lambda v: v.copy())
    x = np.zeros_like(b)
    r = b.copy()
    rt = r.copy()
    bnorm = np.linalg.norm(b)
    hist = [1.0]
    if bnorm == 0.0:
        return x, 0, hist
    rho_prev = 1.0
    u = p = q = None
    it = 0
    while it < maxit:
        rho = rt @ r
        if rho == 0.0:
            break
        if it == 0:
            u = r.copy()
            p = u.copy()
        else:
            beta = rho / rho_prev
            u = r + beta * q
            p = u + beta * (q + beta * p)
        ph = M(p)
        vh = apply_A(ph)
        sigma = rt @ vh
        if sigma == 0.0:
            break
        alpha = rho / sigma
        q = u - alpha * vh
        uh = M(u + q)
        x = x + alpha * uh
        r = r - alpha * apply_A(uh)
        rho_prev = rho
        it += 1
        rel = np.linalg.norm(r) / bnorm
        hist.append(rel)
        if rel <= rtol:
            break
    return x, it, hist


def bicg(apply_A, apply_AT, b: np.ndarray, apply_M=None, apply_MT=None, rtol=1e-10, maxit=1000):
    """Preconditioned biconjugate gradients from x0 = 0 (shadow residual
    r~ = r_0); returns (x, iters, history of ||r||/||b||)."""
    M = apply_M if apply_M else (lambda v: v.copy())
    MT = apply_MT if apply_MT else (lambda v: v.copy())
    x = np.zeros_like(b)
    r = b.copy()
    rt = r.copy()
    bnorm = np.linalg.norm(b)
    hist = [1.0]
    if bnorm == 0.0:
        return x, 0, hist
    rho_prev = 1.0
    p = pt = None
    it = 0
    while it < maxit:
        z = M(r)
        zt = MT(rt)
        rho = z @ rt
        if rho == 0.0:
            break
        if it == 0:
            p, pt = z.copy(), zt.copy()
        else:
            beta = rho / rho_prev
            p = z + beta * p
            pt = zt + beta * pt
        q = apply_A(p)
        qt = apply_AT(pt)
        sigma = pt @ q
        if sigma == 0.0:
            break
        alpha = rho / sigma
        x = x + alpha * p
        r = r - alpha * q
        rt = rt - alpha * qt
        rho_prev = rho
        it += 1
        rel = np.linalg.norm(r) / bnorm
        hist.append(rel)
        if rel <= rtol:
            break
    return x, it, hist


def apply_q(V: np.ndarray, beta: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Q Y for the reflectors of householder_qr (reflectors applied in reverse
    order); Y has V.shape[0] rows."""
    Y = np.array(Y, dtype=np.float64, copy=True)
    for c in range(V.shape[1] - 1, -1, -1):
        if beta[c] != 0.0:
            v = V[c:, c]
            Y[c:] -= beta[c] * np.outer(v, v @ Y[c:])
    return Y


def _round_robin(m: int):
    """The m - 1 rounds (m even) of a round-robin tournament on 0..m-1: each
    round pairs every index with exactly one other, and over all rounds every
    pair meets once."""
    idx = list(range(m))
    rounds = []
    for _ in range(m - 1):
        rounds.append((np.array(idx[: m // 2]), np.array(idx[m // 2:][::-1])))
        idx = [idx[0], idx[-1]] + idx[1:-1]
    return rounds


def _one_sided_jacobi(G: np.ndarray, tol: float, max_sweeps: int):
    """Orthogonalise the columns of G (n x m) by plane rotations G <- G J_pq,
    accumulating V = prod J_pq: for the pair (p, q) with a = |g_p|^2,
    b = |g_q|^2, c = g_p . g_q the rotation that diagonalises [[a, c], [c, b]]
    (zeta = (b - a)/(2c), t = sign(zeta)/(|zeta| + sqrt(1 + zeta^2)),
    cs = 1/sqrt(1 + t^2), sn = cs t).  Pairs with |c| <= tol sqrt(a b) are
    left alone; the sweeps stop when a whole sweep rotates nothing.  The
    columns are held as the rows of G^T and V^T (contiguous).  Returns
    (G V, V, sweeps)."""
    Gt = np.array(np.asarray(G, dtype=np.float64).T, copy=True, order="C")
    m, n = Gt.shape
    pad = m % 2
    if pad:
        Gt = np.concatenate([Gt, np.zeros((1, n))], axis=0)
    mm = m + pad
    Vt = np.eye(mm)
    rounds = _round_robin(mm)
    sweep = 0
    for sweep in range(1, max_sweeps + 1):
        rotated = 0
        for P, Q in rounds:
            gp, gq = Gt[P], Gt[Q]
            a = np.einsum("ij,ij->i", gp, gp)
            b = np.einsum("ij,ij->i", gq, gq)
            c = np.einsum("ij,ij->i", gp, gq)
            act = np.abs(c) > tol * np.sqrt(a * b)
            if not np.any(act):
                continue
            rotated += int(act.sum())
            P, Q, a, b, c = P[act], Q[act], a[act], b[act], c[act]
            zeta = (b - a) / (2.0 * c)
            big = np.abs(zeta) > 1e150               # t = 1/(2 zeta) to rounding; avoids zeta^2 overflow
            zs = np.where(big, 0.0, zeta)
            t = np.where(big, 0.5 / np.where(big, zeta, 1.0),
                         np.where(zeta >= 0, 1.0, -1.0) / (np.abs(zs) + np.sqrt(1.0 + zs * zs)))
            cs = (1.0 / np.sqrt(1.0 + t * t))[:, None]
            sn = cs * t[:, None]
            for M in (Gt, Vt):
                mp, mq = M[P], M[Q]
                M[P] = cs * mp - sn * mq
                M[Q] = sn * mp + cs * mq
        if rotated == 0:
            break
    return Gt[:m].T, Vt[:m, :m].T, sweep


def jacobi_svd(A: np.ndarray, max_sweeps: int = 60):
    """Reduced SVD data of A (n x m): singular values in descending order
    (min(n, m) of them) and the matching right singular vectors as the rows of
    Vt (min(n, m) x m), so that A = U diag(s) Vt with orthonormal U.

    Tall case (n >= m): A = Q R by householder_qr; R (m x m) has the singular
    values and right singular vectors of A, and one-sided Jacobi on R's
    columns gives R V = U_R diag(s).  Wide case (n < m): A^T = Q R, so
    A = R^T Q^T; one-sided Jacobi on R^T (n x n) gives R^T W = U diag(s) and
    the right singular vectors of A are the columns of Q W.  The singular
    values are the column norms of the rotated matrix."""
    A = np.asarray(A, dtype=np.float64)
    n, m = A.shape
    eps = np.finfo(np.float64).eps
    if n >= m:
        _, _, Rf = householder_qr(A)
        Gv, V, _ = _one_sided_jacobi(Rf, m * eps, max_sweeps)
        s = np.sqrt(np.einsum("ij,ij->j", Gv, Gv))
        order = np.argsort(-s, kind="stable")
        return s[order], V[:, order].T.copy()
    Vq, bq, Rf = householder_qr(A.T)
    Gv, W, _ = _one_sided_jacobi(Rf.T, n * eps, max_sweeps)
    s = np.sqrt(np.einsum("ij,ij->j", Gv, Gv))
    order = np.argsort(-s, kind="stable")
    QW = apply_q(Vq, bq, np.concatenate([W, np.zeros((m - n, n))], axis=0))
    return s[order], QW[:, order].T.copy()
