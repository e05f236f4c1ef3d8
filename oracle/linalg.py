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
No LAPACK: every factorisation here is written out.
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
