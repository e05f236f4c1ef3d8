"""Oracle: PCA reduction, Schwarz preconditioners, solves and evaluation.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline use this package; the product path never does.

  * Sec. 4 Eq. (pca)/(pca_net): reduced SVD Psi_j = U S V^T (the oracle's own
    one-sided Jacobi SVD, linalg.jacobi_svd); keep p_j columns of V, by the
    absolute threshold
    sigma_k > tau (Sec. 4) or by the variance rule: the smallest p with
    sum_{k<=p} sigma_k^2 >= (1 - eps) sum_k sigma_k^2.
    Reduced block B_j = H_j V_{p_j} (Eq. (system_new)).
  * Sec. 2: normal equations H^T H W = H^T F.
  * Sec. 3: M_AS^{-1} = sum_i R_i^T A_i^{-1} R_i, A_i = R_i H^T H R_i^T;
    M_RAS^{-1} = sum_i R_i^T D_i A_i^{-1} R_i with sum_i R_i^T D_i R_i = I;
    D_i Boolean (RAS) or 1/(number of sets holding the unknown) (SAS, Sec. 5).
    Reading of R_i: it selects the unknowns of every subdomain whose box
    shares a collocation point with box_i (the extended set N(i)); with
    overlap_level = 0 it selects subdomain i's own unknowns only.
  * Sec. 5: u_hat = L sum_j omega_j (V_{p_j}^T Phi_j) . W_j + G (Eq. (netdd)),
    relative L2 error and normalised L1 error at test points.
  * Differentiation through the least-squares solve (an extension; the
    paper does not differentiate): grad_c0, the derivative of a loss l(W)
    with respect to the reaction coefficient c0 of -Lap u + c0 u, and
    grad_coef, its derivative with respect to the cell values a_c of the
    piecewise diffusion coefficient a = sum_c a_c s_c of -div(a grad u);
    eval_matrix_t, the adjoint of u_hat at the collocation points (for
    losses on u_hat).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

import rann_inputs as ri
from . import assembly as asm
from . import hyperdual as hd
from . import linalg as la


@dataclasses.dataclass
class PCA:
    sigma: np.ndarray     # all singular values of Psi_j, descending
    V: np.ndarray         # m x p_j
    rank: int
    borderline: bool      # a singular value lies within 1e-6 (relative) of the cut


def pca_rank(sigma: np.ndarray, mode: int, thr: float) -> int:
    if mode == ri.PCA_NONE:
        return sigma.shape[0]
    if mode == ri.PCA_ABS:
        return int(np.sum(sigma > thr))
    if mode == ri.PCA_VARIANCE:
        s2 = sigma ** 2
        total = s2.sum()
        csum = np.cumsum(s2)
        return int(np.argmax(csum >= (1.0 - thr) * total) + 1)
    raise ValueError(mode)


def pca(Psi: np.ndarray, mode: int, thr: float, rank: Optional[int] = None) -> PCA:
    """Sec. 4: the p_j leading right singular vectors of Psi_j, p_j by the
    rank rule, or the given rank (a rank that another implementation chose
    at a borderline cut; borderline still refers to the rule)."""
    m = Psi.shape[1]
    s, Vt = la.jacobi_svd(Psi)
    if mode == ri.PCA_NONE:
        return PCA(s, np.eye(m), m, False)
    p = pca_rank(s, mode, thr)
    if rank is not None:
        if not 1 <= rank <= Vt.shape[0]:
            raise ValueError(f"rank {rank} outside 1..{Vt.shape[0]}")
        rule = p
        p = rank
    else:
        rule = p
    # borderline: does a 1e-6 relative wobble of the singular values move the rank?
    lo = pca_rank(s * (1 - 1e-6), mode, thr) if mode == ri.PCA_ABS else pca_rank(
        np.concatenate([s[:rule] * (1 - 1e-6), s[rule:] * (1 + 1e-6)]), mode, thr)
    hi = pca_rank(s * (1 + 1e-6), mode, thr) if mode == ri.PCA_ABS else pca_rank(
        np.concatenate([s[:rule] * (1 + 1e-6), s[rule:] * (1 - 1e-6)]), mode, thr)
    return PCA(s, Vt[:p].T.copy(), p, lo != rule or hi != rule)


@dataclasses.dataclass
class System:
    problem: ri.Problem
    R: np.ndarray
    b: np.ndarray
    rows: List[np.ndarray]      # global point indices of block j
    B: List[np.ndarray]         # reduced blocks N_j x p_j
    pcas: List[PCA]
    F: np.ndarray               # N
    offsets: np.ndarray         # column offset of W_j, length J+1

    @property
    def dof(self) -> int:
        return int(self.offsets[-1])

    @property
    def n_rows(self) -> int:
        return self.F.shape[0]

    # H x and H^T y over the block storage
    def H(self, x: np.ndarray) -> np.ndarray:
        y = np.zeros(self.n_rows)
        for j, Bj in enumerate(self.B):
            np.add.at(y, self.rows[j], Bj @ x[self.offsets[j]:self.offsets[j + 1]])
        return y

    def HT(self, y: np.ndarray) -> np.ndarray:
        return np.concatenate([Bj.T @ y[self.rows[j]] for j, Bj in enumerate(self.B)])

    def normal(self, x: np.ndarray) -> np.ndarray:
        return self.HT(self.H(x))

    def dense(self) -> np.ndarray:
        Hd = np.zeros((self.n_rows, self.dof))
        for j, Bj in enumerate(self.B):
            Hd[self.rows[j], self.offsets[j]:self.offsets[j + 1]] = Bj
        return Hd


def build_system(p: ri.Problem, R=None, b=None, blocks_subset=None, ranks=None) -> System:
    """Algorithm 1 steps 1-5: geometry, networks, windows and C, PCA, reduced system.
    ranks: optional p_j per subdomain in place of the rank rule."""
    if R is None:
        R, b = ri.weights(p)
    js = range(p.J) if blocks_subset is None else blocks_subset
    rows, Bs, pcas = [], [], []
    for j in js:
        r, Psi, Hj = asm.block(p, R, b, j)
        pc = pca(Psi, p.pca_mode, p.pca_thr, None if ranks is None else int(ranks[j]))
        rows.append(r)
        Bs.append(Hj @ pc.V)
        pcas.append(pc)
    F = asm.rhs(p)
    offs = np.concatenate([[0], np.cumsum([B.shape[1] for B in Bs])]).astype(np.int64)
    return System(p, R, b, rows, Bs, pcas, F, offs)


# ------------------------------------------------------------------ Schwarz --

@dataclasses.dataclass
class Schwarz:
    kind: str                    # "as" | "sas" | "ras"
    sets: List[List[int]]        # extended set N(i) (subdomain indices)
    idx: List[np.ndarray]        # unknown indices selected by R_i
    D: List[np.ndarray]          # diagonal of D_i (ones for AS)
    qr: list                     # (V, beta, P) of A_i

    def apply(self, r: np.ndarray) -> np.ndarray:
        z = np.zeros_like(r)
        for i, ix in enumerate(self.idx):
            V, beta, P = self.qr[i]
            s = la.back_substitute(P, la.apply_qt(V, beta, r[ix]))
            z[ix] += self.D[i] * s
        return z

    def apply_t(self, r: np.ndarray) -> np.ndarray:
        """M^T r = sum_i R_i^T A_i^{-T} D_i R_i r (A_i symmetric: A_i^{-T} = A_i^{-1})."""
        z = np.zeros_like(r)
        for i, ix in enumerate(self.idx):
            V, beta, P = self.qr[i]
            z[ix] += la.back_substitute(P, la.apply_qt(V, beta, self.D[i] * r[ix]))
        return z


def extended_sets(S: System, overlap_level: int = 1) -> List[List[int]]:
    p = S.problem
    if overlap_level == 0:
        return [[i] for i in range(p.J)]
    rows = [set(r.tolist()) for r in S.rows]
    return [[k for k in range(p.J) if rows[i] & rows[k]] for i in range(p.J)]


def local_matrix(S: System, ks: List[int]) -> np.ndarray:
    """A_i = R_i H^T H R_i^T: the Gram matrix of the columns of H selected by R_i."""
    blocks = []
    for k in ks:
        blocks.append([])
        for l in ks:
            common, ik, il = np.intersect1d(S.rows[k], S.rows[l], return_indices=True)
            blocks[-1].append(S.B[k][ik].T @ S.B[l][il])
    return np.block(blocks)


def schwarz(S: System, kind: str = "as", overlap_level: int = 1) -> Schwarz:
    sets = extended_sets(S, overlap_level)
    idx = [np.concatenate([np.arange(S.offsets[k], S.offsets[k + 1]) for k in ks]) for ks in sets]
    count = np.zeros(S.dof)
    for ix in idx:
        count[ix] += 1.0
    D = []
    for i, ix in enumerate(idx):
        if kind == "as":
            D.append(np.ones(ix.shape[0]))
        elif kind == "sas":
            D.append(1.0 / count[ix])
        elif kind == "ras":
            own = np.zeros(ix.shape[0])
            own[(ix >= S.offsets[i]) & (ix < S.offsets[i + 1])] = 1.0
            D.append(own)
        else:
            raise ValueError(kind)
    qrs = [la.householder_qr(local_matrix(S, ks)) for ks in sets]
    return Schwarz(kind, sets, idx, D, qrs)


# -------------------------------------------------------------------- solve --

@dataclasses.dataclass
class Solution:
    W: np.ndarray
    iters: int
    history: list
    rel_res_normal: float     # ||H^T(F - H W)|| / ||H^T F||
    res_ls: float             # ||H W - F||


def solve(S: System, solver: str, precond: Optional[Schwarz], rtol=1e-10,
          restart=50, maxit=2000) -> Solution:
    bvec = S.HT(S.F)
    M = precond.apply if precond is not None else None
    if solver == "cg":
        W, it, hist = la.pcg(S.normal, bvec, M, rtol, maxit)
    elif solver == "gmres":
        W, it, hist = la.gmres(S.normal, bvec, M, rtol, restart, maxit)
    elif solver == "cgs":
        W, it, hist = la.cgs(S.normal, bvec, M, rtol, maxit)
    elif solver == "bicg":
        MT = precond.apply_t if precond is not None else None
        W, it, hist = la.bicg(S.normal, S.normal, bvec, M, MT, rtol, maxit)   # H^T H is symmetric
    else:
        raise ValueError(solver)
    res = S.F - S.H(W)
    return Solution(W, it, hist, np.linalg.norm(S.HT(res)) / np.linalg.norm(bvec),
                    np.linalg.norm(res))


def solve_qr(S: System) -> Solution:
    W = la.qr_lstsq(S.dense(), S.F)
    res = S.F - S.H(W)
    bvec = S.HT(S.F)
    return Solution(W, 0, [], np.linalg.norm(S.HT(res)) / np.linalg.norm(bvec),
                    np.linalg.norm(res))


# ---------------------------------------------------------- differentiation --

def grad_c0(S: System, W: np.ndarray, lam: np.ndarray) -> float:
    """dl/dc0 of a loss l(W) through W(c0) = argmin ||H W - F|| (Sec. 2 Eq.
    (system), normal equations), given lam = (H^T H)^{-1} dl/dW, for the
    operator -Lap u + c0 u.  Psi_j and hence the PCA basis V do not depend on
    c0; the reaction term adds c0 L omega_j phi_j to the entries of H_j
    (Sec. 2 Eq. (sum)) and -c0 G to F = f - A[G], so dH/dc0 = H_c with
    (H_c)_j = L Psi_j V_j and dF/dc0 = -G.  Differentiating
    H^T H W = H^T F gives, with r = F - H W,
        dl/dc0 = r . (H_c lam) + (H lam) . (-G) - (H lam) . (H_c W).
    """
    p = S.problem
    xs = asm._coords(ri.grid_points(p), -1)
    Lx = asm.constraint_L(p, xs).a
    Gx = asm.constraint_G(p, xs).a
    Psis = [asm.block(p, S.R, S.b, j)[1] for j in range(len(S.B))]

    def Hc(x: np.ndarray) -> np.ndarray:
        y = np.zeros(S.n_rows)
        for j, Psi in enumerate(Psis):
            np.add.at(y, S.rows[j], Psi @ (S.pcas[j].V @ x[S.offsets[j]:S.offsets[j + 1]]))
        return Lx * y

    r = S.F - S.H(W)
    Hl = S.H(lam)
    return float(r @ Hc(lam) - Hl @ Gx - Hl @ Hc(W))


def grad_coef(S: System, W: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """dl/da_c, c < g*g, of a loss l(W) through the least-squares solution W
    of -div(a grad u) = f with the piecewise coefficient a = sum_c a_c s_c
    (smoothed cell indicators s_c), given lam = (H^T H)^{-1} dl/dW.

    The operator is linear in a, so dH/da_c is the collocation matrix of
    -div(s_c grad .): the blocks H_j assembled with the coefficient values
    e_c (one-hot), times the same V_j (Psi_j, hence the PCA basis, does not
    depend on a); F = f - A[G] gives dF/da_c = -A_c[G], the right-hand side
    assembled with e_c and f = 0.  Differentiating H^T H W = H^T F, with
    r = F - H W and H_c = dH/da_c, F_c = dF/da_c:
        dl/da_c = r . (H_c lam) + (H lam) . (F_c - H_c W).
    """
    import dataclasses
    p = S.problem
    if p.op != ri.OP_DIFFUSION or p.coef != ri.COEF_PIECEWISE:
        raise ValueError("grad_coef: piecewise diffusion coefficient only")
    ncell = p.coef_grid * p.coef_grid
    r = S.F - S.H(W)
    Hl = S.H(lam)
    out = np.zeros(ncell)
    for c in range(ncell):
        e = np.zeros(ncell)
        e[c] = 1.0
        pc = dataclasses.replace(p, coef_vals=e, fc=None, fa=None, f0=0.0)
        Bc = [asm.block(pc, S.R, S.b, j)[2] @ S.pcas[j].V for j in range(len(S.B))]
        Sc = System(p, S.R, S.b, S.rows, Bc, S.pcas, asm.rhs(pc), S.offsets)
        out[c] = r @ Sc.H(lam) + Hl @ (Sc.F - Sc.H(W))
    return out


def eval_matrix_t(S: System, r: np.ndarray) -> np.ndarray:
    """E^T r, with u_hat = E W + G at the collocation points of S
    (Eq. (netdd), (pca_net)): block j of E is diag(L) Psi_j V_j on the rows
    of box_j, so (E^T r)_j = V_j^T Psi_j^T (L r)|_{rows_j}."""
    p = S.problem
    X = ri.grid_points(p)
    Lx = asm.constraint_L(p, asm._coords(X, -1)).a
    out = []
    for j in range(len(S.B)):
        _, Psi, _ = asm.block(p, S.R, S.b, j)
        out.append(S.pcas[j].V.T @ (Psi.T @ (Lx * r)[S.rows[j]]))
    return np.concatenate(out)


# --------------------------------------------------------------- evaluation --

def evaluate(S: System, W: np.ndarray, X: np.ndarray) -> np.ndarray:
    """u_hat(x) = L(x) sum_j omega_j(x) (V_{p_j}^T Phi_j(x)) . W_j + G(x)  (Eq. (netdd), (pca_net))."""
    p = S.problem
    xs = asm._coords(X, -1)
    Lx = asm.constraint_L(p, xs).a
    Gx = asm.constraint_G(p, xs).a
    mu, sig = asm.centres_halfwidths(p)
    total = np.zeros(X.shape[0])
    wsum = None
    what = [asm.window_hat(p, xs, k).a for k in range(p.J)]
    wsum = np.sum(what, axis=0)
    for j in range(p.J):
        wj = np.where(wsum > 0, what[j] / np.where(wsum > 0, wsum, 1.0), 0.0)
        sel = wj != 0.0
        if not np.any(sel):
            continue
        ks = asm.subdomain_multi_index(p, j)
        z = np.broadcast_to(S.b[j][None, :], (int(sel.sum()), S.b.shape[1])).copy()
        for i in range(p.dim):
            z += ((X[sel, i] - mu[i][ks[i]]) / sig[i])[:, None] * S.R[j][None, :, i]
        feat = np.tanh(z) @ S.pcas[j].V
        total[sel] += wj[sel] * (feat @ W[S.offsets[j]:S.offsets[j + 1]])
    return Lx * total + Gx


def errors(u_hat: np.ndarray, u: np.ndarray):
    """Relative L2 error (Sec. 5) and normalised L1 error mean|u_hat-u|/std(u) (Sec. 5)."""
    e2 = np.linalg.norm(u_hat - u) / np.linalg.norm(u)
    e1 = np.mean(np.abs(u_hat - u)) / np.std(u)
    return e2, e1
