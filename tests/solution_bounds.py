"""Parity of an iterative GPU solution with the oracle's direct solution, to the
bound its own float64 normal residual allows.

For the reduced least-squares problem min ||H W - F|| (Sec. 2 Eq. (system),
Sec. 4 Eq. (system_new)) with exact solution W*, every W with normal residual
r_n = H^T (F - H W) satisfies H^T H (W* - W) = r_n, hence
    ||H (W - W*)|| <= ||r_n|| / sigma_min(H),
    ||W - W*||     <= ||r_n|| / sigma_min(H)^2,
and u_hat at test points, u_hat = E W + G, moves by at most ||E|| ||W - W*||.
The checks below form H from the GPU's own reduced blocks (so the basis is
the GPU's), W* by the oracle's Householder-QR least squares, sigma_min(H) and
||E|| as measuring instruments by numpy's SVD (a DoF-wide one-sided Jacobi
in numpy takes minutes), and r_n in float64 on the host from the returned
W: a kernel error that the normal residual does not show (a wrong operator,
a wrong right-hand side, a wrong evaluation) breaks them.
"""
from __future__ import annotations

import numpy as np

import rann_inputs as ri
from oracle import linalg as la
from oracle import solver as sv


class GpuReduced:
    """The GPU's reduced blocks and basis as an oracle System, with the
    oracle's direct solve on it (cached per right-hand side scale)."""

    def __init__(self, p, s, ranks, F):
        R, b = ri.weights(p)
        rows, Bs = [], []
        for j in range(p.J):
            r, B = s.block(j, 2)
            rows.append(r)
            Bs.append(B)
        offs = np.concatenate([[0], np.cumsum(ranks)]).astype(np.int64)
        pcas = [sv.PCA(np.zeros(1), s.pca_of(j)[1], int(ranks[j]), False) for j in range(p.J)]
        Fn = F.cpu().numpy() if hasattr(F, "cpu") else np.asarray(F)
        self.S = sv.System(p, R, b, rows, Bs, pcas, Fn, offs)
        self.H = self.S.dense()
        self.W_star = la.qr_lstsq(self.H, Fn)
        sg = np.linalg.svd(self.H, compute_uv=False)
        self.smax, self.smin = sg[0], sg[-1]
        self._E = {}

    def eval_matrix(self, X):
        key = X.tobytes()
        if key not in self._E:
            g0 = sv.evaluate(self.S, np.zeros(self.S.dof), X)
            E = np.empty((X.shape[0], self.S.dof))
            for c in range(self.S.dof):
                e = np.zeros(self.S.dof)
                e[c] = 1.0
                E[:, c] = sv.evaluate(self.S, e, X) - g0
            self._E[key] = (E, g0, np.linalg.svd(E, compute_uv=False)[0])
        return self._E[key]

    def check(self, W, X=None, u=None, scale=1.0):
        """Asserts the bounds for a solution W of H W ~ scale * F (and its
        u_hat u at X, if given); returns the measured ratios."""
        W = W.cpu().numpy() if hasattr(W, "cpu") else np.asarray(W)
        F = scale * self.S.F
        Ws = scale * self.W_star
        rn = np.linalg.norm(self.H.T @ (F - self.H @ W))
        fit = np.linalg.norm(self.H @ (W - Ws))
        bound = rn / self.smin
        slack = 1e-13 * max(np.linalg.norm(F), 1e-300)
        assert fit <= bound * (1 + 1e-6) + slack, (fit, bound)
        out = {"fit": fit, "fit_bound": bound, "kappa_HtH": (self.smax / self.smin) ** 2}
        if X is not None and u is not None:
            E, g0, nE = self.eval_matrix(X)
            u = u.cpu().numpy() if hasattr(u, "cpu") else np.asarray(u)
            u_star = E @ Ws + g0
            du = np.linalg.norm(u - u_star)
            ub = nE * rn / self.smin ** 2
            assert du <= ub * (1 + 1e-6) + 1e-12 * max(np.linalg.norm(u_star), 1e-300), (du, ub)
            out.update({"du": du / max(np.linalg.norm(u_star), 1e-300),
                        "du_bound": ub / max(np.linalg.norm(u_star), 1e-300)})
        return out
