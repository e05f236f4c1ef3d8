"""GPU parity at the configured full sizes, against the oracle.

The small variants of the other parity tests run the eigensolver's smallest
template (m <= 64) and single tiles of the tensor-core products.  Here the
GPU runs the full-size workloads (m = 300 and 400, blocks of 3136 .. 5808
rows: the m = 300 and m = 400 eigensolver templates and many 128 x 64 tiles
of the digit-slice Gram and projection products), and the oracle computes the
blocks the checks need (in worker processes; it is seconds per block).

  * assembly (Sec. 2 Eq. (sum), Sec. 4): Psi_j and H_j entrywise within
    1e-12 of the block's largest entry;
  * PCA (Sec. 4 Eq. (pca)): the oracle's ranks unless it flags a singular
    value at the cut; eigenvalues sigma_k^2 within 64 m eps lambda_max (the
    backward error of the Gram eigen-decomposition); the kept basis
    orthonormal, Eckart-Young optimal (||Psi - Psi V V^T||_F^2 equals the
    oracle's discarded sum_{k>p} sigma_k^2 up to that backward error), and
    equal to the oracle's singular vectors up to sign where the eigenvalue
    gap exceeds 1e-6 lambda_max (angle bound m eps lambda_max / gap);
  * projection (Eq. (system_new)): B_j against the float64 host product
    H_j V_{p_j} of the oracle's H_j and the GPU's basis, entrywise within
    4 m eps max|H_i.| max|V_.k| plus the 1e-12 of the assembly;
  * one local solve A_i^{-1} r of the Schwarz preconditioner (Sec. 3) at
    m = 300, against the oracle's Householder QR of the same A_i, to the
    factor accuracy kappa(A_i) u (u = 2^-53 for float64 factors, 2^-48 for
    double-float ones), with kappa(A_i) measured;
  * the full multiscale workload solved end to end (SAS-GMRES(50) and
    AS-CG) against the oracle's own Krylov solve at the GPU's ranks: the
    least-squares residuals agree to 1e-8 ||F||, and the u_hat difference is
    printed with the condition estimate and held to 1e-6 (see the test).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

import rann_inputs as ri
from oracle import assembly as asm
from oracle import linalg as la
from oracle import solver as sv

from oracle_pool import hood, householder_qrs, oracle_blocks

EPS = 2.0 ** -52
# blocks checked per workload: the 3x3 neighbourhood of an interior
# subdomain (m = 300), and boundary and interior subdomains (m = 400)
BLOCKS = {
    "multiscale2d": lambda p: hood(p, (4, 4)),
    "poisson3d": lambda p: [0, 21, 42, 63],
    "heat3d": lambda p: [0, 4 + 8 * 4 + 64 * 2, 255],
}


@pytest.fixture(scope="module")
def g():
    from paper_2412_19207_gb300 import build
    build.build()
    import paper_2412_19207_gb300 as pkg
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    return pkg


_handles = {}


def reduced(g, name):
    """Full-size GPU handle after assemble / rhs / pca (precision mode 1)."""
    if name not in _handles:
        p = ri.config(name)
        R, b = ri.weights(p)
        s = g.RannDD(p, R, b)
        s.assemble()
        F = s.rhs()
        ranks = s.pca(p.pca_mode, p.pca_thr)
        _handles[name] = (p, s, F, ranks)
    return _handles[name]


@pytest.mark.parametrize("name", list(BLOCKS))
def test_fullsize_assembly_pca_projection(g, name):
    p, s, F, ranks = reduced(g, name)
    js = BLOCKS[name](p)
    ob = oracle_blocks(name, js, want_dense=True)
    m = p.neurons
    for j in js:
        o = ob[j]
        rows, Psi = s.block(j, 0)
        _, H = s.block(j, 1)
        np.testing.assert_array_equal(rows, o["rows"])
        np.testing.assert_allclose(Psi, o["Psi"], rtol=0, atol=1e-12 * np.abs(o["Psi"]).max())
        np.testing.assert_allclose(H, o["H"], rtol=0, atol=1e-12 * np.abs(o["H"]).max())
        if not o["borderline"]:
            assert ranks[j] == o["rank"], (j, ranks[j], o["rank"])
        eig, V = s.pca_of(j)
        lam = np.zeros(m)
        lam[: o["sigma"].shape[0]] = o["sigma"] ** 2
        tol = 64 * m * EPS * lam[0]
        np.testing.assert_allclose(eig, lam, rtol=0, atol=tol)
        np.testing.assert_allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-11)
        resid = np.linalg.norm(o["Psi"] - (o["Psi"] @ V) @ V.T) ** 2
        tail = float(np.sum(o["sigma"][ranks[j]:] ** 2))
        assert abs(resid - tail) <= 1e-8 * tail + 256 * m * EPS * lam[0], (j, resid, tail)
        # leading vectors with a clear eigenvalue gap: the oracle's up to sign
        Vo = o["V"]
        for k in range(min(ranks[j], o["rank"])):
            gap = min(abs(lam[k] - lam[i]) for i in range(m) if i != k)
            if gap > 1e-6 * lam[0]:
                assert abs(abs(V[:, k] @ Vo[:, k]) - 1.0) <= 1e-8, (j, k)
        # projection: B_j = H_j V_{p_j}
        _, B = s.block(j, 2)
        ref = o["H"] @ V
        bound = (4 * m * EPS * np.abs(o["H"]).max(axis=1)[:, None] * np.abs(V).max(axis=0)[None, :]
                 + 1e-12 * np.abs(o["H"]).max() * np.abs(V).sum(axis=0)[None, :])
        err = np.abs(B - ref)
        assert np.all(err <= bound), (j, float((err / bound).max()))


def _gpu_reduced_system(p, s, ranks, F):
    """The oracle's System on the GPU's own reduced blocks (kernel-level checks)."""
    rows, Bs = [], []
    for j in range(p.J):
        r, B = s.block(j, 2)
        rows.append(r)
        Bs.append(B)
    offs = np.concatenate([[0], np.cumsum(ranks)]).astype(np.int64)
    pcas = [sv.PCA(np.zeros(1), np.zeros((p.neurons, int(ranks[j]))), int(ranks[j]), False) for j in range(p.J)]
    R, b = ri.weights(p)
    return sv.System(p, R, b, rows, Bs, pcas, F.cpu().numpy(), offs)


@pytest.mark.parametrize("mode,kind", [(1, "as"), (0, "as"), (1, "ras")])
def test_fullsize_local_solve(g, mode, kind):
    """r on the unknowns of one interior subdomain k: M^{-1} r sums
    R_i^T D_i A_i^{-1} R_i r over the extended sets holding k (nine of them);
    the oracle forms those A_i from the same reduced blocks and solves them by
    Householder QR."""
    name = "multiscale2d"
    p = ri.config(name)
    R, b = ri.weights(p)
    s = g.RannDD(p, R, b)
    s.set_precision(mode)
    s.assemble()
    F = s.rhs()
    ranks = s.pca(p.pca_mode, p.pca_thr)
    S = _gpu_reduced_system(p, s, ranks, F)
    s.setup_precond(kind)
    k = 4 * 8 + 4
    r = np.zeros(S.dof)
    r[S.offsets[k]:S.offsets[k + 1]] = np.random.default_rng(3).standard_normal(int(ranks[k]))
    z = s.precond_apply(torch.tensor(r, device="cuda")).cpu().numpy()
    sets = sv.extended_sets(S)
    holders = [i for i in range(p.J) if k in sets[i]]
    assert len(holders) == 9
    mats = [sv.local_matrix(S, sets[i]) for i in holders]
    qrs = householder_qrs(mats)
    zo = np.zeros(S.dof)
    kappa = 0.0
    for i, A, (Vq, bq, P) in zip(holders, mats, qrs):
        ix = np.concatenate([np.arange(S.offsets[q], S.offsets[q + 1]) for q in sets[i]])
        si = la.back_substitute(P, la.apply_qt(Vq, bq, r[ix]))
        if kind == "ras":
            own = (ix >= S.offsets[i]) & (ix < S.offsets[i + 1])
            si = np.where(own, si, 0.0)
        zo[ix] += si
        w = np.linalg.eigvalsh(A)
        kappa = max(kappa, w[-1] / w[0])
    u = 2.0 ** -53 if mode == 0 else 2.0 ** -48
    err = np.linalg.norm(z - zo) / np.linalg.norm(zo)
    print(f"\n{name} {kind} mode {mode}: ||z - z_oracle|| / ||z_oracle|| = {err:.3e}, "
          f"max kappa(A_i) = {kappa:.3e}, kappa u = {kappa * u:.3e}")
    assert err <= max(1e-12, kappa * u)
    s.close()


def test_fullsize_multiscale_solve(g):
    """Sec. 5: the full multiscale workload (DoF ~ 6300, 102400 collocation
    points), GPU against the oracle's own AS-CG solve (float64 assembly,
    Jacobi-SVD PCA at the GPU's ranks, Householder-QR local solves).  The two
    reduced bases differ at rounding level (Gram eigen-decomposition against
    Jacobi SVD), so the solutions are compared as functions: the collocated
    residuals H W - F (each side's own H) and u_hat at 101^2 test points.
    The least-squares residual norms agree to 1e-8 ||F|| (both minimise it
    to second order in their normal residuals); the u_hat difference has no
    a-priori bound here (sigma_min of the 102400 x 6300 H is beyond the
    oracle), so it is printed with the GPU's condition estimate and held to
    1e-6, ten times the difference that the small multiscale problem shows
    between the exact solutions of the two bases (7.9e-7)."""
    name = "multiscale2d"
    p, s, F, ranks = reduced(g, name)
    R, b = ri.weights(p)
    ob = oracle_blocks(name, range(p.J), ranks=ranks)
    So = sv.System(p, R, b, [ob[j]["rows"] for j in range(p.J)], [ob[j]["B"] for j in range(p.J)],
                   [sv.PCA(ob[j]["sigma"], ob[j]["V"], ob[j]["rank"], ob[j]["borderline"]) for j in range(p.J)],
                   asm.rhs(p), np.concatenate([[0], np.cumsum(ranks)]).astype(np.int64))
    np.testing.assert_allclose(F.cpu().numpy(), So.F, rtol=0, atol=1e-13 * np.abs(So.F).max())
    sets = sv.extended_sets(So)
    mats = [sv.local_matrix(So, ks) for ks in sets]
    qrs = householder_qrs(mats)
    idx = [np.concatenate([np.arange(So.offsets[k], So.offsets[k + 1]) for k in ks]) for ks in sets]
    M = sv.Schwarz("as", sets, idx, [np.ones(ix.shape[0]) for ix in idx], qrs)
    sol = sv.solve(So, "cg", M, 1e-10, 50, 3000)
    X = ri.test_points(p, 101)
    uo = sv.evaluate(So, sol.W, X)
    Fn = np.linalg.norm(So.F)
    fo = So.H(sol.W)
    for kind, solver in (("sas", "gmres"), ("as", "cg")):
        s.setup_precond(kind)
        if solver == "gmres":
            W, st = s.solve_gmres_ras(F, 1e-10, 50, 3000)
        else:
            W, st = s.solve_cg_as(F, 1e-10, 3000)
        fg = s.matvec(W).cpu().numpy()
        res_g = np.linalg.norm(fg - So.F)
        ug = s.eval(W, torch.tensor(X, device="cuda")).cpu().numpy()
        du = np.linalg.norm(ug - uo) / np.linalg.norm(uo)
        print(f"\n{name} {kind}-{solver}: GPU iters {st['iters']} (normal residual {st['rel_res_true']:.2e}, "
              f"kappa_est(M^-1 A) {st['kappa_est']:.3e}), oracle AS-CG iters {sol.iters} (normal residual "
              f"{sol.rel_res_normal:.2e}); ||HW-F|| GPU {res_g:.9e} oracle {sol.res_ls:.9e}; "
              f"||H_g W_g - H_o W_o|| / ||F|| = {np.linalg.norm(fg - fo) / Fn:.3e}; u_hat difference {du:.3e}")
        assert abs(res_g - sol.res_ls) <= 1e-8 * Fn
        assert du <= 1e-6
