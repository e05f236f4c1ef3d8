"""The adjoint solve (rann_dd_solve_backward) and the differentiable solve.

W(F) = (H^T H)^{-1} H^T F = H^+ F, so H W(F) = P F with P the orthogonal
projector onto range(H).  For a loss on W the sensitivity to F is
dl/dF = H lam with (H^T H) lam = dl/dW.  The tests use losses whose
gradient is consistent with the least-squares structure (dl/dW in
range(H^T)), for which closed forms exist:
  * l = 1/2 ||H W - y||^2:  dl/dF = P (P F - y) = H W(F) - H W(y);
  * l = c . W with c = H^T v:  dl/dF = P v = H W(v);
and, l being quadratic in F, central differences equal the directional
derivative up to the solve tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import rann_inputs as ri


@pytest.fixture(scope="module")
def g():
    from paper_2412_19207_gb300 import build
    build.build()
    import paper_2412_19207_gb300 as pkg
    return pkg


def prepared(g, name, kind, mode=1):
    p = ri.config(name, small=True)
    s = g.RannDD(p)
    s.set_precision(mode)
    s.assemble()
    F = s.rhs()
    ranks = s.pca(p.pca_mode, p.pca_thr)
    s.setup_precond(kind)
    return p, s, F, ranks


CASES = [("heat3d", "as"), ("multiscale2d", "sas"), ("poisson3d", "as"), ("piecewise2d", "ras")]


@pytest.mark.parametrize("name,kind", CASES)
def test_adjoint_of_residual_loss_matches_closed_form_and_differences(g, name, kind):
    p, s, F, ranks = prepared(g, name, kind)
    y = torch.tensor(np.random.default_rng(1).standard_normal(F.numel()), device="cuda")

    def loss_of(Fv):
        W, st = s.solve(Fv, 1e-12, 5000)
        return 0.5 * float(((s.matvec(W) - y) ** 2).sum()), W

    l0, W = loss_of(F)
    gW = s.matvec_t(s.matvec(W) - y)                       # dl/dW = H^T (H W - y)
    lam, st = s.solve_backward(gW, 1e-12, 5000)
    assert st["status"] == "RANN_OK"
    dF = s.matvec(lam)
    Wy, _ = s.solve(y, 1e-12, 5000)
    closed = s.matvec(W) - s.matvec(Wy)                    # P F - P y
    assert float((dF - closed).norm()) <= 1e-7 * float(closed.norm())
    rng = np.random.default_rng(2)
    for _ in range(2):
        d = torch.tensor(rng.standard_normal(F.numel()), device="cuda")
        h = 1e-3 * float(F.norm()) / float(d.norm())
        fd = (loss_of(F + h * d)[0] - loss_of(F - h * d)[0]) / (2 * h)
        an = float((dF * d).sum())
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-9 * float(dF.norm() * d.norm())


@pytest.mark.parametrize("name,kind", CASES[:2])
def test_autograd_gradient_is_the_projected_direction(g, name, kind):
    p, s, F, ranks = prepared(g, name, kind)
    v = torch.tensor(np.random.default_rng(4).standard_normal(F.numel()), device="cuda")
    c = s.matvec_t(v)                                      # c = H^T v
    Fv = F.clone().requires_grad_(True)
    W = g.LeastSquaresSolve.apply(s, Fv, 1e-12, 5000)
    (W * c).sum().backward()
    Wv, _ = s.solve(v, 1e-12, 5000)
    expect = s.matvec(Wv)                                  # P v
    assert float((Fv.grad - expect).norm()) <= 1e-7 * float(expect.norm())


def test_adjoint_matches_dense_float64(g):
    p, s, F, ranks = prepared(g, "heat3d", "as", mode=0)
    blocks = [s.block(j, 2) for j in range(p.J)]
    offs = np.concatenate([[0], np.cumsum(ranks)])
    H = np.zeros((p.n_points(), int(offs[-1])))
    for j, (rows, B) in enumerate(blocks):
        H[rows, offs[j]:offs[j + 1]] = B
    gW = H.T @ np.random.default_rng(3).standard_normal(H.shape[0])
    lam, st = s.solve_backward(torch.tensor(gW, device="cuda"), 1e-12, 5000)
    dF = s.matvec(lam).cpu().numpy()
    dF_dense = H @ np.linalg.solve(H.T @ H, gW)
    assert np.linalg.norm(dF - dF_dense) <= 1e-7 * np.linalg.norm(dF_dense)


def test_backward_needs_a_preconditioner(g):
    p = ri.config("poisson2d_2x2", small=True)
    s = g.RannDD(p)
    s.assemble()
    s.pca(p.pca_mode, p.pca_thr)
    z = torch.zeros(int(s.sizes()["dof"]), dtype=torch.float64, device="cuda")
    with pytest.raises(g.RannError) as e:
        s.solve_backward(z)
    assert e.value.status == g.EORDER


# ---- derivative with respect to the reaction coefficient c0 (rann_dd_grad_c0) ----

def _poisson_c0(g, c0, mode, rtol):
    import dataclasses
    p = dataclasses.replace(ri.config("poisson2d_2x2", small=True), c0=c0, g_kind=ri.G_SINPROD)
    s = g.RannDD(p)
    s.set_precision(mode)
    s.assemble()
    F = s.rhs()
    s.pca(p.pca_mode, p.pca_thr)
    s.setup_precond("as")
    W, st = s.solve_cg_as(F, rtol, 200)
    assert st["status"] == "RANN_OK"
    return p, s, F, W


def test_grad_c0_matches_central_differences(g):
    """l = c . W(c0), c = H^T v, in float64 (precision mode 0): on the 2x2 layout AS-CG
    solves to rounding in a step or two, so central differences of the GPU
    solves resolve dl/dc0 (the PCA basis does not depend on c0)."""
    p, s, F, W = _poisson_c0(g, 0.7, 0, 1e-12)
    v = torch.tensor(np.random.default_rng(21).standard_normal(F.numel()), device="cuda")
    c = s.matvec_t(v)                                      # dl/dW in range(H^T), as above
    lam, st = s.solve_backward(c, 1e-12, 200)
    grad = s.grad_c0(F, W, lam)
    h = 1e-4
    lp = float((c * _poisson_c0(g, 0.7 + h, 0, 1e-12)[3]).sum())
    lm = float((c * _poisson_c0(g, 0.7 - h, 0, 1e-12)[3]).sum())
    fd = (lp - lm) / (2 * h)
    assert abs(grad - fd) <= 1e-4 * abs(fd), (grad, fd)


def test_grad_c0_matches_the_oracle_formula(g):
    """The same formula in the oracle (dense blocks, L Psi V from the oracle's
    assembly) at the GPU's W, lam and PCA basis."""
    from oracle import assembly as asm
    from oracle import solver as sv
    p, s, F, W = _poisson_c0(g, 0.4, 1, 1e-9)
    v = torch.tensor(np.random.default_rng(22).standard_normal(F.numel()), device="cuda")
    c = s.matvec_t(v)
    lam, st = s.solve_backward(c, 1e-9, 200)
    grad = s.grad_c0(F, W, lam)
    R, b = ri.weights(p)
    rows, Bs, pcas = [], [], []
    for j in range(p.J):
        r, Psi, Hj = asm.block(p, R, b, j)
        eig, V = s.pca_of(j)
        rows.append(r)
        Bs.append(Hj @ V)
        pcas.append(sv.PCA(np.sqrt(np.maximum(eig, 0.0)), V, V.shape[1], False))
    offs = np.concatenate([[0], np.cumsum([B.shape[1] for B in Bs])]).astype(np.int64)
    Sg = sv.System(p, R, b, rows, Bs, pcas, asm.rhs(p), offs)
    expect = sv.grad_c0(Sg, W.cpu().numpy(), lam.cpu().numpy())
    assert abs(grad - expect) <= 1e-7 * abs(expect), (grad, expect)


def test_grad_c0_needs_the_poisson_operator(g):
    p = ri.config("multiscale2d", small=True)
    s = g.RannDD(p)
    s.assemble()
    F = s.rhs()
    s.pca(p.pca_mode, p.pca_thr)
    W = torch.zeros(int(s.sizes()["dof"]), dtype=torch.float64, device="cuda")
    with pytest.raises(g.RannError) as e:
        s.grad_c0(F, W, W)
    assert e.value.status == g.EINVAL
