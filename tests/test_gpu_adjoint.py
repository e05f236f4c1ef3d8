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


# ---- the piecewise diffusion coefficient (gradients w.r.t. a_c) ----

def _piecewise(g, g_kind=None, sub=None, mode=0, kind="as"):
    import dataclasses
    p = ri.config("piecewise2d", small=True) if sub is None else ri.piecewise2d(0, sub=sub, pts=8, neurons=20)
    if g_kind is not None:
        p = dataclasses.replace(p, g_kind=g_kind)
    R, b = ri.weights(p)
    s = g.RannDD(p, R, b)
    s.set_precision(mode)
    s.assemble()
    F = s.rhs()
    ranks = s.pca(p.pca_mode, p.pca_thr)
    s.setup_precond(kind)
    return p, R, b, s, F, ranks


def _oracle_on_gpu_basis(p, R, b, s, ranks):
    """The oracle's system with the oracle's blocks projected on the GPU's basis."""
    from oracle import assembly as asm
    from oracle import solver as sv
    rows, Bs, pcas = [], [], []
    for j in range(p.J):
        r, _, H = asm.block(p, R, b, j)
        V = s.pca_of(j)[1]
        rows.append(r)
        Bs.append(H @ V)
        pcas.append(sv.PCA(np.zeros(1), V, int(ranks[j]), False))
    offs = np.concatenate([[0], np.cumsum(ranks)]).astype(np.int64)
    return sv.System(p, R, b, rows, Bs, pcas, asm.rhs(p), offs)


@pytest.mark.parametrize("g_kind", [ri.G_ZERO, ri.G_SINPROD])
def test_grad_coef_matches_the_oracle(g, g_kind):
    """rann_dd_grad_coef against the oracle's grad_coef (one-hot hyper-dual
    assembly of dH/da_c) at the same W, lam and basis; with G = sin sin the
    dF/da_c = -A_c[G] term is exercised too.  The formula is an identity in
    W and lam, so the solves need not be converged far."""
    from oracle import solver as sv
    p, R, b, s, F, ranks = _piecewise(g, g_kind, mode=1, kind="ras")
    W, _ = s.solve_gmres_ras(F, 1e-10, 50, 3000, allow_not_converged=True)
    v = torch.tensor(np.random.default_rng(4).standard_normal(F.numel()), device="cuda")
    lam, _ = s.solve_backward(s.eval_grid_t(v), 1e-10, 3000, allow_not_converged=True)
    got = s.grad_coef(F, W, lam)
    So = _oracle_on_gpu_basis(p, R, b, s, ranks)
    want = sv.grad_coef(So, W.cpu().numpy(), lam.cpu().numpy())
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-9 * np.abs(want).max())


def test_grad_coef_against_central_differences(g):
    """dl/da_c of l = v . u_hat(a) on the collocation grid (a linear functional
    of the solution, well determined where W itself is not) against central
    differences of the GPU solves (2 x 2 subdomains: the AS solve is exact in
    one step; float64 mode); dl/dW = E^T v through rann_dd_eval_grid_t."""
    p, R, b, s, F, ranks = _piecewise(g, sub=2)
    v = torch.tensor(np.random.default_rng(6).standard_normal(F.numel()), device="cuda")
    X = s.points()
    W, _ = s.solve_cg_as(F, 1e-10, 100, allow_not_converged=True)
    lam, _ = s.solve_backward(s.eval_grid_t(v), 1e-10, 100, allow_not_converged=True)
    grad = s.grad_coef(F, W, lam)
    a0 = p.coef_vals.copy()
    h = 1e-5

    def loss(vals):
        s.set_coef(vals)
        s.assemble()
        Fv = s.rhs()
        s.pca(p.pca_mode, p.pca_thr)
        s.setup_precond("as")
        Wv, _ = s.solve_cg_as(Fv, 1e-10, 100, allow_not_converged=True)
        return float(v @ s.eval(Wv, X))

    for cell in (0, 6, 15):
        e = np.zeros_like(a0)
        e[cell] = h
        fd = (loss(a0 + e) - loss(a0 - e)) / (2 * h)
        assert abs(grad[cell] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(grad).max()), (cell, grad[cell], fd)


def test_eval_grid_transpose_matches_the_oracle(g):
    from oracle import solver as sv
    p = ri.config("heat3d", small=True)
    R, b = ri.weights(p)
    s = g.RannDD(p, R, b)
    s.assemble()
    ranks = s.pca(p.pca_mode, p.pca_thr)
    So = _oracle_on_gpu_basis(p, R, b, s, ranks)
    r = np.random.default_rng(3).standard_normal(p.n_points())
    got = s.eval_grid_t(torch.tensor(r, device="cuda")).cpu().numpy()
    want = sv.eval_matrix_t(So, r)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())
    # adjoint identity with the forward evaluation at the grid
    w = torch.tensor(np.random.default_rng(4).standard_normal(int(ranks.sum())), device="cuda")
    X = s.points()
    u = s.eval(w, X) - s.eval(torch.zeros_like(w), X)
    assert abs(float(u @ torch.tensor(r, device="cuda")) - float(w @ torch.tensor(got, device="cuda"))) <= \
        1e-11 * float(u.norm() * np.linalg.norm(r))


def test_misfit_gradients_through_autograd(g):
    """l = ||u_hat(a, F) - u_obs||^2 on the collocation grid, through
    PiecewiseDiffusionSolve and GridEval: dl/da_c against central differences
    and dl/dF along a direction against a central difference (RAS-GMRES
    forward and adjoint, as the piecewise workload runs)."""
    p, R, b, s, F, ranks = _piecewise(g, sub=2, kind="ras")
    a = torch.tensor(p.coef_vals, dtype=torch.float64, requires_grad=True)
    Fv = F.clone().requires_grad_(True)
    u_obs = torch.tensor(np.random.default_rng(2).standard_normal(F.numel()) * 0.01, device="cuda")

    def misfit(av, Fin):
        W = g.PiecewiseDiffusionSolve.apply(s, av, Fin, kind="ras", rtol=1e-13, maxit=200)
        u = g.GridEval.apply(s, W)
        return ((u - u_obs) ** 2).sum()

    l = misfit(a, Fv)
    l.backward()
    ga, gF = a.grad.numpy().copy(), Fv.grad.clone()
    with torch.no_grad():
        h = 1e-5
        for cell in (3, 9):
            e = torch.zeros_like(a)
            e[cell] = h
            fd = (float(misfit(a + e, F)) - float(misfit(a - e, F))) / (2 * h)
            assert abs(ga[cell] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(ga).max()), (cell, ga[cell], fd)
        dF = torch.tensor(np.random.default_rng(9).standard_normal(F.numel()), device="cuda")
        hF = 1e-4
        fd = (float(misfit(a, F + hF * dF)) - float(misfit(a, F - hF * dF))) / (2 * hF)
        assert abs(float(gF @ dF) - fd) <= 1e-5 * abs(fd)
