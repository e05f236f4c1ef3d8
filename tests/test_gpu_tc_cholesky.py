"""The big-panel local factorisation with tensor-core updates (precision mode 1,
local matrices of 512 unknowns and more: the extended sets of a 2 x 2 x 2
space-time grid with 240 neurons hold about 1300 unknowns, so the
factorisation runs five 256-column panels, the lower-triangle trailing
updates, and the inverse's two products per panel).

Checked against the float64 factors of precision mode 0 on the same reduced
system and against the oracle's Householder QR of the same A_i (Sec. 3: the
local inverses A_i^{-1} = P_i^{-1} Q_i^T): M^{-1} r to the double-float
factor accuracy kappa(A_i) 2^-48 (kappa measured); and the AS-CG solve that
uses them reaches rtol with the fitted values inside the bound its normal
residual allows.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import rann_inputs as ri
from oracle import solver as sv

from solution_bounds import GpuReduced


@pytest.fixture(scope="module")
def g():
    from paper_2412_19207_gb300 import build
    build.build()
    import paper_2412_19207_gb300 as pkg
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    return pkg


def problem():
    return ri.heat3d(sub=(2, 2, 2), pts=(7, 7, 5), neurons=240)


@pytest.fixture(scope="module")
def reduced(g):
    p = problem()
    R, b = ri.weights(p)
    s = g.RannDD(p, R, b)
    s.assemble()
    F = s.rhs()
    ranks = s.pca(p.pca_mode, p.pca_thr)
    assert int(ranks.sum()) >= 1024, "the local matrices must take the big-panel path"
    return p, R, b, s, F, ranks


def test_tensor_core_factors_match_the_oracle_and_float64(g, reduced):
    p, R, b, s, F, ranks = reduced
    gr = GpuReduced(p, s, ranks, F)
    M = sv.schwarz(gr.S, "as")
    A = sv.local_matrix(gr.S, M.sets[0])
    w = np.linalg.eigvalsh(A)
    kappa = w[-1] / w[0]
    rng = np.random.default_rng(3)
    out = {}
    for mode in (1, 0):
        s.set_precision(mode)
        status = s.setup_precond("as")
        for k in range(2):
            r = rng.standard_normal(gr.S.dof) if mode == 1 else out[(1, k)][0]
            z = s.precond_apply(torch.tensor(r, device="cuda")).cpu().numpy()
            out[(mode, k)] = (r, z, status)
    for k in range(2):
        r, z1, st1 = out[(1, k)]
        _, z0, st0 = out[(0, k)]
        zo = M.apply(r)
        e1 = np.linalg.norm(z1 - zo) / np.linalg.norm(zo)
        e0 = np.linalg.norm(z0 - zo) / np.linalg.norm(zo)
        print(f"\nkappa(A_i) {kappa:.3e}: ||z - z_oracle|| / ||z_oracle||: tensor-core double-float {e1:.3e}, "
              f"float64 {e0:.3e}; set-up statuses {st1}, {st0}")
        if st1 == g.OK and st0 == g.OK:
            assert e1 <= max(1e-12, kappa * 2.0 ** -48)
            assert e0 <= max(1e-12, kappa * 2.0 ** -53 * 8)


def test_tensor_core_factors_solve(g, reduced):
    p, R, b, s, F, ranks = reduced
    s.set_precision(1)
    s.setup_precond("as")
    W, st = s.solve_cg_as(F, 1e-10, 3000)
    assert st["status"] == "RANN_OK" and st["rel_res_true"] <= 1e-10
    X = ri.test_points(p, 7)
    u = s.eval(W, torch.tensor(X, device="cuda")).cpu().numpy()
    GpuReduced(p, s, ranks, F).check(W, X, u)
    # two set-ups give the same factors (fixed-order sums everywhere)
    z1 = s.precond_apply(torch.ones(int(ranks.sum()), dtype=torch.float64, device="cuda"))
    s.setup_precond("as")
    z2 = s.precond_apply(torch.ones(int(ranks.sum()), dtype=torch.float64, device="cuda"))
    assert torch.equal(z1, z2)


def test_factors_and_apply_on_sets_beyond_two_thousand_unknowns(g):
    """A larger local matrix: on a 2 x 2 x 2 Poisson grid with 600 neurons
    every extended set holds all subdomains (over 2048 unknowns, nine
    panels): M^{-1} r = 8 A^{-1} r.  The double-float apply (tensor-core
    factors) is held to the float64 one (float64 factors, triangular
    products) and to a direct float64 solve of A within kappa(A) 2^-48; two
    applies are identical."""
    p = ri.poisson3d(sub=2, pts=14, neurons=600)
    s = g.RannDD(p, *ri.weights(p))
    s.assemble()
    F = s.rhs()
    ranks = s.pca(p.pca_mode, p.pca_thr)
    n = int(ranks.sum())
    assert n > 2048, n
    rows, Bs = [], []
    for j in range(p.J):
        r, B = s.block(j, 2)
        rows.append(r)
        Bs.append(B)
    offs = np.concatenate([[0], np.cumsum(ranks)]).astype(np.int64)
    pcas = [sv.PCA(np.zeros(1), np.zeros((p.neurons, int(ranks[j]))), int(ranks[j]), False) for j in range(p.J)]
    S = sv.System(p, *ri.weights(p), rows, Bs, pcas, F.cpu().numpy(), offs)
    A = sv.local_matrix(S, list(range(p.J)))
    w = np.linalg.eigvalsh(A)
    kappa = w[-1] / w[0]
    r = np.random.default_rng(8).standard_normal(n)
    zref = 8.0 * np.linalg.solve(A, r)              # a float64 measuring instrument
    out = {}
    for mode in (1, 0):
        s.set_precision(mode)
        s.setup_precond("as")
        rd = torch.tensor(r, device="cuda")
        out[mode] = s.precond_apply(rd).cpu().numpy()
        if mode == 1:
            assert np.array_equal(out[1], s.precond_apply(rd).cpu().numpy())
    e1 = np.linalg.norm(out[1] - zref) / np.linalg.norm(zref)
    e0 = np.linalg.norm(out[0] - zref) / np.linalg.norm(zref)
    print(f"\nn = {n}, kappa(A) {kappa:.3e}: double-float (tensor-core factors) {e1:.3e}, "
          f"float64 {e0:.3e}")
    assert e1 <= max(1e-12, kappa * 2.0 ** -48)
    assert e0 <= max(1e-12, kappa * 2.0 ** -53 * 8)
    s.setup_precond("as")
    W, st = s.solve_cg_as(F, 1e-10, 3000)
    assert st["status"] == "RANN_OK"
