"""The CG variants of Sec. 5 (Table 1b) and the transposed Schwarz
preconditioner on the GPU, against the oracle.

  * M^{-T} is the adjoint of M^{-1}: <M^{-T} r, s> = <r, M^{-1} s> (both
    precision modes; float64 factors to kappa eps, double-float ones to the
    factor's own accuracy), and differs from M^{-1} for SAS/RAS;
  * CGS and BiCG with AS, SAS and RAS reach the least-squares minimum of the
    oracle's direct QR solve (||H W - F|| to 1e-8 ||F||), and their fitted
    values and u_hat match the direct solution on the GPU's reduced blocks
    within the bound their float64 normal residual allows;
  * with J = 2x2 and AS (M^{-1} H^T H = J I, Table 2) both finish in one step.
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


_sys = {}


def system(name):
    if name not in _sys:
        p = ri.config(name, small=True)
        R, b = ri.weights(p)
        S = sv.build_system(p, R, b)
        _sys[name] = (p, R, b, S)
    return _sys[name]


def handle(g, name, kind, mode=1):
    p, R, b, S = system(name)
    s = g.RannDD(p, R, b)
    s.set_precision(mode)
    s.assemble()
    F = s.rhs()
    s.pca(p.pca_mode, p.pca_thr)
    s.setup_precond(kind)
    return s, F


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("kind", ["as", "sas", "ras"])
def test_transposed_preconditioner_is_the_adjoint(g, kind, mode):
    s, F = handle(g, "multiscale2d", kind, mode)
    n = int(s.sizes()["dof"])
    rng = np.random.default_rng(11)
    r = torch.tensor(rng.standard_normal(n), device="cuda")
    v = torch.tensor(rng.standard_normal(n), device="cuda")
    mt_r = s.precond_apply_t(r)
    m_v = s.precond_apply(v)
    lhs, rhs = float(mt_r @ v), float(r @ m_v)
    scale = float(mt_r.norm() * v.norm())
    assert abs(lhs - rhs) <= (1e-9 if mode == 0 else 1e-6) * scale
    if kind != "as":
        assert float((mt_r - s.precond_apply(r)).norm()) > 1e-6 * float(mt_r.norm())
    else:
        assert float((mt_r - s.precond_apply(r)).norm()) <= 1e-12 * float(mt_r.norm())


@pytest.mark.parametrize("solver", ["cgs", "bicg"])
@pytest.mark.parametrize("kind", ["as", "sas", "ras"])
def test_variants_reach_the_least_squares_minimum(g, solver, kind):
    p, R, b, S = system("multiscale2d")
    s, F = handle(g, "multiscale2d", kind)
    W, st = (s.solve_cgs if solver == "cgs" else s.solve_bicg)(F, 1e-10, 3000)
    assert st["status"] == "RANN_OK" and st["rel_res_true"] <= 1e-10
    qr = sv.solve_qr(S)
    res = np.linalg.norm(s.matvec(W).cpu().numpy() - S.F)
    assert abs(res - qr.res_ls) <= 1e-8 * np.linalg.norm(S.F)
    X = ri.test_points(p, 21)
    ug = s.eval(W, torch.tensor(X, device="cuda")).cpu().numpy()
    GpuReduced(p, s, s.ranks, F).check(W, X, ug)


@pytest.mark.parametrize("solver", ["cgs", "bicg"])
def test_variants_one_iteration_on_2x2(g, solver):
    p = ri.config("poisson2d_2x2")
    s = g.RannDD(p)
    s.set_precision(0)          # the identity M^{-1} A = J I holds to float64 rounding only
    s.assemble()
    F = s.rhs()
    s.pca(p.pca_mode, p.pca_thr)
    s.setup_precond("as")
    _, st = (s.solve_cgs if solver == "cgs" else s.solve_bicg)(F, 1e-8, 10)
    assert st["iters"] == 1 and st["status"] == "RANN_OK"
