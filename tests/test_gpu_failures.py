"""Failure detection through the C ABI, with every fault made on the host.

No test faults, traps or hangs the GPU: the inputs are corrupted on the
host (a NaN in F, duplicated hidden neurons), the bounded-wait error word of
the tensor-core pipelines is written from the host exactly as an expired
wait would write it, and the device allocator is capped on the host.  Each
case checks the status the handle returns and that it stays usable.

Also: the solver statistics -- the per-phase device times and the condition
estimate from the Krylov coefficients (the Lanczos tridiagonal of CG, the
Arnoldi Hessenberg matrix of GMRES), which lies inside the spectrum of the
preconditioned normal matrix (Sec. 5, Table 1 reports that condition number).
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


def prepared(g, name="multiscale2d", kind="as", mode=1):
    p = ri.config(name, small=True)
    s = g.RannDD(p, *ri.weights(p))
    s.set_precision(mode)
    s.assemble()
    F = s.rhs()
    s.pca(p.pca_mode, p.pca_thr)
    s.setup_precond(kind)
    return p, s, F


@pytest.mark.parametrize("kind,solver", [("as", "cg"), ("ras", "gmres"), ("sas", "cgs")])
def test_nan_in_the_right_hand_side_is_a_breakdown(g, kind, solver):
    p, s, F = prepared(g, kind=kind)
    Fb = F.clone()
    Fb[7] = float("nan")
    fn = {"cg": s.solve_cg_as, "gmres": s.solve_gmres_ras, "cgs": s.solve_cgs}[solver]
    with pytest.raises(g.RannError) as e:
        fn(Fb)
    assert e.value.status == g.BREAKDOWN
    # the handle still solves the clean problem
    W, st = fn(F)
    assert st["status"] == "RANN_OK"


def test_duplicated_neurons_shift_the_local_factors(g):
    """Two identical hidden neurons in every subdomain make identical columns
    of H (PCA off), so every A_i is singular: the set-up shifts the failed
    Cholesky pivots, reports RANN_LOCAL_SINGULAR (a warning) and the count,
    and the solve still reaches the least-squares minimum."""
    p = ri.config("poisson2d_2x2", small=True)
    R, b = ri.weights(p)
    R[:, 1, :] = R[:, 0, :]
    b[:, 1] = b[:, 0]
    s = g.RannDD(p, R, b)
    s.set_precision(0)
    s.assemble()
    F = s.rhs()
    s.pca(g.PCA_NONE, 0.0)
    assert s.setup_precond("as") == g.LOCAL_SINGULAR
    W, st = s.solve_cg_as(F, 1e-8, 2000, allow_not_converged=True)
    assert st["n_shifted"] == p.J
    assert np.all(np.isfinite(W.cpu().numpy()))


def test_expired_pipeline_wait_is_a_timeout(g):
    """The error word that a bounded mbarrier wait of the tensor-core products
    writes when it gives up: pca and setup_precond read it back and return
    RANN_TIMEOUT; the word is cleared, and the repeated call succeeds with
    the same result as an undisturbed handle."""
    p = ri.config("multiscale2d", small=True)
    R, b = ri.weights(p)
    ref = g.RannDD(p, R, b)
    ref.assemble()
    ranks_ref = ref.pca(p.pca_mode, p.pca_thr)
    s = g.RannDD(p, R, b)
    s.assemble()
    F = s.rhs()
    s.inject_fault(g.FAULT_WAIT_EXPIRED, 3)
    with pytest.raises(g.RannError) as e:
        s.pca(p.pca_mode, p.pca_thr)
    assert e.value.status == g.TIMEOUT
    with pytest.raises(g.RannError) as e:       # not reduced after the failed pca
        s.setup_precond("as")
    assert e.value.status == g.EORDER
    np.testing.assert_array_equal(s.pca(p.pca_mode, p.pca_thr), ranks_ref)
    s.inject_fault(g.FAULT_WAIT_EXPIRED, 5)
    with pytest.raises(g.RannError) as e:
        s.setup_precond("as")
    assert e.value.status == g.TIMEOUT
    with pytest.raises(g.RannError) as e:
        s.solve_cg_as(F)
    assert e.value.status == g.EORDER
    s.setup_precond("as")
    W, st = s.solve_cg_as(F)
    assert st["status"] == "RANN_OK"
    # the streaming Schwarz apply's waits report through the same word at the end of a solve
    s.inject_fault(g.FAULT_WAIT_EXPIRED, 7)
    with pytest.raises(g.RannError) as e:
        s.solve_cg_as(F)
    assert e.value.status == g.TIMEOUT
    W2, st = s.solve_cg_as(F)
    assert st["status"] == "RANN_OK"
    assert torch.equal(W, W2)


def test_allocation_cap_is_out_of_memory(g):
    """A cap on the handle's device memory makes the next allocation fail:
    RANN_ENOMEM, the step is not done, and lifting the cap lets it run."""
    p = ri.config("multiscale2d", small=True)
    s = g.RannDD(p, *ri.weights(p))
    s.assemble()
    F = s.rhs()
    s.inject_fault(g.FAULT_ALLOC_CAP, 0)
    with pytest.raises(g.RannError) as e:
        s.pca(p.pca_mode, p.pca_thr)
    assert e.value.status == g.ENOMEM
    s.inject_fault(g.FAULT_ALLOC_CAP, -1)
    s.pca(p.pca_mode, p.pca_thr)
    s.inject_fault(g.FAULT_ALLOC_CAP, 0)
    with pytest.raises(g.RannError) as e:
        s.setup_precond("ras")
    assert e.value.status == g.ENOMEM
    with pytest.raises(g.RannError) as e:
        s.solve_gmres_ras(F)
    assert e.value.status == g.EORDER
    s.inject_fault(g.FAULT_ALLOC_CAP, -1)
    s.setup_precond("ras")
    W, st = s.solve_gmres_ras(F)
    assert st["status"] == "RANN_OK"
    with pytest.raises(g.RannError) as e:
        s.inject_fault(9, 0)
    assert e.value.status == g.EINVAL


@pytest.mark.parametrize("kind,solver", [("as", "cg"), ("sas", "gmres")])
def test_condition_estimate_and_phase_times(g, kind, solver):
    """kappa_est from the first refinement cycle's Krylov coefficients lies
    inside the spectrum of M^{-1} H^T H (Ritz values of CG's Lanczos
    tridiagonal; singular values of GMRES's Hessenberg matrix), formed here
    densely by the oracle on the GPU's reduced blocks (float64 QR local
    solves), and CG's, which converges from inside, reaches half of it; the
    phase times of assemble, pca and setup are reported."""
    p, s, F = prepared(g, kind=kind, mode=0)
    if solver == "cg":
        W, st = s.solve_cg_as(F, 1e-10, 3000)
    else:
        W, st = s.solve_gmres_ras(F, 1e-10, 50, 3000)
    gr = GpuReduced(p, s, s.ranks, F)
    M = sv.schwarz(gr.S, kind)
    A = gr.H.T @ gr.H
    MA = np.stack([M.apply(A[:, c]) for c in range(A.shape[1])], axis=1)
    if solver == "cg":
        lam = np.linalg.eigvals(MA).real
        kappa = lam.max() / lam.min()
        assert 0.5 * kappa <= st["kappa_est"] <= kappa * (1 + 1e-6), (st["kappa_est"], kappa)
    else:
        sg = np.linalg.svd(MA, compute_uv=False)
        assert 1.0 < st["kappa_est"] <= sg[0] / sg[-1] * (1 + 1e-6), (st["kappa_est"], sg[0] / sg[-1])
    assert st["ms_assemble"] > 0 and st["ms_pca"] > 0 and st["ms_setup"] > 0 and st["ms_solve"] > 0
