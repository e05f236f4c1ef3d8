"""Many right-hand sides per launch (batching over right-hand sides on top of
the batching over subdomains): every column of the multi-RHS Schwarz apply and
of the lockstep AS-preconditioned CG equals the one-column routine bit for bit
(the batched kernels keep the one-column arithmetic per column, reading the
block rows of H^T H once per step for up to four columns; the local factors
are read once per column by the streaming Schwarz apply, and once per four
columns where a set is too large for it).  Edge cases: one column, a column count that is not a multiple of
the four-column launch group, a zero right-hand side, columns converging at
different steps, and the float64 factors of precision mode 0 (handled column
by column).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import rann_inputs as ri
from solution_bounds import GpuReduced


@pytest.fixture(scope="module")
def g():
    from paper_2412_19207_gb300 import build
    build.build()
    import paper_2412_19207_gb300 as pkg
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    return pkg


def handle(g, name, kind, mode=1):
    p = ri.config(name, small=True)
    R, b = ri.weights(p)
    s = g.RannDD(p, R, b)
    s.set_precision(mode)
    s.assemble()
    F = s.rhs()
    s.pca(p.pca_mode, p.pca_thr)
    s.setup_precond(kind)
    return p, s, F


@pytest.mark.parametrize("nrhs", [1, 5])
@pytest.mark.parametrize("kind", ["as", "sas", "ras"])
def test_precond_apply_multi_columns_equal_single(g, kind, nrhs):
    p, s, F = handle(g, "multiscale2d", kind)
    n = int(s.sizes()["dof"])
    rng = np.random.default_rng(3)
    R = torch.tensor(rng.standard_normal((nrhs, n)), device="cuda")
    Z = s.precond_apply_multi(R)
    for c in range(nrhs):
        z1 = s.precond_apply(R[c].contiguous())
        assert torch.equal(Z[c], z1), (kind, c, float((Z[c] - z1).abs().max()))


@pytest.mark.parametrize("mode", [1, 0])
def test_cg_multi_columns_equal_single(g, mode):
    p, s, F = handle(g, "multiscale2d", "as", mode)
    rng = np.random.default_rng(5)
    noise = torch.tensor(rng.standard_normal(F.numel()) * 1e-2, device="cuda")
    Fs = torch.stack([F, 2.0 * F, torch.zeros_like(F), F + noise, -F])
    W, stats = s.solve_cg_as_multi(Fs, 1e-10, 3000)
    iters = []
    for c in range(Fs.shape[0]):
        w1, st1 = s.solve_cg_as(Fs[c].contiguous(), 1e-10, 3000)
        assert torch.equal(W[c], w1), (mode, c, float((W[c] - w1).abs().max()))
        assert stats[c]["iters"] == st1["iters"]
        assert stats[c]["rel_res_true"] == st1["rel_res_true"]
        iters.append(st1["iters"])
    assert torch.count_nonzero(W[2]) == 0 and stats[2]["iters"] == 0
    assert all(st["rel_res_true"] <= 1e-10 for st in stats)
    assert len(set(iters)) > 1            # the columns stop at different steps


def test_cg_multi_solution_matches_the_oracle(g):
    from oracle import solver as sv
    p, s, F = handle(g, "multiscale2d", "as")
    R, b = ri.weights(p)
    S = sv.build_system(p, R, b)
    W, stats = s.solve_cg_as_multi(torch.stack([F, 3.0 * F]), 1e-10, 3000)
    gr = GpuReduced(p, s, s.ranks, F)
    qr = sv.solve_qr(S)
    X = ri.test_points(p, 21)
    for c, f in enumerate([1.0, 3.0]):
        gr.check(W[c], scale=f)
        res = np.linalg.norm(s.matvec(W[c].contiguous()).cpu().numpy() - f * S.F)
        assert abs(res - f * qr.res_ls) <= 1e-8 * f * np.linalg.norm(S.F)


@pytest.mark.parametrize("kind,mode", [("sas", 1), ("ras", 1), ("ras", 0)])
def test_gmres_multi_columns_equal_single(g, kind, mode):
    """Lockstep GMRES(50): every column equals the one-column solve bit for
    bit (columns that stop at different steps and restarts, a zero column)."""
    p, s, F = handle(g, "multiscale2d", kind, mode)
    rng = np.random.default_rng(7)
    noise = torch.tensor(rng.standard_normal(F.numel()) * 1e-2, device="cuda")
    Fs = torch.stack([F, torch.zeros_like(F), F + noise, -2.0 * F])
    W, stats = s.solve_gmres_ras_multi(Fs, 1e-10, 50, 3000)
    iters = []
    for c in range(Fs.shape[0]):
        w1, st1 = s.solve_gmres_ras(Fs[c].contiguous(), 1e-10, 50, 3000)
        assert torch.equal(W[c], w1), (kind, mode, c, float((W[c] - w1).abs().max()))
        assert stats[c]["iters"] == st1["iters"]
        assert stats[c]["rel_res_true"] == st1["rel_res_true"]
        iters.append(st1["iters"])
    assert torch.count_nonzero(W[1]) == 0 and stats[1]["iters"] == 0
    assert len(set(iters)) > 1
