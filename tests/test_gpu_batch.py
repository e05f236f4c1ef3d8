"""Many instances per call (rann_dd_batch_run) and the Schwarz apply tuner.

Piecewise-coefficient diffusion instances on subdomain grids of different
sizes (2 x 2 .. 4 x 4) go through the whole path -- assembly, F, PCA, RAS
set-up, GMRES, and the misfit gradient l = ||u_hat - u_obs||^2 (adjoint
solve, dl/dF, dl/da_c) -- on native worker threads with one CUDA stream
each.  Every instance must equal, bit for bit, the same steps run one
instance at a time through the single-handle entry points (with the same
Schwarz apply configuration): nothing in the path depends on the stream or
on scheduling.  One instance's solution is also held to the bound its normal
residual allows against the oracle's direct least-squares solution on the
same reduced blocks.  The tuner: every configuration a set-up can run gives
the same M^{-1} r to the double-float factor accuracy, each one
deterministically; the tuner keeps the configuration in effect unless another
is more than 10 % faster (then the fastest); instances of one size class
share the tuned choice.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import rann_inputs as ri

from solution_bounds import GpuReduced

SUBS = (2, 3, 4, 2, 3)


@pytest.fixture(scope="module")
def g():
    from paper_2412_19207_gb300 import build
    build.build()
    import paper_2412_19207_gb300 as pkg
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    return pkg


def instance(i, sub):
    return ri.piecewise2d(i, sub=sub, pts=8, neurons=30)


def u_obs_of(s):
    X = s.points()
    return (0.01 * torch.sin(np.pi * X[:, 0]) * torch.sin(np.pi * X[:, 1])).contiguous()


def single(g, p, cfg):
    """The batch's steps through the one-instance entry points."""
    s = g.RannDD(p, *ri.weights(p))
    s.assemble()
    F = s.rhs()
    s.pca(p.pca_mode, p.pca_thr)
    s.setup_precond("ras")
    s.set_apply_config(cfg)
    W, st = s.solve_gmres_ras(F, 1e-10, 50, 3000, allow_not_converged=True)
    X = s.points()
    uo = u_obs_of(s)
    u = s.eval(W, X)
    r = 2.0 * (u - uo)
    lam, _ = s.solve_backward(s.eval_grid_t(r), 1e-10, 3000, allow_not_converged=True)
    gF = s.matvec(lam)
    gc = s.grad_coef(F, W, lam)
    return s, F, W, gF, gc, float(((u - uo) ** 2).sum())


def test_batch_equals_single_instances(g):
    ps = [instance(i, sub) for i, sub in enumerate(SUBS)]
    hs = [g.RannDD(p, *ri.weights(p)) for p in ps]
    uo = [u_obs_of(h) for h in hs]
    b = g.Batch(3)
    res = b.run(hs, ps[0].pca_mode, ps[0].pca_thr, prec="ras", solver=g.SOLVER_GMRES, rtol=1e-10, restart=50,
                maxit=3000, u_obs=uo)
    assert len({r["dof"] for r in res}) > 1                     # instances of different sizes
    for p, r in zip(ps, res):
        s, F, W, gF, gc, loss = single(g, p, r["apply_config"])
        assert torch.equal(r["F"], F)
        assert torch.equal(r["W"], W)
        assert torch.equal(r["grad_F"], gF)
        np.testing.assert_array_equal(r["grad_coef"], gc)
        assert r["loss"] == pytest.approx(loss, rel=1e-12)
    # a repeated batch run gives the same bits
    hs2 = [g.RannDD(p, *ri.weights(p)) for p in ps]
    res2 = b.run(hs2, ps[0].pca_mode, ps[0].pca_thr, prec="ras", solver=g.SOLVER_GMRES, rtol=1e-10,
                 restart=50, maxit=3000, u_obs=[u_obs_of(h) for h in hs2])
    for r, r2 in zip(res, res2):
        assert torch.equal(r["W"], r2["W"]) and torch.equal(r["grad_F"], r2["grad_F"])
    b.close()


def test_batch_instance_against_the_oracle(g):
    ps = [instance(i, sub) for i, sub in enumerate((3, 2))]
    hs = [g.RannDD(p, *ri.weights(p)) for p in ps]
    b = g.Batch(2)
    res = b.run(hs, ps[0].pca_mode, ps[0].pca_thr, prec="as", solver=g.SOLVER_CG, rtol=1e-10, maxit=3000)
    for p, h, r in zip(ps, hs, res):
        X = ri.test_points(p, 7)
        u = h.eval(r["W"], torch.tensor(X, device="cuda")).cpu().numpy()
        GpuReduced(p, h, h.ranks, r["F"]).check(r["W"], X, u)
    b.close()


def test_batch_argument_errors(g):
    p = instance(0, 2)
    h = g.RannDD(p, *ri.weights(p))
    b = g.Batch(1)
    with pytest.raises(g.RannError) as e:
        b.run([h, h], p.pca_mode, p.pca_thr)
    assert e.value.status == g.EINVAL
    assert b.run([], p.pca_mode, p.pca_thr) == []
    with pytest.raises(g.RannError) as e:
        g.Batch(0)
    assert e.value.status == g.EINVAL
    b.close()


def test_apply_configurations_agree_and_the_tuner_keeps_the_fastest(g):
    p = ri.config("multiscale2d", small=True)
    s = g.RannDD(p, *ri.weights(p))
    s.set_precision(1)
    s.assemble()
    s.rhs()
    s.pca(p.pca_mode, p.pca_thr)
    s.setup_precond("sas")
    r = torch.tensor(np.random.default_rng(5).standard_normal(s.sizes()["dof"]), device="cuda")
    z = []
    for cfg in range(g.APPLY_NCFG):
        s.set_apply_config(cfg)
        assert s.get_apply_config() == cfg
        a = s.precond_apply(r)
        assert torch.equal(a, s.precond_apply(r))
        z.append(a.cpu().numpy())
    for a in z[1:]:
        np.testing.assert_allclose(a, z[0], rtol=0, atol=1e-11 * np.abs(z[0]).max())
    cur = s.get_apply_config()
    best, ms = s.tune_apply(2)
    assert all(v is not None and v > 0 for v in ms)
    assert s.get_apply_config() == best
    faster = [c for c in range(g.APPLY_NCFG) if c != cur and ms[c] < 0.9 * ms[cur]]
    if faster:
        assert ms[best] == min(ms[c] for c in faster)
    else:
        assert best == cur
    with pytest.raises(g.RannError) as e:
        s.set_apply_config(g.APPLY_NCFG)
    assert e.value.status == g.EINVAL
    # float64 factors (precision mode 0): only the fused configuration's slot is meaningful
    s.set_precision(0)
    s.setup_precond("sas")
    with pytest.raises(g.RannError) as e:
        s.set_apply_config(1)
    assert e.value.status == g.EINVAL


def test_autotune_shares_the_choice_within_a_size_class(g):
    """Three handles of one problem (one size class) and one of another: the
    class's instances all use the configuration its first instance tuned."""
    ps = [instance(0, 3)] * 3 + [instance(1, 2)]
    hs = [g.RannDD(p, *ri.weights(p)) for p in ps]
    b = g.Batch(4)
    res = b.run(hs, ps[0].pca_mode, ps[0].pca_thr, prec="ras", solver=g.SOLVER_GMRES, rtol=1e-8, maxit=3000,
                autotune=True)
    assert len({r["apply_config"] for r in res[:3]}) == 1
    assert all(0 <= r["apply_config"] < g.APPLY_NCFG for r in res)
    assert torch.equal(res[0]["W"], res[1]["W"]) and torch.equal(res[0]["W"], res[2]["W"])
    b.close()
