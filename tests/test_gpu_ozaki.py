"""The PCA's dense products from bf16 digit slices (precision mode 1) are
float64-accurate.

Sec. 4 forms the Gram matrices Psi_j^T Psi_j and the reduced blocks
B_j = H_j V_{p_j} in float64.  Mode 1 computes both from exact 7-bit digit
slices on the tensor cores (Ozaki splitting); the bound proved in the kernel's
header is a few units of 2^-53 K max|a_i.| max|b_.j| per entry, the float64
product's own bound.  Checked here:
  * B_j against the host float64 product of the device's own H_j and V_{p_j},
    entrywise within 4 m eps max|H_i.| max|V_.k| (either side may err by about
    m eps |H_i.||V_.k|);
  * the Gram matrices through their spectra: by Weyl's inequality the
    eigenvalues move by at most ||dG||_2, so mode 1 and mode 0 (float64 SIMT
    tiles) agree within the eigensolver's own backward error, 64 m eps
    lambda_max, and give the same ranks unless a value sits at the cut.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import rann_inputs as ri

EPS = 2.0 ** -52
NAMES = ["multiscale2d", "heat3d", "poisson3d", "example1", "piecewise2d"]


@pytest.fixture(scope="module")
def g():
    from paper_2412_19207_gb300 import build
    build.build()
    import paper_2412_19207_gb300 as pkg
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    return pkg


def reduced(g, p, mode):
    s = g.RannDD(p)
    s.set_precision(mode)
    s.assemble()
    ranks = s.pca(p.pca_mode, p.pca_thr)
    return s, ranks


@pytest.mark.parametrize("name", NAMES)
def test_projection_matches_float64_product(g, name):
    p = ri.config(name, small=True)
    s, ranks = reduced(g, p, 1)
    m = p.neurons
    for j in range(p.J):
        _, Hj = s.block(j, 1)
        _, Bj = s.block(j, 2)
        _, V = s.pca_of(j)
        ref = Hj @ V
        bound = 4 * m * EPS * np.abs(Hj).max(axis=1)[:, None] * np.abs(V).max(axis=0)[None, :]
        err = np.abs(Bj - ref)
        assert np.all(err <= bound), (j, float((err / np.maximum(bound, 1e-300)).max()))


@pytest.mark.parametrize("name", NAMES)
def test_gram_spectra_match_float64_tiles(g, name):
    p = ri.config(name, small=True)
    s1, r1 = reduced(g, p, 1)
    s0, r0 = reduced(g, p, 0)
    m = p.neurons
    for j in range(p.J):
        e1, _ = s1.pca_of(j)
        e0, _ = s0.pca_of(j)
        tol = 64 * m * EPS * e0[0]
        np.testing.assert_allclose(e1, e0, rtol=0, atol=tol)
        if r1[j] != r0[j]:
            # only a value within the tolerance of the rank cut may flip
            cut = p.pca_thr if p.pca_mode == ri.PCA_ABS else None
            k = min(r1[j], r0[j])
            assert cut is None or abs(np.sqrt(max(e0[k], 0.0)) - cut) <= 1e-6 * max(cut, 1.0), (j, r1[j], r0[j])


def test_solution_from_tensor_core_pca_matches_float64_pca(g):
    """The same problem reduced in mode 1 and mode 0, then solved in float64
    (mode 0), gives the same u_hat to the solve tolerance."""
    p = ri.config("poisson3d", small=True)
    X = torch.tensor(ri.test_points(p, 7), device="cuda")
    out = []
    for mode in (1, 0):
        s, ranks = reduced(g, p, mode)
        s.set_precision(0)
        F = s.rhs()
        s.setup_precond("as")
        W, st = s.solve_cg_as(F, 1e-10, 5000)
        assert st["rel_res_true"] <= 1e-10
        out.append(s.eval(W, X).cpu().numpy())
    assert np.linalg.norm(out[0] - out[1]) <= 1e-8 * np.linalg.norm(out[1])
