"""The allocation-free transposed block product against a host product and the
handle's own.

rann_dd_matvec_t_noalloc serves callers that cannot allocate device memory
(their device memory is all owned by another allocator, or they cannot take
the synchronisation an allocation may imply); it keeps its scratch in a fixed
device array.  This file is collected last so that a failure here comes after
every other test has run; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import rann_inputs as ri


def test_noalloc_transposed_product_matches_handle_product():
    from paper_2412_19207_gb300 import build
    build.build()
    import paper_2412_19207_gb300 as g
    lib = g.load_library()
    p = ri.config("multiscale2d", small=True)
    s = g.RannDD(p)
    s.assemble()
    ranks = s.pca(p.pca_mode, p.pca_thr)
    blocks = [s.block(j, 2) for j in range(p.J)]
    # two more blocks at the edges of the descriptor rules: no rows (its z part
    # is zero), and no columns with a row stride of 3
    rng = np.random.default_rng(5)
    blocks.append((np.zeros(0, dtype=np.int64), np.zeros((0, 5))))
    blocks.append((rng.integers(0, p.n_points(), 10).astype(np.int64), np.zeros((10, 0))))
    J = len(blocks)
    n_rows = np.array([b[1].shape[0] for b in blocks], dtype=np.int32)
    n_cols = np.array([b[1].shape[1] for b in blocks], dtype=np.int32)
    ld = n_cols + 1                               # a row stride wider than the used columns
    ld[-1] = 3
    boff = np.concatenate([[0], np.cumsum(n_rows.astype(np.int64) * ld)])[:J].astype(np.int64)
    row_off = np.concatenate([[0], np.cumsum(n_rows)])[:J].astype(np.int64)
    zoff = np.concatenate([[0], np.cumsum(n_cols)])[:J].astype(np.int64)
    Bh = np.zeros(int(boff[-1] + n_rows[-1] * ld[-1]))
    for j, (rows, B) in enumerate(blocks):
        Bh[boff[j]:boff[j] + n_rows[j] * ld[j]].reshape(n_rows[j], ld[j])[:, : n_cols[j]] = B
    B_dev = torch.tensor(Bh, device="cuda")
    rows_dev = torch.tensor(np.concatenate([b[0] for b in blocks]), dtype=torch.int64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    nz = int(n_cols.sum())
    for trial in range(2):
        yh = np.random.default_rng(trial).standard_normal(p.n_points())
        y = torch.tensor(yh, device="cuda")
        z = torch.full((nz,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.rann_dd_matvec_t_noalloc(J, boff.ctypes.data, n_rows.ctypes.data, n_cols.ctypes.data,
                                          ld.ctypes.data, row_off.ctypes.data, zoff.ctypes.data,
                                          B_dev.data_ptr(), rows_dev.data_ptr(), y.data_ptr(), z.data_ptr(), stream)
        assert st == g.OK, lib.rann_dd_last_error()
        torch.cuda.synchronize()
        zg = z.cpu().numpy()
        # host product z_j = B_j^T y(rows_j)
        zh = np.concatenate([B.T @ yh[rows] for rows, B in blocks])
        assert np.linalg.norm(zg - zh) <= 1e-13 * np.linalg.norm(zh) * np.sqrt(zh.size)
        assert np.all(zg[zoff[-2]:zoff[-2] + 5] == 0.0)
        # and the handle's own transposed product on the configured blocks
        zr = s.matvec_t(y).cpu().numpy()
        assert np.linalg.norm(zg[: zr.size] - zr) <= 1e-13 * np.linalg.norm(zr) * np.sqrt(zr.size)
    # sizes beyond the fixed scratch (16384 row tiles x 128 columns > 2^20) are
    # rejected on the host before anything is enqueued, and so is a row count
    # whose tile count would overflow 32-bit arithmetic
    for rows_big in (1 << 22, 2**31 - 1):
        big = np.array([rows_big], dtype=np.int32)
        st = lib.rann_dd_matvec_t_noalloc(1, np.zeros(1, np.int64).ctypes.data, big.ctypes.data,
                                          np.array([128], np.int32).ctypes.data,
                                          np.array([128], np.int32).ctypes.data,
                                          np.zeros(1, np.int64).ctypes.data, np.zeros(1, np.int64).ctypes.data,
                                          B_dev.data_ptr(), rows_dev.data_ptr(), y.data_ptr(), z.data_ptr(), stream)
        assert st == g.EINVAL and b"scratch" in lib.rann_dd_last_error()
