"""Oracle blocks of full-size problems, computed in parallel worker processes.

The oracle's float64 assembly and Jacobi SVD take seconds per subdomain at
the configured sizes (m = 300 .. 400, thousands of rows per block), so the
full-size parity tests farm the blocks they need out to a process pool.  The
pool uses the "spawn" start method: the parent process has already created a
CUDA context, and a forked child of such a process can hang.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _block(args):
    name, j, rank, want_dense = args
    import rann_inputs as ri
    from oracle import assembly as asm
    from oracle import solver as sv
    p = ri.config(name)
    R, b = ri.weights(p)
    rows, Psi, H = asm.block(p, R, b, j)
    pc = sv.pca(Psi, p.pca_mode, p.pca_thr, rank)
    out = {"j": j, "rows": rows, "sigma": pc.sigma, "V": pc.V, "rank": pc.rank, "borderline": pc.borderline,
           "B": H @ pc.V}
    if want_dense:
        out["Psi"], out["H"] = Psi, H
    return out


def oracle_blocks(name, js, ranks=None, want_dense=False, workers=None):
    """Oracle rows, PCA and reduced block of subdomains js of the full-size
    configured problem `name` (at the given ranks, else by the rank rule);
    with want_dense also Psi_j and H_j."""
    js = list(js)
    workers = workers or max(1, min(len(js), (os.cpu_count() or 2) - 1, 12))
    args = [(name, int(j), None if ranks is None else int(ranks[j]), want_dense) for j in js]
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ["OMP_NUM_THREADS"] = os.environ["OPENBLAS_NUM_THREADS"] = "1"
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            res = pool.map(_block, args, chunksize=1)
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return {r["j"]: r for r in res}


def _qr(A):
    from oracle import linalg as la
    return la.householder_qr(A)


def householder_qrs(mats, workers=None):
    """The oracle's Householder QR of each matrix, in parallel."""
    workers = workers or max(1, min(len(mats), (os.cpu_count() or 2) - 1, 12))
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_qr, mats, chunksize=1)


def hood(p, centre_multi_index, radius=1):
    """Subdomain indices of the (2 radius + 1)^d neighbourhood of a subdomain."""
    import itertools
    l = p.sub[: p.dim]
    out = []
    for off in itertools.product(*[range(-radius, radius + 1)] * p.dim):
        k = [centre_multi_index[i] + off[i] for i in range(p.dim)]
        if all(0 <= k[i] < l[i] for i in range(p.dim)):
            j, s = 0, 1
            for i in range(p.dim):
                j += k[i] * s
                s *= l[i]
            out.append(j)
    return sorted(out)

