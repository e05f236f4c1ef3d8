"""GB300 (sm_103a) RaNN domain-decomposition solver: thin Python binding.

Every step of the method runs in librann_dd.so (hand-written CUDA kernels
behind the C ABI of include/rann_dd.h); this module only marshals arguments:
problem descriptors into the C struct, torch CUDA tensors into device
pointers, and the current torch stream into the library's stream.  There is
no CPU fallback: if the library is missing, importing the binding raises.

Typical use (Algorithm 1 order):

    s = RannDD(problem)            # steps 1-2: subdomains, grid, networks
    s.assemble()                   # steps 3, 5: Psi_j and H_j
    F = s.rhs()                    # F = f - A[G] at the collocation points
    ranks = s.pca(PCA_VARIANCE, 1e-12)    # step 4
    s.setup_precond(PREC_RAS)      # step 6: A_i and their factors
    W, stats = s.solve_gmres_ras(F, rtol=1e-10, restart=50)
    u = s.eval(W, x)               # u_hat at points x
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "librann_dd.so")

OP_POISSON, OP_DIFFUSION, OP_HEAT = 0, 1, 2
COEF_CONST, COEF_MULTISCALE, COEF_PIECEWISE = 0, 1, 2
G_ZERO, G_SINPROD = 0, 1
LAYOUT_CELL, LAYOUT_PAPER = 0, 1
PCA_ABS, PCA_VARIANCE, PCA_NONE = 0, 1, 2
PREC_NONE, PREC_AS, PREC_SAS, PREC_RAS = 0, 1, 2, 3
PREC_BY_NAME = {"none": PREC_NONE, "as": PREC_AS, "sas": PREC_SAS, "ras": PREC_RAS}

STATUS = {0: "RANN_OK", 1: "RANN_EINVAL", 2: "RANN_ENOMEM", 3: "RANN_ECUDA", 4: "RANN_NOT_CONVERGED",
          5: "RANN_BREAKDOWN", 6: "RANN_LOCAL_SINGULAR", 7: "RANN_EORDER", 8: "RANN_TIMEOUT"}
OK, EINVAL, ENOMEM, ECUDA, NOT_CONVERGED, BREAKDOWN, LOCAL_SINGULAR, EORDER, TIMEOUT = range(9)
FAULT_WAIT_EXPIRED, FAULT_ALLOC_CAP = 1, 2


class RannError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Desc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("op", ctypes.c_int), ("c0", ctypes.c_double), ("nu", ctypes.c_double),
        ("coef", ctypes.c_int), ("coef_value", ctypes.c_double), ("eps", ctypes.c_double),
        ("coef_grid", ctypes.c_int), ("coef_vals", ctypes.POINTER(ctypes.c_double)),
        ("layout", ctypes.c_int), ("sub", ctypes.c_int * 3), ("overlap", ctypes.c_double * 3),
        ("delta", ctypes.c_double), ("pts", ctypes.c_int * 3), ("neurons", ctypes.c_int),
        ("w_range", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("R", ctypes.POINTER(ctypes.c_double)), ("b", ctypes.POINTER(ctypes.c_double)),
        ("rho", ctypes.c_double), ("g_kind", ctypes.c_int), ("f0", ctypes.c_double),
        ("f_terms", ctypes.c_int), ("fc", ctypes.POINTER(ctypes.c_double)),
        ("fa", ctypes.POINTER(ctypes.c_double)),
    ]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_res_true", ctypes.c_double), ("rel_res_rec", ctypes.c_double),
                ("rel_res_prec", ctypes.c_double), ("ms_solve", ctypes.c_double), ("n_shifted", ctypes.c_int),
                ("ms_assemble", ctypes.c_double), ("ms_pca", ctypes.c_double), ("ms_setup", ctypes.c_double),
                ("kappa_est", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Pipeline(ctypes.Structure):
    _fields_ = [("pca_mode", ctypes.c_int), ("pca_thr", ctypes.c_double), ("prec_kind", ctypes.c_int),
                ("solver", ctypes.c_int), ("rtol", ctypes.c_double), ("restart", ctypes.c_int),
                ("maxit", ctypes.c_int), ("autotune", ctypes.c_int), ("backward", ctypes.c_int)]


class PipelineOut(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("dof", ctypes.c_int64), ("apply_config", ctypes.c_int),
                ("loss", ctypes.c_double), ("forward", Stats), ("adjoint", Stats)]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_L = ctypes.c_int64

# name -> (restype, argtypes); every entry point declared in include/rann_dd.h
SIGNATURES = {
    "rann_dd_create": (_I, [ctypes.POINTER(Desc), _P, ctypes.POINTER(_P)]),
    "rann_dd_destroy": (None, [_P]),
    "rann_dd_sizes": (_I, [_P, ctypes.POINTER(_L), ctypes.POINTER(_L), ctypes.POINTER(_I), ctypes.POINTER(_I),
                           ctypes.POINTER(_L)]),
    "rann_dd_points": (_I, [_P, _P]),
    "rann_dd_assemble": (_I, [_P]),
    "rann_dd_rhs": (_I, [_P, _P]),
    "rann_dd_pca": (_I, [_P, _I, _D, ctypes.POINTER(_I)]),
    "rann_dd_setup_precond": (_I, [_P, _I, _I]),
    "rann_dd_solve_cg_as": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(Stats)]),
    "rann_dd_solve_gmres_ras": (_I, [_P, _P, _P, _D, _I, _I, ctypes.POINTER(Stats)]),
    "rann_dd_solve_cgs": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(Stats)]),
    "rann_dd_solve_bicg": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(Stats)]),
    "rann_dd_eval": (_I, [_P, _P, _P, _L, _P]),
    "rann_dd_solve_backward": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(Stats)]),
    "rann_dd_grad_c0": (_I, [_P, _P, _P, _P, ctypes.POINTER(_D)]),
    "rann_dd_grad_coef": (_I, [_P, _P, _P, _P, _P]),
    "rann_dd_set_coef": (_I, [_P, _P]),
    "rann_dd_eval_grid_t": (_I, [_P, _P, _P]),
    "rann_dd_set_precision": (_I, [_P, _I]),
    "rann_dd_matvec": (_I, [_P, _P, _P]),
    "rann_dd_matvec_t": (_I, [_P, _P, _P]),
    "rann_dd_normal_matvec": (_I, [_P, _P, _P]),
    "rann_dd_precond_apply": (_I, [_P, _P, _P]),
    "rann_dd_precond_apply_t": (_I, [_P, _P, _P]),
    "rann_dd_precond_apply_multi": (_I, [_P, _P, _P, _I]),
    "rann_dd_solve_cg_as_multi": (_I, [_P, _P, _P, _I, _D, _I, ctypes.POINTER(Stats)]),
    "rann_dd_solve_gmres_ras_multi": (_I, [_P, _P, _P, _I, _D, _I, _I, ctypes.POINTER(Stats)]),
    "rann_dd_block_info": (_I, [_P, _I, ctypes.POINTER(_L), ctypes.POINTER(_I)]),
    "rann_dd_get_block": (_I, [_P, _I, _I, _P, _P]),
    "rann_dd_get_pca": (_I, [_P, _I, _P, _P]),
    "rann_dd_matvec_t_noalloc": (_I, [_I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "rann_dd_profile_enable": (_I, [_P, _I]),
    "rann_dd_profile_get": (_I, [_P, _I, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(_L),
                                 ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_I)]),
    "rann_dd_inject_fault": (_I, [_P, _I, _L]),
    "rann_dd_device_rates": (_I, [ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "rann_dd_set_apply_config": (_I, [_P, _I]),
    "rann_dd_get_apply_config": (_I, [_P, ctypes.POINTER(_I)]),
    "rann_dd_tune_apply": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_float)]),
    "rann_dd_set_stream": (_I, [_P, _P]),
    "rann_dd_batch_create": (_I, [_I, ctypes.POINTER(_P)]),
    "rann_dd_batch_destroy": (None, [_P]),
    "rann_dd_batch_run": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(Pipeline), ctypes.POINTER(_P),
                               ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                               ctypes.POINTER(PipelineOut)]),
    "rann_dd_status_string": (ctypes.c_char_p, [_I]),
    "rann_dd_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads librann_dd.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librann_dd.so not found at {path}: run paper_2412_19207_gb300.build.build() "
                           "(nvcc, sm_103a) first; there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


BOUND_NAMES = {0: "hbm", 1: "alu", 2: "tensor", 3: "alu_df32"}


def _check(status: int, what: str, allow=()):
    if status == OK or status in allow:
        return status
    raise RannError(status, f"{what}: {load_library().rann_dd_last_error().decode()}")


def _dptr(t) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA torch tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _f64p(a: Optional[np.ndarray]):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=np.float64)
    return arr, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_desc(p) -> tuple:
    """C descriptor from a problem object (rann_inputs.Problem or any object with
    the same attributes).  Returns (desc, keepalive) -- keep both alive until
    the handle is created."""
    d = Desc()
    keep = []
    d.dim, d.op, d.c0, d.nu = p.dim, p.op, p.c0, p.nu
    d.coef, d.coef_value, d.eps, d.coef_grid = p.coef, p.coef_value, p.eps, p.coef_grid
    arr, ptr = _f64p(p.coef_vals)
    keep.append(arr)
    d.coef_vals = ptr
    d.layout = p.layout
    for i in range(3):
        d.sub[i] = int(p.sub[i]) if i < p.dim else 1
        d.pts[i] = int(p.pts[i]) if i < p.dim else 1
        d.overlap[i] = float(p.overlap[i]) if i < len(p.overlap) else 0.0
    d.delta = p.delta
    d.neurons, d.w_range, d.seed = p.neurons, p.w_range, p.seed
    R = getattr(p, "R", None)
    b = getattr(p, "b", None)
    arr, ptr = _f64p(R)
    keep.append(arr)
    d.R = ptr
    arr, ptr = _f64p(b)
    keep.append(arr)
    d.b = ptr
    d.rho, d.g_kind, d.f0 = p.rho, p.g_kind, p.f0
    if p.fc is not None:
        d.f_terms = len(p.fc)
        arr, ptr = _f64p(p.fc)
        keep.append(arr)
        d.fc = ptr
        fa = np.zeros((len(p.fc), p.dim))
        fa[:, : np.asarray(p.fa).shape[1]] = np.asarray(p.fa)
        arr, ptr = _f64p(fa)
        keep.append(arr)
        d.fa = ptr
    else:
        d.f_terms = 0
    return d, keep


class RannDD:
    """One problem instance on the current CUDA device and stream."""

    def __init__(self, problem, R: Optional[np.ndarray] = None, b: Optional[np.ndarray] = None, stream=None):
        import torch
        lib = load_library()
        self.problem = problem
        desc, keep = make_desc(problem)
        if R is not None:
            arr, ptr = _f64p(R)
            keep.append(arr)
            desc.R = ptr
            arr, ptr = _f64p(b)
            keep.append(arr)
            desc.b = ptr
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(lib.rann_dd_create(ctypes.byref(desc), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
               "rann_dd_create")
        self._h = h
        self._lib = lib
        self.ranks = None
        self._prec = None

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rann_dd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- sizes ------------------------------------------------------------
    def sizes(self):
        n, rows, dof = _L(), _L(), _L()
        J, m = _I(), _I()
        _check(self._lib.rann_dd_sizes(self._h, ctypes.byref(n), ctypes.byref(rows), ctypes.byref(J),
                                       ctypes.byref(m), ctypes.byref(dof)), "rann_dd_sizes")
        return {"n_points": n.value, "n_block_rows": rows.value, "J": J.value, "m": m.value, "dof": dof.value}

    def _empty(self, n):
        import torch
        return torch.empty(int(n), dtype=torch.float64, device="cuda")

    def points(self):
        sz = self.sizes()
        x = self._empty(sz["n_points"] * self.problem.dim)
        _check(self._lib.rann_dd_points(self._h, _dptr(x)), "rann_dd_points")
        return x.view(-1, self.problem.dim)

    # -- Algorithm 1 ------------------------------------------------------
    def assemble(self):
        _check(self._lib.rann_dd_assemble(self._h), "rann_dd_assemble")

    def rhs(self, out=None):
        F = out if out is not None else self._empty(self.sizes()["n_points"])
        _check(self._lib.rann_dd_rhs(self._h, _dptr(F)), "rann_dd_rhs")
        return F

    def pca(self, mode: int, thr: float):
        J = self.sizes()["J"]
        ranks = (ctypes.c_int * J)()
        _check(self._lib.rann_dd_pca(self._h, mode, thr, ranks), "rann_dd_pca")
        self.ranks = np.array(ranks[:], dtype=np.int64)
        return self.ranks

    def setup_precond(self, kind, overlap_level: int = 1) -> int:
        kind = PREC_BY_NAME[kind] if isinstance(kind, str) else kind
        self._prec = kind
        return _check(self._lib.rann_dd_setup_precond(self._h, kind, overlap_level), "rann_dd_setup_precond",
                      allow=(LOCAL_SINGULAR,))

    def solve_cg_as(self, F, rtol=1e-10, maxit=2000, W=None, allow_not_converged=False):
        W = W if W is not None else self._empty(self.sizes()["dof"])
        st = Stats()
        s = self._lib.rann_dd_solve_cg_as(self._h, _dptr(F), _dptr(W), rtol, maxit, ctypes.byref(st))
        _check(s, "rann_dd_solve_cg_as", allow=(NOT_CONVERGED,) if allow_not_converged else ())
        return W, st.as_dict() | {"status": STATUS[s]}

    def solve_cg_as_multi(self, F, rtol=1e-10, maxit=2000, W=None, allow_not_converged=False):
        """AS-preconditioned CG for the rows of F ([nrhs][N], device float64) in
        lockstep; returns W [nrhs][DoF] and one stats dict per row."""
        nrhs = int(F.shape[0])
        W = W if W is not None else self._empty(nrhs * self.sizes()["dof"]).reshape(nrhs, -1)
        st = (Stats * max(nrhs, 1))()
        s = self._lib.rann_dd_solve_cg_as_multi(self._h, _dptr(F), _dptr(W), nrhs, rtol, maxit, st)
        _check(s, "rann_dd_solve_cg_as_multi", allow=(NOT_CONVERGED,) if allow_not_converged else ())
        return W, [st[c].as_dict() for c in range(nrhs)]

    def set_apply_config(self, cfg: int):
        """Schwarz apply configuration (0: fused 32-row blocks; 1..3: streaming rows)."""
        _check(self._lib.rann_dd_set_apply_config(self._h, int(cfg)), "rann_dd_set_apply_config")

    def get_apply_config(self) -> int:
        c = _I()
        _check(self._lib.rann_dd_get_apply_config(self._h, ctypes.byref(c)), "rann_dd_get_apply_config")
        return c.value

    def tune_apply(self, reps: int = 3):
        """Times every Schwarz apply configuration and keeps the one in effect
        unless another is more than 10 % faster (then the fastest); returns
        (chosen, ms per configuration, None where it cannot run)."""
        best = _I()
        ms = (ctypes.c_float * APPLY_NCFG)()
        _check(self._lib.rann_dd_tune_apply(self._h, int(reps), ctypes.byref(best), ms), "rann_dd_tune_apply")
        return best.value, [None if v < 0 else float(v) for v in ms]

    def solve_gmres_ras_multi(self, F, rtol=1e-10, restart=50, maxit=2000, W=None, allow_not_converged=False):
        """Left-preconditioned GMRES(restart) for the rows of F ([nrhs][N], device
        float64) in lockstep; returns W [nrhs][DoF] and one stats dict per row."""
        nrhs = int(F.shape[0])
        W = W if W is not None else self._empty(nrhs * self.sizes()["dof"]).reshape(nrhs, -1)
        st = (Stats * max(nrhs, 1))()
        s = self._lib.rann_dd_solve_gmres_ras_multi(self._h, _dptr(F), _dptr(W), nrhs, rtol, restart, maxit, st)
        _check(s, "rann_dd_solve_gmres_ras_multi", allow=(NOT_CONVERGED,) if allow_not_converged else ())
        return W, [st[c].as_dict() for c in range(nrhs)]

    def solve_gmres_ras(self, F, rtol=1e-10, restart=50, maxit=2000, W=None, allow_not_converged=False):
        W = W if W is not None else self._empty(self.sizes()["dof"])
        st = Stats()
        s = self._lib.rann_dd_solve_gmres_ras(self._h, _dptr(F), _dptr(W), rtol, restart, maxit, ctypes.byref(st))
        _check(s, "rann_dd_solve_gmres_ras", allow=(NOT_CONVERGED,) if allow_not_converged else ())
        return W, st.as_dict() | {"status": STATUS[s]}

    def _solve_variant(self, fn, F, rtol, maxit, W, allow_not_converged):
        W = W if W is not None else self._empty(self.sizes()["dof"])
        st = Stats()
        s = getattr(self._lib, fn)(self._h, _dptr(F), _dptr(W), rtol, maxit, ctypes.byref(st))
        _check(s, fn, allow=(NOT_CONVERGED,) if allow_not_converged else ())
        return W, st.as_dict() | {"status": STATUS[s]}

    def solve_cgs(self, F, rtol=1e-10, maxit=2000, W=None, allow_not_converged=False):
        """Conjugate gradient squared on the normal equations (Sec. 5, Table 1b)."""
        return self._solve_variant("rann_dd_solve_cgs", F, rtol, maxit, W, allow_not_converged)

    def solve_bicg(self, F, rtol=1e-10, maxit=2000, W=None, allow_not_converged=False):
        """Biconjugate gradients on the normal equations (Sec. 5, Table 1b)."""
        return self._solve_variant("rann_dd_solve_bicg", F, rtol, maxit, W, allow_not_converged)

    def solve_backward(self, gW, rtol=1e-10, maxit=2000, lam=None, allow_not_converged=False):
        """lam = (H^T H)^{-1} gW with the stored preconditioner (adjoint of the solve)."""
        lam = lam if lam is not None else self._empty(self.sizes()["dof"])
        st = Stats()
        s = self._lib.rann_dd_solve_backward(self._h, _dptr(gW), _dptr(lam), rtol, maxit, ctypes.byref(st))
        _check(s, "rann_dd_solve_backward", allow=(NOT_CONVERGED,) if allow_not_converged else ())
        return lam, st.as_dict() | {"status": STATUS[s]}

    def grad_c0(self, F, W, lam) -> float:
        """dl/dc0 through the solve for -Lap u + c0 u, given the right-hand side F,
        the solution W and lam = (H^T H)^{-1} dl/dW (rann_dd_grad_c0)."""
        out = _D(0.0)
        _check(self._lib.rann_dd_grad_c0(self._h, _dptr(F), _dptr(W), _dptr(lam), ctypes.byref(out)),
               "rann_dd_grad_c0")
        return out.value

    def grad_coef(self, F, W, lam) -> np.ndarray:
        """dl/da_c for the piecewise diffusion coefficient (rann_dd_grad_coef),
        given the right-hand side F, the solution W and lam = (H^T H)^{-1} dl/dW."""
        g = self.problem.coef_grid
        out = np.zeros(g * g)
        _check(self._lib.rann_dd_grad_coef(self._h, _dptr(F), _dptr(W), _dptr(lam), out.ctypes.data),
               "rann_dd_grad_coef")
        return out

    def set_coef(self, vals):
        """New piecewise coefficient values (the handle must be re-assembled)."""
        arr = np.ascontiguousarray(vals, dtype=np.float64)
        _check(self._lib.rann_dd_set_coef(self._h, arr.ctypes.data), "rann_dd_set_coef")
        self._prec = None

    def eval_grid_t(self, r, out=None):
        """E^T r for u_hat = E W + G at the collocation points (rann_dd_eval_grid_t)."""
        gW = out if out is not None else self._empty(self.sizes()["dof"])
        _check(self._lib.rann_dd_eval_grid_t(self._h, _dptr(r), _dptr(gW)), "rann_dd_eval_grid_t")
        return gW

    def solve(self, F, rtol=1e-10, maxit=2000, restart=50):
        """The solve matching the preconditioner: AS-CG for AS/none, GMRES otherwise."""
        if self._prec in (PREC_AS, PREC_NONE):
            return self.solve_cg_as(F, rtol, maxit)
        return self.solve_gmres_ras(F, rtol, restart, maxit)

    def set_precision(self, mode: int):
        """1 (default): double-float preconditioner set-up and Krylov iterations with
        float64 residuals; 0: float64 throughout.  Affects the next setup/solve."""
        _check(self._lib.rann_dd_set_precision(self._h, mode), "rann_dd_set_precision")

    def eval(self, W, x, out=None):
        n = x.shape[0]
        u = out if out is not None else self._empty(n)
        _check(self._lib.rann_dd_eval(self._h, _dptr(W), _dptr(x), n, _dptr(u)), "rann_dd_eval")
        return u

    # -- building blocks --------------------------------------------------
    def matvec(self, x, y=None):
        y = y if y is not None else self._empty(self.sizes()["n_points"])
        _check(self._lib.rann_dd_matvec(self._h, _dptr(x), _dptr(y)), "rann_dd_matvec")
        return y

    def matvec_t(self, y, z=None):
        z = z if z is not None else self._empty(self.sizes()["dof"])
        _check(self._lib.rann_dd_matvec_t(self._h, _dptr(y), _dptr(z)), "rann_dd_matvec_t")
        return z

    def normal_matvec(self, x, z=None):
        z = z if z is not None else self._empty(self.sizes()["dof"])
        _check(self._lib.rann_dd_normal_matvec(self._h, _dptr(x), _dptr(z)), "rann_dd_normal_matvec")
        return z

    def precond_apply(self, r, z=None):
        z = z if z is not None else self._empty(self.sizes()["dof"])
        _check(self._lib.rann_dd_precond_apply(self._h, _dptr(r), _dptr(z)), "rann_dd_precond_apply")
        return z

    def precond_apply_multi(self, R, Z=None):
        """Z[c] = M^{-1} R[c] for the rows of R ([nrhs][DoF], device float64)."""
        Z = Z if Z is not None else self._empty(R.numel()).reshape(R.shape)
        _check(self._lib.rann_dd_precond_apply_multi(self._h, _dptr(R), _dptr(Z), int(R.shape[0])),
               "rann_dd_precond_apply_multi")
        return Z

    def precond_apply_t(self, r, z=None):
        z = z if z is not None else self._empty(self.sizes()["dof"])
        _check(self._lib.rann_dd_precond_apply_t(self._h, _dptr(r), _dptr(z)), "rann_dd_precond_apply_t")
        return z

    def inject_fault(self, kind: int, value: int):
        """Host-side fault injection (rann_dd_inject_fault): FAULT_WAIT_EXPIRED
        sets the device error word of the tensor-core pipelines; FAULT_ALLOC_CAP
        caps the handle's live device bytes (value < 0 removes the cap)."""
        _check(self._lib.rann_dd_inject_fault(self._h, kind, int(value)), "rann_dd_inject_fault")

    # -- kernel accounting ------------------------------------------------
    def profile(self, on: bool = True):
        _check(self._lib.rann_dd_profile_enable(self._h, int(on)), "rann_dd_profile_enable")

    def profile_read(self):
        """Per kernel family: launches, device ms, algorithmic bytes and flops, and
        the roofline class ("hbm", "alu" = float64 pipe, "tensor" = bf16 digit-slice
        products, "alu_df32" = double-float on the float32 pipe)."""
        out = {}
        i = 0
        while True:
            name, n, ms, nb, nf, bd = ctypes.c_char_p(), _L(), _D(), _D(), _D(), _I()
            if self._lib.rann_dd_profile_get(self._h, i, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms),
                                             ctypes.byref(nb), ctypes.byref(nf), ctypes.byref(bd)) != OK:
                break
            out[name.value.decode()] = {"launches": n.value, "ms": ms.value, "bytes": nb.value,
                                        "flops": nf.value, "bound": BOUND_NAMES.get(bd.value, "alu")}
            i += 1
        return out

    # -- inspection -------------------------------------------------------
    def block(self, j: int, which: int):
        nr, nc = _L(), _I()
        _check(self._lib.rann_dd_block_info(self._h, j, ctypes.byref(nr), ctypes.byref(nc)), "rann_dd_block_info")
        cols = self.problem.neurons if which < 2 else nc.value
        out = np.empty((nr.value, cols))
        rows = np.empty(nr.value, dtype=np.int64)
        _check(self._lib.rann_dd_get_block(self._h, j, which, out.ctypes.data, rows.ctypes.data), "rann_dd_get_block")
        return rows, out

    def pca_of(self, j: int):
        m = self.problem.neurons
        eig = np.empty(m)
        p = int(self.ranks[j])
        V = np.empty((m, p))
        _check(self._lib.rann_dd_get_pca(self._h, j, eig.ctypes.data, V.ctypes.data), "rann_dd_get_pca")
        return eig, V


class LeastSquaresSolve:
    """Differentiable solve W(F) = (H^T H)^{-1} H^T F of a prepared RannDD
    (assembled, reduced, preconditioner set up): torch.autograd support for
    gradients with respect to the right-hand side F.  The backward pass solves
    the adjoint system with the same preconditioner (rann_dd_solve_backward)
    and returns dl/dF = H lam."""

    @staticmethod
    def apply(solver: "RannDD", F, rtol: float = 1e-10, maxit: int = 2000):
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, Fin):
                W, _ = solver.solve(Fin.detach().contiguous(), rtol, maxit)
                return W

            @staticmethod
            def backward(ctx, gW):
                lam, _ = solver.solve_backward(gW.contiguous(), rtol, maxit)
                return solver.matvec(lam)

        return _Fn.apply(F)


class PiecewiseDiffusionSolve:
    """Differentiable forward solve of -div(a grad u) = f with the piecewise
    coefficient a = sum_c a_c s_c: W(a, F), with torch.autograd support for
    both arguments.  forward sets the coefficient values on the handle and
    runs Algorithm 1 (assemble, PCA, Schwarz set-up, the preconditioned solve
    of the given kind); backward solves the adjoint system with the same
    preconditioner (rann_dd_solve_backward) and returns dl/dF = H lam and
    dl/da = rann_dd_grad_coef (the PCA basis does not depend on a).  The
    collocation right-hand side F is an input: with G = 0 (homogeneous
    Dirichlet data) F = f does not depend on a; otherwise F must be the
    library's rann_dd_rhs for the current a, whose dependence on a through
    A[G] grad_coef includes."""

    @staticmethod
    def apply(solver: "RannDD", a, F, kind: str = "ras", rtol: float = 1e-10, maxit: int = 2000,
              pca_mode: int = PCA_VARIANCE, pca_thr: float = 1e-12):
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, a_in, F_in):
                solver.set_coef(a_in.detach().cpu().numpy())
                solver.assemble()
                solver.pca(pca_mode, pca_thr)
                solver.setup_precond(kind)
                Fc = F_in.detach().contiguous()
                W, _ = solver.solve(Fc, rtol, maxit)
                ctx.save_for_backward(Fc, W)
                return W

            @staticmethod
            def backward(ctx, gW):
                Fc, W = ctx.saved_tensors
                lam, _ = solver.solve_backward(gW.contiguous(), rtol, maxit)
                ga = torch.tensor(solver.grad_coef(Fc, W, lam), dtype=torch.float64)
                return ga, solver.matvec(lam)

        return _Fn.apply(a, F)


class GridEval:
    """u_hat at the collocation points as a differentiable function of W:
    forward rann_dd_eval at the grid, backward the adjoint rann_dd_eval_grid_t
    (for misfits ||u_hat - u_obs||^2 on the grid)."""

    @staticmethod
    def apply(solver: "RannDD", W):
        import torch
        X = solver.points()

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, W_in):
                return solver.eval(W_in.detach().contiguous(), X)

            @staticmethod
            def backward(ctx, gu):
                return solver.eval_grid_t(gu.contiguous())

        return _Fn.apply(W)


def device_rates():
    """Measured (df32, fp64) TFLOP/s of this device (rann_dd_device_rates)."""
    lib = load_library()
    a, b = _D(), _D()
    _check(lib.rann_dd_device_rates(ctypes.byref(a), ctypes.byref(b)), "rann_dd_device_rates")
    return a.value, b.value


APPLY_NCFG = 4
SOLVER_CG, SOLVER_GMRES = 0, 1


class Batch:
    """Many instances through the whole path at once (rann_dd_batch_run): a pool
    of native worker threads, one CUDA stream each; instances of any grid size
    overlap on the device.  run() takes RannDD handles (fresh or assembled) and
    returns one dict per instance: F, W (dof entries), the statistics, the
    Schwarz apply configuration used and, with u_obs given, the misfit
    l = ||u_hat - u_obs||^2 with dl/dF and dl/da_c."""

    def __init__(self, nworkers: int = 8):
        self._lib = load_library()
        b = ctypes.c_void_p()
        _check(self._lib.rann_dd_batch_create(int(nworkers), ctypes.byref(b)), "rann_dd_batch_create")
        self._b = b

    def close(self):
        if getattr(self, "_b", None):
            self._lib.rann_dd_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, handles, pca_mode, pca_thr, prec="ras", solver=SOLVER_GMRES, rtol=1e-10, restart=50,
            maxit=3000, autotune=False, u_obs=None, allow_not_converged=True):
        import torch
        n = len(handles)
        cfg = Pipeline(int(pca_mode), float(pca_thr), PREC_BY_NAME[prec] if isinstance(prec, str) else int(prec),
                       int(solver), float(rtol), int(restart), int(maxit), int(bool(autotune)), int(u_obs is not None))
        sizes = [h.sizes() for h in handles]
        F = [torch.empty(sz["n_points"], dtype=torch.float64, device="cuda") for sz in sizes]
        W = [torch.empty(sz["J"] * sz["m"], dtype=torch.float64, device="cuda") for sz in sizes]
        gF = [torch.empty(sz["n_points"], dtype=torch.float64, device="cuda") for sz in sizes] if u_obs is not None else None
        ncell = [h.problem.coef_grid ** 2 if getattr(h.problem, "coef", 0) == 2 else 0 for h in handles]
        gc = [np.zeros(max(c, 1)) for c in ncell]
        arr = lambda xs: (_P * max(n, 1))(*[_dptr(x) for x in xs])
        hs = (_P * max(n, 1))(*[h._h.value for h in handles])
        out = (PipelineOut * max(n, 1))()
        uo = arr(u_obs) if u_obs is not None else None
        gfp = arr(gF) if gF is not None else None
        gcp = (_P * max(n, 1))(*[g.ctypes.data if c else None for g, c in zip(gc, ncell)])
        torch.cuda.synchronize()
        s = self._lib.rann_dd_batch_run(self._b, n, hs, ctypes.byref(cfg), arr(F), arr(W), uo, gfp,
                                        gcp if u_obs is not None else None, out)
        _check(s, "rann_dd_batch_run", allow=(NOT_CONVERGED,) if allow_not_converged else ())
        res = []
        for k in range(n):
            o = out[k]
            if o.status != OK and not (allow_not_converged and o.status == NOT_CONVERGED):
                raise RannError(o.status, f"batch instance {k}")
            h = handles[k]
            nr, nc = _L(), _I()
            rk = []
            for j in range(sizes[k]["J"]):
                _check(self._lib.rann_dd_block_info(h._h, j, ctypes.byref(nr), ctypes.byref(nc)), "rann_dd_block_info")
                rk.append(nc.value)
            h.ranks = np.array(rk, dtype=np.int64)
            r = {"status": STATUS.get(o.status, o.status), "dof": int(o.dof), "apply_config": int(o.apply_config),
                 "F": F[k], "W": W[k][: int(o.dof)], "forward": o.forward.as_dict()}
            if u_obs is not None:
                r.update({"loss": float(o.loss), "adjoint": o.adjoint.as_dict(), "grad_F": gF[k],
                          "grad_coef": gc[k][: ncell[k]].copy() if ncell[k] else None})
            res.append(r)
        return res
