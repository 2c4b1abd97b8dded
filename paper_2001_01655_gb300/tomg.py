"""ctypes binding of the tomg C ABI (include/tomg.h): argument marshalling only.

Every step of the solve runs in the CUDA library ``_build/libtomg.so``; this module converts
numpy arrays (host) and torch CUDA tensors (device) to pointers and raises on error statuses.
There is no fallback: if the library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libtomg.so")

OK, NOT_CONVERGED, E_INVALID, E_OOM, E_CUDA, E_BREAKDOWN, E_TIMEOUT, E_BUDGET = 0, 1, -1, -2, -3, -4, -5, -6
PC = {"gmg": 0, "amg": 1, "hybrid": 2, "jacobi": 3}
PREC = {"fp64": 0, "fp32": 1, "tc": 2, "tf32x3": 2}
SMOOTHER = {"jacobi": 0, "chebyshev": 1, "gmres": 2}
KRYLOV = {"cg": 0, "fgmres": 1}


class TomgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("tomg status %d: %s" % (status, msg))
        self.status = status


class Options(C.Structure):
    _fields_ = [("pc", C.c_int), ("prec", C.c_int), ("rtol", C.c_double), ("max_iter", C.c_int),
                ("n_levels", C.c_int), ("max_coarse_dofs", C.c_int), ("n_geo_levels", C.c_int),
                ("smoother", C.c_int), ("omega", C.c_double), ("n_pre", C.c_int),
                ("n_post", C.c_int), ("soc_beta", C.c_double), ("check_every", C.c_int),
                ("use_graph", C.c_int), ("max_levels", C.c_int), ("concurrency", C.c_int),
                ("cheb_degree", C.c_int), ("cheb_lower", C.c_double), ("cheb_upper", C.c_double),
                ("adaptive_geo", C.c_int), ("adaptive_iters", C.c_int), ("adaptive_min_geo", C.c_int),
                ("krylov", C.c_int), ("gmres_restart", C.c_int),
                ("gmres_steps", C.c_int), ("block_rhs", C.c_int),
                ("fp64_tc", C.c_int), ("fuse_transfers", C.c_int)]


class Result(C.Structure):
    _fields_ = [("iterations", C.c_int), ("rel_residual", C.c_double), ("compliance", C.c_double),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double), ("status", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LevelInfo(C.Structure):
    _fields_ = [("kind", C.c_int), ("block", C.c_int), ("n_nodes", C.c_int64),
                ("n_dofs", C.c_int64), ("nnzb", C.c_int64), ("nx", C.c_int), ("ny", C.c_int),
                ("nz", C.c_int), ("geometric", C.c_int)]


_lib = None
_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)

_SIGS = {
    "tomg_last_error": (C.c_char_p, []),
    "tomg_options_default": (None, [C.POINTER(Options)]),
    "tomg_ctx_create": (C.c_int, [C.POINTER(_P), C.c_int, _P]),
    "tomg_ctx_destroy": (C.c_int, [_P]),
    "tomg_kernel_launches": (C.c_int, [_P, _I64]),
    "tomg_problem_create": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                      C.c_double, C.c_double, C.c_double, C.POINTER(_P)]),
    "tomg_problem_destroy": (C.c_int, [_P]),
    "tomg_problem_sizes": (C.c_int, [_P, _I64, _I64, _I64]),
    "tomg_set_fixed_dofs": (C.c_int, [_P, _I64, C.c_int64]),
    "tomg_set_density": (C.c_int, [_P, _P, C.c_int]),
    "tomg_setup": (C.c_int, [_P, C.POINTER(Options)]),
    "tomg_solve": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, C.POINTER(Result)]),
    "tomg_num_levels": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "tomg_level_info_get": (C.c_int, [_P, C.c_int, C.POINTER(LevelInfo)]),
    "tomg_level_export": (C.c_int, [_P, C.c_int, _I64, _P, _P, _P]),
    "tomg_prolongation_export": (C.c_int, [_P, C.c_int, _I64, _P, _P, _P]),
    "tomg_aggregates_export": (C.c_int, [_P, C.c_int, _P]),
    "tomg_block_diag_inv_export": (C.c_int, [_P, C.c_int, _P]),
    "tomg_level_apply": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, C.c_int]),
    "tomg_vcycle": (C.c_int, [_P, _P, _P, C.c_int]),
    "tomg_outer_apply": (C.c_int, [_P, _P, _P, C.c_int]),
    "tomg_coarse_solve": (C.c_int, [_P, _P, _P, C.c_int]),
    "tomg_moduli": (C.c_int, [_P, _P, C.c_int]),
    "tomg_element_stiffness": (C.c_int, [_P, _P]),
    "tomg_time_fine_operator": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, _D]),
    "tomg_fine_apply_f32_noalloc": (C.c_int, [_P, _P, _P]),
    "tomg_adaptive_geo_levels": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "tomg_density_filter": (C.c_int, [_P, C.c_double, C.c_int, _P, _P, C.c_int]),
    "tomg_compliance_sensitivity": (C.c_int, [_P, _P, _P, C.c_int]),
    "tomg_stress_stiffness_apply": (C.c_int, [_P, _P, _P, _P, C.c_int]),
    "tomg_buckling_adjoint_rhs": (C.c_int, [_P, C.c_int, _P, _P, C.c_int]),
    "tomg_buckling_sensitivity": (C.c_int, [_P, _P, C.c_int, _P, _P, _P, C.c_double, _P, _P, _P,
                                            C.c_int]),
    "tomg_buckling": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, _P, _P,
                                C.c_int, C.POINTER(C.c_int)]),
    "tomg_server_create": (C.c_int, [_P, C.c_size_t, C.c_int, C.POINTER(_P)]),
    "tomg_server_submit": (C.c_int, [_P, _P, _P, C.c_int, _P, _P, C.POINTER(Options),
                                     C.POINTER(C.c_uint64)]),
    "tomg_server_wait": (C.c_int, [_P, C.c_uint64, C.c_int, C.POINTER(Result)]),
    "tomg_server_stats": (C.c_int, [_P, _D, _D, _D, _I64, C.POINTER(C.c_int),
                                    C.POINTER(C.c_size_t)]),
    "tomg_server_retire": (C.c_int, [_P, _P, C.c_int]),
    "tomg_debug_tc_wait_limit": (C.c_int, [C.c_int]),
    "tomg_debug_grid_wait_limit": (C.c_int, [C.c_int]),
    "tomg_server_destroy": (C.c_int, [_P]),
}


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("tomg CUDA library not built (%s); run paper_2001_01655_gb300.build" % path)
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st, allow_not_converged=True):
    if st == OK or (allow_not_converged and st == NOT_CONVERGED):
        return st
    raise TomgError(st, load().tomg_last_error().decode())


def default_options(**kw) -> Options:
    o = Options()
    load().tomg_options_default(C.byref(o))
    for k, v in kw.items():
        if k == "pc" and isinstance(v, str):
            v = PC[v]
        if k == "prec" and isinstance(v, str):
            v = PREC[v]
        if k == "smoother" and isinstance(v, str):
            v = SMOOTHER[v]
        if k == "krylov" and isinstance(v, str):
            v = KRYLOV[v]
        setattr(o, k, v)
    return o


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype):
    """(pointer, on_device, keepalive) for a numpy array or a torch tensor."""
    if _is_torch(a):
        import torch
        want = torch.float64 if dtype == np.float64 else torch.int64
        if a.dtype != want or not a.is_contiguous():
            raise TypeError("expected a contiguous %s tensor" % want)
        return C.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return C.c_void_p(arr.ctypes.data), 0, arr


class Context:
    """A device and a stream; ``stream`` may be a torch.cuda.Stream or a raw handle."""

    def __init__(self, device: int = 0, stream=None):
        lib = load()
        h = C.c_void_p()
        raw = None
        if stream is not None:
            raw = C.c_void_p(getattr(stream, "cuda_stream", stream))
        _check(lib.tomg_ctx_create(C.byref(h), device, raw))
        self.h = h
        self.device = device

    def kernel_launches(self) -> int:
        v = C.c_int64()
        _check(load().tomg_kernel_launches(self.h, C.byref(v)))
        return v.value

    def close(self):
        if self.h:
            load().tomg_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Problem:
    """SIMP elasticity problem on a structured grid (Sec. 2.1)."""

    def __init__(self, ctx: Context, dim, nx, ny, nz=1, E0=1.0, Emin=1e-9, penal=3.0, nu=0.3):
        lib = load()
        h = C.c_void_p()
        _check(lib.tomg_problem_create(ctx.h, dim, nx, ny, nz, E0, Emin, penal, nu, C.byref(h)))
        self.h, self.ctx = h, ctx
        self.dim, self.nx, self.ny, self.nz = dim, nx, ny, nz
        n, nn, ne = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib.tomg_problem_sizes(h, C.byref(n), C.byref(nn), C.byref(ne)))
        self.n, self.nn, self.nel = n.value, nn.value, ne.value
        self.last_results = []

    @classmethod
    def from_workload(cls, ctx, p):
        """Create from a :class:`workloads.Problem` (density and fixed DOFs set)."""
        P = cls(ctx, p.dim, p.nx, p.ny, p.nz, p.E0, p.Emin, p.penal, p.nu)
        P.set_fixed_dofs(p.fixed)
        P.set_density(p.rho)
        return P

    def close(self):
        if getattr(self, "h", None):
            load().tomg_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fixed_dofs(self, dofs):
        a = np.ascontiguousarray(np.asarray(dofs, dtype=np.int64).ravel())
        _check(load().tomg_set_fixed_dofs(self.h, a.ctypes.data_as(_I64), len(a)))

    def set_density(self, rho):
        p, dev, keep = _ptr(rho, np.float64)
        if not dev and np.asarray(keep).size != self.nel:
            raise ValueError("density has %d entries, expected %d" % (np.asarray(keep).size, self.nel))
        _check(load().tomg_set_density(self.h, p, dev))

    def setup(self, opt: Options | None = None, **kw):
        o = opt if opt is not None else default_options(**kw)
        _check(load().tomg_setup(self.h, C.byref(o)))
        self.opt = o

    def solve(self, f, u0=None, out=None):
        """Solve for right-hand sides f: numpy (nrhs, n) / (n,) on the host, or a torch tensor of
        the same shape (on the device, or on the host, e.g. in pinned memory).  Returns
        (u, [result dicts]); u has f's shape and kind.  With out (a contiguous float64 tensor or
        array of f's shape and kind) the solve starts from out and writes u into it, with no
        copy on the Python side (pinned host buffers stay pinned)."""
        if out is not None:
            nrhs = 1 if len(tuple(out.shape)) == 1 else out.shape[0]
            u = out
        elif _is_torch(f):
            import torch
            nrhs = 1 if f.dim() == 1 else f.shape[0]
            u = torch.zeros_like(f) if u0 is None else u0.clone().contiguous()
        else:
            f = np.ascontiguousarray(f, dtype=np.float64)
            nrhs = 1 if f.ndim == 1 else f.shape[0]
            u = np.zeros_like(f) if u0 is None else np.array(u0, dtype=np.float64, copy=True)
        fp, dev, keepf = _ptr(f, np.float64)
        up, udev, keepu = _ptr(u, np.float64)
        if out is not None and (udev != dev or keepu is not u):
            raise TypeError("out must be a contiguous float64 buffer on the same side as f")
        res = (Result * max(nrhs, 1))()
        st = load().tomg_solve(self.h, nrhs, fp, up, dev, res)
        _check(st)
        self.last_results = [res[i].as_dict() for i in range(nrhs)]
        return u, self.last_results

    # ---- introspection / single steps --------------------------------------------------
    def num_levels(self):
        v = C.c_int()
        _check(load().tomg_num_levels(self.h, C.byref(v)))
        return v.value

    def adaptive_geo_levels(self):
        """Geometric levels the next setup of an adaptive hybrid hierarchy will use (0: none yet)."""
        v = C.c_int()
        _check(load().tomg_adaptive_geo_levels(self.h, C.byref(v)))
        return v.value

    def level_info(self, level):
        li = LevelInfo()
        _check(load().tomg_level_info_get(self.h, level, C.byref(li)))
        return {k: getattr(li, k) for k, _ in li._fields_}

    def _bsr_export(self, fn, level, rows_blocks, br, bc):
        import scipy.sparse as sp
        nnzb = C.c_int64()
        _check(fn(self.h, level, C.byref(nnzb), None, None, None))
        nb = nnzb.value
        rp = np.zeros(rows_blocks + 1, np.int64)
        ci = np.zeros(max(nb, 1), np.int64)
        val = np.zeros(max(nb, 1) * br * bc)
        _check(fn(self.h, level, C.byref(nnzb), C.c_void_p(rp.ctypes.data),
                  C.c_void_p(ci.ctypes.data), C.c_void_p(val.ctypes.data)))
        return rp, ci[:nb], val[:nb * br * bc].reshape(nb, br, bc)

    def level_matrix(self, level):
        """Level operator as a scipy CSR matrix (FP64)."""
        import scipy.sparse as sp
        li = self.level_info(level)
        b, nn = li["block"], li["n_nodes"]
        rp, ci, val = self._bsr_export(load().tomg_level_export, level, nn, b, b)
        return sp.bsr_matrix((val, ci, rp), shape=(nn * b, nn * b)).tocsr()

    def prolongation(self, level):
        import scipy.sparse as sp
        li, lc = self.level_info(level), self.level_info(level + 1)
        b, bc, nn = li["block"], lc["block"], li["n_nodes"]
        rp, ci, val = self._bsr_export(load().tomg_prolongation_export, level, nn, b, bc)
        return sp.bsr_matrix((val, ci, rp), shape=(nn * b, lc["n_nodes"] * bc)).tocsr()

    def block_diag_inv(self, level):
        """The smoother's inverse diagonal blocks of `level`: (n_nodes, block, block), FP64."""
        li = self.level_info(level)
        b, nn = li["block"], li["n_nodes"]
        d = np.zeros((nn, b, b))
        _check(load().tomg_block_diag_inv_export(self.h, level, C.c_void_p(d.ctypes.data)))
        return d

    def aggregates(self, level):
        li = self.level_info(level)
        a = np.zeros(li["n_nodes"], np.int64)
        _check(load().tomg_aggregates_export(self.h, level, C.c_void_p(a.ctypes.data)))
        return a

    def _vec_call(self, fn, x, n_out, *pre):
        if _is_torch(x):
            import torch
            y = torch.zeros(n_out, dtype=torch.float64, device=x.device)
        else:
            x = np.ascontiguousarray(x, dtype=np.float64)
            y = np.zeros(n_out)
        xp, dev, keepx = _ptr(x, np.float64)
        yp, _, keepy = _ptr(y, np.float64)
        _check(fn(self.h, *pre, xp, yp, dev))
        return y

    def level_apply(self, level, x, prec="fp64"):
        li = self.level_info(level)
        return self._vec_call(load().tomg_level_apply, x, li["n_dofs"], level, PREC.get(prec, prec))

    def outer_apply(self, x):
        """y = K x as the outer Krylov loop of the current setup computes it."""
        return self._vec_call(load().tomg_outer_apply, x, self.n)

    def vcycle(self, r):
        return self._vec_call(load().tomg_vcycle, r, self.n)

    def coarse_solve(self, b):
        nl = self.num_levels()
        return self._vec_call(load().tomg_coarse_solve, b, self.level_info(nl - 1)["n_dofs"])

    def moduli(self):
        E = np.zeros(self.nel)
        _check(load().tomg_moduli(self.h, C.c_void_p(E.ctypes.data), 0))
        return E

    def density_filter(self, a, radius=1.5, transpose=False, out=None):
        """rho = S a (or S^T a): the linear density filter of the problem's grid.  numpy in,
        numpy out; or CUDA tensors (device path; `out` a tensor of n_elems doubles)."""
        src, dev, keep = _ptr(a, np.float64)
        if dev:
            import torch
            out = torch.empty_like(a) if out is None else out
            dst, _, _ = _ptr(out, np.float64)
        else:
            out = np.zeros(self.nel)
            dst = C.c_void_p(out.ctypes.data)
        _check(load().tomg_density_filter(self.h, float(radius), int(bool(transpose)), src, dst,
                                          dev))
        return out

    def compliance_sensitivity(self, u, out=None):
        """dF/drho for the current density and displacements u (n_dofs): numpy, or CUDA
        tensors (device path)."""
        if not _is_torch(u):
            u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        src, dev, keep = _ptr(u, np.float64)
        if dev:
            import torch
            out = torch.empty(self.nel, dtype=torch.float64, device=u.device) if out is None else out
            dst, _, _ = _ptr(out, np.float64)
        else:
            out = np.zeros(self.nel)
            dst = C.c_void_p(out.ctypes.data)
        _check(load().tomg_compliance_sensitivity(self.h, src, dst, dev))
        return out

    def stress_stiffness_apply(self, u, x):
        """y = K_sigma(u) x (host arrays)."""
        uu = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        xx = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        y = np.zeros(self.n)
        _check(load().tomg_stress_stiffness_apply(self.h, C.c_void_p(uu.ctypes.data),
                                                  C.c_void_p(xx.ctypes.data),
                                                  C.c_void_p(y.ctypes.data), 0))
        return y

    def buckling(self, u, n_eig=6, j_min=10, j_max=25, tol=1e-6, max_iter=1000, modes=False):
        """The n_eig largest eigenvalues of K_sigma Phi = lambda K Phi (and the K-orthonormal
        modes, n_eig x n_dofs, if requested) by generalized Davidson.  u: numpy, or a CUDA
        tensor (device path: the modes come back as a CUDA tensor).  Returns
        (lambdas, modes or None, iterations, status)."""
        if not _is_torch(u):
            u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        pu, dev, _ = _ptr(u, np.float64)
        lam = np.zeros(n_eig)
        Phi, pm = None, None
        if modes:
            if dev:
                import torch
                Phi = torch.empty((n_eig, self.n), dtype=torch.float64, device=u.device)
                pm = _ptr(Phi, np.float64)[0]
            else:
                Phi = np.zeros((n_eig, self.n))
                pm = C.c_void_p(Phi.ctypes.data)
        it = C.c_int()
        st = load().tomg_buckling(self.h, pu, n_eig, j_min, j_max, float(tol), max_iter,
                                  C.c_void_p(lam.ctypes.data), pm, dev, C.byref(it))
        _check(st)
        return lam, Phi, it.value, st

    def buckling_adjoint_rhs(self, modes):
        """g_k = Phi_k^T (dK_sigma/du) Phi_k for the modes (n_modes x n_dofs, numpy or a CUDA
        tensor): the right-hand sides of the stability adjoint equations, same shape and kind."""
        if not _is_torch(modes):
            modes = np.ascontiguousarray(np.atleast_2d(modes), dtype=np.float64)
        src, dev, keep = _ptr(modes, np.float64)
        if dev:
            import torch
            g = torch.empty_like(modes)
            dst, _, _ = _ptr(g, np.float64)
        else:
            g = np.zeros_like(modes)
            dst = C.c_void_p(g.ctypes.data)
        _check(load().tomg_buckling_adjoint_rhs(self.h, int(modes.shape[0]), src, dst, dev))
        return g

    def buckling_sensitivity(self, u, lambdas, modes, adjoints, pnorm=8.0, per_mode=True):
        """dlambda_k/drho (n_modes x n_elems, if per_mode), dF/drho (n_elems) and F for the
        p-norm aggregate F = (sum lambda_k^p)^(1/p) of the buckling eigenvalues, from the
        displacements u, the K-normalised modes and the adjoint solutions (n_modes x n_dofs).
        numpy arrays, or CUDA tensors for u, modes and adjoints (device path).  Returns
        (dlambda or None, dF, F)."""
        lam = np.ascontiguousarray(lambdas, dtype=np.float64).reshape(-1)
        nm = lam.size
        if not _is_torch(u):
            u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
            modes = np.ascontiguousarray(np.atleast_2d(modes), dtype=np.float64)
            adjoints = np.ascontiguousarray(np.atleast_2d(adjoints), dtype=np.float64)
        pu, dev, _ = _ptr(u, np.float64)
        pm, dm, _ = _ptr(modes, np.float64)
        pa, da, _ = _ptr(adjoints, np.float64)
        if not (dev == dm == da):
            raise TypeError("u, modes and adjoints must all be numpy arrays or all CUDA tensors")
        if tuple(modes.shape) != (nm, self.n) or tuple(adjoints.shape) != (nm, self.n):
            raise ValueError("modes and adjoints must be n_modes x n_dofs")
        if dev:
            import torch
            dl = torch.empty((nm, self.nel), dtype=torch.float64, device=u.device) if per_mode else None
            dF = torch.empty(self.nel, dtype=torch.float64, device=u.device)
            pdl = _ptr(dl, np.float64)[0] if per_mode else None
            pdf = _ptr(dF, np.float64)[0]
        else:
            dl = np.zeros((nm, self.nel)) if per_mode else None
            dF = np.zeros(self.nel)
            pdl = C.c_void_p(dl.ctypes.data) if per_mode else None
            pdf = C.c_void_p(dF.ctypes.data)
        F = C.c_double()
        _check(load().tomg_buckling_sensitivity(self.h, pu, nm, C.c_void_p(lam.ctypes.data), pm, pa,
                                                float(pnorm), pdl, pdf, C.byref(F), dev))
        return dl, dF, F.value

    def fine_apply_f32_noalloc(self, x, y):
        """y = A_0 x in FP32 arithmetic without any device allocation (x, y: contiguous float64
        CUDA tensors of n_dofs entries).  Asynchronous on the context stream."""
        xp, dx, _ = _ptr(x, np.float64)
        yp, dy, _ = _ptr(y, np.float64)
        if not (dx and dy):
            raise TypeError("x and y must be CUDA tensors")
        _check(load().tomg_fine_apply_f32_noalloc(self.h, xp, yp))
        return y

    def time_fine_operator(self, op="apply", prec="fp32", reps=50, cold_l2=True):
        """Mean device time (ms) of one launch of the level-0 operator kernel."""
        ms = C.c_double()
        opi = {"apply": 0, "residual": 1, "jacobi": 2, "outer": 3}[op]
        _check(load().tomg_time_fine_operator(self.h, opi, PREC.get(prec, prec), reps,
                                              1 if cold_l2 else 0, C.byref(ms)))
        return ms.value

    def element_stiffness(self):
        nd = self.dim * (1 << self.dim)
        Ke = np.zeros((nd, nd))
        _check(load().tomg_element_stiffness(self.h, C.c_void_p(Ke.ctypes.data)))
        return Ke


def debug_tc_wait_limit(polls: int):
    """Shorten the tensor-core kernel's MMA waits (tomg_debug_tc_wait_limit; 0 = default)."""
    _check(load().tomg_debug_tc_wait_limit(int(polls)))


def debug_grid_wait_limit(polls: int):
    """Shorten the grid-barrier waits of the cooperative setup kernels
    (tomg_debug_grid_wait_limit; 0 = default)."""
    _check(load().tomg_debug_grid_wait_limit(int(polls)))


class Server:
    """Continuous-batching request loop over many problems (tomg_server_*)."""

    def __init__(self, ctx: Context, hbm_budget_bytes: int, max_slots: int = 4):
        h = C.c_void_p()
        _check(load().tomg_server_create(ctx.h, C.c_size_t(int(hbm_budget_bytes)), max_slots,
                                         C.byref(h)))
        self.h, self.ctx = h, ctx
        self._keep = {}
        self._problems = {}

    def submit(self, problem: Problem, rho, f, u=None, opt: Options | None = None, **kw):
        """Queue one design update; returns a ticket.  rho, f, u: numpy host arrays (copied;
        u receives the solution)."""
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        f = np.ascontiguousarray(f, dtype=np.float64)
        nrhs = 1 if f.ndim == 1 else f.shape[0]
        if u is not None and (u.dtype != np.float64 or not u.flags.c_contiguous):
            raise TypeError("u must be a contiguous float64 array")
        o = opt if opt is not None else default_options(**kw)
        t = C.c_uint64()
        st = load().tomg_server_submit(self.h, problem.h, C.c_void_p(rho.ctypes.data), nrhs,
                                       C.c_void_p(f.ctypes.data),
                                       None if u is None else C.c_void_p(u.ctypes.data),
                                       C.byref(o), C.byref(t))
        _check(st)
        self._keep[t.value] = (rho, f, u, nrhs)
        self._problems[id(problem)] = problem  # problems must outlive the server
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        nrhs = self._keep.get(ticket, (None, None, None, 1))[3]
        res = (Result * nrhs)()
        st = load().tomg_server_wait(self.h, ticket, timeout_ms, res)
        if st == E_TIMEOUT:
            raise TomgError(st, load().tomg_last_error().decode())
        self._keep.pop(ticket, None)
        _check(st)
        return [res[i].as_dict() for i in range(nrhs)]

    def retire(self, problem: Problem, timeout_ms=-1):
        """The client is done with ``problem``: wait for its requests, free its warm start and
        stop counting its device memory (tomg_server_retire)."""
        _check(load().tomg_server_retire(self.h, problem.h, timeout_ms))
        self._problems.pop(id(problem), None)

    def stats(self):
        p50, p99, sps = C.c_double(), C.c_double(), C.c_double()
        done, peak = C.c_int64(), C.c_int()
        pb = C.c_size_t()
        _check(load().tomg_server_stats(self.h, C.byref(p50), C.byref(p99), C.byref(sps),
                                        C.byref(done), C.byref(peak), C.byref(pb)))
        return {"p50_ms": p50.value, "p99_ms": p99.value, "solves_per_s": sps.value,
                "completed": done.value, "peak_active": peak.value, "peak_bytes": pb.value}

    def close(self):
        if getattr(self, "h", None):
            load().tomg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
