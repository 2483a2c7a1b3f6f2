"""Python binding of libwd (argument marshalling only).

Every step of the solver runs in the C/CUDA library ``_build/libwd.so``; this
module converts numpy arrays and torch tensors to pointers, sizes and
streams.  The library is loaded eagerly on first use and its absence is an
error: there is no fallback implementation.

Names follow the C ABI in ``include/wd.h``: analyze -> factor -> solve /
logdet / apply_L.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "_build", "libwd.so")
_lock = threading.Lock()
_lib = None

WD_OK, WD_ERR_INVALID_ARG, WD_ERR_PATTERN, WD_ERR_STATE, WD_ERR_NOT_SPD, WD_ERR_OOM, \
    WD_ERR_CUDA, WD_ERR_TIMEOUT, WD_ERR_NO_CONVERGENCE = range(9)
WD_FP64, WD_MIXED = 0, 1
_PREC = {"fp64": WD_FP64, "mixed": WD_MIXED, WD_FP64: WD_FP64, WD_MIXED: WD_MIXED}

EXPORTED = ["wd_default_options", "wd_create", "wd_destroy", "wd_analyze", "wd_symbolic_export",
            "wd_get_info", "wd_factor", "wd_solve", "wd_logdet", "wd_apply_L", "wd_export_L",
            "wd_status_detail", "wd_status_string", "wd_kernel_stats", "wd_launch_count",
            "wd_selinv", "wd_sym_pattern_outer", "wd_value_gradient", "wd_export_L_noalloc",
            "wd_analyze_batch", "wd_logdet_batch", "wd_backward_error", "wd_theta_step", "wd_set_mass",
            "wd_factor_lu", "wd_solve_lu", "wd_logdet_lu", "wd_export_LU", "wd_factor_ldlt", "wd_inertia",
            "wd_set_level_schedule", "wd_get_level_schedule"]


class WdOptions(ctypes.Structure):
    _fields_ = [("nd_leaf", ctypes.c_int32), ("relax_k", ctypes.c_int32),
                ("relax_pct", ctypes.c_int32), ("ir_max_iter", ctypes.c_int32),
                ("ir_tol", ctypes.c_double), ("use_graphs", ctypes.c_int32),
                ("symbolic_only", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("diag64_min_k", ctypes.c_int32), ("wait_limit", ctypes.c_int32),
                ("test_closed_gate", ctypes.c_int32), ("test_fail_alloc", ctypes.c_int32),
                ("solve_simt", ctypes.c_int32), ("fp64_tc_schur", ctypes.c_int32),
                ("step_launches", ctypes.c_int32)]


class WdGeometry(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("level", ctypes.c_void_p), ("box_lo", ctypes.c_void_p),
                ("box_side", ctypes.c_void_p), ("patch", ctypes.c_void_p)]


class WdInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz_A_lower", ctypes.c_int64), ("nnz_L", ctypes.c_int64),
                ("nnz_L_stored", ctypes.c_int64), ("flops_factor", ctypes.c_double),
                ("nsuper", ctypes.c_int32), ("nlevels", ctypes.c_int32),
                ("max_front", ctypes.c_int32), ("max_width", ctypes.c_int32),
                ("front_bytes", ctypes.c_int64), ("factor_launches", ctypes.c_int64),
                ("analyze_seconds", ctypes.c_double)]


class WdKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int64),
                ("milliseconds", ctypes.c_double), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double)]


class WdSolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("backward_error", ctypes.c_double)]


class WdError(RuntimeError):
    def __init__(self, status, msg, column=-1):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status
        self.column = column


def library_path() -> str:
    return _LIBPATH


def load():
    """Load libwd.so (built by build.py).  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIBPATH):
            raise RuntimeError(f"libwd.so not built ({_LIBPATH}); run build.build() first")
        lib = ctypes.CDLL(_LIBPATH)
        vp, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.wd_default_options.argtypes = [ctypes.POINTER(WdOptions)]
        lib.wd_default_options.restype = None
        lib.wd_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(WdOptions)]
        lib.wd_destroy.argtypes = [vp]
        lib.wd_destroy.restype = None
        lib.wd_analyze.argtypes = [vp, i64, vp, vp, ctypes.POINTER(WdGeometry)]
        lib.wd_symbolic_export.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        lib.wd_get_info.argtypes = [vp, ctypes.POINTER(WdInfo)]
        lib.wd_factor.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp]
        lib.wd_solve.argtypes = [vp, vp, i64, i64, ctypes.c_int, vp, ctypes.POINTER(WdSolveInfo)]
        lib.wd_logdet.argtypes = [vp, ctypes.POINTER(f64)]
        lib.wd_apply_L.argtypes = [vp, vp, vp, i64, i64, ctypes.c_int, vp]
        lib.wd_export_L.argtypes = [vp, vp]
        lib.wd_selinv.argtypes = [vp, vp, ctypes.c_int, vp]
        lib.wd_sym_pattern_outer.argtypes = [vp, vp, vp, i64, i64, vp, ctypes.c_int, vp]
        lib.wd_value_gradient.argtypes = [vp, f64, vp, vp, i64, i64, vp, ctypes.c_int, vp]
        lib.wd_export_L_noalloc.argtypes = [vp, vp, vp]
        lib.wd_analyze_batch.argtypes = [vp, i32, vp, vp, vp, vp]
        lib.wd_logdet_batch.argtypes = [vp, vp]
        lib.wd_backward_error.argtypes = [vp, vp, vp, i64, i64, ctypes.c_int, vp, ctypes.POINTER(f64)]
        lib.wd_theta_step.argtypes = [vp, vp, vp, i64, i64, f64, f64, ctypes.c_int, vp,
                                      ctypes.POINTER(WdSolveInfo)]
        lib.wd_set_mass.argtypes = [vp, vp, ctypes.c_int]
        lib.wd_factor_lu.argtypes = [vp, vp, vp, ctypes.c_int, vp]
        lib.wd_solve_lu.argtypes = [vp, vp, i64, i64, ctypes.c_int, vp]
        lib.wd_logdet_lu.argtypes = [vp, ctypes.POINTER(f64), ctypes.POINTER(i32)]
        lib.wd_export_LU.argtypes = [vp, vp, vp]
        lib.wd_factor_ldlt.argtypes = [vp, vp, ctypes.c_int, vp]
        lib.wd_set_level_schedule.argtypes = [vp, vp, i32]
        lib.wd_get_level_schedule.argtypes = [vp, vp, i32]
        lib.wd_inertia.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.wd_status_detail.argtypes = [vp, ctypes.POINTER(i64), ctypes.c_char_p, ctypes.c_size_t]
        lib.wd_kernel_stats.argtypes = [vp, ctypes.POINTER(WdKernelStat), i32, ctypes.POINTER(i32),
                                        ctypes.c_int]
        lib.wd_launch_count.argtypes = [vp, ctypes.POINTER(i64), ctypes.c_int]
        lib.wd_status_string.argtypes = [ctypes.c_int]
        lib.wd_status_string.restype = ctypes.c_char_p
        for f in ("wd_create", "wd_analyze", "wd_symbolic_export", "wd_get_info", "wd_factor",
                  "wd_solve", "wd_logdet", "wd_apply_L", "wd_export_L", "wd_status_detail",
                  "wd_kernel_stats", "wd_launch_count"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
        return lib


def _status_name(s):
    try:
        return load().wd_status_string(int(s)).decode()
    except Exception:
        return f"status {s}"


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(a):
    """(pointer, on_device) of a numpy array or torch tensor."""
    if _is_torch(a):
        return ctypes.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    return ctypes.c_void_p(a.ctypes.data), 0


def _stream(stream, needed):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    if needed:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


# symbolic defaults (as wd_default_options): nested-dissection leaf size and
# the relaxed amalgamation thresholds (merge a child into its parent while
# the merged width is <= relax_k or the explicit zeros stay <= relax_pct %)
DEFAULTS = {"nd_leaf": 128, "relax_k": 64, "relax_pct": 10}


class Solver:
    """One sparse SPD system: analyze once, factor (re)peatedly, solve many."""

    def __init__(self, nd_leaf=DEFAULTS["nd_leaf"], relax_k=DEFAULTS["relax_k"],
                 relax_pct=DEFAULTS["relax_pct"], ir_max_iter=10, ir_tol=1e-12,
                 symbolic_only=False, profile=False, use_graphs=True, diag64_min_k=None,
                 wait_limit=0, test_closed_gate=False, test_fail_alloc=0, solve_simt=False,
                 fp64_tc_schur=False, step_launches=False):
        self._lib = load()
        o = WdOptions()
        self._lib.wd_default_options(ctypes.byref(o))
        o.nd_leaf, o.relax_k, o.relax_pct = nd_leaf, relax_k, relax_pct
        o.ir_max_iter, o.ir_tol = ir_max_iter, ir_tol
        o.symbolic_only = 1 if symbolic_only else 0
        o.profile = 1 if profile else 0
        o.use_graphs = 1 if use_graphs else 0
        if diag64_min_k is not None:
            o.diag64_min_k = diag64_min_k
        o.wait_limit = wait_limit
        o.test_closed_gate = 1 if test_closed_gate else 0
        o.test_fail_alloc = test_fail_alloc
        o.solve_simt = 1 if solve_simt else 0
        o.fp64_tc_schur = 1 if fp64_tc_schur else 0
        o.step_launches = 1 if step_launches else 0
        # the options that shape the analysis and the factor's launch plan
        self.options = dict(nd_leaf=nd_leaf, relax_k=relax_k, relax_pct=relax_pct,
                            diag64_min_k=o.diag64_min_k, step_launches=o.step_launches)
        self._h = ctypes.c_void_p()
        self._check(self._lib.wd_create(ctypes.byref(self._h), ctypes.byref(o)))
        self.n = None
        self.precision = None

    def close(self):
        if getattr(self, "_h", None):
            self._lib.wd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != WD_OK:
            col = ctypes.c_int64(-1)
            buf = ctypes.create_string_buffer(512)
            if getattr(self, "_h", None):
                self._lib.wd_status_detail(self._h, ctypes.byref(col), buf, 512)
            raise WdError(st, buf.value.decode(errors="replace"), col.value)

    # -- analysis --------------------------------------------------------------
    def analyze(self, colptr, rowidx, basis=None):
        """basis: an object with dim, level, box_lo, box_side (or None)."""
        cp = np.ascontiguousarray(colptr, np.int64)
        ri = np.ascontiguousarray(rowidx, np.int32)
        n = cp.size - 1
        g = None
        keep = []
        if basis is not None:
            lev = np.ascontiguousarray(basis.level, np.int32)
            lo = np.ascontiguousarray(basis.box_lo, np.int32)
            side = np.ascontiguousarray(basis.box_side, np.int32)
            patch = getattr(basis, "patch", None)
            patch = None if patch is None else np.ascontiguousarray(patch, np.int32)
            keep = [lev, lo, side, patch]
            g = WdGeometry(int(basis.dim), lev.ctypes.data, lo.ctypes.data, side.ctypes.data,
                           None if patch is None else patch.ctypes.data)
        self._check(self._lib.wd_analyze(self._h, n, cp.ctypes.data, ri.ctypes.data,
                                         ctypes.byref(g) if g is not None else None))
        del keep
        self.n = n
        self.nnz = int(cp[-1])
        return self

    def analyze_batch(self, patterns, bases=None):
        """Independent instances as one block-diagonal matrix.  patterns: list
        of (colptr, rowidx); bases: list of objects with dim, level, box_lo,
        box_side (or None).  Instances passing the very same arrays share one
        analysis."""
        cnt = len(patterns)
        keep = []
        conv = {}

        def arr(a, dt):
            key = (id(a), dt)
            if key not in conv:
                conv[key] = np.ascontiguousarray(a, dt)
                keep.append(a)
            return conv[key]

        cps = [arr(cp, np.int64) for cp, _ in patterns]
        ris = [arr(ri, np.int32) for _, ri in patterns]
        ns = np.array([c.size - 1 for c in cps], np.int64)
        pcp = (ctypes.c_void_p * cnt)(*[c.ctypes.data for c in cps])
        pri = (ctypes.c_void_p * cnt)(*[r.ctypes.data for r in ris])
        geo = None
        if bases is not None:
            geo = (WdGeometry * cnt)()
            for i, b in enumerate(bases):
                lev, lo, side = arr(b.level, np.int32), arr(b.box_lo, np.int32), arr(b.box_side, np.int32)
                pt = getattr(b, "patch", None)
                pt = None if pt is None else arr(pt, np.int32)
                geo[i] = WdGeometry(int(b.dim), lev.ctypes.data, lo.ctypes.data, side.ctypes.data,
                                    None if pt is None else pt.ctypes.data)
        self._check(self._lib.wd_analyze_batch(self._h, cnt, ns.ctypes.data, pcp, pri, geo))
        del keep
        self.n = int(ns.sum())
        self.nnz = int(sum(int(c[-1]) for c in cps))
        self.batch_sizes = ns
        return self

    def logdet_batch(self) -> np.ndarray:
        out = np.empty(len(self.batch_sizes), np.float64)
        self._check(self._lib.wd_logdet_batch(self._h, ctypes.c_void_p(out.ctypes.data)))
        return out

    def info(self) -> dict:
        i = WdInfo()
        self._check(self._lib.wd_get_info(self._h, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in WdInfo._fields_}

    def symbolic(self) -> dict:
        inf = self.info()
        n, ns = self.n, inf["nsuper"]
        perm = np.empty(n, np.int32)
        parent = np.empty(n, np.int32)
        cc = np.empty(n, np.int64)
        sf = np.empty(ns + 1, np.int32)
        srp = np.empty(ns + 1, np.int64)
        self._check(self._lib.wd_symbolic_export(self._h, perm.ctypes.data, parent.ctypes.data,
                                                 cc.ctypes.data, sf.ctypes.data, srp.ctypes.data,
                                                 None))
        rows = np.empty(max(int(srp[-1]), 1), np.int32)
        self._check(self._lib.wd_symbolic_export(self._h, None, None, None, None, None,
                                                 rows.ctypes.data))
        return dict(perm=perm, parent=parent, colcount=cc, super_first=sf, super_rowptr=srp,
                    super_rows=rows[: int(srp[-1])])

    # -- numeric -----------------------------------------------------------------
    def factor(self, values, precision="fp64", stream=None):
        p, dev = _ptr(values)
        self._check(self._lib.wd_factor(self._h, p, dev, _PREC[precision], _stream(stream, dev)))
        self.precision = precision
        return self

    def solve(self, B, stream=None, with_info=True):
        """Solve A X = B.  A CUDA tensor (n x nrhs, column-major: pass B with
        B.stride(0) == 1, e.g. the transpose of a contiguous (nrhs, n) tensor)
        is overwritten in place; a numpy array gives a new array."""
        info = WdSolveInfo()
        if _is_torch(B):
            if B.dim() == 1:
                B = B.unsqueeze(1)
            if B.stride(0) != 1:
                raise ValueError("B must be column-major (stride(0) == 1)")
            ldb = B.stride(1) if B.shape[1] > 1 else B.shape[0]
            p, dev = _ptr(B)
            self._check(self._lib.wd_solve(self._h, p, B.shape[1], ldb, dev, _stream(stream, dev),
                                           ctypes.byref(info) if with_info else None))
            out = B
        else:
            X = np.array(B, dtype=np.float64, order="F", copy=True)
            if X.ndim == 1:
                X = X[:, None]
            self._check(self._lib.wd_solve(self._h, ctypes.c_void_p(X.ctypes.data), X.shape[1],
                                           X.shape[0], 0, _stream(stream, False),
                                           ctypes.byref(info) if with_info else None))
            out = X
        self.last_solve = {"iterations": info.iterations, "backward_error": info.backward_error}
        return out

    # -- LU without pivoting (nonsymmetric values on the analyzed pattern) ------
    def factor_lu(self, lower, upper, stream=None):
        """P A P^T = L U (FP64, no pivoting).  lower[e] = A[r][c], upper[e] =
        A[c][r] for every stored lower entry e = (r, c)."""
        if _is_torch(lower) != _is_torch(upper):
            raise ValueError("lower and upper must both be numpy arrays or both tensors")
        lo = lower if _is_torch(lower) else np.ascontiguousarray(lower, np.float64)
        up = upper if _is_torch(upper) else np.ascontiguousarray(upper, np.float64)
        if lo.shape[0] != self.nnz or up.shape[0] != self.nnz:
            raise ValueError("one value per stored lower entry of the analyzed pattern")
        pl, dev = _ptr(lo)
        pu, _ = _ptr(up)
        self._check(self._lib.wd_factor_lu(self._h, pl, pu, dev, _stream(stream, dev)))
        self.precision = "lu"
        return self

    def level_schedule(self) -> list:
        """Per elimination-tree level (deepest first): 0 = one launch of
        dependency-ordered tasks for the level's pivot columns, 1 = a
        (panel, update) launch pair per 64-column pivot block."""
        n = self.info()["nlevels"]
        a = np.zeros(max(n, 1), np.int8)
        self._check(self._lib.wd_get_level_schedule(self._h, a.ctypes.data, n))
        return [int(x) for x in a[:n]]

    def set_level_schedule(self, flags):
        a = np.ascontiguousarray(flags, np.int8)
        self._check(self._lib.wd_set_level_schedule(self._h, a.ctypes.data, int(a.size)))
        return self

    def factor_ldlt(self, values, stream=None):
        """P A P^T = L D L^T for a symmetric, possibly indefinite matrix
        (FP64, no pivoting; the LU factorization with U = D L^T).  Solve
        with solve_lu, log |det| with logdet_lu, the inertia with inertia()."""
        v = values if _is_torch(values) else np.ascontiguousarray(values, np.float64)
        if v.shape[0] != self.nnz:
            raise ValueError("one value per stored lower entry of the analyzed pattern")
        p, dev = _ptr(v)
        self._check(self._lib.wd_factor_ldlt(self._h, p, dev, _stream(stream, dev)))
        self.precision = "lu"
        return self

    def inertia(self):
        """(number of positive, number of negative eigenvalues of A) from the
        pivots of the last factor_ldlt."""
        pos = ctypes.c_int64()
        neg = ctypes.c_int64()
        self._check(self._lib.wd_inertia(self._h, ctypes.byref(pos), ctypes.byref(neg)))
        return pos.value, neg.value

    def solve_lu(self, B, stream=None):
        """A^-1 B with the LU factor.  A CUDA tensor (n x nrhs, column-major)
        is overwritten in place; a numpy array gives a new array."""
        if _is_torch(B):
            if B.dim() == 1:
                B = B.unsqueeze(1)
            if B.stride(0) != 1:
                raise ValueError("B must be column-major (stride(0) == 1)")
            self._check(self._lib.wd_solve_lu(self._h, ctypes.c_void_p(B.data_ptr()), B.shape[1], B.stride(1)
                                              if B.shape[1] > 1 else self.n, 1, _stream(stream, True)))
            return B
        X = np.array(B, dtype=np.float64, order="F", copy=True)
        if X.ndim == 1:
            X = X[:, None]
        self._check(self._lib.wd_solve_lu(self._h, ctypes.c_void_p(X.ctypes.data), X.shape[1], self.n, 0,
                                          _stream(stream, False)))
        return X

    def logdet_lu(self):
        """(log |det A|, sign of det A) from the LU factor."""
        v = ctypes.c_double()
        sg = ctypes.c_int32()
        self._check(self._lib.wd_logdet_lu(self._h, ctypes.byref(v), ctypes.byref(sg)))
        return v.value, sg.value

    def export_LU(self):
        """(L, U^T) supernodal panels, each in wd_export_L's layout."""
        size = self._panel_size()
        L = np.empty(size, np.float64)
        Ut = np.empty(size, np.float64)
        self._check(self._lib.wd_export_LU(self._h, L.ctypes.data, Ut.ctypes.data))
        return L, Ut

    def set_mass(self, gvalues=None):
        """The mass matrix G (values on the analyzed lower pattern) used by
        theta_step; None restores G = I."""
        if gvalues is None:
            self._check(self._lib.wd_set_mass(self._h, None, 0))
            return self
        g = gvalues if _is_torch(gvalues) else np.ascontiguousarray(gvalues, np.float64)
        if g.shape[0] != self.nnz:
            raise ValueError("gvalues must hold one value per stored lower entry of the analyzed pattern")
        p, dev = _ptr(g)
        self._check(self._lib.wd_set_mass(self._h, p, dev))
        return self

    def theta_step(self, U, F=None, theta=0.5, dt=1e-2, stream=None):
        """One theta-scheme step with the factored matrix M = I + theta dt K
        (wd_theta_step): U := M^-1 [(1/theta) U - ((1-theta)/theta) M U + dt F].
        A CUDA tensor U (column-major n x nrhs, leading dimension n; F the same
        shape or None) is updated in place; numpy arrays give a new array."""
        info = WdSolveInfo()
        if _is_torch(U):
            if U.dim() == 1:
                U = U.unsqueeze(1)
                F = None if F is None else F.unsqueeze(1)
            n = U.shape[0]
            for t in (U,) if F is None else (U, F):
                if t.stride(0) != 1 or (t.shape[1] > 1 and t.stride(1) != n) or t.shape != U.shape:
                    raise ValueError("U and F must be column-major n x nrhs with leading dimension n")
            pu, dev = _ptr(U)
            pf = None if F is None else _ptr(F)[0]
            self._check(self._lib.wd_theta_step(self._h, pu, pf, U.shape[1], n, float(theta), float(dt), dev,
                                                _stream(stream, dev), ctypes.byref(info)))
            out = U
        else:
            Uc = np.array(U, dtype=np.float64, order="F", copy=True)
            Fc = None if F is None else np.array(F, dtype=np.float64, order="F", copy=True)
            if Uc.ndim == 1:
                Uc = Uc[:, None]
                Fc = None if Fc is None else Fc[:, None]
            if Fc is not None and Fc.shape != Uc.shape:
                raise ValueError("F must have U's shape")
            self._check(self._lib.wd_theta_step(
                self._h, ctypes.c_void_p(Uc.ctypes.data),
                None if Fc is None else ctypes.c_void_p(Fc.ctypes.data), Uc.shape[1], Uc.shape[0],
                float(theta), float(dt), 0, _stream(stream, False), ctypes.byref(info)))
            out = Uc
        self.last_solve = {"iterations": info.iterations, "backward_error": info.backward_error}
        return out

    def backward_error(self, X, B, stream=None) -> float:
        """max over columns of ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)
        (numpy arrays or column-major CUDA tensors with leading dimension n)."""
        be = ctypes.c_double()
        if _is_torch(X):
            if X.dim() == 1:
                X, B = X.unsqueeze(1), B.unsqueeze(1)
            n = X.shape[0]
            for t in (X, B):
                if t.stride(0) != 1 or (t.shape[1] > 1 and t.stride(1) != n) or t.shape != X.shape:
                    raise ValueError("X and B must be column-major n x nrhs with leading dimension n")
            px, dev = _ptr(X)
            pb, _ = _ptr(B)
            self._check(self._lib.wd_backward_error(self._h, px, pb, X.shape[1], n, dev,
                                                    _stream(stream, dev), ctypes.byref(be)))
            return be.value
        Xc = np.array(X, dtype=np.float64, order="F", copy=True)
        Bc = np.array(B, dtype=np.float64, order="F", copy=True)
        if Xc.ndim == 1:
            Xc, Bc = Xc[:, None], Bc[:, None]
        self._check(self._lib.wd_backward_error(self._h, ctypes.c_void_p(Xc.ctypes.data),
                                                ctypes.c_void_p(Bc.ctypes.data), Xc.shape[1], Xc.shape[0],
                                                0, _stream(stream, False), ctypes.byref(be)))
        return be.value

    def logdet(self) -> float:
        v = ctypes.c_double()
        self._check(self._lib.wd_logdet(self._h, ctypes.byref(v)))
        return v.value

    def apply_L(self, Z, S=None, stream=None):
        """S = P^T L Z (Z in factor order).  Torch CUDA tensors (column-major)
        or numpy arrays."""
        if _is_torch(Z):
            import torch
            if Z.dim() == 1:
                Z = Z.unsqueeze(1)
            if S is None:
                S = torch.empty((Z.shape[1], Z.shape[0]), dtype=torch.float64, device=Z.device).T
            pz, dev = _ptr(Z)
            ps, _ = _ptr(S)
            ld = Z.shape[0]
            if Z.stride(0) != 1 or S.stride(0) != 1 or (Z.shape[1] > 1 and (Z.stride(1) != ld or S.stride(1) != ld)):
                raise ValueError("Z and S must be column-major with leading dimension n")
            self._check(self._lib.wd_apply_L(self._h, pz, ps, Z.shape[1], ld, dev, _stream(stream, dev)))
            return S
        Zc = np.array(Z, dtype=np.float64, order="F", copy=True)
        if Zc.ndim == 1:
            Zc = Zc[:, None]
        So = np.empty_like(Zc, order="F")
        self._check(self._lib.wd_apply_L(self._h, ctypes.c_void_p(Zc.ctypes.data),
                                         ctypes.c_void_p(So.ctypes.data), Zc.shape[1], Zc.shape[0], 0,
                                         _stream(stream, False)))
        return So

    def selinv(self, out=None, stream=None):
        """(A^-1)(i, j) at every stored lower entry of A, in the analyzed order
        (needs an fp64 factorization).  out: CUDA float64 tensor (filled in
        place) or None (a new numpy array)."""
        if out is not None and _is_torch(out):
            if out.numel() != self.nnz or not out.is_contiguous():
                raise ValueError("out must be a contiguous tensor with one entry per stored value")
            p, dev = _ptr(out)
            self._check(self._lib.wd_selinv(self._h, p, dev, _stream(stream, dev)))
            return out
        res = np.empty(self.nnz, np.float64)
        self._check(self._lib.wd_selinv(self._h, ctypes.c_void_p(res.ctypes.data), 0,
                                        _stream(stream, False)))
        return res

    def sym_pattern_outer(self, U, V, out=None, stream=None):
        """out[e] = sum_c U(i,c) V(j,c) + U(j,c) V(i,c) (i != j), sum_c U(i,c) V(i,c)
        (i == j) at every stored lower entry e = (i, j).  U, V: n x ncols,
        column-major (torch CUDA tensors with leading dimension n, or numpy)."""
        if _is_torch(U):
            import torch
            if U.dim() == 1:
                U, V = U.unsqueeze(1), V.unsqueeze(1)
            n = U.shape[0]
            for t in (U, V):
                if t.stride(0) != 1 or (t.shape[1] > 1 and t.stride(1) != n) or t.shape != U.shape:
                    raise ValueError("U and V must be column-major n x ncols with leading dimension n")
            if out is None:
                out = torch.empty(self.nnz, dtype=torch.float64, device=U.device)
            pu, dev = _ptr(U)
            pv, _ = _ptr(V)
            po, _ = _ptr(out)
            self._check(self._lib.wd_sym_pattern_outer(self._h, pu, pv, U.shape[1], n, po, dev,
                                                       _stream(stream, dev)))
            return out
        Uc = np.array(U, dtype=np.float64, order="F", copy=True)
        Vc = np.array(V, dtype=np.float64, order="F", copy=True)
        if Uc.ndim == 1:
            Uc, Vc = Uc[:, None], Vc[:, None]
        if Uc.shape != Vc.shape:
            raise ValueError("U and V must have the same shape")
        res = np.empty(self.nnz, np.float64)
        self._check(self._lib.wd_sym_pattern_outer(self._h, ctypes.c_void_p(Uc.ctypes.data),
                                                   ctypes.c_void_p(Vc.ctypes.data), Uc.shape[1],
                                                   Uc.shape[0], ctypes.c_void_p(res.ctypes.data), 0,
                                                   _stream(stream, False)))
        return res

    def value_gradient(self, g_logdet, X, G, out=None, stream=None):
        """dl/d(values) = g_logdet * w * A^-1 - pattern(G X^T + X G^T) at the stored
        lower entries (w = 2 off the diagonal); X = A^-1 B, G = A^-1 dl/dX.
        Torch CUDA tensors (column-major, leading dimension n) or numpy arrays."""
        if _is_torch(X):
            import torch
            if X.dim() == 1:
                X, G = X.unsqueeze(1), G.unsqueeze(1)
            n = X.shape[0]
            for t in (X, G):
                if t.stride(0) != 1 or (t.shape[1] > 1 and t.stride(1) != n) or t.shape != X.shape:
                    raise ValueError("X and G must be column-major n x ncols with leading dimension n")
            if out is None:
                out = torch.empty(self.nnz, dtype=torch.float64, device=X.device)
            px, dev = _ptr(X)
            pg, _ = _ptr(G)
            po, _ = _ptr(out)
            self._check(self._lib.wd_value_gradient(self._h, float(g_logdet), px, pg, X.shape[1], n, po,
                                                    dev, _stream(stream, dev)))
            return out
        Xc = np.array(X, dtype=np.float64, order="F", copy=True)
        Gc = np.array(G, dtype=np.float64, order="F", copy=True)
        if Xc.ndim == 1:
            Xc, Gc = Xc[:, None], Gc[:, None]
        res = np.empty(self.nnz, np.float64)
        self._check(self._lib.wd_value_gradient(self._h, float(g_logdet), ctypes.c_void_p(Xc.ctypes.data),
                                                ctypes.c_void_p(Gc.ctypes.data), Xc.shape[1], Xc.shape[0],
                                                ctypes.c_void_p(res.ctypes.data), 0,
                                                _stream(stream, False)))
        return res

    def kernel_stats(self, reset=False) -> list:
        """Per-kernel launches, event time and algorithmic flops/bytes
        accumulated while profiling (Solver(profile=True))."""
        cnt = ctypes.c_int32()
        self._check(self._lib.wd_kernel_stats(self._h, None, 0, ctypes.byref(cnt), 0))
        arr = (WdKernelStat * max(cnt.value, 1))()
        self._check(self._lib.wd_kernel_stats(self._h, arr, cnt.value, ctypes.byref(cnt),
                                              1 if reset else 0))
        return [dict(name=a.name.decode(), launches=a.launches, ms=a.milliseconds, flops=a.flops,
                     bytes=a.bytes) for a in arr[: cnt.value]]

    def launch_count(self, reset=False) -> int:
        c = ctypes.c_int64()
        self._check(self._lib.wd_launch_count(self._h, ctypes.byref(c), 1 if reset else 0))
        return c.value

    def export_L(self) -> np.ndarray:
        """Stored supernodal panels (see wd_export_L)."""
        out = np.empty(self._panel_size(), np.float64)
        self._check(self._lib.wd_export_L(self._h, ctypes.c_void_p(out.ctypes.data)))
        return out

    def export_L_noalloc(self, out, stream=None):
        """wd_export_L into a preallocated contiguous CUDA float64 tensor of
        _panel_size() entries, enqueued on the stream, without allocating."""
        if not _is_torch(out) or not out.is_cuda or not out.is_contiguous():
            raise ValueError("out must be a contiguous CUDA tensor")
        if out.dtype != __import__("torch").float64 or out.numel() != self._panel_size():
            raise ValueError("out must hold one float64 per stored panel entry")
        p, _ = _ptr(out)
        self._check(self._lib.wd_export_L_noalloc(self._h, p, _stream(stream, True)))
        return out

    def _panel_size(self) -> int:
        sym = self.symbolic()
        k = np.diff(sym["super_first"]).astype(np.int64)
        m = np.diff(sym["super_rowptr"]).astype(np.int64)
        return int((k * m).sum())

    def L_csc_like(self, Lp, Li, panels=None):
        """The factor's entries at the positions of a CSC pattern of L
        (e.g. the oracle's): values of stored panels (export_L's, or the given
        ones in that layout), structural entries only."""
        sym = self.symbolic()
        if panels is None:
            panels = self.export_L()
        sf, srp, rows = sym["super_first"], sym["super_rowptr"], sym["super_rows"]
        n = self.n
        col2s = np.repeat(np.arange(sf.size - 1), np.diff(sf))
        k = np.diff(sf).astype(np.int64)
        m = np.diff(srp).astype(np.int64)
        poff = np.concatenate([[0], np.cumsum(k * m)])
        out = np.empty(Li.size, np.float64)
        for j in range(n):
            s = col2s[j]
            r = rows[srp[s]: srp[s + 1]]
            loc = np.searchsorted(r, Li[Lp[j]: Lp[j + 1]])
            if np.any(loc >= r.size) or np.any(r[np.minimum(loc, r.size - 1)] != Li[Lp[j]: Lp[j + 1]]):
                raise ValueError(f"pattern of column {j} not inside its supernode")
            c = j - sf[s]
            out[Lp[j]: Lp[j + 1]] = panels[poff[s] + c * m[s] + loc]
        return out
