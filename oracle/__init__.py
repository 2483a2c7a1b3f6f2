"""CPU oracle — test infrastructure only.

Plain, slow FP64 reference for everything the solver computes (see
``oracle.c`` for the algorithms and their citations).  Only the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package.  It shares no code with the CUDA path and never imports it.

The C part is compiled with gcc (-O2 -ffp-contract=off) into
``oracle/_build/liboracle.so`` by :func:`build`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (idempotent)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.or_create.restype = ctypes.c_void_p
            lib.or_destroy.argtypes = [ctypes.c_void_p]
            lib.or_analyze.restype = ctypes.c_int
            lib.or_analyze.argtypes = [ctypes.c_void_p, ctypes.c_int64, _i64p, _i32p, ctypes.c_int,
                                       _i32p, _i32p, _i32p, _i32p, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, _i32p]
            lib.or_nd_order_tree.restype = ctypes.c_int
            lib.or_nd_order_tree.argtypes = [ctypes.c_int64, _i64p, _i32p, ctypes.c_int, _i32p,
                                             _i32p, _i32p, _i32p, ctypes.c_int32, _i32p, _i64p,
                                             ctypes.c_int64, _i64p]
            for f in ("or_n", "or_nnzL", "or_nsuper_rows"):
                getattr(lib, f).restype = ctypes.c_int64
                getattr(lib, f).argtypes = [ctypes.c_void_p]
            lib.or_nsuper.restype = ctypes.c_int32
            lib.or_nsuper.argtypes = [ctypes.c_void_p]
            lib.or_get_symbolic.argtypes = [ctypes.c_void_p, _i32p, _i32p, _i64p, _i32p, _i64p,
                                            _i32p]
            lib.or_get_Lpattern.argtypes = [ctypes.c_void_p, _i64p, _i32p]
            lib.or_factor.restype = ctypes.c_int64
            lib.or_factor.argtypes = [ctypes.c_void_p, _f64p]
            lib.or_factor_cols.restype = ctypes.c_int64
            lib.or_factor_cols.argtypes = [ctypes.c_void_p, _f64p, ctypes.c_int64]
            lib.or_get_L.argtypes = [ctypes.c_void_p, _f64p]
            lib.or_solve.restype = ctypes.c_int
            lib.or_solve.argtypes = [ctypes.c_void_p, _f64p, ctypes.c_int64, ctypes.c_int64]
            lib.or_solve_prefix.restype = ctypes.c_int
            lib.or_solve_prefix.argtypes = [ctypes.c_void_p, _f64p, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int64]
            lib.or_factor_lu.restype = ctypes.c_int64
            lib.or_factor_lu.argtypes = [ctypes.c_void_p, _f64p, _f64p]
            lib.or_get_lu.argtypes = [ctypes.c_void_p, _f64p, _f64p]
            lib.or_solve_lu.restype = ctypes.c_int
            lib.or_solve_lu.argtypes = [ctypes.c_void_p, _f64p, ctypes.c_int64, ctypes.c_int64]
            lib.or_logdet_lu.restype = ctypes.c_double
            lib.or_logdet_lu.argtypes = [ctypes.c_void_p, _i32p]
            lib.or_factor_ldlt.restype = ctypes.c_int64
            lib.or_factor_ldlt.argtypes = [ctypes.c_void_p, _f64p]
            lib.or_get_ldlt.argtypes = [ctypes.c_void_p, _f64p, _f64p]
            lib.or_solve_ldlt.restype = ctypes.c_int
            lib.or_solve_ldlt.argtypes = [ctypes.c_void_p, _f64p, ctypes.c_int64, ctypes.c_int64]
            lib.or_logdet_ldlt.restype = ctypes.c_double
            lib.or_logdet_ldlt.argtypes = [ctypes.c_void_p, _i32p, ctypes.POINTER(ctypes.c_int64)]
            lib.or_logdet.restype = ctypes.c_double
            lib.or_logdet.argtypes = [ctypes.c_void_p]
            lib.or_apply_L.restype = ctypes.c_int
            lib.or_apply_L.argtypes = [ctypes.c_void_p, _f64p, _f64p, ctypes.c_int64,
                                       ctypes.c_int64]
            lib.or_selinv.restype = ctypes.c_int
            lib.or_selinv.argtypes = [ctypes.c_void_p, _f64p]
            lib.or_get_permuted_lower.argtypes = [ctypes.c_void_p, _i64p, _i32p, _i64p]
            _lib = lib
    return _lib


def _p(a, t):
    return None if a is None else a.ctypes.data_as(t)


def _geom(basis):
    if basis is None:
        return 0, None, None, None, None
    lev = np.ascontiguousarray(basis.level, np.int32)
    lo = np.ascontiguousarray(basis.box_lo, np.int32)
    side = np.ascontiguousarray(basis.box_side, np.int32)
    patch = getattr(basis, "patch", None)
    patch = None if patch is None else np.ascontiguousarray(patch, np.int32)
    return basis.dim, lev, lo, side, patch


def nd_order(colptr, rowidx, basis, leaf: int = 128, want_tree: bool = False):
    """Geometric nested dissection (perm[new] = old) and, optionally, the
    dissection nodes as rows (V1 start, V2 start, S start, S end)."""
    lib = _load()
    cp = np.ascontiguousarray(colptr, np.int64)
    ri = np.ascontiguousarray(rowidx, np.int32)
    n = cp.size - 1
    dim, lev, lo, side, patch = _geom(basis)
    perm = np.empty(n, np.int32)
    cap = n + 1
    tree = np.empty((cap, 4), np.int64)
    nt = np.zeros(1, np.int64)
    rc = lib.or_nd_order_tree(n, _p(cp, _i64p), _p(ri, _i32p), dim, _p(lev, _i32p),
                              _p(lo, _i32p), _p(side, _i32p), _p(patch, _i32p), leaf, _p(perm, _i32p),
                              _p(tree, _i64p), cap, _p(nt, _i64p))
    if rc:
        raise RuntimeError(f"or_nd_order failed: {rc}")
    return (perm, tree[: int(nt[0])].copy()) if want_tree else perm


class Oracle:
    """Symbolic + numeric sparse Cholesky of a symmetric matrix given by its
    lower CSC (diagonal first in each column, rows sorted, 0-based)."""

    def __init__(self, colptr, rowidx, basis=None, leaf: int = 128, relax_k: int = 64,
                 relax_pct: int = 10, perm=None):
        self._lib = _load()
        self._ctx = ctypes.c_void_p(self._lib.or_create())
        self.colptr = np.ascontiguousarray(colptr, np.int64)
        self.rowidx = np.ascontiguousarray(rowidx, np.int32)
        self.n = self.colptr.size - 1
        dim, lev, lo, side, patch = _geom(basis)
        pin = None if perm is None else np.ascontiguousarray(perm, np.int32)
        rc = self._lib.or_analyze(self._ctx, self.n, _p(self.colptr, _i64p),
                                  _p(self.rowidx, _i32p), dim, _p(lev, _i32p), _p(lo, _i32p),
                                  _p(side, _i32p), _p(patch, _i32p), leaf, relax_k, relax_pct,
                                  _p(pin, _i32p))
        if rc:
            raise ValueError(f"or_analyze failed: {rc}")
        n = self.n
        self.nsuper = int(self._lib.or_nsuper(self._ctx))
        self.nnzL = int(self._lib.or_nnzL(self._ctx))
        nrows = int(self._lib.or_nsuper_rows(self._ctx))
        self.perm = np.empty(n, np.int32)
        self.parent = np.empty(n, np.int32)
        self.colcount = np.empty(n, np.int64)
        self.super_first = np.empty(self.nsuper + 1, np.int32)
        self.super_rowptr = np.empty(self.nsuper + 1, np.int64)
        self.super_rows = np.empty(max(nrows, 1), np.int32)[:nrows]
        self._lib.or_get_symbolic(self._ctx, _p(self.perm, _i32p), _p(self.parent, _i32p),
                                  _p(self.colcount, _i64p), _p(self.super_first, _i32p),
                                  _p(self.super_rowptr, _i64p), _p(self.super_rows, _i32p))
        self.Lp = np.empty(n + 1, np.int64)
        self.Li = np.empty(self.nnzL, np.int32)
        self._lib.or_get_Lpattern(self._ctx, _p(self.Lp, _i64p), _p(self.Li, _i32p))
        self.factored = False

    def __del__(self):
        try:
            self._lib.or_destroy(self._ctx)
        except Exception:
            pass

    # -- numeric ------------------------------------------------------------
    def factor(self, values) -> int:
        """Returns 0, or the first column j (permuted order) whose pivot is
        not positive, as -(j+1)."""
        v = np.ascontiguousarray(values, np.float64)
        rc = int(self._lib.or_factor(self._ctx, _p(v, _f64p)))
        self.factored = rc == 0
        return rc

    def factor_prefix(self, values, ncols: int) -> int:
        """Factor only the first ncols columns of P A P^T (a bounded sample
        of the full factorization, for timing)."""
        v = np.ascontiguousarray(values, np.float64)
        rc = int(self._lib.or_factor_cols(self._ctx, _p(v, _f64p), int(ncols)))
        self.factored = rc == 0 and ncols >= self.n
        return rc

    def solve_prefix(self, Y, ncols: int) -> None:
        """The forward and backward substitution loops of solve() over the
        first ncols columns only, in place on Y (n x nrhs, factor order,
        Fortran order): a bounded share of the solve, for timing (valid after
        factor_prefix(values, ncols))."""
        if not (Y.flags.f_contiguous and Y.dtype == np.float64 and Y.shape[0] == self.n):
            raise ValueError("Y must be an n x nrhs Fortran-ordered float64 array")
        rc = self._lib.or_solve_prefix(self._ctx, _p(Y, _f64p), Y.shape[1], self.n, int(ncols))
        if rc:
            raise RuntimeError("solve_prefix: not factored or bad ncols")

    # -- LU without pivoting (nonsymmetric values on the symmetric pattern) ----
    def factor_lu(self, lower, upper) -> int:
        """P A P^T = L U, L unit lower triangular, no pivoting.  lower[e] =
        A[r][c], upper[e] = A[c][r] for every stored lower entry (r, c).
        Returns 0, or -(j+1) for the first zero pivot (permuted order)."""
        lo = np.ascontiguousarray(lower, np.float64)
        up = np.ascontiguousarray(upper, np.float64)
        return int(self._lib.or_factor_lu(self._ctx, _p(lo, _f64p), _p(up, _f64p)))

    def lu_values(self):
        """(L, U^T) on the pattern of L (Lp, Li): L with its unit diagonal,
        column j of U^T = row j of U."""
        L = np.empty(self.nnzL, np.float64)
        Ut = np.empty(self.nnzL, np.float64)
        self._lib.or_get_lu(self._ctx, _p(L, _f64p), _p(Ut, _f64p))
        return L, Ut

    def solve_lu(self, B) -> np.ndarray:
        X = np.array(B, dtype=np.float64, order="F", copy=True)
        if X.ndim == 1:
            X = X[:, None]
        if self._lib.or_solve_lu(self._ctx, _p(X, _f64p), X.shape[1], self.n):
            raise RuntimeError("not LU-factored")
        return X

    def logdet_lu(self):
        """(log |det A|, sign of det A)"""
        sg = np.zeros(1, np.int32)
        v = float(self._lib.or_logdet_lu(self._ctx, _p(sg, _i32p)))
        return v, int(sg[0])

    # -- LDL^T without pivoting (symmetric, possibly indefinite) ---------------
    def factor_ldlt(self, values) -> int:
        """P A P^T = L D L^T, L unit lower triangular, D diagonal, no
        pivoting.  Returns 0, or -(j+1) for the first zero pivot (permuted
        order)."""
        v = np.ascontiguousarray(values, np.float64)
        return int(self._lib.or_factor_ldlt(self._ctx, _p(v, _f64p)))

    def ldlt_values(self):
        """(L on the pattern of L (Lp, Li) with its unit diagonal, d (n))"""
        L = np.empty(self.nnzL, np.float64)
        d = np.empty(self.n, np.float64)
        self._lib.or_get_ldlt(self._ctx, _p(L, _f64p), _p(d, _f64p))
        return L, d

    def solve_ldlt(self, B) -> np.ndarray:
        X = np.array(B, dtype=np.float64, order="F", copy=True)
        if X.ndim == 1:
            X = X[:, None]
        if self._lib.or_solve_ldlt(self._ctx, _p(X, _f64p), X.shape[1], self.n):
            raise RuntimeError("not LDL^T-factored")
        return X

    def logdet_ldlt(self):
        """(log |det A|, sign of det A, number of negative pivots = number of
        negative eigenvalues of A)"""
        sg = np.zeros(1, np.int32)
        neg = ctypes.c_int64(0)
        v = float(self._lib.or_logdet_ldlt(self._ctx, _p(sg, _i32p), ctypes.byref(neg)))
        return v, int(sg[0]), int(neg.value)

    def L_values(self) -> np.ndarray:
        x = np.empty(self.nnzL, np.float64)
        self._lib.or_get_L(self._ctx, _p(x, _f64p))
        return x

    def L_dense(self) -> np.ndarray:
        Lx = self.L_values()
        L = np.zeros((self.n, self.n))
        cols = np.repeat(np.arange(self.n), np.diff(self.Lp))
        L[self.Li, cols] = Lx
        return L

    def solve(self, B) -> np.ndarray:
        X = np.array(B, dtype=np.float64, order="F", copy=True)
        if X.ndim == 1:
            X = X[:, None]
        rc = self._lib.or_solve(self._ctx, _p(X, _f64p), X.shape[1], self.n)
        if rc:
            raise RuntimeError("not factored")
        return X

    def logdet(self) -> float:
        return float(self._lib.or_logdet(self._ctx))

    def apply_L(self, Z) -> np.ndarray:
        Zc = np.array(Z, dtype=np.float64, order="F", copy=True)
        if Zc.ndim == 1:
            Zc = Zc[:, None]
        S = np.empty_like(Zc, order="F")
        rc = self._lib.or_apply_L(self._ctx, _p(Zc, _f64p), _p(S, _f64p), Zc.shape[1], self.n)
        if rc:
            raise RuntimeError("not factored")
        return S

    def selinv(self) -> np.ndarray:
        """(P A P^T)^-1 on the pattern of L, same layout as L_values()."""
        Z = np.zeros(self.nnzL, np.float64)
        rc = self._lib.or_selinv(self._ctx, _p(Z, _f64p))
        if rc:
            raise RuntimeError(f"or_selinv failed: {rc}")
        return Z

    def permuted_lower(self):
        nnz = int(self.colptr[-1])
        pcp = np.empty(self.n + 1, np.int64)
        prow = np.empty(nnz, np.int32)
        psrc = np.empty(nnz, np.int64)
        self._lib.or_get_permuted_lower(self._ctx, _p(pcp, _i64p), _p(prow, _i32p),
                                        _p(psrc, _i64p))
        return pcp, prow, psrc

    # -- structure helpers ---------------------------------------------------
    def supernodes(self):
        """List of (first, last+1, rows ndarray)."""
        out = []
        for s in range(self.nsuper):
            r = self.super_rows[self.super_rowptr[s]: self.super_rowptr[s + 1]]
            out.append((int(self.super_first[s]), int(self.super_first[s + 1]), r))
        return out

    def factor_flops(self) -> int:
        """sum_j c_j^2, the structural operation count of the factorization."""
        return int(np.sum(self.colcount.astype(np.int64) ** 2))


# ---------------------------------------------------------------------------
# plain FP64 helpers on a symmetric matrix stored as lower CSC
# ---------------------------------------------------------------------------


def sym_lower_to_dense(colptr, rowidx, values, n=None) -> np.ndarray:
    n = len(colptr) - 1 if n is None else n
    A = np.zeros((n, n))
    cols = np.repeat(np.arange(n), np.diff(colptr))
    A[rowidx, cols] = values
    A[cols, rowidx] = values
    return A


def sym_spmv(colptr, rowidx, values, X) -> np.ndarray:
    """A @ X for the symmetric A given by its lower CSC (scipy sparse product
    of the stored triangle, plus its transpose, minus the diagonal)."""
    import scipy.sparse as sp

    n = len(colptr) - 1
    Lo = sp.csc_matrix((values, rowidx, colptr), shape=(n, n))
    d = values[np.asarray(colptr[:-1])]
    Xa = np.asarray(X, dtype=np.float64)
    if Xa.ndim == 1:
        return Lo @ Xa + Lo.T @ Xa - d * Xa
    return Lo @ Xa + Lo.T @ Xa - d[:, None] * Xa


def nonsym_lower_upper_to_dense(colptr, rowidx, lower, upper) -> np.ndarray:
    """Dense A from its stored lower entries: A[r][c] = lower[e], A[c][r] =
    upper[e] for every lower-CSC entry e = (r, c)."""
    n = len(colptr) - 1
    A = np.zeros((n, n))
    cols = np.repeat(np.arange(n), np.diff(colptr))
    A[cols, rowidx] = upper
    A[rowidx, cols] = lower
    return A


def nonsym_spmv(colptr, rowidx, lower, upper, X) -> np.ndarray:
    """A @ X for A given by lower / upper values on a symmetric pattern."""
    import scipy.sparse as sp

    n = len(colptr) - 1
    Lo = sp.csc_matrix((np.asarray(lower, np.float64), rowidx, colptr), shape=(n, n))
    Up = sp.csc_matrix((np.asarray(upper, np.float64), rowidx, colptr), shape=(n, n)).T
    d = np.asarray(lower, np.float64)[np.asarray(colptr[:-1])]
    Xa = np.asarray(X, dtype=np.float64)
    if Xa.ndim == 1:
        return Lo @ Xa + Up @ Xa - d * Xa
    return Lo @ Xa + Up @ Xa - d[:, None] * Xa


def nonsym_backward_error(colptr, rowidx, lower, upper, X, B) -> np.ndarray:
    """Normwise backward error per column for the nonsymmetric A."""
    n = len(colptr) - 1
    X = np.asarray(X).reshape(n, -1)
    B = np.asarray(B).reshape(n, -1)
    R = B - nonsym_spmv(colptr, rowidx, lower, upper, X)
    cols = np.repeat(np.arange(n), np.diff(colptr))
    off = rowidx != cols
    s = np.zeros(n)
    np.add.at(s, rowidx, np.abs(lower))
    np.add.at(s, cols[off], np.abs(np.asarray(upper)[off]))
    return np.abs(R).max(0) / (s.max() * np.abs(X).max(0) + np.abs(B).max(0))


def sym_norm_inf(colptr, rowidx, values) -> float:
    n = len(colptr) - 1
    cols = np.repeat(np.arange(n), np.diff(colptr))
    off = rowidx != cols
    s = np.zeros(n)
    np.add.at(s, rowidx, np.abs(values))
    np.add.at(s, cols[off], np.abs(values[off]))
    return float(s.max())


def backward_error(colptr, rowidx, values, X, B) -> np.ndarray:
    """Normwise backward error per column: ||b-Ax||_inf/(||A||_inf ||x||_inf + ||b||_inf)."""
    X = np.asarray(X).reshape(len(colptr) - 1, -1)
    B = np.asarray(B).reshape(len(colptr) - 1, -1)
    R = B - sym_spmv(colptr, rowidx, values, X)
    an = sym_norm_inf(colptr, rowidx, values)
    return np.abs(R).max(0) / (an * np.abs(X).max(0) + np.abs(B).max(0))


def theta_matrix(colptr, values, theta: float, dt: float, g_values=None) -> np.ndarray:
    """Lower-CSC values of M = G + theta dt K, the matrix the theta-scheme
    inverts at every step (Section 5, Eq. (theta)); K's values (and G's, if
    given; G = I otherwise, an orthonormal basis) on the same pattern,
    diagonal first in each column."""
    m = theta * dt * np.asarray(values, dtype=np.float64)
    if g_values is None:
        m[np.asarray(colptr[:-1])] += 1.0
    else:
        m = m + np.asarray(g_values, dtype=np.float64)
    return m


def theta_step(o, colptr, rowidx, k_values, U, F, theta: float, dt: float, g_values=None) -> np.ndarray:
    """One step of Eq. (theta) with the mass matrix G (identity if g_values is
    None) and the stiffness matrix K (positive semidefinite; the paper's L_J
    enters with the opposite sign):
        G (u_new - u) / dt + K ((1 - theta) u + theta u_new) = F,
    i.e. (G + theta dt K) u_new = (G - (1 - theta) dt K) u + dt F, with the
    oracle `o` factored for M = theta_matrix(...).  U, F: n x nrhs (F may be
    None)."""
    U = np.asarray(U, dtype=np.float64)
    GU = U if g_values is None else sym_spmv(colptr, rowidx, g_values, U)
    rhs = GU - (1.0 - theta) * dt * sym_spmv(colptr, rowidx, k_values, U)
    if F is not None:
        rhs = rhs + dt * np.asarray(F, dtype=np.float64)
    return o.solve(rhs.reshape(len(colptr) - 1, -1)).reshape(U.shape)
