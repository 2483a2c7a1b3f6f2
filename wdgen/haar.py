"""Seeded synthetic workloads: Haar wavelet bases and compressed kernel matrices.

This module only builds INPUTS (a sparse symmetric matrix, its geometry and
right-hand sides).  It holds none of the solver's arithmetic: no ordering,
no factorization, no triangular solve.  Both the CPU oracle and the CUDA path
consume what it produces.

What it builds (the paper's Sections 2 and 3, restated):

* Haar multiresolution bases on a uniform grid of 2^J cells per axis
  (1D or 2D).  Level 0 is the single scaling function (Psi_0 := Phi_0,
  Section 2); level j = 1..J holds wavelets living on the dyadic cells of
  side 2^(1-j) of the unit interval/square (diam supp psi_{j,k} ~ 2^-j).
  1D: psi = (phi_left - phi_right)/sqrt(2) per dyadic interval.
  2D (isotropic): per dyadic square the three tensor wavelets
  psi(x)phi(y), phi(x)psi(y), psi(x)psi(y), sign "+" on the left/bottom half.
  All functions are L2-normalized, so the basis is orthonormal.
* Galerkin matrix in wavelet coordinates (Section 3): with the L2-normalized
  cell indicators as single-scale basis and the one-point (cell-centroid)
  rule,  K_ss[c, c'] = sqrt(|c||c'|) k(x_c, x_c'),  and  A = T K_ss T^T  with
  T the orthonormal fast wavelet transform.
* A-priori compression (Theorem 3.1), first cut-off term with a = 2: the
  entry (lambda, lambda') is kept iff
      dist(D_lambda, D_lambda') <= 2 * 2^(-min(j, j')),
  dist being the Euclidean distance of the closed support boxes, evaluated
  exactly on integers in finest-cell units.  Then the nugget eps*I is added
  (the mass matrix of an orthonormal basis is the identity).

Index order ("canonical levelwise ordering", Section 4): level 0, then level
1, ..., level J; inside a level 1D wavelets by position k, 2D wavelets by
square (row p = y index major, column q = x index) and then by type 0,1,2.
Level j >= 1 starts at index 2^(j-1) in 1D and 4^(j-1) in 2D.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# bases
# --------------------------------------------------------------------------


@dataclass
class Basis:
    """Geometry of a Haar wavelet basis (finest-cell integer units)."""

    dim: int
    J: int
    level: np.ndarray        # int32 [N]
    box_lo: np.ndarray       # int32 [N, dim]   lower corner of supp psi
    box_side: np.ndarray     # int32 [N]        side length of supp psi
    patch: np.ndarray | None = None  # int32 [N] or None

    @property
    def N(self) -> int:
        return int(self.level.shape[0])

    @property
    def n_side(self) -> int:
        return 1 << self.J


def _positions(dim: int, j: int) -> int:
    return 1 if j == 0 else (1 << (j - 1))


def level_side(J: int, j: int) -> int:
    """Support side of a level-j function in finest-cell units."""
    return (1 << J) if j == 0 else (1 << (J + 1 - j))


def haar_basis(dim: int, J: int) -> Basis:
    if dim not in (1, 2):
        raise ValueError("dim must be 1 or 2")
    lev, lo, side = [], [], []
    for j in range(J + 1):
        n = _positions(dim, j)
        s = level_side(J, j)
        if dim == 1:
            k = np.arange(n, dtype=np.int64)
            lev.append(np.full(n, j, np.int32))
            lo.append((k * s)[:, None])
            side.append(np.full(n, s, np.int32))
        else:
            ntype = 1 if j == 0 else 3
            p, q = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
            p = np.repeat(p.reshape(-1), ntype)
            q = np.repeat(q.reshape(-1), ntype)
            lev.append(np.full(p.size, j, np.int32))
            lo.append(np.stack([q * s, p * s], axis=1))
            side.append(np.full(p.size, s, np.int32))
    return Basis(dim, J, np.concatenate(lev), np.concatenate(lo).astype(np.int32),
                 np.concatenate(side))


def fwt(x, dim: int, J: int, xp=np):
    """Orthonormal Haar transform over the trailing cell axes.

    x: (..., n) in 1D or (..., n, n) indexed [iy, ix] in 2D, holding the
    coefficients in the normalized cell basis.  Returns (..., N) wavelet
    coefficients in the canonical levelwise order.  Works for numpy arrays
    and torch tensors (xp = numpy or torch).
    """
    parts = []
    a = x
    r2 = 1.0 / math.sqrt(2.0)
    for _ in range(J, 0, -1):
        if dim == 1:
            a0 = a[..., 0::2]
            a1 = a[..., 1::2]
            parts.append((a0 - a1) * r2)
            a = (a0 + a1) * r2
        else:
            a00 = a[..., 0::2, 0::2]
            a01 = a[..., 0::2, 1::2]
            a10 = a[..., 1::2, 0::2]
            a11 = a[..., 1::2, 1::2]
            d0 = ((a00 + a10) - (a01 + a11)) * 0.5
            d1 = ((a00 + a01) - (a10 + a11)) * 0.5
            d2 = ((a00 + a11) - (a01 + a10)) * 0.5
            a = ((a00 + a01) + (a10 + a11)) * 0.5
            st = xp.stack([d0, d1, d2], -1)
            parts.append(st.reshape(tuple(st.shape[:-3]) + (-1,)))
    parts.append(a.reshape(tuple(a.shape[: a.ndim - dim]) + (1,)))
    parts.reverse()
    if xp is np:
        return np.concatenate(parts, -1)
    return xp.cat(parts, -1)


# --------------------------------------------------------------------------
# compression pattern
# --------------------------------------------------------------------------


def _axis_pairs(J: int, j: int, jp: int):
    """All (k, k', gap) along one axis with gap <= 2*2^(J-min(j,j'))."""
    n, np_ = _positions(1, j), _positions(1, jp)
    s, sp = level_side(J, j), level_side(J, jp)
    thr = 2 * (1 << (J - min(j, jp)))
    k = np.arange(n, dtype=np.int64)
    # k' with  k'*sp - (k+1)*s <= thr  and  k*s - (k'+1)*sp <= thr
    khi = np.minimum(((k + 1) * s + thr) // sp, np_ - 1)
    klo = np.maximum(-((-(k * s - thr)) // sp) - 1, 0)
    cnt = np.maximum(khi - klo + 1, 0)
    kk = np.repeat(k, cnt)
    off = np.arange(int(cnt.sum()), dtype=np.int64) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    kp = np.repeat(klo, cnt) + off
    lo, lop = kk * s, kp * sp
    gap = np.maximum(np.maximum(lop - (lo + s), lo - (lop + sp)), 0)
    keep = gap <= thr
    return kk[keep], kp[keep], gap[keep], thr


def _level_offset(dim: int, j: int) -> int:
    if j == 0:
        return 0
    return (1 << (j - 1)) if dim == 1 else (1 << (2 * (j - 1)))


def compressed_pattern(basis: Basis):
    """Lower CSC pattern (incl. diagonal, rows sorted) of the a=2 mask.

    Returns colptr int64 [N+1], rowidx int32 [nnz_lower].
    """
    dim, J, N = basis.dim, basis.J, basis.N
    rows, cols = [], []
    for j in range(J + 1):
        for jp in range(j, J + 1):
            kk, kp, gap, thr = _axis_pairs(J, j, jp)
            if dim == 1:
                a = _level_offset(1, j) + kk
                b = _level_offset(1, jp) + kp
            else:
                # combine an x-pair and a y-pair: square (p,q) x square (p',q')
                ny = kk.size
                ia = np.repeat(np.arange(ny), ny)   # y pair
                ib = np.tile(np.arange(ny), ny)     # x pair
                ok = gap[ia] ** 2 + gap[ib] ** 2 <= thr * thr
                ia, ib = ia[ok], ib[ok]
                n, np_ = _positions(2, j), _positions(2, jp)
                sq = kk[ia] * n + kk[ib]
                sqp = kp[ia] * np_ + kp[ib]
                t = 1 if j == 0 else 3
                tp = 1 if jp == 0 else 3
                ta = np.repeat(np.arange(t), tp)
                tb = np.tile(np.arange(tp), t)
                a = (_level_offset(2, j) + t * sq)[:, None] + ta[None, :]
                b = (_level_offset(2, jp) + tp * sqp)[:, None] + tb[None, :]
                a = a.reshape(-1)
                b = b.reshape(-1)
            r = np.maximum(a, b)
            c = np.minimum(a, b)
            rows.append(r)
            cols.append(c)
    r = np.concatenate(rows).astype(np.int64)
    c = np.concatenate(cols).astype(np.int64)
    key = np.unique(c * N + r)          # same-level pairs appear twice
    c = key // N
    r = key % N
    colptr = np.zeros(N + 1, np.int64)
    np.cumsum(np.bincount(c, minlength=N), out=colptr[1:])
    return colptr, r.astype(np.int32)


def mass_matrix(basis: Basis, colptr, rowidx, coupling: float = 0.3) -> np.ndarray:
    """Lower-CSC values (on the given pattern) of a synthetic mass matrix G of
    a non-orthonormal basis: the Gram matrix of functions that overlap their
    same-level neighbours, as piecewise linear or bilinear wavelets do
    (Section 6), standing in for those bases (not built here).  G has ones on
    the diagonal and -coupling / max(deg_i, deg_j) between two functions of
    the same level >= 1 whose closed support boxes touch, deg being the
    number of such neighbours; every row's off-diagonal sum is at most
    coupling < 1, so G is symmetric positive definite.  Its pattern lies
    inside the compressed pattern (touching supports are at distance 0), as
    the mass matrix's lies inside the system matrix's (Section 6)."""
    if not 0.0 <= coupling < 1.0:
        raise ValueError("coupling must lie in [0, 1)")
    cp = np.asarray(colptr, np.int64)
    ri = np.asarray(rowidx, np.int64)
    N = cp.size - 1
    cols = np.repeat(np.arange(N), np.diff(cp))
    lev = np.asarray(basis.level)
    lo = np.asarray(basis.box_lo).reshape(N, -1).astype(np.int64)
    side = np.asarray(basis.box_side).astype(np.int64)
    off = ri != cols
    a, b = ri[off], cols[off]
    # closed boxes touch iff on every axis the intervals [lo, lo + side] meet
    touch = np.ones(a.size, bool)
    for ax in range(lo.shape[1]):
        touch &= (lo[a, ax] <= lo[b, ax] + side[b]) & (lo[b, ax] <= lo[a, ax] + side[a])
    nb = touch & (lev[a] == lev[b]) & (lev[a] > 0)
    deg = np.bincount(a[nb], minlength=N) + np.bincount(b[nb], minlength=N)
    g = np.zeros(ri.size)
    g[~off] = 1.0
    idx = np.flatnonzero(off)[nb]
    g[idx] = -coupling / np.maximum(deg[a[nb]], deg[b[nb]])
    return g


def own_pattern(colptr, rowidx, values):
    """(colptr, rowidx, values) of the stored nonzeros of a lower CSC matrix
    given on a larger pattern (the diagonal is always kept): the mass matrix
    on its own, sparser pattern, which its own analysis orders apart from the
    system matrix (Section 6)."""
    cp = np.asarray(colptr, np.int64)
    ri = np.asarray(rowidx, np.int64)
    v = np.asarray(values, np.float64)
    N = cp.size - 1
    cols = np.repeat(np.arange(N), np.diff(cp))
    keep = (v != 0.0) | (ri == cols)
    ncp = np.concatenate([[0], np.cumsum(np.bincount(cols[keep], minlength=N))]).astype(np.int64)
    return ncp, ri[keep].astype(np.int32), v[keep]


def cutoff_parameters(J: int, j: int, jp: int, a: float, delta: float, q: float, dtilde: float):
    """(B_{j,j'}, B^s_{j,j'}) of Theorem 3.1 (Eq. cut-off parameters), in
    domain units: the support-distance and singular-support-distance bounds
    of the a-priori compression for an operator of order 2q, wavelets with
    dtilde vanishing moments, a > 1 and d < delta < dtilde + 2q."""
    lo, hi = min(j, jp), max(j, jp)
    b = a * max(2.0 ** (-lo), 2.0 ** ((2 * J * (delta - q) - (j + jp) * (delta + dtilde)) / (2 * (dtilde + q))))
    bs = a * max(2.0 ** (-hi), 2.0 ** ((2 * J * (delta - q) - (j + jp) * delta - hi * dtilde) / (dtilde + 2 * q)))
    return b, bs


def compressed_pattern_two_term(basis: Basis, a: float, delta: float, q: float, dtilde: float = 1.0,
                                d: float = 1.0):
    """Lower CSC pattern of the full a-priori compression of Theorem 3.1 (both
    terms), for Haar wavelets (d = dtilde = 1) and an operator of order 2q:
    the entry (lambda, lambda') is dropped iff
      dist(D_l, D_l') > B_{|l|,|l'|} and |l|, |l'| > 0, or
      dist(D_l, D_l') <= 2^-min(|l|,|l'|) and the singular support of the
      coarser of the two is farther than B^s_{|l|,|l'|} from the finer's
      support (levels equal: this term does not apply),
    with the supports D and singular supports D^s (box boundaries and the
    lines where the wavelet changes sign) compared exactly in finest-cell
    units.  Needs a > 1 and d < delta < dtilde + 2q.  All pairs of two levels
    are enumerated (blocks of at most 2^22), which suits the small cases it
    is tested on."""
    if not (a > 1 and d < delta < dtilde + 2 * q):
        raise ValueError("Theorem 3.1 needs a > 1 and d < delta < dtilde + 2q")
    dim, J, N = basis.dim, basis.J, basis.N
    lev = np.asarray(basis.level)
    lo = np.asarray(basis.box_lo).reshape(N, -1).astype(np.int64)
    side = np.asarray(basis.box_side).astype(np.int64)
    unit = float(1 << J)                                  # cells per domain unit
    typ = np.zeros(N, np.int64)
    if dim == 2:
        first = np.array([_level_offset(2, j) for j in range(J + 1)])
        typ = np.where(lev > 0, (np.arange(N) - first[lev]) % 3, -1)

    def gap(a0, a1, b0, b1):
        return np.maximum(np.maximum(b0 - a1, a0 - b1), 0)

    def sing_dist2(ia, ib):
        """squared distance (cells^2) from the singular support of ia to the support box of ib"""
        x0, s = lo[ia, 0], side[ia]
        bx0, bs_ = lo[ib, 0][None, :], side[ib][None, :]
        if dim == 1:
            # end points, and the midpoint for a wavelet (level >= 1)
            best = None
            for p_, mid in ((x0, False), (x0 + s, False), (x0 + s // 2, True)):
                g = gap(p_[:, None], p_[:, None], bx0, bx0 + bs_).astype(np.float64)
                if mid:
                    g = np.where((lev[ia] > 0)[:, None], g, np.inf)
                best = g * g if best is None else np.minimum(best, g * g)
            return best
        y0 = lo[ia, 1]
        by0 = lo[ib, 1][None, :]
        X0, X1, Y0, Y1 = x0[:, None], (x0 + s)[:, None], y0[:, None], (y0 + s)[:, None]
        Xm, Ym = (x0 + s // 2)[:, None], (y0 + s // 2)[:, None]
        gxb = gap(X0, X1, bx0, bx0 + bs_)   # x-extent of the box vs the support's x-extent
        gyb = gap(Y0, Y1, by0, by0 + bs_)
        segs = []
        for xc in (X0, X1):                  # vertical boundary edges
            segs.append((gap(xc, xc, bx0, bx0 + bs_), gyb))
        for yc in (Y0, Y1):                  # horizontal boundary edges
            segs.append((gxb, gap(yc, yc, by0, by0 + bs_)))
        t = typ[ia][:, None]
        vm = (gap(Xm, Xm, bx0, bx0 + bs_), gyb)     # vertical midline (types 0, 2)
        hm = (gxb, gap(Ym, Ym, by0, by0 + bs_))     # horizontal midline (types 1, 2)
        best = None
        for gx, gy in segs:
            d2 = (gx * gx + gy * gy).astype(np.float64)
            best = d2 if best is None else np.minimum(best, d2)
        d2 = (vm[0] ** 2 + vm[1] ** 2).astype(np.float64)
        best = np.minimum(best, np.where((t == 0) | (t == 2), d2, np.inf))
        d2 = (hm[0] ** 2 + hm[1] ** 2).astype(np.float64)
        best = np.minimum(best, np.where((t == 1) | (t == 2), d2, np.inf))
        return best

    rows, cols = [], []
    for j in range(J + 1):
        A = np.flatnonzero(lev == j)
        for jp in range(j, J + 1):
            Bi = np.flatnonzero(lev == jp)
            bnd, bnds = cutoff_parameters(J, j, jp, a, delta, q, dtilde)
            near = (unit * 2.0 ** (-min(j, jp))) ** 2
            step = max(1, (1 << 22) // max(1, Bi.size))
            for c0 in range(0, A.size, step):
                ia = A[c0:c0 + step]
                d2 = np.zeros((ia.size, Bi.size))
                for ax in range(dim):
                    g = gap(lo[ia, ax][:, None], (lo[ia, ax] + side[ia])[:, None],
                            lo[Bi, ax][None, :], (lo[Bi, ax] + side[Bi])[None, :]).astype(np.float64)
                    d2 += g * g
                keep = np.ones_like(d2, bool)
                if j > 0:
                    keep &= d2 <= (unit * bnd) ** 2
                if jp > j:
                    far_sing = sing_dist2(ia, Bi) > (unit * bnds) ** 2
                    keep &= ~((d2 <= near) & far_sing)
                ii, kk = np.nonzero(keep)
                ra, cb = ia[ii], Bi[kk]
                rows.append(np.maximum(ra, cb))
                cols.append(np.minimum(ra, cb))
    r = np.concatenate(rows).astype(np.int64)
    c = np.concatenate(cols).astype(np.int64)
    key = np.unique(c * N + r)
    c = key // N
    r = key % N
    colptr = np.zeros(N + 1, np.int64)
    np.cumsum(np.bincount(c, minlength=N), out=colptr[1:])
    return colptr, r.astype(np.int32)


# --------------------------------------------------------------------------
# kernels and values
# --------------------------------------------------------------------------


@dataclass
class Kernel:
    """Isotropic covariance k(r) = sigma2 * f(r / ell)."""

    kind: str = "exponential"     # exponential | matern32 | matern12
    ell: float = 0.2
    sigma2: float = 1.0
    wrt: str = ""                 # "" -> k itself; "ell" / "sigma2" -> dk/d(parameter)

    def __call__(self, r, xp=np):
        t = r / self.ell
        if self.kind in ("exponential", "matern12"):
            e = xp.exp(-t)
            if self.wrt == "ell":
                return self.sigma2 * t * e / self.ell
            return (1.0 if self.wrt == "sigma2" else self.sigma2) * e
        if self.kind == "matern32":
            u = math.sqrt(3.0) * t
            e = xp.exp(-u)
            if self.wrt == "ell":
                return self.sigma2 * u * u * e / self.ell
            return (1.0 if self.wrt == "sigma2" else self.sigma2) * (1.0 + u) * e
        raise ValueError(self.kind)

    def derivative(self, param: str) -> "Kernel":
        """dk/d(param) for param in ("ell", "sigma2") as a kernel of the same
        family (the compressed matrix is linear in k, so mask(T dK T^T) is
        dA/d(param); the nugget's derivative is the identity)."""
        if param not in ("ell", "sigma2"):
            raise ValueError(param)
        return Kernel(self.kind, self.ell, self.sigma2, param)


def _cell_centroids(dim: int, J: int, xp=np, device=None):
    n = 1 << J
    if xp is np:
        c = (np.arange(n, dtype=np.float64) + 0.5) / n
        if dim == 1:
            return c[:, None]
        yy, xx = np.meshgrid(c, c, indexing="ij")
        return np.stack([xx.reshape(-1), yy.reshape(-1)], 1)
    c = (xp.arange(n, dtype=xp.float64, device=device) + 0.5) / n
    if dim == 1:
        return c[:, None]
    yy, xx = xp.meshgrid(c, c, indexing="ij")
    return xp.stack([xx.reshape(-1), yy.reshape(-1)], 1)


def _dist(a, b, xp):
    d2 = None
    for ax in range(a.shape[1]):
        d = a[:, None, ax] - b[None, :, ax]
        d2 = d * d if d2 is None else d2 + d * d
    return xp.sqrt(d2)


def compressed_values(basis: Basis, colptr, rowidx, kernel: Kernel, nugget: float,
                      device: str = "cpu", chunk: int = 2048):
    """Values of the compressed matrix on a lower CSC pattern (float64, numpy).

    A = mask(T K_ss T^T) + nugget*I, with the one-point cell-centroid rule.
    device='cpu' uses numpy; a CUDA device uses torch (the result is the same
    up to rounding; only needed when N^2 doubles do not fit the host).
    """
    dim, J, N = basis.dim, basis.J, basis.N
    n = 1 << J
    vol = 1.0 / float(N)                      # |c| = n^-dim = 1/N
    if device == "cpu":
        xp = np
        X = _cell_centroids(dim, J)
    else:
        import torch as xp  # noqa: N812
        if device.startswith("torch:"):       # torch on an explicit device, e.g. "torch:cpu"
            device = device[len("torch:"):]
        X = _cell_centroids(dim, J, xp, device)
    shape = (n,) if dim == 1 else (n, n)
    # pass 1: Y1 = K_ss T^T  (rows: cells, cols: wavelets)
    if xp is np:
        Y1 = np.empty((N, N), np.float64)
    else:
        Y1 = xp.empty((N, N), dtype=xp.float64, device=device)
    for c0 in range(0, N, chunk):
        c1 = min(N, c0 + chunk)
        K = kernel(_dist(X[c0:c1], X, xp), xp) * vol
        Y1[c0:c1] = fwt(K.reshape((c1 - c0,) + shape), dim, J, xp)
        del K
    # pass 2: A rows = T Y1 (columns of Y1 are cell vectors), gather the pattern
    cp = np.asarray(colptr)
    ri = np.asarray(rowidx).astype(np.int64)
    vals = np.empty(ri.size, np.float64)
    for c0 in range(0, N, chunk):
        c1 = min(N, c0 + chunk)
        Yc = Y1[:, c0:c1].T
        Yc = Yc.copy() if xp is np else Yc.contiguous()
        Arows = fwt(Yc.reshape((c1 - c0,) + shape), dim, J, xp)   # A[c0:c1, :]
        e0, e1 = int(cp[c0]), int(cp[c1])
        colid = np.repeat(np.arange(c0, c1), np.diff(cp[c0:c1 + 1])) - c0
        flat = colid * N + ri[e0:e1]
        if xp is np:
            vals[e0:e1] = Arows.reshape(-1)[flat]
        else:
            idx = xp.from_numpy(flat).to(device)
            vals[e0:e1] = Arows.reshape(-1)[idx].cpu().numpy()
        del Arows, Yc
    del Y1
    # nugget on the diagonal (first entry of every column)
    vals[cp[:-1]] += nugget
    return vals


def compressed_values_nonsym(basis: Basis, colptr, rowidx, kernel: Kernel, nugget: float,
                             beta: float = 0.5, direction=(1.0, 0.0)):
    """(lower, upper) values of a nonsymmetric compressed matrix on a lower
    CSC pattern: lower[e] = A[r][c], upper[e] = A[c][r] for every stored
    entry e = (r, c).  A = mask(T (K_ss + beta K_a) T^T) + nugget I with the
    symmetric kernel of compressed_values and the antisymmetric term
      K_a[c, c'] = sqrt(|c||c'|) ((x_c - x_c') . e / ell) k(x_c, x_c'),
    e = direction (1D: its first component), a transport-like term that
    stands in for the double-layer operator's nonsymmetric part (Section 6,
    PCM example).  The symmetric part of A is the SPD compressed matrix, so A
    has an LU factorization without pivoting.  Dense, for N up to a few
    thousand."""
    dim, J, N = basis.dim, basis.J, basis.N
    n = 1 << J
    vol = 1.0 / float(N)
    X = _cell_centroids(dim, J)
    D = _dist(X, X, np)
    e = np.asarray(direction, np.float64)[:dim]
    proj = X @ e if dim == 2 else X.reshape(-1) * e[0]
    diff = (proj[:, None] - proj[None, :]) / kernel.ell
    K = kernel(D, np) * (1.0 + beta * diff) * vol
    shape = (n,) if dim == 1 else (n, n)
    M1 = fwt(K.reshape((N,) + shape), dim, J, np)             # K T^T (rows transformed)
    A = fwt(np.ascontiguousarray(M1.T).reshape((N,) + shape), dim, J, np).T   # T K T^T
    cp = np.asarray(colptr)
    ri = np.asarray(rowidx).astype(np.int64)
    cols = np.repeat(np.arange(N), np.diff(cp))
    lower = A[ri, cols].copy()
    upper = A[cols, ri].copy()
    lower[cp[:-1]] += nugget
    upper[cp[:-1]] = lower[cp[:-1]]
    return lower, upper


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------


@dataclass
class Workload:
    name: str
    basis: Basis
    colptr: np.ndarray
    rowidx: np.ndarray
    values: np.ndarray
    B: np.ndarray            # (N, nrhs) float64, column-major (Fortran order)
    kernel: Kernel
    nugget: float
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.basis.N

    @property
    def nnz_lower(self) -> int:
        return int(self.rowidx.size)

    @property
    def nnz_full(self) -> int:
        return 2 * self.nnz_lower - self.N


def rhs(N: int, nrhs: int, seed: int = 0) -> np.ndarray:
    """nrhs standard normal vectors, (N, nrhs) column-major, original order."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nrhs, N)).T


def haar_workload(dim: int, J: int, kernel: Kernel, nugget: float, nrhs: int = 1,
                  seed: int = 0, device: str = "cpu", name: str | None = None,
                  values: bool = True) -> Workload:
    basis = haar_basis(dim, J)
    colptr, rowidx = compressed_pattern(basis)
    vals = (compressed_values(basis, colptr, rowidx, kernel, nugget, device)
            if values else np.empty(0))
    return Workload(name or f"haar{dim}d_J{J}", basis, colptr, rowidx, vals,
                    rhs(basis.N, nrhs, seed), kernel, nugget)


def workload_1d(J: int = 10, nrhs: int = 1, **kw) -> Workload:
    """1D: [0,1], 2^J cells, exponential kernel ell=0.2, nugget 1e-2."""
    return haar_workload(1, J, Kernel("exponential", 0.2), 1e-2, nrhs,
                         name=f"1d_haar_J{J}_exp0.2", **kw)


def workload_2d(J: int = 8, nrhs: int = 64, **kw) -> Workload:
    """2D: unit square 2^J x 2^J, Matern-3/2 ell=0.1, nugget 1e-3."""
    return haar_workload(2, J, Kernel("matern32", 0.1), 1e-3, nrhs,
                         name=f"2d_haar_{1 << J}x{1 << J}_matern32", **kw)


def workload_autograd(J: int = 7, nrhs: int = 32, ell: float = 0.15, sigma2: float = 1.0,
                      nugget: float = 1e-2, **kw) -> Workload:
    """2D Matern-1/2 workload of the gradient experiment."""
    return haar_workload(2, J, Kernel("matern12", ell, sigma2), nugget, nrhs,
                         name=f"2d_haar_{1 << J}x{1 << J}_matern12", **kw)


# --------------------------------------------------------------------------
# batch of independent instances
# --------------------------------------------------------------------------
BATCH_LEVELS = {1: (10, 11, 12, 13, 14), 2: (5, 6, 7)}


def batch_instances(count: int = 256, seed: int = 0):
    """Parameters of the batched configuration: instance i has dim 1 (even i)
    or 2 (odd i); J uniform over BATCH_LEVELS[dim] (N = 2^J or 4^J, from 1024
    to 16384); ell ~ U[0.05, 0.5]; exponential kernel, sigma^2 = 1, nugget
    1e-2.  Draw order per instance: J, then ell, from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        dim = 1 if i % 2 == 0 else 2
        levels = BATCH_LEVELS[dim]
        J = int(levels[int(rng.integers(len(levels)))])
        ell = float(rng.uniform(0.05, 0.5))
        out.append(dict(dim=dim, J=J, ell=ell, N=(1 << J) ** dim, nugget=1e-2))
    return out


@dataclass
class BatchWorkload:
    params: list
    bases: list              # one Basis per instance (shared objects per (dim, J))
    patterns: list           # (colptr, rowidx) per instance (shared per (dim, J))
    values: list             # per instance: float64 numpy array
    B: np.ndarray            # (sum N, nrhs): rows of the instances concatenated

    @property
    def N(self) -> int:
        return int(sum(p["N"] for p in self.params))


def batch_workload(count: int = 256, seed: int = 0, nrhs: int = 1, device: str = "cpu",
                   params=None) -> BatchWorkload:
    """The instances of batch_instances(count, seed) (or params): patterns and
    bases are built once per (dim, J) and shared; values per instance; right-
    hand sides rhs(sum N, nrhs, seed) over the concatenated rows."""
    params = batch_instances(count, seed) if params is None else params
    cache = {}
    bases, patterns, values = [], [], []
    for p in params:
        key = (p["dim"], p["J"])
        if key not in cache:
            b = haar_basis(p["dim"], p["J"])
            cache[key] = (b, compressed_pattern(b))
        b, (cp, ri) = cache[key]
        bases.append(b)
        patterns.append((cp, ri))
        values.append(compressed_values(b, cp, ri, Kernel("exponential", p["ell"]), p["nugget"], device))
    N = int(sum(p["N"] for p in params))
    return BatchWorkload(params, bases, patterns, values, rhs(N, nrhs, seed))
