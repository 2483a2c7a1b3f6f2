"""LDL^T without pivoting on the nested-dissection ordering: the symmetric case
of the LU decomposition (Section 4 factors the compressed matrix by a
Cholesky or an LU decomposition on the same ordering and symbolic analysis),
for symmetric matrices that need not be positive definite: P A P^T = L D L^T
with L unit lower triangular on the Cholesky pattern and D diagonal.

CPU: the oracle's LDL^T is pinned by a hand-worked 3 x 3 indefinite example,
by its relation to the Cholesky factor on positive definite matrices
(L = L_chol diag(L_chol)^-1, d = diag(L_chol)^2, against LAPACK's dense
Cholesky), by L D L^T = P A P^T within the textbook backward-error bound,
by Sylvester's law of inertia (the number of negative pivots equals the
number of negative eigenvalues, LAPACK's symmetric eigensolver), by dense
solves and determinants, and by the first zero pivot of a hand-made matrix.
GPU: wd_factor_ldlt / wd_solve_lu / wd_inertia through the C ABI against the
oracle, including the cubed sphere at nugget 1e-3, which is indefinite
(its Cholesky factorization stops with WD_ERR_NOT_SPD).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from wdgen import Kernel, compressed_pattern, compressed_values, haar_basis, rhs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_ldlt_golden_tiny():
    g = json.load(open(os.path.join(GOLDEN, "tiny_ldlt.json")))
    a = g["lower_csc"]
    o = oracle.Oracle(a["colptr"], a["rowidx"])
    assert o.factor_ldlt(g["values"]) == 0
    L, d = o.ldlt_values()
    np.testing.assert_allclose(L, g["L"], rtol=1e-15, atol=0)
    np.testing.assert_allclose(d, g["d"], rtol=1e-15, atol=0)
    v, sgn, neg = o.logdet_ldlt()
    assert sgn == g["sign"] and neg == g["negative_pivots"]
    assert abs(v - g["logabsdet"]) < 1e-14
    np.testing.assert_allclose(o.solve_ldlt(np.array(g["b"]))[:, 0], g["x"], rtol=0, atol=1e-15)


def _dense_factors(o, L, d):
    n = o.n
    Ld = np.zeros((n, n))
    col = np.repeat(np.arange(n), np.diff(o.Lp))
    Ld[o.Li, col] = L
    return Ld, d


@pytest.mark.parametrize("dim,J", [(1, 7), (2, 4)])
def test_ldlt_of_spd_matrix_is_scaled_lapack_cholesky(dim, J):
    b = haar_basis(dim, J)
    cp, ri = compressed_pattern(b)
    v = compressed_values(b, cp, ri, Kernel("exponential", 0.2), 1e-2)
    o = oracle.Oracle(cp, ri, b, leaf=8)
    assert o.factor_ldlt(v) == 0
    L, d = o.ldlt_values()
    A = oracle.sym_lower_to_dense(cp, ri, v)
    C = np.linalg.cholesky(A[np.ix_(o.perm, o.perm)])       # LAPACK
    dc = np.diag(C)
    np.testing.assert_allclose(d, dc ** 2, rtol=1e-12)
    Ld, _ = _dense_factors(o, L, d)
    np.testing.assert_allclose(Ld, C / dc[None, :], rtol=0, atol=1e-12)
    v_, sgn, neg = o.logdet_ldlt()
    assert sgn == 1 and neg == 0


def _indefinite(dim, J):
    """The compressed matrix minus sigma I, sigma the midpoint of the widest
    gap of its spectrum with at least a tenth of the eigenvalues on each
    side: symmetric, indefinite, and as far from singular as a shift into
    the middle of the spectrum allows."""
    b = haar_basis(dim, J)
    cp, ri = compressed_pattern(b)
    v = compressed_values(b, cp, ri, Kernel("exponential", 0.2), 1e-2)
    A = oracle.sym_lower_to_dense(cp, ri, v)
    lam = np.linalg.eigvalsh(A)
    lo, hi = lam.size // 10, lam.size - lam.size // 10
    g = lo + int(np.argmax(np.diff(lam[lo:hi])))
    sigma = 0.5 * (lam[g] + lam[g + 1])
    v = v.copy()
    v[np.asarray(cp)[:-1]] -= sigma                          # the diagonal is first in every column
    return b, cp, ri, v, A - sigma * np.eye(A.shape[0])


@pytest.mark.parametrize("dim,J", [(1, 7), (2, 4)])
def test_ldlt_of_indefinite_matrix(dim, J):
    b, cp, ri, v, A = _indefinite(dim, J)
    o = oracle.Oracle(cp, ri, b, leaf=8)
    assert o.factor(v) != 0                                  # not positive definite
    assert o.factor_ldlt(v) == 0
    L, d = o.ldlt_values()
    Ld, _ = _dense_factors(o, L, d)
    PA = A[np.ix_(o.perm, o.perm)]
    # backward-error bound of LDL^T without pivoting: |L D L^T - P A P^T| <= c u |L| |D| |L|^T
    growth = np.abs(Ld) @ np.diag(np.abs(d)) @ np.abs(Ld).T
    assert np.all(np.abs(Ld @ np.diag(d) @ Ld.T - PA) <= 1e-13 * growth + 1e-15 * np.abs(PA).max())
    # Sylvester's law of inertia
    lam = np.linalg.eigvalsh(A)
    v_, sgn, neg = o.logdet_ldlt()
    assert neg == int(np.sum(lam < 0)) and 0 < neg < o.n
    s_ref, ld_ref = np.linalg.slogdet(A)
    assert sgn == int(s_ref) and abs(v_ - ld_ref) <= 1e-10 * abs(ld_ref)
    B = rhs(o.n, 3, seed=4)
    X = o.solve_ldlt(B)
    Xr = np.linalg.solve(A, B)
    np.testing.assert_allclose(X, Xr, rtol=0, atol=1e-8 * np.abs(Xr).max())


def test_ldlt_first_zero_pivot():
    """A = [[2,0,0,0],[0,1,1,0],[0,1,1,1],[0,0,1,3]] in natural order: d0 = 2,
    d1 = 1, L21 = 1, d2 = 1 - 1 * 1 = 0 exactly (binary arithmetic), so the
    first zero pivot is column 2 although A is nonsingular (det = -2)."""
    A = np.array([[2., 0, 0, 0], [0, 1, 1, 0], [0, 1, 1, 1], [0, 0, 1, 3]])
    assert abs(np.linalg.det(A) + 2) < 1e-12
    cp = [0]
    ri, vals = [], []
    for j in range(4):
        rows = [i for i in range(j, 4) if i == j or A[i, j] != 0]
        ri += rows
        vals += [A[i, j] for i in rows]
        cp.append(len(ri))
    o = oracle.Oracle(np.array(cp), np.array(ri, np.int32))
    assert o.factor_ldlt(np.array(vals)) == -(2 + 1)


# ---------------------------------------------------------------------------
# GPU: the C ABI against the oracle.  Factor entries differ only by summation
# order, but without pivoting an indefinite matrix's rounding errors grow with
# the factorization's growth g = max(|L| |D| |L|^T) / max|A| (the quantity of
# the backward-error bound pinned above): per column 1e-12 g relative, and
# never below the positive definite bar 1e-10.  Solves reach a normwise
# backward error of 1e-12, log |det| 1e-12 relative; the inertia is an
# integer and must be equal.
# ---------------------------------------------------------------------------
_gcache = {}


def _gcase(name):
    if name not in _gcache:
        if name == "sphere_J4_nugget1e-3":
            from wdgen.sphere import sphere_basis, sphere_pattern, sphere_values
            b = sphere_basis(4)
            cp, ri = sphere_pattern(b, "cpu")
            v = sphere_values(b, cp, ri, Kernel("exponential", 0.3), 1e-3, "cpu")
        else:
            dim, J = {"1d_J10_shifted": (1, 10), "2d_J5_shifted": (2, 5)}[name]
            b, cp, ri, v, _ = _indefinite(dim, J)
        o = oracle.Oracle(cp, ri, b)
        assert o.factor_ldlt(v) == 0
        L, d = o.ldlt_values()
        Ld, _ = _dense_factors(o, L, d)
        g = (np.abs(Ld) @ np.diag(np.abs(d)) @ np.abs(Ld).T).max() / np.abs(oracle.sym_lower_to_dense(cp, ri, v)).max()
        _gcache[name] = (b, cp, ri, v, o, max(1e-10, 1e-12 * g))
    return _gcache[name]


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["1d_J10_shifted", "2d_J5_shifted", "sphere_J4_nugget1e-3"])
def test_gpu_ldlt_indefinite(wdlib, cuda, name):
    b, cp, ri, v, o, tol = _gcase(name)
    s = wdlib.Solver().analyze(cp, ri, b)
    with pytest.raises(wdlib.WdError) as e:
        s.factor(v, "fp64")                       # indefinite: no Cholesky factor
    assert e.value.status == wdlib.WD_ERR_NOT_SPD
    s.factor_ldlt(v)
    Lg, Utg = s.export_LU()
    L = s.L_csc_like(o.Lp, o.Li, Lg)
    Ut = s.L_csc_like(o.Lp, o.Li, Utg)
    Lo, do = o.ldlt_values()
    for j in range(o.n):
        a, e_ = o.Lp[j], o.Lp[j + 1]
        assert np.linalg.norm(L[a:e_] - Lo[a:e_]) <= tol * np.linalg.norm(Lo[a:e_]), (j, tol)
    d = Ut[o.Lp[:-1]]                              # D on the diagonal of U^T
    np.testing.assert_allclose(d, do, rtol=tol)
    ld, sg, neg = o.logdet_ldlt()
    pos_g, neg_g = s.inertia()
    assert (pos_g, neg_g) == (o.n - neg, neg) and neg > 0
    v_g, sg_g = s.logdet_lu()
    assert sg_g == sg and abs(v_g - ld) <= 1e-12 * abs(ld)
    B = rhs(o.n, 5, seed=3)
    X = s.solve_lu(B)
    assert oracle.backward_error(cp, ri, v, X, B).max() <= 1e-12
    Xo = o.solve_ldlt(B)
    np.testing.assert_allclose(X, Xo, rtol=0, atol=1e-9 * np.abs(Xo).max())


@pytest.mark.gpu
def test_gpu_ldlt_on_device_values_and_state(wdlib, cuda):
    torch = cuda
    b, cp, ri, v, o, _ = _gcase("2d_J5_shifted")
    s = wdlib.Solver().analyze(cp, ri, b)
    with pytest.raises(wdlib.WdError) as e:
        s.inertia()                                # no LDL^T factor yet
    assert e.value.status == wdlib.WD_ERR_STATE
    s.factor_ldlt(torch.from_numpy(v).cuda())
    assert s.inertia()[1] == o.logdet_ldlt()[2]
    s.factor_lu(v, v)                              # a plain LU factor: no inertia
    with pytest.raises(wdlib.WdError) as e:
        s.inertia()
    assert e.value.status == wdlib.WD_ERR_STATE
