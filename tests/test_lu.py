"""LU without pivoting on the nested-dissection ordering (Section 4: the
nonsymmetric case shares the ordering and the symbolic analysis; U has the
pattern of L transposed), for a nonsymmetric compressed operator (symmetric
kernel plus an antisymmetric transport-like term, standing in for the
double-layer part of Section 6's PCM example).

CPU: the oracle's LU is pinned by a hand-worked 3 x 3 example, by its
relation to the Cholesky factor on symmetric positive definite matrices
(L_lu = L D^-1, U_lu = D L^T with D = diag(L)), by L U = P A P^T and by
dense pivoted solves and determinants (numpy / LAPACK).
GPU: wd_factor_lu / wd_solve_lu / wd_logdet_lu through the C ABI against the
oracle.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from wdgen import (Kernel, compressed_pattern, compressed_values, compressed_values_nonsym, haar_basis,
                   rhs)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_lu_golden_tiny():
    g = json.load(open(os.path.join(GOLDEN, "tiny_lu.json")))
    a = g["lower_csc"]
    o = oracle.Oracle(a["colptr"], a["rowidx"])
    assert o.factor_lu(g["lower"], g["upper"]) == 0
    L, Ut = o.lu_values()
    np.testing.assert_allclose(L, g["L"], rtol=1e-15, atol=0)
    np.testing.assert_allclose(Ut, g["U_transposed"], rtol=1e-15, atol=0)
    v, sgn = o.logdet_lu()
    assert sgn == 1 and abs(v - math.log(96.0)) < 1e-14
    np.testing.assert_allclose(o.solve_lu(np.array(g["b"]))[:, 0], g["x"], rtol=0, atol=1e-14)


@pytest.mark.parametrize("dim,J", [(1, 7), (2, 4)])
def test_lu_of_spd_matrix_is_scaled_cholesky(dim, J):
    b = haar_basis(dim, J)
    cp, ri = compressed_pattern(b)
    v = compressed_values(b, cp, ri, Kernel("exponential", 0.2), 1e-2)
    o = oracle.Oracle(cp, ri, b, leaf=8)
    assert o.factor(v) == 0
    Lc = o.L_values()
    assert o.factor_lu(v, v) == 0
    L, Ut = o.lu_values()
    d = Lc[o.Lp[:-1]]
    col = np.repeat(np.arange(o.n), np.diff(o.Lp))
    np.testing.assert_allclose(L, Lc / d[col], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Ut, Lc * d[col], rtol=1e-12, atol=1e-15)


def _nonsym(dim, J, beta=0.5):
    b = haar_basis(dim, J)
    cp, ri = compressed_pattern(b)
    lo, up = compressed_values_nonsym(b, cp, ri, Kernel("exponential", 0.2), 1e-2, beta=beta)
    return b, cp, ri, lo, up


@pytest.mark.parametrize("dim,J", [(1, 7), (2, 4)])
def test_lu_reproduces_the_matrix_and_solves(dim, J):
    b, cp, ri, lo, up = _nonsym(dim, J)
    A = oracle.nonsym_lower_upper_to_dense(cp, ri, lo, up)
    assert np.abs(A - A.T).max() > 1e-3                      # genuinely nonsymmetric
    o = oracle.Oracle(cp, ri, b, leaf=8)
    assert o.factor_lu(lo, up) == 0
    L, Ut = o.lu_values()
    n = o.n
    Ld = np.zeros((n, n))
    Ud = np.zeros((n, n))
    col = np.repeat(np.arange(n), np.diff(o.Lp))
    Ld[o.Li, col] = L
    Ud[col, o.Li] = Ut
    PA = A[np.ix_(o.perm, o.perm)]
    assert np.abs(Ld @ Ud - PA).max() <= 1e-13 * np.abs(PA).max()
    B = rhs(n, 3, seed=2)
    X = o.solve_lu(B)
    np.testing.assert_allclose(X, np.linalg.solve(A, B), rtol=0, atol=1e-12 * np.abs(X).max())
    sgn, ld = np.linalg.slogdet(A)
    v, s = o.logdet_lu()
    assert s == int(sgn) and abs(v - ld) <= 1e-12 * abs(ld)


def test_lu_first_zero_pivot():
    n = 12
    A = 4 * np.eye(n) - np.eye(n, k=1) - 2 * np.eye(n, k=-1)
    A[5, 5] = 0.0
    A[5, 4] = 0.0
    A[4, 5] = 0.0
    cp = [0]
    ri, lo, up = [], [], []
    for j in range(n):
        rows = [i for i in range(j, n) if i == j or A[i, j] != 0 or A[j, i] != 0]
        ri += rows
        lo += [A[i, j] for i in rows]
        up += [A[j, i] for i in rows]
        cp.append(len(ri))
    o = oracle.Oracle(np.array(cp), np.array(ri, np.int32))
    assert o.factor_lu(np.array(lo), np.array(up)) == -(5 + 1)


# ---------------------------------------------------------------------------
# GPU: the C ABI against the oracle.  Tolerances as for the FP64 Cholesky:
# factor entries differ only by summation order (per column 1e-10 relative),
# solves reach a normwise backward error of 1e-12, log |det| 1e-12 relative.
# ---------------------------------------------------------------------------
GPU_CASES = {"1d_J10": (1, 10, 0.5), "2d_J5": (2, 5, 0.5), "2d_J6": (2, 6, 1.0)}
_gcache = {}


def _gcase(name):
    if name not in _gcache:
        dim, J, beta = GPU_CASES[name]
        b, cp, ri, lo, up = _nonsym(dim, J, beta)
        o = oracle.Oracle(cp, ri, b)
        assert o.factor_lu(lo, up) == 0
        _gcache[name] = (b, cp, ri, lo, up, o)
    return _gcache[name]


def _columns_close(got, ref, Lp, tol):
    for j in range(Lp.size - 1):
        a, e = Lp[j], Lp[j + 1]
        assert np.linalg.norm(got[a:e] - ref[a:e]) <= tol * np.linalg.norm(ref[a:e]), j


@pytest.mark.gpu
@pytest.mark.parametrize("name", list(GPU_CASES))
def test_gpu_lu_factor_entries(wdlib, cuda, name):
    b, cp, ri, lo, up, o = _gcase(name)
    s = wdlib.Solver().analyze(cp, ri, b)
    s.factor_lu(lo, up)
    Lg, Utg = s.export_LU()
    L = s.L_csc_like(o.Lp, o.Li, Lg)
    Ut = s.L_csc_like(o.Lp, o.Li, Utg)
    Lo, Uto = o.lu_values()
    _columns_close(L, Lo, o.Lp, 1e-10)
    _columns_close(Ut, Uto, o.Lp, 1e-10)


@pytest.mark.gpu
@pytest.mark.parametrize("name", list(GPU_CASES))
@pytest.mark.parametrize("nrhs", [1, 5, 16, 37])
def test_gpu_lu_solve(wdlib, cuda, name, nrhs):
    torch = cuda
    b, cp, ri, lo, up, o = _gcase(name)
    s = wdlib.Solver().analyze(cp, ri, b).factor_lu(lo, up)
    B = rhs(o.n, nrhs, seed=nrhs)
    X = s.solve_lu(B)                                     # host arrays
    assert oracle.nonsym_backward_error(cp, ri, lo, up, X, B).max() <= 1e-12
    Xo = o.solve_lu(B)
    assert np.abs(X - Xo).max() <= 1e-9 * np.abs(Xo).max()
    # device tensors, values given on the device, a leading dimension > n
    Bd = torch.empty((nrhs, o.n + 3), dtype=torch.float64, device="cuda").t()[: o.n]
    Bd.copy_(torch.from_numpy(B))
    s2 = wdlib.Solver().analyze(cp, ri, b)
    s2.factor_lu(torch.from_numpy(lo).cuda(), torch.from_numpy(up).cuda())
    s2.solve_lu(Bd)
    torch.cuda.synchronize()
    assert np.abs(Bd.cpu().numpy() - X).max() <= 1e-12 * np.abs(X).max()


@pytest.mark.gpu
@pytest.mark.parametrize("name", list(GPU_CASES))
def test_gpu_lu_logdet(wdlib, cuda, name):
    b, cp, ri, lo, up, o = _gcase(name)
    s = wdlib.Solver().analyze(cp, ri, b).factor_lu(lo, up)
    v, sg = s.logdet_lu()
    vo, so = o.logdet_lu()
    assert sg == so and abs(v - vo) <= 1e-12 * abs(vo)


@pytest.mark.gpu
def test_gpu_lu_negative_determinant(wdlib, cuda):
    """One pivot flipped in sign: the sign of det A follows, |det A| as the
    oracle's."""
    b, cp, ri, lo, up = _nonsym(1, 8)
    lo = lo.copy()
    lo[cp[5]] = -lo[cp[5]]                                # A[5][5] < 0
    o = oracle.Oracle(cp, ri, b)
    if o.factor_lu(lo, up) != 0:
        pytest.skip("the flipped pivot made the matrix singular without pivoting")
    s = wdlib.Solver().analyze(cp, ri, b).factor_lu(lo, up)
    v, sg = s.logdet_lu()
    vo, so = o.logdet_lu()
    assert sg == so and abs(v - vo) <= 1e-12 * abs(vo)
    A = oracle.nonsym_lower_upper_to_dense(cp, ri, lo, up)
    assert sg == int(np.linalg.slogdet(A)[0])


@pytest.mark.gpu
def test_gpu_lu_zero_pivot(wdlib, cuda):
    n = 12
    A = 4 * np.eye(n) - np.eye(n, k=1) - 2 * np.eye(n, k=-1)
    A[5, 5] = A[5, 4] = A[4, 5] = 0.0
    cp = [0]
    ri, lo, up = [], [], []
    for j in range(n):
        rows = [i for i in range(j, n) if i == j or A[i, j] != 0 or A[j, i] != 0]
        ri += rows
        lo += [A[i, j] for i in rows]
        up += [A[j, i] for i in rows]
        cp.append(len(ri))
    cp, ri, lo, up = np.array(cp), np.array(ri, np.int32), np.array(lo), np.array(up)
    o = oracle.Oracle(cp, ri)
    zo = -o.factor_lu(lo, up) - 1
    s = wdlib.Solver().analyze(cp, ri)
    with pytest.raises(wdlib.WdError) as e:
        s.factor_lu(lo, up)
    assert e.value.status == wdlib.WD_ERR_NOT_SPD
    # the same original unknown as the oracle's first zero pivot
    assert s.symbolic()["perm"][e.value.column] == o.perm[zo]
    with pytest.raises(wdlib.WdError):
        s.solve_lu(np.ones(n))                            # no factor after the failure


@pytest.mark.gpu
def test_gpu_lu_and_cholesky_share_a_handle(wdlib, cuda):
    """LU of a symmetric positive definite matrix is the scaled Cholesky factor;
    a Cholesky factor after an LU on the same handle is unaffected by it."""
    b = haar_basis(2, 5)
    cp, ri = compressed_pattern(b)
    v = compressed_values(b, cp, ri, Kernel("matern32", 0.1), 1e-3)
    o = oracle.Oracle(cp, ri, b)
    assert o.factor(v) == 0
    s = wdlib.Solver().analyze(cp, ri, b)
    s.factor_lu(v, v)
    Lg, Utg = s.export_LU()
    L = s.L_csc_like(o.Lp, o.Li, Lg)
    Ut = s.L_csc_like(o.Lp, o.Li, Utg)
    Lc = o.L_values()
    d = Lc[o.Lp[:-1]]
    col = np.repeat(np.arange(o.n), np.diff(o.Lp))
    _columns_close(L, Lc / d[col], o.Lp, 1e-10)
    _columns_close(Ut, Lc * d[col], o.Lp, 1e-10)
    v_lu, sg = s.logdet_lu()
    assert sg == 1 and abs(v_lu - o.logdet()) <= 1e-12 * abs(o.logdet())
    for prec in ("fp64", "mixed"):
        s.factor(v, prec)
        B = rhs(o.n, 4, seed=3)
        X = s.solve(B)
        assert oracle.backward_error(cp, ri, v, X, B).max() <= 1e-12
        tol = 1e-12 if prec == "fp64" else 1e-5      # the mixed factor's pivots are FP32
        assert abs(s.logdet() - o.logdet()) <= tol * abs(o.logdet())
    with pytest.raises(wdlib.WdError):
        s.solve_lu(B)                                     # the LU factor is gone
