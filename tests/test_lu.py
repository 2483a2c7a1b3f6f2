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
