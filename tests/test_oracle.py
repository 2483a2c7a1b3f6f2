"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these compare the oracle with itself: they use a hand-derived example,
dense LAPACK factorizations and inverses, the path characterisation of fill
(Lemma of Section 4), the separator property of nested dissection (Section 4),
closed forms and special cases.
"""
import json
import math
import os
from collections import deque

import numpy as np
import pytest

import oracle
from wdgen import haar_basis, compressed_pattern, compressed_values, Kernel, rhs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_workloads():
    out = []
    for dim, J, ker, nug in ((1, 7, Kernel("exponential", 0.2), 1e-2),
                             (2, 3, Kernel("matern32", 0.1), 1e-3),
                             (2, 4, Kernel("exponential", 0.3), 1e-2)):
        b = haar_basis(dim, J)
        cp, ri = compressed_pattern(b)
        v = compressed_values(b, cp, ri, ker, nug)
        out.append((f"{dim}d_J{J}", b, cp, ri, v))
    return out


WL = _small_workloads()


def _random_spd(n, density, seed):
    rng = np.random.default_rng(seed)
    M = (rng.random((n, n)) < density).astype(float) * rng.standard_normal((n, n))
    A = np.tril(M, -1)
    A = A + A.T
    A += np.diag(np.abs(A).sum(1) + 1.0)
    return A


def _dense_to_lower_csc(A):
    n = A.shape[0]
    cp = [0]
    ri, v = [], []
    for j in range(n):
        rows = [i for i in range(j, n) if i == j or A[i, j] != 0.0]
        ri += rows
        v += [A[i, j] for i in rows]
        cp.append(len(ri))
    return np.array(cp, np.int64), np.array(ri, np.int32), np.array(v)


def test_golden_tiny():
    g = json.load(open(os.path.join(GOLDEN, "tiny_cholesky.json")))
    a = g["lower_csc"]
    o = oracle.Oracle(a["colptr"], a["rowidx"])
    assert list(o.perm) == [0, 1, 2]
    assert list(o.Lp) == g["L_pattern"]["colptr"]
    assert list(o.Li) == g["L_pattern"]["rowidx"]
    assert o.factor(np.array(a["values"])) == 0
    np.testing.assert_allclose(o.L_values(), g["L_values"], rtol=1e-15, atol=0)
    assert abs(o.logdet() - g["logdet"]) < 1e-14
    np.testing.assert_allclose(o.solve(np.array(g["b"]))[:, 0], g["x"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(o.selinv() * 124.0, g["selinv_on_L_pattern_times_124"],
                               rtol=1e-14, atol=1e-13)
    # parent: column 0 -> 1 -> 2; counts 2, 2, 1
    assert list(o.parent) == [1, 2, -1]
    assert list(o.colcount) == [2, 2, 1]


@pytest.mark.parametrize("name,b,cp,ri,v", WL, ids=[w[0] for w in WL])
def test_cholesky_equals_dense_lapack(name, b, cp, ri, v):
    o = oracle.Oracle(cp, ri, b, leaf=8)
    assert o.factor(v) == 0
    A = oracle.sym_lower_to_dense(cp, ri, v)
    P = A[np.ix_(o.perm, o.perm)]
    Ld = np.linalg.cholesky(P)
    L = o.L_dense()
    # per column relative agreement, and no entry outside the structure
    for j in range(o.n):
        assert np.linalg.norm(L[:, j] - Ld[:, j]) <= 1e-13 * np.linalg.norm(Ld[:, j])
    mask = np.zeros_like(L, bool)
    cols = np.repeat(np.arange(o.n), np.diff(o.Lp))
    mask[o.Li, cols] = True
    assert np.abs(Ld[~mask]).max(initial=0.0) <= 1e-13 * np.abs(Ld).max()
    # factorization residual on the whole matrix
    assert np.linalg.norm(P - L @ L.T) <= 1e-13 * np.linalg.norm(P)


@pytest.mark.parametrize("name,b,cp,ri,v", WL, ids=[w[0] for w in WL])
def test_solve_logdet_apply_selinv_dense(name, b, cp, ri, v):
    o = oracle.Oracle(cp, ri, b, leaf=8)
    assert o.factor(v) == 0
    A = oracle.sym_lower_to_dense(cp, ri, v)
    B = rhs(o.n, 3, seed=1)
    X = o.solve(B)
    Xd = np.linalg.solve(A, B)
    assert np.abs(X - Xd).max() <= 1e-11 * np.abs(Xd).max()
    assert oracle.backward_error(cp, ri, v, X, B).max() <= 1e-15
    sign, ld = np.linalg.slogdet(A)
    assert sign > 0 and abs(o.logdet() - ld) <= 1e-12 * abs(ld)
    # apply_L: columns of P^T L from unit vectors, and (P^T L)(P^T L)^T = A
    E = np.eye(o.n)[:, :5]
    S = o.apply_L(E)
    L = o.L_dense()
    PtL = np.empty_like(L)
    PtL[o.perm] = L
    np.testing.assert_allclose(S, PtL[:, :5], rtol=0, atol=1e-15)
    S_all = o.apply_L(np.eye(o.n))
    assert np.abs(S_all @ S_all.T - A).max() <= 1e-13 * np.abs(A).max()
    # selected inverse equals the dense inverse on the pattern of L
    Z = o.selinv()
    Ainv = np.linalg.inv(A[np.ix_(o.perm, o.perm)])
    cols = np.repeat(np.arange(o.n), np.diff(o.Lp))
    np.testing.assert_allclose(Z, Ainv[o.Li, cols], rtol=0, atol=1e-11 * np.abs(Ainv).max())


def _lemma_structure(n, adj_sets):
    """struct(L_{:,j}) from the path characterisation of the Lemma in
    Section 4: i > j is in it iff a path i ... j exists whose interior
    vertices are all numbered below j."""
    out = []
    for j in range(n):
        seen = {j}
        dq = deque([j])
        reach = []
        while dq:
            u = dq.popleft()
            for w in adj_sets[u]:
                if w < j and w not in seen:
                    seen.add(w)
                    dq.append(w)
            reach.append(u)
        s = set()
        for u in reach:
            for w in adj_sets[u]:
                if w > j:
                    s.add(w)
        out.append(sorted(s))
    return out


@pytest.mark.parametrize("case", ["1d", "2d", "rand"])
def test_fill_lemma_bruteforce(case):
    if case == "1d":
        b = haar_basis(1, 7)
        cp, ri = compressed_pattern(b)
        o = oracle.Oracle(cp, ri, b, leaf=8)
    elif case == "2d":
        b = haar_basis(2, 3)
        cp, ri = compressed_pattern(b)
        o = oracle.Oracle(cp, ri, b, leaf=8)
    else:
        A = _random_spd(150, 0.03, 7)
        cp, ri, _ = _dense_to_lower_csc(A)
        o = oracle.Oracle(cp, ri)
    n = o.n
    assert n <= 200
    iperm = np.empty(n, np.int64)
    iperm[o.perm] = np.arange(n)
    adj = [set() for _ in range(n)]
    cols = np.repeat(np.arange(n), np.diff(cp))
    for i, j in zip(ri, cols):
        if i != j:
            a, c = int(iperm[i]), int(iperm[j])
            adj[a].add(c)
            adj[c].add(a)
    ref = _lemma_structure(n, adj)
    for j in range(n):
        got = list(o.Li[o.Lp[j] + 1: o.Lp[j + 1]])
        assert got == ref[j], j
        assert o.colcount[j] == len(ref[j]) + 1
        assert o.parent[j] == (ref[j][0] if ref[j] else -1)
        assert o.parent[j] == -1 or o.parent[j] > j


@pytest.mark.parametrize("dim,J,leaf", [(1, 8, 8), (2, 4, 16), (2, 5, 32)])
def test_nd_separator_property(dim, J, leaf):
    b = haar_basis(dim, J)
    cp, ri = compressed_pattern(b)
    perm, tree = oracle.nd_order(cp, ri, b, leaf=leaf, want_tree=True)
    n = b.N
    assert sorted(perm) == list(range(n))
    assert len(tree) > 0
    pos = np.empty(n, np.int64)
    pos[perm] = np.arange(n)
    cols = np.repeat(np.arange(n), np.diff(cp))
    off = ri != cols
    pa, pb = pos[ri[off]], pos[cols[off]]
    for s0, s1, s2, s3 in tree:
        assert s0 <= s1 <= s2 <= s3
        in1a = (pa >= s0) & (pa < s1)
        in2a = (pa >= s1) & (pa < s2)
        in1b = (pb >= s0) & (pb < s1)
        in2b = (pb >= s1) & (pb < s2)
        # no edge between V1 and V2 (block form of P A P^T in Section 4)
        assert not np.any((in1a & in2b) | (in2a & in1b))


def test_nd_coarsest_last():
    """The root separator ends with the level-0 function; separators are
    ordered finest level first."""
    b = haar_basis(2, 5)
    cp, ri = compressed_pattern(b)
    perm, tree = oracle.nd_order(cp, ri, b, leaf=64, want_tree=True)
    assert b.level[perm[-1]] == 0
    root = max(tree, key=lambda t: t[3] - t[0])
    assert root[3] == b.N
    seg = b.level[perm[root[2]:root[3]]]
    assert np.all(np.diff(seg) <= 0)


def test_closed_form_scaled_identity():
    b = haar_basis(1, 6)
    cp, ri = compressed_pattern(b)
    eps = 1e-2
    v = np.zeros(ri.size)
    v[cp[:-1]] = eps
    o = oracle.Oracle(cp, ri, b, leaf=8)
    assert o.factor(v) == 0
    Lx = o.L_values()
    diag = Lx[o.Lp[:-1]]
    np.testing.assert_allclose(diag, math.sqrt(eps), rtol=1e-16)
    off = np.ones(Lx.size, bool)
    off[o.Lp[:-1]] = False
    assert np.all(Lx[off] == 0.0)
    assert abs(o.logdet() - b.N * math.log(eps)) <= 1e-13 * abs(b.N * math.log(eps))


def test_special_case_diagonal_and_tridiagonal():
    n = 50
    cp = np.arange(n + 1, dtype=np.int64)
    ri = np.arange(n, dtype=np.int32)
    o = oracle.Oracle(cp, ri)
    assert np.all(o.parent == -1) and o.nnzL == n
    # tridiagonal in natural order: no fill, chain etree
    A = 4 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    cp, ri, v = _dense_to_lower_csc(A)
    o = oracle.Oracle(cp, ri, relax_k=16, relax_pct=10)
    assert o.nnzL == 2 * n - 1
    assert list(o.parent) == list(range(1, n)) + [-1]
    assert o.factor(v) == 0
    # path graph: fundamental supernodes are singletons except {n-2, n-1};
    # the merge scan joins consecutive ones while the width stays <= 16
    # (width 17 would add 136 explicit zeros to a 170-entry trapezoid)
    assert list(o.super_first) == [0, 16, 32, 48, 50]
    # with width 64 allowed the whole path is one supernode
    assert list(oracle.Oracle(cp, ri, relax_k=64, relax_pct=10).super_first) == [0, 50]


def test_supernode_rows_and_partition():
    b = haar_basis(2, 5)
    cp, ri = compressed_pattern(b)
    o = oracle.Oracle(cp, ri, b)
    assert o.super_first[0] == 0 and o.super_first[-1] == o.n
    assert np.all(np.diff(o.super_first) > 0)
    for f, e, rows in o.supernodes():
        assert list(rows[: e - f]) == list(range(f, e))
        assert np.all(np.diff(rows) > 0)
        # every column's structure lies inside the supernode's rows
        rs = set(rows.tolist())
        for j in range(f, e):
            assert set(o.Li[o.Lp[j]: o.Lp[j + 1]].tolist()) <= rs
        # the last column's structure is exactly the rows from it onward
        assert list(o.Li[o.Lp[e - 1]: o.Lp[e]]) == list(rows[e - 1 - f:])


def test_dense_matrix_single_supernode():
    n = 30
    A = _random_spd(n, 1.0, 3)
    cp, ri, v = _dense_to_lower_csc(A)
    o = oracle.Oracle(cp, ri)
    assert o.nsuper == 1 and o.nnzL == n * (n + 1) // 2
    assert o.factor(v) == 0
    np.testing.assert_allclose(o.L_dense(), np.linalg.cholesky(A), rtol=0, atol=1e-13)


def test_not_spd_reports_first_column():
    n = 20
    A = 4 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    A[7, 7] = -1.0
    A[12, 12] = -1.0
    cp, ri, v = _dense_to_lower_csc(A)
    o = oracle.Oracle(cp, ri)
    assert o.factor(v) == -(7 + 1)


def test_malformed_pattern_rejected():
    cp = np.array([0, 2, 3], np.int64)
    with pytest.raises(ValueError):
        oracle.Oracle(cp, np.array([1, 0, 1], np.int32))   # diagonal not first
    with pytest.raises(ValueError):
        oracle.Oracle(cp, np.array([0, 5, 1], np.int32))   # row out of range


def test_backward_error_definition():
    A = np.array([[2.0, 1.0], [1.0, 3.0]])
    cp, ri, v = _dense_to_lower_csc(A)
    x = np.array([[1.0], [1.0]])
    b = np.array([[3.0], [4.5]])          # A x = [3, 4]: residual 0.5
    be = oracle.backward_error(cp, ri, v, x, b)
    # ||A||_inf = 4, ||x|| = 1, ||b|| = 4.5
    assert abs(be[0] - 0.5 / (4.0 + 4.5)) < 1e-16


def _amalgamation_cases():
    g = json.load(open(os.path.join(GOLDEN, "amalgamation.json")))
    return [(c, r) for c in g["cases"] for r in c["runs"]]


@pytest.mark.parametrize("case,run", _amalgamation_cases(),
                         ids=[f"{c['name'][:4]}-k{r['relax_k']}-p{r['relax_pct']}" for c, r in _amalgamation_cases()])
def test_amalgamation_percentage_branch(case, run):
    """Hand-worked merges decided by the explicit-zero percentage (the width
    threshold lies below every merged width), one run just below and one just
    above each threshold: an off-by-one in the trapezoid or in the zero count
    moves a threshold across one of them."""
    a = case["lower_csc"]
    o = oracle.Oracle(a["colptr"], a["rowidx"], relax_k=run["relax_k"], relax_pct=run["relax_pct"])
    assert list(o.perm) == list(range(len(a["colptr"]) - 1))
    assert list(o.parent) == case["parent"]
    assert list(o.colcount) == case["colcount"]
    assert list(o.super_first) == run["super_first"]


def test_solve_prefix_over_all_columns_is_the_solve():
    """The timing helper runs solve()'s loops over a prefix of the columns:
    over all of them it is the solve (in factor order)."""
    name, b, cp, ri, v = WL[0]
    o = oracle.Oracle(cp, ri, b, leaf=8)
    assert o.factor(v) == 0
    B = rhs(o.n, 3, 0)
    X = o.solve(B)
    Y = np.asfortranarray(B[o.perm])
    o.solve_prefix(Y, o.n)
    np.testing.assert_array_equal(Y, X[o.perm])
