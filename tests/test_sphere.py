"""Cubed-sphere generator and the patch-first dissection (CPU).

Pins: the panel areas tile the sphere (sum 4 pi); the paired patches share an
edge; the compressed pattern and values against their definitions written
out densely (brute force over all pairs, T K T^T with T from the transform of
the identity); the library's ordering and symbolic analysis bit-exact
against the oracle's independent implementation; the separator property and
the patch split at the root of the dissection.
"""
import math

import numpy as np
import pytest

import oracle
from wdgen import Kernel, fwt
from wdgen.sphere import (NPATCH, panel_grid, sphere_basis, sphere_pattern, sphere_values,
                          support_spheres)


@pytest.mark.parametrize("J", [1, 2, 3, 5])
def test_panels_tile_the_sphere(J):
    pts, areas, corners = panel_grid(J)
    assert abs(areas.sum() - 4 * math.pi) <= 1e-12
    assert areas.min() > 0
    np.testing.assert_allclose(np.linalg.norm(pts, axis=-1), 1.0, atol=1e-15)
    np.testing.assert_allclose(np.linalg.norm(corners, axis=-1), 1.0, atol=1e-15)


def test_paired_patches_share_an_edge():
    J = 3
    _, _, corners = panel_grid(J)
    n1 = (1 << J) + 1
    for a, b in [(0, 1), (2, 3), (4, 5)]:
        ca = corners[a].reshape(-1, 3)
        cb = corners[b].reshape(-1, 3)
        d = np.linalg.norm(ca[:, None, :] - cb[None, :, :], axis=-1)
        assert (d.min(1) < 1e-12).sum() == n1       # one full edge of grid points in common
    # opposite faces share nothing
    d = np.linalg.norm(corners[0].reshape(-1, 3)[:, None] - corners[2].reshape(-1, 3)[None], axis=-1)
    assert d.min() > 1.0


def _dense_T(J):
    n = 1 << J
    return fwt(np.eye(n * n).reshape(n * n, n, n), 2, J)   # rows: cells, cols: wavelets -> T^T


def test_pattern_and_values_match_their_definitions():
    J, ell, nug = 3, 0.3, 1e-3
    b = sphere_basis(J)
    cp, ri = sphere_pattern(b)
    N = b.N
    # pattern: brute force over all pairs
    m, r = support_spheres(b)
    d = np.linalg.norm(m[:, None] - m[None], axis=-1) - r[:, None] - r[None]
    d = np.maximum(d, 0.0)
    jmin = np.minimum(b.level[:, None], b.level[None]).astype(np.float64)
    keep = np.tril(d <= 2.0 * 2.0 ** -jmin)
    Pd = np.zeros((N, N), bool)
    col = np.repeat(np.arange(N), np.diff(cp))
    Pd[ri, col] = True
    assert np.array_equal(Pd, keep)
    # support spheres contain their corner points (by construction) and every
    # support's panel midpoints
    pts, areas, _ = panel_grid(J)
    for v in range(0, N, 7):
        x0, y0 = b.box_lo[v]
        s = b.box_side[v]
        mid = pts[b.patch[v], y0:y0 + s, x0:x0 + s].reshape(-1, 3)
        assert np.linalg.norm(mid - m[v], axis=-1).max() <= r[v] + 1e-12
    # values: A = mask(T K_ss T^T) + nug I, K_ss = sqrt(|c||c'|) k(|x_c - x_c'|)
    n2 = (1 << J) ** 2
    X = pts.reshape(NPATCH * n2, 3)
    w = np.sqrt(areas.reshape(-1))
    K = np.exp(-np.linalg.norm(X[:, None] - X[None], axis=-1) / ell) * w[:, None] * w[None]
    Tt = _dense_T(J)
    T = np.zeros((N, N))
    for p in range(NPATCH):
        T[p * n2:(p + 1) * n2, p * n2:(p + 1) * n2] = Tt.T
    np.testing.assert_allclose(T @ T.T, np.eye(N), atol=1e-14)
    A = T @ K @ T.T + nug * np.eye(N)
    v = sphere_values(b, cp, ri, Kernel("exponential", ell), nug)
    np.testing.assert_allclose(v, A[ri, col], rtol=0, atol=1e-14 * np.abs(A).max())


@pytest.mark.parametrize("J", [2, 3, 4])
def test_patch_dissection_bitexact_and_separators(wdlib, J):
    b = sphere_basis(J)
    cp, ri = sphere_pattern(b)
    # leaf 64: the smallest sphere (96 vertices) is still dissected
    s = wdlib.Solver(symbolic_only=True, nd_leaf=64).analyze(cp, ri, b)
    got = s.symbolic()
    o = oracle.Oracle(cp, ri, b, leaf=64)
    assert np.array_equal(got["perm"], o.perm)
    assert np.array_equal(got["parent"], o.parent)
    assert np.array_equal(got["colcount"], o.colcount)
    assert np.array_equal(got["super_first"], o.super_first)
    assert np.array_equal(got["super_rows"], o.super_rows)
    perm, tree = oracle.nd_order(cp, ri, b, leaf=64, want_tree=True)
    assert np.array_equal(perm, o.perm)
    # the root node (recorded last) cuts patches {0, 1} from {2, 3, 4, 5}
    t0, t1, t2, t3 = tree[-1]
    assert t0 == 0 and t3 == b.N
    assert set(b.patch[perm[t0:t1]].tolist()) <= {0, 1}
    assert set(b.patch[perm[t1:t2]].tolist()) <= {2, 3, 4, 5}
    # separator property at every node: no edge between V1 and V2
    col = np.repeat(np.arange(b.N), np.diff(cp))
    pos = np.empty(b.N, np.int64)
    pos[perm] = np.arange(b.N)
    pi, pj = pos[ri], pos[col]
    for t0, t1, t2, _ in tree:
        in1 = lambda x: (x >= t0) & (x < t1)
        in2 = lambda x: (x >= t1) & (x < t2)
        assert not np.any((in1(pi) & in2(pj)) | (in2(pi) & in1(pj)))
