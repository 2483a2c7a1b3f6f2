"""The synthetic input generator against its definitions (Sections 2 and 3)."""
import numpy as np
import pytest

from wdgen import Kernel, compressed_pattern, compressed_values, fwt, haar_basis, rhs


def _T(dim, J):
    N = (1 << J) ** dim
    I = np.eye(N).reshape((N,) + ((1 << J,) * dim))
    return fwt(I, dim, J).T          # T[lambda, c]


@pytest.mark.parametrize("dim,J", [(1, 6), (2, 3), (2, 4)])
def test_haar_orthonormal(dim, J):
    T = _T(dim, J)
    assert np.abs(T @ T.T - np.eye(T.shape[0])).max() < 1e-15


@pytest.mark.parametrize("dim,J", [(1, 5), (2, 3)])
def test_wavelet_supports_and_vanishing_mean(dim, J):
    b = haar_basis(dim, J)
    T = _T(dim, J)
    n = 1 << J
    for lam in range(b.N):
        w = T[lam].reshape((n,) * dim)
        nz = np.argwhere(np.abs(w) > 1e-14)
        lo = nz.min(0)[::-1] if dim == 2 else nz.min(0)
        hi = nz.max(0)[::-1] if dim == 2 else nz.max(0)
        np.testing.assert_array_equal(lo, b.box_lo[lam])
        np.testing.assert_array_equal(hi - lo + 1, [b.box_side[lam]] * dim)
        if b.level[lam] > 0:                    # one vanishing moment
            assert abs(w.sum()) < 1e-13


def _brute_pattern(b):
    N, J = b.N, b.J
    pairs = set()
    for i in range(N):
        for j in range(i + 1):
            thr = 2 * (1 << (J - min(b.level[i], b.level[j])))
            g2 = 0
            for a in range(b.dim):
                lo1, hi1 = b.box_lo[i, a], b.box_lo[i, a] + b.box_side[i]
                lo2, hi2 = b.box_lo[j, a], b.box_lo[j, a] + b.box_side[j]
                g = max(0, lo2 - hi1, lo1 - hi2)
                g2 += g * g
            if g2 <= thr * thr:
                pairs.add((i, j))
    return pairs


@pytest.mark.parametrize("dim,J", [(1, 6), (2, 3), (2, 4)])
def test_pattern_matches_cutoff_definition(dim, J):
    b = haar_basis(dim, J)
    cp, ri = compressed_pattern(b)
    cols = np.repeat(np.arange(b.N), np.diff(cp))
    got = set(zip(ri.tolist(), cols.tolist()))
    assert got == _brute_pattern(b)
    for j in range(b.N):
        assert ri[cp[j]] == j and np.all(np.diff(ri[cp[j]:cp[j + 1]]) > 0)


def _kss(b, ker):
    n = 1 << b.J
    c = (np.arange(n) + 0.5) / n
    if b.dim == 1:
        X = c[:, None]
    else:
        yy, xx = np.meshgrid(c, c, indexing="ij")
        X = np.stack([xx.ravel(), yy.ravel()], 1)
    r = np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    return ker(r) / b.N


@pytest.mark.parametrize("dim,J,ker", [(1, 6, Kernel("exponential", 0.2)),
                                       (2, 3, Kernel("matern32", 0.1)),
                                       (2, 4, Kernel("matern12", 0.15, 2.0))])
def test_values_are_masked_galerkin_matrix(dim, J, ker):
    b = haar_basis(dim, J)
    cp, ri = compressed_pattern(b)
    eps = 1e-3
    v = compressed_values(b, cp, ri, ker, eps, chunk=37)
    T = _T(dim, J)
    K = _kss(b, ker)
    A = T @ K @ T.T + eps * np.eye(b.N)
    cols = np.repeat(np.arange(b.N), np.diff(cp))
    np.testing.assert_allclose(v, A[ri, cols], rtol=0, atol=1e-14 * np.abs(A).max())


def test_unmasked_spectrum_is_kernel_spectrum_plus_nugget():
    b = haar_basis(2, 3)
    N = b.N
    cp = np.array([N * j - j * (j - 1) // 2 for j in range(N + 1)], np.int64)
    ri = np.concatenate([np.arange(j, N) for j in range(N)]).astype(np.int32)
    ker = Kernel("exponential", 0.3)
    v = compressed_values(b, cp, ri, ker, 1e-2)
    A = np.zeros((N, N))
    cols = np.repeat(np.arange(N), np.diff(cp))
    A[ri, cols] = v
    A[cols, ri] = v
    ev = np.linalg.eigvalsh(A)
    ek = np.linalg.eigvalsh(_kss(b, ker)) + 1e-2
    np.testing.assert_allclose(ev, ek, rtol=0, atol=1e-14)


def test_rhs_seeded():
    B = rhs(100, 4, seed=0)
    ref = np.random.default_rng(0).standard_normal((4, 100)).T
    np.testing.assert_array_equal(B, ref)
    assert B.flags.f_contiguous


def test_sizes_of_paper_like_configs():
    # 1D: 1 + sum_{j=1}^{10} 2^(j-1) = 1024; 2D 256^2: 1 + 3 sum_{j=1}^{8} 4^(j-1) = 65536
    assert haar_basis(1, 10).N == 1024
    assert haar_basis(2, 8).N == 65536
    b = haar_basis(1, 10)
    cp, ri = compressed_pattern(b)
    assert 2 * ri.size - b.N == 51892


@pytest.mark.parametrize("kind", ["exponential", "matern32"])
@pytest.mark.parametrize("param", ["ell", "sigma2"])
def test_kernel_parameter_derivatives(kind, param):
    """dk/d(param) against central differences of k (relative step 1e-6)."""
    r = np.linspace(0.0, 1.5, 301)
    k = Kernel(kind, 0.17, 1.3)
    d = k.derivative(param)(r)
    h = 1e-6 * getattr(k, param)
    kp = Kernel(kind, **{**dict(ell=0.17, sigma2=1.3), param: getattr(k, param) + h})
    km = Kernel(kind, **{**dict(ell=0.17, sigma2=1.3), param: getattr(k, param) - h})
    fd = (kp(r) - km(r)) / (2 * h)
    np.testing.assert_allclose(d, fd, rtol=1e-7, atol=1e-9)


# ---- the full a-priori compression of Theorem 3.1 (both terms) -------------


def _pattern_set(cp, ri):
    cols = np.repeat(np.arange(cp.size - 1), np.diff(cp))
    return set(zip(ri.tolist(), cols.tolist()))


def test_two_term_cutoff_golden():
    import json
    import os

    from wdgen import compressed_pattern_two_term, cutoff_parameters

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "two_term_cutoff.json")))
    p = g["parameters"]
    b = haar_basis(p["dim"], p["J"])
    cp, ri = compressed_pattern_two_term(b, a=p["a"], delta=p["delta"], q=p["q"], dtilde=p["dtilde"])
    S = _pattern_set(cp, ri)
    for e in g["entries"]:
        assert ((e["row"], e["col"]) in S) == e["kept"], e["why"]
    bs15 = cutoff_parameters(5, 1, 5, 1.5, 1.2, 1.0, 1.0)[1]
    assert abs(bs15 - 1.5 * 2 ** (-10.2 / 3)) < 1e-15
    assert cutoff_parameters(5, 5, 5, 1.5, 1.2, 1.0, 1.0) == (0.046875, 0.046875)


def test_two_term_cutoff_structure_and_growth():
    """Diagonal kept, rows sorted, larger a keeps a superset; the number of
    entries per unknown grows by less and less from level to level (the
    theorem's O(N) entries), while the first-term mask with a = 2 grows by a
    constant amount per level."""
    from wdgen import compressed_pattern_two_term

    prev = None
    inc1, inc2 = [], []
    for J in range(6, 12):
        b = haar_basis(1, J)
        cp, ri = compressed_pattern_two_term(b, a=1.5, delta=1.2, q=1.0)
        assert np.all(ri[cp[:-1]] == np.arange(b.N))
        for c in range(0, b.N, 97):
            assert np.all(np.diff(ri[cp[c]:cp[c + 1]]) > 0)
        c1, _ = compressed_pattern(b)
        anz = (2.0 * cp[-1] - b.N) / b.N, (2.0 * c1[-1] - b.N) / b.N
        if prev is not None:
            inc2.append(anz[0] - prev[0])
            inc1.append(anz[1] - prev[1])
        prev = anz
    assert all(x > y for x, y in zip(inc2, inc2[1:]))          # shrinking increments
    assert inc2[-1] < 0.3 * inc1[-1]
    b = haar_basis(2, 4)
    small = _pattern_set(*compressed_pattern_two_term(b, a=1.5, delta=1.2, q=1.0))
    big = _pattern_set(*compressed_pattern_two_term(b, a=3.0, delta=1.2, q=1.0))
    assert small < big


def test_two_term_cutoff_needs_the_theorems_parameters():
    from wdgen import compressed_pattern_two_term

    b = haar_basis(1, 4)
    for kw in (dict(a=1.0, delta=1.2, q=1.0), dict(a=2.0, delta=0.9, q=1.0), dict(a=2.0, delta=1.5, q=0.2)):
        with pytest.raises(ValueError):
            compressed_pattern_two_term(b, **kw)
