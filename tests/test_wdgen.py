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
