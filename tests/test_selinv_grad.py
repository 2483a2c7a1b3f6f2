"""Selected inverse and value gradients through the C ABI (needs a GB300).

Pins: the oracle's selected inverse (itself pinned to the dense inverse) and,
at sizes where it is cheap, the dense FP64 inverse and gradient; central
finite differences of the log-likelihood in a kernel hyperparameter.
Tolerances: FP64 throughout; entries of A^-1 within 1e-10 of max |A^-1|
(the supernodal recurrences and the oracle's scalar ones round differently,
both backward stable for these condition numbers, cond(A) <= 1e3);
gradients within 1e-9 relative in the max norm; finite differences with a
relative step of 1e-5 agree to 1e-6.
"""
import numpy as np
import pytest

import oracle
from wdgen import Kernel, compressed_pattern, compressed_values, haar_basis, rhs

pytestmark = pytest.mark.gpu

CASES = {
    "1d_J10": (1, 10, Kernel("exponential", 0.2), 1e-2),
    "2d_J5": (2, 5, Kernel("matern12", 0.15), 1e-2),
    "2d_J6": (2, 6, Kernel("matern32", 0.1), 1e-3),
}
_cache = {}


def _case(name):
    if name not in _cache:
        dim, J, ker, nug = CASES[name]
        b = haar_basis(dim, J)
        cp, ri = compressed_pattern(b)
        v = compressed_values(b, cp, ri, ker, nug)
        _cache[name] = (b, cp, ri, v)
    return _cache[name]


def _lower_entries(cp, ri):
    n = cp.size - 1
    col = np.repeat(np.arange(n), np.diff(cp))
    return ri.astype(np.int64), col


def _on_pattern(M, cp, ri):
    i, j = _lower_entries(cp, ri)
    return M[i, j]


def _weights(cp, ri):
    i, j = _lower_entries(cp, ri)
    return np.where(i == j, 1.0, 2.0)


@pytest.mark.parametrize("name", list(CASES))
def test_selinv_matches_oracle_and_dense(wdlib, cuda, name):
    b, cp, ri, v = _case(name)
    s = wdlib.Solver().analyze(cp, ri, b).factor(v, "fp64")
    z = s.selinv()
    n = cp.size - 1
    if n <= 4096:
        Ainv = np.linalg.inv(oracle.sym_lower_to_dense(cp, ri, v))
        ref = _on_pattern(Ainv, cp, ri)
    else:
        o = oracle.Oracle(cp, ri, b)
        assert o.factor(v) == 0
        Zl = o.selinv()
        pcp, prow, psrc = o.permuted_lower()
        ref = np.empty(ri.size)
        # (P A P^T)^-1 on L's pattern -> A's stored entries
        for jp in range(n):
            for e in range(pcp[jp], pcp[jp + 1]):
                ip = prow[e]
                lo, hi = min(ip, jp), max(ip, jp)
                a, c = o.Lp[lo], o.Lp[lo + 1]
                ref[psrc[e]] = Zl[a + np.searchsorted(o.Li[a:c], hi)]
    scale = np.abs(ref).max()
    assert np.abs(z - ref).max() <= 1e-10 * scale


def test_selinv_device_tensor_and_repeat(wdlib, cuda):
    import torch
    b, cp, ri, v = _case("2d_J5")
    s = wdlib.Solver().analyze(cp, ri, b).factor(torch.tensor(v, device="cuda"), "fp64")
    out = torch.empty(ri.size, dtype=torch.float64, device="cuda")
    s.selinv(out)
    first = out.cpu().numpy().copy()
    s.selinv(out)
    assert np.array_equal(first, out.cpu().numpy())
    assert np.array_equal(first, s.selinv())
    # refactor with scaled values: A^-1 scales inversely
    s.factor(2.0 * v, "fp64")
    np.testing.assert_allclose(s.selinv(), 0.5 * first, rtol=1e-12, atol=1e-14 * np.abs(first).max())


def test_selinv_needs_fp64_factor(wdlib, cuda):
    b, cp, ri, v = _case("1d_J10")
    s = wdlib.Solver().analyze(cp, ri, b)
    with pytest.raises(wdlib.WdError) as e:
        s.selinv()
    assert e.value.status == wdlib.WD_ERR_STATE
    s.factor(v, "mixed")
    with pytest.raises(wdlib.WdError) as e:
        s.selinv()
    assert e.value.status == wdlib.WD_ERR_STATE


@pytest.mark.parametrize("kind", ["diagonal", "tridiagonal", "dense150"])
def test_selinv_edge_structures(wdlib, cuda, kind):
    rng = np.random.default_rng(5)
    if kind == "diagonal":
        n = 300
        A = np.diag(rng.uniform(1, 2, n))
    elif kind == "tridiagonal":
        n = 257
        A = np.diag(np.full(n, 4.0)) + np.diag(np.full(n - 1, -1.0), 1) + np.diag(np.full(n - 1, -1.0), -1)
    else:
        n = 150
        G = rng.standard_normal((n, n))
        A = G @ G.T / n + np.eye(n)
    cols = [np.nonzero(np.tril(A)[:, j])[0] for j in range(n)]
    cp = np.concatenate([[0], np.cumsum([c.size for c in cols])]).astype(np.int64)
    ri = np.concatenate(cols).astype(np.int32)
    v = np.concatenate([A[c, j] for j, c in enumerate(cols)])
    s = wdlib.Solver().analyze(cp, ri).factor(v, "fp64")
    ref = _on_pattern(np.linalg.inv(A), cp, ri)
    assert np.abs(s.selinv() - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["1d_J10", "2d_J5"])
def test_value_gradient_matches_dense(wdlib, cuda, name):
    """l = <W, X> + c log det A with X = A^-1 B: dl/dA = c A^-1 - G X^T,
    G = A^-1 W; on the pattern with off-diagonals counted twice."""
    b, cp, ri, v = _case(name)
    n = cp.size - 1
    s = wdlib.Solver().analyze(cp, ri, b).factor(v, "fp64")
    B = rhs(n, 3, 7)
    W = rhs(n, 3, 8)
    c = 0.75
    X = s.solve(B)
    G = s.solve(W)
    g = s.value_gradient(c, X, G)
    A = oracle.sym_lower_to_dense(cp, ri, v)
    Ainv = np.linalg.inv(A)
    Xd, Gd = Ainv @ B, Ainv @ W
    D = c * Ainv - Gd @ Xd.T
    i, j = _lower_entries(cp, ri)
    ref = np.where(i == j, D[i, j], D[i, j] + D[j, i])
    assert np.abs(g - ref).max() <= 1e-9 * np.abs(ref).max()
    # pattern outer product alone
    o = s.sym_pattern_outer(G, X)
    P = Gd @ Xd.T
    ref_o = np.where(i == j, P[i, j], P[i, j] + P[j, i])
    assert np.abs(o - ref_o).max() <= 1e-9 * np.abs(ref_o).max()
    # logdet term alone: w * A^-1
    g0 = s.value_gradient(1.0, X[:, :0], G[:, :0])
    np.testing.assert_allclose(g0, _weights(cp, ri) * _on_pattern(Ainv, cp, ri), rtol=0,
                               atol=1e-10 * np.abs(Ainv).max())


def test_autograd_nll_values_and_rhs(wdlib, cuda):
    import torch
    from paper_2007_01541_gb300.autograd import SPDSystem, gp_negative_log_likelihood
    b, cp, ri, v = _case("2d_J5")
    n = cp.size - 1
    sysm = SPDSystem(cp, ri, b)
    vals = torch.tensor(v, device="cuda", requires_grad=True)
    Y = torch.tensor(rhs(n, 4, 0), device="cuda", requires_grad=True)
    loss = gp_negative_log_likelihood(sysm, vals, Y)
    loss.backward()
    A = oracle.sym_lower_to_dense(cp, ri, v)
    Ainv = np.linalg.inv(A)
    Yn = rhs(n, 4, 0)
    X = Ainv @ Yn
    ref_loss = 0.5 * (Yn * X).sum() + 0.5 * 4 * np.linalg.slogdet(A)[1]
    assert abs(loss.item() - ref_loss) <= 1e-11 * abs(ref_loss)
    D = 0.5 * 4 * Ainv - 0.5 * X @ X.T
    i, j = _lower_entries(cp, ri)
    ref = np.where(i == j, D[i, j], D[i, j] + D[j, i])
    gv = vals.grad.cpu().numpy()
    assert np.abs(gv - ref).max() <= 1e-9 * np.abs(ref).max()
    np.testing.assert_allclose(Y.grad.cpu().numpy(), X, rtol=0, atol=1e-11 * np.abs(X).max())


def test_autograd_hyperparameter_finite_differences(wdlib, cuda):
    """d nll / d ell through the value gradient and dA/d ell (the same
    compressed matrix with dk/d ell) against central differences."""
    import torch
    from paper_2007_01541_gb300.autograd import SPDSystem, gp_negative_log_likelihood
    b = haar_basis(2, 5)
    cp, ri = compressed_pattern(b)
    ker = Kernel("matern12", 0.15, 1.0)
    nug = 1e-2
    n = b.N
    Y = torch.tensor(rhs(n, 8, 0), device="cuda")
    sysm = SPDSystem(cp, ri, b)

    def nll(k):
        vals = torch.tensor(compressed_values(b, cp, ri, k, nug), device="cuda", requires_grad=True)
        loss = gp_negative_log_likelihood(sysm, vals, Y)
        loss.backward()
        return loss.item(), vals.grad.cpu().numpy()

    _, g = nll(ker)
    dA = compressed_values(b, cp, ri, ker.derivative("ell"), 0.0)
    d_ell = float(g @ dA)
    h = 1e-5 * ker.ell
    lp, _ = nll(Kernel("matern12", ker.ell + h, 1.0))
    lm, _ = nll(Kernel("matern12", ker.ell - h, 1.0))
    fd = (lp - lm) / (2 * h)
    assert abs(d_ell - fd) <= 1e-6 * max(1.0, abs(fd))
    # sigma^2 and nugget
    dS = compressed_values(b, cp, ri, ker.derivative("sigma2"), 0.0)
    d_s2 = float(g @ dS)
    lp, _ = nll(Kernel("matern12", ker.ell, 1.0 + 1e-5))
    lm, _ = nll(Kernel("matern12", ker.ell, 1.0 - 1e-5))
    assert abs(d_s2 - (lp - lm) / 2e-5) <= 1e-6 * max(1.0, abs(d_s2))
    i, j = _lower_entries(cp, ri)
    d_nug = float(g[i == j].sum())
    vals0 = compressed_values(b, cp, ri, ker, nug)
    eps = 1e-5 * nug

    def nll_nug(dn):
        vv = torch.tensor(vals0 + np.where(i == j, dn, 0.0), device="cuda")
        return gp_negative_log_likelihood(sysm, vv, Y).item()

    fd_n = (nll_nug(eps) - nll_nug(-eps)) / (2 * eps)
    assert abs(d_nug - fd_n) <= 1e-6 * max(1.0, abs(fd_n))


def test_autograd_configuration_full_size(wdlib, cuda):
    """The gradient configuration at full size (2D 128^2, N = 16,384, Matern-1/2
    l = 0.15, sigma^2 = 1, nugget 1e-2, 32 observation vectors): selected-
    inverse entries of sampled columns against solves with unit vectors
    (refined to backward error 1e-12 against A itself), the value gradient
    against central differences of the loss in a random direction, and the
    l-derivative against central differences in l."""
    import torch
    from paper_2007_01541_gb300.autograd import SPDSystem, gp_negative_log_likelihood
    from wdgen import workload_autograd
    w = workload_autograd(device="cuda")
    b, cp, ri = w.basis, w.colptr, w.rowidx
    n = b.N
    assert n == 16384 and w.B.shape[1] == 32
    sysm = SPDSystem(cp, ri, b)
    vals = torch.tensor(w.values, device="cuda", requires_grad=True)
    Y = torch.tensor(np.ascontiguousarray(w.B.T), device="cuda").T
    loss = gp_negative_log_likelihood(sysm, vals, Y)
    loss.backward()
    g = vals.grad.cpu().numpy()
    assert np.all(np.isfinite(g))
    # selected inverse at sampled columns: A^-1 e_j by the refined FP64 solve
    s = sysm.solver
    s.factor(w.values, "fp64")
    z = s.selinv()
    rng = np.random.default_rng(3)
    cols = rng.choice(n, 8, replace=False)
    E = np.zeros((n, cols.size))
    E[cols, np.arange(cols.size)] = 1.0
    Xe = s.solve(E)
    assert s.last_solve["backward_error"] <= 1e-12
    i, j = _lower_entries(cp, ri)
    scale = np.abs(z).max()
    for q, c in enumerate(cols):
        sel = np.nonzero(j == c)[0]                  # stored entries (i, c), i >= c
        assert np.abs(z[sel] - Xe[i[sel], q]).max() <= 1e-10 * scale
        sel = np.nonzero(i == c)[0]                  # stored entries (c, j), j < c
        assert np.abs(z[sel] - Xe[j[sel], q]).max() <= 1e-10 * scale
    # value gradient: directional central difference
    d = rng.standard_normal(ri.size) * np.abs(w.values)
    h = 1e-6

    def nll(v):
        return gp_negative_log_likelihood(sysm, torch.tensor(v, device="cuda"), Y).item()

    fd = (nll(w.values + h * d) - nll(w.values - h * d)) / (2 * h)
    assert abs(float(g @ d) - fd) <= 1e-6 * max(1.0, abs(fd))
    # hyperparameter l through dA/dl
    ker = w.kernel
    dA = compressed_values(b, cp, ri, ker.derivative("ell"), 0.0, "cuda")
    d_ell = float(g @ dA)
    he = 1e-5 * ker.ell
    vp = compressed_values(b, cp, ri, Kernel(ker.kind, ker.ell + he, ker.sigma2), w.nugget, "cuda")
    vm = compressed_values(b, cp, ri, Kernel(ker.kind, ker.ell - he, ker.sigma2), w.nugget, "cuda")
    fd_ell = (nll(vp) - nll(vm)) / (2 * he)
    assert abs(d_ell - fd_ell) <= 1e-6 * max(1.0, abs(fd_ell))
