"""Theta-scheme steps (Section 5, Eq. (theta), G = I).

CPU: the oracle's step is pinned by two facts of the scheme that do not
restate its formula: an eigenvector v of K (K v = lambda v) is only scaled,
by r = (1 - (1 - theta) dt lambda) / (1 + theta dt lambda) per step (source
0), and u* = K^-1 F is a fixed point of the step.  The library's step is
checked against argument errors without a GPU.

GPU: wd_theta_step (which forms the step from M alone: (1/theta) U -
((1 - theta)/theta) M U + dt F) against the oracle's step (which uses K)
over five steps, FP64 and mixed precision, few and many right-hand sides,
device and host arrays.
"""
import numpy as np
import pytest

import oracle
from wdgen import Kernel, compressed_pattern, compressed_values, haar_basis, rhs


def _k(dim, J, ker, nug):
    b = haar_basis(dim, J)
    cp, ri = compressed_pattern(b)
    return b, cp, ri, compressed_values(b, cp, ri, ker, nug)


@pytest.mark.parametrize("theta,dt", [(0.5, 0.3), (1.0, 2.0), (0.25, 0.05)])
def test_oracle_step_scales_an_eigenvector(theta, dt):
    b, cp, ri, k = _k(1, 6, Kernel("exponential", 0.2), 1e-2)
    K = oracle.sym_lower_to_dense(cp, ri, k)
    lam, V = np.linalg.eigh(K)
    o = oracle.Oracle(cp, ri, b)
    assert o.factor(oracle.theta_matrix(cp, k, theta, dt)) == 0
    for idx in (0, len(lam) // 2, len(lam) - 1):
        u = V[:, idx].copy()
        r = (1 - (1 - theta) * dt * lam[idx]) / (1 + theta * dt * lam[idx])
        for step in range(1, 4):
            u = oracle.theta_step(o, cp, ri, k, u[:, None], None, theta, dt)[:, 0]
            np.testing.assert_allclose(u, r ** step * V[:, idx], rtol=0, atol=1e-12)


def test_oracle_step_fixed_point():
    b, cp, ri, k = _k(2, 4, Kernel("matern32", 0.1), 1e-3)
    K = oracle.sym_lower_to_dense(cp, ri, k)
    F = rhs(K.shape[0], 3, seed=4)
    ustar = np.linalg.solve(K, F)
    for theta, dt in ((0.5, 0.1), (1.0, 1.0)):
        o = oracle.Oracle(cp, ri, b)
        assert o.factor(oracle.theta_matrix(cp, k, theta, dt)) == 0
        u1 = oracle.theta_step(o, cp, ri, k, ustar, F, theta, dt)
        assert np.abs(u1 - ustar).max() <= 1e-11 * np.abs(ustar).max()


def test_theta_step_argument_errors(wdlib):
    b, cp, ri, k = _k(1, 6, Kernel("exponential", 0.2), 1e-2)
    s = wdlib.Solver(symbolic_only=True).analyze(cp, ri, b)
    with pytest.raises(wdlib.WdError) as e:
        s.theta_step(np.zeros((cp.size - 1, 1)))
    assert e.value.status == wdlib.WD_ERR_STATE


_cases = {}


def _case(name):
    if name not in _cases:
        dim, J, ker, nug = {"1d_J10": (1, 10, Kernel("exponential", 0.2), 1e-2),
                            "2d_J6": (2, 6, Kernel("matern32", 0.1), 1e-3)}[name]
        _cases[name] = _k(dim, J, ker, nug)
    return _cases[name]


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["1d_J10", "2d_J6"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nrhs,theta", [(1, 0.5), (3, 1.0), (12, 0.5)])
def test_theta_steps_against_the_oracle(wdlib, cuda, name, prec, nrhs, theta):
    torch = cuda
    b, cp, ri, k = _case(name)
    dt = 0.05
    m = oracle.theta_matrix(cp, k, theta, dt)
    o = oracle.Oracle(cp, ri, b)
    assert o.factor(m) == 0
    n = cp.size - 1
    U0 = rhs(n, nrhs, seed=nrhs)
    F = rhs(n, nrhs, seed=100 + nrhs)
    s = wdlib.Solver().analyze(cp, ri, b).factor(m, prec)
    with pytest.raises(wdlib.WdError) as e:
        s.theta_step(U0, F, theta=0.0, dt=dt)
    assert e.value.status == wdlib.WD_ERR_INVALID_ARG
    Uo = U0.copy()
    Uh = U0.copy()
    Ud = torch.tensor(np.ascontiguousarray(U0.T), device="cuda").T       # column-major, ld n
    Fd = torch.tensor(np.ascontiguousarray(F.T), device="cuda").T
    for _ in range(5):
        Uo = oracle.theta_step(o, cp, ri, k, Uo, F, theta, dt)
        Uh = s.theta_step(Uh, F, theta=theta, dt=dt)
        assert s.last_solve["backward_error"] <= 1e-12
        s.theta_step(Ud, Fd, theta=theta, dt=dt)
    scale = np.abs(Uo).max()
    assert np.abs(Uh - Uo).max() <= 1e-10 * scale
    assert np.abs(Ud.cpu().numpy() - Uo).max() <= 1e-10 * scale


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_theta_step_without_source_and_with_zero_dt(wdlib, cuda, prec):
    """F = NULL follows the oracle's source-free step; dt = 0 makes M = I and
    leaves U unchanged."""
    b, cp, ri, k = _case("1d_J10")
    n = cp.size - 1
    U0 = rhs(n, 2, seed=7)
    theta, dt = 0.5, 0.1
    m = oracle.theta_matrix(cp, k, theta, dt)
    o = oracle.Oracle(cp, ri, b)
    assert o.factor(m) == 0
    s = wdlib.Solver().analyze(cp, ri, b).factor(m, prec)
    U = s.theta_step(U0, None, theta=theta, dt=dt)
    Uo = oracle.theta_step(o, cp, ri, k, U0, None, theta, dt)
    assert np.abs(U - Uo).max() <= 1e-10 * np.abs(Uo).max()
    s0 = wdlib.Solver().analyze(cp, ri, b).factor(oracle.theta_matrix(cp, k, theta, 0.0), prec)
    U1 = s0.theta_step(U0, rhs(n, 2, seed=8), theta=theta, dt=0.0)
    assert np.abs(U1 - U0).max() <= 1e-13 * np.abs(U0).max()


# ---- a non-orthonormal basis: mass matrix G != I --------------------------


@pytest.mark.parametrize("theta,dt", [(0.5, 0.3), (1.0, 2.0)])
def test_oracle_step_with_mass_scales_a_generalized_eigenvector(theta, dt):
    """K v = lambda G v (scipy's generalized symmetric eigensolver): the step
    with mass matrix G scales v by (1 - (1 - theta) dt lambda) / (1 + theta dt
    lambda), source 0."""
    import scipy.linalg as sla
    from wdgen import mass_matrix

    b, cp, ri, k = _k(1, 6, Kernel("exponential", 0.2), 1e-2)
    g = mass_matrix(b, cp, ri, 0.3)
    K = oracle.sym_lower_to_dense(cp, ri, k)
    G = oracle.sym_lower_to_dense(cp, ri, g)
    assert np.abs(G - np.eye(G.shape[0])).max() > 0.01          # G is not the identity
    lam, V = sla.eigh(K, G)
    o = oracle.Oracle(cp, ri, b)
    assert o.factor(oracle.theta_matrix(cp, k, theta, dt, g)) == 0
    for idx in (0, len(lam) // 2, len(lam) - 1):
        v = V[:, idx] / np.abs(V[:, idx]).max()
        r = (1 - (1 - theta) * dt * lam[idx]) / (1 + theta * dt * lam[idx])
        u = v.copy()
        for step in range(1, 4):
            u = oracle.theta_step(o, cp, ri, k, u[:, None], None, theta, dt, g)[:, 0]
            np.testing.assert_allclose(u, r ** step * v, rtol=0, atol=1e-11)


def test_oracle_step_with_mass_fixed_point_and_identity():
    """u* = K^-1 F is a fixed point for any G; G = I given explicitly is the
    orthonormal step."""
    from wdgen import mass_matrix

    b, cp, ri, k = _k(2, 4, Kernel("matern32", 0.1), 1e-3)
    g = mass_matrix(b, cp, ri, 0.25)
    K = oracle.sym_lower_to_dense(cp, ri, k)
    F = rhs(K.shape[0], 2, seed=5)
    ustar = np.linalg.solve(K, F)
    o = oracle.Oracle(cp, ri, b)
    assert o.factor(oracle.theta_matrix(cp, k, 0.5, 0.1, g)) == 0
    u1 = oracle.theta_step(o, cp, ri, k, ustar, F, 0.5, 0.1, g)
    assert np.abs(u1 - ustar).max() <= 1e-11 * np.abs(ustar).max()
    eye = np.zeros_like(k)
    eye[cp[:-1]] = 1.0
    o1 = oracle.Oracle(cp, ri, b)
    assert o1.factor(oracle.theta_matrix(cp, k, 0.5, 0.1, eye)) == 0
    U = rhs(K.shape[0], 2, seed=6)
    np.testing.assert_allclose(oracle.theta_step(o1, cp, ri, k, U, F, 0.5, 0.1, eye),
                               oracle.theta_step(o1, cp, ri, k, U, F, 0.5, 0.1), rtol=0, atol=1e-14)


def test_mass_matrix_is_spd_on_the_pattern():
    from wdgen import mass_matrix

    for dim, J in ((1, 7), (2, 4)):
        b = haar_basis(dim, J)
        cp, ri = compressed_pattern(b)
        g = mass_matrix(b, cp, ri, 0.3)
        G = oracle.sym_lower_to_dense(cp, ri, g)
        ev = np.linalg.eigvalsh(G)
        assert ev.min() >= 0.7 - 1e-12 and ev.max() <= 1.3 + 1e-12   # Gershgorin: row sums <= 0.3
        assert np.count_nonzero(g) > b.N                             # off-diagonal coupling exists


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["1d_J10", "2d_J6"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nrhs,theta", [(1, 0.5), (12, 1.0)])
def test_theta_steps_with_mass_against_the_oracle(wdlib, cuda, name, prec, nrhs, theta):
    """wd_set_mass + wd_theta_step (the library forms (1/theta) G U -
    ((1 - theta)/theta) M U + dt F) against the oracle's step from K and G,
    five steps; then G = I restored."""
    from wdgen import mass_matrix

    b, cp, ri, k = _case(name)
    g = mass_matrix(b, cp, ri, 0.3)
    dt = 0.05
    m = oracle.theta_matrix(cp, k, theta, dt, g)
    o = oracle.Oracle(cp, ri, b)
    assert o.factor(m) == 0
    n = cp.size - 1
    U0 = rhs(n, nrhs, seed=20 + nrhs)
    F = rhs(n, nrhs, seed=120 + nrhs)
    s = wdlib.Solver().analyze(cp, ri, b).set_mass(g).factor(m, prec)
    Uo, Uh = U0.copy(), U0.copy()
    for _ in range(5):
        Uo = oracle.theta_step(o, cp, ri, k, Uo, F, theta, dt, g)
        Uh = s.theta_step(Uh, F, theta=theta, dt=dt)
        assert s.last_solve["backward_error"] <= 1e-12
    assert np.abs(Uh - Uo).max() <= 1e-10 * np.abs(Uo).max()
    # G = I again: the step of M = I + theta dt K
    mi = oracle.theta_matrix(cp, k, theta, dt)
    oi = oracle.Oracle(cp, ri, b)
    assert oi.factor(mi) == 0
    s.set_mass(None).factor(mi, prec)
    Ui = s.theta_step(U0, F, theta=theta, dt=dt)
    Uoi = oracle.theta_step(oi, cp, ri, k, U0, F, theta, dt)
    assert np.abs(Ui - Uoi).max() <= 1e-10 * np.abs(Uoi).max()


@pytest.mark.parametrize("dim,J", [(1, 8), (2, 5)])
def test_mass_matrix_on_its_own_pattern_has_less_fill(wdlib, dim, J):
    """G analyzed on its own (sparser) pattern gets its own ordering, with far
    less fill than G ordered as the system matrix (Section 6); the oracle's
    factor of G on its own pattern reproduces G."""
    from wdgen import mass_matrix, own_pattern

    b = haar_basis(dim, J)
    cp, ri = compressed_pattern(b)
    g = mass_matrix(b, cp, ri, 0.3)
    gcp, gri, gv = own_pattern(cp, ri, g)
    assert gri.size < ri.size
    nnz_as_A = wdlib.Solver(symbolic_only=True).analyze(cp, ri, b).info()["nnz_L"]
    nnz_own = wdlib.Solver(symbolic_only=True).analyze(gcp, gri, b).info()["nnz_L"]
    assert nnz_own < nnz_as_A
    o = oracle.Oracle(gcp, gri, b)
    assert o.factor(gv) == 0
    G = oracle.sym_lower_to_dense(gcp, gri, gv)
    Ld = o.L_dense()
    PG = G[np.ix_(o.perm, o.perm)]
    assert np.abs(Ld @ Ld.T - PG).max() <= 1e-13


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_mass_matrix_inverse_on_its_own_ordering(wdlib, cuda, prec):
    """G^-1 applied by a handle analyzed on G's own pattern (its own ordering):
    backward error <= 1e-12 against G, and the same solution as the oracle's."""
    from wdgen import mass_matrix, own_pattern

    b = haar_basis(2, 6)
    cp, ri = compressed_pattern(b)
    gcp, gri, gv = own_pattern(cp, ri, mass_matrix(b, cp, ri, 0.3))
    s = wdlib.Solver().analyze(gcp, gri, b).factor(gv, prec)
    B = rhs(b.N, 4, seed=7)
    X = s.solve(B)
    assert oracle.backward_error(gcp, gri, gv, X, B).max() <= 1e-12
    o = oracle.Oracle(gcp, gri, b)
    assert o.factor(gv) == 0
    assert np.abs(X - o.solve(B)).max() <= 1e-10 * np.abs(X).max()
