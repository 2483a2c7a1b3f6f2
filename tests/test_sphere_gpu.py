"""Cubed sphere through the C ABI (needs a GB300).

The cubed-sphere configuration (6 x 128^2 panels, N = 98,304, exponential
kernel l = 0.3 on the chordal distance, nugget 1e-3) is not positive definite
under the compression reading used here (Lanczos: lambda_min of the masked
matrix without nugget is about -3.3e-3 at 6 x 32^2 and -3.8e-3 at 6 x 64^2):
the factorization must report WD_ERR_NOT_SPD, at the same first column as the
oracle.  The sampling path (s = P^T L z, 128 samples) runs on the same
structure with nugget 1e-2, where the matrix is positive definite.

Small spheres: against the oracle (solve, log det, apply_L).  Full size:
S^T A^-1 S = Z^T Z for S = P^T L Z (A^-1 S by the refined solve, whose FP64
residual uses A itself, so this checks L L^T = P A P^T), FP64 to 1e-9 and
mixed precision to 1e-3 relative, and the two precisions' samples agree to
1e-4.
"""
import numpy as np
import pytest

import oracle
from wdgen import Kernel, rhs
from wdgen.sphere import sphere_basis, sphere_pattern, sphere_values

pytestmark = pytest.mark.gpu
_cache = {}


def _sphere(J, nug, device="cpu"):
    key = (J, nug)
    if key not in _cache:
        b = sphere_basis(J)
        cp, ri = sphere_pattern(b, device)
        v = sphere_values(b, cp, ri, Kernel("exponential", 0.3), nug, device)
        _cache[key] = (b, cp, ri, v)
    return _cache[key]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_small_sphere_against_oracle(wdlib, cuda, prec):
    b, cp, ri, v = _sphere(4, 1e-2)
    o = oracle.Oracle(cp, ri, b)
    assert o.factor(v) == 0
    s = wdlib.Solver().analyze(cp, ri, b).factor(v, prec)
    B = rhs(b.N, 3, 1)
    X = s.solve(B)
    assert oracle.backward_error(cp, ri, v, X, B).max() <= 1e-12
    np.testing.assert_allclose(X, o.solve(B), rtol=0, atol=1e-9 * np.abs(X).max())
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert abs(s.logdet() - o.logdet()) <= tol * abs(o.logdet())
    Z = rhs(b.N, 4, 2)
    S = s.apply_L(Z)
    So = o.apply_L(Z)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.abs(S - So).max() <= tol * np.abs(So).max()


def test_small_sphere_not_spd_at_the_oracles_column(wdlib, cuda):
    b, cp, ri, v = _sphere(4, 1e-3)
    o = oracle.Oracle(cp, ri, b)
    rc = o.factor(v)
    assert rc < 0
    s = wdlib.Solver().analyze(cp, ri, b)
    with pytest.raises(wdlib.WdError) as e:
        s.factor(v, "fp64")
    assert e.value.status == wdlib.WD_ERR_NOT_SPD
    assert e.value.column == -rc - 1


def test_full_sphere_configuration_is_not_spd(wdlib, cuda):
    b, cp, ri, v = _sphere(7, 1e-3, "cuda")
    assert b.N == 98304
    s = wdlib.Solver().analyze(cp, ri, b)
    with pytest.raises(wdlib.WdError) as e:
        s.factor(v, "fp64")
    assert e.value.status == wdlib.WD_ERR_NOT_SPD


def test_full_sphere_sampling(wdlib, cuda):
    torch = cuda
    b, cp, ri, v = _sphere(7, 1e-2, "cuda")
    Z = rhs(b.N, 128, 0)
    Zt = torch.tensor(np.ascontiguousarray(Z.T), device="cuda").T
    out = {}
    for prec in ("fp64", "mixed"):
        s = wdlib.Solver().analyze(cp, ri, b).factor(torch.tensor(v, device="cuda"), prec)
        S = s.apply_L(Zt)
        X = S.clone()
        s.solve(X)
        assert s.last_solve["backward_error"] <= 1e-12
        G = (S.T @ X).cpu().numpy()
        ZZ = Z.T @ Z
        tol = 1e-9 if prec == "fp64" else 1e-3
        assert np.abs(G - ZZ).max() <= tol * np.abs(ZZ).max(), prec
        out[prec] = S.cpu().numpy()
    assert np.abs(out["mixed"] - out["fp64"]).max() <= 1e-4 * np.abs(out["fp64"]).max()
