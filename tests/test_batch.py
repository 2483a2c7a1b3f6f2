"""Batches of independent systems (wd_analyze_batch) through the C ABI
(needs a GB300).

Small batches: every instance against the oracle (solve, log det, factor
entries through the per-instance backward error).  The batched configuration
at full size (256 instances, N from 1024 to 16384, 1.85M unknowns): every
instance's normwise backward error <= 1e-12 (a property that holds at any
size) and the two smallest instances against the oracle.
"""
import numpy as np
import pytest

import oracle
from wdgen import batch_instances, batch_workload

pytestmark = pytest.mark.gpu


def _slices(sizes):
    off = np.concatenate([[0], np.cumsum(sizes)])
    return [slice(int(off[i]), int(off[i + 1])) for i in range(len(sizes))]


def _small_batch():
    params = [dict(dim=1, J=8, ell=0.3, N=256, nugget=1e-2), dict(dim=2, J=4, ell=0.2, N=256, nugget=1e-2),
              dict(dim=1, J=9, ell=0.07, N=512, nugget=1e-2), dict(dim=2, J=5, ell=0.45, N=1024, nugget=1e-2),
              dict(dim=1, J=8, ell=0.11, N=256, nugget=1e-2), dict(dim=2, J=4, ell=0.05, N=256, nugget=1e-2)]
    return batch_workload(params=params, nrhs=3, seed=4)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_small_batch_against_oracle(wdlib, cuda, prec):
    w = _small_batch()
    s = wdlib.Solver().analyze_batch(w.patterns, w.bases)
    s.factor(np.concatenate(w.values), prec)
    X = s.solve(w.B)
    assert s.last_solve["backward_error"] <= 1e-12
    ld = s.logdet_batch()
    for i, sl in enumerate(_slices([p["N"] for p in w.params])):
        cp, ri = w.patterns[i]
        o = oracle.Oracle(cp, ri, w.bases[i])
        assert o.factor(w.values[i]) == 0
        Xo = o.solve(w.B[sl])
        assert oracle.backward_error(cp, ri, w.values[i], X[sl], w.B[sl]).max() <= 1e-12
        np.testing.assert_allclose(X[sl], Xo, rtol=0, atol=1e-9 * np.abs(Xo).max())
        tol = 1e-12 if prec == "fp64" else 1e-5
        assert abs(ld[i] - o.logdet()) <= tol * abs(o.logdet())
    assert abs(s.logdet() - ld.sum()) <= 1e-10 * np.abs(ld).sum()


def test_batch_not_spd_names_the_instance(wdlib, cuda):
    w = _small_batch()
    vals = [v.copy() for v in w.values]
    cp, ri = w.patterns[3]
    vals[3][cp[:-1]] *= -1.0                       # negate instance 3's diagonal
    s = wdlib.Solver().analyze_batch(w.patterns, w.bases)
    with pytest.raises(wdlib.WdError) as e:
        s.factor(np.concatenate(vals), "fp64")
    assert e.value.status == wdlib.WD_ERR_NOT_SPD
    assert "instance 3" in str(e.value)


def test_batch_refactor_and_device_values(wdlib, cuda):
    torch = cuda
    w = _small_batch()
    s = wdlib.Solver().analyze_batch(w.patterns, w.bases)
    v = np.concatenate(w.values)
    s.factor(torch.tensor(v, device="cuda"), "mixed")
    X1 = s.solve(w.B)
    s.factor(torch.tensor(2.0 * v, device="cuda"), "mixed")
    X2 = s.solve(w.B)
    np.testing.assert_allclose(X2, 0.5 * X1, rtol=0, atol=1e-11 * np.abs(X1).max())


def test_batched_configuration_full_size(wdlib, cuda):
    """256 instances (the batched configuration), mixed precision with
    refinement, one right-hand side each."""
    torch = cuda
    params = batch_instances(256, 0)
    w = batch_workload(params=params, nrhs=1, seed=0, device="cuda")
    s = wdlib.Solver().analyze_batch(w.patterns, w.bases)
    vals = torch.tensor(np.concatenate(w.values), device="cuda")
    s.factor(vals, "mixed")
    Bt = torch.tensor(w.B, device="cuda")
    Xt = Bt.T.contiguous().T
    s.solve(Xt)
    assert s.last_solve["backward_error"] <= 1e-12
    X = Xt.cpu().numpy()
    ld = s.logdet_batch()
    assert np.all(np.isfinite(ld))
    sizes = [p["N"] for p in params]
    sl = _slices(sizes)
    # every instance's own backward error (oracle's FP64 residual)
    for i in range(len(params)):
        cp, ri = w.patterns[i]
        v = w.values[i]
        assert oracle.backward_error(cp, ri, v, X[sl[i]], w.B[sl[i]]).max() <= 1e-12, i
    # the two smallest instances against the oracle
    for i in np.argsort(sizes, kind="stable")[:2]:
        cp, ri = w.patterns[i]
        v = w.values[i]
        o = oracle.Oracle(cp, ri, w.bases[i])
        assert o.factor(v) == 0
        Xo = o.solve(w.B[sl[i]])
        np.testing.assert_allclose(X[sl[i]], Xo, rtol=0, atol=1e-9 * np.abs(Xo).max())
        assert abs(ld[i] - o.logdet()) <= 1e-5 * abs(o.logdet())
