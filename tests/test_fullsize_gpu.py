"""The 2D 256^2 configuration at full size (N = 65,536, Matern-3/2 l = 0.1,
nugget 1e-3, 64 right-hand sides), in the launch configuration the benchmark
times: values and right-hand sides on the device, CUDA-graph replay, mixed
precision with refinement (FP64 beside it).  Needs a GB300.

The oracle factors the whole matrix once per session (1.0e11 flops, about a
minute or two on one host core), and parity is taken on every column of L,
the top separator fronts included (the largest Schur updates and the deepest
super-block inverses run there), on log det, and on the normwise backward
error of every solution column from the oracle's own FP64 residual.
"""
import numpy as np
import pytest

import oracle
from wdgen import Kernel, compressed_pattern, compressed_values, haar_basis, rhs

pytestmark = pytest.mark.gpu
_c = {}


def _full():
    if not _c:
        b = haar_basis(2, 8)
        cp, ri = compressed_pattern(b)
        v = compressed_values(b, cp, ri, Kernel("matern32", 0.1), 1e-3, device="cuda")
        o = oracle.Oracle(cp, ri, b)
        assert o.factor(v) == 0
        _c.update(b=b, cp=cp, ri=ri, v=v, o=o, Lo=o.L_values())
    return _c


def _solver(wdlib, torch, c, prec):
    # "fp64_tc": the FP64 factorization with its Schur updates on the tensor
    # cores (bf16 slices), held to the FP64 bar
    opts = {"fp64_tc_schur": True} if prec == "fp64_tc" else {}
    p = "fp64" if prec == "fp64_tc" else prec
    return wdlib.Solver(**opts).analyze(c["cp"], c["ri"], c["b"]).factor(torch.tensor(c["v"], device="cuda"), p)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp64_tc", 1e-10), ("mixed", 2e-5)])
def test_fullsize_factor_every_column(wdlib, cuda, prec, tol):
    """||L_gpu[:, j] - L_oracle[:, j]||_2 <= tol ||L_oracle[:, j]||_2 for all
    65,536 columns; the last supernode (the root separator) is also checked on
    its own, so that a failure there cannot hide behind the column count."""
    c = _full()
    o = c["o"]
    s = _solver(wdlib, cuda, c, prec)
    L = s.L_csc_like(o.Lp, o.Li)
    starts = o.Lp[:-1]
    d2 = np.add.reduceat((L - c["Lo"]) ** 2, starts)
    n2 = np.add.reduceat(c["Lo"] ** 2, starts)
    rel = np.sqrt(d2 / n2)
    assert rel.size == o.n
    assert float(rel.max()) <= tol, (prec, float(rel.max()), int(rel.argmax()))
    root = int(o.super_first[-2])
    assert o.n - root > 1000          # the root separator is a wide dense front
    assert float(rel[root:].max()) <= tol


def test_fullsize_mixed_solve_64_rhs(wdlib, cuda):
    torch = cuda
    c = _full()
    s = _solver(wdlib, torch, c, "mixed")
    n = c["o"].n
    B = rhs(n, 64, seed=0)
    Bt = torch.tensor(np.ascontiguousarray(B.T), device="cuda")   # (64, n): Bt.T is column-major
    s.solve(Bt.T)
    X = Bt.T.cpu().numpy()
    be = oracle.backward_error(c["cp"], c["ri"], c["v"], X, B)
    assert be.max() <= 1e-12, be.max()
    assert s.last_solve["iterations"] >= 1
    # the library's own (double-float) residual agrees with the oracle's FP64 one
    assert abs(s.last_solve["backward_error"] - be.max()) <= 5e-15, (s.last_solve, be.max())


def test_fullsize_logdet(wdlib, cuda):
    """FP64: log det agrees with the oracle's 2 sum log L_jj; mixed: with FP64
    to the FP32 factor's accuracy (scale: sum |2 log L_jj|)."""
    c = _full()
    o = c["o"]
    s64 = _solver(wdlib, cuda, c, "fp64")
    L = s64.L_csc_like(o.Lp, o.Li)
    ld64 = s64.logdet()
    assert abs(ld64 - o.logdet()) <= 1e-12 * np.abs(2.0 * np.log(c["Lo"][o.Lp[:-1]])).sum()
    scale = np.abs(2.0 * np.log(L[o.Lp[:-1]])).sum()     # sum |2 log L_jj| over all columns
    assert abs(ld64 - 2.0 * np.log(L[o.Lp[:-1]]).sum()) <= 1e-12 * scale
    ldm = _solver(wdlib, cuda, c, "mixed").logdet()
    assert abs(ldm - ld64) <= 1e-6 * scale, (ldm, ld64, scale)
