"""Error paths of the library that can be driven without a GPU fault (needs a
GB300): a bounded device wait that expires (WD_ERR_TIMEOUT), device memory
that runs out (WD_ERR_OOM, injected on the host side of the allocator), and
refinement that stops short of the requested backward error
(WD_ERR_NO_CONVERGENCE).  After each, the handle and the CUDA context stay
usable.  Nothing here faults, traps or hangs the GPU: the timeout is a wait
for a device word that nothing sets, bounded by a short poll limit, after
which every CTA drains its own work, frees its tensor memory and returns.
"""
import numpy as np
import pytest

import oracle
from wdgen import Kernel, compressed_pattern, compressed_values, haar_basis, rhs

pytestmark = pytest.mark.gpu

_c = {}


def _small():
    if not _c:
        b = haar_basis(2, 6)
        cp, ri = compressed_pattern(b)
        v = compressed_values(b, cp, ri, Kernel("matern32", 0.1), 1e-3)
        _c.update(b=b, cp=cp, ri=ri, v=v)
    return _c


def test_timeout_of_a_bounded_wait(wdlib, cuda):
    c = _small()
    s = wdlib.Solver(wait_limit=2000, test_closed_gate=True).analyze(c["cp"], c["ri"], c["b"])
    with pytest.raises(wdlib.WdError) as e:
        s.factor(c["v"], "mixed")          # the tensor-core updates wait on the closed gate
    assert e.value.status == wdlib.WD_ERR_TIMEOUT
    # the handle stays usable: the FP64 factor has no tensor-core waits
    s.factor(c["v"], "fp64")
    B = rhs(c["b"].N, 3, seed=0)
    X = s.solve(B)
    assert oracle.backward_error(c["cp"], c["ri"], c["v"], X, B).max() <= 1e-12
    # and so does the context: a default handle factors in mixed precision
    s2 = wdlib.Solver().analyze(c["cp"], c["ri"], c["b"]).factor(c["v"], "mixed")
    X2 = s2.solve(B)
    assert oracle.backward_error(c["cp"], c["ri"], c["v"], X2, B).max() <= 1e-12


def test_out_of_memory_at_every_allocation(wdlib, cuda):
    """The k-th device allocation fails, for every k up to the number the
    analysis, both factorizations and a solve make: the call reports
    WD_ERR_OOM, and destroying the handle gives every byte back."""
    torch = cuda
    c = _small()
    B = rhs(c["b"].N, 4, seed=0)

    def run(s):
        s.analyze(c["cp"], c["ri"], c["b"])
        s.factor(c["v"], "mixed")
        s.solve(B)
        s.factor(c["v"], "fp64")
        s.solve(B)

    run(wdlib.Solver())                     # warm-up: modules, pools
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for k in range(1, 200):
        s = wdlib.Solver(test_fail_alloc=k)
        try:
            run(s)
        except wdlib.WdError as err:
            assert err.status == wdlib.WD_ERR_OOM, (k, str(err))
            failures += 1
        else:
            s.close()
            break
        s.close()
    else:
        pytest.fail("more than 199 device allocations")
    assert failures >= 10
    torch.cuda.synchronize()
    # nothing leaked: the free memory is back (the CUDA runtime's own pools
    # may move by less than a page)
    assert torch.cuda.mem_get_info()[0] >= free0 - (2 << 20)


def test_refinement_without_steps_does_not_converge(wdlib, cuda):
    c = _small()
    B = rhs(c["b"].N, 8, seed=1)
    s = wdlib.Solver(ir_max_iter=0).analyze(c["cp"], c["ri"], c["b"]).factor(c["v"], "mixed")
    with pytest.raises(wdlib.WdError) as e:
        s.solve(B)
    assert e.value.status == wdlib.WD_ERR_NO_CONVERGENCE
    assert "backward error" in str(e.value)
    # FP64 on the same handle reaches the target without refinement
    s.factor(c["v"], "fp64")
    X = s.solve(B)
    assert oracle.backward_error(c["cp"], c["ri"], c["v"], X, B).max() <= 1e-12
