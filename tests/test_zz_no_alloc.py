"""wd_export_L_noalloc (static device scratch, no allocation) against
wd_export_L on the same factor; two calls in a row, the output poisoned in
between.  Named to be collected last; it also passes run alone."""
import numpy as np
import pytest

from wdgen import Kernel, compressed_pattern, compressed_values, haar_basis

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_export_matches_export(wdlib, cuda, prec):
    torch = cuda
    b = haar_basis(2, 6)
    cp, ri = compressed_pattern(b)
    v = compressed_values(b, cp, ri, Kernel("matern32", 0.1), 1e-3)
    s = wdlib.Solver().analyze(cp, ri, b).factor(v, prec)
    ref = s.export_L()
    out = torch.empty(ref.size, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    for _ in range(2):
        out.fill_(float("nan"))
        torch.cuda.current_stream().synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        with torch.cuda.stream(stream):
            s.export_L_noalloc(out, stream=stream.cuda_stream)
        stream.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0      # no device memory was taken
        assert np.array_equal(out.cpu().numpy(), ref)


def test_noalloc_export_is_ordered_before_the_next_factor(wdlib, cuda):
    """The export returns without waiting; a refactorization with other
    values issued right after it on another stream must not overwrite the
    fronts before the export has read them."""
    torch = cuda
    b = haar_basis(2, 7)
    cp, ri = compressed_pattern(b)
    v1 = compressed_values(b, cp, ri, Kernel("matern32", 0.1), 1e-3)
    v2 = compressed_values(b, cp, ri, Kernel("matern32", 0.2), 1e-2)
    s = wdlib.Solver().analyze(cp, ri, b)
    ref1 = s.factor(v1, "fp64").export_L()
    ref2 = s.factor(v2, "fp64").export_L()
    assert not np.array_equal(ref1, ref2)
    s.factor(v1, "fp64")
    out = torch.full((ref1.size,), float("nan"), dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    s.export_L_noalloc(out, stream=side.cuda_stream)
    s.factor(v2, "fp64")                       # default stream, no synchronization in between
    side.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref1)
    assert np.array_equal(s.export_L(), ref2)


def test_noalloc_export_rejects_too_many_supernodes(wdlib, cuda):
    torch = cuda
    n = 70000                                   # a diagonal matrix: n singleton supernodes
    cp = np.arange(n + 1, dtype=np.int64)
    ri = np.arange(n, dtype=np.int32)
    s = wdlib.Solver().analyze(cp, ri).factor(np.full(n, 2.0), "fp64")
    assert s.info()["nsuper"] > 65536
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(wdlib.WdError) as e:
        s.export_L_noalloc(out)
    assert e.value.status == wdlib.WD_ERR_INVALID_ARG
    assert "static scratch" in str(e.value)
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0        # nothing was enqueued


def test_noalloc_export_needs_factor(wdlib, cuda):
    torch = cuda
    b = haar_basis(1, 6)
    cp, ri = compressed_pattern(b)
    s = wdlib.Solver().analyze(cp, ri, b)
    with pytest.raises(wdlib.WdError) as e:
        s.export_L_noalloc(torch.empty(s._panel_size(), dtype=torch.float64, device="cuda"))
    assert e.value.status == wdlib.WD_ERR_STATE


def test_noalloc_export_can_be_captured_in_a_cuda_graph(wdlib, cuda):
    """Stream capture rejects cudaMalloc, cudaFree and synchronizing calls: a
    capture of the export that succeeds and replays to the same panels shows
    the call makes none of them."""
    torch = cuda
    b = haar_basis(2, 6)
    cp, ri = compressed_pattern(b)
    v = compressed_values(b, cp, ri, Kernel("matern32", 0.1), 1e-3)
    s = wdlib.Solver().analyze(cp, ri, b).factor(v, "fp64")
    ref = s.export_L()
    out = torch.empty(ref.size, dtype=torch.float64, device="cuda")
    s.export_L_noalloc(out, stream=torch.cuda.current_stream().cuda_stream)   # warm-up: module, address
    torch.cuda.synchronize()
    out.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        s.export_L_noalloc(out, stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    g.replay()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.array_equal(out.cpu().numpy(), ref)
