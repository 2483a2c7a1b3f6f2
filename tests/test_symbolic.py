"""Host symbolic analysis of the library against the independent oracle
(bit-exact), input validation, and the exported C ABI (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from wdgen import compressed_pattern, haar_basis

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _compare(wd, cp, ri, basis, **opt):
    dflt = wd.DEFAULTS
    o = oracle.Oracle(cp, ri, basis, leaf=opt.get("nd_leaf", dflt["nd_leaf"]),
                      relax_k=opt.get("relax_k", dflt["relax_k"]), relax_pct=opt.get("relax_pct", dflt["relax_pct"]))
    s = wd.Solver(symbolic_only=True, **opt).analyze(cp, ri, basis)
    sy = s.symbolic()
    for key in ("perm", "parent", "colcount", "super_first", "super_rowptr", "super_rows"):
        np.testing.assert_array_equal(sy[key], getattr(o, key), err_msg=key)
    inf = s.info()
    assert inf["nnz_L"] == o.nnzL
    assert inf["flops_factor"] == float(np.sum(o.colcount.astype(np.float64) ** 2))
    return s, o


@pytest.mark.parametrize("dim,J", [(1, 10), (2, 4), (2, 5), (2, 6), (2, 7)])
def test_symbolic_bitexact(wdlib, dim, J):
    b = haar_basis(dim, J)
    cp, ri = compressed_pattern(b)
    _compare(wdlib, cp, ri, b)


@pytest.mark.parametrize("opt", [dict(nd_leaf=16), dict(relax_k=1, relax_pct=0),
                                 dict(relax_k=64, relax_pct=30), dict(nd_leaf=200)])
def test_symbolic_bitexact_options(wdlib, opt):
    b = haar_basis(2, 6)
    cp, ri = compressed_pattern(b)
    _compare(wdlib, cp, ri, b, **opt)


@pytest.mark.slow
def test_symbolic_bitexact_full_2d(wdlib):
    """The 2D 256 x 256 workload (N = 65,536), at full size."""
    b = haar_basis(2, 8)
    cp, ri = compressed_pattern(b)
    s, o = _compare(wdlib, cp, ri, b)
    assert s.info()["n"] == 65536


def test_symbolic_no_geometry(wdlib):
    rng = np.random.default_rng(3)
    n = 300
    M = np.tril((rng.random((n, n)) < 0.02), -1)
    cp = [0]
    ri = []
    for j in range(n):
        rows = [j] + [i for i in range(j + 1, n) if M[i, j]]
        ri += rows
        cp.append(len(ri))
    _compare(wdlib, np.array(cp), np.array(ri), None)


@pytest.mark.parametrize("bad", ["unsorted", "nodiag", "range", "dup"])
def test_malformed_pattern(wdlib, bad):
    cp = np.array([0, 3, 5, 6], np.int64)
    ri = {"unsorted": [0, 2, 1, 1, 2, 2], "nodiag": [1, 2, 0, 1, 2, 2],
          "range": [0, 1, 7, 1, 2, 2], "dup": [0, 1, 1, 1, 2, 2]}[bad]
    s = wdlib.Solver(symbolic_only=True)
    with pytest.raises(wdlib.WdError) as e:
        s.analyze(cp, np.array(ri, np.int32))
    assert e.value.status == wdlib.WD_ERR_PATTERN


def test_state_errors_host_only(wdlib):
    s = wdlib.Solver(symbolic_only=True)
    with pytest.raises(wdlib.WdError) as e:
        s.info()
    assert e.value.status == wdlib.WD_ERR_STATE
    b = haar_basis(1, 6)
    cp, ri = compressed_pattern(b)
    s.analyze(cp, ri, b)
    with pytest.raises(wdlib.WdError) as e:
        s.factor(np.ones(ri.size))
    assert e.value.status == wdlib.WD_ERR_STATE


def test_library_exports_every_declared_symbol(wdlib):
    hdr = open(os.path.join(ROOT, "include", "wd.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"\b(wd_[A-Za-z_0-9]+)\s*\(", hdr))
    assert len(names) >= 12
    lib = ctypes.CDLL(wdlib.library_path())
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(wdlib.EXPORTED) <= names


def test_batch_analysis_is_the_block_diagonal_union(wdlib):
    """wd_analyze_batch equals the instances' own analyses, shifted by the
    running column / row offsets (and instances passing the same arrays share
    one analysis)."""
    specs = [(1, 7), (2, 4), (1, 7), (2, 5), (1, 6)]
    cache = {}
    pats, bases = [], []
    for d, J in specs:
        if (d, J) not in cache:
            b = haar_basis(d, J)
            cache[(d, J)] = (b, compressed_pattern(b))
        b, p = cache[(d, J)]
        bases.append(b)
        pats.append(p)
    sb = wdlib.Solver(symbolic_only=True).analyze_batch(pats, bases)
    got = sb.symbolic()
    coff = roff = 0
    perm, parent, cc, sf, srp, rows = [], [], [], [], [0], []
    for (cp, ri), b in zip(pats, bases):
        one = wdlib.Solver(symbolic_only=True).analyze(cp, ri, b).symbolic()
        n = cp.size - 1
        perm.append(one["perm"] + coff)
        parent.append(np.where(one["parent"] < 0, -1, one["parent"] + coff))
        cc.append(one["colcount"])
        sf.append(one["super_first"][:-1] + coff)
        srp.extend((one["super_rowptr"][1:] + roff).tolist())
        rows.append(one["super_rows"] + coff)
        coff += n
        roff += int(one["super_rowptr"][-1])
    assert np.array_equal(got["perm"], np.concatenate(perm))
    assert np.array_equal(got["parent"], np.concatenate(parent))
    assert np.array_equal(got["colcount"], np.concatenate(cc))
    assert np.array_equal(got["super_first"], np.concatenate(sf + [[coff]]))
    assert np.array_equal(got["super_rowptr"], np.array(srp))
    assert np.array_equal(got["super_rows"], np.concatenate(rows))
    inf = sb.info()
    assert inf["n"] == coff and inf["nnz_A_lower"] == sum(p[1].size for p in pats)


def test_batch_analysis_rejects_bad_instance(wdlib):
    b = haar_basis(1, 5)
    cp, ri = compressed_pattern(b)
    bad = cp.copy()
    bad[-1] += 1
    s = wdlib.Solver(symbolic_only=True)
    with pytest.raises(wdlib.WdError) as e:
        s.analyze_batch([(cp, ri), (bad, ri)], [b, b])
    assert "instance 1" in str(e.value)


def test_symbolic_amalgamation_golden(wdlib):
    """The library's merge scan on the hand-worked amalgamation cases."""
    import json
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "amalgamation.json")))
    for case in g["cases"]:
        a = case["lower_csc"]
        cp = np.array(a["colptr"], np.int64)
        ri = np.array(a["rowidx"], np.int32)
        for run in case["runs"]:
            s = wdlib.Solver(symbolic_only=True, relax_k=run["relax_k"],
                             relax_pct=run["relax_pct"]).analyze(cp, ri)
            sy = s.symbolic()
            assert list(sy["parent"]) == case["parent"]
            assert list(sy["colcount"]) == case["colcount"]
            assert list(sy["super_first"]) == run["super_first"], (case["name"], run)


def test_invalid_options_are_rejected(wdlib):
    for kw in (dict(wait_limit=-1), dict(diag64_min_k=-1), dict(test_fail_alloc=-2), dict(nd_leaf=0)):
        with pytest.raises(wdlib.WdError) as e:
            wdlib.Solver(symbolic_only=True, **kw)
        assert e.value.status == wdlib.WD_ERR_INVALID_ARG


@pytest.mark.parametrize("dim,J", [(1, 10), (2, 5)])
def test_symbolic_bitexact_two_term_pattern(wdlib, dim, J):
    """The full two-term compression of Theorem 3.1 gives a sparser coarse
    coupling; the analysis stays bit-exact with the oracle on it."""
    from wdgen import compressed_pattern_two_term

    b = haar_basis(dim, J)
    cp, ri = compressed_pattern_two_term(b, a=1.5, delta=1.2, q=1.0)
    _compare(wdlib, cp, ri, b)
