"""CUDA path against the CPU oracle, through the C ABI (needs a GB300).

Tolerances, derived from the arithmetic: FP64 factor entries differ from the
oracle's only by summation order (a few thousand terms per entry, cond(A) up to
~1e3), and the refinement target is a backward error of 1e-12:
  * FP64 factor: per column ||L_gpu(:,j) - L_or(:,j)||_2 <= 1e-10 ||L_or(:,j)||_2;
    amalgamation zeros stay exactly 0.
  * solves: normwise backward error <= 1e-12 per right-hand side, residual in
    FP64 by the oracle's own sparse product.
  * logdet: FP64 within 1e-12 relative; apply_L within 1e-12 relative.
"""
import math

import numpy as np
import pytest

import oracle
from wdgen import Kernel, compressed_pattern, compressed_values, haar_basis, rhs

pytestmark = pytest.mark.gpu

CASES = {
    "1d_J10": (1, 10, Kernel("exponential", 0.2), 1e-2),
    "2d_J5": (2, 5, Kernel("matern32", 0.1), 1e-3),
    "2d_J6": (2, 6, Kernel("matern32", 0.1), 1e-3),
    "2d_J7_exp": (2, 7, Kernel("exponential", 0.3), 1e-2),
}
_cache = {}


def _case(name):
    if name not in _cache:
        dim, J, ker, nug = CASES[name]
        b = haar_basis(dim, J)
        cp, ri = compressed_pattern(b)
        v = compressed_values(b, cp, ri, ker, nug)
        o = oracle.Oracle(cp, ri, b)
        assert o.factor(v) == 0
        _cache[name] = (b, cp, ri, v, o)
    return _cache[name]


def _panel_mask_check(s, o):
    """Stored entries outside L's structure (amalgamation zeros) are 0."""
    sym = s.symbolic()
    panels = s.export_L()
    sf, srp, rows = sym["super_first"], sym["super_rowptr"], sym["super_rows"]
    k = np.diff(sf).astype(np.int64)
    m = np.diff(srp).astype(np.int64)
    poff = np.concatenate([[0], np.cumsum(k * m)])
    bad = 0.0
    for sn in range(k.size):
        r = rows[srp[sn]: srp[sn + 1]]
        for c in range(k[sn]):
            j = sf[sn] + c
            struct = set(o.Li[o.Lp[j]: o.Lp[j + 1]].tolist())
            col = panels[poff[sn] + c * m[sn]: poff[sn] + (c + 1) * m[sn]]
            zero = np.array([ri not in struct for ri in r])
            if zero.any():
                bad = max(bad, float(np.abs(col[zero]).max()))
    return bad


@pytest.mark.parametrize("name", list(CASES))
def test_factor_fp64_entries(wdlib, cuda, name):
    b, cp, ri, v, o = _case(name)
    s = wdlib.Solver().analyze(cp, ri, b)
    s.factor(v, "fp64")
    L = s.L_csc_like(o.Lp, o.Li)
    Lo = o.L_values()
    for j in range(o.n):
        a, e = o.Lp[j], o.Lp[j + 1]
        assert np.linalg.norm(L[a:e] - Lo[a:e]) <= 1e-10 * np.linalg.norm(Lo[a:e]), j
    if name in ("1d_J10", "2d_J5"):
        assert _panel_mask_check(s, o) == 0.0


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("nrhs", [1, 2, 5, 33])
def test_solve_fp64(wdlib, cuda, name, nrhs):
    b, cp, ri, v, o = _case(name)
    s = wdlib.Solver().analyze(cp, ri, b).factor(v, "fp64")
    B = rhs(o.n, nrhs, seed=nrhs)
    X = s.solve(B)
    be = oracle.backward_error(cp, ri, v, X, B)
    assert be.max() <= 1e-12
    Xo = o.solve(B)
    assert np.abs(X - Xo).max() <= 1e-8 * np.abs(Xo).max()
    assert 0 <= s.last_solve["backward_error"] <= 1e-12


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("nrhs", [2, 7])
def test_solve_mixed_refined(wdlib, cuda, name, nrhs):
    b, cp, ri, v, o = _case(name)
    s = wdlib.Solver().analyze(cp, ri, b).factor(v, "mixed")
    B = rhs(o.n, nrhs, seed=11)
    X = s.solve(B)
    be = oracle.backward_error(cp, ri, v, X, B)
    assert be.max() <= 1e-12
    assert s.last_solve["iterations"] >= 1
    assert s.last_solve["backward_error"] <= 1e-12


def test_solve_device_tensor_in_place(wdlib, cuda):
    torch = cuda
    b, cp, ri, v, o = _case("2d_J6")
    s = wdlib.Solver().analyze(cp, ri, b)
    s.factor(torch.from_numpy(v).cuda(), "fp64")
    B = rhs(o.n, 4, seed=5)
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda().T   # column-major view
    s.solve(Bt)
    torch.cuda.synchronize()
    X = Bt.cpu().numpy()
    assert oracle.backward_error(cp, ri, v, X, B).max() <= 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_logdet(wdlib, cuda, name):
    b, cp, ri, v, o = _case(name)
    s = wdlib.Solver().analyze(cp, ri, b).factor(v, "fp64")
    ref = o.logdet()
    assert abs(s.logdet() - ref) <= 1e-12 * abs(ref)
    s.factor(v, "mixed")
    assert abs(s.logdet() - ref) <= 1e-5 * abs(ref)


@pytest.mark.parametrize("name", ["1d_J10", "2d_J6"])
def test_apply_L(wdlib, cuda, name):
    b, cp, ri, v, o = _case(name)
    s = wdlib.Solver().analyze(cp, ri, b).factor(v, "fp64")
    Z = rhs(o.n, 9, seed=2)
    S = s.apply_L(Z)
    So = o.apply_L(Z)
    assert np.abs(S - So).max() <= 1e-12 * np.abs(So).max()
    s.factor(v, "mixed")
    S32 = s.apply_L(Z)
    assert np.abs(S32 - So).max() <= 1e-5 * np.abs(So).max()


def _dense_lower(A):
    n = A.shape[0]
    cp, ri, vv = [0], [], []
    for j in range(n):
        rows = [i for i in range(j, n) if i == j or A[i, j] != 0.0]
        ri += rows
        vv += [A[i, j] for i in rows]
        cp.append(len(ri))
    return np.array(cp, np.int64), np.array(ri, np.int32), np.array(vv)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_not_spd_first_column(wdlib, cuda, prec):
    n = 300
    A = 4 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    A[120, 120] = -2.0
    A[250, 250] = -2.0
    cp, ri, v = _dense_lower(A)
    o = oracle.Oracle(cp, ri)
    col = -o.factor(v) - 1
    s = wdlib.Solver().analyze(cp, ri)
    with pytest.raises(wdlib.WdError) as e:
        s.factor(v, prec)
    assert e.value.status == wdlib.WD_ERR_NOT_SPD
    assert e.value.column == col == 120
    with pytest.raises(wdlib.WdError) as e2:
        s.solve(np.ones(n))
    assert e2.value.status == wdlib.WD_ERR_STATE


@pytest.mark.parametrize("kind", ["n1", "diagonal", "tridiagonal", "dense200", "random"])
def test_edge_structures(wdlib, cuda, kind):
    rng = np.random.default_rng(7)
    if kind == "n1":
        A = np.array([[3.0]])
    elif kind == "diagonal":
        A = np.diag(rng.random(77) + 0.5)
    elif kind == "tridiagonal":
        n = 1000
        A = 4 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    elif kind == "dense200":
        M = rng.standard_normal((200, 200))
        A = M @ M.T + 200 * np.eye(200)
    else:
        n = 700
        M = (rng.random((n, n)) < 0.01) * rng.standard_normal((n, n))
        A = np.tril(M, -1)
        A = A + A.T
        A += np.diag(np.abs(A).sum(1) + 1)
    cp, ri, v = _dense_lower(A)
    o = oracle.Oracle(cp, ri)
    assert o.factor(v) == 0
    s = wdlib.Solver().analyze(cp, ri).factor(v, "fp64")
    L = s.L_csc_like(o.Lp, o.Li)
    np.testing.assert_allclose(L, o.L_values(), rtol=0, atol=1e-12 * np.abs(o.L_values()).max())
    B = rhs(A.shape[0], 3)
    X = s.solve(B)
    assert oracle.backward_error(cp, ri, v, X, B).max() <= 1e-12
    assert abs(s.logdet() - o.logdet()) <= 1e-12 * max(1.0, abs(o.logdet()))


def test_refactor_same_pattern_and_zero_rhs(wdlib, cuda):
    b, cp, ri, v, o = _case("1d_J10")
    s = wdlib.Solver().analyze(cp, ri, b)
    for scale in (1.0, 2.0):
        s.factor(v * scale, "fp64")
        assert abs(s.logdet() - (o.logdet() + o.n * math.log(scale))) <= 1e-11 * abs(o.logdet())
    assert s.solve(np.zeros((o.n, 0))).shape == (o.n, 0)


@pytest.mark.parametrize("graphs", [True, False])
def test_profiled_and_direct_launches(wdlib, cuda, graphs):
    b, cp, ri, v, o = _case("2d_J6")
    s = wdlib.Solver(profile=True, use_graphs=graphs).analyze(cp, ri, b)
    B = rhs(o.n, 3, seed=4)
    for prec in ("fp64", "mixed"):
        s.factor(v, prec)
        X = s.solve(B)
        assert oracle.backward_error(cp, ri, v, X, B).max() <= 1e-12
    st = s.kernel_stats(reset=True)
    names = {k["name"] for k in st}
    assert {"schur_update_fp64", "tc_schur_syrk_fp32", "fwd_xapply_fp32", "bwd_reduce_fp64",
            "sbinv_stage_fp32", "fwd_bupdate_fp64"} <= names
    assert all(k["launches"] > 0 and k["ms"] > 0 for k in st)
    assert s.kernel_stats() == []
    assert s.launch_count() > 0


@pytest.mark.parametrize("step_launches", [False, True])
@pytest.mark.parametrize("name", ["1d_J10", "2d_J6", "2d_J7_exp"])
def test_factor_mixed_entries(wdlib, cuda, name, step_launches):
    """FP32 fronts with tensor-core (3xTF32) Schur updates: every column of L
    within 2e-5 of the FP64 oracle (relative 2-norm), amalgamation zeros
    exactly 0 in the 1D case.  Both schedules of the pivot columns: one
    launch per level of dependency-ordered tasks (the default), and a
    (panel, update) launch pair per 64-column pivot block."""
    b, cp, ri, v, o = _case(name)
    s = wdlib.Solver(step_launches=step_launches).analyze(cp, ri, b)
    s.factor(v, "mixed")
    L = s.L_csc_like(o.Lp, o.Li)
    Lo = o.L_values()
    worst = 0.0
    for j in range(o.n):
        a, e = o.Lp[j], o.Lp[j + 1]
        worst = max(worst, np.linalg.norm(L[a:e] - Lo[a:e]) / np.linalg.norm(Lo[a:e]))
    assert worst <= 2e-5, worst
    if name == "1d_J10":
        assert _panel_mask_check(s, o) == 0.0


@pytest.mark.parametrize("nrhs", [3, 40])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_backward_error_call_matches_fp64_residual(wdlib, cuda, nrhs, prec):
    """wd_backward_error (FP64 residual up to 8 columns, double-float beyond)
    against the oracle's FP64 residual, on solutions perturbed so that the
    residual is well above rounding, and on exact solves (tiny residual)."""
    b, cp, ri, v, o = _case("2d_J6")
    s = wdlib.Solver().analyze(cp, ri, b).factor(v, prec)
    B = rhs(o.n, nrhs, seed=9)
    X = s.solve(B)
    be0 = s.backward_error(X, B)
    assert be0 <= 1e-12
    assert abs(be0 - oracle.backward_error(cp, ri, v, X, B).max()) <= 2e-15
    rng = np.random.default_rng(2)
    for scale in (1e-13, 1e-9, 1e-5):
        Xp = X + scale * np.abs(X).max() * rng.standard_normal(X.shape)
        ref = oracle.backward_error(cp, ri, v, Xp, B).max()
        got = s.backward_error(Xp, B)
        assert abs(got - ref) <= 1e-6 * ref + 2e-15, (scale, got, ref)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nrhs", [3, 40])
def test_solve_device_padded_leading_dimension(wdlib, cuda, prec, nrhs):
    """A column-major device B with leading dimension n + 5: the solution lands
    in the first n rows of every column and the padding is left untouched."""
    torch = cuda
    b, cp, ri, v, o = _case("2d_J6")
    s = wdlib.Solver().analyze(cp, ri, b).factor(v, prec)
    B = rhs(o.n, nrhs, seed=21)
    store = torch.full((nrhs, o.n + 5), 7.0, dtype=torch.float64, device="cuda")
    store[:, : o.n] = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    view = store[:, : o.n].T                      # n x nrhs, stride (1, n + 5)
    assert view.stride() == (1, o.n + 5)
    s.solve(view)
    X = view.cpu().numpy()
    assert oracle.backward_error(cp, ri, v, X, B).max() <= 1e-12
    assert torch.all(store[:, o.n:] == 7.0)


def test_mixed_with_fp64_diagonal_blocks(wdlib, cuda):
    """WD_MIXED with every diagonal block factored in FP64 (diag64_min_k = 1):
    the factor agrees with the oracle at the mixed tolerance, the refined
    solve reaches the target, and refinement needs no more steps than with
    FP32 diagonal blocks."""
    b, cp, ri, v, o = _case("2d_J6")
    B = rhs(o.n, 33, seed=2)
    its = {}
    for d64 in (0, 1):
        s = wdlib.Solver(diag64_min_k=d64).analyze(cp, ri, b)
        s.factor(v, "mixed")
        L = s.L_csc_like(o.Lp, o.Li)
        Lo = o.L_values()
        starts = o.Lp[:-1]
        rel = np.sqrt(np.add.reduceat((L - Lo) ** 2, starts) / np.add.reduceat(Lo ** 2, starts))
        assert rel.max() <= 2e-5, (d64, rel.max())
        X = s.solve(B)
        assert oracle.backward_error(cp, ri, v, X, B).max() <= 1e-12
        its[d64] = s.last_solve["iterations"]
    assert its[1] <= its[0], its


def test_fp64_diagonal_block_of_a_leaf_front(wdlib, cuda):
    """A front without children assembles F11 = fl32(A11) exactly; with FP64
    diagonal blocks its stored L11 is the FP64 Cholesky factor of that block
    rounded to FP32 (within one FP32 ulp: the two FP64 factorizations differ
    only in summation order)."""
    b, cp, ri, v, o = _case("2d_J6")
    s = wdlib.Solver(diag64_min_k=1).analyze(cp, ri, b).factor(v, "mixed")
    sym = s.symbolic()
    sf, srp = sym["super_first"], sym["super_rowptr"]
    k = np.diff(sf).astype(np.int64)
    m = np.diff(srp).astype(np.int64)
    poff = np.concatenate([[0], np.cumsum(k * m)])
    col2s = np.repeat(np.arange(k.size), k)
    has_child = np.zeros(k.size, bool)
    for t in range(k.size):
        p = sym["parent"][sf[t + 1] - 1]
        if p >= 0:
            has_child[col2s[p]] = True
    panels = s.export_L()
    A = oracle.sym_lower_to_dense(cp, ri, v)[np.ix_(o.perm, o.perm)]
    checked = 0
    for t in np.flatnonzero(~has_child):
        nb = int(min(k[t], 64))
        if nb < 8:
            continue
        j0 = int(sf[t])
        A11 = A[j0:j0 + nb, j0:j0 + nb].astype(np.float32).astype(np.float64)
        ref = np.linalg.cholesky(A11).astype(np.float32)
        pan = panels[poff[t]: poff[t + 1]].reshape(int(k[t]), int(m[t])).T   # m x k
        L11 = pan[:nb, :nb].astype(np.float32)
        ulp = np.spacing(np.abs(ref))
        assert np.all(np.abs(L11 - ref) <= ulp), (t, float((np.abs(L11 - ref) / ulp).max()))
        checked += 1
    assert checked >= 10


@pytest.mark.parametrize("name", ["1d_J10", "2d_J6", "2d_J7_exp"])
@pytest.mark.parametrize("nrhs", [9, 64, 130])
def test_tensor_core_solve_products_match_simt(wdlib, cuda, name, nrhs):
    """Mixed precision, more than 8 right-hand sides: the solves' products on
    the tensor cores (3xTF32, the default) against the FP32 SIMT kernels, on
    the unrefined solution (ir_tol = 1 stops before any refinement step): both
    are FP32-accurate solves of the same FP32 factor, so they agree to a few
    FP32 roundings times the condition number; refined, both reach 1e-12."""
    b, cp, ri, v, o = _case(name)
    B = rhs(o.n, nrhs, seed=3)
    X = {}
    for simt in (False, True):
        s = wdlib.Solver(ir_tol=1.0, solve_simt=simt).analyze(cp, ri, b).factor(v, "mixed")
        X[simt] = s.solve(B)
        assert s.last_solve["iterations"] == 0
    ref = o.solve(B)
    scale = np.abs(ref).max(0)
    for simt in (False, True):
        assert (np.abs(X[simt] - ref).max(0) / scale).max() <= 1e-3
    assert (np.abs(X[False] - X[True]).max(0) / scale).max() <= 1e-4
    s = wdlib.Solver().analyze(cp, ri, b).factor(v, "mixed")
    Xr = s.solve(B)
    assert oracle.backward_error(cp, ri, v, Xr, B).max() <= 1e-12


@pytest.mark.parametrize("dim,J,ker,nug", [(1, 10, Kernel("exponential", 0.2), 1e-2),
                                           (2, 6, Kernel("exponential", 0.3), 1e-2)])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 2e-5)])
def test_two_term_pattern_factor_and_solve(wdlib, cuda, dim, J, ker, nug, prec, tol):
    """Matrices on the full two-term compression pattern of Theorem 3.1:
    factor columns and refined solves against the oracle."""
    from wdgen import compressed_pattern_two_term

    b = haar_basis(dim, J)
    cp, ri = compressed_pattern_two_term(b, a=1.5, delta=1.2, q=1.0)
    v = compressed_values(b, cp, ri, ker, nug)
    o = oracle.Oracle(cp, ri, b)
    assert o.factor(v) == 0
    s = wdlib.Solver().analyze(cp, ri, b).factor(v, prec)
    L = s.L_csc_like(o.Lp, o.Li)
    Lo = o.L_values()
    starts = o.Lp[:-1]
    rel = np.sqrt(np.add.reduceat((L - Lo) ** 2, starts) / np.add.reduceat(Lo ** 2, starts))
    assert rel.max() <= tol
    B = rhs(o.n, 16, seed=9)
    X = s.solve(B)
    assert oracle.backward_error(cp, ri, v, X, B).max() <= 1e-12


# ---------------------------------------------------------------------------
# FP64 factorization with the Schur updates on the tensor cores (bf16 slices,
# exact products, FP64 combination): the FP64 bar
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", list(CASES))
def test_factor_fp64_tensor_core_updates(wdlib, cuda, name):
    b, cp, ri, v, o = _case(name)
    s = wdlib.Solver(fp64_tc_schur=True).analyze(cp, ri, b)
    s.factor(v, "fp64")
    L = s.L_csc_like(o.Lp, o.Li)
    Lo = o.L_values()
    for j in range(o.n):
        a, e = o.Lp[j], o.Lp[j + 1]
        assert np.linalg.norm(L[a:e] - Lo[a:e]) <= 1e-10 * np.linalg.norm(Lo[a:e]), j
    ref = o.logdet()
    assert abs(s.logdet() - ref) <= 1e-12 * abs(ref)
    B = rhs(o.n, 5, seed=11)
    X = s.solve(B)
    assert oracle.backward_error(cp, ri, v, X, B).max() <= 1e-12
    assert s.last_solve["iterations"] == 0


@pytest.mark.parametrize("tc", [False, True])
def test_fp64_factor_of_a_matrix_with_large_and_small_rows(wdlib, cuda, tc):
    """D A D with D = 2^k_i, k_i in -20..20 (exact scaling): its factor is
    D L, L the factor of A, so D^-1 times the computed factor is held to the
    FP64 bar against the oracle's L -- the slices' per-row scales must follow
    the rows' sizes (an error relative to the scaled factor's columns would
    not be a fair bar: FP64's own error in entry (i, j) scales with D_i)."""
    b, cp, ri, v, o = _case("2d_J5")
    rng = np.random.default_rng(3)
    dsc = 2.0 ** rng.integers(-20, 21, size=o.n)
    cols = np.repeat(np.arange(o.n), np.diff(cp))
    vs = v * dsc[ri] * dsc[cols]
    s = wdlib.Solver(fp64_tc_schur=tc).analyze(cp, ri, b).factor(vs, "fp64")
    assert np.array_equal(s.symbolic()["perm"], o.perm)
    dp = dsc[o.perm]                               # D in the factor's order
    L = s.L_csc_like(o.Lp, o.Li) / dp[o.Li]
    Lo = o.L_values()
    for j in range(o.n):
        a, e = o.Lp[j], o.Lp[j + 1]
        assert np.linalg.norm(L[a:e] - Lo[a:e]) <= 1e-10 * np.linalg.norm(Lo[a:e]), j
