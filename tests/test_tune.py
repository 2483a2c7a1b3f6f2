"""The schedule tuner: the C ABI's per-level schedule flags (host-only
handles on CPU; the factor's arithmetic is the same on both schedules, which
the GPU parity tests check for the all-tasks and all-pairs schedules), and the
tuner's measurement, choice and cache on a GB300."""
import json

import numpy as np
import pytest

from wdgen import Kernel, compressed_pattern, compressed_values, haar_basis, rhs


def _case(J=5):
    b = haar_basis(2, J)
    cp, ri = compressed_pattern(b)
    return b, cp, ri


def test_level_schedule_flags_on_a_host_only_handle(wdlib):
    b, cp, ri = _case()
    s = wdlib.Solver(symbolic_only=True).analyze(cp, ri, b)
    n = s.info()["nlevels"]
    assert s.level_schedule() == [0] * n
    flags = [l % 2 for l in range(n)]
    s.set_level_schedule(flags)
    assert s.level_schedule() == flags
    with pytest.raises(wdlib.WdError) as e:
        s.set_level_schedule([0] * (n + 1))
    assert e.value.status == wdlib.WD_ERR_INVALID_ARG
    with pytest.raises(wdlib.WdError) as e:
        s.set_level_schedule([2] * n)
    assert e.value.status == wdlib.WD_ERR_INVALID_ARG
    # a new analysis resets the flags
    s.analyze(cp, ri, b)
    assert s.level_schedule() == [0] * n
    # launch pairs everywhere when the option asks for them
    t = wdlib.Solver(symbolic_only=True, step_launches=True).analyze(cp, ri, b)
    assert t.level_schedule() == [1] * n


def test_structure_key_depends_on_the_analysis(wdlib):
    from paper_2007_01541_gb300 import tune
    b, cp, ri = _case(5)
    k1 = tune.structure_key(wdlib.Solver(symbolic_only=True).analyze(cp, ri, b))
    k2 = tune.structure_key(wdlib.Solver(symbolic_only=True).analyze(cp, ri, b))
    k3 = tune.structure_key(wdlib.Solver(symbolic_only=True, relax_k=16).analyze(cp, ri, b))
    b6, cp6, ri6 = _case(6)
    k4 = tune.structure_key(wdlib.Solver(symbolic_only=True).analyze(cp6, ri6, b6))
    assert k1 == k2 and len({k1, k3, k4}) == 3


@pytest.mark.gpu
def test_tuner_chooses_caches_and_keeps_the_factor(wdlib, cuda, tmp_path):
    import oracle
    from paper_2007_01541_gb300 import tune
    b, cp, ri = _case(7)
    v = compressed_values(b, cp, ri, Kernel("matern32", 0.1), 1e-3)
    s = wdlib.Solver().analyze(cp, ri, b)
    path = str(tmp_path / "cache.json")
    r = tune.tune_schedule(s, v, reps=2, cache_path=path)
    n = s.info()["nlevels"]
    assert not r["cached"] and r["evaluations"] == n + 1 and len(r["schedule"]) == n
    assert s.level_schedule() == r["schedule"]
    assert r["ms"] <= r["ms_default"]
    # the chosen schedule factors and solves to the refinement target
    s.factor(v, "mixed")
    B = rhs(b.N, 4, seed=2)
    X = s.solve(B)
    assert oracle.backward_error(cp, ri, v, X, B).max() <= 1e-12
    # a second solver with the same structure takes the cached choice
    s2 = wdlib.Solver().analyze(cp, ri, b)
    r2 = tune.tune_schedule(s2, v, cache_path=path)
    assert r2["cached"] and s2.level_schedule() == r["schedule"]
    assert list(json.load(open(path)).values())[0]["schedule"] == r["schedule"]
