"""Batched problems (several lambda fields of uneven size, one batched
persistent pressure launch per sweep) against the same problems solved one
by one, and against the FP64 oracle."""
import numpy as np
import pytest

from paper_2606_06135_gb300 import geometry as G
from oracle import hfdib_oracle as O

pytestmark = pytest.mark.gpu


def uneven_cases(model="kepsilon"):
    return [G.case_grf(64, 32, seed=1, model=model), G.case_grf(48, 24, seed=2, model=model),
            G.case_cylinder(40, 20, model=model)]


OPTION_SETS = {"defaults": {}, "maskB_vanleer": dict(continuity_mask=1, convection=2)}


@pytest.mark.parametrize("options", sorted(OPTION_SETS))
@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_individual_solves_bit_for_bit(precision, options):
    """Same per-problem arithmetic, block partition and summation order as
    the single-problem persistent kernel: identical results, also with
    reading B of the continuity mask and vanLeer convection."""
    from paper_2606_06135_gb300.hfdib import BatchSolver, Solver
    opts = OPTION_SETS[options]
    cases = uneven_cases()
    bs = BatchSolver(cases, precision=precision, **opts)
    r = bs.sweep(12)
    assert r.shape == (3, 10)
    assert np.all(np.isfinite(r))
    for i, c in enumerate(cases):
        s = Solver(c, precision=precision, **opts)
        s.sweep(12)
        fb = bs.problem(i).fields()
        fs = s.fields()
        for n in fs:
            np.testing.assert_array_equal(fb[n], fs[n], err_msg="%d %s" % (i, n))
        s.close()
    bs.close()


def test_batch_converges_to_the_oracle_states():
    from paper_2606_06135_gb300.hfdib import BatchSolver
    cases = [G.case_cylinder(48, 24), G.case_cylinder(40, 20)]
    bs = BatchSolver(cases, precision=1)
    rc, iters, res = bs.solve(tol=1e-12, max_iter=6000, check_every=20)
    assert rc == 0, (rc, iters, res)
    for i, c in enumerate(cases):
        o = O.Oracle(c)
        o.solve(tol=1e-12, max_iter=2000)
        f = bs.problem(i).fields()
        for name, ref in (("ux", o.u[0]), ("uy", o.u[1]), ("p", o.p), ("k", o.k), ("eps", o.eps)):
            err = np.linalg.norm(f[name] - ref) / np.linalg.norm(ref)
            assert err < 1e-9, (i, name, err)
    bs.close()


def test_batch_autotune_picks_a_valid_configuration():
    from paper_2606_06135_gb300.hfdib import BatchSolver
    bs = BatchSolver(uneven_cases(), precision=1)
    best = bs.autotune(trial_sweeps=1)
    assert best["threads"] in (512, 1024)
    assert best["tail_cells"] in (256, 1024, 4096)
    assert best["coarse_sweeps"] in (2, 4, 8)
    assert best["candidates"] >= 1 and best["us_per_sweep"] > 0
    r = bs.sweep(5)
    assert np.all(np.isfinite(r))
    # a second batch of the same shape reuses the cached choice
    bs2 = BatchSolver(uneven_cases(), precision=1)
    r2 = bs2.sweep(2)
    assert np.all(np.isfinite(r2))
    bs.close()
    bs2.close()
