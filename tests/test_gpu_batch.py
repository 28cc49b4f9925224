"""Batched problems (several lambda fields of uneven size: every sweep phase
one launch for all problems, one persistent pressure launch) against the same
problems solved one by one, and against the FP64 oracle.

A problem gets the block partition and the reduction order of its own
launch inside a batch, so a wrong partition or index shows as an O(1)
difference.  The batched and the per-problem kernels are separate
instantiations of the same code, which the compiler may fuse into different
multiply-adds, so the comparison is to round-off (1e-12 relative per field)
rather than bit for bit.  (The persistent pressure kernel is one kernel for
both.)"""
import numpy as np
import pytest

from paper_2606_06135_gb300 import geometry as G
from oracle import hfdib_oracle as O

pytestmark = pytest.mark.gpu


ROUNDOFF = 1e-12


def same_fields(fa, fb, tol=ROUNDOFF, tag=""):
    for n in fb:
        scale = max(np.abs(fb[n]).max(), 1e-300)
        err = np.abs(fa[n] - fb[n]).max() / scale
        assert err <= tol, (tag, n, err)


def uneven_cases(model="kepsilon"):
    return [G.case_grf(64, 32, seed=1, model=model), G.case_grf(48, 24, seed=2, model=model),
            G.case_cylinder(40, 20, model=model)]


OPTION_SETS = {"defaults": {}, "maskB_vanleer": dict(continuity_mask=1, convection=2), "sst": {}}


@pytest.mark.parametrize("options", sorted(OPTION_SETS))
@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_individual_solves(precision, options):
    """Every phase of the batched sweep is one launch for all problems, each
    problem on its own range of blocks with the block partition of its own
    launch, and one persistent launch solves all pressure equations: the
    results equal those of the problems solved one by one to round-off --
    with k-epsilon, with reading B of the continuity mask and vanLeer
    convection, and with k-omega SST."""
    from paper_2606_06135_gb300.hfdib import BatchSolver, Solver
    opts = OPTION_SETS[options]
    cases = uneven_cases("komegasst" if options == "sst" else "kepsilon")
    bs = BatchSolver(cases, precision=precision, **opts)
    r = bs.sweep(12)
    assert r.shape == (3, 10)
    assert np.all(np.isfinite(r))
    for i, c in enumerate(cases):
        s = Solver(c, precision=precision, **opts)
        s.sweep(12)
        same_fields(bs.problem(i).fields(), s.fields(), tag=i)
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


@pytest.mark.parametrize("precision", [0, 1])
def test_3d_batch_equals_individual_solves(precision):
    """3D problems of different size.  FP64 agrees to round-off.  On the mixed
    path the FP32 correction solves stop at a relative residual of 1e-6, and
    where the stop falls depends on FP32 rounding, so the instantiations'
    rounding differences can move each sweep's pressure correction by up to
    ~1e-6 of itself; the corrections of these sweeps are below 1e-2 of the
    fields, so 8 sweeps stay within 8 * 1e-6 * 1e-2 ~ 1e-7."""
    from paper_2606_06135_gb300.hfdib import BatchSolver, Solver
    cases = [G.case_sphere(24, 12, 12), G.case_sphere(20, 12, 10)]
    bs = BatchSolver(cases, precision=precision)
    bs.sweep(8)
    for i, c in enumerate(cases):
        s = Solver(c, precision=precision)
        s.sweep(8)
        same_fields(bs.problem(i).fields(), s.fields(), tol=ROUNDOFF if precision == 0 else 1e-7, tag=i)
        s.close()
    bs.close()


def test_batch_solve_stops_each_problem_on_the_device():
    """The batch solve loops on the device and applies the stop test at the end
    of every sweep: a problem that meets the tolerance at sweep n sits out the
    later sweeps, so its state is that of n sweeps of the same problem alone
    (to round-off), and its reported count is n."""
    from paper_2606_06135_gb300.hfdib import BatchSolver, Solver
    cases = [G.case_cylinder(32, 16), G.case_cylinder(64, 32)]
    bs = BatchSolver(cases, precision=0)
    rc, iters, res = bs.solve(tol=1e-8, max_iter=4000)
    assert rc == 0, (rc, iters, res)
    assert iters[0] != iters[1], iters
    for i, c in enumerate(cases):
        assert max(res[i, :6]) <= 1e-8
        s = Solver(c, precision=0)
        s.sweep(int(iters[i]))
        same_fields(bs.problem(i).fields(), s.fields(), tol=1e-10, tag=i)
        # one sweep fewer does not meet the tolerance
        s2 = Solver(c, precision=0)
        r = s2.sweep(int(iters[i]) - 1)
        assert max(r[:6]) > 1e-8
        s.close()
        s2.close()
    # the problems go on sweeping together afterwards
    r = bs.sweep(2)
    assert np.all(np.isfinite(r))
    bs.close()
