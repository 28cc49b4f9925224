"""The persistent pressure kernels' bounded barrier waits: a wait that runs
out of polls is reported as HFDIB_ERR_TIMEOUT by the next residual read, and
the handle stays usable.

The timeout is provoked without a fault or a hang: a poll budget of one
makes every barrier wait that is not already complete give up at once (the
waits bound themselves; no kernel waits forever or traps).  After the
timed-out sweep the state is restored from a checkpoint taken before it, and
the next sweep reproduces, bit for bit, the same sweep of an untouched twin.
"""
import numpy as np
import pytest

from paper_2606_06135_gb300 import geometry as G
from paper_2606_06135_gb300 import hfdib

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_single_problem_timeout(precision):
    case = G.case_cylinder(64, 32)
    s = hfdib.Solver(case, precision=precision)
    twin = hfdib.Solver(case, precision=precision)
    s.sweep(3)
    twin.sweep(3)
    state = s.get_state()
    s.set_barrier_polls(1)
    with pytest.raises(hfdib.HfdibError) as e:
        s.sweep(1)
    assert e.value.code == hfdib.ERR_TIMEOUT
    # reported once: the flag is cleared by the read that reported it
    s.set_barrier_polls(0)
    s.set_state(state)
    r1 = s.sweep(1)
    r2 = twin.sweep(1)
    np.testing.assert_array_equal(r1, r2)
    for name in ("ux", "uy", "p", "k", "eps"):
        np.testing.assert_array_equal(s.field(name).cpu().numpy(), twin.field(name).cpu().numpy())
    # solve_steady reports it as well
    s.set_barrier_polls(1)
    with pytest.raises(hfdib.HfdibError) as e:
        s.solve(tol=1e-12, max_iter=5, check_every=1, raise_on_fail=True)
    assert e.value.code == hfdib.ERR_TIMEOUT
    s.set_barrier_polls(0)
    s.set_state(state)
    assert np.all(np.isfinite(s.sweep(1)))
    s.close()
    twin.close()


def test_batch_timeout():
    cases = [G.case_cylinder(48, 24), G.case_cylinder(64, 32)]
    b = hfdib.BatchSolver(cases, precision=1)
    twin = hfdib.BatchSolver(cases, precision=1)
    b.sweep(2)
    twin.sweep(2)
    states = [b.problem(i).get_state() for i in range(len(cases))]
    b.set_barrier_polls(1)
    with pytest.raises(hfdib.HfdibError) as e:
        b.sweep(1)
    assert e.value.code == hfdib.ERR_TIMEOUT
    b.set_barrier_polls(0)
    for i, st in enumerate(states):
        b.problem(i).set_state(st)
    np.testing.assert_array_equal(b.sweep(1), twin.sweep(1))
    for i in range(len(cases)):
        np.testing.assert_array_equal(b.problem(i).field("p").cpu().numpy(),
                                      twin.problem(i).field("p").cpu().numpy())
    b.close()
    twin.close()
