"""Per-cell pins of the oracle's wall functions against hand values.

* Eq. kws: the surface k of the quadratic profile is k_vis(y+) u_tau^2 with
  u_tau = C_mu^(1/4) sqrt(k_P) (Eq. frictionvel); k_vis at y+ = 1, 5, 11 is
  read from tests/golden/kws_kvis.txt, derived there in exact rational
  arithmetic.  The imposed k_ib then follows the quadratic weights.
* Eq. omegaws, P_ib: on a flat immersed wall with the linear shear
  u = (s (y - y_w), 0) and a uniform k set for a chosen y+, every bc cell has
  n = (0, 1) and |(n.grad) u| = s, so P_ib = kappa nu y+ s^2 / ln^2(E y+)
  in the log branch (y+ = 30), P_k = nu_t s^2 in the laminar branch (y+ = 5),
  and 0 in ic cells.
* On a converged high-Re step (every bc cell in the log branch) the log
  branch equals the wall-function form (nu + nu_tw)|du/dn| u_tau,log/(kappa y)
  with u_tau,log = kappa y |du/dn| / ln(E y+) and nu_tw = nu (kappa y+ /
  ln(E y+) - 1), cell by cell.
"""
import math
import os

import numpy as np
import pytest

from paper_2606_06135_gb300 import geometry as G
from oracle import hfdib_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
# published wall-function constants, written out (not read from the oracle)
C_MU, KAPPA, E_WF = 0.09, 0.41, 9.8


def kvis_golden():
    out = {}
    for line in open(os.path.join(GOLDEN, "kws_kvis.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            a, b = line.split()
            out[float(a)] = float(b)
    return out


def flat_wall(yw=2.3):
    """8 x 8 unit cells, a flat immersed wall at y = yw (solid below), k-eps,
    nu = 0.01.  Row j = 2 (centres at y = 2.5) holds the bc cells."""
    g = G.make_grid(8, 8, 1, 0.0, 0.0, 8.0, 8.0)
    X, Y, _ = G.cell_centres(g)
    sigma = Y - yw
    case = G._base_case("flat", g, sigma, np.maximum(sigma, 0), "kepsilon", 100.0, G.bc2d())
    return O.Oracle(case), Y


def k_for_yplus(o, yplus):
    """uniform k with y_eff u_tau / nu = y+ at the bc cells (one y_eff)"""
    ye = o.geo["y_eff"]
    assert np.ptp(ye) == 0.0
    return (yplus * o.nu / (ye[0] * C_MU ** 0.25)) ** 2


@pytest.mark.parametrize("yplus", [1.0, 5.0, 11.0])
def test_kws_surface_k(yplus):
    o, _ = flat_wall()
    k0 = k_for_yplus(o, yplus)
    o.k = np.full(o.m.shape, k0)
    o.imposed_fields()
    np.testing.assert_allclose(o.yplus_bc, yplus, rtol=1e-13)
    assert o.lam_branch.all()            # y+ <= 11: laminar branch
    ut2 = math.sqrt(C_MU) * k0           # u_tau^2 of Eq. frictionvel
    kS = kvis_golden()[yplus] * ut2
    np.testing.assert_allclose(o.k_surface, kS, rtol=1e-12)
    # uniform k: both interpolated values are k0, so the quadratic gives
    # k_ib = wS kS + (w1 + w2) k0 at every bc cell
    geo = o.geo
    want = geo["wS"] * kS + (geo["w1"] + geo["w2"]) * k0
    np.testing.assert_allclose(o.k_ib.ravel()[geo["cell"]], want, rtol=1e-12)


def test_kws_zero_at_the_wall():
    """C_f(0) = 0: k_vis(0) = 0, so k_S vanishes as y+ -> 0."""
    o, _ = flat_wall()
    o.k = np.full(o.m.shape, k_for_yplus(o, 1e-9))
    o.imposed_fields()
    assert np.abs(o.k_surface).max() <= 1e-20


@pytest.mark.parametrize("yplus", [30.0, 5.0])
def test_pib_on_a_linear_shear(yplus):
    o, Y = flat_wall()
    s, nut = 2.0, 0.03
    o.u = [s * (Y - 2.3), np.zeros_like(Y)]
    o.k = np.full(o.m.shape, k_for_yplus(o, yplus))
    o.nut = np.full(o.m.shape, nut)
    o.imposed_fields()
    np.testing.assert_allclose(o.geo["n"][:, :2], np.tile([0.0, 1.0], (len(o.geo["cell"]), 1)), atol=0)
    _, _, _, P = o._production()
    cells = o.geo["cell"]
    Pb = P.ravel()[cells]
    if yplus > 11.0:
        assert not o.lam_branch.any()
        want = KAPPA * o.nu * yplus * s * s / math.log(E_WF * yplus) ** 2
        np.testing.assert_allclose(Pb, want, rtol=1e-12)
    else:
        assert o.lam_branch.all()
        # the full production nu_t 2 S:S; 2 S:S = s^2 away from the inlet and
        # outlet columns, where du_x/dx takes the boundary values
        inner = (cells % 8 > 0) & (cells % 8 < 7)
        np.testing.assert_allclose(Pb[inner], nut * s * s, rtol=1e-12)
    assert np.all(P[o.ic] == 0.0)


@pytest.fixture(scope="module")
def step_converged():
    case = G.case_bfs(64, 16, model="kepsilon")
    o = O.Oracle(case)
    it, res = o.solve(tol=1e-11, max_iter=800)
    assert o.max_residual(res) <= 1e-11
    return o


def test_pib_log_branch_wall_function_form(step_converged):
    o = step_converged
    o.imposed_fields()
    assert not o.lam_branch.any()
    Gr, _, _, P = o._production()
    cells = o.geo["cell"]
    n = o.geo["n"]
    dudn = np.zeros((len(cells), 3))
    for b in range(o.m.dims):
        for a in range(o.m.dims):
            dudn[:, b] += n[:, a] * Gr[a][b].ravel()[cells]
    g = np.sqrt((dudn ** 2).sum(axis=1))
    yp = o.yplus_bc
    y = o.geo["y_eff"]
    ln = np.log(E_WF * yp)
    ut_log = KAPPA * y * g / ln
    nu_tw = o.nu * (KAPPA * yp / ln - 1.0)
    want = (o.nu + nu_tw) * g * ut_log / (KAPPA * y)
    np.testing.assert_allclose(P.ravel()[cells], want, rtol=1e-12)
