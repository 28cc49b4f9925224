"""Pins of the oracle's k-omega SST model (Menter, the model Sec. 2.1 cites;
the coefficients are his published ones, the paper prints none).

* Homogeneous decay (lambda == 0, uniform flow, no shear) in both limits of
  the blend.  A tiny wall distance gives F1 = 1: omega = 1/(beta1 (t + t0))
  and k ~ (t + t0)^(-beta*/beta1), beta1 = 0.075.  A huge one gives F1 = 0:
  the same with beta2 = 0.0828.  The two exponents differ by 10 %.
* With a wall distance that makes F1 and F2 differ along the decay, the
  omega equation's local sink coefficient -U d(omega)/dx / omega^2 follows
  F1 beta1 + (1 - F1) beta2, not the F2 blend.
* F1, F2 and CD_kw at hand-evaluated cells, one per branch of arg1, and the
  three limiters (nu_t, the k production, the omega source) at cells where
  they bind and where they do not.  Every expected number is derived in the
  comments from Menter's definitions with round inputs.
"""
import math

import numpy as np
import pytest

from paper_2606_06135_gb300 import geometry as G
from oracle import hfdib_oracle as O

SWEEPS = 900
# Menter's published SST constants, written out here rather than read from
# the oracle's table, so that a wrong table entry fails the pins
BETA1, BETA2, BETA_STAR = 0.075, 0.0828, 0.09


def decayed_sst(ywall):
    """Uniform inflow at I = 10 %, l_t = 0.02, Re 1e8 (nu ~ 0), 400 x 4 cells
    over x in [0, 2]; converged, so k(x), omega(x) are the decay in time t = x/U."""
    case = G.case_uniform(400, 4, Re=1e8, I_in=0.1, model="komegasst")
    case["lt_in"] = 0.02
    case["ywall"] = np.full_like(case["ywall"], ywall)
    o = O.Oracle(case)
    for _ in range(SWEEPS):
        res = o.sweep()
    assert res["k"] <= 1e-12 and res["omega"] <= 1e-12, res
    X, _, _ = G.cell_centres(case["grid"])
    return o, X[0, 0]


def decay_exponent(t, k, t0):
    sel = (t > 0.5) & (t < 1.8)
    return -np.polyfit(np.log(t[sel] + t0), np.log(k[sel]), 1)[0]


@pytest.mark.parametrize("limit", ["inner", "outer"])
def test_sst_homogeneous_decay_limits(limit):
    # inner: y = 1e-9 (clipped to 1e-3 h) -> sqrt(k)/(beta* omega y) ~ 1e4 -> F1 = 1
    # outer: y = 1e3 -> arg1 ~ 2e-4 -> F1 = tanh(arg1^4) ~ 0
    o, t = decayed_sst(1e-9 if limit == "inner" else 1e3)
    beta = BETA1 if limit == "inner" else BETA2
    other = BETA2 if limit == "inner" else BETA1
    t0 = 1.0 / (beta * o.omega_in)
    expo = BETA_STAR / beta
    got = decay_exponent(t, o.k[0, 0], t0)
    assert abs(got - expo) <= 5e-3 * expo, (got, expo)
    # the other limit's exponent is ~10 % away
    assert abs(got - BETA_STAR / other) > 5e-2 * expo
    # d omega/dt = -beta omega^2: omega (t + t0) beta = 1
    sel = (t > 0.5) & (t < 1.8)
    prod = o.omega[0, 0][sel] * (t[sel] + t0) * beta
    assert np.abs(prod - 1.0).max() <= 3e-3, np.abs(prod - 1.0).max()
    # no shear: the stress limiter is inactive and nu_t = k/omega
    np.testing.assert_allclose(o.nut, o.k / o.omega, rtol=1e-9)


def test_sst_omega_sink_blends_with_F1():
    """y = 0.278 puts sqrt(k)/(beta* omega y) near 0.8 at the inlet: F1 =
    tanh(a^4) runs 0.39 -> 0.85 along the decay while F2 = tanh(4 a^2) stays
    above 0.98, so the blend function is told apart by the local sink."""
    o, t = decayed_sst(0.278)
    w = o.omega[0, 0]
    dx = t[1] - t[0]
    # upwind march of d omega/dt = -beta omega^2 (+ diffusion and cross
    # diffusion, each ~0.2 % here): beta ~ -U (w_i - w_{i-1}) / (dx w_i^2)
    beta_loc = -(w[1:] - w[:-1]) / (dx * w[1:] ** 2)
    k = np.maximum(o.k, O.K_MIN)
    gk = O.gauss_grad(o.m, o.k, o.bnd.scalar_spec(o.k_in))
    gw = O.gauss_grad(o.m, o.omega, o.bnd.scalar_spec(o.omega_in))
    _, F1, F2 = o._sst_blend(k, o.omega, np.zeros(o.m.shape), gk, gw)
    F1, F2 = F1[0, 0][1:], F2[0, 0][1:]
    b_f1 = F1 * BETA1 + (1.0 - F1) * BETA2
    b_f2 = F2 * BETA1 + (1.0 - F2) * BETA2
    sel = slice(50, -5)
    assert F1[sel].min() < 0.5 and F2[sel].min() > 0.95
    assert (np.abs(beta_loc / b_f1 - 1.0)[sel]).max() <= 1e-2
    # where the two blends differ by more than 3 % (most of the decay), the
    # local sink is far from the F2 blend
    far = np.abs(b_f1 / b_f2 - 1.0)[sel] > 0.03
    assert far.sum() >= 100
    assert (np.abs(beta_loc / b_f2 - 1.0)[sel][far]).min() > 2e-2


def _blend_at(cells):
    """Evaluate the oracle's blend at hand-chosen cells: each cell is
    (k, omega, y, nu, grad k, grad omega) on a 4 x 4 grid (2D)."""
    case = G.case_uniform(4, 4, model="komegasst")
    o = O.Oracle(case)
    shape = o.m.shape
    out = []
    for k, w, y, nu, gk, gw in cells:
        o.ywall = np.full(shape, y)
        o.nu = nu
        gkf = [np.full(shape, v) for v in gk]
        gwf = [np.full(shape, v) for v in gw]
        CD, F1, F2 = o._sst_blend(np.full(shape, k), np.full(shape, w), np.zeros(shape), gkf, gwf)
        out.append((float(CD.ravel()[0]), float(F1.ravel()[0]), float(F2.ravel()[0])))
    return out


def test_sst_blend_hand_cells():
    (cdA, f1A, f2A), (cdB, f1B, f2B), (cdC, f1C, f2C), (cdD, f1D, f2D) = _blend_at([
        # A: k = 0.0081 (sqrt 0.09), omega = 1, y = 1, nu = 1e-4, no gradients.
        #    sqrt(k)/(beta* omega y) = 0.09/0.09 = 1; 500 nu/(y^2 omega) = 0.05;
        #    CD = 0 -> CD+ = 1e-10 -> 4 sigma_w2 k/(CD+ y^2) huge; arg1 = 1.
        #    arg2 = max(2, 0.05) = 2.
        (0.0081, 1.0, 1.0, 1e-4, (0.0, 0.0), (0.0, 0.0)),
        # B: k = 0.0009 (sqrt 0.03), nu = 1e-3: sqrt(k)/(beta* omega y) = 1/3,
        #    500 nu/(y^2 omega) = 0.5 wins arg1 = 0.5; arg2 = max(2/3, 0.5) = 2/3.
        (0.0009, 1.0, 1.0, 1e-3, (0.0, 0.0), (0.0, 0.0)),
        # C: as A with grad k = (0.1, 0), grad omega = (0.5, 0): CD = 2 sigma_w2
        #    0.05 / 1 = 0.0856; 4 sigma_w2 k/(CD y^2) = 4 0.0081 (0.856/0.0856)
        #    = 0.324 wins arg1 (sigma_w2 = 0.856).  arg2 = 2.
        (0.0081, 1.0, 1.0, 1e-4, (0.1, 0.0), (0.5, 0.0)),
        # D: as C with grad omega = (-0.5, 0): CD = -0.0856 (returned signed);
        #    CD+ = 1e-10, so arg1 = 1 as in A.
        (0.0081, 1.0, 1.0, 1e-4, (0.1, 0.0), (-0.5, 0.0)),
    ])
    assert cdA == 0.0
    assert math.isclose(f1A, math.tanh(1.0), rel_tol=1e-14), f1A
    assert math.isclose(f2A, math.tanh(4.0), rel_tol=1e-14), f2A
    assert cdB == 0.0
    assert math.isclose(f1B, math.tanh(0.5 ** 4), rel_tol=1e-12), f1B
    assert math.isclose(f2B, math.tanh((2.0 / 3.0) ** 2), rel_tol=1e-12), f2B
    assert math.isclose(cdC, 0.0856, rel_tol=1e-13), cdC
    assert math.isclose(f1C, math.tanh(0.324 ** 4), rel_tol=1e-12), f1C
    assert math.isclose(f2C, math.tanh(4.0), rel_tol=1e-14), f2C
    assert math.isclose(cdD, -0.0856, rel_tol=1e-13), cdD
    assert math.isclose(f1D, math.tanh(1.0), rel_tol=1e-14), f1D
    assert math.isclose(f2D, math.tanh(4.0), rel_tol=1e-14), f2D


def test_sst_limiters_hand_cells():
    nut = O.Oracle.sst_nut
    # nu_t = a1 k / max(a1 omega, b1 F2 sqrt(2 S:S)), a1 = 0.31, b1 = 1.
    # k = 0.31, omega = 1, 2 S:S = 4: F2 = 1 -> max(0.31, 2) = 2 -> 0.0961/2
    assert math.isclose(float(nut(0.31, 1.0, 4.0, 1.0)), 0.04805, rel_tol=1e-13)
    # F2 = 0.5 -> max(0.31, 1) = 1 -> 0.0961
    assert math.isclose(float(nut(0.31, 1.0, 4.0, 0.5)), 0.0961, rel_tol=1e-13)
    # F2 = 0.1 -> max(0.31, 0.2) = 0.31: the limiter is off, nu_t = k/omega
    assert math.isclose(float(nut(0.31, 1.0, 4.0, 0.1)), 0.31, rel_tol=1e-13)
    prod = O.Oracle.sst_k_production
    # min(G, c1 beta* k omega), c1 = 10: k = 0.5, omega = 2 -> 0.9
    assert math.isclose(float(prod(10.0, 0.5, 2.0)), 0.9, rel_tol=1e-13)
    assert float(prod(0.5, 0.5, 2.0)) == 0.5
    gbn = O.Oracle.sst_gbynu
    # min(2 S:S, (c1/a1) beta* omega max(a1 omega, b1 F2 sqrt(2 S:S))):
    # 2 S:S = 100, omega = 1, F2 = 1 -> (10/0.31) 0.09 max(0.31, 10) = 900/31
    assert math.isclose(float(gbn(100.0, 1.0, 1.0)), 900.0 / 31.0, rel_tol=1e-13)
    # 2 S:S = 0.25, omega = 1, F2 = 1 -> bound (10/0.31) 0.09 0.5 > 0.25
    assert float(gbn(0.25, 1.0, 1.0)) == 0.25
