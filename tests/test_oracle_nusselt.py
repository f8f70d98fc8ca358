"""Pins of the oracle's hot-wall Nusselt number (reduce()["nu_hot"]).

The paper does not define a Nusselt number; the reading used throughout is
the mean over the left wall's rows of -H dT/dx / dT at the wall node, with the
second-order one-sided difference (-3 T_0 + 4 T_1 - T_2) / 2.  Three pins,
none of which re-types that formula:

* exactness on quadratic profiles: a second-order one-sided difference is
  exact for T = T_w - x / L + c x^2, so a state with that profile in every
  row has Nu = mean(H / L_y) to rounding, whatever c is.  A first-order or
  shifted stencil, a wrong sign, a wrong H or dT, or wall rows in the mean
  all miss it by O(c) or more;
* the one-phase Neumann solution of Sec. 4.1 (Eq. (43)-(46) with T_i = T_m):
  the wall gradient of Eq. (44) gives
  Nu(t) = H (T_b - T_m) / (dT erf(eta) sqrt(pi D t)), D = alpha_e / sigma;
  the scheme is second-order, so the gap closes like 1 / (D t);
* the wall flux balances the stored heat: per row, the enthalpy
  sum (T + a f_l) grows at the rate D Nu dT / H that enters through the wall.
"""
import numpy as np
import pytest
from scipy.optimize import brentq
from scipy.special import erf

import lbm_workloads as W


def _quadratic_state(o, w, Tw_rows, L_rows, c_rows, wall_rows_value=None):
    """g with node temperatures T(x, y) = Tw(y) - x / L(y) + c(y) x^2; the sum
    of a node's five populations is all that defines its temperature, so the
    whole value goes into the rest population."""
    f, g, fl = o.get_state()
    x = np.arange(w.nx, dtype=np.float64)
    T = Tw_rows[:, None] - x[None, :] / L_rows[:, None] + c_rows[:, None] * x[None, :] ** 2
    if wall_rows_value is not None:
        T[0, :] = wall_rows_value
        T[-1, :] = wall_rows_value
    g[:] = 0.0
    g[0] = T
    o.set_state(g=g)


@pytest.mark.parametrize("walled", [False, True])
def test_nusselt_exact_on_quadratic_profiles(oracle_mod, walled):
    ny = 9
    rng = np.random.default_rng(5)
    if walled:
        w = W.convection_cavity(12)
        w.params = {**w.params, "flow": 0, "tau_T": 0.7}
        ny = w.ny
    else:
        w = W.conduction_slab(nx=12, ny=ny)
    Tw = 1.0 + 0.3 * rng.random(ny)
    L = rng.uniform(3.0, 40.0, ny)
    c = rng.uniform(-0.05, 0.05, ny)
    o = oracle_mod.Oracle(w.nx, w.ny, **w.params)
    o.set_fields(w.phi, w.K, w.T0, w.fl0, Tw)
    _quadratic_state(o, w, Tw, L, c, wall_rows_value=(-7.0 if walled else None))
    H, dT = w.params["H"], w.params["dT"]
    rows = slice(1, ny - 1) if walled else slice(0, ny)
    expect = np.mean(H / (dT * L[rows]))
    got = o.reduce()["nu_hot"]
    assert abs(got - expect) < 1e-12 * abs(expect), (got, expect)
    # the curvature does not enter: a first-order or shifted stencil would see c
    assert abs(np.mean(H * c[rows]) / expect) > 1e-3


def _one_phase_eta(st_eff):
    return brentq(lambda e: e * np.exp(e * e) * erf(e) - st_eff / np.sqrt(np.pi), 1e-6, 5)


def test_nusselt_follows_neumann_wall_gradient_and_heat_balance(oracle_mod):
    """Config-1 slab (256 x 4, phi = 0.5, St = 1, alpha = 0.02, H = 256)."""
    w = W.conduction_slab()
    o = oracle_mod.Oracle(w.nx, w.ny, **w.params)
    o.set_fields(w.phi, w.K, w.T0, w.fl0)
    D = o.derived()["alpha_e"] / w.params["sigma"]
    eta = _one_phase_eta(w.params["sigma"] * w.params["St"] / w.phi[0, 0])
    H, dT = w.params["H"], w.params["dT"]
    times = [2000, 5000, 10000, 20000]
    done, nu_sum = 0, 0.0
    ent0 = o.reduce()["enthalpy"]
    rec = {}
    for t in times:
        while done < t:
            o.step(1)
            done += 1
            nu_sum += o.reduce()["nu_hot"]
        r = o.reduce()
        rec[t] = (r["nu_hot"], (r["enthalpy"] - ent0) / w.ny, D * dT * nu_sum / H)
    rel = []
    for t in times:
        nu_an = H * 1.0 / (dT * erf(eta) * np.sqrt(np.pi * D * t))
        rel.append(rec[t][0] / nu_an - 1)
        # second order: the relative gap times D t stays bounded (measured ~0.25)
        assert abs(rel[-1]) * D * t < 0.4, (t, rel[-1])
    # and it does shrink like 1 / t (not a fixed offset of a wrong factor)
    assert abs(rel[-1]) < 0.2 * abs(rel[0])
    # heat balance between t = 5000 and 20000: stored heat per row grows by the
    # time integral of the wall flux D Nu dT / H
    stored = rec[20000][1] - rec[5000][1]
    flux = rec[20000][2] - rec[5000][2]
    assert abs(flux / stored - 1) < 2e-3, (flux, stored)
