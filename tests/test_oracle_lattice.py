"""Lattice-level pins of the FP64 oracle: closed-form flows, conservation,
the enthalpy fixed point, and the analytic phase-change solutions of Sec. 4."""
import numpy as np
import pytest
from scipy.optimize import brentq
from scipy.special import erf, erfc

import lbm_workloads as W


def _run(oracle_mod, w, steps, literal=False, threads=None):
    o = oracle_mod.Oracle(w.nx, w.ny, threads=threads, **w.params)
    o.set_fields(w.phi, w.K, w.T0, w.fl0, w.wall_T_left)
    if steps:
        o.step(steps, literal=literal)
    return o


# ---- flow: closed forms ------------------------------------------------------

@pytest.mark.parametrize("fl,phi,K", [(1.0, 0.4, 1.0), (0.6, 0.5, 4.0)])
def test_uniform_darcy_forchheimer_steady_state(oracle_mod, fl, phi, K):
    """Uniform periodic flow driven by a constant buoyancy reaches
    phi nu/K_eff u + phi C_F/sqrt(K_eff) u^2 = phi G, the steady form of Eq. (2)
    with Eq. (4) (no gradients)."""
    n = 6
    G = 1e-4
    # a mushy band [1 - fl, 2 - fl] makes f_l = fl the enthalpy equilibrium at T = 1
    params = dict(bc=("periodic",) * 4, flow=1, tau_nu=0.8, tau_T=0.9, g_beta=G, Pr=1.0,
                  T_ref=0.0, T_s=1.0 - fl, T_l=2.0 - fl)
    w = W.Workload("uniform", n, n, params, np.full((n, n), phi), np.full((n, n), K),
                   np.ones((n, n)), np.full((n, n), fl))
    o = _run(oracle_mod, w, 3000)
    m = o.macros()
    nu = o.derived()["nu_l"]
    varphi = phi * fl
    Keff = K * fl ** 3 * ((1 - phi) / (1 - varphi)) ** 2
    CF = 1.75 / np.sqrt(175 * varphi ** 3)
    a, b = CF / np.sqrt(Keff), nu / Keff
    u_exact = (-b + np.sqrt(b * b + 4 * a * G)) / (2 * a)
    assert np.abs(m["ux"]).max() < 1e-15
    np.testing.assert_allclose(m["uy"], u_exact, rtol=1e-10)
    np.testing.assert_allclose(m["T"], 1.0, atol=1e-13)
    np.testing.assert_allclose(m["fl"], fl, atol=1e-13)


def test_brinkman_channel_profile(oracle_mod):
    """Fully developed flow between halfway-bounce-back walls:
    u(x) = (G K / nu_l) [1 - cosh(r (x - c)) / cosh(r h)], r^2 = phi nu_l / (nu_e K),
    walls at x = 1/2 and nx - 3/2 (nodes 0 and nx-1 are wall nodes)."""
    nx, ny, phi, K, G = 66, 4, 0.5, 12.5, 1e-8
    params = dict(bc=("dirichlet", "dirichlet", "periodic", "periodic"), T_bc=(1.0, 1.0, 0, 0),
                  flow=1, tau_nu=1.0, tau_T=1.0, g_beta=G, Pr=1.0, T_ref=0.0)
    w = W.Workload("channel", nx, ny, params, np.full((ny, nx), phi), np.full((ny, nx), K),
                   np.ones((ny, nx)), np.ones((ny, nx)))
    o = _run(oracle_mod, w, 6000)
    uy = o.macros()["uy"][1, 1:-1]
    d = o.derived()
    r = np.sqrt(phi * d["nu_l"] / (d["nu_e"] * K))
    x = np.arange(1, nx - 1)
    c, h = (nx - 1) / 2.0, (nx - 2) / 2.0
    u_exact = G * K / d["nu_l"] * (1 - np.cosh(r * (x - c)) / np.cosh(r * h))
    err = np.abs(uy - u_exact).max() / u_exact.max()
    assert err < 5e-3, err
    # away from the walls the profile is exact to the Forchheimer correction (< 1e-5 here)
    core = slice(len(x) // 2 - 8, len(x) // 2 + 8)
    assert np.abs(uy[core] / u_exact[core] - 1).max() < 1e-4


# ---- conservation on closed domains -----------------------------------------

@pytest.mark.parametrize("flow,T_s,T_l", [(1, 0.0, 0.0), (0, -0.05, 0.05)])
def test_mass_and_enthalpy_conserved_on_periodic_box(oracle_mod, flow, T_s, T_l):
    w = W.periodic_box(32, flow=flow, T_s=T_s, T_l=T_l)
    o = _run(oracle_mod, w, 0)
    r0 = o.reduce()
    fl0 = o.macros()["fl"]
    o.step(300)
    r1 = o.reduce()
    fl1 = o.macros()["fl"]
    assert abs(r1["mass"] / r0["mass"] - 1) < 1e-12
    assert abs(r1["enthalpy"] - r0["enthalpy"]) / np.abs(w.T0).sum() < 1e-12
    # the step really changed phase (and, with flow, the flow mask)
    assert np.abs(fl1 - fl0).max() > 0.05
    if flow:
        assert ((fl1 >= 1e-3) != (fl0 >= 1e-3)).sum() > 0


# ---- the enthalpy iteration -------------------------------------------------

def test_literal_and_superposed_source_agree(oracle_mod):
    """Re-running collision + streaming for each inner iteration (Sec. 3.2, literal)
    equals adding the streamed source to the source-free field (Eq. 35-36 are
    linear in S~)."""
    w = W.melted_cavity(32)
    a = _run(oracle_mod, w, 40, literal=True)
    b = _run(oracle_mod, w, 40, literal=False)
    ma, mb = a.macros(), b.macros()
    for k in ma:
        np.testing.assert_allclose(ma[k], mb[k], atol=1e-12, rtol=0)
    fa, ga, _ = a.get_state()
    fb, gb, _ = b.get_state()
    np.testing.assert_allclose(ga, gb, atol=1e-12, rtol=0)


def test_fixed_point_of_enthalpy_relation(oracle_mod):
    """After a step, f_l(n+1) and T(n+1) satisfy Eq. (40)-(42) in the form
    f_l = clamp((T + a f_l - T_s) / (T_l - T_s + a), 0, 1) at every non-wall node."""
    for w in (W.melted_cavity(32), W.corner_solidification(24, alpha=0.02)):
        o = _run(oracle_mod, w, 25)
        m = o.macros()
        a = w.phi * o.derived()["lat"]
        T_s, T_l = w.params["T_s"], w.params["T_l"]
        pred = np.clip((m["T"] + a * m["fl"] - T_s) / (T_l - T_s + a), 0, 1)
        inner = (slice(1, -1), slice(1, -1))
        np.testing.assert_allclose(m["fl"][inner], pred[inner], atol=1e-12, rtol=0)
        assert 0 < m["fl"][inner].mean() < 1


def test_thread_count_does_not_change_results(oracle_mod):
    w = W.periodic_box(32)
    a = _run(oracle_mod, w, 60, threads=1)
    b = _run(oracle_mod, w, 60, threads=4)
    for x, y in zip(a.get_state(), b.get_state()):
        np.testing.assert_array_equal(x, y)


# ---- Sec. 4.1: conduction melting, analytic Neumann solution ----------------

def _neumann_one_phase_eta(st_eff):
    return brentq(lambda e: e * np.exp(e * e) * erf(e) - st_eff / np.sqrt(np.pi), 1e-6, 5)


def test_conduction_melting_matches_neumann(oracle_mod):
    """One-phase case of Eq. (43)-(46) (T_i = T_m): the effective Stefan number
    is sigma St / phi = 2, so eta e^eta^2 erf(eta) = 2 / sqrt(pi), eta = 0.800601,
    and x_m = 2 eta sqrt(D t), D = alpha_e / sigma."""
    w = W.conduction_slab()
    o = _run(oracle_mod, w, 0)
    d = o.derived()
    D = d["alpha_e"] / w.params["sigma"]
    st_eff = w.params["sigma"] * w.params["St"] / w.phi[0, 0]
    eta = _neumann_one_phase_eta(st_eff)
    assert abs(eta - 0.800601) < 1e-6
    times, xm = [5000, 10000, 15000, 20000], []
    done = 0
    for t in times:
        o.step(t - done)
        done = t
        fl = o.macros()["fl"].mean(axis=0)
        xm.append(0.5 * fl[0] + fl[1:].sum())
    xa = 2 * eta * np.sqrt(D * np.array(times))
    rel = np.array(xm) / xa - 1
    assert abs(rel[-1]) < 0.01, rel          # interface position within 1% at t = 20,000
    slope = np.polyfit(np.sqrt(times), xm, 1)[0]
    assert abs(slope / (2 * eta * np.sqrt(D)) - 1) < 5e-3  # x_m grows like sqrt(t)
    # liquid temperature profile, Eq. (44) with T_b = 1, T_m = 0
    T = o.macros()["T"].mean(axis=0)
    x = np.arange(1, int(xa[-1]) - 2)
    T_an = 1 - erf(x / (2 * np.sqrt(D * times[-1]))) / erf(eta)
    assert np.abs(T[x] - T_an).max() < 2e-3


# ---- Sec. 4.2: solidification in a corner ------------------------------------

def _neumann_two_phase_solidification(T_i, T_m, T_c, a):
    """1-D freezing of liquid at T_i from a wall at T_c (equal properties):
    a lam sqrt(pi) = (T_m - T_c) e^-lam^2 / erf(lam) - (T_i - T_m) e^-lam^2 / erfc(lam),
    the solidification form of Eq. (46)."""
    f = lambda l: ((T_m - T_c) * np.exp(-l * l) / erf(l)
                   - (T_i - T_m) * np.exp(-l * l) / erfc(l) - a * l * np.sqrt(np.pi))
    return brentq(f, 1e-6, 5)


def test_corner_solidification_symmetry_and_far_field(oracle_mod):
    """Sec. 4.2 set-up (T_i = 0.3, T_c = -1, St = 4, mushy band +-0.02, phi = sigma = 1)
    on a 60 x 60 lattice, H = N_x / 2, run to Fo = 0.25 with alpha = 0.02 (the only
    diffusivity the paper states, Sec. 4.1; at tau_T >= 0.75 the paper's
    zeta_e = zeta_nu = 1.5 let an odd-even mode grow along slow mushy fronts)."""
    n = 60
    w = W.corner_solidification(n, alpha=0.02)
    o = _run(oracle_mod, w, 0)
    d = o.derived()
    H = n / 2.0
    t = int(round(0.25 * H * H / d["alpha_e"]))  # Fo = 0.25 (Sec. 4.2, H = N_x / 2)
    o.step(t)
    fl = o.macros()["fl"]
    # the problem is symmetric about the diagonal
    assert np.abs(fl - fl.T).max() < 1e-10
    # far from the corner (next to the adiabatic right wall) the front is the
    # 1-D two-phase Neumann front measured from the bottom wall node
    a = w.phi[0, 0] * d["lat"]
    lam = _neumann_two_phase_solidification(w.meta["T_i"], 0.0, w.meta["T_c"], a)
    X_an = 2 * lam * np.sqrt(d["alpha_e"] * t)
    col = fl[:, -3]
    X = 0.5 * (1 - col[0]) + (1 - col[1:]).sum()
    assert abs(X / X_an - 1) < 0.02, (X, X_an)
    # along the diagonal two walls cool the material: the front is further out
    diag = np.array([fl[i, i] for i in range(n)])
    X_diag = np.sqrt(2) * (0.5 * (1 - diag[0]) + (1 - diag[1:]).sum())
    assert X_diag > X
