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


def test_brinkman_channel_with_extrapolated_walls(oracle_mod):
    """flow_walls = 1 (Sec. 4's non-equilibrium extrapolation for the no-slip
    walls): the wall is on the wall nodes, so the fully developed profile is
    u(x) = (G K / nu_l) [1 - cosh(r (x - c)) / cosh(r h)] with c = h = (nx - 1)/2;
    the oracle's is within 1e-3 of it, and next to the wall 90% above the
    halfway bounce-back profile (wall half a node further out)."""
    nx, ny, phi, K, G = 66, 4, 0.5, 12.5, 1e-8
    params = dict(bc=("dirichlet", "dirichlet", "periodic", "periodic"), T_bc=(1.0, 1.0, 0, 0),
                  flow=1, tau_nu=1.0, tau_T=1.0, g_beta=G, Pr=1.0, T_ref=0.0, flow_walls=1)
    w = W.Workload("channel", nx, ny, params, np.full((ny, nx), phi), np.full((ny, nx), K),
                   np.ones((ny, nx)), np.ones((ny, nx)))
    o = _run(oracle_mod, w, 6000)
    uy = o.macros()["uy"][1]
    d = o.derived()
    r = np.sqrt(phi * d["nu_l"] / (d["nu_e"] * K))
    x = np.arange(nx)
    u_node = G * K / d["nu_l"] * (1 - np.cosh(r * (x - (nx - 1) / 2)) / np.cosh(r * (nx - 1) / 2))
    u_half = G * K / d["nu_l"] * (1 - np.cosh(r * (x - (nx - 1) / 2)) / np.cosh(r * (nx - 2) / 2))
    assert np.abs(uy[1:-1] - u_node[1:-1]).max() < 1e-3 * u_node.max()
    assert uy[1] > 1.9 * u_half[1]
    assert np.abs(o.macros()["ux"]).max() < 1e-15


def test_brinkman_channel_between_solid_columns_with_front_extrapolation(oracle_mod):
    """flow_front = 1 (Sec. 4's non-equilibrium extrapolation for the no-slip
    condition on the solid-liquid interface): a channel, periodic both ways, no
    wall nodes, bounded by two solid columns (f_l = 0, held at T_m with the
    isothermal melting point, so that neither phase changes) and driven by a
    uniform buoyancy (T - T_ref = 1).  The no-slip sits on the solid nodes: the
    developed profile is the flow-wall one, within 1e-3 of
    (G K / nu_l) [1 - cosh(r (x - c)) / cosh(r c)], c = (nx - 1)/2, and next to
    the solid 90% above the halfway bounce-back profile."""
    nx, ny, phi, K, G = 66, 4, 0.5, 12.5, 1e-8
    params = dict(bc=("periodic",) * 4, T_bc=(0.0, 0.0, 0.0, 0.0), flow=1, tau_nu=1.0,
                  tau_T=1.0, g_beta=G, Pr=1.0, T_ref=-1.0, T_s=0.0, T_l=0.0, flow_front=1)
    fl0 = np.ones((ny, nx))
    fl0[:, 0] = fl0[:, -1] = 0.0
    w = W.Workload("solid_channel", nx, ny, params, np.full((ny, nx), phi), np.full((ny, nx), K),
                   np.zeros((ny, nx)), fl0)
    o = _run(oracle_mod, w, 6000)
    m = o.macros()
    uy = m["uy"][1]
    assert np.array_equal(m["fl"], fl0)   # no phase change
    d = o.derived()
    r = np.sqrt(phi * d["nu_l"] / (d["nu_e"] * K))
    x = np.arange(nx)
    c = (nx - 1) / 2.0
    u_node = G * K / d["nu_l"] * (1 - np.cosh(r * (x - c)) / np.cosh(r * c))
    u_half = G * K / d["nu_l"] * (1 - np.cosh(r * (x - c)) / np.cosh(r * (nx - 2) / 2))
    assert np.abs(uy[1:-1] - u_node[1:-1]).max() < 1e-3 * u_node.max()
    assert uy[1] > 1.9 * u_half[1]
    assert np.abs(m["ux"]).max() < 1e-15
    # halfway bounce-back on the same columns puts the wall half a node further in
    o2 = _run(oracle_mod, W.Workload("solid_channel_bb", nx, ny, {**params, "flow_front": 0},
                                     w.phi, w.K, w.T0, fl0), 6000)
    uy2 = o2.macros()["uy"][1]
    assert np.abs(uy2[1:-1] - u_half[1:-1]).max() < 2e-3 * u_half.max()


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


# ---- Sec. 4.1: two-phase conduction melting with alpha_l != alpha_s ------------

def _neumann_two_phase_melting(ratio, St=1.0, T_b=1.0, T_m=0.0, T_i=-1.0):
    """eta of Eq. (46) with k_s / k_l = alpha_s / alpha_l (equal rho c_p), written out
    from the melting problem: the flux balance at x_m = 2 eta sqrt(alpha_l t)."""
    r = ratio
    f = lambda e: (np.exp(-e * e) / erf(e)
                   + (1.0 / r) * np.sqrt(r) * (T_i - T_m) / (T_b - T_m)
                   * np.exp(-e * e * r) / erfc(e * np.sqrt(r))
                   - e * np.sqrt(np.pi) / St)
    return brentq(f, 1e-6, 3.0)


@pytest.mark.parametrize("ratio,front_tol,T_tol", [(1.0, 0.01, 5e-3), (10.0, 0.02, 5e-2)])
def test_two_phase_conduction_melting(oracle_mod, ratio, front_tol, T_tol):
    """Sec. 4.1 set-up: 200 x 6 periodic in y, T_b = 1, T_i = -1, mushy band +-0.02,
    St = 1, alpha_s = 0.02, alpha_l = ratio alpha_s through a liquid-fraction
    weighted tau_T; at Fo = t alpha_s / H^2 = 0.01 (H = 200) the front is the
    two-phase Neumann front, and the liquid and solid profiles follow Eq. (44), (45).
    With one diffusivity for both phases (ratio ignored) the ratio-10 front would
    sit 15% short of it."""
    w = W.two_phase_slab(ratio)
    o = _run(oracle_mod, w, 0)
    t = int(round(0.01 * 200 ** 2 / w.meta["alpha_s"]))
    o.step(t)
    m = o.macros()
    eta = _neumann_two_phase_melting(ratio)
    a_l, a_s = w.meta["alpha_l"], w.meta["alpha_s"]
    fl = m["fl"].mean(axis=0)
    x_m = 0.5 * fl[0] + fl[1:].sum()
    x_an = 2 * eta * np.sqrt(a_l * t)
    assert abs(x_m / x_an - 1) < front_tol, (x_m, x_an)
    x = np.arange(w.nx, dtype=float)
    T_an = np.where(x <= x_an, 1 - erf(x / (2 * np.sqrt(a_l * t))) / erf(eta),
                    -1 + erfc(x / (2 * np.sqrt(a_s * t))) / erfc(eta * np.sqrt(a_l / a_s)))
    assert np.abs(m["T"].mean(axis=0) - T_an).max() < T_tol
    # the solution is one-dimensional
    assert np.abs(m["T"] - m["T"][0]).max() < 1e-12


def test_two_phase_eta_matches_paper_values():
    """eta for alpha_l / alpha_s = 1 and 10 (St = 1, T_b = 1, T_m = 0, T_i = -1)."""
    assert abs(_neumann_two_phase_melting(1.0) - 0.37776) < 1e-5
    assert abs(_neumann_two_phase_melting(10.0) - 0.44697) < 1e-5


def test_theta_follows_liquid_fraction(oracle_mod):
    """zeta_alpha(f_l) = 1 / (1/2 + alpha_e(f_l) / (sigma c_sT^2)), alpha_e linear in f_l."""
    w = W.two_phase_slab(10.0)
    o = oracle_mod.Oracle(w.nx, w.ny, **w.params)
    for fl, alpha in ((0.0, 0.02), (1.0, 0.2), (0.25, 0.25 * 0.2 + 0.75 * 0.02)):
        assert abs(o.theta_T(fl) - 1.0 / (0.5 + alpha / 0.2)) < 1e-14


def test_porous_gallium_cavity_relaxation_times(oracle_mod):
    """Sec. 4.3's parameter set through the oracle's derivation of tau_nu and
    tau_T (Ma = 0.1, J = 1, H = 200, Pr = 0.0208, Ra = 8.409e5,
    lambda = 0.2719, sigma = 0.8604, c_s^2 = 1/3, c_sT^2 = 1/5): worked out by
    hand from the section's two formulas, tau_nu = 0.5054482 and
    tau_T = 0.6379572; the thermal diffusivity alpha_l = nu_l / Pr = 0.0873103
    and the latent coefficient a = phi / (sigma St) = 3.605691."""
    w = W.porous_gallium_cavity(200)
    o = oracle_mod.Oracle(w.nx, w.ny, **w.params)
    d = o.derived()
    assert abs(d["tau_nu"] - 0.5054482) < 1e-7
    assert abs(d["tau_T"] - 0.6379572) < 1e-7
    assert abs(d["nu_l"] / 0.0208 - 0.0873103) < 1e-7
    assert abs(0.385 * d["lat"] - 3.605691) < 1e-6
    assert abs(w.params["T_s"] - 0.3712) < 1e-12 and abs(w.params["T_l"] - 0.4112) < 1e-12


# ---- Eq. (7): heat capacity ratio following the liquid fraction ---------------

def _neumann_front(k_l, D_l, k_s, D_s, latent, T_b=1.0, T_m=0.0, T_i=-1.0):
    """lambda of the front x_m = 2 lambda sqrt(t) of a two-phase Neumann
    problem: dT/dt = D d2T/dx2 in each phase, and at the front
    latent dx_m/dt = -k_l dT_l/dx + k_s dT_s/dx."""
    f = lambda L: (k_l * (T_b - T_m) * np.exp(-L * L / D_l)
                   / (np.sqrt(np.pi * D_l) * erf(L / np.sqrt(D_l)))
                   - k_s * (T_m - T_i) * np.exp(-L * L / D_s)
                   / (np.sqrt(np.pi * D_s) * erfc(L / np.sqrt(D_s))) - latent * L)
    return brentq(f, 1e-9, 0.5)


def test_theta_follows_heat_capacity(oracle_mod):
    """tau_T(f_l) = 1/2 + alpha_e(f_l) / (sigma(f_l) c_sT^2) with sigma linear in
    f_l (Eq. (7)) and alpha_l = sigma_l c_sT^2 (tau_T - 1/2): for the Sec. 4.1 slab
    with alpha_l / alpha_s = 10 (alpha_s = 0.02, tau_T = 1.5, c_sT^2 = 0.2,
    sigma_l = 1) and sigma_s = 0.5, worked by hand: f_l = 0: 0.5 + 0.02 / 0.1 =
    0.7; f_l = 1: 0.5 + 0.2 / 0.2 = 1.5; f_l = 0.5: alpha_e = 0.11, sigma = 0.75,
    0.5 + 0.11 / 0.15."""
    w = W.two_phase_slab(10.0)
    o = oracle_mod.Oracle(w.nx, w.ny, **{**w.params, "sigma_solid": 0.5})
    for fl, tau in ((0.0, 0.7), (1.0, 1.5), (0.5, 0.5 + 0.11 / 0.15)):
        assert abs(1.0 / o.theta_T(fl) - tau) < 1e-13, (fl, 1.0 / o.theta_T(fl), tau)


@pytest.mark.parametrize("sigma_s", [0.5, 2.0])
def test_two_phase_melting_with_solid_heat_capacity(oracle_mod, sigma_s):
    """The Sec. 4.1 slab (alpha_l = alpha_s = 0.02, sigma_l = 1) with a different
    solid heat capacity: after 20,000 steps the front sits within 2% of the
    Neumann front of the scheme's continuum problem (D = alpha / sigma per
    phase, latent = int_0^1 phi / (St sigma(f)) df = ln(sigma_l / sigma_s) /
    (sigma_l - sigma_s)).  The physical problem (fluxes alpha dT/dx, latent
    phi / St) puts the front 27% (sigma_s = 0.5) and 41% (sigma_s = 2)
    elsewhere: with sigma varying in space the scheme carries D dT/dx across
    the front, not alpha dT/dx."""
    w = W.two_phase_slab(1.0)
    o = oracle_mod.Oracle(w.nx, w.ny, **{**w.params, "sigma_solid": sigma_s})
    o.set_fields(w.phi, w.K, w.T0, w.fl0)
    t = 20000
    o.step(t)
    fl = o.macros()["fl"].mean(axis=0)
    x_m = 0.5 * fl[0] + fl[1:].sum()
    D_l, D_s = 0.02, 0.02 / sigma_s
    latent = np.log(1.0 / sigma_s) / (1.0 - sigma_s)
    x_an = 2 * _neumann_front(D_l, D_l, D_s, D_s, latent) * np.sqrt(t)
    assert abs(x_m / x_an - 1) < 0.02, (x_m, x_an)
    # the physical problem: fluxes alpha dT/dx, latent phi / St = 1
    x_phys = 2 * _neumann_front(0.02, D_l, 0.02, D_s, 1.0) * np.sqrt(t)
    assert abs(x_m / x_phys - 1) > 0.15, (x_m, x_phys)


def test_sigma_solid_equal_to_sigma_is_constant_sigma(oracle_mod):
    """sigma_solid = sigma is the constant-sigma model, bit for bit, on a
    convecting cavity."""
    w = W.melted_cavity(32)
    a = oracle_mod.Oracle(w.nx, w.ny, **w.params)
    b = oracle_mod.Oracle(w.nx, w.ny, **{**w.params, "sigma_solid": w.params.get("sigma", 1.0)})
    for o in (a, b):
        o.set_fields(w.phi, w.K, w.T0, w.fl0)
        o.step(20)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
