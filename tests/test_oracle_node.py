"""Single-node pins of the FP64 oracle against identities the paper fixes.

Each check is built independently of the oracle's own formula: moment
polynomials are constructed from the velocity sets, inverses come from
numpy, the BGK+Guo-Zhao step is written out here from its definition.
"""
import numpy as np
import pytest

EX9 = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY9 = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
EX5 = np.array([0, 1, 0, -1, 0])
EY5 = np.array([0, 0, 1, 0, -1])
CS2 = 1 / 3


def _ctx(oracle_mod, **kw):
    base = dict(bc=("periodic",) * 4, flow=1, tau_nu=0.8, tau_T=0.9, g_beta=1e-4, Pr=1.0)
    base.update(kw)
    return oracle_mod.Oracle(5, 5, **base)


def test_velocity_sets_eq15_eq31():
    # Eq. (15): e_i = (cos((i-1) pi/2), sin((i-1) pi/2)) for i = 1..4,
    # sqrt(2) (cos((2i-9) pi/4), sin((2i-9) pi/4)) for i = 5..8
    for i in range(1, 5):
        a = (i - 1) * np.pi / 2
        assert (EX9[i], EY9[i]) == (round(np.cos(a)), round(np.sin(a)))
        assert (EX5[i], EY5[i]) == (round(np.cos(a)), round(np.sin(a)))
    for i in range(5, 9):
        a = (2 * i - 9) * np.pi / 4
        assert (EX9[i], EY9[i]) == (round(np.sqrt(2) * np.cos(a)), round(np.sqrt(2) * np.sin(a)))


def test_M_rows_are_the_moments_of_eq17(oracle_mod):
    M, Minv, N, Ninv = oracle_mod.matrices()
    e2 = EX9 ** 2 + EY9 ** 2
    # rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy as polynomials of the velocities
    rows = np.array([
        np.ones(9), 3 * e2 - 4, 4.5 * e2 ** 2 - 10.5 * e2 + 4,
        EX9, (3 * e2 - 5) * EX9, EY9, (3 * e2 - 5) * EY9,
        EX9 ** 2 - EY9 ** 2, EX9 * EY9])
    np.testing.assert_array_equal(M, rows)
    MMt = M @ M.T
    np.testing.assert_array_equal(MMt, np.diag([9, 36, 36, 6, 12, 6, 12, 4, 4]))
    np.testing.assert_allclose(Minv, np.linalg.inv(M), atol=1e-15)
    np.testing.assert_allclose(M @ Minv, np.eye(9), atol=1e-15)


def test_N_rows_eq32(oracle_mod):
    _, _, N, Ninv = oracle_mod.matrices()
    e2 = EX5 ** 2 + EY5 ** 2
    rows = np.array([np.ones(5), EX5, EY5, 5 * e2 - 4, EX5 ** 2 - EY5 ** 2])
    np.testing.assert_array_equal(N, rows)
    np.testing.assert_array_equal(N @ N.T, np.diag([5, 2, 2, 20, 4]))
    np.testing.assert_allclose(Ninv, np.linalg.inv(N), atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_feq_moments_match_meq_eq19_eq29(oracle_mod, seed):
    o = _ctx(oracle_mod)
    M, _, _, _ = oracle_mod.matrices()
    rng = np.random.default_rng(seed)
    rho = 1 + 0.05 * rng.standard_normal()
    ux, uy = 0.05 * rng.standard_normal(2)
    varphi = rng.uniform(0.2, 1.0)
    feq = o.feq(rho, ux, uy, varphi)
    np.testing.assert_allclose(M @ feq, o.meq(rho, ux, uy, varphi), atol=1e-15)
    # hydrodynamic moments of the incompressible porous equilibrium
    assert abs(feq.sum() - rho) < 1e-15
    assert abs((EX9 * feq).sum() - ux) < 1e-15  # rho0 = 1
    assert abs((EY9 * feq).sum() - uy) < 1e-15
    assert abs((EX9 * EX9 * feq).sum() - (CS2 * rho + ux * ux / varphi)) < 1e-15
    assert abs((EX9 * EY9 * feq).sum() - ux * uy / varphi) < 1e-15
    assert abs((EY9 * EY9 * feq).sum() - (CS2 * rho + uy * uy / varphi)) < 1e-15


def _guo_force(u, F, varphi, rho0=1.0):
    """Guo-Zhao velocity-space forcing (without the 1 - 1/(2 tau) factor)."""
    eu = EX9 * u[0] + EY9 * u[1]
    eF = EX9 * F[0] + EY9 * F[1]
    uF = u[0] * F[0] + u[1] * F[1]
    return W9 * rho0 * (eF / CS2 + (eu * eF - CS2 * uF) / (CS2 ** 2 * varphi))


@pytest.mark.parametrize("seed", range(5))
def test_forcing_moments_eq22_are_guo_force(oracle_mod, seed):
    o = _ctx(oracle_mod)
    M, _, _, _ = oracle_mod.matrices()
    rng = np.random.default_rng(100 + seed)
    u = 0.05 * rng.standard_normal(2)
    F = 1e-3 * rng.standard_normal(2)
    varphi = rng.uniform(0.2, 1.0)
    S = o.force_moments(u[0], u[1], F[0], F[1], varphi)
    np.testing.assert_allclose(S, M @ _guo_force(u, F, varphi), atol=1e-16)


def _random_f(rng):
    return W9 * (1 + 0.02 * rng.standard_normal(9))


@pytest.mark.parametrize("seed", range(6))
def test_velocity_solve_satisfies_eq25(oracle_mod, seed):
    """u from the explicit Eq. (26)-(28) makes Eq. (25) hold with F(u) of Eq. (4)."""
    rng = np.random.default_rng(200 + seed)
    o = _ctx(oracle_mod, g_beta=1e-3)
    f = _random_f(rng)
    fl = rng.uniform(0.05, 1.0)
    phi = rng.uniform(0.3, 0.7)
    K = 10 ** rng.uniform(-1, 2)
    T = rng.uniform(-1, 2)
    ux, uy, Fx, Fy = o.velocity(f, T, fl, phi, K)
    res_x = ux - ((EX9 * f).sum() + 0.5 * Fx)
    res_y = uy - ((EY9 * f).sum() + 0.5 * Fy)
    assert abs(res_x) < 1e-15 and abs(res_y) < 1e-15
    # Eq. (4) with Eq. (6) at varphi = phi f_l, K the fully liquid permeability
    varphi = phi * fl
    Keff = K * fl ** 3 * ((1 - phi) / (1 - varphi)) ** 2
    CF = 1.75 / np.sqrt(175 * varphi ** 3)
    d = o.derived()
    um = np.hypot(ux, uy)
    G = d["g_beta"] * T
    Fx_ref = -varphi * d["nu_l"] / Keff * ux - varphi * CF / np.sqrt(Keff) * um * ux
    Fy_ref = -varphi * d["nu_l"] / Keff * uy - varphi * CF / np.sqrt(Keff) * um * uy + varphi * G
    assert abs(Fx - Fx_ref) < 1e-15 and abs(Fy - Fy_ref) < 1e-15


def test_velocity_solve_without_porous_matrix_is_v(oracle_mod):
    """K -> infinity, varphi -> 1 removes the drag: u = v (reading d_0 = l_0)."""
    o = _ctx(oracle_mod, g_beta=0.0)
    f = _random_f(np.random.default_rng(3))
    ux, uy, Fx, Fy = o.velocity(f, 0.0, 1.0, 0.999999, np.inf)
    assert abs(ux - (EX9 * f).sum()) < 1e-15
    assert abs(uy - (EY9 * f).sum()) < 1e-15
    assert Fx == 0 and Fy == 0


@pytest.mark.parametrize("seed", range(4))
def test_collision_conserves_mass_and_momentum(oracle_mod, seed):
    rng = np.random.default_rng(300 + seed)
    o = _ctx(oracle_mod, g_beta=1e-3)
    f = _random_f(rng)
    fl, phi, K, T = 0.7, 0.45, 5.0, 0.6
    fp = o.collide_flow(f, T, fl, phi, K)
    ux, uy, Fx, Fy = o.velocity(f, T, fl, phi, K)
    assert abs(fp.sum() - f.sum()) < 1e-15
    # post-collision momentum: sum e f + rho0 F (= rho0 u + rho0 F / 2)
    assert abs((EX9 * fp).sum() - ((EX9 * f).sum() + Fx)) < 1e-15
    assert abs((EY9 * fp).sum() - ((EY9 * f).sum() + Fy)) < 1e-15


@pytest.mark.parametrize("tau", [0.6, 0.9, 1.4])
def test_mrt_with_equal_rates_is_bgk_guo(oracle_mod, tau):
    """Sec. 3.1: with every relaxation rate 1/tau_nu the MRT step is the BGK
    step with the Guo-Zhao porous forcing."""
    s = 1 / tau
    o = _ctx(oracle_mod, tau_nu=tau, s_e=s, s_eps=s, s_q=s, g_beta=2e-3)
    rng = np.random.default_rng(int(tau * 10))
    f = _random_f(rng)
    fl, phi, K, T = 0.8, 0.5, 3.0, 0.4
    ux, uy, Fx, Fy = o.velocity(f, T, fl, phi, K)
    varphi = phi * fl
    feq = o.feq(f.sum(), ux, uy, varphi)
    bgk = f - (f - feq) / tau + (1 - 1 / (2 * tau)) * _guo_force((ux, uy), (Fx, Fy), varphi)
    np.testing.assert_allclose(o.collide_flow(f, T, fl, phi, K), bgk, atol=2e-16)


@pytest.mark.parametrize("seed", range(4))
def test_thermal_equilibrium_eq34_eq39(oracle_mod, seed):
    rng = np.random.default_rng(400 + seed)
    sigma = rng.uniform(0.8, 1.2)
    o = _ctx(oracle_mod, sigma=sigma)
    _, _, N, Ninv = oracle_mod.matrices()
    T = rng.uniform(-1, 2)
    ux, uy = 0.05 * rng.standard_normal(2)
    geq = o.geq(T, ux, uy)
    np.testing.assert_allclose(N @ geq, o.thermal_meq(T, ux, uy), atol=1e-15)
    assert abs(geq.sum() - T) < 1e-15
    assert abs((EX5 * geq).sum() - ux * T / sigma) < 1e-15
    # N^-1 (1, 0, 0, varpi, 0) gives the weights w~ of Eq. (39)
    varpi = -2.0
    wt = Ninv @ np.array([1, 0, 0, varpi, 0])
    np.testing.assert_allclose(wt, [(1 - varpi) / 5] + [(4 + varpi) / 20] * 4, atol=1e-16)
    np.testing.assert_allclose(o.geq(1.0, 0, 0), wt, atol=1e-16)


def test_thermal_collision_source_and_relaxation(oracle_mod):
    o = _ctx(oracle_mod, tau_T=0.75, zeta_e=1.3, zeta_nu=1.7)
    _, _, N, _ = oracle_mod.matrices()
    rng = np.random.default_rng(5)
    g = np.array([0.6, 0.1, 0.1, 0.1, 0.1]) * 0.7 + 0.01 * rng.standard_normal(5)
    ux, uy, s0 = 0.03, -0.02, -0.013
    gp = o.collide_thermal(g, ux, uy, s0)
    T = g.sum()
    # temperature moment: T + S~_0; other moments relax at Theta of Eq. (37)
    assert abs(gp.sum() - (T + s0)) < 1e-15
    n, neq, npost = N @ g, o.thermal_meq(T, ux, uy), N @ gp
    theta = np.array([1, 1 / 0.75, 1 / 0.75, 1.3, 1.7])
    src = np.array([s0, 0, 0, -2.0 * s0, 0])
    np.testing.assert_allclose(npost, n - theta * (n - neq) + src, atol=1e-15)


def test_derived_parameters_recover_dimensionless_groups(oracle_mod):
    """tau_nu, tau_T, g beta from Sec. 4.3 reproduce Ra, Pr and alpha_e of Eq. (9), (39)."""
    Ra, Pr, H, lam, sigma = 1e5, 0.7, 256.0, 0.8, 0.9
    o = oracle_mod.Oracle(8, 8, bc=("dirichlet", "dirichlet", "adiabatic", "adiabatic"),
                          flow=1, Ra=Ra, Pr=Pr, Ma=0.1, H=H, lambda_=lam, sigma=sigma)
    d = o.derived()
    nu_l = d["nu_l"]
    alpha_l = nu_l / Pr
    assert abs(d["g_beta"] * H ** 3 / (nu_l * alpha_l) / Ra - 1) < 1e-14
    assert abs(d["alpha_e"] / alpha_l / lam - 1) < 1e-14
    assert abs(d["nu_e"] - (d["tau_nu"] - 0.5) / 3) < 1e-16
    # Mach number: u_c = sqrt(g beta dT H) = Ma c_s
    assert abs(np.sqrt(d["g_beta"] * H) / np.sqrt(CS2) - 0.1) < 1e-12
