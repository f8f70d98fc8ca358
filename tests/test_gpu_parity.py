"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Error measure: for each field, max_x |gpu - oracle| / max_x |oracle| (a
normwise relative error; pointwise relative error is undefined where a field
crosses zero).  The bar is 1e-4 after 10,000 steps for u, T and f_l; short
runs are held tighter, at 2e-5, since FP32 rounding (6e-8 per operation)
accumulates roughly linearly in the step count before the fields' own
dynamics damp it.
"""
import numpy as np
import pytest

import lbm_workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("ux", "uy", "T", "fl")


@pytest.fixture(scope="module")
def lbm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1503_08406_gb300 as P
    return P


def _f32(w):
    """Round the workload's fields to float32 in place: the CUDA path takes
    float32 inputs, so the oracle must see the same numbers."""
    for k in ("phi", "K", "T0", "fl0"):
        setattr(w, k, getattr(w, k).astype(np.float32).astype(np.float64))
    return w


def _gpu(P, w, steps, **over):
    lat = P.Lattice(w.nx, w.ny, **{**w.params, **over})
    lat.set_fields(w.phi, w.K, w.T0, w.fl0, w.wall_T_left)
    if steps:
        lat.step(steps)
    assert lat.status() == 0
    return lat


def _ora(oracle_mod, w, steps):
    o = oracle_mod.Oracle(w.nx, w.ny, **w.params)
    o.set_fields(w.phi, w.K, w.T0, w.fl0, w.wall_T_left)
    if steps:
        o.step(steps)
    return o


def _errors(got, exp, fields=FIELDS):
    out = {}
    for k in fields:
        scale = np.abs(exp[k]).max()
        if scale == 0:
            out[k] = float(np.abs(got[k]).max())
        else:
            out[k] = float(np.abs(got[k].astype(np.float64) - exp[k]).max() / scale)
    return out


@pytest.mark.parametrize("steps", [1, 2, 3, 8, 51])
def test_melted_cavity_matches_oracle(lbm, oracle_mod, steps):
    """Ragged 40 x 40 cavity (tiles of 32): flow, moving front and walls, both
    step parities."""
    w = _f32(W.melted_cavity(40))
    got = _gpu(lbm, w, steps).macros()
    exp = _ora(oracle_mod, w, steps).macros()
    err = _errors(got, exp, FIELDS + ("rho",))
    assert max(err.values()) < 2e-5, err


@pytest.mark.parametrize("shape,flow", [((45, 37), 1), ((33, 70), 0)])
def test_ragged_periodic_box_matches_oracle(lbm, oracle_mod, shape, flow):
    w = _f32(W.periodic_box(shape[0], ny=shape[1], flow=flow, T_s=-0.02 * (1 - flow),
                            T_l=0.02 * (1 - flow)))
    steps = 120
    got = _gpu(lbm, w, steps).macros()
    exp = _ora(oracle_mod, w, steps).macros()
    fields = FIELDS if flow else ("T", "fl")
    err = _errors(got, exp, fields)
    assert max(err.values()) < 5e-5, err
    # the flow mask really moved in this run
    if flow:
        assert ((exp["fl"] >= 1e-3) != (w.fl0 >= 1e-3)).sum() > 0


def test_narrow_periodic_lattice(lbm, oracle_mod):
    """ny = 3 periodic: the enthalpy halo (8 nodes) wraps the lattice several times."""
    w = _f32(W.conduction_slab(nx=70, ny=3, alpha=0.05))
    got = _gpu(lbm, w, 400).macros()
    exp = _ora(oracle_mod, w, 400).macros()
    err = _errors(got, exp, ("T", "fl"))
    assert max(err.values()) < 2e-5, err


def test_conduction_melting_config(lbm, oracle_mod):
    """256 x 4 conduction melting, 20,000 steps: interface within 1% of the
    one-phase Neumann solution (eta = 0.800601) and parity with the oracle."""
    w = _f32(W.conduction_slab())
    lat = _gpu(lbm, w, 20000)
    got = lat.macros()
    D = lat.derived()["alpha_e"]
    fl = got["fl"].mean(axis=0)
    xm = 0.5 * fl[0] + fl[1:].sum()
    xa = 2 * 0.8006013628 * np.sqrt(D * 20000)
    assert abs(xm / xa - 1) < 0.01, (xm, xa)
    exp = _ora(oracle_mod, w, 20000).macros()
    err = _errors(got, exp, ("T", "fl"))
    assert max(err.values()) < 1e-4, err


@pytest.mark.parametrize("ratio", [1.0, 10.0])
def test_two_phase_conduction_config(lbm, oracle_mod, ratio):
    """Sec. 4.1 two-phase melting (alpha_l / alpha_s = ratio, tau_T by phase),
    200 x 6 to Fo = 0.01 (20,000 steps): parity with the oracle and the
    two-phase Neumann front (eta = 0.37776, 0.44697) within 1% / 2%.

    Here the solid diffuses from T_i = -1, changing by ~1e-5 per step against
    populations of order 0.1-0.6, so FP32 rounding accumulates to 2e-5 (ratio 1)
    and 9e-5 (ratio 10) in T after 20,000 steps (measured; 3e-7 in the
    convection cavity).  A front node's f_l, at the steep end of the mushy band,
    then differs by up to 1.2e-3; the front position by under 0.01 node."""
    w = _f32(W.two_phase_slab(ratio))
    steps = 20000
    got = _gpu(lbm, w, steps).macros()
    exp = _ora(oracle_mod, w, steps).macros()
    err = _errors(got, exp, ("T", "fl"))
    assert err["T"] < 2e-4 and err["fl"] < 5e-3, err
    eta = {1.0: 0.37776, 10.0: 0.44697}[ratio]
    fl = got["fl"].mean(axis=0)
    x_m = 0.5 * fl[0] + fl[1:].sum()
    fo = exp["fl"].mean(axis=0)
    assert abs(x_m - (0.5 * fo[0] + fo[1:].sum())) < 0.01
    x_an = 2 * eta * np.sqrt(w.meta["alpha_l"] * steps)
    assert abs(x_m / x_an - 1) < (0.01 if ratio == 1.0 else 0.02), (x_m, x_an)


def test_phase_dependent_diffusivity_with_flow(lbm, oracle_mod):
    """alpha_l / alpha_s = 3 in the melted cavity (flow, TMA-staged kernel)."""
    w = _f32(W.melted_cavity(64))
    w.params = {**w.params, "alpha_ratio": 3.0}
    lat = _gpu(lbm, w, 51)
    assert lat.kernel_variant() == 2
    err = _errors(lat.macros(), _ora(oracle_mod, w, 51).macros())
    assert max(err.values()) < 2e-5, err


def test_parity_cavity_10000_steps(lbm, oracle_mod):
    """The convection-melting cavity (256^2, Ra = 1e5, heterogeneous porosity
    seed 1): u, T and f_l within 1e-4 of the FP64 oracle after 10,000 steps."""
    w = _f32(W.parity_cavity(256))
    steps = 10000
    lat = _gpu(lbm, w, steps)
    got = lat.macros()
    o = _ora(oracle_mod, w, steps)
    exp = o.macros()
    err = _errors(got, exp)
    assert max(err.values()) < 1e-4, err
    r_g, r_o = lat.reduce(), o.reduce()
    assert abs(r_g["melt_frac"] / r_o["melt_frac"] - 1) < 1e-4
    assert abs(r_g["nu_hot"] / r_o["nu_hot"] - 1) < 1e-4


def _front(fl):
    """Melted length per row: sum over x of f_l (the row's front position)."""
    return fl.sum(axis=1)


def test_convection_cavity_config2(lbm, oracle_mod):
    """Convection melting in the uniform porous cavity (256^2, phi = 0.4,
    Da = 1e-4, Ra = 1e5, Pr = 1, Ste = 1): u, T and f_l within 1e-4 of the
    oracle after 2,000 steps; then on the GPU alone to 50,000 steps, where the
    front leans: liquid heated at the left wall rises and spreads under the
    top wall, so the top rows melt further than the bottom rows."""
    w = _f32(W.convection_cavity(256))
    steps = 2000
    lat = _gpu(lbm, w, steps)
    o = _ora(oracle_mod, w, steps)
    err = _errors(lat.macros(), o.macros())
    assert max(err.values()) < 1e-4, err
    lat.step(50000 - steps)
    assert lat.status() == 0
    fl = lat.macros()["fl"]
    x = _front(fl[1:-1, :])                 # interior rows, bottom to top
    q = len(x) // 4
    top, bottom = x[-q:].mean(), x[:q].mean()
    assert top > bottom + 2.0, (top, bottom)
    assert np.all(np.diff(x[q:-q]) > -0.5)   # the lean is monotone away from the walls


def test_porous_gallium_cavity_matches_oracle(lbm, oracle_mod):
    """Sec. 4.3's parameter set (200^2, Ra = 8.409e5, Pr = 0.0208,
    tau_nu = 0.5054, St = 0.1241): u, T and f_l within 1e-4 of the FP64
    oracle after 4,000 steps, the melted fraction and hot-wall Nusselt number
    too."""
    w = _f32(W.porous_gallium_cavity(200))
    steps = 4000
    lat = _gpu(lbm, w, steps)
    o = _ora(oracle_mod, w, steps)
    err = _errors(lat.macros(), o.macros())
    assert max(err.values()) < 1e-4, err
    r_g, r_o = lat.reduce(), o.reduce()
    assert r_o["melt_frac"] > 0.005   # the front has left the wall
    assert abs(r_g["melt_frac"] / r_o["melt_frac"] - 1) < 1e-4
    assert abs(r_g["nu_hot"] / r_o["nu_hot"] - 1) < 1e-4


@pytest.mark.parametrize("sigma_s", [0.5, 2.0])
def test_solid_heat_capacity_slab_matches_oracle(lbm, oracle_mod, sigma_s):
    """Eq. (7) with sigma_s != sigma_l (sigma linear in f_l, taken at f_l(n) in
    tau_T, n^eq and the latent coefficient) on the Sec. 4.1 slab, 20,000 steps:
    T within 2e-4 of the oracle (the solid's slow diffusion from T_i = -1
    accumulates FP32 rounding, as with the two-phase diffusivity), f_l within
    1e-3 and the front within 0.01 node."""
    w = _f32(W.two_phase_slab(1.0))
    w.params = {**w.params, "sigma_solid": sigma_s}
    steps = 20000
    got = _gpu(lbm, w, steps).macros()
    exp = _ora(oracle_mod, w, steps).macros()
    err = _errors(got, exp, ("T", "fl"))
    assert err["T"] < 2e-4 and err["fl"] < 1e-3, err
    xm = lambda fl: 0.5 * fl.mean(axis=0)[0] + fl.mean(axis=0)[1:].sum()
    assert abs(xm(got["fl"]) - xm(exp["fl"])) < 0.01


def test_solid_heat_capacity_with_flow(lbm, oracle_mod):
    """sigma(f_l) of Eq. (7) in the melted cavity (flow, TMA-staged kernel)."""
    w = _f32(W.melted_cavity(64))
    w.params = {**w.params, "sigma_solid": 0.5}
    lat = _gpu(lbm, w, 51)
    assert lat.kernel_variant() == 2
    o = _ora(oracle_mod, w, 51)
    err = _errors(lat.macros(), o.macros())
    assert max(err.values()) < 2e-5, err
    rg, ro = lat.reduce(), o.reduce()
    assert abs(rg["enthalpy"] - ro["enthalpy"]) <= 1e-5 * abs(ro["enthalpy"])


def test_porous_gallium_cavity_with_solid_sigma(lbm, oracle_mod):
    """Sec. 4.3 with the paper's two heat-capacity ratios (0.8604 liquid,
    0.8352 solid, Eq. (7)): 4,000 steps within 1e-4 of the oracle."""
    w = _f32(W.porous_gallium_cavity(200, solid_sigma=True))
    steps = 4000
    lat = _gpu(lbm, w, steps)
    o = _ora(oracle_mod, w, steps)
    err = _errors(lat.macros(), o.macros())
    assert max(err.values()) < 1e-4, err
    r_g, r_o = lat.reduce(), o.reduce()
    assert abs(r_g["melt_frac"] / r_o["melt_frac"] - 1) < 1e-4


def _walls_errors(lat, o):
    """Field errors with rho on the lattice nodes only: what a wall node's
    slots hold between steps differs by design (the extrapolation rewrites
    them before they are used)."""
    got, exp = lat.macros(), o.macros()
    err = _errors(got, exp)
    inner = (slice(1, -1), slice(1, -1))
    err["rho"] = _errors({"rho": got["rho"][inner]}, {"rho": exp["rho"][inner]}, ("rho",))["rho"]
    return err


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("steps", [1, 2, 3, 51])
def test_extrapolated_flow_walls_match_oracle(lbm, oracle_mod, steps, variant):
    """flow_walls = 1, the non-equilibrium extrapolation of Sec. 4 on the
    no-slip walls, in the melted cavity (walls on all four sides, corners
    included), with both stream-collide kernels and both step parities."""
    w = _f32(W.melted_cavity(64))
    w.params = {**w.params, "flow_walls": 1}
    lat = _gpu(lbm, w, steps, kernel_variant=variant)
    assert lat.kernel_variant() == variant
    err = _walls_errors(lat, _ora(oracle_mod, w, steps))
    assert max(err.values()) < 2e-5, err


@pytest.mark.parametrize("variant", [1, 2])
def test_extrapolated_flow_walls_with_moving_front(lbm, oracle_mod, variant):
    """flow_walls = 1 while the front runs along the top and bottom walls:
    wall nodes start and stop carrying flow with their inward nodes, so the
    links into them are re-paired as the phase changes (ragged 40^2, tiles
    of 32), 400 steps."""
    w = _f32(W.melted_cavity(40))
    w.params = {**w.params, "flow_walls": 1}
    steps = 400
    lat = _gpu(lbm, w, steps, kernel_variant=variant)
    o = _ora(oracle_mod, w, steps)
    err = _walls_errors(lat, o)
    assert max(err.values()) < 5e-5, err
    fl = o.macros()["fl"]
    rows = [1, w.ny - 2]
    changed = (fl[rows, 1:-1] >= 1e-3) != (w.fl0[rows, 1:-1] >= 1e-3)
    assert changed.sum() > 0   # wall nodes did change activity in this run


def test_extrapolated_flow_walls_brinkman_channel(lbm, oracle_mod):
    """Body-force-driven channel between two flow walls (periodic in y, 66 x
    4): after 6,000 steps the GPU profile is the oracle's to 1e-5 and the
    fully developed Brinkman-Forchheimer profile with the no-slip wall on the
    wall nodes to 1e-3."""
    nx, ny, phi, K, G = 66, 4, 0.5, 12.5, 1e-8
    params = dict(bc=("dirichlet", "dirichlet", "periodic", "periodic"), T_bc=(1.0, 1.0, 0, 0),
                  flow=1, tau_nu=1.0, tau_T=1.0, g_beta=G, Pr=1.0, T_ref=0.0, flow_walls=1)
    w = _f32(W.Workload("channel", nx, ny, params, np.full((ny, nx), phi), np.full((ny, nx), K),
                        np.ones((ny, nx)), np.ones((ny, nx))))
    steps = 6000
    lat = _gpu(lbm, w, steps)
    o = _ora(oracle_mod, w, steps)
    got, exp = lat.macros(), o.macros()
    uy, uy_o = got["uy"][1].astype(np.float64), exp["uy"][1]
    assert np.abs(uy - uy_o).max() < 1e-5 * np.abs(uy_o).max()
    d = o.derived()
    r = np.sqrt(phi * d["nu_l"] / (d["nu_e"] * K))
    x = np.arange(nx)
    c = (nx - 1) / 2.0
    u_node = G * K / d["nu_l"] * (1 - np.cosh(r * (x - c)) / np.cosh(r * c))
    assert np.abs(uy[1:-1] - u_node[1:-1]).max() < 1e-3 * u_node.max()


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("steps,walls", [(1, 0), (2, 0), (51, 0), (51, 1)])
def test_front_extrapolation_matches_oracle(lbm, oracle_mod, steps, walls, variant):
    """flow_front = 1 (no-slip on the moving solid-liquid interface by the
    extrapolation of Sec. 4) in the melted cavity, both stream-collide kernels,
    with halfway bounce-back or extrapolated flow walls."""
    w = _f32(W.melted_cavity(64))
    w.params = {**w.params, "flow_front": 1, "flow_walls": walls}
    lat = _gpu(lbm, w, steps, kernel_variant=variant)
    assert lat.kernel_variant() == variant
    err = _walls_errors(lat, _ora(oracle_mod, w, steps))
    assert max(err.values()) < 2e-5, err


@pytest.mark.parametrize("variant", [1, 2])
def test_front_extrapolation_with_moving_front(lbm, oracle_mod, variant):
    """flow_front = 1 while the front moves (ragged 40^2, 400 steps): links
    turn from extrapolated to streaming as nodes melt."""
    w = _f32(W.melted_cavity(40))
    w.params = {**w.params, "flow_front": 1}
    steps = 400
    lat = _gpu(lbm, w, steps, kernel_variant=variant)
    o = _ora(oracle_mod, w, steps)
    err = _walls_errors(lat, o)
    assert max(err.values()) < 5e-5, err
    fl = o.macros()["fl"]
    assert ((fl >= 1e-3) != (w.fl0 >= 1e-3)).sum() > 0   # the flow mask moved


def test_front_extrapolation_channel_between_solid_columns(lbm, oracle_mod):
    """The solid-column channel (periodic both ways, no wall nodes, uniform
    buoyancy): after 6,000 steps the GPU profile is the oracle's to 1e-5 and
    the Brinkman-Forchheimer profile with the no-slip on the solid nodes to
    1e-3."""
    nx, ny, phi, K, G = 66, 4, 0.5, 12.5, 1e-8
    params = dict(bc=("periodic",) * 4, T_bc=(0.0, 0.0, 0.0, 0.0), flow=1, tau_nu=1.0,
                  tau_T=1.0, g_beta=G, Pr=1.0, T_ref=-1.0, T_s=0.0, T_l=0.0, flow_front=1)
    fl0 = np.ones((ny, nx))
    fl0[:, 0] = fl0[:, -1] = 0.0
    w = _f32(W.Workload("solid_channel", nx, ny, params, np.full((ny, nx), phi),
                        np.full((ny, nx), K), np.zeros((ny, nx)), fl0))
    steps = 6000
    lat = _gpu(lbm, w, steps)
    o = _ora(oracle_mod, w, steps)
    uy, uy_o = lat.macros()["uy"][1].astype(np.float64), o.macros()["uy"][1]
    assert np.abs(uy - uy_o).max() < 1e-5 * np.abs(uy_o).max()
    d = o.derived()
    r = np.sqrt(phi * d["nu_l"] / (d["nu_e"] * K))
    x = np.arange(nx)
    c = (nx - 1) / 2.0
    u_node = G * K / d["nu_l"] * (1 - np.cosh(r * (x - c)) / np.cosh(r * c))
    assert np.abs(uy[1:-1] - u_node[1:-1]).max() < 1e-3 * u_node.max()


def test_full_size_cavity_matches_oracle(lbm, oracle_mod):
    """2048^2 (the benchmark size), left third melted so flow runs on a
    third of the lattice: full-field comparison after 3 steps."""
    w = _f32(W.melted_cavity(2048, seed=3, Ra=1e6, Da=1e-4))
    got = _gpu(lbm, w, 3).macros()
    exp = _ora(oracle_mod, w, 3).macros()
    err = _errors(got, exp)
    assert max(err.values()) < 2e-5, err


def test_reductions_match_oracle(lbm, oracle_mod):
    w = W.melted_cavity(64)
    lat = _gpu(lbm, w, 100)
    o = _ora(oracle_mod, w, 100)
    rg, ro = lat.reduce(), o.reduce()
    for k in ("mass", "enthalpy", "melt_frac", "nu_hot"):
        assert abs(rg[k] - ro[k]) <= 1e-5 * abs(ro[k]), (k, rg[k], ro[k])


def test_conservation_on_periodic_box(lbm):
    """Closed domain: FP64 sums of the FP32 state conserve mass and enthalpy to
    FP32 rounding."""
    w = W.periodic_box(96)
    lat = _gpu(lbm, w, 0)
    r0 = lat.reduce()
    lat.step(500)
    r1 = lat.reduce()
    assert abs(r1["mass"] / r0["mass"] - 1) < 1e-6
    assert abs(r1["enthalpy"] - r0["enthalpy"]) / np.abs(w.T0).sum() < 1e-5
    assert abs(r1["melt_frac"] - r0["melt_frac"]) > 1e-3


def test_state_roundtrip_continues_exactly(lbm):
    w = W.melted_cavity(64)
    a = _gpu(lbm, w, 7)                      # odd count: swapped layout
    f, g, fl = a.get_state()
    a.step(6)
    b = _gpu(lbm, w, 0)
    b.set_state(f, g, fl)
    b.step(6)
    ma, mb = a.macros(), b.macros()
    for k in ("ux", "uy", "rho", "T", "fl"):
        np.testing.assert_array_equal(ma[k], mb[k])


def test_host_and_device_pointer_paths_agree(lbm):
    w = W.melted_cavity(48)
    a = _gpu(lbm, w, 0)
    b = lbm.Lattice(w.nx, w.ny, **w.params)
    b.set_fields_host(w.phi, w.K, w.T0, w.fl0)
    a.step(9)
    b.step(9)
    ma, mb = a.macros(), b.macros_host()
    for k in ma:
        np.testing.assert_array_equal(ma[k], mb[k])


def test_inner_iteration_cap_is_reported(lbm):
    w = W.melted_cavity(48)
    lat = _gpu(lbm, w, 0, max_inner_iters=1)
    lat.step(20)
    assert lat.status() == -4          # LBM_ERR_NOT_CONVERGED, read once ...
    assert lat.status() == 0           # ... and cleared


def test_invalid_fields_rejected(lbm):
    w = W.melted_cavity(32)
    lat = lbm.Lattice(w.nx, w.ny, **w.params)
    bad = w.phi.copy()
    bad[3, 3] = 1.0          # flow needs porosity < 1
    with pytest.raises(lbm.LBMError) as e:
        lat.set_fields(bad, w.K, w.T0, w.fl0)
    assert e.value.code == -1
    with pytest.raises(lbm.LBMError):
        lat.set_fields_host(w.phi, -w.K, w.T0, w.fl0)
    fl = w.fl0.copy()
    fl[0, 5] = 1.5
    with pytest.raises(lbm.LBMError):
        lat.set_fields(w.phi, w.K, w.T0, fl)
