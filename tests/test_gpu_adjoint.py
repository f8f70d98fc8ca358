"""The CUDA adjoint of the conduction step against the FP64 reference.

lbm_adjoint_melt differentiates the melted fraction after N steps with
respect to the porosity field and the left wall's temperature profile by the
discrete adjoint (reverse of the step, the enthalpy fixed point by the
implicit function theorem) with checkpointing; the FP64 reference
(oracle/adjoint_ref.py) differentiates the same map by autograd and is itself
pinned to finite differences of the C oracle.  The CUDA path runs in FP32, so
the bars are relative, 1e-3 for the wall profile and
for the porosity field normwise.
"""
import numpy as np
import pytest

import lbm_workloads as W

pytestmark = pytest.mark.gpu

STEPS = 400


def _case():
    w = W.two_phase_slab(1.0, nx=40, ny=4)
    params = dict(w.params)
    params.pop("alpha_ratio")
    params.update(T_s=-0.3, T_l=0.3)
    y = np.arange(w.ny)
    Tw = (1.0 + 0.2 * np.sin(2 * np.pi * y / w.ny)).astype(np.float32).astype(np.float64)
    phi = (0.6 + 0.2 * np.random.default_rng(0).random((w.ny, w.nx))).astype(np.float32)
    return w, params, Tw, phi.astype(np.float64)


@pytest.fixture(scope="module")
def lbm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1503_08406_gb300 as P
    return P


@pytest.fixture(scope="module")
def reference(oracle_mod):
    from oracle.adjoint_ref import ConductionRef
    w, params, Tw, phi = _case()
    return ConductionRef(w.nx, w.ny, params).gradients(STEPS, w.T0, w.fl0, phi, Tw)


def _lattice(P, w, params, phi, Tw):
    lat = P.Lattice(w.nx, w.ny, **params)
    lat.set_fields(phi, w.K, w.T0, w.fl0, Tw)
    return lat


def test_adjoint_matches_fp64_reference(lbm, reference):
    w, params, Tw, phi = _case()
    J_ref, dphi_ref, dtw_ref = reference
    lat = _lattice(lbm, w, params, phi, Tw)
    J, dphi, dtw = lat.adjoint_melt(STEPS)
    assert lat.status() == 0
    assert abs(J - J_ref) < 1e-5 * abs(J_ref) + 1e-7, (J, J_ref)
    assert np.abs(dtw - dtw_ref).max() < 1e-3 * np.abs(dtw_ref).max(), (dtw, dtw_ref)
    assert np.abs(dphi - dphi_ref).max() < 1e-3 * np.abs(dphi_ref).max(), \
        (np.abs(dphi - dphi_ref).max(), np.abs(dphi_ref).max())


def test_checkpoint_spacing_does_not_change_the_gradient(lbm):
    w, params, Tw, phi = _case()
    a = _lattice(lbm, w, params, phi, Tw).adjoint_melt(STEPS, checkpoint_every=1)
    b = _lattice(lbm, w, params, phi, Tw).adjoint_melt(STEPS, checkpoint_every=37)
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_keeping_every_step_matches_recomputation(lbm):
    """checkpoint_every = 0 keeps f_l of every step from a graph-replayed
    forward run; K > 0 recomputes from checkpoints step by step."""
    w, params, Tw, phi = _case()
    a = _lattice(lbm, w, params, phi, Tw).adjoint_melt(STEPS)
    b = _lattice(lbm, w, params, phi, Tw).adjoint_melt(STEPS, checkpoint_every=37)
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("K", [0, 37])
def test_context_ends_where_the_forward_run_does(lbm, K):
    w, params, Tw, phi = _case()
    lat = _lattice(lbm, w, params, phi, Tw)
    lat.step(3)   # an odd start: the forward run begins with a single step
    lat.adjoint_melt(STEPS, checkpoint_every=K)
    plain = _lattice(lbm, w, params, phi, Tw)
    plain.step(3)
    plain.step(STEPS)
    assert lat.steps_done() == STEPS + 3
    ma, mb = lat.macros(), plain.macros()
    for k in ("T", "fl"):
        np.testing.assert_array_equal(ma[k], mb[k])


def test_autograd_function(lbm, reference):
    import torch
    from paper_1503_08406_gb300.autograd import MeltedFraction
    w, params, Tw, phi = _case()
    lat = lbm.Lattice(w.nx, w.ny, **params)
    phi_t = torch.tensor(phi, dtype=torch.float32, requires_grad=True)
    tw_t = torch.tensor(Tw, dtype=torch.float32, requires_grad=True)
    J = MeltedFraction.apply(phi_t, tw_t, lat, w.K, w.T0, w.fl0, STEPS)
    (2.0 * J).backward()
    _, dphi_ref, dtw_ref = reference
    assert np.abs(tw_t.grad.numpy() - 2 * dtw_ref).max() < 2e-3 * np.abs(dtw_ref).max()
    assert np.abs(phi_t.grad.numpy() - 2 * dphi_ref).max() < 2e-3 * np.abs(dphi_ref).max()


@pytest.fixture(scope="module")
def reference_nu(oracle_mod):
    from oracle.adjoint_ref import ConductionRef
    w, params, Tw, phi = _case()
    return ConductionRef(w.nx, w.ny, params).gradients(STEPS, w.T0, w.fl0, phi, Tw,
                                                        objective="nusselt")


def test_nusselt_adjoint_matches_fp64_reference(lbm, reference_nu):
    w, params, Tw, phi = _case()
    J_ref, dphi_ref, dtw_ref = reference_nu
    lat = _lattice(lbm, w, params, phi, Tw)
    J, dphi, dtw = lat.adjoint(STEPS, "nusselt")
    assert lat.status() == 0
    assert abs(J - J_ref) < 1e-5 * abs(J_ref), (J, J_ref)
    assert np.abs(dtw - dtw_ref).max() < 1e-3 * np.abs(dtw_ref).max(), (dtw, dtw_ref)
    assert np.abs(dphi - dphi_ref).max() < 1e-3 * np.abs(dphi_ref).max(), \
        (np.abs(dphi - dphi_ref).max(), np.abs(dphi_ref).max())
    # the same run through the checkpointed path, bit for bit
    again = _lattice(lbm, w, params, phi, Tw).adjoint(STEPS, "nusselt", checkpoint_every=37)
    assert again[0] == J and np.array_equal(again[1], dphi) and np.array_equal(again[2], dtw)


def test_nusselt_autograd_function(lbm, reference_nu):
    import torch
    from paper_1503_08406_gb300.autograd import HotWallNusselt
    w, params, Tw, phi = _case()
    lat = lbm.Lattice(w.nx, w.ny, **params)
    phi_t = torch.tensor(phi, dtype=torch.float32, requires_grad=True)
    tw_t = torch.tensor(Tw, dtype=torch.float32, requires_grad=True)
    (0.5 * HotWallNusselt.apply(phi_t, tw_t, lat, w.K, w.T0, w.fl0, STEPS)).backward()
    _, dphi_ref, dtw_ref = reference_nu
    assert np.abs(tw_t.grad.numpy() - 0.5 * dtw_ref).max() < 2e-3 * np.abs(dtw_ref).max()
    assert np.abs(phi_t.grad.numpy() - 0.5 * dphi_ref).max() < 2e-3 * np.abs(dphi_ref).max()


def test_unsupported_configuration_rejected(lbm):
    w = W.melted_cavity(48)   # flow on, walls on all sides
    lat = lbm.Lattice(w.nx, w.ny, **w.params)
    lat.set_fields(w.phi, w.K, w.T0, w.fl0)
    with pytest.raises(lbm.LBMError):
        lat.adjoint_melt(10)
    w, params, Tw, phi = _case()
    narrow = W.two_phase_slab(1.0, nx=4, ny=4)
    p4 = dict(narrow.params)
    p4.pop("alpha_ratio")
    lat = lbm.Lattice(4, 4, **p4)
    lat.set_fields(narrow.phi, narrow.K, narrow.T0, narrow.fl0)
    with pytest.raises(lbm.LBMError):
        lat.adjoint(10, "nusselt")   # x = 2 would be the right wall


@pytest.mark.parametrize("objective", ["melt", "nusselt"])
def test_adjoint_64x64_against_fp64_reference(lbm, oracle_mod, objective):
    """A 64 x 64 slab with seeded porosity and a varying wall profile, 400
    steps: the FP64 reference (autograd through every step and inner
    iteration) against the CUDA adjoint, both objectives."""
    from oracle.adjoint_ref import ConductionRef
    w = W.adjoint_slab(64, 64, seed=1)
    phi = w.phi.astype(np.float32).astype(np.float64)
    tw = w.wall_T_left.astype(np.float32).astype(np.float64)
    J_ref, dphi_ref, dtw_ref = ConductionRef(w.nx, w.ny, w.params).gradients(
        400, w.T0, w.fl0, phi, tw, objective=objective)
    lat = lbm.Lattice(w.nx, w.ny, **w.params)
    lat.set_fields(phi, w.K, w.T0, w.fl0, tw)
    J, dphi, dtw = lat.adjoint(400, objective)
    assert lat.status() == 0
    assert abs(J - J_ref) < 1e-5 * abs(J_ref), (J, J_ref)
    assert np.abs(dtw - dtw_ref).max() < 1e-3 * np.abs(dtw_ref).max()
    assert np.abs(dphi - dphi_ref).max() < 1e-3 * np.abs(dphi_ref).max()
    assert (np.abs(dphi_ref) > 0).sum() > 64   # the front has crossed several columns
