"""The CUDA adjoint of the coupled step (flow on) against the FP64 reference.

lbm_adjoint_coupled differentiates the melted fraction, or the hot-wall
Nusselt number averaged over the steps, with respect to porosity, ln K and
the left wall profile; oracle/coupled_ref.py differentiates the same map by
autograd and is pinned to finite differences of the C oracle.  FP32 on the
GPU: bars of 2e-3 of the largest entry.
"""
import numpy as np
import pytest

import lbm_workloads as W

pytestmark = pytest.mark.gpu

STEPS = 40


def _case():
    w = W.melted_cavity(24)
    params = dict(w.params)
    params.update(T_s=0.1, T_l=0.4)
    tw = (1.0 + 0.1 * np.sin(2 * np.pi * np.arange(w.ny) / w.ny)).astype(np.float32)
    for k in ("phi", "K", "T0", "fl0"):
        setattr(w, k, getattr(w, k).astype(np.float32).astype(np.float64))
    return w, params, tw.astype(np.float64)


@pytest.fixture(scope="module")
def lbm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1503_08406_gb300 as P
    return P


@pytest.mark.parametrize("objective", ["melt", "nusselt"])
def test_coupled_adjoint_matches_fp64_reference(lbm, oracle_mod, objective):
    from oracle.coupled_ref import CoupledRef
    w, params, tw = _case()
    J_ref, dphi_ref, dlnK_ref, dtw_ref = CoupledRef(w.nx, w.ny, params).gradients(
        STEPS, w.T0, w.fl0, w.phi, w.K, tw, objective)
    lat = lbm.Lattice(w.nx, w.ny, **params)
    lat.set_fields(w.phi, w.K, w.T0, w.fl0, tw)
    J, dphi, dlnK, dtw = lat.adjoint_coupled(STEPS, objective)
    assert lat.status() == 0 and lat.steps_done() == STEPS
    assert abs(J - J_ref) < 1e-4 * abs(J_ref), (J, J_ref)
    for got, exp in ((dphi, dphi_ref), (dlnK, dlnK_ref), (dtw, dtw_ref)):
        scale = np.abs(exp).max()
        assert scale > 0
        assert np.abs(got - exp).max() < 2e-3 * scale, (np.abs(got - exp).max(), scale)


def test_coupled_adjoint_rejects_conduction(lbm):
    w = W.two_phase_slab(1.0, nx=40, ny=4)
    p = dict(w.params)
    p.pop("alpha_ratio")
    lat = lbm.Lattice(w.nx, w.ny, **p)
    lat.set_fields(w.phi, w.K, w.T0, w.fl0)
    with pytest.raises(lbm.LBMError):
        lat.adjoint_coupled(10)
