"""FP64 reference for the adjoint of the conduction step, pinned to the C
oracle: its forward map equals the oracle's, and its gradients (autograd
through every step and inner iteration) equal central finite differences of
the oracle itself, which shares no code with it."""
import numpy as np
import pytest

import lbm_workloads as W

torch = pytest.importorskip("torch")


def _case():
    w = W.two_phase_slab(1.0, nx=40, ny=4)
    params = dict(w.params)
    params.pop("alpha_ratio")
    params.update(T_s=-0.3, T_l=0.3)   # a wide mushy band: fronts stay off the clamps
    y = np.arange(w.ny)
    Tw = 1.0 + 0.2 * np.sin(2 * np.pi * y / w.ny)
    phi = 0.6 + 0.2 * np.random.default_rng(0).random((w.ny, w.nx))
    return w, params, Tw, phi


STEPS = 400


def _J_oracle(oracle_mod, w, params, phi, Tw):
    o = oracle_mod.Oracle(w.nx, w.ny, **params)
    o.set_fields(phi, w.K, w.T0, w.fl0, Tw)
    o.step(STEPS)
    return o.macros()["fl"][:, 1:-1].mean(), o


@pytest.fixture(scope="module")
def reference(oracle_mod):
    from oracle.adjoint_ref import ConductionRef
    w, params, Tw, phi = _case()
    ref = ConductionRef(w.nx, w.ny, params)
    J, d_phi, d_tw = ref.gradients(STEPS, w.T0, w.fl0, phi, Tw)
    return w, params, Tw, phi, ref, J, d_phi, d_tw


def test_forward_equals_oracle(oracle_mod, reference):
    w, params, Tw, phi, ref, J, _, _ = reference
    g, fl = ref.run(STEPS, w.T0, w.fl0, torch.tensor(phi), torch.tensor(Tw))
    J_o, o = _J_oracle(oracle_mod, w, params, phi, Tw)
    m = o.macros()
    assert np.abs(fl.numpy() - m["fl"]).max() < 1e-12
    T = g.sum(dim=0).numpy()
    assert np.abs(T[:, 1:-1] - m["T"][:, 1:-1]).max() < 1e-12
    assert abs(J - J_o) < 1e-13


def test_gradients_equal_finite_differences(oracle_mod, reference):
    w, params, Tw, phi, _, _, d_phi, d_tw = reference
    h = 1e-6
    for yy in range(w.ny):
        tp, tm = Tw.copy(), Tw.copy()
        tp[yy] += h
        tm[yy] -= h
        fd = (_J_oracle(oracle_mod, w, params, phi, tp)[0]
              - _J_oracle(oracle_mod, w, params, phi, tm)[0]) / (2 * h)
        assert abs(d_tw[yy] - fd) < 1e-6 * abs(fd), (yy, d_tw[yy], fd)
    # cells behind, inside and ahead of the mushy front
    for yy, xx in ((0, 1), (1, 2), (2, 3), (0, 3), (3, 6)):
        pp, pm = phi.copy(), phi.copy()
        pp[yy, xx] += h
        pm[yy, xx] -= h
        fd = (_J_oracle(oracle_mod, w, params, pp, Tw)[0]
              - _J_oracle(oracle_mod, w, params, pm, Tw)[0]) / (2 * h)
        assert abs(d_phi[yy, xx] - fd) < 1e-6 * max(abs(fd), 1e-12), (yy, xx, d_phi[yy, xx], fd)
    # the wall profile matters, and porosity only where the front has been
    assert (np.abs(d_tw) > 1e-3).all()
    assert np.abs(d_phi[:, 10:]).max() == 0.0


def _nu_oracle(oracle_mod, w, params, phi, Tw):
    """The oracle's left-wall Nusselt number after each step, averaged."""
    o = oracle_mod.Oracle(w.nx, w.ny, **params)
    o.set_fields(phi, w.K, w.T0, w.fl0, Tw)
    acc = 0.0
    for _ in range(STEPS):
        o.step(1)
        acc += o.reduce()["nu_hot"]
    return acc / STEPS


@pytest.fixture(scope="module")
def reference_nu(oracle_mod):
    from oracle.adjoint_ref import ConductionRef
    w, params, Tw, phi = _case()
    ref = ConductionRef(w.nx, w.ny, params)
    J, d_phi, d_tw = ref.gradients(STEPS, w.T0, w.fl0, phi, Tw, objective="nusselt")
    return w, params, Tw, phi, J, d_phi, d_tw


def test_nusselt_objective_equals_oracle(oracle_mod, reference_nu):
    w, params, Tw, phi, J, _, _ = reference_nu
    J_o = _nu_oracle(oracle_mod, w, params, phi, Tw)
    assert abs(J - J_o) < 1e-11 * abs(J_o), (J, J_o)


def test_nusselt_gradients_equal_finite_differences(oracle_mod, reference_nu):
    """The time-averaged hot-wall Nusselt number: the wall profile enters
    directly (T_0) and through the field; porosity only through the field."""
    w, params, Tw, phi, _, d_phi, d_tw = reference_nu
    h = 1e-6
    for yy in range(w.ny):
        tp, tm = Tw.copy(), Tw.copy()
        tp[yy] += h
        tm[yy] -= h
        fd = (_nu_oracle(oracle_mod, w, params, phi, tp)
              - _nu_oracle(oracle_mod, w, params, phi, tm)) / (2 * h)
        assert abs(d_tw[yy] - fd) < 1e-6 * abs(fd), (yy, d_tw[yy], fd)
    for yy, xx in ((0, 1), (1, 2), (2, 3), (3, 6)):
        pp, pm = phi.copy(), phi.copy()
        pp[yy, xx] += h
        pm[yy, xx] -= h
        fd = (_nu_oracle(oracle_mod, w, params, pp, Tw)
              - _nu_oracle(oracle_mod, w, params, pm, Tw)) / (2 * h)
        assert abs(d_phi[yy, xx] - fd) < 1e-5 * max(abs(fd), 1e-9), (yy, xx, d_phi[yy, xx], fd)
    # the direct term alone would give 1.5 H / (dT ny) per row; the field adds to it
    H = float(params["H"])
    assert np.all(np.abs(d_tw - 1.5 * H / w.ny) > 1e-3 * 1.5 * H / w.ny)
