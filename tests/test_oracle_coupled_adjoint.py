"""FP64 reference for the adjoint of the coupled step (flow lattice on),
pinned to the C oracle: its forward map equals the oracle's (populations,
liquid fraction), and its gradients with respect to ln K, phi and the left
wall profile (autograd through every step and inner iteration) equal central
finite differences of the oracle, which shares no code with it."""
import numpy as np
import pytest

import lbm_workloads as W

torch = pytest.importorskip("torch")

STEPS = 80


def _case():
    """A 24^2 cavity whose left third starts liquid (flow, the moving front and
    the flow mask all active), mushy band [0.1, 0.4] so that the front is not
    a kink, and a varying hot-wall profile."""
    w = W.melted_cavity(24)
    params = dict(w.params)
    params.update(T_s=0.1, T_l=0.4)
    tw = 1.0 + 0.1 * np.sin(2 * np.pi * np.arange(w.ny) / w.ny)
    return w, params, tw


def _J_oracle(oracle_mod, w, params, phi, K, tw, objective):
    o = oracle_mod.Oracle(w.nx, w.ny, **params)
    o.set_fields(phi, K, w.T0, w.fl0, tw)
    if objective == "melt":
        o.step(STEPS)
        return o.reduce()["melt_frac"]
    acc = 0.0
    for _ in range(STEPS):
        o.step(1)
        acc += o.reduce()["nu_hot"]
    return acc / STEPS


@pytest.mark.parametrize("which", ["cavity", "periodic"])
def test_forward_equals_oracle(oracle_mod, which):
    from oracle.coupled_ref import CoupledRef
    if which == "cavity":
        w, params, tw = _case()
    else:
        w = W.periodic_box(16, flow=1)
        params, tw = dict(w.params), np.zeros(w.ny)
    ref = CoupledRef(w.nx, w.ny, params)
    f, g, fl, _ = ref.run(60, w.T0, w.fl0, torch.tensor(w.phi), torch.tensor(w.K),
                          torch.tensor(tw))
    o = oracle_mod.Oracle(w.nx, w.ny, **params)
    o.set_fields(w.phi, w.K, w.T0, w.fl0, tw if which == "cavity" else None)
    o.step(60)
    fo, go, flo = o.get_state()
    assert np.abs(f.numpy() - fo).max() < 1e-12
    assert np.abs(g.numpy() - go).max() < 1e-12
    assert np.abs(fl.numpy() - flo).max() < 1e-12
    if which == "cavity":
        assert (flo[1:-1, 1:-1] >= 1e-3).sum() > 100   # flow runs on a good part of it


@pytest.mark.parametrize("objective", ["melt", "nusselt"])
def test_gradients_equal_finite_differences(oracle_mod, objective):
    """ln K and phi at cells behind and at the front, and far ahead of it
    (zero), and the wall profile; tolerance: 2e-3 relative plus 5e-9, the
    finite differences' own noise (inner iterations stop at 1e-13)."""
    from oracle.coupled_ref import CoupledRef
    w, params, tw = _case()
    J, d_phi, d_lnK, d_tw = CoupledRef(w.nx, w.ny, params).gradients(
        STEPS, w.T0, w.fl0, w.phi, w.K, tw, objective)
    assert abs(J - _J_oracle(oracle_mod, w, params, w.phi, w.K, tw, objective)) < 1e-12 * abs(J)
    h = 1e-6
    ok = lambda ad, fd: abs(ad - fd) <= 2e-3 * abs(fd) + 5e-9
    for yy, xx in ((12, 6), (5, 8), (18, 9)):
        Kp, Km = w.K.copy(), w.K.copy()
        Kp[yy, xx] *= np.exp(h)
        Km[yy, xx] *= np.exp(-h)
        fd = (_J_oracle(oracle_mod, w, params, w.phi, Kp, tw, objective)
              - _J_oracle(oracle_mod, w, params, w.phi, Km, tw, objective)) / (2 * h)
        assert ok(d_lnK[yy, xx], fd), ("lnK", yy, xx, d_lnK[yy, xx], fd)
        pp, pm = w.phi.copy(), w.phi.copy()
        pp[yy, xx] += h
        pm[yy, xx] -= h
        fd = (_J_oracle(oracle_mod, w, params, pp, w.K, tw, objective)
              - _J_oracle(oracle_mod, w, params, pm, w.K, tw, objective)) / (2 * h)
        assert ok(d_phi[yy, xx], fd), ("phi", yy, xx, d_phi[yy, xx], fd)
    for yy in (3, 12):
        tp, tm = tw.copy(), tw.copy()
        tp[yy] += h
        tm[yy] -= h
        fd = (_J_oracle(oracle_mod, w, params, w.phi, w.K, tp, objective)
              - _J_oracle(oracle_mod, w, params, w.phi, w.K, tm, objective)) / (2 * h)
        assert ok(d_tw[yy], fd), ("tw", yy, d_tw[yy], fd)
    # the permeability matters where the liquid moves, not in the far solid
    assert np.abs(d_lnK[:, 1:10]).max() > 1e-8
    assert np.abs(d_lnK[:, 14:]).max() == 0.0


def test_gradients_on_64x64_cavity(oracle_mod):
    """The same reference on a 64^2 melting cavity (100 steps, the hot-wall
    Nusselt number averaged over them): ln K gradients at two cells near the
    hot wall (about -1.7e-6 and -3.9e-7) and a wall row (about 0.66), against
    finite differences of the oracle."""
    from oracle.coupled_ref import CoupledRef
    w = W.melted_cavity(64)
    params = dict(w.params)
    params.update(T_s=0.1, T_l=0.4)
    tw = 1.0 + 0.1 * np.sin(2 * np.pi * np.arange(w.ny) / w.ny)
    steps = 100

    def J(K=None, t=None):
        o = oracle_mod.Oracle(w.nx, w.ny, **params)
        o.set_fields(w.phi, w.K if K is None else K, w.T0, w.fl0, tw if t is None else t)
        acc = 0.0
        for _ in range(steps):
            o.step(1)
            acc += o.reduce()["nu_hot"]
        return acc / steps

    _, _, d_lnK, d_tw = CoupledRef(w.nx, w.ny, params).gradients(
        steps, w.T0, w.fl0, w.phi, w.K, tw, "nusselt")
    h = 1e-6
    for yy, xx in ((3, 4), (10, 5)):
        Kp, Km = w.K.copy(), w.K.copy()
        Kp[yy, xx] *= np.exp(h)
        Km[yy, xx] *= np.exp(-h)
        fd = (J(K=Kp) - J(K=Km)) / (2 * h)
        assert abs(fd) > 1e-7
        assert abs(d_lnK[yy, xx] - fd) <= 2e-3 * abs(fd) + 5e-9, (yy, xx, d_lnK[yy, xx], fd)
    tp, tm = tw.copy(), tw.copy()
    tp[20] += h
    tm[20] -= h
    fd = (J(t=tp) - J(t=tm)) / (2 * h)
    assert abs(d_tw[20] - fd) <= 2e-3 * abs(fd) + 5e-9, (d_tw[20], fd)
    assert (np.abs(d_lnK) > 0).sum() > 500
