"""The CUDA adjoint of the coupled step (flow on) against the FP64 reference
and against finite differences of the FP64 oracle.

lbm_adjoint_coupled differentiates the melted fraction, or the hot-wall
Nusselt number averaged over the steps, with respect to porosity, ln K and
the left wall profile; oracle/coupled_ref.py differentiates the same map by
autograd and is pinned to finite differences of the C oracle.  The GPU runs
in FP32: its gradients are held to 1e-3 of the largest entry of the FP64
reference's (normwise), and, at sampled cells, to central
differences of the oracle's objective with h = 1e-4.

Memory schedules: keeping every state, and keeping one every K steps with
each segment recomputed from a CUDA graph, give the same bits.
"""
import numpy as np
import pytest

import lbm_workloads as W

pytestmark = pytest.mark.gpu

STEPS = 40
TOL = 1e-3


def _f32(w):
    for k in ("phi", "K", "T0", "fl0"):
        setattr(w, k, getattr(w, k).astype(np.float32).astype(np.float64))
    if w.wall_T_left is not None:
        w.wall_T_left = w.wall_T_left.astype(np.float32).astype(np.float64)
    return w


def _case():
    w = W.melted_cavity(24)
    params = dict(w.params)
    params.update(T_s=0.1, T_l=0.4)
    w.wall_T_left = 1.0 + 0.1 * np.sin(2 * np.pi * np.arange(w.ny) / w.ny)
    w.params = params
    return _f32(w)


def _copy64():
    """The 64^2 copy of the 512^2 inverse-problem cavity (fields block-averaged
    from the large draw), started a quarter melted so that 100 steps move
    the front and the flow."""
    w = W.adjoint_cavity(64, melted=0.25)
    w.wall_T_left = 1.0 + 0.1 * np.sin(2 * np.pi * np.arange(w.ny) / w.ny)
    return _f32(w)


@pytest.fixture(scope="module")
def lbm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1503_08406_gb300 as P
    return P


def _gpu(lbm, w, steps, objective, **kw):
    lat = lbm.Lattice(w.nx, w.ny, **w.params)
    lat.set_fields(w.phi, w.K, w.T0, w.fl0, w.wall_T_left)
    out = lat.adjoint_coupled(steps, objective, **kw)
    assert lat.status() == 0 and lat.steps_done() == steps
    return out


def _check_normwise(got, ref):
    J, dphi, dlnK, dtw = got
    J_ref, dphi_ref, dlnK_ref, dtw_ref = ref
    assert abs(J - J_ref) < 1e-4 * abs(J_ref), (J, J_ref)
    for name, g, e in (("phi", dphi, dphi_ref), ("lnK", dlnK, dlnK_ref), ("Tw", dtw, dtw_ref)):
        scale = np.abs(e).max()
        assert scale > 0
        err = np.abs(np.asarray(g, dtype=np.float64) - e).max() / scale
        assert err < TOL, (name, err)


@pytest.mark.parametrize("objective", ["melt", "nusselt"])
def test_coupled_adjoint_matches_fp64_reference(lbm, oracle_mod, objective):
    from oracle.coupled_ref import CoupledRef
    w = _case()
    ref = CoupledRef(w.nx, w.ny, w.params).gradients(STEPS, w.T0, w.fl0, w.phi, w.K,
                                                     w.wall_T_left, objective)
    _check_normwise(_gpu(lbm, w, STEPS, objective), ref)


@pytest.mark.parametrize("objective", ["melt", "nusselt"])
def test_coupled_adjoint_64_copy_matches_fp64_reference(lbm, oracle_mod, objective):
    from oracle.coupled_ref import CoupledRef
    w = _copy64()
    steps = 100
    ref = CoupledRef(w.nx, w.ny, w.params).gradients(steps, w.T0, w.fl0, w.phi, w.K,
                                                     w.wall_T_left, objective)
    _check_normwise(_gpu(lbm, w, steps, objective, checkpoint_every=10), ref)


def test_coupled_adjoint_64_copy_300_steps(lbm, oracle_mod):
    """The 64^2 copy started solid (subcooled to T_s - 0.05) with only the hot
    wall column melted, 300 steps: the gradients stay within 1e-3 of the FP64
    reference's (with the solid held at T_s itself, FP32 rounding put solid
    nodes on the mushy side of the clamp's kink, and the linearised step grew
    without bound)."""
    from oracle.coupled_ref import CoupledRef
    w = _f32(W.adjoint_cavity(64))
    steps = 300
    ref = CoupledRef(w.nx, w.ny, w.params).gradients(steps, w.T0, w.fl0, w.phi, w.K,
                                                     w.wall_T_left, "melt")
    _check_normwise(_gpu(lbm, w, steps, "melt"), ref)


def test_coupled_adjoint_long_run_matches_differences(lbm):
    """128^2 copy of the inverse-problem cavity, 4,000 steps (the front about
    ten cells from the hot wall, flow on behind it): dJ/dphi of the melted
    fraction at the largest entry and at front cells equals central
    differences of the GPU forward run, on the cells where the differences
    at h = 1e-3 and 1e-2 agree within 1% (the objective is smooth there),
    within 1e-3 of the gradient's largest entry plus the two differences'
    gap."""
    w = _f32(W.adjoint_cavity(128))
    steps = 4000
    lat = lbm.Lattice(w.nx, w.ny, **w.params)
    lat.set_fields(w.phi, w.K, w.T0, w.fl0, w.wall_T_left)
    J0, dphi, dlnK, dtw = lat.adjoint_coupled(steps, "melt")
    assert lat.status() == 0
    for gr in (dphi, dlnK, dtw):
        assert np.all(np.isfinite(gr))
    fl = lat.macros()["fl"]
    scale = np.abs(dphi).max()
    rng = np.random.default_rng(3)
    front = np.argwhere((fl > 0.05) & (fl < 0.95))
    cells = [np.unravel_index(np.argmax(np.abs(dphi)), dphi.shape)]
    cells += [tuple(front[k]) for k in rng.choice(len(front), size=6, replace=False)]

    def J(phi):
        lat.set_fields(phi, w.K, w.T0, w.fl0, w.wall_T_left)
        lat.step(steps)
        return lat.reduce()["melt_frac"]

    checked = 0
    for (y, x) in cells:
        fd = []
        for h in (1e-3, 1e-2):
            p = w.phi.copy()
            p[y, x] += h
            a = J(p)
            p[y, x] -= 2 * h
            fd.append((a - J(p)) / (2 * h))
        gap = abs(fd[0] - fd[1])
        if gap > 0.01 * max(abs(fd[0]), 1e-3 * scale):
            continue
        checked += 1
        assert abs(dphi[y, x] - fd[0]) <= 1e-3 * scale + gap, ((y, x), dphi[y, x], fd)
    assert checked >= 3, checked


def test_checkpointed_schedule_gives_the_same_bits(lbm):
    w = _f32(W.melted_cavity(48))
    w.params = {**w.params, "T_s": 0.1, "T_l": 0.4}
    for objective in ("melt", "nusselt"):
        full = _gpu(lbm, w, 61, objective, checkpoint_every=0)
        for K in (7, 8, 61):
            seg = _gpu(lbm, w, 61, objective, checkpoint_every=K)
            assert full[0] == seg[0], (objective, K)
            for a, b in zip(full[1:], seg[1:]):
                assert np.array_equal(a, b), (objective, K)


def test_device_gradients_equal_host_gradients(lbm):
    import torch
    w = _case()
    host = _gpu(lbm, w, 20, "melt")
    dev = _gpu(lbm, w, 20, "melt", device=True)
    assert host[0] == dev[0]
    for a, b in zip(host[1:], dev[1:]):
        assert isinstance(b, torch.Tensor) and b.is_cuda
        assert np.array_equal(a, b.cpu().numpy())


def test_coupled_objective_autograd_on_device(lbm):
    """CoupledObjective with CUDA tensors: gradients land on the device and
    equal the adjoint's."""
    import torch
    from paper_1503_08406_gb300.autograd import CoupledObjective
    w = _case()
    lat = lbm.Lattice(w.nx, w.ny, **w.params)
    phi = torch.tensor(w.phi, dtype=torch.float32, device="cuda", requires_grad=True)
    lnK = torch.tensor(np.log(w.K), dtype=torch.float32, device="cuda", requires_grad=True)
    tw = torch.tensor(w.wall_T_left, dtype=torch.float32, device="cuda", requires_grad=True)
    J = CoupledObjective.apply(phi, lnK, tw, lat, w.T0, w.fl0, 20, "nusselt")
    J.backward()
    assert phi.grad.is_cuda and lnK.grad.is_cuda and tw.grad.is_cuda
    lat2 = lbm.Lattice(w.nx, w.ny, **w.params)
    lat2.set_fields(phi.detach(), torch.exp(lnK.detach()), w.T0, w.fl0, tw.detach())
    J2, dphi, dlnK, dtw = lat2.adjoint_coupled(20, "nusselt")
    assert abs(J.item() - J2) <= 1e-12 * abs(J2)
    np.testing.assert_array_equal(phi.grad.cpu().numpy(), dphi)
    np.testing.assert_array_equal(lnK.grad.cpu().numpy(), dlnK)
    np.testing.assert_array_equal(tw.grad.cpu().numpy(), dtw)


def _oracle_objective(oracle_mod, w, steps, objective, phi=None, K=None, tw=None):
    o = oracle_mod.Oracle(w.nx, w.ny, **{**w.params, "inner_tol": 1e-13})
    o.set_fields(w.phi if phi is None else phi, w.K if K is None else K, w.T0, w.fl0,
                 w.wall_T_left if tw is None else tw)
    if objective == "melt":
        o.step(steps)
        return o.reduce()["melt_frac"]
    acc = 0.0
    for _ in range(steps):
        o.step(1)
        acc += o.reduce()["nu_hot"]
    return acc / steps


@pytest.mark.parametrize("objective", ["melt", "nusselt"])
def test_coupled_adjoint_matches_oracle_finite_differences(lbm, oracle_mod, objective):
    """Central differences of the FP64 oracle's objective, h = 1e-4 (in phi,
    ln K and the wall profile), at 16 seeded cells away from the clamps (f_l
    after the run in (0.05, 0.95), or liquid at least 0.05 above T_l) whose gradient
    is at least 5% of the field's largest (an FP32 gradient carries an
    absolute error of ~1e-5 of the largest entry, so smaller entries cannot be
    held to 1e-3 of themselves), and at 4 wall rows, after 400 steps.  Each
    difference is taken at h and 2h: their gap is the difference's own noise
    (the objective's FP64 rounding over the run against a change of 2 h |dJ| -- large for the
    melted fraction's tiny ln K and wall gradients), which the bar adds to
    1e-3 relative."""
    w = _copy64()
    steps = 400   # the subcooled front melts a column at a time: mushy cells by then
    J, dphi, dlnK, dtw = _gpu(lbm, w, steps, objective)
    o = oracle_mod.Oracle(w.nx, w.ny, **w.params)
    o.set_fields(w.phi, w.K, w.T0, w.fl0, w.wall_T_left)
    o.step(steps)
    mac = o.macros()
    fl_end = mac["fl"]
    # away from the clamp kinks: the front (0.05 < f_l < 0.95) and the liquid
    # well above T_l (where the Nusselt number's gradient sits)
    smooth = ((fl_end > 0.05) & (fl_end < 0.95)) | \
        ((fl_end == 1.0) & (mac["T"] >= w.params["T_l"] + 0.05))
    rng = np.random.default_rng(12)
    h = 1e-4

    def cd(name, y, x, hh):
        vals = []
        for sgn in (1, -1):
            if name == "phi":
                p = w.phi.copy()
                p[y, x] += sgn * hh
                vals.append(_oracle_objective(oracle_mod, w, steps, objective, phi=p))
            elif name == "lnK":
                K = w.K.copy()
                K[y, x] *= np.exp(sgn * hh)
                vals.append(_oracle_objective(oracle_mod, w, steps, objective, K=K))
            else:
                tw = w.wall_T_left.copy()
                tw[y] += sgn * hh
                vals.append(_oracle_objective(oracle_mod, w, steps, objective, tw=tw))
        return (vals[0] - vals[1]) / (2 * hh)

    worst, checked = {}, {}
    for name, grad in (("phi", dphi), ("lnK", dlnK)):
        big = np.abs(grad) >= 0.05 * np.abs(grad).max()
        cand = np.argwhere(smooth & big)
        assert len(cand) >= 8, (name, len(cand))
        cells = cand[rng.choice(len(cand), size=min(16, len(cand)), replace=False)]
        for (y, x) in cells:
            fd1, fd2 = cd(name, y, x, h), cd(name, y, x, 2 * h)
            err = (abs(grad[y, x] - fd1) - 2 * abs(fd1 - fd2)) / abs(fd1)
            worst[name] = max(worst.get(name, -1.0), err)
        checked[name] = len(cells)
    for y in rng.choice(np.arange(1, w.ny - 1), size=4, replace=False):
        fd1, fd2 = cd("Tw", y, 0, h), cd("Tw", y, 0, 2 * h)
        err = (abs(dtw[y] - fd1) - 2 * abs(fd1 - fd2)) / abs(fd1)
        worst["Tw"] = max(worst.get("Tw", -1.0), err)
    print("cells checked", checked, "worst gap beyond the differences' noise, relative:", worst)
    for name, err in worst.items():
        assert err < TOL, (name, err, worst)


@pytest.mark.parametrize("which,objective", [("slab_alpha10", "melt"),
                                             ("slab_alpha10", "nusselt"),
                                             ("cavity_alpha3", "melt")])
def test_coupled_adjoint_with_phase_dependent_diffusivity(lbm, oracle_mod, which, objective):
    """alpha_l != alpha_s (Sec. 4.1: the flux moments' rate follows f_l(n)):
    the Sec. 4.1 slab with alpha_l = 10 alpha_s and the flow lattice off, and
    the melting cavity with alpha_l = 3 alpha_s, against the FP64 reference."""
    from oracle.coupled_ref import CoupledRef
    if which == "slab_alpha10":
        w = W.adjoint_slab(40, 4)
        w.params = {**w.params, "alpha_ratio": 10.0, "tau_T": 0.5 + 10 * 0.02 / 0.2}
        steps = 200
    else:
        w = _case()
        w.params = {**w.params, "alpha_ratio": 3.0}
        steps = STEPS
    w = _f32(w)
    ref = CoupledRef(w.nx, w.ny, w.params).gradients(steps, w.T0, w.fl0, w.phi, w.K,
                                                     w.wall_T_left, objective)
    got = _gpu(lbm, w, steps, objective)
    J, dphi, dlnK, dtw = got
    J_ref, dphi_ref, dlnK_ref, dtw_ref = ref
    assert abs(J - J_ref) < 1e-4 * abs(J_ref), (J, J_ref)
    for name, g, e in (("phi", dphi, dphi_ref), ("Tw", dtw, dtw_ref)):
        scale = np.abs(e).max()
        assert np.abs(np.asarray(g, dtype=np.float64) - e).max() < TOL * scale, name
    if w.params.get("flow", 1):
        scale = np.abs(dlnK_ref).max()
        assert np.abs(np.asarray(dlnK, dtype=np.float64) - dlnK_ref).max() < TOL * scale
    else:
        assert np.abs(dlnK).max() == 0   # no flow: the permeability plays no part


def test_adjoint_phase_timing(lbm):
    w = _case()
    lat = lbm.Lattice(w.nx, w.ny, **w.params)
    assert lat.adjoint_timing() == (0.0, 0.0)
    lat.set_fields(w.phi, w.K, w.T0, w.fl0, w.wall_T_left)
    lat.adjoint_coupled(20, "melt", checkpoint_every=5)
    fwd, rev = lat.adjoint_timing()
    assert fwd > 0 and rev > 0
