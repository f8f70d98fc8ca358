"""The flow collision's adjoint written for the reverse-sweep kernels
(paper_1503_08406_gb300/csrc/lbm_flow_adjoint.cuh), built for the host in
float64 and checked against the FP64 reference (oracle/coupled_ref.py): its
forward map equals the reference's collision, and its vector-Jacobian
product equals torch.autograd's through that collision, on random nodes
(liquid fractions from near f_act to 1, speeds from rest to the lattice's
usual range, porosity, permeability and temperature spread)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import lbm_workloads as W

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1503_08406_gb300", "csrc")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("flowadj") / "libflowadj.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, "-o", out,
                    os.path.join(HERE, "native", "flow_adjoint_host.cpp")], check=True)
    return ctypes.CDLL(out)


def _P(a):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(ctypes.c_void_p)


def _nodes(n, seed):
    rng = np.random.default_rng(seed)
    w9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    rho = 1 + 0.01 * rng.standard_normal(n)
    u = 0.02 * rng.standard_normal((2, n)) * (rng.random(n) > 0.1)   # some at rest
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    eu = ex[:, None] * u[0] + ey[:, None] * u[1]
    f = w9[:, None] * (rho + 3 * eu + 4.5 * eu ** 2 - 1.5 * (u ** 2).sum(0))
    f += 1e-4 * rng.standard_normal(f.shape)
    T = rng.uniform(-0.5, 1.5, n)
    fl = np.concatenate([[1.0, 1e-3 * 1.01], rng.uniform(0.002, 1.0, n - 2)])
    phi = rng.uniform(0.3, 0.7, n)
    K = np.exp(rng.uniform(np.log(0.1), np.log(1e3), n))
    return f, T, fl, phi, K


def _ref():
    from oracle.coupled_ref import CoupledRef
    w = W.melted_cavity(24)
    return CoupledRef(w.nx, w.ny, w.params)


def _prm(ref):
    return np.concatenate([[ref.rho0, ref.nu_l, ref.g_beta, ref.T_ref], ref.lam.numpy(),
                           [1e-300]])


def test_forward_equals_reference_collision(lib):
    ref = _ref()
    n = 256
    f, T, fl, phi, K = _nodes(n, 0)
    fpost, ux, uy = np.zeros((n, 9)), np.zeros(n), np.zeros(n)
    lib.flow_collide_f64(_P(_prm(ref)), n, _P(f.T.copy()), _P(T), _P(fl), _P(phi), _P(K),
                         fpost.ctypes.data_as(ctypes.c_void_p), ux.ctypes.data_as(ctypes.c_void_p),
                         uy.ctypes.data_as(ctypes.c_void_p))
    t = lambda a: torch.tensor(a, dtype=torch.float64)
    fp_r, ux_r, uy_r = ref.collide_flow(t(f), t(T), t(fl), t(phi), t(K))
    assert np.abs(fpost.T - fp_r.numpy()).max() < 1e-13
    assert np.abs(ux - ux_r.numpy()).max() < 1e-15 and np.abs(uy - uy_r.numpy()).max() < 1e-15


def test_adjoint_equals_autograd(lib):
    ref = _ref()
    n = 256
    f, T, fl, phi, K = _nodes(n, 1)
    rng = np.random.default_rng(2)
    lf = rng.standard_normal((n, 9))
    lux, luy = rng.standard_normal(n), rng.standard_normal(n)
    outs = {k: np.zeros(s) for k, s in (("lfin", (n, 9)), ("lT", n), ("lfl", n), ("lphi", n),
                                         ("lK", n))}
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    lib.flow_adjoint_f64(_P(_prm(ref)), n, _P(f.T.copy()), _P(T), _P(fl), _P(phi), _P(K),
                         _P(lf), _P(lux), _P(luy), vp(outs["lfin"]), vp(outs["lT"]),
                         vp(outs["lfl"]), vp(outs["lphi"]), vp(outs["lK"]))
    ins = [torch.tensor(a, dtype=torch.float64, requires_grad=True) for a in (f, T, fl, phi, K)]
    fp, ux, uy = ref.collide_flow(*ins)
    J = (torch.tensor(lf.T) * fp).sum() + (torch.tensor(lux) * ux).sum() + \
        (torch.tensor(luy) * uy).sum()
    g = torch.autograd.grad(J, ins)
    exp = {"lfin": g[0].numpy().T, "lT": g[1].numpy(), "lfl": g[2].numpy(),
           "lphi": g[3].numpy(), "lK": g[4].numpy()}
    for k in exp:
        scale = np.abs(exp[k]).max()
        err = np.abs(outs[k] - exp[k]).max() / scale
        assert err < 1e-11, (k, err, scale)


def _tprm(ref):
    return np.concatenate([[ref.sigma, ref.csT2, ref.varpi], ref.theta.numpy(),
                           [ref.w5[0].item(), ref.w5[1].item()]])


def _thermal_nodes(n, seed):
    rng = np.random.default_rng(seed)
    g = np.array([0.6] + [0.1] * 4)[:, None] * rng.uniform(-0.5, 1.5, n) \
        + 0.01 * rng.standard_normal((5, n))
    ux, uy = 0.03 * rng.standard_normal(n), 0.03 * rng.standard_normal(n)
    return g, ux, uy


def test_thermal_collision_and_its_adjoint(lib):
    ref = _ref()
    n = 256
    g, ux, uy = _thermal_nodes(n, 3)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    gpost = np.zeros((n, 5))
    lib.thermal_collide_f64(_P(_tprm(ref)), n, _P(g.T.copy()), _P(ux), _P(uy), vp(gpost))
    ins = [torch.tensor(a, dtype=torch.float64, requires_grad=True) for a in (g, ux, uy)]
    gp = ref.collide_thermal(*ins)
    assert np.abs(gpost.T - gp.detach().numpy()).max() < 1e-14
    lg = np.random.default_rng(4).standard_normal((n, 5))
    lgin, lux, luy = np.zeros((n, 5)), np.zeros(n), np.zeros(n)
    lib.thermal_adjoint_f64(_P(_tprm(ref)), n, _P(g.T.copy()), _P(ux), _P(uy), _P(lg), vp(lgin),
                            vp(lux), vp(luy))
    d = torch.autograd.grad((torch.tensor(lg.T) * gp).sum(), ins)
    for got, exp in ((lgin.T, d[0]), (lux, d[1]), (luy, d[2])):
        exp = exp.numpy()
        assert np.abs(got - exp).max() < 1e-12 * np.abs(exp).max()


def test_wall_extrapolation_adjoint(lib):
    ref = _ref()
    n = 128
    g, ux, uy = _thermal_nodes(n, 5)
    Tw = np.random.default_rng(6).uniform(0, 1, n)
    lgb = np.random.default_rng(7).standard_normal((n, 5))
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    lgf, lTw, lux, luy = np.zeros((n, 5)), np.zeros(n), np.zeros(n), np.zeros(n)
    lib.wall_adjoint_f64(_P(_tprm(ref)), n, _P(g.T.copy()), _P(ux), _P(uy), _P(lgb), vp(lgf),
                         vp(lTw), vp(lux), vp(luy))
    ins = [torch.tensor(a, dtype=torch.float64, requires_grad=True) for a in (g, Tw, ux, uy)]
    gb = ref.extrapolate_wall(ins[0], ins[1], ins[2], ins[3])
    d = torch.autograd.grad((torch.tensor(lgb.T) * gb).sum(), ins)
    for got, exp in ((lgf.T, d[0]), (lTw, d[1]), (lux, d[2]), (luy, d[3])):
        exp = exp.numpy()
        assert np.abs(got - exp).max() < 1e-12 * np.abs(exp).max()


@pytest.fixture(scope="module")
def rev(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("coupledrev") / "libcoupledrev.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, "-o", out,
                    os.path.join(HERE, "native", "coupled_reverse_host.cpp")], check=True)
    return ctypes.CDLL(out)


def _geometry(which):
    """(workload, params, wall profile) of a test geometry: a walled melting
    cavity, the same fields in a channel (periodic in y, adiabatic right
    wall) and a doubly periodic box."""
    if which == "box":
        w = W.periodic_box(16, flow=1, T_s=-0.1, T_l=0.1)
        return w, dict(w.params), np.zeros(w.ny)
    if which == "twophase":   # Sec. 4.1 slab, alpha_l = 10 alpha_s, flow off
        w = W.adjoint_slab(40, 4)
        params = dict(w.params)
        params["alpha_ratio"] = 10.0
        params["tau_T"] = 0.5 + 10 * 0.02 / 0.2
        return w, params, w.wall_T_left
    w = W.melted_cavity(24)
    params = dict(w.params)
    params.update(T_s=0.1, T_l=0.4)
    if which == "channel":
        params["bc"] = ("dirichlet", "adiabatic", "periodic", "periodic")
    if which == "cavity_alpha":
        params["alpha_ratio"] = 3.0
    tw = 1.0 + 0.1 * np.sin(2 * np.pi * np.arange(w.ny) / w.ny)
    return w, params, tw


@pytest.mark.parametrize("which,objective", [("cavity", "melt"), ("cavity", "nusselt"),
                                             ("channel", "melt"), ("channel", "nusselt"),
                                             ("box", "melt"), ("twophase", "melt"),
                                             ("twophase", "nusselt"), ("cavity_alpha", "melt")])
def test_reverse_sweep_from_node_functions_equals_autograd(rev, which, objective):
    """The reverse sweep of the coupled step from lbm::coupled_reverse_node, the
    reverse-sweep kernel's body (run over every node on the host, after a
    Jacobi solve of the fixed point's adjoint on the band, by
    tests/native/coupled_reverse_host.cpp), over 40 steps: the gradients in
    ln K, phi and the wall profile equal autograd of the FP64 reference, on a
    walled cavity, a channel periodic in y, a doubly periodic box, the
    Sec. 4.1 slab with alpha_l = 10 alpha_s (flow off) and the cavity with
    alpha_l = 3 alpha_s."""
    from oracle.coupled_ref import BC, CoupledRef
    w, params, tw = _geometry(which)
    steps = 40
    ref = CoupledRef(w.nx, w.ny, params)
    J, d_phi, d_lnK, d_tw = ref.gradients(steps, w.T0, w.fl0, w.phi, w.K, tw, objective)
    t = lambda a: torch.tensor(a, dtype=torch.float64)
    f, g, fl = ref.initial(w.T0, w.fl0)
    states = []
    for _ in range(steps):
        states.append((f.numpy().copy(), g.numpy().copy(), fl.numpy().copy()))
        f, g, fl = ref.step(f, g, fl, t(w.phi), t(w.K), t(tw))
    states.append((f.numpy().copy(), g.numpy().copy(), fl.numpy().copy()))
    n = w.nx * w.ny
    wall = ref.wall.numpy()
    lf, lg, lfl = np.zeros(9 * n), np.zeros(5 * n), np.zeros(n)
    lphi, lK, lTw = np.zeros(n), np.zeros(n), np.zeros(w.ny)
    bcv = [BC[b] if isinstance(b, str) else int(b) for b in params["bc"]]
    per_x, per_y = int(bcv[0] == 0), int(bcv[2] == 0)
    nuprm = np.zeros(8)
    nuprm[7] = ref.flow
    if ref.alpha_ratio is not None:
        nuprm[5], nuprm[6] = ref.tau_T, 1.0 / ref.alpha_ratio
    if objective == "melt":
        lfl[:] = np.where(wall.ravel(), 0.0, 1.0 / (~wall).sum())
    else:
        # Nu = -(-3 T_w + 4 T_1 - T_2)/2 H/dT over the rows without a
        # horizontal wall, after each step, averaged: its terms per state; those
        # of the last state seed the sweep, each reversed step adds those of
        # the state before it (the wall term for the states 0..N-1: the same
        # constant N times)
        y0, y1 = (0, w.ny) if per_y else (1, w.ny - 1)
        k = ref.H / (ref.dT * (y1 - y0) * steps)
        nuprm[:5] = (-2 * k, 0.5 * k, 1.5 * k, y0, y1)
        src = np.zeros((w.ny, w.nx))
        src[y0:y1, 1] = -2 * k
        src[y0:y1, 2] = 0.5 * k
        lg += np.tile(src.ravel(), 5)
    bc = (ctypes.c_int * 4)(*bcv)
    fprm = np.concatenate([[ref.rho0, ref.nu_l, ref.g_beta, ref.T_ref], ref.lam.numpy(), [1e-300]])
    tprm = np.concatenate([[ref.sigma, ref.csT2, ref.varpi], ref.theta.numpy(),
                           [ref.w5[0].item(), ref.w5[1].item()]])
    sc = np.array([ref.f_act, ref.T_s, ref.T_l, ref.lat])
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    phi, K = np.ascontiguousarray(w.phi.ravel()), np.ascontiguousarray(w.K.ravel())
    for m in range(steps - 1, -1, -1):
        f0, g0, fl0 = states[m]
        fl1 = states[m + 1][2]
        rev.coupled_reverse_step_f64(w.nx, w.ny, per_x, per_y, bc, _P(fprm), _P(tprm), _P(sc),
                                     _P(nuprm), _P(f0.ravel()), _P(g0.ravel()),
                                     _P(fl0.ravel()), _P(fl1.ravel()), _P(phi), _P(K), vp(lf),
                                     vp(lg), vp(lfl), vp(lphi), vp(lK), vp(lTw))
    got = {"phi": lphi.reshape(w.ny, w.nx), "lnK": (lK * K).reshape(w.ny, w.nx), "tw": lTw}
    exp = {"phi": d_phi, "lnK": d_lnK, "tw": d_tw}
    for k in exp:
        scale = np.abs(exp[k]).max()
        if (which == "box" and k == "tw") or (which == "twophase" and k == "lnK"):
            assert scale == 0 and np.abs(got[k]).max() == 0   # no wall / no flow
            continue
        assert scale > 0, k
        err = np.abs(got[k] - exp[k]).max() / scale
        assert err < 1e-9, (k, err, scale)
