"""FP64 CPU oracle for the double-MRT phase-change LBM (Liu & He, arXiv:1503.08406).

TEST INFRASTRUCTURE ONLY.  ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers.  The product path (``paper_1503_08406_gb300``) never imports this
module, and this module never imports the product: they share no code.

The arithmetic lives in ``lbm_oracle.c`` (plain C, double precision, compiled
with gcc by :func:`build`).  This file only marshals arguments through ctypes.

Pinned by ``tests/test_oracle_*.py``: matrix identities of Eq. (18), (32);
equilibrium and forcing moments, Eq. (19), (22), (29), (34), (39); the
velocity solve, Eq. (25)-(28); the BGK limit stated in Sec. 3.1; closed-form
uniform Darcy-Forchheimer and Brinkman-channel flows; mass and enthalpy
conservation; the one-phase Neumann solution, Eq. (43) with Eq. (46); the
corner-solidification symmetry and far-field 1-D Neumann front (Sec. 4.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "liblbm_oracle.so")

BC = {"periodic": 0, "dirichlet": 1, "adiabatic": 2}
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile lbm_oracle.c into oracle/_build/liblbm_oracle.so with gcc."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                               os.path.getmtime(os.path.join(_HERE, "lbm_oracle.h")))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
           "-std=c11", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("bc", ctypes.c_int32 * 4), ("T_bc", ctypes.c_double * 4),
        ("flow", ctypes.c_int32),
        ("Ra", ctypes.c_double), ("Pr", ctypes.c_double), ("Ma", ctypes.c_double),
        ("J", ctypes.c_double), ("lambda_", ctypes.c_double), ("sigma", ctypes.c_double),
        ("St", ctypes.c_double), ("dT", ctypes.c_double), ("H", ctypes.c_double),
        ("T_ref", ctypes.c_double), ("T_s", ctypes.c_double), ("T_l", ctypes.c_double),
        ("varpi", ctypes.c_double), ("rho0", ctypes.c_double),
        ("tau_nu", ctypes.c_double), ("tau_T", ctypes.c_double), ("g_beta", ctypes.c_double),
        ("s_e", ctypes.c_double), ("s_eps", ctypes.c_double), ("s_q", ctypes.c_double),
        ("zeta_e", ctypes.c_double), ("zeta_nu", ctypes.c_double),
        ("f_act", ctypes.c_double),
        ("max_inner_iters", ctypes.c_int32), ("inner_tol", ctypes.c_double),
        ("alpha_ratio", ctypes.c_double), ("sigma_solid", ctypes.c_double),
        ("flow_walls", ctypes.c_int32), ("flow_front", ctypes.c_int32),
    ]


_D = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            vp = ctypes.c_void_p
            lib.ora_create.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(vp)]
            lib.ora_destroy.argtypes = [vp]
            lib.ora_set_threads.argtypes = [ctypes.c_int]
            lib.ora_get_derived.argtypes = [vp, _D]
            lib.ora_set_fields.argtypes = [vp, _D, _D, _D, _D, _D]
            lib.ora_step.argtypes = [vp, ctypes.c_int64, ctypes.c_int]
            lib.ora_inner_iterations.argtypes = [vp]
            lib.ora_inner_iterations.restype = ctypes.c_int64
            lib.ora_get_macros.argtypes = [vp, _D, _D, _D, _D, _D]
            lib.ora_reduce.argtypes = [vp, _D]
            lib.ora_get_state.argtypes = [vp, _D, _D, _D]
            lib.ora_set_state.argtypes = [vp, _D, _D, _D]
            lib.ora_matrices.argtypes = [_D, _D, _D, _D]
            for name in ("ora_feq", "ora_meq"):
                getattr(lib, name).argtypes = [vp] + [ctypes.c_double] * 4 + [_D]
            lib.ora_force_moments.argtypes = [vp] + [ctypes.c_double] * 5 + [_D]
            lib.ora_geq.argtypes = [vp] + [ctypes.c_double] * 3 + [_D]
            lib.ora_thermal_meq.argtypes = [vp] + [ctypes.c_double] * 3 + [_D]
            lib.ora_velocity.argtypes = [vp, _D] + [ctypes.c_double] * 4 + [_D]
            lib.ora_collide_flow.argtypes = [vp, _D] + [ctypes.c_double] * 4 + [_D]
            lib.ora_theta_T.argtypes = [vp, ctypes.c_double]
            lib.ora_theta_T.restype = ctypes.c_double
            lib.ora_collide_thermal.argtypes = [vp, _D] + [ctypes.c_double] * 3 + [_D]
            _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


DEFAULTS = dict(
    bc=("dirichlet", "dirichlet", "adiabatic", "adiabatic"), T_bc=(1.0, 0.0, 0.0, 0.0),
    flow=1, Ra=0.0, Pr=0.0, Ma=0.1, J=1.0, lambda_=1.0, sigma=1.0, St=1.0, dT=1.0, H=0.0,
    T_ref=0.0, T_s=0.0, T_l=0.0, varpi=-2.0, rho0=1.0, tau_nu=-1.0, tau_T=-1.0, g_beta=-1.0,
    s_e=0.0, s_eps=0.0, s_q=0.0, zeta_e=0.0, zeta_nu=0.0, f_act=1e-3,
    max_inner_iters=1000, inner_tol=1e-13, alpha_ratio=0.0, sigma_solid=0.0,
    flow_walls=0, flow_front=0,
)


def make_params(nx: int, ny: int, **kw) -> _Params:
    d = dict(DEFAULTS)
    unknown = set(kw) - set(d)
    if unknown:
        raise KeyError(f"unknown oracle parameters: {sorted(unknown)}")
    d.update(kw)
    p = _Params()
    p.nx, p.ny = nx, ny
    for i, b in enumerate(d.pop("bc")):
        p.bc[i] = BC[b] if isinstance(b, str) else int(b)
    for i, t in enumerate(d.pop("T_bc")):
        p.T_bc[i] = float(t)
    for k, v in d.items():
        setattr(p, k, v)
    return p


class OracleError(RuntimeError):
    pass


class Oracle:
    """One lattice (flow + thermal) held by the C oracle."""

    def __init__(self, nx: int, ny: int, threads: int | None = None, **params):
        self.lib = _load()
        self.nx, self.ny = nx, ny
        self.n = nx * ny
        self._h = ctypes.c_void_p()
        rc = self.lib.ora_create(ctypes.byref(make_params(nx, ny, **params)), ctypes.byref(self._h))
        if rc != 0:
            raise OracleError(f"ora_create failed ({rc})")
        if threads:
            self.lib.ora_set_threads(int(threads))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self.lib.ora_destroy(h)
            self._h = ctypes.c_void_p()

    def theta_T(self, fl: float) -> float:
        """Thermal relaxation rate 1/tau_T at liquid fraction fl (Sec. 4.1)."""
        return float(self.lib.ora_theta_T(self._h, float(fl)))

    def derived(self) -> dict:
        out = np.zeros(8)
        self.lib.ora_get_derived(self._h, _ptr(out))
        keys = ("tau_nu", "tau_T", "nu_e", "nu_l", "alpha_e", "g_beta", "csT2", "lat")
        return dict(zip(keys, out.tolist()))

    def set_fields(self, phi, K, T0, fl0, wall_T_left=None):
        n = self.n
        arrs = [_f64(a, n) for a in (phi, K, T0, fl0)]
        wt = None if wall_T_left is None else _f64(wall_T_left, self.ny)
        rc = self.lib.ora_set_fields(self._h, *[_ptr(a) for a in arrs], _ptr(wt))
        if rc != 0:
            raise OracleError(f"ora_set_fields failed ({rc})")

    def step(self, nsteps: int = 1, literal: bool = False, check: bool = True) -> int:
        rc = self.lib.ora_step(self._h, int(nsteps), int(bool(literal)))
        if check and rc != 0:
            raise OracleError(f"ora_step failed ({rc})")
        return rc

    def inner_iterations(self) -> int:
        return int(self.lib.ora_inner_iterations(self._h))

    def macros(self) -> dict:
        outs = {k: np.zeros(self.n) for k in ("ux", "uy", "rho", "T", "fl")}
        self.lib.ora_get_macros(self._h, *[_ptr(outs[k]) for k in ("ux", "uy", "rho", "T", "fl")])
        return {k: v.reshape(self.ny, self.nx) for k, v in outs.items()}

    def reduce(self) -> dict:
        out = np.zeros(4)
        self.lib.ora_reduce(self._h, _ptr(out))
        return dict(zip(("mass", "enthalpy", "melt_frac", "nu_hot"), out.tolist()))

    def get_state(self):
        f = np.zeros((9, self.ny, self.nx))
        g = np.zeros((5, self.ny, self.nx))
        fl = np.zeros((self.ny, self.nx))
        self.lib.ora_get_state(self._h, _ptr(f), _ptr(g), _ptr(fl))
        return f, g, fl

    def set_state(self, f=None, g=None, fl=None):
        f = None if f is None else _f64(f, 9 * self.n)
        g = None if g is None else _f64(g, 5 * self.n)
        fl = None if fl is None else _f64(fl, self.n)
        self.lib.ora_set_state(self._h, _ptr(f), _ptr(g), _ptr(fl))

    # ---- single-node pieces -------------------------------------------------
    def feq(self, rho, ux, uy, varphi):
        out = np.zeros(9)
        self.lib.ora_feq(self._h, rho, ux, uy, varphi, _ptr(out))
        return out

    def meq(self, rho, ux, uy, varphi):
        out = np.zeros(9)
        self.lib.ora_meq(self._h, rho, ux, uy, varphi, _ptr(out))
        return out

    def force_moments(self, ux, uy, Fx, Fy, varphi):
        out = np.zeros(9)
        self.lib.ora_force_moments(self._h, ux, uy, Fx, Fy, varphi, _ptr(out))
        return out

    def geq(self, T, ux, uy):
        out = np.zeros(5)
        self.lib.ora_geq(self._h, T, ux, uy, _ptr(out))
        return out

    def thermal_meq(self, T, ux, uy):
        out = np.zeros(5)
        self.lib.ora_thermal_meq(self._h, T, ux, uy, _ptr(out))
        return out

    def velocity(self, f, T, fl, phi, K):
        f = _f64(f, 9)
        out = np.zeros(4)
        self.lib.ora_velocity(self._h, _ptr(f), T, fl, phi, K, _ptr(out))
        return out

    def collide_flow(self, f, T, fl, phi, K):
        f = _f64(f, 9)
        out = np.zeros(9)
        self.lib.ora_collide_flow(self._h, _ptr(f), T, fl, phi, K, _ptr(out))
        return out

    def collide_thermal(self, g, ux, uy, src0):
        g = _f64(g, 5)
        out = np.zeros(5)
        self.lib.ora_collide_thermal(self._h, _ptr(g), ux, uy, src0, _ptr(out))
        return out


def matrices():
    lib = _load()
    M, Mi, N, Ni = np.zeros(81), np.zeros(81), np.zeros(25), np.zeros(25)
    lib.ora_matrices(_ptr(M), _ptr(Mi), _ptr(N), _ptr(Ni))
    return M.reshape(9, 9), Mi.reshape(9, 9), N.reshape(5, 5), Ni.reshape(5, 5)
