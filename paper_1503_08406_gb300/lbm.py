"""Python binding of liblbm (include/lbm.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of liblbm.so.  PyTorch supplies device memory (the context workspace and
output tensors) and the CUDA stream.  There is no CPU fallback: if
liblbm.so has not been built, or no GPU is present, the calls raise.

The functions named like the C entry points (``lbm_create`` ...) are one-to-
one wrappers; :class:`Lattice` strings them together for Python users.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblbm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "lbm.h")

LBM_OK = 0
ERRORS = {
    -1: "LBM_ERR_INVALID_ARG", -2: "LBM_ERR_CUDA", -3: "LBM_ERR_NONFINITE",
    -4: "LBM_ERR_NOT_CONVERGED", -5: "LBM_ERR_OOM", -6: "LBM_ERR_NO_DEVICE",
    -7: "LBM_ERR_TIMEOUT",
}
BC = {"periodic": 0, "dirichlet": 1, "adiabatic": 2}


class LBMError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {ERRORS.get(code, code)}")


class lbm_params(ctypes.Structure):
    """Mirror of the C struct lbm_params (include/lbm.h)."""
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
        ("screen_tol", ctypes.c_double),
        ("kernel_variant", ctypes.c_int32),
        ("storage", ctypes.c_int32),
        ("alpha_ratio", ctypes.c_double),
        ("check_every", ctypes.c_int32),
        ("sigma_solid", ctypes.c_double),
        ("flow_walls", ctypes.c_int32),
        ("flow_front", ctypes.c_int32),
    ]


PARAM_DEFAULTS = dict(
    bc=("dirichlet", "dirichlet", "adiabatic", "adiabatic"), T_bc=(1.0, 0.0, 0.0, 0.0),
    flow=1, Ra=0.0, Pr=0.0, Ma=0.1, J=1.0, lambda_=1.0, sigma=1.0, St=1.0, dT=1.0, H=0.0,
    T_ref=0.0, T_s=0.0, T_l=0.0, varpi=-2.0, rho0=1.0, tau_nu=-1.0, tau_T=-1.0, g_beta=-1.0,
    s_e=0.0, s_eps=0.0, s_q=0.0, zeta_e=0.0, zeta_nu=0.0, f_act=1e-3,
    max_inner_iters=1000, inner_tol=1e-6, screen_tol=0.0, kernel_variant=0, storage=0, alpha_ratio=0.0,
    check_every=0, sigma_solid=0.0, flow_walls=0, flow_front=0,
)


STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}


def make_params(nx: int, ny: int, **kw) -> lbm_params:
    d = dict(PARAM_DEFAULTS)
    unknown = set(kw) - set(d)
    if unknown:
        raise KeyError(f"unknown lbm parameters: {sorted(unknown)}")
    d.update(kw)
    p = lbm_params()
    p.nx, p.ny = int(nx), int(ny)
    for i, b in enumerate(d.pop("bc")):
        p.bc[i] = BC[b] if isinstance(b, str) else int(b)
    for i, t in enumerate(d.pop("T_bc")):
        p.T_bc[i] = float(t)
    if isinstance(d.get("storage"), str):
        d["storage"] = STORAGE[d["storage"]]
    for k, v in d.items():
        setattr(p, k, v)
    return p


_lock = threading.Lock()
_lib = None
_VP = ctypes.c_void_p
_FP = ctypes.POINTER(ctypes.c_float)
_DP = ctypes.POINTER(ctypes.c_double)


def declared_functions() -> list[str]:
    """Names of the functions include/lbm.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


def load():
    """Load liblbm.so (built by paper_1503_08406_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER(lbm_params)
        lib.lbm_workspace_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        lib.lbm_create.argtypes = [P, _VP, _VP, ctypes.c_size_t, ctypes.POINTER(_VP)]
        lib.lbm_destroy.argtypes = [_VP]
        lib.lbm_destroy.restype = None
        lib.lbm_derived.argtypes = [_VP, _DP]
        lib.lbm_set_fields.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_int]
        lib.lbm_step.argtypes = [_VP, ctypes.c_int64]
        lib.lbm_prepare.argtypes = [_VP, ctypes.c_int64]
        lib.lbm_check_wait.argtypes = [_VP, ctypes.c_int64]
        lib.lbm_status.argtypes = [_VP]
        lib.lbm_steps_done.argtypes = [_VP]
        lib.lbm_steps_done.restype = ctypes.c_int64
        lib.lbm_kernel_launches.argtypes = [_VP]
        lib.lbm_kernel_launches.restype = ctypes.c_int64
        lib.lbm_kernel_variant.argtypes = [_VP]
        lib.lbm_kernel_variant.restype = ctypes.c_int
        lib.lbm_autotune.argtypes = [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_int32)]
        lib.lbm_adjoint_melt.argtypes = [_VP, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                         _VP, _VP, _DP, ctypes.c_int]
        lib.lbm_adjoint.argtypes = [_VP, ctypes.c_int, ctypes.c_int64, ctypes.c_int32,
                                    ctypes.c_int32, _VP, _VP, _DP, ctypes.c_int]
        lib.lbm_adjoint_coupled.argtypes = [_VP, ctypes.c_int, ctypes.c_int64, ctypes.c_int32,
                                            ctypes.c_int32, _VP, _VP, _VP, _DP, ctypes.c_int]
        lib.lbm_adjoint_timing.argtypes = [_VP, _DP]
        lib.lbm_trace.argtypes = [_VP, ctypes.c_int64]
        lib.lbm_trace_read.argtypes = [_VP, _VP, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
        lib.lbm_batch_create.argtypes = [ctypes.POINTER(_VP), ctypes.c_int, _VP,
                                         ctypes.POINTER(_VP)]
        lib.lbm_batch_step.argtypes = [_VP, ctypes.c_int64]
        lib.lbm_batch_mode.argtypes = [_VP]
        lib.lbm_batch_mode.restype = ctypes.c_int
        lib.lbm_batch_destroy.argtypes = [_VP]
        lib.lbm_batch_destroy.restype = None
        lib.lbm_get_macros.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_int]
        lib.lbm_reduce.argtypes = [_VP, _DP]
        lib.lbm_get_state.argtypes = [_VP, _VP, _VP, _VP, ctypes.c_int]
        lib.lbm_set_state.argtypes = [_VP, _VP, _VP, _VP, ctypes.c_int]
        lib.lbm_timing.argtypes = [_VP, ctypes.c_int]
        lib.lbm_timing_read.argtypes = [_VP, _DP, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]
        lib.lbm_error_string.argtypes = [ctypes.c_int]
        lib.lbm_error_string.restype = ctypes.c_char_p
        _lib = lib
    return _lib


def _check(rc: int, what: str):
    if rc != LBM_OK:
        raise LBMError(rc, what)


# ---- one-to-one wrappers of the C entry points --------------------------------

def lbm_workspace_bytes(params: lbm_params) -> int:
    n = ctypes.c_size_t()
    _check(load().lbm_workspace_bytes(ctypes.byref(params), ctypes.byref(n)), "lbm_workspace_bytes")
    return n.value


def lbm_create(params: lbm_params, stream: int = 0, workspace: int = 0, workspace_bytes: int = 0):
    h = _VP()
    _check(load().lbm_create(ctypes.byref(params), _VP(stream or None), _VP(workspace or None),
                             workspace_bytes, ctypes.byref(h)), "lbm_create")
    return h


def lbm_destroy(h) -> None:
    load().lbm_destroy(h)


def lbm_step(h, nsteps: int) -> None:
    _check(load().lbm_step(h, int(nsteps)), "lbm_step")


def lbm_status(h) -> int:
    return load().lbm_status(h)


def lbm_error_string(code: int) -> str:
    return load().lbm_error_string(code).decode()


# ---- Python-side convenience ---------------------------------------------------

def _torch():
    import torch
    return torch


class Lattice:
    """One coupled flow + temperature lattice on the current CUDA device.

    Parameters are the fields of ``lbm_params`` (see include/lbm.h); the
    workspace is a torch uint8 tensor owned by this object.
    """

    def __init__(self, nx: int, ny: int, stream=None, **params):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("liblbm needs a CUDA device; there is no CPU path")
        self.lib = load()
        self.nx, self.ny, self.n = int(nx), int(ny), int(nx) * int(ny)
        self.params = make_params(nx, ny, **params)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        nbytes = lbm_workspace_bytes(self.params)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        self._h = lbm_create(self.params, self.stream.cuda_stream, aligned, nbytes)

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self.lib.lbm_destroy(h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- inputs -------------------------------------------------------------------
    def _dev(self, a, count=None):
        torch = _torch()
        count = self.n if count is None else count
        if isinstance(a, torch.Tensor):
            t = a.detach().to(device="cuda", dtype=torch.float32).contiguous()
        else:
            t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
        if t.numel() != count:
            raise ValueError(f"expected {count} values, got {t.numel()}")
        return t

    def set_fields(self, phi, K, T0, fl0, wall_T_left=None):
        ts = [self._dev(a) for a in (phi, K, T0, fl0)]
        wt = None if wall_T_left is None else self._dev(wall_T_left, self.ny)
        self.stream.wait_stream(_torch().cuda.current_stream())
        rc = self.lib.lbm_set_fields(self._h, *[t.data_ptr() for t in ts],
                                     None if wt is None else wt.data_ptr(), 1)
        _check(rc, "lbm_set_fields")

    def set_fields_host(self, phi, K, T0, fl0, wall_T_left=None):
        """Same as set_fields from host (numpy) arrays through the host-pointer path."""
        arrs = [np.ascontiguousarray(a, dtype=np.float32).ravel() for a in (phi, K, T0, fl0)]
        wt = None if wall_T_left is None else np.ascontiguousarray(wall_T_left, dtype=np.float32)
        rc = self.lib.lbm_set_fields(self._h, *[a.ctypes.data for a in arrs],
                                     None if wt is None else wt.ctypes.data, 0)
        _check(rc, "lbm_set_fields")

    # -- stepping -----------------------------------------------------------------
    def step(self, nsteps: int = 1):
        lbm_step(self._h, nsteps)

    def prepare(self, nsteps: int):
        """Capture the CUDA graphs step(nsteps) would use now, without stepping."""
        _check(self.lib.lbm_prepare(self._h, int(nsteps)), "lbm_prepare")

    def status(self) -> int:
        return lbm_status(self._h)

    def check_wait(self, limit_ns: int):
        """Queue the bounded-wait self-check (lbm_check_wait): a wait that must
        give up after limit_ns, after which status() reports LBM_ERR_TIMEOUT."""
        _check(self.lib.lbm_check_wait(self._h, int(limit_ns)), "lbm_check_wait")

    def steps_done(self) -> int:
        return int(self.lib.lbm_steps_done(self._h))

    def kernel_launches(self) -> int:
        return int(self.lib.lbm_kernel_launches(self._h))

    def autotune(self, trial_steps: int = 32) -> tuple[int, int]:
        """Pick the fastest stream-collide configuration for this lattice (real
        steps of the run); returns (kernel variant, tiles per CTA)."""
        v, t = ctypes.c_int32(), ctypes.c_int32()
        _check(self.lib.lbm_autotune(self._h, int(trial_steps), ctypes.byref(v), ctypes.byref(t)),
               "lbm_autotune")
        return v.value, t.value

    OBJECTIVES = {"melt": 0, "nusselt": 1}

    def _grad_buffers(self, shapes, device: bool):
        """Gradient outputs: torch CUDA tensors (device=True, written in place
        by the library) or numpy arrays; returns (arrays, pointers)."""
        if device:
            torch = _torch()
            outs = [torch.zeros(sh, dtype=torch.float32, device="cuda") for sh in shapes]
            _torch().cuda.current_stream().synchronize()
            return outs, [t.data_ptr() for t in outs]
        outs = [np.zeros(sh, dtype=np.float32) for sh in shapes]
        return outs, [a.ctypes.data for a in outs]

    def adjoint(self, nsteps: int, objective: str = "melt", checkpoint_every: int = 0,
                mu_sweeps: int = 0, device: bool = False):
        """Run nsteps steps; return the objective and its gradient with respect
        to the porosity field ([ny, nx]) and the left wall's temperature
        profile ([ny]) (lbm_adjoint in include/lbm.h).  objective "melt": the
        melted fraction after the steps; "nusselt": the left-wall Nusselt
        number after each step, averaged over the steps.  device=True returns
        the gradients as CUDA tensors (no host copy)."""
        (dphi, dtw), ptrs = self._grad_buffers([(self.ny, self.nx), (self.ny,)], device)
        J = ctypes.c_double()
        _check(self.lib.lbm_adjoint(self._h, self.OBJECTIVES[objective], int(nsteps),
                                    int(checkpoint_every), int(mu_sweeps), *ptrs,
                                    ctypes.byref(J), int(device)), "lbm_adjoint")
        return J.value, dphi, dtw

    def adjoint_coupled(self, nsteps: int, objective: str = "melt", checkpoint_every: int = 0,
                        mu_sweeps: int = 0, device: bool = False):
        """The flow lattice on: run nsteps steps; return the objective and its
        gradients with respect to the porosity field ([ny, nx]), ln K
        ([ny, nx]) and the left wall's temperature profile ([ny])
        (lbm_adjoint_coupled in include/lbm.h).  checkpoint_every: 0 keeps
        every state when it fits, K > 0 keeps one every K steps and recomputes
        the rest.  device=True returns CUDA tensors."""
        (dphi, dlnK, dtw), ptrs = self._grad_buffers(
            [(self.ny, self.nx), (self.ny, self.nx), (self.ny,)], device)
        J = ctypes.c_double()
        _check(self.lib.lbm_adjoint_coupled(self._h, self.OBJECTIVES[objective], int(nsteps),
                                            int(checkpoint_every), int(mu_sweeps), *ptrs,
                                            ctypes.byref(J), int(device)),
               "lbm_adjoint_coupled")
        return J.value, dphi, dlnK, dtw

    def adjoint_melt(self, nsteps: int, checkpoint_every: int = 0, mu_sweeps: int = 0):
        """The melted fraction after nsteps steps and its gradients
        (lbm_adjoint_melt in include/lbm.h)."""
        dphi = np.zeros((self.ny, self.nx), dtype=np.float32)
        dtw = np.zeros(self.ny, dtype=np.float32)
        J = ctypes.c_double()
        _check(self.lib.lbm_adjoint_melt(self._h, int(nsteps), int(checkpoint_every),
                                         int(mu_sweeps), dphi.ctypes.data, dtw.ctypes.data,
                                         ctypes.byref(J), 0), "lbm_adjoint_melt")
        return J.value, dphi, dtw

    def trace(self, capacity: int):
        """Start (capacity > 0 records) or stop (0) the kernel trace (lbm_trace)."""
        _check(self.lib.lbm_trace(self._h, int(capacity)), "lbm_trace")

    def trace_read(self, max_records: int = 1 << 22) -> np.ndarray:
        """The trace records so far, int64 [n, 4]: kind, step stamp, start ns, end ns."""
        out = np.zeros((max_records, 4), dtype=np.int64)
        n = ctypes.c_int64()
        _check(self.lib.lbm_trace_read(self._h, out.ctypes.data, int(max_records), ctypes.byref(n)),
               "lbm_trace_read")
        return out[:n.value]

    def adjoint_timing(self) -> tuple[float, float]:
        """Device ms of the last adjoint call: (forward run, reverse sweep)."""
        ms = (ctypes.c_double * 2)()
        _check(self.lib.lbm_adjoint_timing(self._h, ms), "lbm_adjoint_timing")
        return ms[0], ms[1]

    def kernel_variant(self) -> int:
        """1: ordinary-load stream-collide kernel, 2: TMA-staged kernel."""
        return int(self.lib.lbm_kernel_variant(self._h))

    def derived(self) -> dict:
        out = (ctypes.c_double * 8)()
        _check(self.lib.lbm_derived(self._h, out), "lbm_derived")
        keys = ("tau_nu", "tau_T", "nu_e", "nu_l", "alpha_e", "g_beta", "csT2", "lat")
        return dict(zip(keys, list(out)))

    # -- outputs ------------------------------------------------------------------
    def macros(self, numpy: bool = True) -> dict:
        torch = _torch()
        outs = {k: torch.empty((self.ny, self.nx), dtype=torch.float32, device="cuda")
                for k in ("ux", "uy", "rho", "T", "fl")}
        rc = self.lib.lbm_get_macros(self._h, *[outs[k].data_ptr() for k in
                                                ("ux", "uy", "rho", "T", "fl")], 1)
        _check(rc, "lbm_get_macros")
        self.stream.synchronize()
        if numpy:
            return {k: v.cpu().numpy() for k, v in outs.items()}
        return outs

    def macros_host(self) -> dict:
        """Macroscopic fields through the host-pointer path of lbm_get_macros."""
        outs = {k: np.empty((self.ny, self.nx), dtype=np.float32)
                for k in ("ux", "uy", "rho", "T", "fl")}
        rc = self.lib.lbm_get_macros(self._h, *[outs[k].ctypes.data for k in
                                                ("ux", "uy", "rho", "T", "fl")], 0)
        _check(rc, "lbm_get_macros")
        return outs

    def reduce(self) -> dict:
        out = (ctypes.c_double * 4)()
        rc = self.lib.lbm_reduce(self._h, out)
        vals = dict(zip(("mass", "enthalpy", "melt_frac", "nu_hot"), list(out)))
        _check(rc, "lbm_reduce")
        return vals

    def get_state(self):
        f = np.empty((9, self.ny, self.nx), dtype=np.float32)
        g = np.empty((5, self.ny, self.nx), dtype=np.float32)
        fl = np.empty((self.ny, self.nx), dtype=np.float32)
        _check(self.lib.lbm_get_state(self._h, f.ctypes.data, g.ctypes.data, fl.ctypes.data, 0),
               "lbm_get_state")
        return f, g, fl

    def set_state(self, f=None, g=None, fl=None):
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float32) for a in (f, g, fl)]
        _check(self.lib.lbm_set_state(self._h, *[None if a is None else a.ctypes.data for a in arrs], 0),
               "lbm_set_state")

    # -- measurement --------------------------------------------------------------
    def timing(self, enable: bool = True):
        _check(self.lib.lbm_timing(self._h, int(enable)), "lbm_timing")

    def timing_read(self) -> dict:
        ms = (ctypes.c_double * 4)()
        n, t, m = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(self.lib.lbm_timing_read(self._h, ms, ctypes.byref(n), ctypes.byref(t),
                                        ctypes.byref(m)), "lbm_timing_read")
        return dict(fused_ms=ms[0], prep_ms=ms[1], solve_ms=ms[2], commit_ms=ms[3], steps=n.value,
                    tiles_solved=t.value, max_sweeps=m.value)


TRACE_KINDS = {10: "stream-collide, all tiles", 11: "stream-collide, tiles away from the front",
               12: "stream-collide, tiles near the front", 20: "enthalpy solve",
               30: "enthalpy commit"}


def trace_launches(records: np.ndarray) -> list[dict]:
    """Group lbm_trace records into launches (one per kind and step stamp):
    start of the first CTA, end of the last, CTA count and median CTA time,
    times in us from the first record, in start order."""
    if len(records) == 0:
        return []
    t0 = int(records[:, 2].min())
    out = []
    keys = np.unique(records[:, :2], axis=0)
    for kind, stamp in keys:
        m = (records[:, 0] == kind) & (records[:, 1] == stamp)
        st, en = records[m, 2], records[m, 3]
        out.append(dict(kind=int(kind), parity=int(kind) // 100,
                        what=TRACE_KINDS.get(int(kind) % 100, str(kind)), step=int(stamp),
                        start_us=(int(st.min()) - t0) / 1e3, end_us=(int(en.max()) - t0) / 1e3,
                        ctas=int(m.sum()), median_cta_us=float(np.median(en - st)) / 1e3))
    out.sort(key=lambda r: r["start_us"])
    return out


class Batch:
    """Several lattices advanced together through one CUDA graph per 32 steps
    (lbm_batch_* in include/lbm.h).  Keeps references to the lattices."""

    def __init__(self, lattices, stream=None):
        torch = _torch()
        self.lattices = list(lattices)
        self.lib = load()
        self.stream = stream or torch.cuda.Stream()
        arr = (_VP * len(self.lattices))(*[lat._h.value for lat in self.lattices])
        h = _VP()
        _check(self.lib.lbm_batch_create(arr, len(self.lattices), self.stream.cuda_stream,
                                         ctypes.byref(h)), "lbm_batch_create")
        self._h = h

    def step(self, nsteps: int):
        _check(self.lib.lbm_batch_step(self._h, int(nsteps)), "lbm_batch_step")

    def mode(self) -> int:
        """1: one launch per pass over every lattice; 0: one graph branch per lattice."""
        rc = int(self.lib.lbm_batch_mode(self._h))
        _check(rc if rc < 0 else 0, "lbm_batch_mode")
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self.lib.lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
