"""lbm_reduce_state_noalloc: the conservation sums for callers that cannot
allocate device memory (a framework whose allocator owns all device memory,
or monitoring code held to a fixed memory budget).  It reads an FP32
checkpoint the caller already holds and keeps its scratch in a fixed array
inside the library.

Checked through the C ABI against lbm_reduce, the entry point that uses the
context's own (allocated) scratch, on two calls in a row.  Both sum the same
float32 state in FP64, in different orders, so they agree to 1e-12 relative.
Cases: a walled melting cavity with a uniform and with a non-uniform left-wall
profile (the profile enters the Nusselt sum), a doubly periodic box, and a
context storing its populations in FP16 (its checkpoint is still FP32).
"""
import ctypes

import numpy as np
import pytest

import lbm_workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1503_08406_gb300 as P
    lib = P.load()
    lib.lbm_reduce_state_noalloc.argtypes = [ctypes.POINTER(P.lbm_params)] + [ctypes.c_void_p] * 7
    lib.lbm_reduce_state_noalloc.restype = ctypes.c_int
    return torch, P, lib


def _checkpoint(torch, lat, w):
    n = w.nx * w.ny
    f = torch.empty(9 * n, dtype=torch.float32, device="cuda")
    g = torch.empty(5 * n, dtype=torch.float32, device="cuda")
    fl = torch.empty(n, dtype=torch.float32, device="cuda")
    rc = lat.lib.lbm_get_state(lat._h, f.data_ptr(), g.data_ptr(), fl.data_ptr(), 1)
    assert rc == 0
    torch.cuda.synchronize()
    return f, g, fl


def _profiled_cavity():
    w = W.melted_cavity(64)
    y = np.arange(w.ny)
    w.wall_T_left = 1.0 + 0.25 * np.sin(2 * np.pi * y / w.ny)
    return w


CASES = {
    "cavity": (lambda: W.melted_cavity(64), 37, {}),
    "cavity_wall_profile": (_profiled_cavity, 41, {}),
    "periodic_box": (lambda: W.periodic_box(48, ny=40), 60, {}),
    "cavity_fp16_storage": (lambda: W.melted_cavity(64), 29, {"storage": "fp16"}),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_reduce_matches_lbm_reduce(setup, case):
    torch, P, lib = setup
    maker, steps, over = CASES[case]
    w = maker()
    lat = P.Lattice(w.nx, w.ny, **{**w.params, **over})
    lat.set_fields(w.phi, w.K, w.T0, w.fl0, w.wall_T_left)
    lat.step(steps)
    expected = lat.reduce()
    f, g, fl = _checkpoint(torch, lat, w)
    phi = torch.from_numpy(w.phi.astype(np.float32).ravel()).cuda()
    wall = None
    if w.wall_T_left is not None:
        wall = torch.from_numpy(w.wall_T_left.astype(np.float32)).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = (ctypes.c_double * 4)()
        rc = lib.lbm_reduce_state_noalloc(ctypes.byref(lat.params), f.data_ptr(), g.data_ptr(),
                                          fl.data_ptr(), phi.data_ptr(),
                                          None if wall is None else wall.data_ptr(), stream, out)
        assert rc == 0, (call, rc)
        got = dict(zip(("mass", "enthalpy", "melt_frac", "nu_hot"), list(out)))
        for k, v in expected.items():
            assert abs(got[k] - v) <= 1e-12 * max(abs(v), 1.0), (call, k, got[k], v)
    if w.wall_T_left is not None:
        # the profile matters: the uniform wall value gives another Nusselt number
        out = (ctypes.c_double * 4)()
        rc = lib.lbm_reduce_state_noalloc(ctypes.byref(lat.params), f.data_ptr(), g.data_ptr(),
                                          fl.data_ptr(), phi.data_ptr(), None, stream, out)
        assert rc == 0
        assert abs(out[3] - expected["nu_hot"]) > 1e-3 * abs(expected["nu_hot"])


def test_noalloc_reduce_rejects_too_many_rows(setup):
    torch, P, lib = setup
    max_rows = 16384   # LBM_NOALLOC_MAX_ROWS in include/lbm.h
    p = P.make_params(8, max_rows + 1, flow=0, tau_T=0.8)
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = (ctypes.c_double * 4)()
    rc = lib.lbm_reduce_state_noalloc(ctypes.byref(p), *[dummy.data_ptr()] * 4, None, None, out)
    assert rc == -1   # LBM_ERR_INVALID_ARG, before any kernel runs
