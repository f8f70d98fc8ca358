"""Failure detection on the GPU, in the forms that fault and hang nothing:

* a NaN put into a population through lbm_set_state is reported by
  lbm_reduce (LBM_ERR_NONFINITE), and by the every-K-steps sentinel of
  lbm_step through lbm_status;
* the bounded device-side wait gives up: lbm_check_wait waits, with the
  stream-collide kernel's bounded wait and a 1 ms limit, on a barrier that
  nothing completes, and lbm_status reports LBM_ERR_TIMEOUT once;
* a forced low inner-iteration cap is reported as LBM_ERR_NOT_CONVERGED.

Also: how lbm_step splits a step count into CUDA graphs (exact-length graphs
from either parity, the sentinel's chunk ends, lbm_prepare) does not change
the result by a bit.
"""
import numpy as np
import pytest

import lbm_workloads as W

pytestmark = pytest.mark.gpu

NONFINITE, TIMEOUT, NOT_CONVERGED = -3, -7, -4


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1503_08406_gb300 as P
    return P


def _lattice(P, w, **over):
    lat = P.Lattice(w.nx, w.ny, **{**w.params, **over})
    lat.set_fields(w.phi, w.K, w.T0, w.fl0, w.wall_T_left)
    return lat


def test_nan_in_state_reported_by_reduce(P):
    w = W.melted_cavity(40)
    lat = _lattice(P, w)
    lat.step(3)
    assert lat.reduce()   # healthy
    f, g, fl = lat.get_state()
    f[4, 20, 17] = np.nan
    lat.set_state(f, g, fl)
    with pytest.raises(P.LBMError) as e:
        lat.reduce()
    assert e.value.code == NONFINITE


@pytest.mark.parametrize("where", ["f", "g", "fl"])
def test_sentinel_reports_nonfinite_state(P, where):
    w = W.melted_cavity(48)
    lat = _lattice(P, w, check_every=4)
    lat.step(9)
    assert lat.status() == 0        # healthy run: the sentinel finds nothing
    f, g, fl = lat.get_state()
    {"f": lambda: f.__setitem__((2, 30, 31), np.inf),
     "g": lambda: g.__setitem__((0, 5, 5), np.nan),
     "fl": lambda: fl.__setitem__((40, 3), np.nan)}[where]()
    lat.set_state(f, g, fl)
    lat.step(3)                     # the sentinel is not due yet
    assert lat.status() == 0
    lat.step(1)                     # now it is
    assert lat.status() == NONFINITE
    assert lat.status() == NONFINITE   # kept until a new state is loaded
    lat.set_fields(w.phi, w.K, w.T0, w.fl0)
    lat.step(8)
    assert lat.status() == 0


def test_bounded_wait_gives_up_and_is_reported_once(P):
    w = W.melted_cavity(40)
    lat = _lattice(P, w)
    lat.step(2)
    before = lat.get_state()
    lat.check_wait(1_000_000)       # 1 ms on a barrier nothing completes
    assert lat.status() == TIMEOUT
    assert lat.status() == 0        # reported once
    after = lat.get_state()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)  # the probe touches no state
    with pytest.raises(P.LBMError):
        lat.check_wait(10)           # below the accepted range


def test_forced_low_inner_cap_reported(P):
    w = W.melted_cavity(48)
    lat = _lattice(P, w, max_inner_iters=1)
    lat.step(4)
    assert lat.status() == NOT_CONVERGED
    assert lat.status() == 0


def test_graph_splits_give_the_same_bits(P):
    w = W.melted_cavity(64)
    ref = _lattice(P, w)
    ref.timing(True)                 # kernel by kernel, no graphs
    ref.step(75)
    ref.timing(False)
    exp = ref.get_state()
    for split in ([75], [5, 20, 50], [1, 64, 10], [3, 2, 70]):
        lat = _lattice(P, w, check_every=7)
        for k in split:
            lat.prepare(k)
            lat.step(k)
        got = lat.get_state()
        assert lat.status() == 0
        assert lat.steps_done() == 75
        for a, b in zip(exp, got):
            assert np.array_equal(a, b), split
