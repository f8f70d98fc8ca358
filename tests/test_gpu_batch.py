"""Batches of uneven lattices in one CUDA graph, and the per-lattice autotuner.

A batch replays one graph per 32 steps holding every lattice's kernels on its
own branch; each lattice keeps its own parameters, size, storage and kernel
configuration.  The step each lattice takes is the same computation as when
it is stepped alone, so the results must agree bit for bit.  The autotuner
switches between stream-collide configurations that compute the same step,
so a tuned run must also match an untuned one bit for bit.
"""
import ctypes

import numpy as np
import pytest

import lbm_workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
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


def _same(a, b):
    for x, y in zip(a.get_state(), b.get_state()):
        if not np.array_equal(x.view(np.uint32), y.view(np.uint32)):
            return False
    return True


def _members():
    ws = W.batched_cavities(3, seed=4)   # sides drawn from 64..512
    return [(ws[0], {}), (ws[1], {}), (ws[2], {"storage": "fp16"}),
            (W.melted_cavity(64), {"kernel_variant": 1}),   # ordinary-load kernel
            (W.periodic_box(48, ny=40), {})]                 # periodic: ordinary loads


@pytest.mark.parametrize("lead,steps", [(0, 70), (3, 67)])
def test_batch_matches_lattices_stepped_alone(lbm, lead, steps):
    """lead: steps each lattice takes alone first (an odd count makes the batch
    take one single step before its graphs); then the batch advances steps."""
    import torch
    members = _members()
    batch_lats = [_lattice(lbm, w, **o) for w, o in members]
    for lat in batch_lats:
        lat.step(lead)
    b = lbm.Batch(batch_lats)
    b.step(steps)
    torch.cuda.synchronize()
    for (w, o), lat in zip(members, batch_lats):
        assert lat.status() == 0 and lat.steps_done() == lead + steps
        alone = _lattice(lbm, w, **o)
        alone.step(lead + steps)
        assert _same(lat, alone), w.name
    b.close()


@pytest.mark.parametrize("lead,steps", [(0, 70), (1, 96)])
def test_batched_launches_match_lattices_stepped_alone(lbm, lead, steps):
    """Six uneven cavities of the batch workload (FP32, TMA-staged kernel):
    each pass of a step is one launch over all of them, each cavity on its
    own range of CTAs, and every cavity ends bit for bit where it ends when
    stepped alone."""
    import torch
    ws = W.batched_cavities(6, seed=4)
    lats = [_lattice(lbm, w) for w in ws]
    for lat in lats:
        lat.step(lead)
    b = lbm.Batch(lats)
    assert b.mode() == 1
    b.step(steps)
    torch.cuda.synchronize()
    for w, lat in zip(ws, lats):
        assert lat.status() == 0 and lat.steps_done() == lead + steps
        alone = _lattice(lbm, w)
        alone.step(lead + steps)
        assert _same(lat, alone), w.name
    b.close()


def test_mixed_batch_takes_one_branch_per_lattice(lbm):
    b = lbm.Batch([_lattice(lbm, w, **o) for w, o in _members()])
    assert b.mode() == 0
    b.close()


def test_batch_rejects_repeated_and_empty(lbm):
    w = W.melted_cavity(48)
    lat = _lattice(lbm, w)
    lib = lbm.load()
    h = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 2)(lat._h.value, lat._h.value)
    assert lib.lbm_batch_create(arr, 2, None, ctypes.byref(h)) == -1 and not h.value
    assert lib.lbm_batch_create(arr, 0, None, ctypes.byref(h)) == -1


def test_autotuned_run_matches_untuned(lbm):
    w = W.bench_cavity(256, melted=0.5)
    tuned = _lattice(lbm, w)
    variant, tpc = tuned.autotune(8)
    assert variant in (1, 2) and tuned.kernel_variant() == variant
    assert (variant == 1 and tpc == 0) or (variant == 2 and tpc in (2, 3, 4, 5, 6, 8))
    done = tuned.steps_done()
    assert done == 7 * 2 * 8      # seven configurations, 2 x 8 steps each
    tuned.step(40)
    plain = _lattice(lbm, w)
    plain.step(done + 40)
    assert tuned.status() == 0 and _same(tuned, plain)


def test_autotune_without_tma_tries_only_the_ordinary_kernel(lbm):
    w = W.periodic_box(48)
    lat = _lattice(lbm, w)
    assert lat.autotune(4) == (1, 0)
    assert lat.steps_done() == 8


def _normwise(got, exp, fields=("ux", "uy", "T", "fl")):
    out = {}
    for k in fields:
        scale = np.abs(exp[k]).max()
        out[k] = float(np.abs(got[k].astype(np.float64) - exp[k]).max() / scale) if scale else \
            float(np.abs(got[k]).max())
    return out


def test_batch_members_match_oracle(lbm, oracle_mod):
    """Members of the 64-cavity batch workload (seed 4) stepped in a batch of
    four, 320 steps (ten graph replays) from the workload's own initial state,
    against the FP64 oracle: the one with the smallest tau_nu (0.5036: 64^2,
    Ra = 9.7e6), the 96^2 one at tau_nu = 0.5058 and a 512^2 one (tau_nu =
    0.535, Ra = 6.6e6), each within 5e-5 normwise in u, T and f_l.  (Members
    with tau_T above ~0.75, 15 of the 64, grow the scheme's odd-even mode at
    their isothermal front: there the FP32 and FP64 runs part after about a
    hundred steps, as any two roundings do.)"""
    import torch
    ws = W.batched_cavities(64, seed=4)
    picks = [55, 38, 7, 40]
    members = [W.Workload(ws[i].name, ws[i].nx, ws[i].ny, ws[i].params,
                          *(getattr(ws[i], k).astype(np.float32).astype(np.float64)
                            for k in ("phi", "K", "T0", "fl0"))) for i in picks]
    lats = [_lattice(lbm, w) for w in members]
    b = lbm.Batch(lats)
    assert b.mode() == 1
    steps = 320
    b.step(steps)
    torch.cuda.synchronize()
    for w, lat in zip(members[:3], lats[:3]):
        assert lat.status() == 0 and lat.steps_done() == steps
        o = oracle_mod.Oracle(w.nx, w.ny, **w.params)
        o.set_fields(w.phi, w.K, w.T0, w.fl0, w.wall_T_left)
        o.step(steps)
        if w is members[0]:
            assert abs(o.derived()["tau_nu"] - 0.5036) < 1e-4
        err = _normwise(lat.macros(), o.macros())
        assert max(err.values()) < 5e-5, (w.name, err)
    b.close()
