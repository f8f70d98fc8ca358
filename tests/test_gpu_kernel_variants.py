"""The two stream-collide kernels give the same bits.

The TMA-staged kernel copies each 32 x 8 tile's populations (with
a one-node halo on odd steps), f_l (with halo), phi and K into shared memory
through bulk tensor copies, then runs the same per-node update as the
ordinary-load kernel.  Same inputs, same arithmetic: the state after any
number of steps must match bit for bit, on ragged tiles, with and without the
flow lattice, through the direct path (single steps) and the CUDA graphs
(where each step's fused pass is split into far and near tiles).
"""
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


def _run(P, w, steps, variant, chunks=1):
    lat = P.Lattice(w.nx, w.ny, **{**w.params, "kernel_variant": variant})
    lat.set_fields(w.phi, w.K, w.T0, w.fl0, w.wall_T_left)
    for _ in range(chunks):
        lat.step(steps // chunks)
    assert lat.status() == 0
    return lat


def test_variant_selection(lbm):
    P = lbm
    w = W.melted_cavity(64)
    assert _run(P, w, 0, 0).kernel_variant() == 2      # walled, nx % 4 == 0: TMA
    assert _run(P, w, 0, 1).kernel_variant() == 1      # forced ordinary loads
    w42 = W.melted_cavity(42)                            # rows not 16-byte strided
    assert _run(P, w42, 0, 2).kernel_variant() == 1
    wp = W.periodic_box(48)                              # periodic halos: no tensor maps
    assert _run(P, wp, 0, 2).kernel_variant() == 1


def _cropped(w, ny):
    """The cavity's lower ny rows, walled again on top (row ny - 1 becomes the wall row)."""
    import dataclasses
    return dataclasses.replace(w, name="%s_%dx%d" % (w.name, w.nx, ny), ny=ny,
                               phi=w.phi[:ny].copy(), K=w.K[:ny].copy(), T0=w.T0[:ny].copy(),
                               fl0=w.fl0[:ny].copy())


CASES = {
    # ny - 1 = 96 is a multiple of the tile height: the top wall row is a tile row of its
    # own, holding no node to update, whose wall slots only the row below writes
    "cropped_cavity_100x97": (lambda: _cropped(W.melted_cavity(100), 97), 37, 1),
    # ragged in x (100 = 3 tiles + 4) and y (100 = 12 rows of tiles + 4)
    "melted_cavity_100": (lambda: W.melted_cavity(100), 57, 1),
    # no flow lattice, Dirichlet and adiabatic walls, a moving solidification front
    "corner_100": (lambda: W.corner_solidification(100), 41, 1),
    # graph path: a 64-step graph with far/near split passes, then a 6-step graph
    "bench_cavity_256": (lambda: W.bench_cavity(256, melted=0.5), 70, 1),
    # one step per call: only the direct path, both parities
    "melted_cavity_64_direct": (lambda: W.melted_cavity(64), 9, 9),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_tma_kernel_matches_plain_kernel_bitwise(lbm, name):
    maker, steps, chunks = CASES[name]
    w = maker()
    plain = _run(lbm, w, steps, 1, chunks)
    tma = _run(lbm, w, steps, 2, chunks)
    assert plain.kernel_variant() == 1 and tma.kernel_variant() == 2
    for k, (a, b) in enumerate(zip(plain.get_state(), tma.get_state())):
        diff = np.flatnonzero(a.view(np.uint32) != b.view(np.uint32))
        assert diff.size == 0, (name, ("f", "g", "fl")[k], diff[:8], a.ravel()[diff[:4]],
                                b.ravel()[diff[:4]])
    assert plain.reduce() == tma.reduce()
