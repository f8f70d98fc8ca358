"""The seeded input recipes (lbm_workloads): shapes, ranges and the readings
they implement, checked on the host.  The recipes hold no arithmetic of the
method; these tests pin what the design notes state about them."""
import numpy as np

import lbm_workloads as W


def test_inverse_problem_cavity_recipe():
    """512^2 inverse-problem cavity: ln K with standard deviation ~0.5 and
    mean K = Da H^2; porosity in [0.3, 0.6]; the solid starts, and the right
    wall is held, below the melting range by its width (no node on the
    clamp's kink); only the hot wall column starts liquid."""
    w = W.adjoint_cavity(512)
    assert (w.nx, w.ny) == (512, 512)
    lnK = np.log(w.K)
    assert 0.35 < lnK.std() < 0.6
    assert abs(w.K.mean() / (1e-4 * 512 * 512) - 1) < 1e-12
    assert w.phi.min() >= 0.3 and w.phi.max() <= 0.6
    p = w.params
    T_c = p["T_bc"][1]
    assert T_c == p["T_s"] - (p["T_l"] - p["T_s"])
    assert np.all(w.T0[:, 1:] == T_c) and np.all(w.T0[:, 0] == 1.0)
    assert np.all(w.fl0[:, 0] == 1.0) and np.all(w.fl0[:, 1:] == 0.0)
    assert np.all(w.wall_T_left == 1.0)


def test_inverse_problem_copies_keep_the_large_draw():
    """The 64^2 copy is the 512^2 draw block-averaged 8 x 8 (porosity exactly,
    ln K up to the renormalisation of its mean)."""
    big, small = W.adjoint_cavity(512), W.adjoint_cavity(64)
    avg = big.phi.reshape(64, 8, 64, 8).mean(axis=(1, 3))
    assert np.allclose(small.phi, avg, atol=1e-12)
    lk_big = np.log(big.K).reshape(64, 8, 64, 8).mean(axis=(1, 3))
    d = np.log(small.K) - lk_big
    assert d.std() < 0.05   # the same pattern


def test_melted_start_is_consistent():
    """melted > 0: the left fraction of the columns liquid and above T_l, the
    rest solid at T_c."""
    w = W.adjoint_cavity(64, melted=0.25)
    m = 16
    assert np.all(w.fl0[:, :m] == 1.0) and np.all(w.fl0[:, m:] == 0.0)
    assert w.T0[:, :m].min() > w.params["T_l"]
    assert np.all(w.T0[:, m:] == w.params["T_bc"][1])


def test_batch_workload_recipe():
    """64 cavities: sides from the stated set, Ra log-uniform in [1e4, 1e7],
    porosity in [0.3, 0.9], St in [0.1, 1]; the draw is seeded."""
    a, b = W.batched_cavities(64, seed=4), W.batched_cavities(64, seed=4)
    assert len(a) == 64
    for x, y in zip(a, b):
        assert x.nx == y.nx and x.meta == y.meta
        assert x.nx in W.BATCH_SIDES and x.nx == x.ny
        assert 1e4 <= x.meta["Ra"] <= 1e7
        assert 0.3 <= x.meta["phi"] <= 0.9
        assert 0.1 <= x.meta["St"] <= 1.0
    assert len({x.nx for x in a}) >= 5   # uneven sizes
