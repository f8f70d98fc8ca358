"""The kernel trace (lbm_trace / lbm_trace_read): every CTA of the traced
kernels leaves one record; the launches of a graph-replayed step group by
step stamp into a full or far-tile stream-collide pass, a near-tile pass, a
solve and a commit, in dependency order; tracing changes no result."""
import numpy as np
import pytest

import lbm_workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1503_08406_gb300 as P
    return P


def test_trace_records_each_launch_in_order(P):
    from paper_1503_08406_gb300.lbm import trace_launches
    w = W.bench_cavity(256, melted=0.5)
    ref = P.Lattice(w.nx, w.ny, **w.params)
    lat = P.Lattice(w.nx, w.ny, **w.params)
    for x in (ref, lat):
        x.set_fields(w.phi, w.K, w.T0, w.fl0)
    assert lat.kernel_variant() == 2
    lat.trace(1 << 16)
    lat.step(6)
    recs = lat.trace_read()
    lat.trace(0)
    assert len(recs) > 0 and np.all(recs[:, 3] >= recs[:, 2])
    launches = trace_launches(recs)
    steps = sorted({r["step"] for r in launches})
    assert len(steps) == 6 and steps == list(range(steps[0], steps[0] + 6))
    by_step = {s: {r["kind"] % 100: r for r in launches if r["step"] == s} for s in steps}
    first = by_step[steps[0]]
    assert 10 in first and 20 in first and 30 in first      # full pass, solve, commit
    for s in steps[1:]:
        k = by_step[s]
        assert 11 in k and 12 in k and 20 in k and 30 in k  # far and near passes in a graph
        # the near tiles wait for the previous commit, the solve for both passes
        assert k[12]["start_us"] >= by_step[s - 1][30]["end_us"]
        assert k[20]["start_us"] >= max(k[11]["end_us"], k[12]["end_us"])
        assert k[30]["start_us"] >= k[20]["end_us"]
    assert all(r["parity"] == (r["step"] - steps[0]) % 2 for r in launches) or \
        all(r["parity"] == (r["step"] - steps[0] + 1) % 2 for r in launches)
    assert len(lat.trace_read()) == 0                       # off: nothing recorded
    ref.step(6)
    for a, b in zip(ref.get_state(), lat.get_state()):
        assert np.array_equal(a, b)
