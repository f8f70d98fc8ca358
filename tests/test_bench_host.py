"""Host-side logic of bench.py, on CPU: multi-rank aggregation over gloo
(world size 2), the reference arm end to end, and the clock / peak parsing."""
import json
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 100.0 + 50.0 * rank          # rank 1 is the slow one
    value, ms = bench.aggregate(ms_local, cells=1000, steps=10, world=world, dist=dist,
                                device="cpu")
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_takes_slowest_rank_and_sums_replicas():
    world = 2
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank, args=(world, 29533, out), nprocs=world, join=True)
    for r in range(world):
        value, ms = out[r]
        assert ms == 150.0
        assert abs(value - world * 1000 * 10 / 0.150 / 1e6) < 1e-12


def test_aggregate_single_rank():
    value, ms = bench.aggregate(200.0, cells=4096, steps=100, world=1)
    assert ms == 200.0 and abs(value - 4096 * 100 / 0.2 / 1e6) < 1e-12


def test_reference_arm_prints_one_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "3", "--warmup", "1"], capture_output=True, text=True,
                       env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["higher_is_better"] is True


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "3", "--warmup", "1"], capture_output=True, text=True,
                       env=env, cwd=ROOT, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_clock_summary_parses_nvidia_smi_csv(tmp_path):
    s = bench.ClockSampler("0")
    s.path = str(tmp_path / "c.csv")
    s.proc = object()
    with open(s.path, "w") as f:
        f.write("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1987, 2070, 1200.5, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    out = s.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3


def test_measured_peak_falls_back(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7100.0}))
    assert bench.measured_peak() == (7100.0, "measured")


def test_traffic_record_matches_kernel_source():
    # the committed ncu record is only used while the fused kernel is unchanged
    d = json.load(open(bench.TRAFFIC_FILE))
    t = bench.traffic_per_launch(2048)
    if d["kernel_hash"] == bench.kernel_hash():
        assert t == pytest.approx(d["dram_bytes_per_launch"])
    else:
        assert t is None
