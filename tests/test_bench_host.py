"""bench.py's host logic without a GPU: the max over ranks (gloo, world
sizes 2 and 3) and the reference arm's rank handling."""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest
import torch.multiprocessing as mp

import dist_workers
from dist_workers import free_port

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("world", [2, 3])
def test_max_over_ranks_gloo(world):
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(dist_workers.bench_max_body, args=(world, free_port(), d), nprocs=world, join=True)
        got = [float(np.load(f"{d}/max{r}.npy")[0]) for r in range(world)]
    assert got == [1.5 * world] * world


def test_max_over_ranks_single_process():
    import bench
    assert bench.max_over_ranks(2.5, "cpu") == 2.5


def test_reference_arm_only_on_rank0():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_warmup_below_three_is_refused():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--warmup", "2"],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0


def test_reference_arm_prints_one_complete_line():
    """The oracle arm on the host cores: one JSON line with the keys the
    measurement contract asks for."""
    import json
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"]


def test_roofline_states_both_pair_counts():
    """frac_executed counts the pairs the symmetrised kernel visits, P(N);
    frac_effective_pairs the 27 N^6 / 64 valid pairs of the plain sum; both
    at 6 FMA-pipe lane operations per pair and the same launch time."""
    import bench
    for N in (16, 32):
        r = bench.conv_roofline(N, 256, 10.0)
        ratio = r["frac_effective_pairs"] / r["frac_executed"]
        assert abs(ratio - bench.valid_pairs_per_cell(N) / bench.unique_pairs_per_cell(N)) < 1e-12
        assert 1.8 < ratio < 2.1  # the symmetrisation halves the work, up to the centre tiles
        assert bench.valid_pairs_per_cell(N) == 27 * N ** 6 // 64
        assert r["frac"] == r["frac_executed"]
        assert abs(r["achieved"] - 6.0 * bench.unique_pairs_per_cell(N) * 256 / 10e-3 / 1e12) < 1e-9


def test_traffic_is_reported_only_for_the_captured_launch_shape():
    """The roofline's DRAM traffic belongs to one launch shape: the default
    and explicit choices that select a captured kernel map to its entry,
    anything else (another tile shape, rebuilt weights, no L2 priorities, a
    shape the group count cannot take) is reported as null."""
    import bench
    base = {"groups_per_cta": 0, "ctas_per_sm": 0, "tile_split": 0, "weights": "stored tiles", "l2_hint": 0,
            "tile": 0}
    assert bench.traffic_key(32, 256, base) == (32, 256, 2, 1)
    assert bench.traffic_key(32, 256, dict(base, groups_per_cta=4)) == (32, 256, 4, 1)
    assert bench.traffic_key(32, 256, dict(base, groups_per_cta=2, tile_split=2)) == (32, 256, 2, 2)
    assert bench.traffic_key(16, 128, dict(base, groups_per_cta=2, tile_split=4)) == (16, 128, 2, 4)
    assert bench.traffic_key(32, 96, dict(base, groups_per_cta=4)) == (32, 96, 1, 1)  # three groups: one per CTA
    assert bench.traffic_key(32, 256, dict(base, tile=3)) is None
    assert bench.traffic_key(32, 256, dict(base, weights="radius tables")) is None
    assert bench.traffic_key(32, 256, dict(base, l2_hint=1)) is None
    for key in ((32, 256, 4, 1), (32, 256, 2, 1), (32, 256, 2, 2), (16, 128, 2, 4)):
        assert bench.TRAFFIC[key] > 0
    r = bench.conv_roofline(32, 256, 12.5, None, dict(base, groups_per_cta=4))
    assert r["traffic"] == bench.TRAFFIC[(32, 256, 4, 1)]
    assert bench.conv_roofline(32, 256, 12.5, None, dict(base, tile=2))["traffic"] is None
