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
