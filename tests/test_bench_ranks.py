"""bench.py's multi-rank aggregation on CPU ranks (gloo, world size 2): the
whole-job step time is the maximum over ranks and the units are summed; the
reference arm prints only on rank 0."""
import os
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms, units, rate = bench.whole_job(10.0 + 5.0 * rank, 1000 * (rank + 1), world)
    out[rank] = (ms, units, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_max_time_sum_units_gloo():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, 29517, out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        ms, units, rate = out[r]
        assert ms == 15.0 and units == 3000.0
        assert abs(rate - 3000.0 / 15e-3) < 1e-6


def test_reference_arm_prints_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_traffic_record_is_current_and_goes_null_on_change(tmp_path):
    """The committed ncu traffic figure is read only while the profiled
    kernel's source (and its planner) is the one it was captured on: the
    bench reports it for the current source, and null once that code
    changes."""
    import json
    import shutil
    sys.path.insert(0, ROOT)
    import bench
    tag = "sketch_slab_kernel_fp16_kr_256x256x256x16"
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[tag]
    assert bench.traffic_record(tag) == rec["dram_bytes_per_launch"]
    # the same check on a copy of the tree whose kernel source differs by one byte
    fake = tmp_path / "root"
    (fake / "profiles").mkdir(parents=True)
    shutil.copy(os.path.join(ROOT, "profiles", "traffic.json"), fake / "profiles" / "traffic.json")
    src = open(os.path.join(ROOT, rec["source"]), "rb").read()
    a = src.index(rec["region"][0].encode()) + len(rec["region"][0])
    dst = fake / rec["source"]
    dst.parent.mkdir(parents=True)
    dst.write_bytes(src[:a] + b" " + src[a:])
    old = bench.ROOT
    try:
        bench.ROOT = str(fake)
        assert bench.traffic_record(tag) is None
    finally:
        bench.ROOT = old
