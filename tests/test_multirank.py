"""The N > 1 path of bench.py on CPU: frames are independent, so ranks are
replicas (no data-path collective). Two gloo ranks check that each rank gets
its own frame, that the timing is the maximum over ranks on every rank, and
that the job value counts every rank's photons; the reference arm runs on
rank 0 only."""
import os
import socket
import subprocess
import sys

import numpy as np
import torch.multiprocessing as mp

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, REPO)
    import bench
    from paper_2203_00952_gb300 import synth

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    spec = synth.FrameSpec(rows=6, cols=7, T=256, sigma=2.0, mean_photons=40.0, sbr=1.0)
    fr = bench.rank_frame(spec, rank)
    digest = torch.tensor([int(fr.offsets[-1]), int(fr.stamps.astype(np.int64).sum())], dtype=torch.int64)
    all_d = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(all_d, digest)
    local_ms = 10.0 + 5.0 * rank
    total = bench.max_over_ranks(local_ms, world, "cpu")
    value = bench.job_value(world, 1000, 4, total)
    out[rank] = (total, value, [tuple(d.tolist()) for d in all_d])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_are_independent_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    expect_max = 10.0 + 5.0 * (world - 1)
    for r in range(world):
        total, value, digests = res[r]
        assert total == expect_max  # max over ranks, on every rank
        assert value == world * 1000 * 4 / (expect_max / 1e3)
        assert digests[0] != digests[1]  # each rank its own frame
    assert res[0][2] == res[1][2]


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(REPO, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_prints_its_line_on_rank_zero():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(REPO, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--ref-sample-seconds", "0.05"], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    import json

    line = json.loads(r.stdout.strip().splitlines()[-1])
    sys.path.insert(0, REPO)
    import bench

    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == bench.WORKLOAD_NAME
