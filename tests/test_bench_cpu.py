"""Host-side logic of bench.py on CPU: rank aggregation over a 2-process gloo group, the reference
arm's JSON contract, and the profile/traffic bookkeeping."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = bench.max_over_ranks(float(10 * rank + 1), world)
    bench.barrier(world)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"max": m}, f)
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    vals = [json.load(open(tmp_path / f"r{r}.json"))["max"] for r in range(2)]
    assert vals == [11.0, 11.0]


def test_single_rank_aggregation_is_identity():
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_reference_arm_contract(monkeypatch):
    # small grid so the CPU test stays quick; the JSON keys are what the driver reads
    monkeypatch.setattr(bench, "NX", 64)
    args = bench.argparse.Namespace(steps=2, warmup=3, gpus=1)
    line = bench.run_reference(args, 0, 1)
    assert line["impl"] == "reference" and line["unit"] == "MLUPS" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert bench.run_reference(args, 1, 2) is None  # other ranks print nothing
    assert line["config"] == bench.bench_config(1)  # the same workload description as our arm
    json.dumps(line)


def test_headline_error_against_oracle():
    import numpy as np

    want = np.linspace(1.0, 2.0, 16)
    got = want * (1 + 1e-7)
    r = bench.rel_l2_vs_oracle(got, want)
    assert abs(r["value"] - 1e-7) < 1e-12 and r["field"] == "rho'"
    assert bench.rel_l2_vs_oracle(got, None)["value"] is None


def test_profiled_traffic_is_null_when_kernel_changed(tmp_path, monkeypatch):
    p = tmp_path / "prof.md"
    p.write_text("kernel_source_sha256_16: deadbeefdeadbeef\ndram_bytes_per_launch: 1.0e8\n")
    monkeypatch.setattr(bench, "PROFILES", {3: str(p)})
    assert bench.profiled_traffic(3) is None
    p.write_text(f"kernel_source_sha256_16: {bench.kernel_source_sha()}\ndram_bytes_per_launch: 1.0e8\n")
    assert bench.profiled_traffic(3) == pytest.approx(1.0e8)
    assert bench.profiled_traffic(2) is None  # no summary for that kernel
