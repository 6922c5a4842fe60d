"""bench.py host logic without a GPU: the replica aggregation across ranks (two
gloo ranks on 127.0.0.1), the reference arm's JSON line, and the silent exit of
non-zero ranks in the reference arm."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    # each replica reports its own elapsed time; the slowest one sets the job time
    m = bench.reduce_max(10.0 + 3.5 * rank, world)
    with open(os.path.join(out_dir, "r%d.txt" % rank), "w") as f:
        f.write(repr(m))
    dist.destroy_process_group()


def test_replica_time_is_max_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    vals = [float(open(os.path.join(tmp_path, "r%d.txt" % r)).read()) for r in range(2)]
    assert vals == [13.5, 13.5]


def _run_bench(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    e.setdefault("OMP_NUM_THREADS", "4")
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True,
                          text=True, env=e, cwd=ROOT, timeout=600)


def test_reference_arm_prints_one_json_line():
    r = _run_bench(["--impl", "reference", "--steps", "2", "--warmup", "1", "--nx", "512"])
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "cell-updates/s" and d["value"] > 0
    assert d["metric"].startswith("cell-updates/s")
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1


def test_reference_arm_other_ranks_exit_silently():
    r = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "1", "--nx", "512"],
                   env={"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_roofline_uses_the_counters_of_the_launch_shape():
    """The bench's roofline object takes ncu traffic only for the block shape the
    dominant kernel ran with, and null for a shape no capture saw."""
    sys.path.insert(0, ROOT)
    import bench
    kt = {"k_face_y": (10.0, 10), "k_update": (5.0, 10)}
    cells = 4096 * 4096
    r = bench.roofline("hsgn", "mixed", kt, cells, 61, 7, 4, 6787.2, "measured", {"face_y": "32x8"})
    assert r["kernel"] == "k_face_y" and r["block"] == "32x8"
    assert r["traffic"] == bench.TRAFFIC_PER_CELL[("hsgn", "mixed", "k_face_y", "32x8")] * cells
    assert abs(r["achieved"] - 61 * cells / 1e-3 / 1e9) < 1e-6 * r["achieved"]
    r = bench.roofline("hsgn", "mixed", kt, cells, 61, 7, 4, 6787.2, "measured", {"face_y": "16x16"})
    assert r["traffic"] is None
    # compulsory bytes per cell: no primitive planes in the mixed path
    assert bench.kernel_bytes("k_face_y", 7, 4) == (7 + 3) * 4 + 8 + (2 * 7 + 9) * 4
    assert bench.kernel_bytes("k_face_y", 7, 8) == (2 * 7 + 4) * 8 + 8 + (2 * 7 + 9) * 8
