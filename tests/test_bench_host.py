"""Host logic of bench.py on CPU: the multi-rank timing reductions (2 gloo
ranks on 127.0.0.1) and the reference arm (the FP64 oracle) JSON line."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, local, dist = bench.dist_init()
    assert (r, w) == (rank, world) and dist.get_backend() == "gloo"
    bench.barrier(dist)
    mx = bench.max_over_ranks(10.0 + rank, dist)
    sm = bench.sum_over_ranks(100.0 * (rank + 1), dist)
    out.put((rank, mx, sm))
    dist.destroy_process_group()


def test_two_rank_max_and_sum_over_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 11.0, 300.0), (1, 11.0, 300.0)]


def test_reference_arm_prints_one_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "dam_break_small", "--steps", "3", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "interactions/s"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["higher_is_better"] is True
    # whole oracle steps of the same window as the GPU arm
    assert d["steps"] == 3 and "steps 3-6" in d["config"]["window"]
    assert d["ms_per_step"] > 0 and d["cpu_baseline"]["value"] == d["value"]


def test_profile_figures_follow_their_capture(tmp_path, monkeypatch):
    """traffic and limiter come from the committed capture only while the
    kernel source and the build flags are the ones it was taken with, and
    only for its workload (a copy of the repository layout under tmp_path)."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    (tmp_path / "profiles").mkdir()
    (tmp_path / "k.cu").write_text("kernel source")
    (tmp_path / "build.py").write_text("FLAGS = ['-ftz=true']")
    sha = lambda p: hashlib.sha256(p.read_bytes()).hexdigest()
    lim = {"unit": "L1 data pipe", "pct_of_peak": 89.0}
    d = {"source": "k.cu", "source_sha256": sha(tmp_path / "k.cu"),
         "build": "build.py", "build_sha256": sha(tmp_path / "build.py"),
         "variants": {"4": {"eval_bytes": 300, "build_bytes": 200, "limiter": lim},
                      "5": {"eval_bytes": 330, "build_bytes": 200, "limiter": lim},
                      "5p": {"eval_bytes": 260, "build_bytes": 130, "limiter": lim}}}
    (tmp_path / "profiles" / "k_interact_list_traffic.json").write_text(json.dumps(d))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic(1, "dam_break", 4) == (200 + 2 * 300) / 2
    assert bench.measured_traffic(1, "dam_break", 5, 0.25) == 330 + 0.25 * 200 / 2
    assert bench.measured_limiter(1, "dam_break", 5) == lim
    # the pair-once mode has its own entry (and none for variant 4 here)
    assert bench.measured_traffic(1, "dam_break", 5, 0.25, pair_once=True) == 260 + 0.25 * 130 / 2
    assert bench.measured_limiter(1, "dam_break", 5, pair_once=True) == lim
    assert bench.measured_traffic(1, "dam_break", 4, pair_once=True) is None
    # another workload, cell size or variant: nothing
    assert bench.measured_traffic(1, "wave_flume", 5) is None
    assert bench.measured_traffic(0, "dam_break", 5) is None
    assert bench.measured_limiter(1, "dam_break", 0) is None
    # the flags changed since the capture: nothing
    (tmp_path / "build.py").write_text("FLAGS = []")
    assert bench.measured_traffic(1, "dam_break", 5) is None
    assert bench.measured_limiter(1, "dam_break", 5) is None
    # the kernel source changed: nothing
    (tmp_path / "build.py").write_text("FLAGS = ['-ftz=true']")
    assert bench.measured_traffic(1, "dam_break", 4) is not None
    (tmp_path / "k.cu").write_text("kernel source, edited")
    assert bench.measured_traffic(1, "dam_break", 4) is None
