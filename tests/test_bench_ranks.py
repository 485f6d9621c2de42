"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): every rank takes rank 0's
decision on the number of timed repeats, the reported times are the max over ranks repeat by
repeat, and the value counts every rank's replica; under torchrun the reference arm runs on
rank 0 only (the other ranks exit at once, printing nothing), and rank 0's reference line carries
the bench line's keys with the warm-up and timed steps it ran."""
import json
import os
import socket
import subprocess
import sys

import pytest

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, repeats, times_by_rank, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seq = iter(times_by_rank[rank])
        got = bench.repeat_times(lambda: next(seq), repeats, world, "cpu")
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def _run(repeats, times_by_rank):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, repeats, times_by_rank, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


def test_every_rank_takes_rank0s_repeat_count_and_the_max_time():
    # rank 0 is slow (its 5 repeats pass 0.5 s) while rank 1 alone would run 50 repeats; rank 1's
    # third repeat is the slowest of all
    t0 = [200.0] * 60
    t1 = [1.0, 1.0, 900.0] + [1.0] * 60
    out = _run(0, [t0, t1])
    assert out[0] == out[1] == [200.0, 200.0, 900.0, 200.0, 200.0]


def test_a_fixed_repeat_count_is_taken_by_every_rank():
    t0 = [3.0, 1.0, 2.0, 5.0]
    t1 = [1.0, 4.0, 1.0, 5.0]
    out = _run(3, [t0, t1])
    assert out[0] == out[1] == [3.0, 4.0, 2.0]


def test_the_value_counts_every_ranks_replica():
    sys.path.insert(0, ROOT)
    import bench
    one = bench.whole_job_mlups(1024 * 2048, 20, 1, 7.3)
    assert bench.whole_job_mlups(1024 * 2048, 20, 2, 7.3) == pytest.approx(2 * one, rel=1e-15)
    assert one == pytest.approx(1024 * 2048 * 20 / 7.3e-3 / 1e6, rel=1e-15)


def test_reference_arm_runs_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_line_on_rank0():
    """The reference arm (the oracle on the host cores) prints one JSON line with the keys of the
    bench line, the warm-up and timed steps it ran, and its cpu_baseline and e2e records."""
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "2"], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "2 of the 2 requested warm-up steps" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["ms_per_step"] == pytest.approx(1024 * 2048 / d["value"] / 1e3, rel=1e-9)
