"""Host logic of bench.py on CPU: the max-over-ranks step time of a multi-rank
run (two gloo ranks on 127.0.0.1) and the reference arm, which only rank 0 runs."""
import contextlib
import io
import json
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, value, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        out.put((rank, bench.max_over_ranks(value, dist, device="cpu")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_single_rank_is_identity():
    assert bench.max_over_ranks(12.5, None) == 12.5


def test_max_over_ranks_two_gloo_ranks_agree_on_the_slowest():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    values = [41.25, 43.75]                   # rank 1 is the slower one
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, values[r], out)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: max(values), 1: max(values)}


def _reference_args(**over):
    argv = ["--impl", "reference", "--workload", "1", "--steps", "1", "--warmup", "0"]
    for k, v in over.items():
        argv += [f"--{k}", str(v)]
    old = sys.argv
    sys.argv = ["bench.py"] + argv
    try:
        return bench.parse()
    finally:
        sys.argv = old


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(_reference_args(gpus=2))
    assert buf.getvalue() == ""


def test_reference_arm_rank0_prints_one_line(monkeypatch):
    pytest.importorskip("oracle")
    monkeypatch.setenv("RANK", "0")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(_reference_args())
    lines = [ln for ln in buf.getvalue().splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "fits/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
