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


def _fake_tree(tmp_path, source_text, recorded_sha):
    csrc = tmp_path / "paper_1808_06992_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "gram_tc.cu").write_bytes(source_text)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.txt").write_text(
        "# comment line\n"
        f"kernel=k_gram_tc source_sha={recorded_sha} dram_bytes_per_launch=1234000 capture=x.md\n")


def test_traffic_figure_used_only_while_the_source_hash_matches(tmp_path, monkeypatch):
    import hashlib
    src = b"__global__ void k_gram_tc() {}\n"
    _fake_tree(tmp_path, src, hashlib.sha256(src).hexdigest()[:16])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_per_launch("k_gram_tc") == 1234000.0
    # another workload than the one the figure was scaled to: no figure
    assert bench.traffic_per_launch("k_gram_tc", applies=False) is None
    # the source changed since the capture: no figure
    (tmp_path / "paper_1808_06992_gb300" / "csrc" / "gram_tc.cu").write_bytes(src + b"// edit\n")
    assert bench.traffic_per_launch("k_gram_tc") is None


def test_committed_traffic_record_has_no_stale_line():
    # a line whose kernel source changed since its capture would be silently
    # ignored by the bench: re-capture it (or drop the line) when the kernel changes
    with open(os.path.join(ROOT, "profiles", "traffic.txt")) as f:
        kernels = [dict(kv.split("=", 1) for kv in ln.split() if "=" in kv).get("kernel")
                   for ln in f if ln.startswith("kernel=")]
    assert kernels
    for k in kernels:
        assert bench.traffic_per_launch(k) is not None, k


_FAKE_SMI = r"""
import sys, time
flag = sys.argv[1]
while True:
    phase = open(flag).read().strip()
    if phase == "before":
        print("0, 1000, 2070, 300.0, 0x8, Active, Not Active, Not Active, Not Active", flush=True)
    elif phase == "during":
        print("0, 2070, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active", flush=True)
    else:
        print("0, 1500, 2070, 200.0, 0x0, Not Active, Not Active, Not Active, Not Active", flush=True)
    time.sleep(0.02)
"""


def test_clock_sampler_summarises_only_the_timed_region(tmp_path):
    import time
    fake = tmp_path / "fake_smi.py"
    fake.write_text(_FAKE_SMI)
    flag = tmp_path / "phase"
    flag.write_text("before")
    smp = bench.ClockSampler(0, cmd=[sys.executable, str(fake), str(flag)])
    smp.start()
    assert smp.lines                                  # sampling runs before the region opens
    time.sleep(0.2)
    flag.write_text("during")
    time.sleep(0.1)
    smp.mark_start()
    time.sleep(0.5)
    smp.mark_stop()
    flag.write_text("after")
    time.sleep(0.2)
    c = smp.stop()
    assert c["samples"] >= 10
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]           # the hw_slowdown before the region is not counted


def test_clock_sampler_without_nvidia_smi_says_so():
    smp = bench.ClockSampler(0, cmd=["/nonexistent/nvidia-smi"])
    smp.start()
    c = smp.stop()
    assert c["sm_mhz"] is None and c["reasons"] == ["nvidia-smi unavailable"]
