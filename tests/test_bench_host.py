"""Host-side logic of bench.py on the CPU: the slowest-rank reduction over a
world_size-2 gloo group, the reference arm (the oracle) alone and under a
2-process torchrun, and the parsing of sampled GPU clocks."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    out.put((rank, got, bench.whole_job_rate(world, 3, 1 << 20, got)))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]  # every rank sees the slowest time
    want = 2 * 3 * (1 << 20) / 0.015 / 1e9
    assert all(abs(r[2] - want) < 1e-9 for r in res)


def test_max_over_ranks_single_process():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5


def _json_lines(text):
    return [json.loads(line) for line in text.splitlines() if line.startswith("{")]


def test_reference_arm_alone():
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr
    lines = _json_lines(res.stdout)
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["unit"] == "Gkeys/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_under_torchrun_world2():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "3"]
    res = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = _json_lines(res.stdout)
    assert len(lines) == 1 and lines[0]["n_gpus"] == 2  # rank 0 alone prints


def test_clock_summary_parsing():
    c = bench.ClockSampler(0)
    c.lines = ["0, 1980, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2070, 2070, 1200.1, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2010, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    s = c.summary()
    assert s["sm_mhz"] == 2010 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_kernel_source_hash_ignores_comments(tmp_path, monkeypatch):
    """The DRAM-traffic figure is keyed by a hash of the pass's code: comments
    and blank lines do not change it, code does."""
    csrc = tmp_path / "paper_1511_03404_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in bench.ONESWEEP_SOURCES:
        (csrc / name).write_text("int a = 1;  // one\n\nint b = 2;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    first = csrc / bench.ONESWEEP_SOURCES[0]
    first.write_text("// a new comment\nint a = 1;  // changed comment\nint b = 2;\n\n")
    assert bench.kernel_source_hash() == h0
    first.write_text("int a = 3;\nint b = 2;\n")
    assert bench.kernel_source_hash() != h0
