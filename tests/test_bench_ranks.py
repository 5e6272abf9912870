"""Multi-rank logic of bench.py on CPU (gloo, world size 2): the job time is the
slowest rank's and the throughput counts every rank's particle-steps."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, n = bench.aggregate_ranks(100.0 + 50.0 * rank, 1e6 * (rank + 1), dist)
    out.put((rank, t, n))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, n in res:
        assert t == 150.0
        assert n == 3e6


def test_aggregate_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(12.5, 7.0) == (12.5, 7.0)


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    """--impl reference times the oracle and prints one JSON line with the
    contract's keys (the 64^2 x 16 box, one step)."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "1", "--workload", "periodic_thermal_2d"])
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("periodic_thermal_2d")
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


@pytest.mark.parametrize("procs", [1, 2])
def test_reference_arm_process_count(monkeypatch, capsys, procs):
    """One process: the single thread in place, one 64^2 x 16 box; two:
    two boxes, their particle-steps together."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    bench.main(["--impl", "reference", "--steps", "2", "--warmup", "1", "--workload", "periodic_thermal_2d",
                "--ref-procs", str(procs)])
    d = json.loads([l for l in capsys.readouterr().out.splitlines() if l.startswith("{")][0])
    assert d["cpu_baseline"]["cores"] == procs
    assert ("single thread" in d["config"]["sample"]) == (procs == 1)
    n = 65536 * procs
    assert abs(d["value"] * d["ms_per_step"] / 1e3 - n) < 1e-6 * n


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "1", "--workload", "periodic_thermal_2d"])
    assert capsys.readouterr().out.strip() == ""


def test_oracle_on_every_core_figure():
    """The all-core oracle figure: one spawned process and box per core, the
    particle-steps of all of them over the common wall time."""
    import argparse
    sys.path.insert(0, ROOT)
    import bench
    a = argparse.Namespace(workload="periodic_thermal_2d", sample_n=0, ppc=16, err_n=0)
    r = bench._cpu_all_cores(a, 1, nproc=2)
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["unit"] == bench.UNIT
    assert "2 processes" in r["sample"] and "(131072 CRs in all)" in r["sample"]
    assert r["value"] > 0 and abs(r["value"] * r["seconds"] - 131072) < 1e-6 * 131072


def test_oracle_on_every_core_reports_a_failed_process():
    """A process that cannot build its box ends the figure with the reason
    instead of leaving the others waiting."""
    import argparse
    sys.path.insert(0, ROOT)
    import bench
    a = argparse.Namespace(workload="alfvenic_beam_3d", sample_n=-4, ppc=32, err_n=0)
    r = bench._cpu_all_cores(a, 1, nproc=2)
    assert set(r) == {"unavailable"} and r["unavailable"]


def test_oracle_on_every_core_gives_up_at_its_limit():
    """No result within the time limit (here far shorter than starting the
    processes) ends the figure with the reason; no process is left behind."""
    import argparse
    import multiprocessing as mp
    sys.path.insert(0, ROOT)
    import bench
    a = argparse.Namespace(workload="alfvenic_beam_3d", sample_n=40, ppc=32, err_n=0)
    r = bench._cpu_all_cores(a, 1, nproc=2, limit_s=0.2)
    assert set(r) == {"unavailable"}
    assert not mp.active_children()


def test_shared_atomic_roofline_arithmetic():
    """3-D TSC: 27 cells x (1 + 7 x 2) words + 2 contribution counts = 407
    atomic adds per particle, 12.71875 warp instructions; 2-D: 9 x 15 + 2 =
    137, 4.28125.  At one instruction per 1.1 SM-cycles on 152 SMs at
    2000 MHz the pipe does 276.36 G/s."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench.smem_atomic_roofline(3, 32 * 1000, 1e-6, 2000.0, 152)
    assert r["atomics_per_particle"] == 407
    assert abs(r["achieved"] - 407 * 1000 / 1e-6 / 1e9) < 1e-9 * r["achieved"]
    assert abs(r["peak"] - 152 * 2000e6 / 1.1 / 1e9) < 1e-9 * r["peak"]
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15
    r2 = bench.smem_atomic_roofline(2, 32, 1.0, 2000.0, 152)
    assert r2["atomics_per_particle"] == 137 and abs(r2["achieved"] - 137e-9) < 1e-20


def test_shared_pipe_roofline_arithmetic():
    """36.669 wavefronts per particle over 32,000 particles in 1 us is 1173.4
    G wavefronts/s; the pipe does 0.93 per SM-cycle on 152 SMs at 2000 MHz,
    282.72 G/s.  The figures per particle are those of the captures."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench.shared_pipe_roofline(36.669, 32 * 1000, 1e-6, 2000.0, 152)
    assert abs(r["achieved"] - 36.669 * 32000 / 1e-6 / 1e9) < 1e-9 * r["achieved"]
    assert abs(r["peak"] - 152 * 2000e6 * 0.93 / 1e9) < 1e-9 * r["peak"]
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15
    w = bench.PUSH_SHARED_WAVEFRONTS_PER_PARTICLE
    assert abs(w["alfvenic_beam_3d"] - 36.669) < 1e-3 and abs(w["bell_2d"] - 11.119) < 1e-3


def test_clock_record_parsing(tmp_path):
    """The nvidia-smi rows sampled during the timed region: median SM clock
    under load, the maximum clock, and every throttle reason seen active."""
    sys.path.insert(0, ROOT)
    import bench
    rows = ["0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2010, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
            "garbage line"]
    f = tmp_path / "clocks.csv"
    f.write_text("\n".join(rows) + "\n")

    class _File:
        name = str(f)

        def flush(self):
            pass

    c = bench.ClockSampler(0)
    c.proc, c.f = object(), _File()
    s = c.summary()
    assert s["sm_mhz"] == 2010.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 4
    f.write_text("0, 1100, 2070, 500.0, 0x0, Active, Not Active, Active, Not Active\n")
    c.f = _File()
    s = c.summary()
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and s["sm_mhz"] == 1100.0
    f.write_text("")
    c.f = _File()
    assert c.summary()["reasons"] == ["no samples"]
    c.proc = None
    assert c.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_profile_commands_use_the_current_bench_flags():
    """Every bench command quoted in the committed ncu summaries still parses
    with the bench's flags, so the summaries can be re-made as written."""
    import glob
    import re
    import shlex
    sys.path.insert(0, ROOT)
    import bench
    ap = bench.build_parser()
    found = 0
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read().replace("\\\n", " ")
        for cmd in re.findall(r"python bench\.py([^&\n`]*)", text):
            ap.parse_args(shlex.split(cmd))
            found += 1
        for ncu in re.findall(r"^ncu [^\n]*", text, flags=re.M):    # never one that locks the clocks
            assert "--clock-control none" in ncu, (path, ncu)
    assert found >= 4
