"""The multi-process path of bench.py on CPU (gloo, world size 2): the
replicas exchange nothing but the max-over-ranks timing reduction, and under
torchrun only rank 0 runs and prints the reference arm."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.max_over_ranks(1.5 + rank, dist, "cpu")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    got = dict(q.get(timeout=5) for _ in procs)
    assert got == {0: 2.5, 1: 2.5}


def test_max_over_ranks_without_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25


def test_reference_arm_under_torchrun_prints_once_on_rank_0():
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0"]
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    r = json.loads(lines[0])
    assert r["impl"] == "reference" and r["value"] > 0 and r["steps"] == 1
    assert r["e2e"]["h2d_bytes_per_step"] == 0 and r["cpu_baseline"]["kind"] == "oracle"


def _fake_smi(tmp_path, lines):
    """A stand-in for nvidia-smi that prints fixed samples and then waits to
    be terminated, as the real one does under -lms."""
    smi = tmp_path / "nvidia-smi"
    body = "".join("echo '%s'\n" % ln for ln in lines)
    smi.write_text("#!/bin/sh\n" + body + "sleep 30\n")
    smi.chmod(0o755)
    return str(tmp_path)


def _sample_clocks(monkeypatch, bindir, keep_path=None):
    import time
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("PATH", bindir + os.pathsep + os.environ["PATH"])
    if keep_path:
        monkeypatch.setenv("BH_CLOCKS_CSV", keep_path)
    else:
        monkeypatch.delenv("BH_CLOCKS_CSV", raising=False)
    with bench.Clocks(0) as clk:
        time.sleep(0.5)
    return clk, clk.summary()


def test_clock_summary_median_max_and_reasons(tmp_path, monkeypatch):
    lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2055, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage line"]
    clk, s = _sample_clocks(monkeypatch, _fake_smi(tmp_path, lines))
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(clk.path)  # the temporary sample file is removed


def test_clock_summary_keeps_samples_where_asked(tmp_path, monkeypatch):
    lines = ["0, 2070, 2070, 900.1, 0x0, Active, Not Active, Not Active, Not Active"]
    keep = str(tmp_path / "clocks.csv")
    clk, s = _sample_clocks(monkeypatch, _fake_smi(tmp_path, lines), keep)
    assert s["reasons"] == ["hw_slowdown"] and s["samples"] == 1
    assert clk.path == keep and os.path.exists(keep)


def test_clock_summary_without_nvidia_smi(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("PATH", str(tmp_path))
    with bench.Clocks(0) as clk:
        pass
    assert clk.summary()["reasons"] == ["nvidia-smi unavailable"]
    assert clk.fh.closed and not os.path.exists(clk.path)


def test_table_entries_cover_every_printed_value():
    """The --tables mode runs one solve per printed entry of Tables 1-3, with
    the DoF count (kN+1)^d of the paper's convention, smallest first."""
    sys.path.insert(0, ROOT)
    import bench
    golden = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_tables_nu_frac.json")))
    assert set(bench.TABLE_COLUMNS) == {n for n in golden if n.startswith("tab") and n != "tab3_levels"}
    entries = bench.table_entries(golden)
    printed = sum(v is not None for n in bench.TABLE_COLUMNS for row in golden[n] for v in row)
    assert len(entries) == printed == 192
    assert [e[0] for e in entries] == sorted(e[0] for e in entries)
    for dofs, name, i, j, d, k, L in entries:
        assert golden[name][i][j] is not None and dofs == (k * 2 ** L + 1) ** d
        assert d == (3 if name.startswith("tab3") else 2)
    # the paper's caption: only levels with 5e4 to 1e7 DoFs (2D) were computed
    assert min(e[0] for e in entries if e[4] == 2) >= 5e4


def test_cpu_baseline_on_all_degrees_with_a_small_budget():
    """The CPU baseline leg: the six degrees solved concurrently by spawned
    oracle processes; with a budget of a second it stops after the first
    size, and reports that size, its cores and the sizes it did not run."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench.cpu_baseline(budget_s=1.0, reps=1)
    assert r["kind"] == "oracle" and r["value"] > 0
    assert r["largest_cells"] == 8 and len(r["sizes"]) == 1
    assert r["cores"] >= 6 and r["host_cpus"] == os.cpu_count()
    top = r["sizes"][0]
    assert top["dofs"] == sum((k * 8 + 1) ** 2 for k in range(2, 8))
    assert top["true_relres_max"] <= 1.0001e-8 and "512^2" in r["not_run"]
