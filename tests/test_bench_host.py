"""Host-side logic of bench.py: replica timing over ranks (gloo, two CPU
processes), the whole-job value, the workload bookkeeping, and the clock
sampler (against a stand-in nvidia-smi)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.0 + rank, None)
    q.put((rank, t, bench.job_value(100, 5, world, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_time_is_max_over_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == 2.0
        assert v == pytest.approx(world * 100 * 5 / 2.0)


def test_workload_bookkeeping():
    sys.path.insert(0, ROOT)
    import bench
    case = bench.make_case(0)
    assert case.P == 64 and case.M == 64 * 1810 and case.Ns == 5
    lb = bench.level_band_cells(case)
    assert len(lb) == bench.wavefront_levels(case)
    assert sum(m for _, m in lb) == case.M
    assert sum(b for b, _ in lb) >= bench.band_cells(case)
    assert bench.launches_per_step(5, 5) == 69


def _fake_smi(tmp_path, reasons):
    """A stand-in nvidia-smi printing one CSV sample every 20 ms."""
    f = tmp_path / "nvidia-smi"
    f.write_text("#!/bin/sh\nwhile true; do echo \"0, 1980, 2070, 900.0, x, %s\"; sleep 0.02; done\n"
                 % ", ".join(reasons))
    f.chmod(0o755)
    return str(tmp_path)


def test_clock_sampler_reads_samples_and_reasons(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import time

    import bench
    d = _fake_smi(tmp_path, ["Not Active", "Active", "Not Active", "Active"])
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ["PATH"])
    c = bench.ClockSampler(0)
    c.start()
    assert c.skip >= 1  # returned after the first sample, which is left out
    time.sleep(0.2)
    out = c.stop()
    assert out["sm_mhz"] == 1980.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert out["samples"] >= 3


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.ClockSampler(0)
    c.start()
    assert c.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
