"""Host logic of bench.py.  Multi-process path (one rank per GPU, replicas of the workload):
the slowest rank's time is what every rank reports, and the value counts the units of all
ranks; run as two gloo ranks on the CPU; the reference arm does no work on rank 1.  And the
roofline's algorithmic work counter."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    local_ms = [1000.0, 3000.0][rank]
    m = b.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (m, b.whole_job_rate(world, 2, 1e9, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_report_the_slowest_time_and_the_whole_job_rate():
    port = _free_port()
    out = tmp.Manager().dict()
    tmp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        m, v = out[r]
        assert m == 3000.0
        assert v == pytest.approx(2 * 2 * 1e9 / 3.0)


def test_single_process_needs_no_group():
    b = _bench()
    assert b.max_over_ranks(12.5, None, "cpu") == 12.5
    assert b.whole_job_rate(1, 4, 2e9, 1000.0) == pytest.approx(8e9)


def test_reference_arm_does_nothing_on_other_ranks(capsys, monkeypatch):
    b = _bench()
    monkeypatch.setenv("RANK", "1")
    calls = []
    monkeypatch.setattr(b, "cpu_baseline_sample", lambda *a, **k: calls.append(a) or {})

    class A:
        workload, warmup, steps, gpus, ref_tents, cpu_max_procs = "graded", 3, 2, 2, 20, 16
    assert b.run_reference(A()) is None
    assert calls == [] and capsys.readouterr().out == ""


@pytest.mark.parametrize("dim,p,flop", [(2, 2, 60), (3, 2, 156), (3, 3, 264), (3, 4, 414)])
def test_algorithmic_flops_per_dof_update(dim, p, flop):
    """The roofline's work counter: per element and operator application, volume d n_f N_p^2,
    facets d n_f 2 N_fp N_p and mass solve + M' 2 n_f^2 N_p multiply-adds, 2 flop each,
    divided by the n_f N_p DOFs updated."""
    assert _bench().flops_per_dof_update(dim, p) == pytest.approx(flop)


def test_traffic_figure_is_tied_to_the_kernel_sources(monkeypatch):
    """The stored DRAM traffic per tent is reported only while the kernel sources hash to the
    stamp taken with it; any change to the sources turns it into null."""
    bench = _bench()
    rec = bench.TRAFFIC_BYTES_PER_TENT[("fp32", "tent_persistent_kernel")]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["sources"])
    assert bench.traffic_per_tent("fp32", "tent_persistent_kernel") == rec["bytes_per_tent"]
    assert bench.traffic_per_tent("fp64", "tent_persistent_kernel") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.traffic_per_tent("fp32", "tent_persistent_kernel") is None
