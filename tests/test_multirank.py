"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas only, no data-path collective).
The job's figures combine the slowest rank's time with the units of all ranks, and under torchrun
only rank 0 runs and prints the reference arm."""
import contextlib
import importlib.util
import io
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _bench()
        dist.barrier()
        # rank r timed (r + 1) seconds for 10 (r + 1) PCG iterations
        dev_s, iters = bench.combine_ranks(float(rank + 1), 10 * (rank + 1), 0.5, world, "cpu")
        dist.barrier()
        out.put((rank, dev_s, iters))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_max_time_and_summed_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, dev_s, iters in res:
        assert dev_s == 2.0 and iters == 30.0, (rank, dev_s, iters)


def test_single_rank_needs_no_process_group():
    bench = _bench()
    assert bench.combine_ranks(1.5, 7, 0.1, 1, "cpu") == (1.5, 7.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    bench = _bench()
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"steps": 1, "warmup": 0, "gpus": 2})()
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""
