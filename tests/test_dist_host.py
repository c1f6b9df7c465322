"""bench.py's multi-rank harness on CPU: two gloo ranks (one process per GPU on a real
box, replicas only) agree on the barrier and on the max-over-ranks timing, and the
reference arm runs on rank 0 only."""
import importlib.util
import os
import socket

import pytest
import torch.multiprocessing as mp

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


def _rank_main(rank, world, port, out):
    os.environ.update({"WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    bench = _bench()
    w, r, local = bench.dist_setup()
    bench.barrier(w)
    # each rank "measured" a different time; every rank must see the slowest one
    slowest = bench.max_over_ranks(w, 1.0 + 0.25 * r)

    class Args:
        steps, warmup = 1, 0
    ref_rc = bench.run_reference(Args(), w, r) if r != 0 else None
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    out.put((r, w, local, slowest, ref_rc))


def test_two_gloo_ranks_barrier_and_max():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, *_ in res] == [0, 1]
    for r, w, local, slowest, ref_rc in res:
        assert w == world and local == r
        assert slowest == pytest.approx(1.25)
    # the reference arm does no work on ranks other than 0
    assert res[1][4] == 0


def test_single_rank_needs_no_process_group():
    bench = _bench()
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (1, 0, 0)
    assert bench.max_over_ranks(1, 3.5) == 3.5
    bench.barrier(1)
