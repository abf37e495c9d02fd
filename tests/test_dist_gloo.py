"""The benchmark's multi-rank plumbing on two CPU ranks (gloo).

`bench.py --gpus N` runs one process per GPU as independent replicas: the
product path exchanges nothing between GPUs, so the only cross-rank steps are
a barrier on both sides of the timed region, the maximum of the ranks' times
and the whole-job throughput computed from it; the reference arm runs on
rank 0 alone. These are the same functions the GPU runs use (there over NCCL),
exercised here on host cores with world size 2."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# per-rank time of the "timed region" in this test, in ms
RANK_MS = (12.5, 20.0)


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    try:
        w, r, local = bench.dist_setup(None, backend="gloo")
        bench.barrier(w)
        slowest = bench.allreduce_max(RANK_MS[r], w)
        value = bench.job_value(1e9, 4, slowest, w)
        # the reference arm: every rank but 0 returns at once, without work or output
        skipped = r != 0 and bench.run_reference(None, w, r) is None
        bench.barrier(w)
        out.put((r, w, local, slowest, value, skipped))
    finally:
        if dist.is_initialized():
            dist.destroy_process_group()


def test_two_gloo_ranks_barrier_max_and_job_value():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(out.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    want_ms = max(RANK_MS)
    # whole-job value: both ranks' work over the slower rank's time
    want_value = 2 * 1e9 * 4 / (want_ms / 1e3) / 1e9
    for r, (rank, world, local, slowest, value, skipped) in enumerate(got):
        assert (rank, world, local) == (r, 2, r)
        assert slowest == want_ms
        assert abs(value - want_value) <= 1e-9 * want_value
        assert skipped == (r != 0)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        assert bench.dist_setup(None) == (1, 0, 0)
        bench.barrier(1)
        assert bench.allreduce_max(7.25, 1) == 7.25
        assert bench.job_value(2e9, 3, 1500.0, 1) == 4.0
    finally:
        os.environ.update(env)
