"""The bench's multi-rank host path on CPU: two gloo ranks, the environment contract of
torchrun (RANK / WORLD_SIZE / LOCAL_RANK, rendezvous on 127.0.0.1), the job time as the
maximum over ranks, and the reference arm running on rank 0 only."""
import os
import socket

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    r, w, lr = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    ms = bench.max_over_ranks(10.0 + 5.0 * r, w, "cpu")
    # a non-zero rank's reference arm does no work and prints nothing
    ref = bench.run_reference(None, r) if r != 0 else None
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, lr, ms, ref))


def test_two_gloo_ranks_take_the_slowest_time():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out) and [o[2] for o in out] == [0, 1]
    assert all(o[3] == 15.0 for o in out)
    assert out[1][4] is None


def test_single_rank_time_is_unchanged():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
