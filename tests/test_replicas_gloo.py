"""Multi-GPU is replicas only: each rank solves its own LPs, no collective on
the data path; the job's time is the maximum over ranks.  This runs that
logic of bench.py with world size 2 on the gloo backend (CPU processes), the
oracle standing in for each rank's solver."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        B = 2
        offs = bench.replica_offsets(rank, B)
        objs, ms = [], 0.0
        for o in offs:
            lp = bench.make_lp("tiny", seed_offset=o)
            x, y, s, info = oracle.lp_solve_lp(lp, inner_sweeps=1)
            assert info["status_name"] == "OK"
            objs.append(info["obj_primal"])
            ms += 10.0 * (rank + 1)          # a stand-in step time per rank
        tmax = bench.max_over_ranks(ms, dist)
        gathered = [None] * world
        dist.all_gather_object(gathered, (offs, objs, ms))
        if rank == 0:
            out.put((gathered, tmax, bench.weak_throughput(world, B, 1, tmax)))
    finally:
        dist.destroy_process_group()


def test_replicas_two_ranks_gloo():
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, tmax, value = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    offs = [g[0] for g in gathered]
    assert set(offs[0]).isdisjoint(offs[1])            # every rank solves its own LPs
    assert len({round(o, 9) for g in gathered for o in g[1]}) == 4   # four different LPs
    assert tmax == max(g[2] for g in gathered) == 40.0  # the job's time is the slowest rank's
    assert value == pytest.approx(2 * 2 * 1 / 0.040)   # whole-job LPs/s over both ranks
