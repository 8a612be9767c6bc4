"""The multi-rank timing path of bench.py on two gloo ranks (CPU): barrier,
max-over-ranks elapsed time and the weak-scaling job throughput."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1611_03226_b300 import ranks
    assert ranks.world() == (world, rank, rank)
    ranks.barrier()
    # rank r "took" 1 + r seconds for 300 frames
    value, slowest = ranks.job_throughput(300.0, 1.0 + rank)
    q.put((rank, value, slowest, ranks.max_over_ranks(10.0 * rank)))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, value, slowest, m in out:
        assert slowest == 2.0                 # slowest rank's time
        assert value == 2 * 300.0 / 2.0       # all ranks' units / slowest time
        assert m == 10.0
