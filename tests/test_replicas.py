"""Multi-GPU host logic, on CPU with gloo (world size 2): the planner shards as
independent replicas -- each rank plans its own requests, no data-path
collective -- so the only cross-rank steps are the barrier and the max-over-ranks
timing reduction of the benchmark, and the per-rank request sets must be disjoint."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    reqs = bench.workload_requests(6, rank)
    seeds = torch.tensor([[w.path_seed, w.cand_seed] for w in reqs], dtype=torch.int64)
    gathered = [torch.zeros_like(seeds) for _ in range(world)]
    dist.all_gather(gathered, seeds)
    t = torch.tensor([10.0 * (rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    if rank == 0:
        out.put((torch.cat(gathered).tolist(), float(t.item())))
    dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    seeds, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = [tuple(s) for s in seeds]
    assert len(flat) == 12 and len(set(flat)) == 12   # no request planned twice
    assert tmax == 20.0                                # slowest rank sets the step time
