"""Worker bodies for the multi-process CPU tests (importable by spawned
children)."""
import os


def max_over_ranks_worker(rank: int, world: int, port: int, queue) -> None:
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slowest = bench.max_over_ranks(10.0 + 3.0 * rank, dist, "cpu")
    rate = bench.job_rate(1000.0, world, slowest)
    queue.put((rank, slowest, rate, bench.dist_env()))
    dist.barrier()
    dist.destroy_process_group()
