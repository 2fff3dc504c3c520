"""One process per GPU of a node: the plumbing around the solve.

The collision solve is pointwise (every node is an independent problem), so
ranks share nothing on the data path: each rank solves its own nodes, drawn
from its own seed.  Ranks meet only to time a step (a barrier on both sides,
the maximum of the elapsed times) and to add up counts for the report, and a
rate is the units of all ranks over that maximum time (weak scaling).
torch.distributed provides the process group: NCCL for CUDA tensors, gloo on
the CPU.
"""

import os


def world():
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0 without one)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def workload_seed(rank, stream=0):
    """Seed of rank `rank`'s inputs for workload stream `stream` (distinct across ranks and streams)."""
    return 1000 * stream + rank


def weak_scaling_value(units_all_ranks, steps, max_ms):
    """Rate of the whole job: the units every rank processed per step, over the slowest rank's time."""
    return units_all_ranks * steps / (max_ms * 1e-3)


class Group:
    """Barrier and reductions over the ranks; a no-op when the world has one rank."""

    def __init__(self, device=None, backend=None):
        import torch
        self.ws, self.rank, self.local = world()
        self.device = device if device is not None else torch.device("cpu")
        self.cuda = self.device.type == "cuda"
        if self.ws > 1:
            import torch.distributed as dist
            if backend is None:
                backend = "nccl" if self.cuda else "gloo"
            kw = dict(device_id=self.device) if (self.cuda and backend == "nccl") else {}
            dist.init_process_group(backend, **kw)

    def barrier(self):
        import torch
        if self.cuda:
            torch.cuda.synchronize()
        if self.ws > 1:
            torch.distributed.barrier()
        if self.cuda:
            torch.cuda.synchronize()

    def allmax(self, x):
        if self.ws == 1:
            return x
        import torch
        t = torch.tensor([float(x)], device=self.device, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    def allsum(self, x):
        if self.ws == 1:
            return x
        import torch
        t = torch.tensor([int(x)], device=self.device, dtype=torch.int64)
        torch.distributed.all_reduce(t)
        return int(t.item())

    def close(self):
        if self.ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
