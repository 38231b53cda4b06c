"""Host-side logic for running one acquisition on several GPUs.

Protons are independent, so the path shards without any exchange on the
data path: each rank simulates a contiguous block of projection angles (the
acquisition-structured partition the paper proposes for GPU clusters,
Sec. IV) with the full phantom.  The only exchanges are
  - an all-gather of the per-rank nonzero counts, to place the local CSR
    blocks in one global CSR (row offsets are known from the angle blocks);
  - a sum-reduction of A^T r over the row shards for the adjoint;
  - a max-reduction of the step time for the benchmark.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def angle_shard(n_angles: int, rank: int, world: int):
    """[k0, k1): the contiguous block of angles of `rank` (sizes differ by at most 1)."""
    base, extra = divmod(n_angles, world)
    k0 = rank * base + min(rank, extra)
    return k0, k0 + base + (1 if rank < extra else 0)


def shard_workload(w: dict, rank: int, world: int) -> dict:
    """The workload restricted to this rank's angles.  Its local row i is
    global row first_row + i of the full acquisition (first_row =
    row_base()), and the library keys each proton's random numbers by that
    global index, so the shard's rows are exactly those rows of the whole
    acquisition."""
    k0, k1 = angle_shard(len(w["angles"]), rank, world)
    s = dict(w)
    s["angles"] = w["angles"][k0:k1]
    s["first_row"] = int(w.get("first_row", 0)) + k0 * int(w["paths_per_angle"])
    return s


def row_base(w: dict, rank: int, world: int) -> int:
    k0, _ = angle_shard(len(w["angles"]), rank, world)
    return k0 * int(w["paths_per_angle"])


def nnz_offsets(local_nnz: int, group=None):
    """Exclusive prefix of the ranks' nonzero counts (all-gather), and the total."""
    world = dist.get_world_size(group)
    t = torch.tensor([int(local_nnz)], dtype=torch.int64)
    if torch.cuda.is_available() and dist.get_backend(group) == "nccl":
        t = t.cuda()
    out = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(out, t, group=group)
    counts = [int(v.item()) for v in out]
    rank = dist.get_rank(group)
    return sum(counts[:rank]), sum(counts)


def reduce_adjoint(g: torch.Tensor, group=None) -> torch.Tensor:
    """g = sum over ranks of their A_rank^T r_rank (in place)."""
    dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
    return g


def max_over_ranks(value: float, device=None, group=None) -> float:
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
