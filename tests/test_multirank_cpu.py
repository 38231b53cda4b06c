"""The multi-GPU host logic with two gloo ranks on CPU: angle-block shards
reassemble the single-process CSR exactly (through the all-gathered nonzero
offsets), the summed shard adjoints equal the full A^T r, and timings reduce
to the maximum.  The per-shard rows come from the CPU oracle; each rank also
builds the library's geometry of its block (global first row) and has the
library accept it on the host.  The GPU side of the same partition (blocks
concatenating into the whole CSR bit for bit) is tests/test_gpu_shards.py."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2108_12369_gb300 import shard, workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        import scipy.sparse as sp
        w = W.neo2_2d_spline(n_angles=7, paths_per_angle=60, n=96, h=2.0)
        rows = np.arange(shard.row_base(w, rank, world),
                         shard.row_base(w, rank, world) + len(shard.shard_workload(w, rank, world)["angles"])
                         * w["paths_per_angle"], dtype=np.int64)
        ph = O.Phantom(w["phantom"])
        x = ph.raster().astype(np.float32)
        sim = O.Simulation(ph, x, w["angles"], w["paths_per_angle"], w["model"], w["seed"])
        rp, col, val, bc, bn = sim.rows(rows)
        # the library's view of this rank's block: its geometry carries the
        # global first row, which keys the block's random numbers
        from paper_2108_12369_gb300 import pct as P
        sw = shard.shard_workload(w, rank, world)
        geo = P.GeometryArgs(sw)
        assert geo.c.first_row == rows[0] and geo.n_rows == len(rows)
        assert list(geo.angles) == list(w["angles"][shard.angle_shard(7, rank, world)[0]:][:len(sw["angles"])])
        ph_lib = P.Phantom(w["phantom"])
        assert P.simulate_workspace_size(ph_lib, geo, P.PREC_MIXED) > 0  # accepted on the host
        off, total = shard.nnz_offsets(int(rp[-1]))
        # the shard's adjoint contribution
        A = sp.csr_matrix((val, col, rp), shape=(len(rows), ph.nvox))
        r = np.cos(rows.astype(np.float64))
        g = torch.from_numpy(A.T @ r)
        shard.reduce_adjoint(g)
        t = shard.max_over_ranks(0.5 + rank)
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), rows=rows, rp=rp, col=col, val=val, b=bn, off=off,
                 total=total, g=g.numpy(), t=t)
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_reassemble_the_full_system(tmp_path):
    from paper_2108_12369_gb300 import build
    build.build()  # the ranks load the library's host side
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    parts = [np.load(tmp_path / f"r{k}.npz") for k in range(world)]
    from oracle import oracle as O
    import scipy.sparse as sp
    w = W.neo2_2d_spline(n_angles=7, paths_per_angle=60, n=96, h=2.0)
    full = O.simulate(w["phantom"], w["angles"], w["paths_per_angle"], w["model"], w["seed"])
    # angle blocks are contiguous and cover every row once
    assert np.array_equal(np.concatenate([p["rows"] for p in parts]), np.arange(len(full["b"])))
    # all-gathered offsets place each shard's nonzeros
    assert parts[0]["off"] == 0 and parts[1]["off"] == parts[0]["rp"][-1]
    assert parts[0]["total"] == parts[1]["total"] == full["row_ptr"][-1]
    col = np.concatenate([p["col"] for p in parts])
    val = np.concatenate([p["val"] for p in parts])
    rp = np.concatenate([parts[0]["rp"][:-1], parts[1]["rp"] + parts[1]["off"]])
    assert np.array_equal(rp, full["row_ptr"]) and np.array_equal(col, full["col"])
    assert np.array_equal(val, full["val"])
    assert np.array_equal(np.concatenate([p["b"] for p in parts]), full["b"])
    # summed shard adjoints equal the full adjoint, identical on both ranks
    A = sp.csr_matrix((full["val"], full["col"], full["row_ptr"]), shape=(len(full["b"]), 96 * 96))
    want = A.T @ np.cos(np.arange(len(full["b"]), dtype=np.float64))
    for p in parts:
        assert np.allclose(p["g"], want, rtol=1e-12, atol=1e-12)
    assert parts[0]["t"] == parts[1]["t"] == 1.5


@pytest.mark.parametrize("n,world", [(7, 2), (360, 8), (3, 4), (0, 2)])
def test_angle_shards_partition(n, world):
    blocks = [shard.angle_shard(n, r, world) for r in range(world)]
    assert blocks[0][0] == 0 and blocks[-1][1] == n
    for (a0, a1), (b0, b1) in zip(blocks[:-1], blocks[1:]):
        assert a1 == b0
    sizes = [b - a for a, b in blocks]
    assert max(sizes) - min(sizes) <= 1
