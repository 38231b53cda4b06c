"""The system on disk (Sec. II-C: A written to a file that reads back as
CSR, with b and x_true): a single writer, blocks written in any order, two
gloo ranks writing their angle blocks into one shared file, and the checks
on malformed calls.  Host I/O only."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2108_12369_gb300 import shard, workloads as W


@pytest.fixture(scope="module")
def pct():
    from paper_2108_12369_gb300 import build, pct as P
    build.build()
    return P


def _system(orc, n_angles=6, ppa=40):
    w = W.neo2_2d_spline(n_angles=n_angles, paths_per_angle=ppa, n=64, h=3.2)
    ref = orc.simulate(w["phantom"], w["angles"], w["paths_per_angle"], w["model"], w["seed"])
    return w, ref


def _check_equal(got, ref):
    assert np.array_equal(got["row_ptr"], ref["row_ptr"])
    assert np.array_equal(got["col"], ref["col"])
    assert np.array_equal(got["val"], ref["val"].astype(np.float32))
    assert np.array_equal(got["b"], ref["b"].astype(np.float32))
    assert np.array_equal(got["x_true"], ref["x_true"])


def test_single_writer_round_trip(pct, orc, tmp_path):
    w, ref = _system(orc)
    p = tmp_path / "a.pctcsr"
    n = len(ref["b"])
    pct.csr_file_create(p, n, len(ref["x_true"]), int(ref["row_ptr"][-1]), ref["x_true"])
    pct.csr_file_write_rows(p, 0, 0, ref["row_ptr"], ref["col"], ref["val"], ref["b"])
    got = pct.csr_file_read(p)
    assert got["n_rows"] == n and got["nnz"] == ref["row_ptr"][-1]
    _check_equal(got, ref)
    with open(p, "rb") as f:  # sections on 4096-byte boundaries
        head = np.frombuffer(f.read(128)[8:72], dtype="<i8")
    assert all(int(o) % 4096 == 0 for o in head[3:])


def test_blocks_in_any_order(pct, orc, tmp_path):
    w, ref = _system(orc)
    rp = ref["row_ptr"]
    p = tmp_path / "b.pctcsr"
    pct.csr_file_create(p, len(ref["b"]), len(ref["x_true"]), int(rp[-1]), ref["x_true"])
    cuts = [0, 17, 100, 101, len(ref["b"])]
    for r0, r1 in reversed(list(zip(cuts[:-1], cuts[1:]))):
        lo, hi = rp[r0], rp[r1]
        pct.csr_file_write_rows(p, r0, int(lo), rp[r0:r1 + 1] + 1000, ref["col"][lo:hi], ref["val"][lo:hi],
                                ref["b"][r0:r1])  # any base of the local row pointers
    _check_equal(pct.csr_file_read(p), ref)


def test_rejects_blocks_beyond_the_file_and_foreign_files(pct, tmp_path):
    p = tmp_path / "c.pctcsr"
    pct.csr_file_create(p, 4, 3, 5, np.ones(3, np.float32))
    with pytest.raises(pct.PctError):
        pct.csr_file_write_rows(p, 3, 0, [0, 1, 2], [0, 1], [1.0, 1.0], [1.0, 2.0])  # rows 3, 4 of 4
    with pytest.raises(pct.PctError):
        pct.csr_file_write_rows(p, 0, 4, [0, 2], [0, 1], [1.0, 1.0], [1.0])  # nonzeros 4, 5 of 5
    q = tmp_path / "d.bin"
    q.write_bytes(b"x" * 256)
    with pytest.raises(pct.PctError):
        pct.csr_file_write_rows(q, 0, 0, [0, 1], [0], [1.0], [1.0])
    with pytest.raises(pct.PctError):
        pct.csr_file_create(tmp_path / "no" / "dir" / "e", 1, 1, 1, np.ones(1, np.float32))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _writer(rank, world, port, path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        from paper_2108_12369_gb300 import pct as P
        w = W.neo2_2d_spline(n_angles=7, paths_per_angle=30, n=64, h=3.2)
        sw = shard.shard_workload(w, rank, world)
        r0 = sw["first_row"]
        rows = np.arange(r0, r0 + len(sw["angles"]) * sw["paths_per_angle"], dtype=np.int64)
        ph = O.Phantom(w["phantom"])
        x = ph.raster().astype(np.float32)
        sim = O.Simulation(ph, x, w["angles"], w["paths_per_angle"], w["model"], w["seed"])
        rp, col, val, _, b = sim.rows(rows)
        nz0, total = shard.nnz_offsets(int(rp[-1]))
        if rank == 0:
            P.csr_file_create(path, len(w["angles"]) * w["paths_per_angle"], ph.nvox, total, x)
        dist.barrier()  # the file exists before any block is written
        P.csr_file_write_rows(path, r0, nz0, rp, col, val, b)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_write_one_file(pct, orc, tmp_path):
    p = str(tmp_path / "shared.pctcsr")
    mp.spawn(_writer, args=(2, _free_port(), p), nprocs=2, join=True)
    w = W.neo2_2d_spline(n_angles=7, paths_per_angle=30, n=64, h=3.2)
    ref = orc.simulate(w["phantom"], w["angles"], w["paths_per_angle"], w["model"], w["seed"])
    _check_equal(pct.csr_file_read(p), ref)
