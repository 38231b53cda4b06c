"""Acquisition-structured partition (Sec. IV: blocks of projection angles per
GPU): each block simulated on its own, with the global index of its first row,
gives exactly its rows of the whole acquisition, so the blocks' CSRs
concatenate, with nonzero offsets from the blocks' counts, into the CSR of one
call over all angles -- bit for bit, in both precisions."""
import pytest

from paper_2108_12369_gb300 import shard, workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_12369_gb300 import build, pct as P
    build.build()
    return P


CASES = {
    "neo2_2d": lambda: W.neo2_2d_spline(n_angles=11, paths_per_angle=700, n=256, h=0.8),
    "head_3d": lambda: W.head_3d_spline(n_angles=7, paths_per_angle=900, n=(60, 60, 48), h=(3.3, 3.3, 3.4)),
}


def _sim(pct, w, prec):
    out = pct.simulate(pct.Phantom(w["phantom"]), pct.GeometryArgs(w), prec)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec_name", ["mixed", "f64"])
@pytest.mark.parametrize("world", [2, 3])
def test_angle_blocks_concatenate_into_the_whole_acquisition(pct, case, prec_name, world):
    prec = {"mixed": pct.PREC_MIXED, "f64": pct.PREC_F64}[prec_name]
    w = CASES[case]()
    full = _sim(pct, w, prec)
    rp, cols, vals, bs, nz0 = [torch.zeros(1, dtype=torch.int64, device="cuda")], [], [], [], 0
    for r in range(world):
        sw = shard.shard_workload(w, r, world)
        assert sw["first_row"] == shard.row_base(w, r, world)
        part = _sim(pct, sw, prec)
        rp.append(part["row_ptr"][1:] + nz0)
        nz0 += part["nnz"]
        cols.append(part["col"])
        vals.append(part["val"])
        bs.append(part["b"])
    assert nz0 == full["nnz"]
    assert torch.equal(torch.cat(rp), full["row_ptr"])
    assert torch.equal(torch.cat(cols), full["col"])
    assert torch.equal(torch.cat(vals), full["val"])
    assert torch.equal(torch.cat(bs), full["b"])


def test_block_without_row_base_differs(pct):
    """The row base is what makes a block reproduce its rows: the same angles
    keyed from row 0 give other protons."""
    w = CASES["neo2_2d"]()
    full = _sim(pct, w, pct.PREC_MIXED)
    sw = shard.shard_workload(w, 1, 2)
    base = sw["first_row"]
    alone = _sim(pct, dict(sw, first_row=0), pct.PREC_MIXED)
    n = len(sw["angles"]) * sw["paths_per_angle"]
    assert not torch.equal(alone["b"], full["b"][base:base + n])


def test_matrix_free_forward_of_a_block_equals_its_rows(pct):
    w = CASES["head_3d"]()
    ph = pct.Phantom(w["phantom"])
    x = torch.empty(ph.nvox, dtype=torch.float32, device="cuda")
    pct.phantom_rasterize(ph, x)
    geo = pct.GeometryArgs(w)
    n = geo.n_rows
    ws = torch.empty(pct.projector_workspace_size(ph, geo, n), dtype=torch.uint8, device="cuda")
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    pct.forward(ph, geo, None, 0, n, x, y, ws)
    sw = shard.shard_workload(w, 1, 3)
    sgeo = pct.GeometryArgs(sw)
    ys = torch.empty(sgeo.n_rows, dtype=torch.float32, device="cuda")
    wss = torch.empty(pct.projector_workspace_size(ph, sgeo, sgeo.n_rows), dtype=torch.uint8, device="cuda")
    pct.forward(ph, sgeo, None, 0, sgeo.n_rows, x, ys, wss)
    torch.cuda.synchronize()
    b = sw["first_row"]
    assert torch.equal(ys, y[b:b + sgeo.n_rows])
