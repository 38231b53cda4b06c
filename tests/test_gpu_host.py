"""pct_simulate_host (Sec. II-C: the simulator's output A, b, straight into
host memory): the acquisition in angle blocks, each counted and filled with a
one-block workspace while the previous block's copies run, gives the row
pointers, entries and WEPL of pct_simulate_count + pct_simulate_fill bit for
bit: 2D and 3D, every precision, blocks of one angle and a ragged last block,
a staging buffer of a few rows; the capacity contract (count only, entries
not written, exact nnz returned) and a short workspace."""
import pytest

from paper_2108_12369_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_12369_gb300 import build, pct as P
    build.build()
    return P


def host_sim(pct, ph, geo, prec, apb, staging_bytes, capacity=None):
    ws = torch.empty(pct.simulate_host_workspace_size(ph, geo, prec, apb), dtype=torch.uint8, device="cuda")
    x = torch.empty(ph.nvox, dtype=torch.float32, device="cuda")
    pct.phantom_rasterize(ph, x)
    h_rp = torch.empty(geo.n_rows + 1, dtype=torch.int64, pin_memory=True)
    h_b = torch.empty(max(geo.n_rows, 1), dtype=torch.float32, pin_memory=True)
    staging = torch.empty(staging_bytes, dtype=torch.uint8, device="cuda")
    if capacity == 0:
        h_col = h_val = None
    else:
        h_col = torch.empty(capacity, dtype=torch.int32, pin_memory=True)
        h_val = torch.empty(capacity, dtype=torch.float32, pin_memory=True)
    nnz = pct.simulate_host(ph, geo, prec, apb, ws, x, staging, h_rp, h_col, h_val, h_b)
    return nnz, h_rp, h_col, h_val, h_b[: geo.n_rows]


CASES = {
    "neo2": lambda: W.neo2_2d_spline(n_angles=7, paths_per_angle=500, n=256, h=0.8),
    "head3d": lambda: W.head_3d_spline(n_angles=5, paths_per_angle=2000, n=(48, 48, 40)),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec_name", ["mixed", "lean", "f64"])
@pytest.mark.parametrize("apb", [1, 3])
def test_host_simulation_equals_device_simulation(pct, case, prec_name, apb):
    prec = {"mixed": pct.PREC_MIXED, "lean": pct.PREC_MIXED_LEAN, "f64": pct.PREC_F64}[prec_name]
    w = CASES[case]()
    ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
    dev = pct.simulate(ph, geo, prec)
    nnz = dev["nnz"]
    got, h_rp, h_col, h_val, h_b = host_sim(pct, ph, geo, prec, apb, 96 << 10, capacity=nnz)
    assert got == nnz
    assert torch.equal(h_rp, dev["row_ptr"].cpu())
    assert torch.equal(h_col, dev["col"].cpu())
    assert torch.equal(h_val, dev["val"].cpu())  # bit for bit
    assert torch.equal(h_b, dev["b"].cpu())
    # the one-block workspace (records of one block) is smaller than the whole
    # simulation's; the FP64 form keeps no records
    if apb < len(w["angles"]) and prec != pct.PREC_F64:
        assert pct.simulate_host_workspace_size(ph, geo, prec, apb) < pct.simulate_workspace_size(ph, geo, prec)


def test_capacity_contract(pct):
    w = CASES["head3d"]()
    ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
    dev = pct.simulate(ph, geo, pct.PREC_MIXED)
    nnz = dev["nnz"]
    rp = dev["row_ptr"].cpu()
    # capacity 0: a count with a one-block workspace
    got, h_rp, _, _, _ = host_sim(pct, ph, geo, pct.PREC_MIXED, 2, 1 << 20, capacity=0)
    assert got == nnz and torch.equal(h_rp, rp)
    # one entry short: row pointers complete, the exact count returned
    got, h_rp, _, _, _ = host_sim(pct, ph, geo, pct.PREC_MIXED, 2, 1 << 20, capacity=nnz - 1)
    assert got == nnz and torch.equal(h_rp, rp)
    # a larger capacity than needed
    got, h_rp, h_col, h_val, _ = host_sim(pct, ph, geo, pct.PREC_MIXED, 2, 1 << 20, capacity=nnz + 1000)
    assert got == nnz and torch.equal(h_col[:nnz], dev["col"].cpu()) and torch.equal(h_val[:nnz], dev["val"].cpu())


def test_short_workspace_and_staging(pct):
    w = CASES["neo2"]()
    ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
    need = pct.simulate_host_workspace_size(ph, geo, pct.PREC_MIXED, 2)
    ws = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    x = torch.empty(ph.nvox, dtype=torch.float32, device="cuda")
    h_rp = torch.empty(geo.n_rows + 1, dtype=torch.int64)
    h_b = torch.empty(geo.n_rows, dtype=torch.float32)
    staging = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(pct.PctError) as e:
        pct.simulate_host(ph, geo, pct.PREC_MIXED, 2, ws, x, staging, h_rp, None, None, h_b)
    assert e.value.status == pct.ENOMEM
    # a staging half smaller than one row
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    pct.phantom_rasterize(ph, x)
    h_col = torch.empty(10_000_000, dtype=torch.int32)
    h_val = torch.empty(10_000_000, dtype=torch.float32)
    with pytest.raises(pct.PctError) as e:
        pct.simulate_host(ph, geo, pct.PREC_MIXED, 2, ws, x, torch.empty(1024, dtype=torch.uint8, device="cuda"),
                          h_rp, h_col, h_val, h_b)
    assert e.value.status == pct.EINVAL
