"""pct_simulate_fill_host (Sec. II-C: the simulator's output A, b) writes the
same row pointers, entries and WEPL into host memory as pct_simulate_fill
does into device memory, block by block through a staging buffer: many
blocks with a ragged last one, a single block, both precisions, and the
rejection of a staging buffer too small for one row."""
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


def host_fill(pct, ph, geo, prec, staging_bytes):
    ws = torch.empty(pct.simulate_workspace_size(ph, geo, prec), dtype=torch.uint8, device="cuda")
    x = torch.empty(ph.nvox, dtype=torch.float32, device="cuda")
    rp = torch.empty(geo.n_rows + 1, dtype=torch.int64, device="cuda")
    pct.phantom_rasterize(ph, x)
    pct.simulate_count(ph, geo, prec, ws, rp)
    nnz = int(rp[-1])
    h_rp = torch.empty(geo.n_rows + 1, dtype=torch.int64, pin_memory=True)
    h_col = torch.empty(max(nnz, 1), dtype=torch.int32, pin_memory=True)
    h_val = torch.empty(max(nnz, 1), dtype=torch.float32, pin_memory=True)
    h_b = torch.empty(max(geo.n_rows, 1), dtype=torch.float32, pin_memory=True)
    staging = torch.empty(staging_bytes, dtype=torch.uint8, device="cuda")
    pct.simulate_fill_host(ph, geo, prec, ws, rp, x, staging, h_rp, h_col, h_val, h_b)
    return h_rp, h_col[:nnz], h_val[:nnz], h_b[: geo.n_rows]


@pytest.mark.parametrize("prec_name", ["mixed", "f64"])
@pytest.mark.parametrize("staging_bytes", [64 << 10, 256 << 20])
def test_host_fill_equals_device_fill(pct, prec_name, staging_bytes):
    prec = {"mixed": pct.PREC_MIXED, "f64": pct.PREC_F64}[prec_name]
    w = W.neo2_2d_spline(n_angles=24, paths_per_angle=400, n=256, h=0.8)
    ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
    dev = pct.simulate(ph, geo, prec)
    h_rp, h_col, h_val, h_b = host_fill(pct, ph, geo, prec, staging_bytes)
    assert torch.equal(h_rp, dev["row_ptr"].cpu())
    assert torch.equal(h_col, dev["col"].cpu())
    assert torch.equal(h_val, dev["val"].cpu())  # bit for bit
    assert torch.equal(h_b, dev["b"].cpu())


def test_host_fill_3d_blocks(pct):
    w = W.head_3d_spline(n_angles=4, paths_per_angle=3000, n=(48, 48, 40))
    ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
    dev = pct.simulate(ph, geo, pct.PREC_MIXED)
    h_rp, h_col, h_val, h_b = host_fill(pct, ph, geo, pct.PREC_MIXED, 96 << 10)
    assert torch.equal(h_rp, dev["row_ptr"].cpu())
    assert torch.equal(h_col, dev["col"].cpu())
    assert torch.equal(h_val, dev["val"].cpu())
    assert torch.equal(h_b, dev["b"].cpu())


def test_host_fill_rejects_staging_smaller_than_a_row(pct):
    w = W.neo2_2d_spline(n_angles=2, paths_per_angle=200, n=256, h=0.8)
    ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
    for nbytes in (1024, 2 * 1056):  # no room at all; 128 entries per half, rows hold more
        with pytest.raises(pct.PctError):
            host_fill(pct, ph, geo, pct.PREC_MIXED, nbytes)


def test_host_fill_rejects_null_entry_buffers_before_any_fill(pct):
    """With nonzeros to write, a NULL col_host or val_host is refused once the
    row pointers are read back, before any fill is launched."""
    import ctypes as C
    w = W.neo2_2d_spline(n_angles=2, paths_per_angle=50, n=128, h=1.6)
    ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
    ws = torch.empty(pct.simulate_workspace_size(ph, geo, pct.PREC_MIXED), dtype=torch.uint8, device="cuda")
    x = torch.empty(ph.nvox, dtype=torch.float32, device="cuda")
    rp = torch.empty(geo.n_rows + 1, dtype=torch.int64, device="cuda")
    pct.phantom_rasterize(ph, x)
    pct.simulate_count(ph, geo, pct.PREC_MIXED, ws, rp)
    assert int(rp[-1]) > 0
    h_rp = torch.empty(geo.n_rows + 1, dtype=torch.int64, pin_memory=True)
    h = torch.empty(int(rp[-1]), dtype=torch.float32, pin_memory=True)
    h_b = torch.full((geo.n_rows,), -7.0, dtype=torch.float32, pin_memory=True)
    staging = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    L = pct.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for col_p, val_p in ((None, h.data_ptr()), (h.data_ptr(), None)):
        st = L.pct_simulate_fill_host(ph.handle, C.byref(geo.c), pct.PREC_MIXED, C.c_void_p(ws.data_ptr()),
                                      ws.numel(), C.c_void_p(rp.data_ptr()), C.c_void_p(x.data_ptr()),
                                      C.c_void_p(staging.data_ptr()), staging.numel(),
                                      C.c_void_p(h_rp.data_ptr()), C.c_void_p(col_p), C.c_void_p(val_p),
                                      C.c_void_p(h_b.data_ptr()), stream)
        assert st == pct.EINVAL and b"NULL col_host or val_host" in L.pct_last_error()
    torch.cuda.synchronize()
    assert torch.all(h_b == -7.0)  # nothing was filled
