"""The C ABI without a GPU: the library builds, exports every function
include/pct.h declares, and its host-only calls validate arguments."""
import ctypes as C
import re
from pathlib import Path

import pytest

from paper_2108_12369_gb300 import workloads as W

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def pct():
    from paper_2108_12369_gb300 import build, pct as P
    build.build()
    return P


def declared_functions():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = h.read_text()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(pct_[a-z0-9_]+)\s*\(", text))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_every_declared_function_is_exported(pct):
    L = pct.lib()
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/ but not exported"
    assert set(pct.EXPORTS) <= set(names)


def test_version(pct):
    assert "sm_103a" in pct.version()


def test_phantom_create_validates(pct):
    ph = pct.Phantom(W.phantom(2, (200, 200), (1.0, 1.0), skin=False))
    assert ph.nvox == 40000
    ph3 = pct.Phantom(W.phantom(3, (20, 30, 40), (1.0, 1.0, 1.0), skin=True))
    assert ph3.nvox == 24000
    for bad in ({"dim": 4}, {"n": (0, 10, 1)}, {"h": (1.0, -1.0, 1.0)}, {"raster": 7}, {"kind": 9},
                {"raster": W.AREA, "area_samples": 0}, {"raster": W.AREA, "area_samples": 65}):
        d = dict(W.phantom(2, (10, 10), (1.0, 1.0), skin=False), **bad)
        with pytest.raises(pct.PctError) as e:
            pct.Phantom(d)
        assert e.value.status == pct.EINVAL
    d = W.phantom(2, (10, 10), (1.0, 1.0), skin=False)
    d["regions"] = d["regions"] * 4  # 20 > 16 regions
    with pytest.raises(ValueError):
        pct.Phantom(d)
    d = W.phantom(2, (10, 10), (1.0, 1.0), skin=False)
    d["regions"] = [dict(d["regions"][0], a=(0.0, 1.0, 1.0))]
    with pytest.raises(pct.PctError):
        pct.Phantom(d)
    assert "semi-axis" in pct.last_error()


def test_workspace_size_and_geometry_checks(pct):
    w = W.neo2_2d_spline(n_angles=10, paths_per_angle=100)
    ph = pct.Phantom(w["phantom"])
    geo = pct.GeometryArgs(w)
    for prec in (pct.PREC_MIXED, pct.PREC_F64):
        n = pct.simulate_workspace_size(ph, geo, prec)
        assert n >= 10 * 16 + 33 * 32
    bad_models = [dict(w["model"], model=5), dict(w["model"], spline_segments=0),
                  dict(w["model"], rho=1.5), dict(w["model"], sigma_lat=-1.0),
                  dict(w["model"], t_range=(5.0, -5.0)), dict(w["model"], chord=3),
                  dict(w["model"], mcs=2), dict(w["model"], mcs=W.MCS_HIGHLAND, beam_mev=0.0),
                  dict(w["model"], mcs=W.MCS_HIGHLAND, x0_mm=float("nan"))]
    for m in bad_models:
        g = pct.GeometryArgs(dict(w, model=m))
        with pytest.raises(pct.PctError) as e:
            pct.simulate_workspace_size(ph, g, pct.PREC_F64)
        assert e.value.status == pct.EINVAL
    with pytest.raises(pct.PctError):
        pct.simulate_workspace_size(ph, geo, 7)
    w0 = dict(w, angles=W.angles(0))
    assert pct.simulate_workspace_size(ph, pct.GeometryArgs(w0), pct.PREC_F64) > 0


def test_batch_workspace_size_validates(pct):
    ws = [W.neo1_2d_straight(n_angles=3, paths_per_angle=10), W.head_3d_spline(n_angles=2, paths_per_angle=5)]
    assert pct.batch_workspace_size(ws) > 0
    bad = [dict(ws[0], model=dict(ws[0]["model"], model=9))]
    with pytest.raises(pct.PctError) as e:
        pct.batch_workspace_size(bad)
    assert e.value.status == pct.EINVAL


def test_fill_host_validates_before_any_device_work(pct):
    """pct_simulate_fill_host checks its pointers on the host (no GPU needed)."""
    w = W.neo2_2d_spline(n_angles=2, paths_per_angle=10, n=64, h=3.2)
    ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
    L = pct.lib()
    st = L.pct_simulate_fill_host(ph.handle, C.byref(geo.c), pct.PREC_MIXED, None, 0, None, None, None, 0,
                                  None, None, None, None, None)
    assert st == pct.EINVAL and b"NULL row pointers" in L.pct_last_error()
    buf = (C.c_int64 * 64)()
    p = C.cast(buf, C.c_void_p)
    st = L.pct_simulate_fill_host(ph.handle, C.byref(geo.c), pct.PREC_MIXED, None, 0, p, None, None, 0,
                                  p, None, None, None, None)
    assert st == pct.EINVAL and b"NULL argument" in L.pct_last_error()
    odd = C.c_void_p((p.value + 255) // 256 * 256 + 8)  # not 256-byte aligned (never dereferenced)
    st = L.pct_simulate_fill_host(ph.handle, C.byref(geo.c), pct.PREC_MIXED, None, 0, p, p, odd, 1 << 20,
                                  p, p, p, p, None)
    assert st == pct.EINVAL and b"aligned" in L.pct_last_error()


def test_simulate_host_validates_before_any_device_work(pct):
    """pct_simulate_host checks its arguments and workspace on the host; its
    workspace is one angle block's (no GPU needed)."""
    w = W.head_3d_spline(n_angles=9, paths_per_angle=100, n=(32, 32, 24))
    ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
    L = pct.lib()
    sizes = [pct.simulate_host_workspace_size(ph, geo, pct.PREC_MIXED, k) for k in (1, 3, 9, 20)]
    assert sizes[0] < sizes[1] < sizes[2] == sizes[3]
    assert sizes[1] < pct.simulate_workspace_size(ph, geo, pct.PREC_MIXED)
    with pytest.raises(pct.PctError) as e:
        pct.simulate_host_workspace_size(ph, geo, pct.PREC_MIXED, 0)
    assert e.value.status == pct.EINVAL
    buf = (C.c_int64 * 64)()
    p = C.cast(buf, C.c_void_p)
    nnz = C.c_int64(-1)

    stg = C.c_void_p((p.value + 255) // 256 * 256)  # fake device staging address (never dereferenced)
    odd = C.c_void_p(stg.value + 8)  # not 256-byte aligned

    def call(apb, ws_bytes, x, staging, rp, col, cap, out, why):
        st = L.pct_simulate_host(ph.handle, C.byref(geo.c), pct.PREC_MIXED, apb, p, ws_bytes, x, staging, 1 << 20,
                                 rp, col, col, p, cap, out, None)
        assert why.encode() in L.pct_last_error(), (why, L.pct_last_error())
        return st
    assert call(0, 1 << 40, p, stg, p, p, 10, C.byref(nnz), "angles_per_block") == pct.EINVAL
    assert call(2, 1 << 40, p, stg, None, p, 10, C.byref(nnz), "NULL row_ptr_host") == pct.EINVAL
    assert call(2, 1 << 40, p, stg, p, p, 10, None, "nnz_out") == pct.EINVAL
    assert call(2, 1 << 40, p, stg, p, p, -1, C.byref(nnz), "nnz_capacity") == pct.EINVAL
    assert call(2, 1 << 40, None, stg, p, p, 10, C.byref(nnz), "NULL argument") == pct.EINVAL
    assert call(2, 1 << 40, p, stg, p, None, 10, C.byref(nnz), "NULL col_host") == pct.EINVAL
    assert call(2, 1 << 40, p, odd, p, p, 10, C.byref(nnz), "aligned") == pct.EINVAL
    assert L.pct_simulate_check(None, C.byref(nnz), None) == pct.EINVAL
    assert L.pct_simulate_check(p, None, None) == pct.EINVAL
    need = pct.simulate_host_workspace_size(ph, geo, pct.PREC_MIXED, 2)
    buf[0] = 7
    assert call(2, need - 1, p, stg, p, None, 0, C.byref(nnz), "workspace") == pct.ENOMEM
    assert nnz.value == 0 and buf[0] == 0


class _FakeAllocator:
    """Allocator callbacks that hand out fake, never-dereferenced addresses and
    return NULL on call number `fail_at` (1-based); counts every call."""

    def __init__(self, pct, fail_at):
        self.fail_at, self.calls, self.live, self.freed = fail_at, 0, set(), []

        def alloc(nbytes, ctx):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            p = 0x7f0000000000 + 0x1000000 * self.calls
            self.live.add(p)
            return p

        def free(p, ctx):
            self.freed.append(p)
            self.live.discard(p)

        self.af, self.ff = pct.ALLOC_FN(alloc), pct.FREE_FN(free)


@pytest.mark.parametrize("fail_at", [1, 2, 3, 4])
def test_simulate_allocator_failure_frees_everything(pct, fail_at):
    """pct_simulate allocates its workspace, x_true, row pointers and b first;
    when the caller's allocator returns NULL for any of them the call returns
    PCT_ENOMEM before any device work and frees every block it received."""
    w = W.neo2_2d_spline(n_angles=3, paths_per_angle=20, n=64, h=3.2)
    ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
    fa = _FakeAllocator(pct, fail_at)
    out = pct.Csr()
    st = pct.lib().pct_simulate(ph.handle, C.byref(geo.c), pct.PREC_MIXED, fa.af, fa.ff, None, C.byref(out), None)
    assert st == pct.ENOMEM and "allocator returned NULL" in pct.last_error()
    assert fa.calls == 4  # the four up-front blocks, nothing after the failure
    assert not fa.live and len(fa.freed) == 3 and len(set(fa.freed)) == 3
    assert out.row_ptr is None and out.col is None  # nothing handed out


@pytest.mark.parametrize("prec_name", ["mixed", "f64"])
def test_workspace_one_byte_short_is_refused_before_any_device_work(pct, prec_name):
    prec = {"mixed": pct.PREC_MIXED, "f64": pct.PREC_F64}[prec_name]
    w = W.head_3d_spline(n_angles=2, paths_per_angle=30, n=(20, 20, 16), h=(10.0, 10.0, 10.0))
    ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
    need = pct.simulate_workspace_size(ph, geo, prec)
    fake = C.c_void_p(0x7f0000000000)  # never dereferenced: the size check comes first
    L = pct.lib()
    st = L.pct_simulate_count(ph.handle, C.byref(geo.c), prec, fake, need - 1, fake, None)
    assert st == pct.ENOMEM and "smaller than" in pct.last_error()
    st = L.pct_simulate_fill(ph.handle, C.byref(geo.c), prec, fake, need - 1, fake, fake, fake, fake, fake, None)
    assert st == pct.ENOMEM
    pneed = pct.projector_workspace_size(ph, geo, 10, prec)
    st = L.pct_forward(ph.handle, C.byref(geo.c), None, prec, 0, 10, fake, fake, fake, pneed - 1, None)
    assert st == pct.ENOMEM
    st = L.pct_adjoint(ph.handle, C.byref(geo.c), None, prec, 0, 10, fake, fake, fake, pneed - 1, None)
    assert st == pct.ENOMEM


def test_first_row_is_validated(pct):
    w = W.neo2_2d_spline(n_angles=4, paths_per_angle=10, n=64, h=3.2)
    ph = pct.Phantom(w["phantom"])
    assert pct.simulate_workspace_size(ph, pct.GeometryArgs(dict(w, first_row=123456789)), pct.PREC_MIXED) > 0
    for bad in (-1, (1 << 62) - 39):
        with pytest.raises(pct.PctError) as e:
            pct.simulate_workspace_size(ph, pct.GeometryArgs(dict(w, first_row=bad)), pct.PREC_MIXED)
        assert e.value.status == pct.EINVAL and "first_row" in pct.last_error()


def test_lean_form_workspace(pct):
    for w in (W.neo2_2d_spline(n_angles=10, paths_per_angle=1000), W.head_3d_spline(n_angles=4, paths_per_angle=1000)):
        ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
        full = pct.simulate_workspace_size(ph, geo, pct.PREC_MIXED)
        lean = pct.simulate_workspace_size(ph, geo, pct.PREC_MIXED_LEAN)
        assert lean < 0.25 * full
        assert lean >= geo.n_rows * (160 + 184 + 2 * 112 + 1)  # row records, lead segments, row flags
    assert pct.batch_workspace_size(W.batch_instances(count=4, max_paths=50000), lean=True) < \
        pct.batch_workspace_size(W.batch_instances(count=4, max_paths=50000))
