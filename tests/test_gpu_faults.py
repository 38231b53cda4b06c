"""Failures made on the host, with the GPU doing real work around them:
pct_simulate's col / val allocations come after the count and the nonzero
read-back; when the caller's allocator returns NULL there, the call returns
PCT_ENOMEM and every block it had received is freed.  No GPU fault is made."""
import ctypes as C

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


@pytest.mark.parametrize("fail_at", [5, 6])
@pytest.mark.parametrize("prec_name", ["mixed", "f64"])
def test_allocator_failure_after_the_count_frees_everything(pct, fail_at, prec_name):
    prec = {"mixed": pct.PREC_MIXED, "f64": pct.PREC_F64}[prec_name]
    w = W.neo2_2d_spline(n_angles=3, paths_per_angle=200, n=128, h=1.6)
    ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
    live, calls = {}, [0]

    def alloc(nbytes, ctx):
        calls[0] += 1
        if calls[0] == fail_at:
            return None
        t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    def free(p, ctx):
        assert p in live, "freed a block the allocator never handed out"
        live.pop(p)

    af, ff = pct.ALLOC_FN(alloc), pct.FREE_FN(free)
    out = pct.Csr()
    st = pct.lib().pct_simulate(ph.handle, C.byref(geo.c), prec, af, ff, None, C.byref(out),
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == pct.ENOMEM and "allocator returned NULL" in pct.last_error()
    assert calls[0] == 6 and not live
    # the library stays usable
    good = pct.simulate(ph, geo, prec)
    assert good["nnz"] > 0
