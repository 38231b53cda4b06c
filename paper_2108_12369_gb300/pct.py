"""Python binding of libpct (include/pct.h): argument marshalling only.

Every computation runs in the CUDA library; this module turns PyTorch
tensors into device pointers and workload dicts into the C structs.  It
raises if libpct.so is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

from . import workloads as W

LIB_PATH = Path(__file__).resolve().parent / "_build" / "libpct.so"

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = range(6)
PREC_MIXED, PREC_F64, PREC_MIXED_LEAN = 0, 1, 2
MAX_REGIONS = 16


class PctError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libpct status {status}: {msg}")
        self.status = status


class Region(C.Structure):
    _fields_ = [("c", C.c_double * 3), ("a", C.c_double * 3), ("rsp", C.c_double)]


class PhantomDesc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("kind", C.c_int32), ("raster", C.c_int32),
                ("n", C.c_int32 * 3), ("h", C.c_double * 3), ("n_regions", C.c_int32),
                ("regions", C.POINTER(Region)), ("area_samples", C.c_int32)]


class PathModel(C.Structure):
    _fields_ = [("model", C.c_int32), ("chord", C.c_int32), ("spline_segments", C.c_int32),
                ("noise", C.c_int32), ("t_range", C.c_double * 2), ("v_range", C.c_double * 2),
                ("sigma_lat", C.c_double), ("sigma_in", C.c_double), ("sigma_out", C.c_double),
                ("rho", C.c_double), ("noise_rel", C.c_double), ("mcs", C.c_int32), ("beam_mev", C.c_double),
                ("x0_mm", C.c_double)]


class Geometry(C.Structure):
    _fields_ = [("angles_rad", C.POINTER(C.c_double)), ("n_angles", C.c_int32),
                ("paths_per_angle", C.c_int64), ("model", PathModel), ("seed", C.c_uint64),
                ("stream_id", C.c_uint64), ("first_row", C.c_int64)]


class Csr(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("n_cols", C.c_int64), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p),
                ("b", C.c_void_p), ("x_true", C.c_void_p)]


class BatchTuning(C.Structure):
    _fields_ = [("order", C.c_int32), ("rows_per_item", C.c_int32 * 3), ("grid_mult", C.c_int32 * 3),
                ("fill_prefetch", C.c_int32)]


class BatchItem(C.Structure):
    _fields_ = [("phantom", C.c_void_p), ("geo", Geometry), ("row_ptr_dev", C.c_void_p),
                ("x_true_dev", C.c_void_p)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

# every symbol include/pct.h declares
EXPORTS = ["pct_phantom_create", "pct_phantom_destroy", "pct_phantom_nvox", "pct_phantom_rasterize",
           "pct_simulate_workspace_size", "pct_simulate_count", "pct_simulate_fill", "pct_simulate_fill_host",
           "pct_simulate_host_workspace_size", "pct_simulate_host", "pct_simulate_check", "pct_simulate",
           "pct_projector_workspace_size", "pct_forward", "pct_adjoint", "pct_batch_workspace_size", "pct_batch_create",
           "pct_batch_count", "pct_batch_nnz", "pct_batch_fill", "pct_batch_params", "pct_batch_destroy",
           "pct_scan_counts_static", "pct_sap_workspace_size", "pct_sap", "pct_csr_file_create",
           "pct_csr_file_write_rows", "pct_last_error", "pct_version"]
BATCH_AUTOTUNE, BATCH_LEAN = 1, 2
STATIC_SCAN_MAX_ROWS = 1 << 28

_lib = None


def lib():
    """Load libpct.so (built by build.build()); raises when it is missing."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2108_12369_gb300.build.build()")
        L = C.CDLL(str(LIB_PATH))
        P, vp = C.POINTER, C.c_void_p
        sig = {
            "pct_phantom_create": ([P(PhantomDesc), P(vp)], C.c_int),
            "pct_phantom_destroy": ([vp], C.c_int),
            "pct_phantom_nvox": ([vp], C.c_int64),
            "pct_phantom_rasterize": ([vp, vp, vp], C.c_int),
            "pct_simulate_workspace_size": ([vp, P(Geometry), C.c_int32, P(C.c_size_t)], C.c_int),
            "pct_simulate_count": ([vp, P(Geometry), C.c_int32, vp, C.c_size_t, vp, vp], C.c_int),
            "pct_simulate_fill": ([vp, P(Geometry), C.c_int32, vp, C.c_size_t, vp, vp, vp, vp, vp, vp],
                                  C.c_int),
            "pct_simulate_fill_host": ([vp, P(Geometry), C.c_int32, vp, C.c_size_t, vp, vp, vp, C.c_size_t, vp, vp,
                                        vp, vp, vp], C.c_int),
            "pct_simulate_host_workspace_size": ([vp, P(Geometry), C.c_int32, C.c_int32, P(C.c_size_t)], C.c_int),
            "pct_simulate_host": ([vp, P(Geometry), C.c_int32, C.c_int32, vp, C.c_size_t, vp, vp, C.c_size_t, vp, vp,
                                   vp, vp, C.c_int64, P(C.c_int64), vp], C.c_int),
            "pct_simulate_check": ([vp, P(C.c_int64), vp], C.c_int),
            "pct_simulate": ([vp, P(Geometry), C.c_int32, ALLOC_FN, FREE_FN, vp, P(Csr), vp], C.c_int),
            "pct_projector_workspace_size": ([vp, P(Geometry), C.c_int32, C.c_int64, P(C.c_size_t)],
                                             C.c_int),
            "pct_forward": ([vp, P(Geometry), P(Csr), C.c_int32, C.c_int64, C.c_int64, vp, vp, vp,
                             C.c_size_t, vp], C.c_int),
            "pct_adjoint": ([vp, P(Geometry), P(Csr), C.c_int32, C.c_int64, C.c_int64, vp, vp, vp,
                             C.c_size_t, vp], C.c_int),
            "pct_scan_counts_static": ([vp, C.c_int64, vp], C.c_int),
            "pct_batch_workspace_size": ([P(BatchItem), C.c_int32, C.c_int32, P(C.c_size_t)], C.c_int),
            "pct_batch_create": ([P(BatchItem), C.c_int32, vp, C.c_size_t, C.c_int32, vp, P(vp)], C.c_int),
            "pct_batch_count": ([vp, vp], C.c_int),
            "pct_batch_nnz": ([vp, P(C.c_int64), vp], C.c_int),
            "pct_batch_fill": ([vp, P(vp), P(vp), P(vp), vp], C.c_int),
            "pct_batch_params": ([vp, P(BatchTuning)], C.c_int),
            "pct_batch_destroy": ([vp], C.c_int),
            "pct_sap_workspace_size": ([C.c_int64, C.c_int32, P(C.c_size_t)], C.c_int),
            "pct_sap": ([P(Csr), vp, C.c_int32, P(C.c_double), C.c_double, C.c_int32, vp, vp, C.c_size_t, vp],
                        C.c_int),
            "pct_csr_file_create": ([C.c_char_p, C.c_int64, C.c_int64, C.c_int64, vp], C.c_int),
            "pct_csr_file_write_rows": ([C.c_char_p, C.c_int64, C.c_int64, C.c_int64, vp, vp, vp, vp], C.c_int),
            "pct_last_error": ([], C.c_char_p),
            "pct_version": ([], C.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(status: int):
    if status != OK:
        raise PctError(status, lib().pct_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def last_error() -> str:
    return lib().pct_last_error().decode()


def version() -> str:
    return lib().pct_version().decode()


class Phantom:
    """Handle of pct_phantom_create(desc) for a workloads.phantom() dict."""

    def __init__(self, desc: dict):
        regs = desc["regions"]
        if not 1 <= len(regs) <= MAX_REGIONS:
            raise ValueError("1..16 regions")
        self._regs = (Region * len(regs))(*[Region((C.c_double * 3)(*r["c"]), (C.c_double * 3)(*r["a"]),
                                                   r["rsp"]) for r in regs])
        n = list(desc["n"]) + [1] * (3 - len(desc["n"]))
        h = list(desc["h"]) + [1.0] * (3 - len(desc["h"]))
        self._desc = PhantomDesc(desc["dim"], desc.get("kind", W.ELLIPSOID), desc.get("raster", W.CORNER),
                                 (C.c_int32 * 3)(*n), (C.c_double * 3)(*h), len(regs),
                                 C.cast(self._regs, C.POINTER(Region)), int(desc.get("area_samples", 4)))
        self.handle = C.c_void_p()
        _check(lib().pct_phantom_create(C.byref(self._desc), C.byref(self.handle)))
        self.nvox = int(lib().pct_phantom_nvox(self.handle))
        self.desc = desc

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.pct_phantom_destroy(self.handle)
            self.handle = None


def phantom_create(desc: dict) -> Phantom:
    return Phantom(desc)


def phantom_rasterize(ph: Phantom, x_true, stream=None):
    _check(lib().pct_phantom_rasterize(ph.handle, _ptr(x_true), _stream(stream)))


class GeometryArgs:
    """pct_geometry for a workload dict (keeps the angle array alive).  A
    workload that is a block of angles of a larger acquisition carries the
    global index of its first row as w["first_row"]."""

    def __init__(self, w: dict, stream_id: int = 0):
        self.angles = np.ascontiguousarray(w["angles"], dtype=np.float64)
        m = w["model"]
        pm = PathModel(m["model"], m.get("chord", W.CHORD_EXACT), m.get("spline_segments", 32),
                       m.get("noise", W.NOISE_NONE), (C.c_double * 2)(*m["t_range"]),
                       (C.c_double * 2)(*m.get("v_range", (0.0, 0.0))), m.get("sigma_lat", 0.0),
                       m.get("sigma_in", 0.0), m.get("sigma_out", 0.0), m.get("rho", 0.0),
                       m.get("noise_rel", 0.0), m.get("mcs", W.MCS_FIXED), m.get("beam_mev", 200.0),
                       m.get("x0_mm", W.X0_WATER_MM))
        self.c = Geometry(self.angles.ctypes.data_as(C.POINTER(C.c_double)), len(self.angles),
                          int(w["paths_per_angle"]), pm, C.c_uint64(int(w["seed"])),
                          C.c_uint64(int(stream_id)), int(w.get("first_row", 0)))
        self.n_rows = len(self.angles) * int(w["paths_per_angle"])


def simulate_workspace_size(ph: Phantom, geo: GeometryArgs, precision: int = PREC_MIXED) -> int:
    n = C.c_size_t()
    _check(lib().pct_simulate_workspace_size(ph.handle, C.byref(geo.c), precision, C.byref(n)))
    return n.value


def simulate_count(ph, geo, precision, workspace, row_ptr, stream=None):
    _check(lib().pct_simulate_count(ph.handle, C.byref(geo.c), precision, _ptr(workspace),
                                    workspace.numel() * workspace.element_size(), _ptr(row_ptr),
                                    _stream(stream)))


def simulate_fill(ph, geo, precision, workspace, row_ptr, x_true, col, val, b, stream=None):
    _check(lib().pct_simulate_fill(ph.handle, C.byref(geo.c), precision, _ptr(workspace),
                                   workspace.numel() * workspace.element_size(), _ptr(row_ptr),
                                   _ptr(x_true), _ptr(col), _ptr(val), _ptr(b), _stream(stream)))


def simulate_fill_host(ph, geo, precision, workspace, row_ptr, x_true, staging, row_ptr_h, col_h, val_h, b_h,
                       stream=None):
    """Phase 2 into host tensors (pinned for overlapped copies) through a
    device staging buffer; returns when the host tensors are complete."""
    _check(lib().pct_simulate_fill_host(ph.handle, C.byref(geo.c), precision, _ptr(workspace),
                                        workspace.numel() * workspace.element_size(), _ptr(row_ptr),
                                        _ptr(x_true), _ptr(staging), staging.numel() * staging.element_size(),
                                        _ptr(row_ptr_h), _ptr(col_h), _ptr(val_h), _ptr(b_h), _stream(stream)))


def simulate_check(workspace, stream=None) -> int:
    """Rows whose fill disagreed with row_ptr since the count that used this
    workspace (synchronises the stream); 0 for a consistent fill."""
    n = C.c_int64()
    _check(lib().pct_simulate_check(_ptr(workspace), C.byref(n), _stream(stream)))
    return n.value


def simulate_host_workspace_size(ph: Phantom, geo: GeometryArgs, precision: int, angles_per_block: int) -> int:
    n = C.c_size_t()
    _check(lib().pct_simulate_host_workspace_size(ph.handle, C.byref(geo.c), precision, int(angles_per_block),
                                                  C.byref(n)))
    return n.value


def simulate_host(ph, geo, precision, angles_per_block, workspace, x_true, staging, row_ptr_h, col_h, val_h, b_h,
                  stream=None) -> int:
    """The whole simulation into host tensors (pinned for overlapped copies),
    angle block by angle block; returns nnz.  col_h / val_h hold the CSR
    entries when nnz <= their length; otherwise only row_ptr_h is complete
    (col_h / val_h may then be None, e.g. to learn nnz with a small
    workspace)."""
    cap = 0 if col_h is None else min(col_h.numel(), val_h.numel())
    nnz = C.c_int64()
    st = lib().pct_simulate_host(ph.handle, C.byref(geo.c), precision, int(angles_per_block), _ptr(workspace),
                                 workspace.numel() * workspace.element_size(), _ptr(x_true), _ptr(staging),
                                 staging.numel() * staging.element_size(), _ptr(row_ptr_h), _ptr(col_h), _ptr(val_h),
                                 _ptr(b_h), cap, C.byref(nnz), _stream(stream))
    if st == ENOMEM and nnz.value > cap:
        return nnz.value  # the capacity case: row pointers complete, entries not written
    _check(st)
    return nnz.value


def simulate(ph: Phantom, geo: GeometryArgs, precision: int = PREC_MIXED, stream=None, device="cuda"):
    """Two-phase simulation into PyTorch-owned buffers; returns a dict of tensors."""
    import torch
    ws = torch.empty(simulate_workspace_size(ph, geo, precision), dtype=torch.uint8, device=device)
    x = torch.empty(ph.nvox, dtype=torch.float32, device=device)
    rp = torch.empty(geo.n_rows + 1, dtype=torch.int64, device=device)
    b = torch.empty(max(geo.n_rows, 1), dtype=torch.float32, device=device)[: geo.n_rows]
    phantom_rasterize(ph, x, stream)
    simulate_count(ph, geo, precision, ws, rp, stream)
    nnz = int(rp[-1].item())
    col = torch.empty(max(nnz, 1), dtype=torch.int32, device=device)
    val = torch.empty(max(nnz, 1), dtype=torch.float32, device=device)
    simulate_fill(ph, geo, precision, ws, rp, x, col, val, b, stream)
    return {"x_true": x, "row_ptr": rp, "col": col[:nnz], "val": val[:nnz], "b": b, "nnz": nnz,
            "workspace": ws}


def simulate_c_alloc(ph: Phantom, geo: GeometryArgs, precision: int = PREC_MIXED, stream=None,
                     device="cuda"):
    """pct_simulate(): the library allocates through callbacks (here: torch)."""
    import torch
    keep = {}

    def _alloc(nbytes, ctx):
        t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)
        keep[t.data_ptr()] = t
        return t.data_ptr()

    def _free(p, ctx):
        keep.pop(p, None)

    af, ff = ALLOC_FN(_alloc), FREE_FN(_free)
    out = Csr()
    _check(lib().pct_simulate(ph.handle, C.byref(geo.c), precision, af, ff, None, C.byref(out),
                              _stream(stream)))

    def view(p, dtype, n):
        return keep[p].view(dtype)[:n]

    return {"x_true": view(out.x_true, torch.float32, out.n_cols),
            "row_ptr": view(out.row_ptr, torch.int64, out.n_rows + 1),
            "col": view(out.col, torch.int32, out.nnz), "val": view(out.val, torch.float32, out.nnz),
            "b": view(out.b, torch.float32, out.n_rows), "nnz": out.nnz}


def _csr(A):
    if A is None:
        return None
    return C.byref(Csr(A["row_ptr"].numel() - 1, A["x_true"].numel() if "x_true" in A else 0,
                       A["col"].numel(), A["row_ptr"].data_ptr(), A["col"].data_ptr(),
                       A["val"].data_ptr(), 0, 0))


def scan_counts_static(row_ptr, n_rows: int, stream=None):
    """pct_scan_counts_static: row pointers from the counts in row_ptr[1..n_rows],
    in place, with the library's static scratch (no device allocation)."""
    _check(lib().pct_scan_counts_static(_ptr(row_ptr), int(n_rows), _stream(stream)))


def projector_workspace_size(ph: Phantom, geo: GeometryArgs, max_rows: int, precision: int = PREC_MIXED) -> int:
    n = C.c_size_t()
    _check(lib().pct_projector_workspace_size(ph.handle, C.byref(geo.c), precision, int(max_rows), C.byref(n)))
    return n.value


def forward(ph, geo, A, row0, n_rows, x, y, workspace=None, stream=None, precision=PREC_MIXED):
    """y = A x over rows [row0, row0 + n_rows) (CSR if A is given, else matrix-free)."""
    ws = workspace
    _check(lib().pct_forward(ph.handle if ph else None, C.byref(geo.c) if geo else None, _csr(A), precision,
                             row0, n_rows, _ptr(x), _ptr(y), _ptr(ws),
                             0 if ws is None else ws.numel() * ws.element_size(), _stream(stream)))


def adjoint(ph, geo, A, row0, n_rows, r, g, workspace=None, stream=None, precision=PREC_MIXED):
    """g += A^T r over rows [row0, row0 + n_rows)."""
    ws = workspace
    _check(lib().pct_adjoint(ph.handle if ph else None, C.byref(geo.c) if geo else None, _csr(A), precision,
                             row0, n_rows, _ptr(r), _ptr(g), _ptr(ws),
                             0 if ws is None else ws.numel() * ws.element_size(), _stream(stream)))


class Batch:
    """pct_batch_* over a list of workload dicts: one persistent launch per
    phase for all of them, replayed from CUDA graphs."""

    def __init__(self, workloads, autotune: bool = False, stream=None, device="cuda", lean: bool = False,
                 workspace_bytes: int = 0):
        """lean: items may take the lean form; workspace_bytes beyond the
        all-lean size lets the largest items keep the full form."""
        import torch
        self.n = len(workloads)
        self.phantoms = [Phantom(w["phantom"]) for w in workloads]
        self.geos = [GeometryArgs(w) for w in workloads]
        self.row_ptr = [torch.empty(g.n_rows + 1, dtype=torch.int64, device=device) for g in self.geos]
        self.x_true = [torch.empty(max(p.nvox, 1), dtype=torch.float32, device=device) for p in self.phantoms]
        self._items = (BatchItem * self.n)(*[
            BatchItem(p.handle, g.c, rp.data_ptr(), x.data_ptr())
            for p, g, rp, x in zip(self.phantoms, self.geos, self.row_ptr, self.x_true)])
        nbytes = C.c_size_t()
        flags = (BATCH_AUTOTUNE if autotune else 0) | (BATCH_LEAN if lean else 0)
        _check(lib().pct_batch_workspace_size(self._items, self.n, flags, C.byref(nbytes)))
        size = max(nbytes.value, int(workspace_bytes))
        self.workspace = torch.empty(size, dtype=torch.uint8, device=device)
        self.handle = C.c_void_p()
        _check(lib().pct_batch_create(self._items, self.n, _ptr(self.workspace), size,
                                      flags, _stream(stream),
                                      C.byref(self.handle)))
        self.device = device

    def count(self, stream=None):
        _check(lib().pct_batch_count(self.handle, _stream(stream)))

    def nnz(self, stream=None):
        out = (C.c_int64 * self.n)()
        _check(lib().pct_batch_nnz(self.handle, out, _stream(stream)))
        return [int(v) for v in out]

    def fill(self, nnz=None, stream=None):
        """Allocates col / val / b per simulation (kept for the next fill of
        the same sizes) and runs the fill phase."""
        import torch
        nnz = self.nnz(stream) if nnz is None else nnz
        if getattr(self, "_sizes", None) != list(nnz):  # outputs of the previous fill are reused
            self.col = self.val = None  # freed before the new ones are allocated
            self.col = [torch.empty(max(z, 1), dtype=torch.int32, device=self.device) for z in nnz]
            self.val = [torch.empty(max(z, 1), dtype=torch.float32, device=self.device) for z in nnz]
            self.b = [torch.empty(max(g.n_rows, 1), dtype=torch.float32, device=self.device) for g in self.geos]
            self._sizes = list(nnz)
        cols = (C.c_void_p * self.n)(*[t.data_ptr() for t in self.col])
        vals = (C.c_void_p * self.n)(*[t.data_ptr() for t in self.val])
        bs = (C.c_void_p * self.n)(*[t.data_ptr() for t in self.b])
        _check(lib().pct_batch_fill(self.handle, cols, vals, bs, _stream(stream)))
        return [{"row_ptr": rp, "col": c[:z], "val": v[:z], "b": bb[:g.n_rows], "x_true": x, "nnz": z}
                for rp, c, v, bb, x, z, g in zip(self.row_ptr, self.col, self.val, self.b, self.x_true,
                                                  nnz, self.geos)]

    def params(self):
        """The launch shape in use (pct_batch_tuning) as a dict."""
        t = BatchTuning()
        _check(lib().pct_batch_params(self.handle, C.byref(t)))
        return {"order": t.order, "rows_per_item": list(t.rows_per_item), "grid_mult": list(t.grid_mult),
                "fill_prefetch": t.fill_prefetch}

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.pct_batch_destroy(self.handle)
            self.handle = None


def batch_workspace_size(workloads, lean: bool = False) -> int:
    phs = [Phantom(w["phantom"]) for w in workloads]
    geos = [GeometryArgs(w) for w in workloads]
    items = (BatchItem * len(phs))(*[BatchItem(p.handle, g.c, None, None) for p, g in zip(phs, geos)])
    n = C.c_size_t()
    _check(lib().pct_batch_workspace_size(items, len(phs), BATCH_LEAN if lean else 0, C.byref(n)))
    return n.value


def sap_workspace_size(n_cols: int, n_strings: int) -> int:
    n = C.c_size_t()
    _check(lib().pct_sap_workspace_size(int(n_cols), int(n_strings), C.byref(n)))
    return n.value


def sap(A, b, n_cols: int, n_strings: int, lam: float, iterations: int, x, weights=None, workspace=None,
        stream=None):
    """String-averaging projections (Sec. II-D) on the CSR dict A (row_ptr,
    col, val) and b, in place on the float32 device tensor x."""
    import torch
    ws = workspace
    if ws is None:
        ws = torch.empty(sap_workspace_size(n_cols, n_strings), dtype=torch.uint8, device=x.device)
    csr = Csr(A["row_ptr"].numel() - 1, int(n_cols), A["col"].numel(), A["row_ptr"].data_ptr(),
              A["col"].data_ptr(), A["val"].data_ptr(), 0, 0)
    wts = None
    if weights is not None:
        warr = np.ascontiguousarray(weights, dtype=np.float64)
        wts = warr.ctypes.data_as(C.POINTER(C.c_double))
    _check(lib().pct_sap(C.byref(csr), _ptr(b), int(n_strings), wts, float(lam), int(iterations), _ptr(x),
                         _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))
    return x


def _host_ptr(a):
    """data pointer of a host numpy array or CPU tensor (None for None)"""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if a.is_cuda:
            raise ValueError("host arrays expected")
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def csr_file_create(path, n_rows: int, n_cols: int, nnz: int, x_true):
    """pct_csr_file_create: the file of an n_rows x n_cols system with nnz
    nonzeros, with x_true (host float32) written."""
    x = np.ascontiguousarray(x_true, dtype=np.float32) if not hasattr(x_true, "data_ptr") else x_true
    _check(lib().pct_csr_file_create(str(path).encode(), int(n_rows), int(n_cols), int(nnz), _host_ptr(x)))


def csr_file_write_rows(path, row0: int, nz0: int, row_ptr, col, val, b):
    """pct_csr_file_write_rows: a block of rows (host arrays; row_ptr local,
    any base) at global row row0 and global nonzero offset nz0."""
    arrs = [np.ascontiguousarray(a, dtype=t) if not hasattr(a, "data_ptr") else a
            for a, t in ((row_ptr, np.int64), (col, np.int32), (val, np.float32), (b, np.float32))]
    n = (arrs[0].numel() if hasattr(arrs[0], "numel") else len(arrs[0])) - 1
    _check(lib().pct_csr_file_write_rows(str(path).encode(), int(row0), int(n), int(nz0),
                                         *[_host_ptr(a) for a in arrs]))


def csr_file_read(path):
    """The system in a file made by csr_file_create / _write_rows, as numpy
    arrays mapped from the file: dict(row_ptr, col, val, b, x_true)."""
    with open(path, "rb") as f:
        head = f.read(128)
    if head[:8] != b"PCTCSR1\0":
        raise ValueError(f"{path} is not a libpct CSR file")
    n_rows, n_cols, nnz, o_rp, o_col, o_val, o_b, o_x = np.frombuffer(head[8:72], dtype="<i8")
    mm = lambda off, dt, n: np.memmap(path, dtype=dt, mode="r", offset=int(off), shape=(int(n),))
    return {"row_ptr": mm(o_rp, "<i8", n_rows + 1), "col": mm(o_col, "<i4", nnz), "val": mm(o_val, "<f4", nnz),
            "b": mm(o_b, "<f4", n_rows), "x_true": mm(o_x, "<f4", n_cols),
            "n_rows": int(n_rows), "n_cols": int(n_cols), "nnz": int(nnz)}
