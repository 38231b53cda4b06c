"""ctypes front end of the FP64 CPU oracle (``pct_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` import this
module; the product package never does.  It shares no code with the CUDA
library: it only takes the same plain workload descriptions (dicts of
numbers) as inputs.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "pct_oracle.c"
LIB = HERE / "_build" / "liboracle.so"

ELLIPSOID, EXTRUDED = 0, 1
CENTER, CORNER, AREA = 0, 1, 2
STRAIGHT, STRAIGHT_MCS, SPLINE = 0, 1, 2
CHORD_EXACT, CHORD_CONSTANT = 0, 1
NOISE_NONE, NOISE_GAUSS_REL = 0, 1
MCS_FIXED, MCS_HIGHLAND = 0, 1


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (no FMA contraction, OpenMP for timing)."""
    LIB.parent.mkdir(exist_ok=True)
    if force or not LIB.exists() or LIB.stat().st_mtime < max(
        SRC.stat().st_mtime, (HERE / "pct_oracle.h").stat().st_mtime
    ):
        tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
             "-shared", "-o", str(tmp), str(SRC), "-lm"]
        )
        os.replace(tmp, LIB)
    return LIB


class _Phantom(C.Structure):
    _fields_ = [("dim", C.c_int32), ("kind", C.c_int32), ("raster", C.c_int32),
                ("n", C.c_int32 * 3), ("h", C.c_double * 3), ("n_regions", C.c_int32),
                ("regions", C.POINTER(C.c_double)), ("area_samples", C.c_int32)]


class _Model(C.Structure):
    _fields_ = [("model", C.c_int32), ("chord", C.c_int32), ("spline_segments", C.c_int32),
                ("noise", C.c_int32), ("t_lo", C.c_double), ("t_hi", C.c_double),
                ("v_lo", C.c_double), ("v_hi", C.c_double), ("sigma_lat", C.c_double),
                ("sigma_in", C.c_double), ("sigma_out", C.c_double), ("rho", C.c_double),
                ("noise_rel", C.c_double), ("mcs", C.c_int32), ("beam_mev", C.c_double),
                ("x0_mm", C.c_double)]


class _Sim(C.Structure):
    _fields_ = [("ph", C.POINTER(_Phantom)), ("x_true", C.POINTER(C.c_float)),
                ("angles", C.POINTER(C.c_double)), ("n_angles", C.c_int32),
                ("paths_per_angle", C.c_int64), ("model", C.POINTER(_Model)),
                ("seed", C.c_uint64), ("stream", C.c_uint64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(str(build()))
        P = C.POINTER
        _lib.orc_philox4x64_10.argtypes = [P(C.c_uint64), P(C.c_uint64), P(C.c_uint64)]
        _lib.orc_log.argtypes = [C.c_double]
        _lib.orc_log.restype = C.c_double
        _lib.orc_uniform.argtypes = [C.c_uint64] * 4
        _lib.orc_uniform.restype = C.c_double
        _lib.orc_normal_pairs.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64,
                                          C.c_int32, P(C.c_double)]
        _lib.orc_normal_pairs.restype = C.c_uint64
        _lib.orc_hull_hit.argtypes = [P(_Phantom), C.c_int32, P(C.c_double), P(C.c_double),
                                      P(C.c_double), P(C.c_double)]
        _lib.orc_hull_hit.restype = C.c_int
        _lib.orc_raster.argtypes = [P(_Phantom), P(C.c_double)]
        _lib.orc_segment.argtypes = [P(_Phantom), P(C.c_double), P(C.c_double), P(C.c_int32),
                                     P(C.c_double), C.c_int64]
        _lib.orc_segment.restype = C.c_int64
        _lib.orc_path.argtypes = [P(_Sim), C.c_int64, P(C.c_double), C.c_int32]
        _lib.orc_path.restype = C.c_int32
        _lib.orc_row.argtypes = [P(_Sim), C.c_int64, P(C.c_int32), P(C.c_double), C.c_int64,
                                 P(C.c_double), P(C.c_double)]
        _lib.orc_row.restype = C.c_int64
        _lib.orc_count_rows.argtypes = [P(_Sim), P(C.c_int64), C.c_int64, P(C.c_int64), C.c_int32]
        _lib.orc_fill_rows.argtypes = [P(_Sim), P(C.c_int64), C.c_int64, P(C.c_int64),
                                       P(C.c_int32), P(C.c_double), P(C.c_double), P(C.c_double),
                                       C.c_int32]
        _lib.orc_highland.argtypes = [C.c_double, C.c_double, C.c_double, P(C.c_double)]
        _lib.orc_highland.restype = C.c_double
        _lib.orc_sap.argtypes = [C.c_int64, C.c_int64, P(C.c_int64), P(C.c_int32), P(C.c_double),
                                 P(C.c_double), C.c_int32, P(C.c_double), C.c_double, C.c_int32,
                                 P(C.c_double)]
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


class Phantom:
    """Oracle-side copy of a phantom description (see workloads.py for fields)."""

    def __init__(self, desc: dict):
        self.desc = desc
        self.regions = np.ascontiguousarray(
            [list(r["c"]) + list(r["a"]) + [r["rsp"]] for r in desc["regions"]], dtype=np.float64
        ).reshape(-1, 7)
        n = list(desc["n"]) + [1] * (3 - len(desc["n"]))
        h = list(desc["h"]) + [1.0] * (3 - len(desc["h"]))
        self.c = _Phantom(int(desc["dim"]), int(desc.get("kind", ELLIPSOID)),
                          int(desc.get("raster", CORNER)), (C.c_int32 * 3)(*n),
                          (C.c_double * 3)(*h), len(self.regions),
                          _ptr(self.regions, C.c_double), int(desc.get("area_samples", 4)))
        self.nvox = int(np.prod(n[: desc["dim"]]))

    def raster(self) -> np.ndarray:
        x = np.zeros(self.nvox, dtype=np.float64)
        lib().orc_raster(C.byref(self.c), _ptr(x, C.c_double))
        return x

    def segment(self, P, Q, cap: int = 1 << 16):
        P = np.ascontiguousarray(list(P) + [0.0] * (3 - len(P)), dtype=np.float64)
        Q = np.ascontiguousarray(list(Q) + [0.0] * (3 - len(Q)), dtype=np.float64)
        cols = np.zeros(cap, np.int32)
        lens = np.zeros(cap, np.float64)
        n = lib().orc_segment(C.byref(self.c), _ptr(P, C.c_double), _ptr(Q, C.c_double),
                              _ptr(cols, C.c_int32), _ptr(lens, C.c_double), cap)
        assert n <= cap
        return cols[:n].copy(), lens[:n].copy()

    def hull_hit(self, region: int, A, g):
        A = np.ascontiguousarray(list(A) + [0.0] * (3 - len(A)), dtype=np.float64)
        g = np.ascontiguousarray(list(g) + [0.0] * (3 - len(g)), dtype=np.float64)
        li, lo = C.c_double(), C.c_double()
        hit = lib().orc_hull_hit(C.byref(self.c), region, _ptr(A, C.c_double),
                                 _ptr(g, C.c_double), C.byref(li), C.byref(lo))
        return bool(hit), li.value, lo.value


def _model_struct(m: dict) -> _Model:
    return _Model(int(m["model"]), int(m.get("chord", CHORD_EXACT)),
                  int(m.get("spline_segments", 32)), int(m.get("noise", NOISE_NONE)),
                  float(m["t_range"][0]), float(m["t_range"][1]),
                  float(m.get("v_range", (0.0, 0.0))[0]), float(m.get("v_range", (0.0, 0.0))[1]),
                  float(m.get("sigma_lat", 0.0)), float(m.get("sigma_in", 0.0)),
                  float(m.get("sigma_out", 0.0)), float(m.get("rho", 0.0)),
                  float(m.get("noise_rel", 0.0)), int(m.get("mcs", MCS_FIXED)),
                  float(m.get("beam_mev", 200.0)), float(m.get("x0_mm", 360.8)))


class Simulation:
    """Oracle simulation of one workload: phantom, angles, protons, model, seed."""

    def __init__(self, phantom: Phantom, x_true: np.ndarray, angles, paths_per_angle: int,
                 model: dict, seed: int, stream: int = 0):
        self.phantom = phantom
        self.x_true = np.ascontiguousarray(x_true, dtype=np.float32)
        self.angles = np.ascontiguousarray(angles, dtype=np.float64)
        self.P = int(paths_per_angle)
        self.model = _model_struct(model)
        self.n_rows = len(self.angles) * self.P
        self.c = _Sim(C.pointer(phantom.c), _ptr(self.x_true, C.c_float),
                      _ptr(self.angles, C.c_double), len(self.angles), self.P,
                      C.pointer(self.model), C.c_uint64(seed), C.c_uint64(stream))

    def path(self, row: int, cap: int = 8192) -> np.ndarray:
        v = np.zeros((cap, 3), np.float64)
        n = lib().orc_path(C.byref(self.c), row, _ptr(v, C.c_double), cap)
        return v[:n].copy()

    def row(self, row: int):
        n = lib().orc_row(C.byref(self.c), row, None, None, 0, None, None)
        cols = np.zeros(max(n, 1), np.int32)
        vals = np.zeros(max(n, 1), np.float64)
        bc, bn = C.c_double(), C.c_double()
        lib().orc_row(C.byref(self.c), row, _ptr(cols, C.c_int32), _ptr(vals, C.c_double), n,
                      C.byref(bc), C.byref(bn))
        return cols[:n], vals[:n], bc.value, bn.value

    def rows(self, rows=None, threads: int = 1):
        """CSR of the given rows (default: all), FP64 values.

        Returns (row_ptr int64 [n+1], cols int32, vals float64, b_clean, b_noisy)."""
        if rows is None:
            rows = np.arange(self.n_rows, dtype=np.int64)
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        n = len(rows)
        counts = np.zeros(n, np.int64)
        lib().orc_count_rows(C.byref(self.c), _ptr(rows, C.c_int64), n,
                             _ptr(counts, C.c_int64), threads)
        row_ptr = np.zeros(n + 1, np.int64)
        np.cumsum(counts, out=row_ptr[1:])
        nnz = int(row_ptr[-1])
        cols = np.zeros(max(nnz, 1), np.int32)
        vals = np.zeros(max(nnz, 1), np.float64)
        bc = np.zeros(n, np.float64)
        bn = np.zeros(n, np.float64)
        lib().orc_fill_rows(C.byref(self.c), _ptr(rows, C.c_int64), n,
                            _ptr(row_ptr, C.c_int64), _ptr(cols, C.c_int32),
                            _ptr(vals, C.c_double), _ptr(bc, C.c_double),
                            _ptr(bn, C.c_double), threads)
        return row_ptr, cols[:nnz], vals[:nnz], bc, bn


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, np.uint64)
    lib().orc_philox4x64_10(_ptr(c, C.c_uint64), _ptr(k, C.c_uint64), _ptr(out, C.c_uint64))
    return out


def log(x: float) -> float:
    return lib().orc_log(float(x))


def uniform(seed: int, stream: int, row: int, j: int) -> float:
    return lib().orc_uniform(seed, stream, row, j)


def normal_pairs(seed: int, stream: int, row: int, j0: int, n_pairs: int):
    z = np.zeros(2 * n_pairs, np.float64)
    j = lib().orc_normal_pairs(seed, stream, row, j0, n_pairs, _ptr(z, C.c_double))
    return z, int(j)


def raster_f32(desc: dict) -> np.ndarray:
    """x_true as stored: the FP64 raster rounded once to FP32."""
    return Phantom(desc).raster().astype(np.float32)


def simulate(desc: dict, angles, paths_per_angle: int, model: dict, seed: int, rows=None,
             threads: int = 1, stream: int = 0):
    """Convenience: raster + rows.  Returns dict of numpy arrays."""
    ph = Phantom(desc)
    x = ph.raster().astype(np.float32)
    sim = Simulation(ph, x, angles, paths_per_angle, model, seed, stream)
    rp, cols, vals, bc, bn = sim.rows(rows, threads)
    return {"x_true": x, "row_ptr": rp, "col": cols, "val": vals, "b_clean": bc, "b": bn}


def sap(row_ptr, col, val, b, n_cols: int, n_strings: int, lam: float, iterations: int, x0=None,
        weights=None) -> np.ndarray:
    """String-averaging projections (Sec. II-D) in FP64: `iterations` sweeps
    from x0 (default 0); string t = rows t, t + M, ...; returns x."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    c = np.ascontiguousarray(col, dtype=np.int32)
    v = np.ascontiguousarray(val, dtype=np.float64)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n_cols, np.float64) if x0 is None else np.array(x0, dtype=np.float64)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    lib().orc_sap(len(rp) - 1, n_cols, _ptr(rp, C.c_int64), _ptr(c, C.c_int32), _ptr(v, C.c_double),
                  _ptr(bb, C.c_double), int(n_strings), None if w is None else _ptr(w, C.c_double),
                  float(lam), int(iterations), _ptr(x, C.c_double))
    return x


def highland(beam_mev: float, x0_mm: float, x_mm: float):
    """(theta0 in rad, beta c p in MeV) of the Highland / PDG formula."""
    bcp = C.c_double()
    th = lib().orc_highland(float(beam_mev), float(x0_mm), float(x_mm), C.byref(bcp))
    return th, bcp.value
