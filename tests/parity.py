"""Comparison of a GPU simulation against the CPU oracle.

Rule (from the statement that indices must match exactly and lengths / WEPL
within 1e-6 relative per proton):
  row_ptr and col: equal;
  per row: max_j |a_gpu - a_orc| <= tol * sum_j a_orc;
  b: |b_gpu - b_orc| <= tol * max(|b_orc|, sum_j a_orc * max(x)).
"""
import numpy as np


def to_np(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)


def compare(gpu: dict, ref: dict, tol: float = 1e-6, exact_values: bool = False, x_max=None):
    rp_g = to_np(gpu["row_ptr"]).astype(np.int64)
    rp_o = np.asarray(ref["row_ptr"], dtype=np.int64)
    assert rp_g.shape == rp_o.shape
    bad = np.flatnonzero(rp_g != rp_o)
    assert bad.size == 0, f"row_ptr differs first at {bad[:5]}"
    col_g = to_np(gpu["col"])
    assert np.array_equal(col_g, ref["col"]), f"col differs at {np.flatnonzero(col_g != ref['col'])[:10]}"
    n = len(rp_o) - 1
    val_g = to_np(gpu["val"]).astype(np.float64)
    val_o = np.asarray(ref["val"], dtype=np.float64)
    rows = np.repeat(np.arange(n), np.diff(rp_o))
    rowsum = np.bincount(rows, weights=val_o, minlength=n)
    b_g = to_np(gpu["b"]).astype(np.float64)
    b_o = np.asarray(ref["b"], dtype=np.float64)
    if x_max is None:
        x_max = float(np.max(to_np(gpu["x_true"]))) if "x_true" in gpu else 1.0
    stats = {}
    if len(val_o):
        aerr = np.abs(val_g - val_o)
        rel = aerr / np.maximum(rowsum[rows], 1e-30)
        stats.update(val_max_rel=float(rel.max()), val_rms_abs=float(np.sqrt(np.mean(aerr ** 2))),
                     val_max_abs=float(aerr.max()))
        if exact_values:
            assert np.array_equal(to_np(gpu["val"]), val_o.astype(np.float32))
        assert rel.max() <= tol, f"value error {rel.max():.3g} > {tol} at entry {int(rel.argmax())}"
    if n:
        berr = np.abs(b_g - b_o)
        scale = np.maximum(np.abs(b_o), rowsum * x_max)
        relb = berr / np.maximum(scale, 1e-30)
        relb[scale == 0] = berr[scale == 0]
        stats.update(b_max_rel=float(relb.max()), b_rms_abs=float(np.sqrt(np.mean(berr ** 2))))
        if exact_values:
            assert np.array_equal(to_np(gpu["b"]), b_o.astype(np.float32))
        assert relb.max() <= tol, f"b error {relb.max():.3g} > {tol} at row {int(relb.argmax())}"
    return stats
