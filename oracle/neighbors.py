"""Brute-force neighbour pairs (the sparsity mask M of Sec. II.A) -- oracle, test-only.

Pairs (i, j) with |r_j - r_i|^2 <= cutoff^2, self included, found by an O(N^2) loop.  The
squared distance is evaluated as ((dx*dx) + (dy*dy)) + (dz*dz) in FP64 with one rounding per
operation (NumPy element-wise ops do not fuse), which is the rounding the pattern is defined
with.  Periodic boxes use the minimum image dx - L * rint(dx / L).
"""
from __future__ import annotations

import numpy as np


def min_image(dx: np.ndarray, box) -> np.ndarray:
    """Minimum-image displacement per component (box None or 0 => open)."""
    if box is None:
        return dx
    out = dx.copy()
    for c in range(3):
        L = float(box[c])
        if L > 0.0:
            out[..., c] = dx[..., c] - L * np.rint(dx[..., c] / L)
    return out


def neighbor_csr(pos: np.ndarray, cutoff: float, box=None, chunk: int = 2048):
    """CSR (row_ptr int64, col int32) of all pairs with r^2 <= cutoff^2, columns ascending."""
    pos = np.asarray(pos, dtype=np.float64)
    n = pos.shape[0]
    rc2 = float(cutoff) * float(cutoff)
    cols = []
    counts = np.zeros(n, dtype=np.int64)
    for i0 in range(0, n, chunk):
        i1 = min(n, i0 + chunk)
        d = pos[None, :, :] - pos[i0:i1, None, :]
        d = min_image(d, box)
        r2 = d[..., 0] * d[..., 0]
        r2 = r2 + d[..., 1] * d[..., 1]
        r2 = r2 + d[..., 2] * d[..., 2]
        hit = r2 <= rc2
        for k in range(i1 - i0):
            js = np.nonzero(hit[k])[0]
            counts[i0 + k] = js.size
            cols.append(js.astype(np.int32))
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = np.concatenate(cols) if cols else np.zeros(0, dtype=np.int32)
    return row_ptr, col
