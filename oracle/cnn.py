"""FP64 CPU oracle for the learned initial proposal (delay-and-sum volume and
the small 3D CNN on it).

TEST INFRASTRUCTURE ONLY: only `tests/`, `__graft_entry__.smoke()` and the
CPU legs of `bench.py` may import this module. The product library never
calls it and shares no code with it.

* conv3d: 3x3x3 taps, zero padding, stride 1, on a channels-last volume
  x[z][y][x][c]; weight w[cout][tap][cin] with tap = (dz+1)*9 + (dy+1)*3 +
  (dx+1); out[v][n] = bias[n] + sum_{tap,c} x[v + offset(tap)][c] w[n][tap][c].
  Written as 27 shifted copies of the padded volume and one matrix product
  per tap (numpy), so each output is the plain sum of its 27*Cin terms.
* bf16: round-to-nearest-even of float32 to 8 mantissa bits, the storage
  type of the CNN's activations and weights.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    x = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32)
    return np.where(np.isnan(x), x, out).reshape(np.shape(a))


def conv3d(x, w, bias=None) -> np.ndarray:
    """x: (nz, ny, nx, cin); w: (cout, 27, cin); returns float64
    (nz, ny, nx, cout)."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    nz, ny, nx, cin = x.shape
    cout = w.shape[0]
    xp = np.zeros((nz + 2, ny + 2, nx + 2, cin))
    xp[1:-1, 1:-1, 1:-1] = x
    out = np.zeros((nz, ny, nx, cout))
    for tap in range(27):
        dz, dy, dx = tap // 9 - 1, (tap // 3) % 3 - 1, tap % 3 - 1
        sl = xp[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
        out += sl @ w[:, tap, :].T
    if bias is not None:
        out += np.asarray(bias, dtype=np.float64)
    return out
