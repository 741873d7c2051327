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


def das_volume(y, pos, normal, c: float, dt: float, origin, spacing: float, dims,
               wmode: str = "clamp") -> np.ndarray:
    """Delay-and-sum volume: voxel v (centre x_v = origin + (index + 1/2)
    spacing) takes sum_m w_m(v) y_m(tau), tau = |x_v - s_m| / c, with y_m
    linearly interpolated between cell centres (sample j stands for the cell
    [j dt, (j+1) dt), centre (j + 1/2) dt; zero outside the record) and
    w = max(0, n_m . u), u = (x_v - s_m) / d (the radiator's orientation
    weight; wmode "none" gives w = 1). dims = (nx, ny, nz); returns float64
    [nz][ny][nx]."""
    y = np.asarray(y, dtype=np.float64)
    M, T = y.shape
    nx, ny, nz = (int(v) for v in dims)
    cx = float(origin[0]) + (np.arange(nx) + 0.5) * spacing
    cy = float(origin[1]) + (np.arange(ny) + 0.5) * spacing
    cz = float(origin[2]) + (np.arange(nz) + 0.5) * spacing
    Z, Y, X = np.meshgrid(cz, cy, cx, indexing="ij")
    vol = np.zeros((nz, ny, nx))
    P = np.asarray(pos, dtype=np.float64)
    N = np.asarray(normal, dtype=np.float64)
    for m in range(M):
        dx, dy, dz = X - P[m, 0], Y - P[m, 1], Z - P[m, 2]
        d = np.sqrt(dx * dx + dy * dy + dz * dz)
        w = np.ones_like(d) if wmode == "none" else np.maximum(
            (N[m, 0] * dx + N[m, 1] * dy + N[m, 2] * dz) / d, 0.0)
        q = d / (c * dt) - 0.5
        j = np.floor(q).astype(np.int64)
        f = q - j
        y0 = np.where((j >= 0) & (j < T), y[m, np.clip(j, 0, T - 1)], 0.0)
        y1 = np.where((j + 1 >= 0) & (j + 1 < T), y[m, np.clip(j + 1, 0, T - 1)], 0.0)
        vol += w * ((1.0 - f) * y0 + f * y1)
    return vol


# --------------------------------------------------------------------------
# the proposal CNN: 1 -> 16 -> 32 -> 64 channels of 3x3x3 convolutions with
# ReLU and a 1x1x1 head with two outputs (logit, pressure) per voxel
# --------------------------------------------------------------------------

PARAM_SHAPES = (("w1", (16, 27, 1)), ("b1", (16,)), ("w2", (32, 27, 16)), ("b2", (32,)),
                ("w3", (64, 27, 32)), ("b3", (64,)), ("wh", (2, 64)), ("bh", (2,)))


def unpack_params(p) -> dict:
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in PARAM_SHAPES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    assert o == p.size
    return out


def scaled_input(vol) -> np.ndarray:
    """The network input: vol / max|vol| rounded to bf16, shape (nz, ny, nx, 1)."""
    v = np.asarray(vol, dtype=np.float64)
    mx = np.max(np.abs(v))
    x = (v / mx if mx > 0 else v).astype(np.float32)
    return bf16_round(x)[..., None].astype(np.float64)


def cnn_forward(p, vol, round_activations: bool = True) -> np.ndarray:
    """Forward pass in float64 with bf16 weights and input; with
    round_activations the three hidden activations are rounded to bf16 as
    they are stored on the GPU. Returns (V, 2) in voxel order."""
    P = unpack_params(p)
    r = (lambda a: bf16_round(a.astype(np.float32)).astype(np.float64)) if round_activations \
        else (lambda a: a)
    bw = lambda w: bf16_round(w.astype(np.float32)).astype(np.float64)
    h = scaled_input(vol)
    for k in (1, 2, 3):
        h = r(np.maximum(conv3d(h, bw(P[f"w{k}"]), P[f"b{k}"]), 0.0))
    out = h @ P["wh"].T + P["bh"]
    return out.reshape(-1, 2)


def cnn_loss_grad(p, vol, occ, p0, pos_weight: float, bf16_storage: bool = False):
    """Loss and its gradient with respect to the FP32 parameters, by torch
    autograd in float64 on the CPU (weights used through their bf16 values,
    input bf16). Returns (loss0, loss1, grad).

    With bf16_storage the tensors the network stores in bf16 are rounded to
    bf16 at the points where they are stored, the precision the network is
    specified in (BF16 storage, FP32 accumulation): the hidden activations
    h1, h2, h3 after their ReLU; the gradient with respect to the third
    convolution's output, after the ReLU mask; and the gradients with
    respect to h2 and h1, before their ReLU masks. Every sum is still taken
    in float64. Without it nothing is rounded past the input and weights."""
    import torch
    import torch.nn.functional as F

    def to_bf16(a):
        return a.float().bfloat16().double() if bf16_storage else a

    class Store(torch.autograd.Function):  # rounds the stored value
        @staticmethod
        def forward(ctx, a):
            return to_bf16(a)

        @staticmethod
        def backward(ctx, g):
            return g

    class GradStore(torch.autograd.Function):  # rounds the stored gradient
        @staticmethod
        def forward(ctx, a):
            return a.clone()

        @staticmethod
        def backward(ctx, g):
            return to_bf16(g)

    P = unpack_params(p)
    x = torch.from_numpy(scaled_input(vol)[..., 0])[None, None]  # (1, 1, nz, ny, nx)
    t = torch.from_numpy(np.asarray(occ, dtype=np.float64).reshape(-1))
    q0 = torch.from_numpy(np.asarray(p0, dtype=np.float64).reshape(-1))
    leaves = {}
    for name, _ in PARAM_SHAPES:
        a = P[name]
        if name.startswith("w") and name != "wh":
            a = bf16_round(a.astype(np.float32)).astype(np.float64)
        leaves[name] = torch.tensor(a, requires_grad=True)

    def kern(w):  # (cout, 27, cin) -> (cout, cin, 3, 3, 3), tap = (dz+1)*9 + (dy+1)*3 + (dx+1)
        co, _, ci = w.shape
        return w.permute(0, 2, 1).reshape(co, ci, 3, 3, 3)

    h = x
    for k in (1, 2):
        pre = F.conv3d(h, kern(leaves[f"w{k}"]), leaves[f"b{k}"], padding=1)
        h = GradStore.apply(Store.apply(torch.relu(pre)))
    pre = GradStore.apply(F.conv3d(h, kern(leaves["w3"]), leaves["b3"], padding=1))
    h = Store.apply(torch.relu(pre))
    h = h[0].permute(1, 2, 3, 0).reshape(-1, P["wh"].shape[1])
    out = h @ leaves["wh"].T + leaves["bh"]
    z, q = out[:, 0], out[:, 1]
    V = z.shape[0]
    l0 = (pos_weight * t * F.softplus(-z) + (1 - t) * F.softplus(z)).sum() / V
    l1 = (t * (q - q0) ** 2).sum() / V
    (l0 + l1).backward()
    grad = np.concatenate([leaves[n].grad.numpy().reshape(-1) for n, _ in PARAM_SHAPES])
    return float(l0.detach()), float(l1.detach()), grad
