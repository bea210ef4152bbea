"""Plain numpy definition of the 3D U-Net dose denoiser -- TEST INFRASTRUCTURE ONLY.

Only tests/ may use it. It restates, from the layer definitions, what the CUDA
denoiser computes, so that each layer, the network output and every parameter
gradient can be compared with it. Arrays are channels-last, (z, y, x, c), float64.
Weights are (taps, cin, cout) with tap t = dx + 3 dy + 9 dz for 3x3x3 kernels
(offsets -1..1) and t = dx + 2 dy + 4 dz for 2x2x2 kernels; the flat parameter
vector lists, layer by layer, W then b, and finally the 1x1x1 head (16 weights,
1 bias). Input channels: the dose over its maximum s, the density, and (optional) the dose's
statistical uncertainty over s; the other 13 channels are zero. With bf16=True, weights,
inputs and every stored activation are rounded to bfloat16 (round to nearest even), as the
model's arithmetic specifies.
"""
from __future__ import annotations

import numpy as np

CH = (16, 32, 64, 128)


def bf16(a):
    """Round float values to bfloat16 (round to nearest, ties to even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _shift(x, dz, dy, dx):
    """x[z+dz, y+dy, x+dx] with zero padding."""
    out = np.zeros_like(x)
    Z, Y, X = x.shape[:3]
    zs, ze = max(0, -dz), min(Z, Z - dz)
    ys, ye = max(0, -dy), min(Y, Y - dy)
    xs, xe = max(0, -dx), min(X, X - dx)
    out[zs:ze, ys:ye, xs:xe] = x[zs + dz:ze + dz, ys + dy:ye + dy, xs + dx:xe + dx]
    return out


def taps3():
    return [(t % 3 - 1, t // 3 % 3 - 1, t // 9 - 1) for t in range(27)]   # (dx, dy, dz)


def taps2():
    return [(t & 1, (t >> 1) & 1, t >> 2) for t in range(8)]


# ---- layers: forward, data gradient, weight gradient --------------------------------------
def conv3(x, W):
    """y[v] = sum_t x[v + d_t] W[t]  (3x3x3, stride 1, zero padding 1)."""
    return sum(_shift(x, dz, dy, dx) @ W[t] for t, (dx, dy, dz) in enumerate(taps3()))


def conv3_dx(dy, W):
    return sum(_shift(dy, -dz, -dy_, -dx) @ W[t].T for t, (dx, dy_, dz) in enumerate(taps3()))


def conv3_dw(x, dy):
    n = dy.shape[-1]
    return np.stack([_shift(x, dz, dy_, dx).reshape(-1, x.shape[-1]).T @ dy.reshape(-1, n)
                     for (dx, dy_, dz) in taps3()])


def down(x, W):
    """y[u] = sum_t x[2u + d_t] W[t]  (2x2x2, stride 2)."""
    return sum(x[dz::2, dy::2, dx::2] @ W[t] for t, (dx, dy, dz) in enumerate(taps2()))


def down_dx(dy, W, fine_shape):
    dx = np.zeros(fine_shape[:3] + (W.shape[1],))
    for t, (ox, oy, oz) in enumerate(taps2()):
        dx[oz::2, oy::2, ox::2] = dy @ W[t].T
    return dx


def down_dw(x, dy):
    n = dy.shape[-1]
    return np.stack([x[oz::2, oy::2, ox::2].reshape(-1, x.shape[-1]).T @ dy.reshape(-1, n)
                     for (ox, oy, oz) in taps2()])


def up(x, W):
    """y[2u + p] = x[u] W[p]  (transposed 2x2x2, stride 2)."""
    Z, Y, X, _ = x.shape
    y = np.zeros((2 * Z, 2 * Y, 2 * X, W.shape[2]))
    for p, (ox, oy, oz) in enumerate(taps2()):
        y[oz::2, oy::2, ox::2] = x @ W[p]
    return y


def up_dx(dy, W):
    return sum(dy[oz::2, oy::2, ox::2] @ W[p].T for p, (ox, oy, oz) in enumerate(taps2()))


def up_dw(x, dy):
    n = dy.shape[-1]
    return np.stack([x.reshape(-1, x.shape[-1]).T @ dy[oz::2, oy::2, ox::2].reshape(-1, n)
                     for (ox, oy, oz) in taps2()])


FWD = {0: conv3, 1: down, 2: up}


# ---- network ----------------------------------------------------------------------------
def architecture():
    """(mode, cin, cout, input, output) per layer; activations named by strings; 'cat{l}'
    holds [up-path output, skip] along channels."""
    L = []
    inp, cin = "x", 16
    for l, C in enumerate(CH):
        last = l == len(CH) - 1
        L.append((0, cin, C, inp, f"e{l}"))
        L.append((0, C, C, f"e{l}", f"s{l}"))
        if not last:
            L.append((1, C, CH[l + 1], f"s{l}", f"d{l}"))
            inp, cin = f"d{l}", CH[l + 1]
    prev, pc = f"s{len(CH) - 1}", CH[-1]
    for l in range(len(CH) - 2, -1, -1):
        C = CH[l]
        L.append((2, pc, C, prev, f"u{l}"))
        L.append((0, 2 * C, C, f"cat{l}", f"f{l}"))
        L.append((0, C, C, f"f{l}", f"g{l}"))
        prev, pc = f"g{l}", C
    return L


def param_layout():
    off, lay = 0, []
    for mode, cin, cout, _, _ in architecture():
        taps = 27 if mode == 0 else 8
        lay.append((off, (taps, cin, cout), off + taps * cin * cout, cout))
        off += taps * cin * cout + cout
    return lay, off, off + 16


def num_params():
    return param_layout()[2] + 1


class UNet:
    def __init__(self, params, bf16_storage=True):
        self.p = np.asarray(params, np.float64)
        self.q = bf16 if bf16_storage else (lambda a: np.asarray(a, np.float64))
        self.lay, self.hw, self.hb = param_layout()

    def weights(self, i):
        off, shape, boff, cout = self.lay[i]
        W = self.p[off:off + np.prod(shape)].reshape(shape)
        return self.q(W), self.p[boff:boff + cout]

    def _inputs(self, dose, dens, sigma=None):
        s = dose.max()
        x0 = dose / s if s > 0 else np.zeros_like(dose)
        x = np.zeros(dose.shape + (16,))
        x[..., 0] = x0
        x[..., 1] = dens
        if sigma is not None:
            x[..., 2] = np.asarray(sigma, np.float64) / s if s > 0 else 0.0
        return self.q(x), x0, s

    def forward(self, dose, dens, keep=False, sigma=None):
        x, x0, s = self._inputs(np.asarray(dose, np.float64), np.asarray(dens, np.float64), sigma)
        A = {"x": x}
        for i, (mode, cin, cout, a_in, a_out) in enumerate(architecture()):
            if a_in.startswith("cat"):
                l = a_in[3:]
                A[a_in] = np.concatenate([A[f"u{l}"], A[f"s{l}"]], axis=-1)
            W, b = self.weights(i)
            A[a_out] = self.q(np.maximum(FWD[mode](A[a_in], W) + b, 0.0))
        h = A["g0"]
        out = x0 + h @ self.p[self.hw:self.hw + 16] + self.p[self.hb]
        if keep:
            return out, s, A
        return out * s

    def loss_and_grads(self, dose, dens, target, sigma=None):
        """Masked mean squared error of (out - target/s) and its gradient w.r.t. every parameter."""
        dose = np.asarray(dose, np.float64)
        out, s, A = self.forward(dose, dens, keep=True, sigma=sigma)
        mask = np.asarray(dens) >= 0.1
        e = np.where(mask, out - np.asarray(target, np.float64) / s, 0.0)
        cnt = mask.sum()
        loss = (e ** 2).sum() / cnt
        gout = 2 * e / cnt
        G = np.zeros_like(self.p)
        h = A["g0"]
        G[self.hw:self.hw + 16] = (h * gout[..., None]).reshape(-1, 16).sum(0)
        G[self.hb] = gout.sum()
        dA = {"g0": self.q(gout[..., None] * self.p[self.hw:self.hw + 16] * (h > 0))}
        arch = architecture()
        for i in range(len(arch) - 1, -1, -1):
            mode, cin, cout, a_in, a_out = arch[i]
            off, shape, boff, _ = self.lay[i]
            W, _ = self.weights(i)
            dy = dA[a_out]
            x = A[a_in]
            dW = {0: conv3_dw, 1: down_dw, 2: up_dw}[mode](x, dy)
            G[off:off + np.prod(shape)] = dW.ravel()
            G[boff:boff + cout] = dy.reshape(-1, cout).sum(0)
            if i == 0:
                continue
            if mode == 0:
                dx = conv3_dx(dy, W)
            elif mode == 1:
                dx = down_dx(dy, W, x.shape)
            else:
                dx = up_dx(dy, W)
            dx = dx * (x > 0)
            if a_in.startswith("cat"):
                l = a_in[3:]
                C = dx.shape[-1] // 2
                dA[f"u{l}"] = self.q(dx[..., :C])
                dA[f"s{l}"] = self.q(dx[..., C:])
            elif a_in in dA:
                dA[a_in] = self.q(dA[a_in] + dx)
            else:
                dA[a_in] = self.q(dx)
        return loss, G
