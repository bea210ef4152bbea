"""Pins of the denoiser oracle (oracle/unet.py): each layer against SciPy's
correlation, adjoint identities for the data and weight gradients, and finite
differences of the full masked-MSE loss."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import unet as U


def rnd(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.14159], np.float32)
    r = U.bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -6 and r[3] == -2.5
    assert abs(r[4] - 3.140625) < 1e-12


def test_conv3_matches_scipy_correlate():
    x = rnd((6, 5, 7, 3), 1)
    W = rnd((27, 3, 2), 2)
    y = U.conv3(x, W)
    for n in range(2):
        ref = np.zeros(x.shape[:3])
        for c in range(3):
            k = np.zeros((3, 3, 3))
            for t in range(27):
                k[t // 9, t // 3 % 3, t % 3] = W[t, c, n]     # (z, y, x) order
            ref += ndimage.correlate(x[..., c], k, mode="constant", cval=0.0)
        assert np.allclose(y[..., n], ref, atol=1e-12)


def test_down_and_up_match_definitions():
    x = rnd((4, 6, 8, 3), 3)
    W = rnd((8, 3, 5), 4)
    y = U.down(x, W)
    for z, yy, xx in [(0, 0, 0), (1, 2, 3), (1, 1, 0)]:
        ref = sum(x[2 * z + (t >> 2), 2 * yy + ((t >> 1) & 1), 2 * xx + (t & 1)] @ W[t] for t in range(8))
        assert np.allclose(y[z, yy, xx], ref)
    xc = rnd((2, 3, 4, 5), 5)
    Wu = rnd((8, 5, 3), 6)
    yu = U.up(xc, Wu)
    assert np.allclose(yu[3, 5, 7], xc[1, 2, 3] @ Wu[7])
    assert np.allclose(yu[2, 4, 6], xc[1, 2, 3] @ Wu[0])


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_layer_adjoints(mode):
    fine = (6, 4, 8)
    if mode == 0:
        x, W = rnd(fine + (3,), 7), rnd((27, 3, 4), 8)
        y = U.conv3(x, W)
        dy = rnd(y.shape, 9)
        dx, dW = U.conv3_dx(dy, W), U.conv3_dw(x, dy)
    elif mode == 1:
        x, W = rnd(fine + (3,), 7), rnd((8, 3, 4), 8)
        y = U.down(x, W)
        dy = rnd(y.shape, 9)
        dx, dW = U.down_dx(dy, W, x.shape), U.down_dw(x, dy)
    else:
        x, W = rnd((3, 2, 4, 3), 7), rnd((8, 3, 4), 8)
        y = U.up(x, W)
        dy = rnd(y.shape, 9)
        dx, dW = U.up_dx(dy, W), U.up_dw(x, dy)
    # <dy, L(x, W)> is bilinear: its gradients are the adjoint maps
    s = (dy * y).sum()
    assert abs((dx * x).sum() - s) < 1e-9 * abs(s)
    assert abs((dW * W).sum() - s) < 1e-9 * abs(s)


def test_network_gradients_by_finite_differences():
    rng = np.random.default_rng(11)
    n = U.num_params()
    p = rng.standard_normal(n) * 0.05
    net_shape = (8, 8, 8)
    dose = rng.random(net_shape)
    dens = rng.uniform(0.0, 1.5, net_shape)
    target = dose * 1.1 + 0.05
    net = U.UNet(p, bf16_storage=False)
    loss, G = net.loss_and_grads(dose, dens, target)
    lay, hw, hb = U.param_layout()
    picks = [lay[0][0] + 5, lay[3][0] + 17, lay[9][2] + 3, lay[11][0] + 40, lay[19][0] + 2, lay[19][2], hw + 3, hb]
    for i in picks:
        h = 1e-6
        pp = p.copy(); pp[i] += h
        lp, _ = U.UNet(pp, bf16_storage=False).loss_and_grads(dose, dens, target)
        pm = p.copy(); pm[i] -= h
        lm, _ = U.UNet(pm, bf16_storage=False).loss_and_grads(dose, dens, target)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - G[i]) <= 1e-5 * max(1.0, abs(fd)) + 1e-9, (i, fd, G[i])


def test_parameter_count():
    # 3x3x3 convolutions and 2x2x2 up/down convolutions of the 16-32-64-128 U-Net plus the head
    n = U.num_params()
    assert 1_500_000 < n < 2_500_000
