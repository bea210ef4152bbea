"""The tensor-core denoiser against its numpy oracle (oracle/unet.py): every layer kind's
forward, data gradient and weight gradient, the whole network's output and parameter
gradients, training progress, and the plain-Monte-Carlo fallback."""
import numpy as np
import pytest

from oracle import unet as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ocmc():
    from paper_1503_01722_gb300 import build
    build.build()
    from paper_1503_01722_gb300 import ocmc as m
    return m


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-30))


CASES = [(0, 16, 16), (0, 32, 16), (0, 16, 32), (0, 32, 32), (0, 64, 32), (0, 32, 64), (0, 64, 64), (0, 64, 128),
         (0, 128, 64), (0, 128, 128),
         (1, 16, 32), (1, 32, 64), (1, 64, 128), (2, 128, 64), (2, 64, 32), (2, 32, 16)]


@pytest.mark.parametrize("mode,cin,cout", CASES)
def test_layer_matches_oracle(ocmc, mode, cin, cout):
    rng = np.random.default_rng(mode * 1000 + cin + cout)
    fine = (10, 12, 14)                       # 1680 voxels: several 128-row tiles and a ragged tail
    coarse = tuple(s // 2 for s in fine)
    gin = coarse if mode == 2 else fine
    gout = coarse if mode == 1 else fine
    taps = 27 if mode == 0 else 8
    x = U.bf16(rng.standard_normal(gin + (cin,)))
    W = U.bf16(rng.standard_normal((taps, cin, cout)) / np.sqrt(taps * cin))
    dy = U.bf16(rng.standard_normal(gout + (cout,)))
    y, dx, dw = ocmc.unet_test_layer(mode, fine, cin, cout, x, W, dy)
    if mode == 0:
        yr, dxr, dwr = U.conv3(x, W), U.conv3_dx(dy, W), U.conv3_dw(x, dy)
    elif mode == 1:
        yr, dxr, dwr = U.down(x, W), U.down_dx(dy, W, x.shape), U.down_dw(x, dy)
    else:
        yr, dxr, dwr = U.up(x, W), U.up_dx(dy, W), U.up_dw(x, dy)
    # y and dx are stored in BF16 (relative rounding 2^-9); dW is FP32
    assert np.allclose(y, yr, rtol=8e-3, atol=1e-2 * np.abs(yr).max())
    assert np.allclose(dx, dxr, rtol=8e-3, atol=1e-2 * np.abs(dxr).max())
    assert rel_l2(y, yr) < 4e-3 and rel_l2(dx, dxr) < 4e-3
    assert np.allclose(dw, dwr, rtol=1e-4, atol=1e-4 * np.abs(dwr).max())


@pytest.mark.parametrize("cin,cout", [(16, 16), (32, 16), (32, 32), (32, 64), (64, 32), (64, 64), (128, 64),
                                      (128, 128)])
def test_conv3_large_grid(ocmc, cin, cout):
    """A grid of 190+ output tiles per channel slice, so every block of the persistent
    tensor-memory kernel runs several tiles (both accumulator sets, every halo stage reused);
    for 64 and 128 input channels the blocks also split the output channels into slices. The
    weight gradient of the 16- and 32-channel layers runs on tcgen05 too: every block then
    accumulates over dozens of rows (all stages reused), with two or more row segments per x
    line where the grid is 128 voxels wide."""
    rng = np.random.default_rng(cin * 7 + cout)
    fine = (48, 80, 128) if cin < 64 else (32, 48, 64)
    x = U.bf16(rng.standard_normal(fine + (cin,)))
    W = U.bf16(rng.standard_normal((27, cin, cout)) / np.sqrt(27 * cin))
    dy = U.bf16(rng.standard_normal(fine + (cout,)))
    y, dx, dw = ocmc.unet_test_layer(0, fine, cin, cout, x, W, dy)
    yr, dxr = U.conv3(x, W), U.conv3_dx(dy, W)
    assert np.allclose(y, yr, rtol=8e-3, atol=1e-2 * np.abs(yr).max())
    assert np.allclose(dx, dxr, rtol=8e-3, atol=1e-2 * np.abs(dxr).max())
    dwr = U.conv3_dw(x, dy)
    assert np.allclose(dw, dwr, rtol=1e-4, atol=1e-4 * np.abs(dwr).max())


@pytest.mark.parametrize("mode,cin,cout", [(2, 32, 16), (2, 64, 32), (2, 128, 64), (1, 16, 32), (1, 32, 64),
                                            (1, 64, 128)])
def test_strided_conv_large_grid(ocmc, mode, cin, cout):
    """The 2x2x2 convolutions on the tensor-memory path -- DOWN (stride 2) and UP (transposed),
    forward and data gradient of each layer kind -- over 288 to 576 tiles of 128 coarse voxels,
    so that every persistent block runs several tiles through its accumulator sets and input
    stages."""
    rng = np.random.default_rng(mode * 100 + cin + cout)
    fine = (48, 96, 64) if max(cin, cout) >= 64 else (48, 80, 128)
    coarse = tuple(s // 2 for s in fine)
    gin = coarse if mode == 2 else fine
    gout = coarse if mode == 1 else fine
    x = U.bf16(rng.standard_normal(gin + (cin,)))
    W = U.bf16(rng.standard_normal((8, cin, cout)) / np.sqrt(8 * cin))
    dy = U.bf16(rng.standard_normal(gout + (cout,)))
    y, dx, _ = ocmc.unet_test_layer(mode, fine, cin, cout, x, W, dy)
    if mode == 2:
        pairs = ((y, U.up(x, W)), (dx, U.up_dx(dy, W)))
    else:
        pairs = ((y, U.down(x, W)), (dx, U.down_dx(dy, W, x.shape)))
    for got, ref in pairs:
        assert np.allclose(got, ref, rtol=8e-3, atol=1e-2 * np.abs(ref).max())
        assert rel_l2(got, ref) < 4e-3


def test_tensor_memory_path_matches_mma_path(ocmc, monkeypatch):
    """The network with its 3x3x3 convolutions on tcgen05 and with every layer on mma.sync:
    the same arithmetic in a different summation order (outputs and gradients agree to BF16
    rounding)."""
    import torch
    shape = (32, 32, 32)
    dose, dens, target = random_case(shape, 13)
    td, tr, tt = (torch.from_numpy(a).cuda() for a in (dose, dens, target))
    res = []
    for mode in ("tc", "mma"):
        if mode == "mma":
            monkeypatch.setenv("OCMC_UNET_KERNELS", "mma")
        net = ocmc.UNet(shape, seed=21)
        p = net.params()
        p[-17:-1] = np.random.default_rng(5).standard_normal(16) * 0.2
        net.set_params(p)
        out = torch.empty_like(td)
        net.forward(td, tr, out)
        net.train_step(td, tr, tt, lr=0.0)
        res.append((out.cpu().numpy(), net.params(grads=True)))
        net.close()
    assert rel_l2(res[0][0], res[1][0]) < 1e-2
    assert rel_l2(res[0][1], res[1][1]) < 0.1


def random_case(shape, seed):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*[np.linspace(-1, 1, n) for n in shape], indexing="ij")
    target = np.exp(-4 * (x ** 2 + y ** 2)) * np.exp(-0.5 * (z + 1))
    dose = np.maximum(target * (1 + 0.3 * rng.standard_normal(shape)), 0)
    dens = np.where(rng.random(shape) < 0.1, 0.05, rng.uniform(0.3, 1.8, shape))
    return dose.astype(np.float32), dens.astype(np.float32), target.astype(np.float32)


def test_network_output_and_gradients_match_oracle(ocmc):
    import torch
    shape = (16, 16, 16)
    net = ocmc.UNet(shape, seed=3)
    p = net.params().astype(np.float64)
    p[-17:-1] = np.random.default_rng(5).standard_normal(16) * 0.2     # a head that passes signal
    net.set_params(p)
    dose, dens, target = random_case(shape, 7)
    sigma = (0.05 * dose + 0.01 * dose.max()).astype(np.float32)
    td, tr, tt, ts = (torch.from_numpy(a).cuda() for a in (dose, dens, target, sigma))
    out = torch.empty_like(td)
    net.forward(td, tr, out, sigma=ts)
    ref = U.UNet(p.astype(np.float32).astype(np.float64), bf16_storage=True)
    assert rel_l2(out.cpu().numpy(), ref.forward(dose, dens, sigma=sigma)) < 1e-2
    net.forward(td, tr, out)                              # without sigma: channel 2 is zero
    assert rel_l2(out.cpu().numpy(), ref.forward(dose, dens)) < 1e-2
    loss = net.train_step(td, tr, tt, lr=0.0, sigma=ts)
    G = net.params(grads=True)
    lr_, Gr = ref.loss_and_grads(dose, dens, target, sigma=sigma)
    assert abs(loss - lr_) < 1e-2 * lr_
    # Deep-layer gradients are sums with heavy cancellation at random initialisation, so the
    # BF16 rounding of stored activations and gradients moves them by up to ~25% (fp64 oracle
    # vs BF16 oracle: the "gap"). Two BF16 evaluations that sum in different orders round some
    # stored values differently; from there on their rounding errors are independent, so they
    # may differ by up to about sqrt(2) x the gap. The bound per layer is 1.5 x the gap (at
    # least 3%); measured, mma.sync kernels sit at 0.5-0.7 and tcgen05 kernels at 0.7-1.1 of
    # it. A wiring mistake (wrong skip, missing ReLU mask, swapped operand) gives errors of
    # order 1, and every kernel is checked on its own to BF16 rounding by the layer tests.
    _, G64 = U.UNet(p.astype(np.float32).astype(np.float64), bf16_storage=False).loss_and_grads(
        dose, dens, target, sigma=sigma)
    lay, hw, hb = U.param_layout()
    rows, bad = [], []
    for i, (off, shp, boff, cout) in enumerate(lay):
        n = int(np.prod(shp))
        for name, sl in (("W", slice(off, off + n)), ("b", slice(boff, boff + cout))):
            err, gap = rel_l2(G[sl], Gr[sl]), rel_l2(Gr[sl], G64[sl])
            tol = max(0.03, 1.5 * gap)
            rows.append(f"{i:2d} {name} err {err:.4f} gap {gap:.4f} tol {tol:.4f}")
            if err > tol:
                bad.append(rows[-1])
    assert not bad, "\n".join(rows)
    assert rel_l2(G[hw:hw + 17], Gr[hw:hw + 17]) < 2e-2


def test_adam_first_step(ocmc):
    """Adam's first step (bias-corrected moments m = g, v = g^2) moves every parameter by
    lr * g / (|g| + eps) against its gradient."""
    import torch
    shape = (16, 16, 16)
    net = ocmc.UNet(shape, seed=4)
    dose, dens, target = random_case(shape, 11)
    td, tr, tt = (torch.from_numpy(a).cuda() for a in (dose, dens, target))
    p0 = net.params()
    net.train_step(td, tr, tt, lr=0.0)
    g = net.params(grads=True)
    assert np.array_equal(net.params(), p0)                     # lr = 0: gradients only
    lr = 1e-3
    net.train_step(td, tr, tt, lr=lr)
    assert np.array_equal(net.params(grads=True), g)           # deterministic gradients
    g64 = g.astype(np.float64)
    expect = p0 - lr * g64 / (np.abs(g64) + 1e-8)
    assert np.allclose(net.params(), expect, rtol=0, atol=2e-6 * lr + 1e-7 * np.abs(p0).max())
    net.set_params(p0)                                         # restarts Adam
    net.train_step(td, tr, tt, lr=lr)
    assert np.allclose(net.params(), expect, rtol=0, atol=2e-6 * lr + 1e-7 * np.abs(p0).max())


def test_training_reduces_loss(ocmc):
    import torch
    shape = (32, 32, 32)
    net = ocmc.UNet(shape, seed=1)
    dose, dens, target = random_case(shape, 9)
    td, tr, tt = (torch.from_numpy(a).cuda() for a in (dose, dens, target))
    losses = [net.train_step(td, tr, tt, lr=1e-3) for _ in range(150)]
    assert np.mean(losses[-10:]) < 0.85 * losses[0], (losses[0], losses[-10:])


def test_denoise_fallback(ocmc):
    import torch
    import ocmc_inputs as I
    ph = I.homogeneous((16, 16, 16), (1.0, 1.0, 1.0))
    net = ocmc.UNet(ph.density.shape, seed=2)
    with ocmc.Engine(0) as e:
        e.create_phantom(ph)
        e.set_source(I.beam_on(ph, 0, I.mono(2.0), (6, 6), 100.0))
        e.run(200_000, seed=1)
        D, S = e.dose()
        out = torch.empty(ph.density.shape, dtype=torch.float32, device="cuda")
        flag = torch.empty_like(out)
        # tiny k: every voxel whose network value differs from plain MC keeps the plain value
        ocmc.denoise(e, net, 1e-6, out, flag)
        o, f = out.cpu().numpy(), flag.cpu().numpy()
        assert np.array_equal(o[f == 1], D[f == 1]) and f.mean() > 0.5
        # huge k: the network output
        ocmc.denoise(e, net, 1e30, out, flag)
        ref = torch.empty_like(out)
        net.forward(torch.from_numpy(D).cuda(), torch.from_numpy(ph.density).cuda(), ref,
                    sigma=torch.from_numpy(S).cuda())
        assert flag.sum().item() == 0 and torch.equal(out, ref)
        # moderate k: the rule itself, |denoised - plain| > k * pooled sigma, with sigma pooled
        # as the root of the mean variance over the 3x3x3 neighbourhood (float32, same order)
        r = ref.cpu().numpy()
        S2 = (S.astype(np.float32) ** 2).astype(np.float32)
        nz, ny, nx = S2.shape
        pad = np.zeros((nz + 2, ny + 2, nx + 2), np.float32)
        pad[1:-1, 1:-1, 1:-1] = S2
        one = np.zeros_like(pad)
        one[1:-1, 1:-1, 1:-1] = 1
        s2 = np.zeros_like(S2)
        cnt = np.zeros_like(S2)
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    sl = (slice(1 + dz, 1 + dz + nz), slice(1 + dy, 1 + dy + ny), slice(1 + dx, 1 + dx + nx))
                    s2 = (s2 + pad[sl]).astype(np.float32)
                    cnt = cnt + one[sl]
        sig = np.sqrt((s2 / cnt).astype(np.float32))
        ratio = np.abs(r - D)[sig > 0] / sig[sig > 0]
        k = np.float32(np.median(ratio))          # a k that splits the voxels
        ocmc.denoise(e, net, float(k), out, flag)
        expect = np.abs(r - D) > k * np.sqrt((s2 / cnt).astype(np.float32))
        f = flag.cpu().numpy() == 1
        assert 0 < f.sum() < f.size and np.array_equal(f, expect)
        assert np.array_equal(out.cpu().numpy(), np.where(expect, D, r))


def test_tensor_memory_wait_timeout_is_reported_and_recoverable(ocmc):
    """The bounded waits of the tcgen05 convolution: the test hook makes one wait per block run
    out (a barrier that nothing completes, 1 ms limit) after the block's first tile, so copies
    and MMAs are in flight when it gives up. A training step (learning rate 0: the weights stay)
    must return OCMC_ERR_TIMEOUT, and with the hook off the same network gives the same output
    as before, bit for bit."""
    import torch
    shape = (64, 64, 64)
    rng = np.random.default_rng(5)
    dose = torch.from_numpy(rng.random(shape, dtype=np.float32)).cuda()
    dens = torch.from_numpy(np.full(shape, 1.0, np.float32)).cuda()
    net = ocmc.UNet(shape, seed=3)
    out0 = torch.empty_like(dose)
    net.forward(dose, dens, out0)
    torch.cuda.synchronize()
    try:
        ocmc.unet_test_stall(1, 1_000_000)
        with pytest.raises(ocmc.OcmcError) as x:
            net.train_step(dose, dens, dose, 0.0)
        assert x.value.status == ocmc.ERR_TIMEOUT
    finally:
        ocmc.unet_test_stall(-1, 0)
    out2 = torch.empty_like(dose)
    net.forward(dose, dens, out2)
    torch.cuda.synchronize()
    assert torch.equal(out0, out2)
    net.close()
