"""GPU parity of the network kernels and the executor against the FP64 oracle.

Inputs are bfloat16-exact, so the oracle sees exactly the values the kernels read.
Tolerances follow the arithmetic:
* float32 accumulation of K products: |error| <= (K + 2) 2^-24 sum |x_i w_i|  (the
  standard bound for recursive summation, plus the bias add);
* a bfloat16 result adds round-to-nearest-even: <= 2^-8 relative (8-bit significand);
* the whole network stores every activation and gradient in bfloat16: each rounding
  adds a relative error of RMS about 2^-8/sqrt(3) ~ 0.23 %, and ~30 roundings in a row
  (forward and backward through 15 convolutions) give sqrt(30) x 0.23 % ~ 1.2 % RMS;
  the gate is 3 % relative L2 and cosine similarity >= 0.998;
* against the oracle that rounds the same stored tensors to bfloat16, only the rare
  roundings that float32 (vs float64) accumulation sends the other way remain:
  0.5 % overall, 2 % per layer (small weight gradients are sums with cancellation).
"""
import numpy as np
import pytest
import torch

from oracle import unet_oracle as U

pytestmark = pytest.mark.gpu

dev = "cuda"


def _bf(a):
    """float64 numpy -> (bfloat16 CUDA tensor, the float64 values it holds)."""
    t = torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.to(dev).contiguous(), t.to(torch.float64).numpy()


def _nn():
    from paper_2604_06257_gb300 import build, nn
    build.build()
    return nn


CONV_CASES = [  # (ci, co, (N, nz, ny, nx)) -- every BN tile, ragged voxel counts
    (16, 16, (2, 5, 6, 7)),
    (16, 32, (1, 3, 5, 9)),
    (48, 16, (2, 4, 4, 4)),
    (32, 64, (1, 5, 3, 6)),
    (64, 128, (1, 3, 4, 5)),
    (192, 64, (1, 2, 3, 4)),
    (96, 32, (2, 3, 3, 3)),
]


@pytest.mark.parametrize("ci,co,shape", CONV_CASES)
@pytest.mark.parametrize("act", [False, True])
def test_conv3d_forward(ci, co, shape, act):
    nn = _nn()
    r = np.random.default_rng(ci * 1000 + co)
    x, xh = _bf(r.standard_normal(shape + (ci,)))
    w, wh = _bf(r.standard_normal((27, ci, co)) * np.sqrt(2.0 / (27 * ci)))
    b = torch.as_tensor(r.standard_normal(co).astype(np.float32)).to(dev)
    y = torch.empty(shape + (co,), dtype=torch.bfloat16, device=dev)
    yf = torch.empty(shape + (co,), dtype=torch.float32, device=dev)
    nn.mach_nn_conv3d(x, w, b, y, yf, act=act)
    torch.cuda.synchronize()
    z = U.conv3d(xh, wh, b.cpu().double().numpy())
    ref = U.lrelu(z) if act else z
    bound = (27 * ci + 2) * 2.0 ** -24 * (U.conv3d(np.abs(xh), np.abs(wh)) + np.abs(b.cpu().double().numpy()))
    got = yf.cpu().double().numpy()
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) - bound)
    gb = y.cpu().double().numpy()
    assert np.all(np.abs(gb - ref) <= 2.0 ** -8 * (np.abs(ref) + bound) + bound)


@pytest.mark.parametrize("ci,co,shape", CONV_CASES)
def test_conv3d_flip_is_the_data_gradient(ci, co, shape):
    nn = _nn()
    r = np.random.default_rng(ci * 7 + co)
    gy, gyh = _bf(r.standard_normal(shape + (co,)))
    w, wh = _bf(r.standard_normal((27, ci, co)) * 0.1)
    wt = w.transpose(1, 2).contiguous()          # [27, co, ci]
    gx = torch.empty(shape + (ci,), dtype=torch.float32, device=dev)
    nn.mach_nn_conv3d(gy, wt, None, None, gx, flip=True)
    torch.cuda.synchronize()
    ref = U.conv3d_grad_input(gyh, wh)
    bound = (27 * co + 2) * 2.0 ** -24 * U.conv3d_grad_input(np.abs(gyh), np.abs(wh))
    got = gx.cpu().double().numpy()
    assert np.all(np.abs(got - ref) <= bound)


TC_CASES = CONV_CASES + [(16, 16, (2, 16, 64, 64)), (32, 128, (2, 4, 40, 24)), (16, 256, (1, 3, 17, 9))]


def test_packed_weight_layouts():
    nn = _nn()
    r = np.random.default_rng(5)
    ci, co = 48, 32
    w = torch.as_tensor(r.standard_normal((27, ci, co)).astype(np.float32)).to(dev)
    wpk, wpkt = nn.mach_nn_pack_weights(w, ci, co)
    wb = w.to(torch.bfloat16)
    # forward: [ci/16][27][2][co][8], element (kc, t, g, o, j) = W[t][16kc + 8g + j][o]
    ref = wb.view(27, ci // 16, 2, 8, co).permute(1, 0, 2, 4, 3).reshape(-1)
    assert torch.equal(wpk, ref)
    # flipped: [co/16][27][2][ci][8], element (kc, t, g, i, j) = W[t][i][16kc + 8g + j]
    ref = wb.view(27, ci, co // 16, 2, 8).permute(2, 0, 3, 1, 4).reshape(-1)
    assert torch.equal(wpkt, ref)


@pytest.mark.parametrize("ci,co,shape", TC_CASES)
@pytest.mark.parametrize("act", [False, True])
def test_conv3d_tcgen05_forward(ci, co, shape, act):
    nn = _nn()
    r = np.random.default_rng(ci * 1000 + co + 17)
    x, xh = _bf(r.standard_normal(shape + (ci,)))
    w32 = (r.standard_normal((27, ci, co)) * np.sqrt(2.0 / (27 * ci))).astype(np.float32)
    w, wh = _bf(w32)
    wpk, _ = nn.mach_nn_pack_weights(w.float(), ci, co, flipped=False)
    b = torch.as_tensor(r.standard_normal(co).astype(np.float32)).to(dev)
    y = torch.empty(shape + (co,), dtype=torch.bfloat16, device=dev)
    yf = torch.empty(shape + (co,), dtype=torch.float32, device=dev)
    nn.mach_nn_conv3d_tc(x, wpk, co, b, y, yf, act=act)
    assert nn.mach_nn_device_status() == 0
    z = U.conv3d(xh, wh, b.cpu().double().numpy())
    ref = U.lrelu(z) if act else z
    bound = (27 * ci + 2) * 2.0 ** -24 * (U.conv3d(np.abs(xh), np.abs(wh)) + np.abs(b.cpu().double().numpy()))
    got = yf.cpu().double().numpy()
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) - bound)
    gb = y.cpu().double().numpy()
    assert np.all(np.abs(gb - ref) <= 2.0 ** -8 * (np.abs(ref) + bound) + bound)


@pytest.mark.parametrize("ci,co,shape", CONV_CASES)
def test_conv3d_tcgen05_flip_is_the_data_gradient(ci, co, shape):
    nn = _nn()
    r = np.random.default_rng(ci * 7 + co + 3)
    gy, gyh = _bf(r.standard_normal(shape + (co,)))
    w, wh = _bf(r.standard_normal((27, ci, co)) * 0.1)
    _, wpkt = nn.mach_nn_pack_weights(w.float(), ci, co, forward=False)
    gx = torch.empty(shape + (ci,), dtype=torch.float32, device=dev)
    nn.mach_nn_conv3d_tc(gy, wpkt, ci, None, None, gx, flip=True)
    assert nn.mach_nn_device_status() == 0
    ref = U.conv3d_grad_input(gyh, wh)
    bound = (27 * co + 2) * 2.0 ** -24 * U.conv3d_grad_input(np.abs(gyh), np.abs(wh))
    assert np.all(np.abs(gx.cpu().double().numpy() - ref) <= bound)


FOLD_CASES = [  # 16 output channels: x tiles of 14 with ragged ends, 1 ... 6 input steps, and 7 (27-tap kernel)
    (16, (1, 5, 9, 29)), (32, (2, 3, 17, 15)), (48, (1, 4, 8, 14)), (96, (1, 3, 5, 30)), (112, (1, 2, 4, 6)),
]


@pytest.mark.parametrize("ci,shape", FOLD_CASES)
@pytest.mark.parametrize("tz,stages", [(1, 0), (2, 0), (4, 0), (2, 2), (4, 3)])
@pytest.mark.parametrize("flip", [False, True])
def test_conv3d_tcgen05_x_folded_matches_oracle(ci, shape, tz, stages, flip):
    # the x-folded kernel (three x taps in one N = 48 MMA, partial sums shifted in the
    # epilogue) against the oracle, forward and flipped, and against the 27-tap kernel
    nn = _nn()
    r = np.random.default_rng(ci + 10 * tz + int(flip))
    x, xh = _bf(r.standard_normal(shape + (ci,)))
    w, wh = _bf(r.standard_normal((27, ci, 16)) * np.sqrt(2.0 / (27 * ci)))
    b = torch.as_tensor(r.standard_normal(16).astype(np.float32)).to(dev)
    wt, wth = _bf(r.standard_normal((27, 16, ci)) * 0.1)   # flipped case: a 16 -> ci convolution
    ys = []
    try:
        for fold in (True, False):
            nn.mach_nn_set_conv_fold(fold, tz, stages)
            y = torch.empty(shape + (16,), dtype=torch.float32, device=dev)
            if flip:   # data gradient of the 16 -> ci convolution: input = its output gradient
                _, wpkt = nn.mach_nn_pack_weights(wt.float(), 16, ci, forward=False)
                nn.mach_nn_conv3d_tc(x, wpkt, 16, None, None, y, flip=True)
                ref = U.conv3d_grad_input(xh, wth)
                bound = (27 * ci + 2) * 2.0 ** -24 * U.conv3d_grad_input(np.abs(xh), np.abs(wth))
            else:
                wpk, _ = nn.mach_nn_pack_weights(w.float(), ci, 16, flipped=False)
                nn.mach_nn_conv3d_tc(x, wpk, 16, b, None, y, act=True)
                bb = b.cpu().double().numpy()
                ref = U.lrelu(U.conv3d(xh, wh, bb))
                bound = (27 * ci + 2) * 2.0 ** -24 * (U.conv3d(np.abs(xh), np.abs(wh)) + np.abs(bb))
            assert nn.mach_nn_device_status() == 0
            got = y.cpu().double().numpy()
            assert np.all(np.abs(got - ref) <= bound), (fold, np.max(np.abs(got - ref) - bound))
            ys.append(y)
    finally:
        nn.mach_nn_set_conv_fold(True, 4)
    assert float((ys[0] - ys[1]).abs().max()) <= 1e-5 * float(ys[1].abs().max())


def test_tcgen05_and_mma_sync_agree():
    # the two convolution kernels sum the same products in different orders
    nn = _nn()
    r = np.random.default_rng(8)
    ci, co, shape = 64, 64, (2, 8, 32, 16)
    x, _ = _bf(r.standard_normal(shape + (ci,)))
    w, _ = _bf(r.standard_normal((27, ci, co)) * 0.05)
    wpk, _ = nn.mach_nn_pack_weights(w.float(), ci, co, flipped=False)
    a = torch.empty(shape + (co,), dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    nn.mach_nn_conv3d_tc(x, wpk, co, None, None, a)
    nn.mach_nn_conv3d(x, w, None, None, b)
    torch.cuda.synchronize()
    assert float((a - b).abs().max()) <= 1e-4 * float(b.abs().max())


WGRAD_CASES = [(16, 16), (16, 32), (16, 64), (32, 16), (32, 32), (32, 64), (48, 16), (96, 32), (192, 64),
               (64, 128)]


@pytest.mark.parametrize("ci,co", WGRAD_CASES)
def test_conv3d_weight_gradient(ci, co):
    nn = _nn()
    shape = (2, 6, 9, 10) if ci * co <= 2048 else (1, 5, 6, 7)
    r = np.random.default_rng(ci + 31 * co)
    x, xh = _bf(r.standard_normal(shape + (ci,)))
    g, gh = _bf(r.standard_normal(shape + (co,)))
    dw = torch.zeros((27, ci, co), dtype=torch.float32, device=dev)
    nn.mach_nn_conv3d_wgrad(x, g, dw)
    torch.cuda.synchronize()
    ref = U.conv3d_grad_weight(xh, gh)
    M = int(np.prod(shape))
    bound = (M + 64) * 2.0 ** -24 * U.conv3d_grad_weight(np.abs(xh), np.abs(gh))
    got = dw.cpu().double().numpy()
    assert np.all(np.abs(got - ref) <= bound)


def _ulp_close(got, ref, extra=0.0):
    """Within one bfloat16 rounding of the exact value (plus `extra`)."""
    return np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + extra + 1e-30)


def test_pool_upsample_copy_and_adjoints():
    nn = _nn()
    r = np.random.default_rng(11)
    x, xh = _bf(r.standard_normal((2, 4, 6, 8, 32)))
    p = torch.empty((2, 2, 3, 4, 32), dtype=torch.bfloat16, device=dev)
    nn.mach_nn_pool2(x, p)
    assert _ulp_close(p.cpu().double().numpy(), U.pool2(xh))
    # adjoint, accumulated onto an existing gradient
    gp, gph = _bf(r.standard_normal((2, 2, 3, 4, 32)))
    acc, acch = _bf(r.standard_normal((2, 4, 6, 8, 32)))
    nn.mach_nn_pool2(gp, acc, backward=True, accumulate=True)
    assert _ulp_close(acc.cpu().double().numpy(), acch + U.pool2_adjoint(gph))
    # upsampling into a channel slice, and back
    c, cy, off = 16, 48, 32
    src, srch = _bf(r.standard_normal((2, 2, 3, 4, c)))
    cat = torch.zeros((2, 4, 6, 8, cy), dtype=torch.bfloat16, device=dev)
    nn.mach_nn_up2(src, cat, off=off)
    got = cat.cpu().double().numpy()
    np.testing.assert_array_equal(got[..., off:off + c], U.up2(srch))
    assert not got[..., :off].any()
    gcat, gcath = _bf(r.standard_normal((2, 4, 6, 8, cy)))
    back = torch.empty((2, 2, 3, 4, c), dtype=torch.bfloat16, device=dev)
    nn.mach_nn_up2(gcat, back, off=off, backward=True)
    assert _ulp_close(back.cpu().double().numpy(), U.up2_adjoint(gcath[..., off:off + c]), 2.0 ** -20)
    # channel copies are exact both ways
    e, eh = _bf(r.standard_normal((2, 4, 6, 8, 16)))
    nn.mach_nn_copy_channels(e, cat, off=0)
    np.testing.assert_array_equal(cat.cpu().double().numpy()[..., :16], eh)
    out = torch.empty_like(e)
    nn.mach_nn_copy_channels(gcat, out, off=8, back=True)
    np.testing.assert_array_equal(out.cpu().double().numpy(), gcath[..., 8:24])


def test_data_movement_scalar_paths():
    # channel counts and offsets that are not multiples of 8 take the element-wise kernels
    nn = _nn()
    r = np.random.default_rng(14)
    x, xh = _bf(r.standard_normal((1, 4, 2, 6, 5)))
    p = torch.empty((1, 2, 1, 3, 5), dtype=torch.bfloat16, device=dev)
    nn.mach_nn_pool2(x, p)
    assert _ulp_close(p.cpu().double().numpy(), U.pool2(xh))
    src, srch = _bf(r.standard_normal((1, 2, 1, 3, 5)))
    cat = torch.zeros((1, 4, 2, 6, 13), dtype=torch.bfloat16, device=dev)
    nn.mach_nn_up2(src, cat, off=3)
    np.testing.assert_array_equal(cat.cpu().double().numpy()[..., 3:8], U.up2(srch))
    back = torch.empty((1, 2, 1, 3, 5), dtype=torch.bfloat16, device=dev)
    gcat, gcath = _bf(r.standard_normal((1, 4, 2, 6, 13)))
    nn.mach_nn_up2(gcat, back, off=3, backward=True)
    assert _ulp_close(back.cpu().double().numpy(), U.up2_adjoint(gcath[..., 3:8]), 2.0 ** -20)
    out = torch.empty((1, 4, 2, 6, 5), dtype=torch.bfloat16, device=dev)
    nn.mach_nn_copy_channels(gcat, out, off=7, back=True)
    np.testing.assert_array_equal(out.cpu().double().numpy(), gcath[..., 7:12])


def test_lrelu_backward_and_bias_gradient():
    nn = _nn()
    r = np.random.default_rng(12)
    g, gh = _bf(r.standard_normal((3, 5, 7, 9, 32)))
    y, yh = _bf(r.standard_normal((3, 5, 7, 9, 32)))
    nn.mach_nn_lrelu_bwd(g, y)
    np.testing.assert_array_equal(g.cpu().double().numpy(), np.where(yh > 0, gh, gh / 64.0))
    g1, g1h = _bf(r.standard_normal(37))          # a count the 16-byte path cannot take
    y1, y1h = _bf(r.standard_normal(37))
    nn.mach_nn_lrelu_bwd(g1, y1)
    np.testing.assert_array_equal(g1.cpu().double().numpy(), np.where(y1h > 0, g1h, g1h / 64.0))
    for c in (16, 32, 64, 128):
        gg, ggh = _bf(r.standard_normal((2, 5, 7, 9, c)))
        db = torch.zeros(c, dtype=torch.float32, device=dev)
        nn.mach_nn_bias_grad(gg, db)
        ref = ggh.reshape(-1, c).sum(0)
        bound = (ggh.size // c + 2048) * 2.0 ** -24 * np.abs(ggh).reshape(-1, c).sum(0)
        assert np.all(np.abs(db.cpu().double().numpy() - ref) <= bound)


def test_adam_matches_oracle_and_refreshes_bfloat16_copies():
    nn = _nn()
    r = np.random.default_rng(13)
    ci, co = 32, 16
    n = 27 * ci * co
    w0 = r.standard_normal(n).astype(np.float32)
    w = torch.as_tensor(w0).to(dev)
    m = torch.zeros(n, device=dev)
    v = torch.zeros(n, device=dev)
    wb = torch.empty(n, dtype=torch.bfloat16, device=dev)
    wbt = torch.empty(n, dtype=torch.bfloat16, device=dev)
    wh, mh, vh = w0.astype(np.float64), np.zeros(n), np.zeros(n)
    for step in (1, 2, 3):
        g0 = r.standard_normal(n).astype(np.float32)
        nn.mach_nn_adam(w, m, v, torch.as_tensor(g0).to(dev), step, 1e-2, w_bf16=wb, w_bf16_t=wbt, ci=ci, co=co)
        wh, mh, vh = U.adam(wh, mh, vh, g0.astype(np.float64), step, 1e-2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(w.cpu().double().numpy(), wh, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(m.cpu().double().numpy(), mh, rtol=1e-5, atol=1e-7)
    assert torch.equal(wb, w.to(torch.bfloat16))
    assert torch.equal(wbt.view(27, co, ci), wb.view(27, ci, co).transpose(1, 2))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _cos(a, b):
    return float((a * b).sum() / (np.linalg.norm(a) * np.linalg.norm(b)))


def _layer_tolerances(p64, y, t, dims, levels, base, gain, Gq, floor=2e-2):
    """Per-layer gate for the gradients against the bfloat16-storing oracle: the GPU
    accumulates in float32, so a bfloat16 rounding of a stored tensor flips now and then.
    The oracle's own spread under perturbations of that size (relative 2^-24 before each
    rounding) measures how far such flips move each layer's gradient; the gate is twice
    that spread, and never below `floor`."""
    rng = np.random.default_rng(1234)

    def nudged(x):
        return U.round_bf16(x * (1.0 + rng.uniform(-2.0 ** -24, 2.0 ** -24, np.shape(x))))

    _, Gn, _ = U.loss_and_grads(p64, y, t, dims, levels, base, gain, store=nudged)
    out = {}
    for s in U.layout(levels, base):
        sl = slice(s.w_off, s.b_off + s.co)
        out[s.w_off] = max(floor, 2.0 * _rel(Gn[sl], Gq[sl]))
    return out


@pytest.mark.parametrize("backend", ["tcgen05", "mma.sync"])
@pytest.mark.parametrize("levels,dims,batch", [(4, (16, 8, 8), 2), (2, (6, 4, 10), 3), (1, (3, 5, 7), 1),
                                               (5, (32, 32, 32), 1)])
def test_network_forward_backward_matches_oracle(levels, dims, batch, backend):
    nn = _nn()
    nz, ny, nx = dims
    V = nz * ny * nx
    r = np.random.default_rng(levels * 10 + batch)
    base = 16
    p = U.he_like(levels, base, r).astype(np.float32)
    y = (r.standard_normal((V, batch)) + 1j * r.standard_normal((V, batch))) * (1.0 + np.arange(batch))
    t = 1.5 * y + 0.5 * (r.standard_normal((V, batch)) + 1j * r.standard_normal((V, batch)))
    y = y.astype(np.complex64)
    t = t.astype(np.complex64)
    gain = 0.8
    with nn.UNet(nx, ny, nz, batch, levels=levels, base_ch=base, seed=1) as net:
        assert net.n_params == U.n_params(levels, base)
        net.set_params(p)
        np.testing.assert_array_equal(net.params(), p)
        net.set_gain(gain)
        net.set_backend(backend)
        yd = torch.as_tensor(y).to(dev)
        td = torch.as_tensor(t).to(dev)
        loss = torch.zeros(1, device=dev)
        net.backward(yd, td, loss)
        pred = net.forward(yd)
        torch.cuda.synchronize()
        G = net.grads()
    pr = pred.cpu().numpy().astype(np.complex128)
    p64 = p.astype(np.float64)
    # (1) against the oracle storing the same tensors in bfloat16: the remaining
    # differences come from float32 vs float64 accumulation flipping a rounding now and then
    lq, Gq, Aq = U.loss_and_grads(p64, y, t, dims, levels, base, gain, store=U.round_bf16)
    assert float(loss.item()) == pytest.approx(lq, rel=2e-3)
    assert _rel(pr - gain * y, Aq["pred"] - gain * y) <= 5e-3
    assert _rel(G, Gq) <= 5e-3
    tol = _layer_tolerances(p64, y, t, dims, levels, base, gain, Gq)
    for s in U.layout(levels, base):                                # every layer gets its gradient
        sl = slice(s.w_off, s.b_off + s.co)
        assert _rel(G[sl], Gq[sl]) <= tol[s.w_off], (s, tol[s.w_off])
    # (2) against plain float64: the whole effect of bfloat16 storage
    l64, G64, A64 = U.loss_and_grads(p64, y, t, dims, levels, base, gain)
    assert float(loss.item()) == pytest.approx(l64, rel=3e-2)
    assert _rel(pr - gain * y, A64["pred"] - gain * y) <= 3e-2
    assert _rel(G, G64) <= 3e-2 and _cos(G, G64) >= 0.998


@pytest.mark.parametrize("dims", [(16, 8, 8), (6, 4, 10)])
def test_network_with_coordinate_channels_matches_oracle(dims):
    """Position channels (mach_unet_desc.coords): forward and gradients against the oracle
    storing the same tensors in bfloat16, including the first layer's weights on the
    coordinate channels."""
    nn = _nn()
    nz, ny, nx = dims
    V = nz * ny * nx
    levels, batch, base = 2, 2, 16
    r = np.random.default_rng(77)
    p = U.he_like(levels, base, r, coords=True).astype(np.float32)
    y = (r.standard_normal((V, batch)) + 1j * r.standard_normal((V, batch))).astype(np.complex64)
    t = (1.5 * y + 0.5 * (r.standard_normal((V, batch)) + 1j * r.standard_normal((V, batch)))).astype(np.complex64)
    gain = 0.8
    with nn.UNet(nx, ny, nz, batch, levels=levels, base_ch=base, seed=1, coords=True) as net:
        net.set_params(p)
        net.set_gain(gain)
        yd, td = torch.as_tensor(y).to(dev), torch.as_tensor(t).to(dev)
        loss = torch.zeros(1, device=dev)
        net.backward(yd, td, loss)
        pred = net.forward(yd)
        torch.cuda.synchronize()
        G = net.grads()
    p64 = p.astype(np.float64)
    lq, Gq, Aq = U.loss_and_grads(p64, y, t, dims, levels, base, gain, store=U.round_bf16, coords=True)
    assert float(loss.item()) == pytest.approx(lq, rel=2e-3)
    pr = pred.cpu().numpy().astype(np.complex128)
    assert _rel(pr - gain * y, Aq["pred"] - gain * y) <= 5e-3
    assert _rel(G, Gq) <= 5e-3
    s0 = U.layout(levels, base)[0]
    w0 = G[s0.w_off:s0.b_off].reshape(27, s0.ci, s0.co)
    w0q = Gq[s0.w_off:s0.b_off].reshape(27, s0.ci, s0.co)
    assert np.abs(w0[:, 2:5]).max() > 0
    assert _rel(w0[:, 2:5], w0q[:, 2:5]) <= 2e-2
    # without coordinates the same parameters give another prediction
    with nn.UNet(nx, ny, nz, batch, levels=levels, base_ch=base, seed=1) as net:
        net.set_params(p)
        net.set_gain(gain)
        pred0 = net.forward(yd)
        torch.cuda.synchronize()
    assert _rel(pred0.cpu().numpy() - gain * y, pr - gain * y) > 1e-2


@pytest.mark.parametrize("backend", ["tcgen05", "mma.sync"])
def test_five_levels_training_step_keeps_every_weight_copy_current(backend):
    """Five levels: the level-3 decoder convolution reads 256 + 128 channels, so its data
    gradient has 384 output channels and runs on the warp-MMA kernel even in tcgen05 mode.
    After an Adam step, the gradients must be those of the updated parameters, so every
    bfloat16 weight copy a kernel reads is current."""
    nn = _nn()
    levels, base, batch, dims = 5, 16, 1, (32, 32, 32)
    nz, ny, nx = dims
    V = nz * ny * nx
    r = np.random.default_rng(55)
    p = U.he_like(levels, base, r).astype(np.float32)
    y = ((r.standard_normal((V, batch)) + 1j * r.standard_normal((V, batch)))).astype(np.complex64)
    t = (1.5 * y + 0.5 * (r.standard_normal((V, batch)) + 1j * r.standard_normal((V, batch)))).astype(np.complex64)
    gain = 0.8
    with nn.UNet(nx, ny, nz, batch, levels=levels, base_ch=base, seed=1) as net:
        net.set_params(p)
        net.set_gain(gain)
        net.set_backend(backend)
        yd = torch.as_tensor(y).to(dev)
        td = torch.as_tensor(t).to(dev)
        loss = torch.zeros(1, device=dev)
        net.train_step(yd, td, 1e-2, loss)
        p1 = net.params().copy()
        net.backward(yd, td, loss)
        torch.cuda.synchronize()
        G = net.grads()
    assert np.abs(p1 - p).max() > 1e-3                                # the step moved the weights
    lq, Gq, Aq = U.loss_and_grads(p1.astype(np.float64), y, t, dims, levels, base, gain, store=U.round_bf16)
    assert float(loss.item()) == pytest.approx(lq, rel=2e-3)
    assert _rel(G, Gq) <= 5e-3
    tol = _layer_tolerances(p1.astype(np.float64), y, t, dims, levels, base, gain, Gq)
    for s in U.layout(levels, base):
        sl = slice(s.w_off, s.b_off + s.co)
        assert _rel(G[sl], Gq[sl]) <= tol[s.w_off], (s, tol[s.w_off])


def test_fresh_network_predicts_gain_times_input_and_learns():
    nn = _nn()
    nz, ny, nx, batch = 16, 16, 16, 2
    V = nz * ny * nx
    r = np.random.default_rng(21)
    y = ((r.standard_normal((V, batch)) + 1j * r.standard_normal((V, batch)))).astype(np.complex64)
    yd = torch.as_tensor(y).to(dev)
    # a target the network can fit: a smoothed copy of the input
    yv = torch.as_tensor(y.T.reshape(batch, nz, ny, nx))
    sm = sum(torch.roll(yv, s, d) for d in (1, 2, 3) for s in (-1, 1)) / 6.0
    td = sm.reshape(batch, V).T.contiguous().to(dev)
    with nn.UNet(nx, ny, nz, batch, levels=4, base_ch=16, seed=3) as net:
        net.set_gain(0.5)
        pred = net.forward(yd)
        torch.cuda.synchronize()
        np.testing.assert_allclose(pred.cpu().numpy(), 0.5 * y, rtol=1e-6, atol=1e-6)
        loss = torch.zeros(1, device=dev)
        hist = []
        for _ in range(60):
            net.train_step(yd, td, 2e-3, loss)
            hist.append(float(loss.item()))
    assert hist[-1] < 0.5 * hist[0], hist[::10]


def test_inference_only_network_matches_and_refuses_training():
    nn = _nn()
    r = np.random.default_rng(31)
    p = U.he_like(4, 16, r).astype(np.float32)
    x = torch.as_tensor((r.standard_normal((16 * 16 * 16, 2)) + 1j * r.standard_normal((16 * 16 * 16, 2)))
                        .astype(np.complex64)).to(dev)
    with nn.UNet(16, 16, 16, 2) as full, nn.UNet(16, 16, 16, 2, inference_only=True) as lite:
        assert lite.device_bytes < 0.6 * full.device_bytes
        for net in (full, lite):
            net.set_params(p)
            net.set_gain(0.7)
        a, b = full.forward(x), lite.forward(x)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        loss = torch.zeros(1, device=dev)
        with pytest.raises(Exception):
            lite.train_step(x, x, 1e-3, loss)
        with pytest.raises(Exception):
            lite.grads()


def test_das_and_network_replay_from_one_cuda_graph():
    # the learned path (few-angle DAS, then the network) captured once and replayed: every
    # launch is stream-ordered and nothing synchronises the host
    nn = _nn()
    import synth
    import paper_2604_06257_gb300 as m
    from paper_2604_06257_gb300 import learned as Lc
    acq = Lc.acquisition(16, 8, "few", 512)
    iq = synth.random_iq(acq, 9, device=dev)
    r = np.random.default_rng(32)
    with m.Plan(**m.plan_kwargs(acq)) as plan, nn.UNet(16, 16, 16, 8, inference_only=True) as net:
        net.set_params(U.he_like(4, 16, r).astype(np.float32))
        y = torch.empty((acq.n_vox, 8), dtype=torch.complex64, device=dev)
        out = torch.empty_like(y)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            plan.run(iq, y, stream=s)
            net.forward(y, out, stream=s)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        eager = out.clone()
        out.zero_()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            plan.run(iq, y)
            net.forward(y, out)
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, eager)


@pytest.mark.parametrize("ci,co", [(16, 16), (64, 128)])   # resident and streamed weights
def test_tcgen05_bounded_waits_report_timeout_and_context_survives(ci, co):
    nn = _nn()
    r = np.random.default_rng(ci + co)
    shape = (1, 4, 16, 16)
    x, xh = _bf(r.standard_normal(shape + (ci,)))
    w, wh = _bf(r.standard_normal((27, ci, co)) * 0.1)
    wpk, _ = nn.mach_nn_pack_weights(w.float(), ci, co, flipped=False)
    y = torch.empty(shape + (co,), dtype=torch.float32, device=dev)
    assert nn.mach_nn_device_status() == 0
    nn.mach_nn_debug_conv(True, 1 << 12)          # no copies are issued: every wait runs out
    try:
        nn.mach_nn_conv3d_tc(x, wpk, co, None, None, y)
        assert nn.mach_nn_device_status() == 5     # MACH_ERR_TIMEOUT, reported once
    finally:
        nn.mach_nn_debug_conv(False, 0)
    assert nn.mach_nn_device_status() == 0
    nn.mach_nn_conv3d_tc(x, wpk, co, None, None, y)   # the same context computes correctly
    assert nn.mach_nn_device_status() == 0
    ref = U.conv3d(xh, wh)
    bound = (27 * ci + 2) * 2.0 ** -24 * U.conv3d(np.abs(xh), np.abs(wh))
    assert np.all(np.abs(y.cpu().double().numpy() - ref) <= bound)
