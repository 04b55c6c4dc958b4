"""Pins for the FP64 network oracle (CPU): an independent library convolution, adjoint
identities, finite differences, closed forms and the Adam update rule."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import unet_oracle as U


def _rng(seed=0):
    return np.random.default_rng(seed)


def test_conv3d_matches_scipy_correlate():
    # ci != co and an anisotropic grid catch transposed weights and swapped axes;
    # correlate (not convolve) fixes the tap direction.
    r = _rng(1)
    x = r.standard_normal((2, 4, 5, 6, 3))
    w = r.standard_normal((27, 3, 2))
    b = r.standard_normal(2)
    y = U.conv3d(x, w, b)
    for n in range(2):
        for co in range(2):
            ref = np.full(x.shape[1:4], b[co])
            for ci in range(3):
                k = np.zeros((3, 3, 3))
                for t, (dz, dy, dx) in enumerate(U.TAPS):
                    k[dz + 1, dy + 1, dx + 1] = w[t, ci, co]
                ref += ndimage.correlate(x[n, ..., ci], k, mode="constant", cval=0.0)
            np.testing.assert_allclose(y[n, ..., co], ref, rtol=1e-12, atol=1e-12)


def test_tap_convention_reads_the_stated_neighbour():
    # a single nonzero weight at tap (dz, dy, dx) = (1, -1, 0) copies x[z+1, y-1, x]
    x = _rng(2).standard_normal((1, 4, 4, 4, 1))
    w = np.zeros((27, 1, 1))
    t = (1 + 1) * 9 + (-1 + 1) * 3 + (0 + 1)
    w[t, 0, 0] = 1.0
    y = U.conv3d(x, w)
    assert y[0, 1, 2, 3, 0] == x[0, 2, 1, 3, 0]
    assert y[0, 3, 2, 3, 0] == 0.0   # z + 1 out of range reads zero


def test_conv3d_adjoints():
    r = _rng(3)
    x = r.standard_normal((2, 3, 4, 5, 3))
    w = r.standard_normal((27, 3, 4))
    g = r.standard_normal((2, 3, 4, 5, 4))
    lhs = (U.conv3d(x, w) * g).sum()
    np.testing.assert_allclose(lhs, (x * U.conv3d_grad_input(g, w)).sum(), rtol=1e-12)
    np.testing.assert_allclose(lhs, (w * U.conv3d_grad_weight(x, g)).sum(), rtol=1e-12)


def test_pool_and_upsample_adjoints_and_closed_forms():
    r = _rng(4)
    x = r.standard_normal((2, 4, 6, 8, 3))
    g = r.standard_normal((2, 2, 3, 4, 3))
    np.testing.assert_allclose((U.pool2(x) * g).sum(), (x * U.pool2_adjoint(g)).sum(), rtol=1e-12)
    np.testing.assert_allclose((U.up2(g) * x).sum(), (g * U.up2_adjoint(x)).sum(), rtol=1e-12)
    np.testing.assert_allclose(U.pool2(U.up2(g)), g, rtol=1e-15)
    assert U.pool2(x)[1, 1, 2, 3, 2] == pytest.approx(x[1, 2:4, 4:6, 6:8, 2].mean(), rel=1e-14)


def _problem(levels=3, base=2, dims=(4, 4, 8), N=2, seed=5):
    r = _rng(seed)
    V = int(np.prod(dims))
    y = (r.standard_normal((V, N)) + 1j * r.standard_normal((V, N))) * np.array([1.0, 3.0])[:N]
    t = 2.0 * y + 0.3 * (r.standard_normal((V, N)) + 1j * r.standard_normal((V, N)))
    p = U.he_like(levels, base, r)
    return p, y, t


def test_network_gradient_matches_finite_differences():
    levels, base, dims = 3, 2, (4, 4, 8)
    p, y, t = _problem(levels, base, dims)
    gain = 1.3
    _, G, _ = U.loss_and_grads(p, y, t, dims, levels, base, gain)
    f = lambda q: U.loss_and_grads(q, y, t, dims, levels, base, gain)[0]
    r = _rng(6)
    idx = []
    for s in U.layout(levels, base):   # a weight and the bias of every convolution
        lo = s.w_off + (2 * s.co if s is U.layout(levels, base)[0] else 0)
        idx.append(int(r.integers(lo, s.b_off)))
        idx.append(s.b_off + int(r.integers(0, s.co)))
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (f(p + e) - f(p - e)) / (2 * h)
        assert G[i] == pytest.approx(fd, rel=2e-5, abs=1e-9), i


def test_zero_output_layer_predicts_gain_times_input():
    levels, base, dims = 2, 2, (2, 4, 4)
    p, y, t = _problem(levels, base, dims, seed=7)
    s = U.layout(levels, base)[-1]
    p[s.w_off:s.b_off + s.co] = 0.0
    gain = 0.7
    loss, _, A = U.loss_and_grads(p, y, t, dims, levels, base, gain)
    np.testing.assert_allclose(A["pred"], gain * y, rtol=1e-13)
    rms = np.sqrt((np.abs(y) ** 2).mean(axis=0))
    ref = (np.abs(gain * y / rms - t / rms) ** 2).sum() / (2 * y.size)
    assert loss == pytest.approx(ref, rel=1e-13)


def test_skip_connection_sits_after_the_upsampled_channels():
    # Two levels, c0 = 2: cat_0 = [up(e_1) (4 channels) | e_0 (2 channels)].  A decoder
    # weight on input channel 4 (the first skip channel) at the centre tap, identity
    # afterwards, must reproduce lrelu(e_0[..., 0]) in output channel 0.
    levels, base, dims = 2, 2, (2, 2, 4)
    p, y, _ = _problem(levels, base, dims, seed=8)
    L = U.layout(levels, base)
    for s in L[4:]:
        p[s.w_off:s.b_off + s.co] = 0.0
    centre = 13
    w = np.zeros((27, L[4].ci, L[4].co)); w[centre, 4, 0] = 1.0
    p[L[4].w_off:L[4].b_off] = w.ravel()
    w = np.zeros((27, 2, 2)); w[centre, 0, 0] = 1.0
    p[L[5].w_off:L[5].b_off] = w.ravel()
    w = np.zeros((27, 2, 2)); w[centre, 0, 0] = 1.0
    p[L[6].w_off:L[6].b_off] = w.ravel()
    A = U.forward(p, y, dims, levels, base, 0.0)
    # b_0 and d_0 apply the leaky ReLU twice more to the copied channel
    np.testing.assert_allclose(A["o"][..., 0], U.lrelu(U.lrelu(A["e0"][..., 0])), rtol=1e-15)
    assert not np.allclose(A["o"][..., 0], U.lrelu(U.lrelu(A["cat0"][..., 0])))


def test_adam_closed_forms():
    g = np.array([0.5, -2.0, 1e-3])
    w0 = np.zeros(3)
    lr = 0.01
    w, m, v = U.adam(w0, np.zeros(3), np.zeros(3), g, 1, lr)
    np.testing.assert_allclose(w, -lr * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # a constant gradient keeps the bias-corrected moments at g and g^2
    for step in (2, 3):
        w_prev = w
        w, m, v = U.adam(w, m, v, g, step, lr)
        np.testing.assert_allclose(w - w_prev, -lr * g / (np.abs(g) + 1e-8), rtol=1e-9)


def test_layout_counts():
    # 4 levels of 16..128 channels: 15 convolutions
    L = U.layout(4, 16)
    assert len(L) == 15
    assert [(s.ci, s.co) for s in L] == [(16, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (64, 128),
                                         (128, 128), (192, 64), (64, 64), (96, 32), (32, 32), (48, 16), (16, 16),
                                         (16, 16)]
    assert U.n_params(4, 16) == sum(27 * s.ci * s.co + s.co for s in L)


def test_round_bf16_matches_torch_and_ties_to_even():
    import torch
    r = _rng(9)
    a = (r.standard_normal(20000) * np.exp(r.uniform(-20, 20, 20000))).astype(np.float32)
    ref = torch.as_tensor(a).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(U.round_bf16(a.astype(np.float64)), ref)
    assert U.round_bf16(1 + 2.0 ** -8) == 1.0                   # tie -> even significand
    assert U.round_bf16(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6
    assert U.round_bf16(-(1 + 3 * 2.0 ** -8)) == -(1 + 2.0 ** -6)
    assert U.round_bf16(0.0) == 0.0


def test_storage_rounding_is_applied_only_where_stored():
    # With rounding of stored tensors the loss moves by about the bfloat16 precision,
    # and the identity rounding reproduces the float64 result exactly.
    levels, base, dims = 2, 2, (2, 4, 4)
    p, y, t = _problem(levels, base, dims, seed=10)
    l64, G64, _ = U.loss_and_grads(p, y, t, dims, levels, base, 1.1)
    lid, Gid, _ = U.loss_and_grads(p, y, t, dims, levels, base, 1.1, store=lambda a: a)
    assert lid == l64 and np.array_equal(Gid, G64)
    lq, Gq, A = U.loss_and_grads(p, y, t, dims, levels, base, 1.1, store=U.round_bf16)
    assert 0 < abs(lq - l64) / l64 < 0.05
    assert np.array_equal(A["a0"], U.round_bf16(A["a0"]))   # activations are representable


def test_coordinate_channels():
    """The optional position channels: closed-form values, exact in bfloat16 for grids up
    to 256, placed in channels 2, 3, 4 (x, y, z) of the packed input, and gradients with
    respect to first-layer weights on them that match finite differences."""
    np.testing.assert_array_equal(U.coord_channel(4), [-0.75, -0.25, 0.25, 0.75])
    np.testing.assert_array_equal(U.coord_channel(5), [-0.5, -0.25, 0.0, 0.25, 0.5])
    for n in (1, 3, 64, 100, 128, 255, 256):
        c = U.coord_channel(n)
        assert np.all(np.abs(c) < 1)
        np.testing.assert_array_equal(c, -c[::-1])
        np.testing.assert_array_equal(U.round_bf16(c), c)
    dims = (3, 4, 5)                                   # (nz, ny, nx), x fastest
    x, _ = U.to_channels(np.ones((60, 1)), dims, 8, coords=True)
    assert x[0, 2, 1, 3, 2] == U.coord_channel(5)[3]
    assert x[0, 2, 1, 3, 3] == U.coord_channel(4)[1]
    assert x[0, 2, 1, 3, 4] == U.coord_channel(3)[2]
    assert np.all(x[..., 5:] == 0)
    levels, base, dims, N = 2, 8, (2, 4, 4), 2
    r = _rng(9)
    V = int(np.prod(dims))
    y = r.standard_normal((V, N)) + 1j * r.standard_normal((V, N))
    t = 1.5 * y + 0.3 * (r.standard_normal((V, N)) + 1j * r.standard_normal((V, N)))
    p = U.he_like(levels, base, r, coords=True)
    gain = 1.1
    _, G, _ = U.loss_and_grads(p, y, t, dims, levels, base, gain, coords=True)
    f = lambda q: U.loss_and_grads(q, y, t, dims, levels, base, gain, coords=True)[0]
    s0 = U.layout(levels, base)[0]
    h = 1e-6
    for tap, ci, co in [(13, 2, 0), (4, 3, 5), (22, 4, 7)]:
        i = s0.w_off + (tap * s0.ci + ci) * s0.co + co
        e = np.zeros_like(p)
        e[i] = h
        fd = (f(p + e) - f(p - e)) / (2 * h)
        assert G[i] != 0.0
        assert G[i] == pytest.approx(fd, rel=2e-5, abs=1e-9), (tap, ci, co)


def test_x_taps_folded_into_partial_sums_reproduce_the_convolution():
    """The identity the x-folded tensor-core kernel evaluates: per (dz, dy) pair the three
    x taps' partial sums P_j[x'] = sum_ci W[dz, dy, j - 1][ci] X[x', ci] on the unshifted x
    positions, then Y[x] = P_0[x - 1] + P_1[x] + P_2[x + 1] (zero outside the volume), and
    the mirrored shifts for the data gradient."""
    r = np.random.default_rng(21)
    x = r.standard_normal((1, 4, 5, 9, 16))
    w = r.standard_normal((27, 16, 16))
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    _, D, H, W, _ = x.shape
    for flip in (False, True):
        s = -1 if flip else 1
        y = np.zeros(x.shape[:4] + (16,))
        for pr in range(9):
            dz, dy = s * (pr // 3 - 1), s * (pr % 3 - 1)
            rows = xp[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, :, :]      # all x (with the zero border)
            for j in range(3):
                pj = rows @ w[3 * pr + j]                                  # P_j on x' = -1 .. W
                dx = s * (j - 1)
                y += pj[:, :, :, 1 + dx:1 + dx + W, :]
        ref = U.conv3d_grad_input(x, np.transpose(w, (0, 2, 1))) if flip else U.conv3d(x, w)
        np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)

