"""FP64 oracle of the learned compounding network (a small 3D U-Net).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's
CPU-baseline leg may import this; the product path never does.  It shares no code with
the CUDA library.  Plain numpy in float64; every operation is its definition written
out (one library matmul per convolution tap), with no blocking or fusion.

The paper has no learned component (it only notes, in Sec. 4, that beamformed volumes
can stay on the GPU for downstream machine learning); the network follows the stated
design of the learned-compounding configuration: 4 levels, 16-128 channels, 3x3x3
kernels.  Definitions used here (and by the library):

* activations channels-last [N, D, H, W, C]; weights [27, C_in, C_out], tap
  t = (dz+1)*9 + (dy+1)*3 + (dx+1) reading voxel (z+dz, y+dy, x+dx), zero outside;
* leaky ReLU with slope 1/64; 2x average pooling; nearest-neighbour 2x upsampling;
* level l has c0 * 2^l channels; encoder a_l = lrelu(conv(in_l)), e_l = lrelu(conv(a_l)),
  in_l = pool(e_{l-1}); decoder (L-2 .. 0) cat_l = [up(d_{l+1}) | e_l] with d_{L-1} = e_{L-1},
  b_l = lrelu(conv(cat_l)), d_l = lrelu(conv(b_l)); output o = conv(d_0);
* input x = volume / rms (rms over the volume's voxels of |y|), channels (re, im, 0, ...), or
  (re, im, cx, cy, cz, 0, ...) with the voxel position as coordinate channels;
  prediction = rms * (gain * x + o[..., :2]); loss = mean over volumes, voxels and
  (re, im) of (o + gain * x - target / rms)^2;
* Adam (Kingma & Ba 2015, Algorithm 1) with bias correction.

Backward passes are the adjoints of these definitions, derived by hand; the tests pin
them against finite differences and adjoint identities.

``store``: optional rounding applied wherever the library stores a tensor in bfloat16
(``round_bf16``: round to 8 significant bits, ties to even): the packed input, every
activation, every activation gradient, and the weights used by the convolutions (the
weight gradient is then taken with respect to the rounded weights, as the library's
float32 master weights receive it).  With ``store=None`` everything stays float64.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Tuple

import numpy as np

LEAK = 1.0 / 64.0
TAPS = [(t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1) for t in range(27)]


# ------------------------------------------------------------------------ ops ----
def round_bf16(a):
    """Round to the nearest number with 8 significant bits, ties to even (the bfloat16
    significand; exponent range not modelled)."""
    a = np.asarray(a, dtype=np.float64)
    m, e = np.frexp(a)                  # a = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.round(m * 256.0) / 256.0, e)


def _shifted(xp: np.ndarray, off, shape) -> np.ndarray:
    """View of the zero-padded tensor xp at offset (dz, dy, dx) with the unpadded shape."""
    dz, dy, dx = off
    _, D, H, W, _ = shape
    return xp[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W, :]


def _pad(x: np.ndarray) -> np.ndarray:
    return np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))


def conv3d(x: np.ndarray, w: np.ndarray, b=None) -> np.ndarray:
    """y[n,z,y,x,co] = b[co] + sum_{t,ci} x[n, z+dz, y+dy, x+dx, ci] w[t, ci, co]."""
    xp = _pad(np.asarray(x, dtype=np.float64))
    y = np.zeros(x.shape[:4] + (w.shape[2],))
    for t, off in enumerate(TAPS):
        y += _shifted(xp, off, x.shape) @ w[t]
    if b is not None:
        y += b
    return y


def conv3d_grad_input(gy: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Adjoint of conv3d in x: every output gradient goes back to the voxel it read,
    gx[n, z+dz, y+dy, x+dx, ci] += gy[n, z, y, x, co] w[t, ci, co]."""
    N, D, H, W, _ = gy.shape
    shape = (N, D, H, W, w.shape[1])
    gxp = np.zeros((N, D + 2, H + 2, W + 2, w.shape[1]))
    for t, off in enumerate(TAPS):
        _shifted(gxp, off, shape)[...] += gy @ w[t].T
    return gxp[:, 1:-1, 1:-1, 1:-1, :]


def conv3d_grad_weight(x: np.ndarray, gy: np.ndarray) -> np.ndarray:
    """gw[t, ci, co] = sum over voxels of x[v + off(t), ci] gy[v, co]."""
    xp = _pad(np.asarray(x, dtype=np.float64))
    Ci, Co = x.shape[4], gy.shape[4]
    gw = np.zeros((27, Ci, Co))
    g2 = gy.reshape(-1, Co)
    for t, off in enumerate(TAPS):
        gw[t] = _shifted(xp, off, x.shape).reshape(-1, Ci).T @ g2
    return gw


def lrelu(z):
    return np.where(z > 0, z, LEAK * z)


def lrelu_grad(g, z):
    return np.where(z > 0, g, LEAK * g)


def pool2(x):
    N, D, H, W, C = x.shape
    return x.reshape(N, D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4, 6))


def pool2_adjoint(g):
    """Adjoint of pool2: each of the 8 children receives g / 8."""
    return np.repeat(np.repeat(np.repeat(g, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up2_adjoint(g):
    """Adjoint of up2: sum over the 8 children."""
    N, D, H, W, C = g.shape
    return g.reshape(N, D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4, 6))


def adam(w, m, v, g, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Algorithm 1 of Kingma & Ba); returns (w, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


# -------------------------------------------------------------------- network ----
@dataclass
class ConvSpec:
    ci: int
    co: int
    level: int
    w_off: int
    b_off: int


def layout(levels: int, base_ch: int) -> List[ConvSpec]:
    """Convolutions in execution order (encoder 0..L-1, decoder L-2..0, output) with
    their offsets in the flat parameter vector (W [27, ci, co] then bias [co])."""
    ch = [base_ch << l for l in range(levels)]
    spec = []
    for l in range(levels):
        spec.append((base_ch if l == 0 else ch[l - 1], ch[l], l))
        spec.append((ch[l], ch[l], l))
    for l in range(levels - 2, -1, -1):
        spec.append((ch[l + 1] + ch[l], ch[l], l))
        spec.append((ch[l], ch[l], l))
    spec.append((base_ch, base_ch, 0))
    out, off = [], 0
    for ci, co, lv in spec:
        w_off = off
        off += 27 * ci * co
        out.append(ConvSpec(ci, co, lv, w_off, off))
        off += co
    return out


def n_params(levels: int, base_ch: int) -> int:
    s = layout(levels, base_ch)[-1]
    return s.b_off + s.co


def unpack(params: np.ndarray, levels: int, base_ch: int):
    return [(params[s.w_off:s.b_off].reshape(27, s.ci, s.co).astype(np.float64),
             params[s.b_off:s.b_off + s.co].astype(np.float64)) for s in layout(levels, base_ch)]


def coord_channel(n: int) -> np.ndarray:
    """Position of the voxels along an axis of n: (2 i + 1 - n) / P, P the smallest power of
    two >= n (so |c| < 1, symmetric about the centre)."""
    P = 1
    while P < n:
        P *= 2
    return (2.0 * np.arange(n) + 1.0 - n) / P


def to_channels(y: np.ndarray, dims, base_ch: int, coords: bool = False) -> Tuple[np.ndarray, np.ndarray]:
    """DAS output complex [V, N] -> (x [N, nz, ny, nx, base_ch] with x = y / rms in
    channels 0, 1 and, with ``coords``, the voxel's x, y, z position in channels 2, 3, 4;
    rms [N])."""
    nz, ny, nx = dims
    y = np.asarray(y, dtype=np.complex128)
    V, N = y.shape
    ms = (np.abs(y) ** 2).mean(axis=0)
    rms = np.where(ms > 0, np.sqrt(ms), 1.0)
    x = np.zeros((N, nz, ny, nx, base_ch))
    yn = (y / rms).T.reshape(N, nz, ny, nx)
    x[..., 0] = yn.real
    x[..., 1] = yn.imag
    if coords:
        x[..., 2] = coord_channel(nx)[None, None, None, :]
        x[..., 3] = coord_channel(ny)[None, None, :, None]
        x[..., 4] = coord_channel(nz)[None, :, None, None]
    return x, rms


def forward(params, y_in, dims, levels: int, base_ch: int, gain: float, store=None, coords: bool = False) -> Dict:
    """Forward pass; returns every pre-activation (z_*), activation and the prediction
    (complex [V, N])."""
    q = store if store is not None else (lambda a: a)
    P = [(q(W), b) for W, b in unpack(params, levels, base_ch)]
    L = levels
    enc = lambda l, k: 2 * l + k
    dec = lambda l, k: 2 * L + 2 * (L - 2 - l) + k
    x, rms = to_channels(y_in, dims, base_ch, coords)
    A: Dict = {"x": x, "rms": rms, "P": P}
    inp = q(x)
    for l in range(L):
        if l > 0:
            inp = q(pool2(A[f"e{l - 1}"]))
        A[f"in{l}"] = inp
        W, b = P[enc(l, 0)]
        A[f"za{l}"] = conv3d(inp, W, b)
        A[f"a{l}"] = q(lrelu(A[f"za{l}"]))
        W, b = P[enc(l, 1)]
        A[f"ze{l}"] = conv3d(A[f"a{l}"], W, b)
        A[f"e{l}"] = q(lrelu(A[f"ze{l}"]))
    for l in range(L - 2, -1, -1):
        src = A[f"e{L - 1}"] if l == L - 2 else A[f"d{l + 1}"]
        A[f"cat{l}"] = np.concatenate([up2(src), A[f"e{l}"]], axis=-1)
        W, b = P[dec(l, 0)]
        A[f"zb{l}"] = conv3d(A[f"cat{l}"], W, b)
        A[f"b{l}"] = q(lrelu(A[f"zb{l}"]))
        W, b = P[dec(l, 1)]
        A[f"zd{l}"] = conv3d(A[f"b{l}"], W, b)
        A[f"d{l}"] = q(lrelu(A[f"zd{l}"]))
    top = A["d0"] if L > 1 else A["e0"]
    W, b = P[4 * L - 2]
    A["o"] = conv3d(top, W, b)
    res = gain * x[..., :2] + A["o"][..., :2]                       # [N, nz, ny, nx, 2]
    pred = (res[..., 0] + 1j * res[..., 1]).reshape(len(rms), -1) * rms[:, None]
    A["pred"] = pred.T                                               # [V, N]
    return A


def loss_and_grads(params, y_in, target, dims, levels: int, base_ch: int, gain: float, store=None,
                   coords: bool = False):
    """(loss, flat gradient, activations) of the loss defined in the module docstring."""
    q = store if store is not None else (lambda a: a)
    L = levels
    A = forward(params, y_in, dims, levels, base_ch, gain, store, coords)
    P = A["P"]
    spec = layout(levels, base_ch)
    enc = lambda l, k: 2 * l + k
    dec = lambda l, k: 2 * L + 2 * (L - 2 - l) + k
    N = len(A["rms"])
    t = (np.asarray(target, dtype=np.complex128) / A["rms"]).T.reshape(A["x"].shape[:4])
    e = np.stack([A["o"][..., 0] + gain * A["x"][..., 0] - t.real,
                  A["o"][..., 1] + gain * A["x"][..., 1] - t.imag], axis=-1)
    count = e.size
    loss = float((e ** 2).sum() / count)
    go = np.zeros_like(A["o"])
    go[..., :2] = q(2.0 * e / count)
    G = np.zeros(n_params(levels, base_ch))

    def conv_back(idx, x_in, gz, need_input=True):
        W, _ = P[idx]
        s = spec[idx]
        G[s.w_off:s.b_off] += conv3d_grad_weight(x_in, gz).ravel()
        G[s.b_off:s.b_off + s.co] += gz.reshape(-1, s.co).sum(axis=0)
        return q(conv3d_grad_input(gz, W)) if need_input else None

    top = A["d0"] if L > 1 else A["e0"]
    g_top = conv_back(4 * L - 2, top, go)
    gd = {}
    ge = {}
    if L > 1:
        gd[0] = g_top
    else:
        ge[0] = g_top
    for l in range(0, L - 1):
        c_up = spec[dec(l, 0)].ci - A[f"e{l}"].shape[-1]
        gz = q(lrelu_grad(gd[l], A[f"zd{l}"]))
        gb = conv_back(dec(l, 1), A[f"b{l}"], gz)
        gz = q(lrelu_grad(gb, A[f"zb{l}"]))
        gcat = conv_back(dec(l, 0), A[f"cat{l}"], gz)
        g_src = q(up2_adjoint(gcat[..., :c_up]))
        if l == L - 2:
            ge[L - 1] = g_src
        else:
            gd[l + 1] = g_src
        ge[l] = gcat[..., c_up:].copy()
    for l in range(L - 1, -1, -1):
        gz = q(lrelu_grad(ge[l], A[f"ze{l}"]))
        ga = conv_back(enc(l, 1), A[f"a{l}"], gz)
        gz = q(lrelu_grad(ga, A[f"za{l}"]))
        gin = conv_back(enc(l, 0), A[f"in{l}"], gz, need_input=l > 0)
        if l > 0:
            ge[l - 1] = q(ge[l - 1] + pool2_adjoint(gin))
    return loss, G, A


def he_like(levels: int, base_ch: int, rng: np.random.Generator, scale: float = 1.0, coords: bool = False) -> np.ndarray:
    """Random parameters (normal, std sqrt(2 / (27 ci)) * scale, biases included) for
    tests; padded input channels are kept at zero like the library's initialisation."""
    p = np.zeros(n_params(levels, base_ch))
    for i, s in enumerate(layout(levels, base_ch)):
        w = rng.standard_normal((27, s.ci, s.co)) * np.sqrt(2.0 / (27 * s.ci)) * scale
        if i == 0:
            w[:, 5 if coords else 2:, :] = 0.0
        p[s.w_off:s.b_off] = w.ravel()
        p[s.b_off:s.b_off + s.co] = 0.1 * scale * rng.standard_normal(s.co)
    return p
