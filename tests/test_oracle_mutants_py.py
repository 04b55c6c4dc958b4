"""The pins of the network and RF oracles must catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's source (a wrong slope, a missing
factor, a transposed operand, a swapped concatenation, a dropped bias correction, a wrong
sign or index), loads it as a separate module, swaps it in for the real one and runs the
pins; at least one pin must fail.  The real oracle is untouched."""
import inspect
import os
import sys
import types

import pytest

import test_rf_oracle as rf_pins
import test_unet_oracle as unet_pins

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _mutant(rel, old, new, tag):
    path = os.path.join(ROOT, rel)
    src = open(path).read()
    assert src.count(old) >= 1, old
    src = src.replace(old, new, 1)
    name = f"_mutant_{tag}"
    mod = types.ModuleType(name)
    sys.modules[name] = mod           # dataclasses resolve annotations through sys.modules
    try:
        exec(compile(src, path, "exec"), mod.__dict__)
    except Exception:
        del sys.modules[name]
        raise
    return mod


def _caught(pin_module, attr, mutant, pins):
    # every pin must run without arguments: a parametrised pin would raise for want of them
    # and count every mutant as caught
    for fn in pins:
        assert not inspect.signature(fn).parameters, fn.__name__
    real = getattr(pin_module, attr)
    setattr(pin_module, attr, mutant)
    try:
        for fn in pins:
            try:
                fn()
            except Exception:
                return True
        return False
    finally:
        setattr(pin_module, attr, real)


UNET_MUTANTS = [
    ("relu instead of leaky relu", "return np.where(z > 0, z, LEAK * z)", "return np.where(z > 0, z, 0.0 * z)"),
    ("leaky relu gradient slope", "return np.where(z > 0, g, LEAK * g)", "return np.where(z > 0, g, g)"),
    ("convolution tap direction", "        y += _shifted(xp, off, x.shape) @ w[t]",
     "        y += _shifted(xp, (-off[0], -off[1], -off[2]), x.shape) @ w[t]"),
    ("data gradient with the mirrored tap", "gy @ w[t].T", "gy @ w[26 - t].T"),
    ("weight gradient tap direction", "gw[t] = _shifted(xp, off, x.shape)", "gw[t] = _shifted(xp, (-off[0], -off[1], -off[2]), x.shape)"),
    ("pooling adjoint scale", "axis=2), 2, axis=3) / 8.0", "axis=2), 2, axis=3) / 4.0"),
    ("upsampling adjoint averages", "return g.reshape(N, D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4, 6))",
     "return g.reshape(N, D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4, 6))"),
    ("skip concatenated first", 'A[f"cat{l}"] = np.concatenate([up2(src), A[f"e{l}"]], axis=-1)',
     'A[f"cat{l}"] = np.concatenate([A[f"e{l}"], up2(src)], axis=-1)'),
    ("rms of magnitudes", "ms = (np.abs(y) ** 2).mean(axis=0)", "ms = np.abs(y).mean(axis=0) ** 2 * 1.1"),
    ("adam without bias correction", "mh = m / (1 - beta1 ** step)", "mh = m"),
    ("gain on the target", 'A["o"][..., 0] + gain * A["x"][..., 0] - t.real', 'A["o"][..., 0] + A["x"][..., 0] - gain * t.real'),
    ("seven significand bits", "np.round(m * 256.0) / 256.0", "np.round(m * 128.0) / 128.0"),
    ("skip gradient slice", 'c_up = spec[dec(l, 0)].ci - A[f"e{l}"].shape[-1]', 'c_up = A[f"e{l}"].shape[-1]'),
    ("bias gradient summed over channels", "G[s.b_off:s.b_off + s.co] += gz.reshape(-1, s.co).sum(axis=0)",
     "G[s.b_off:s.b_off + s.co] += gz.reshape(-1, s.co).sum()"),
    ("pooling takes the maximum", "2, W // 2, 2, C).mean(axis=(2, 4, 6))", "2, W // 2, 2, C).max(axis=(2, 4, 6))"),
    ("bias left out of the forward pass", "    if b is not None:\n        y += b", "    if b is not None:\n        y += 0.0 * b"),
    ("second moment of |g|", "v = beta2 * v + (1 - beta2) * g * g", "v = beta2 * v + (1 - beta2) * np.abs(g)"),
    ("epsilon inside the root", "(np.sqrt(vh) + eps)", "np.sqrt(vh + eps)"),
    ("coordinates not centred", "(2.0 * np.arange(n) + 1.0 - n) / P", "(2.0 * np.arange(n) - n) / P"),
    ("rms over all volumes of a batch", "ms = (np.abs(y) ** 2).mean(axis=0)", "ms = np.full(y.shape[1], (np.abs(y) ** 2).mean())"),
    ("upsampling shifted by a voxel",
     "def up2(x):\n    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)",
     "def up2(x):\n    return np.roll(np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3), 1, axis=3)"),
]
UNET_PINS = [getattr(unet_pins, n) for n in dir(unet_pins) if n.startswith("test_")]


@pytest.mark.parametrize("what,old,new", UNET_MUTANTS, ids=[m[0] for m in UNET_MUTANTS])
def test_network_oracle_pins_catch(what, old, new):
    mod = _mutant("oracle/unet_oracle.py", old, new, what.replace(" ", "_"))
    assert _caught(unet_pins, "U", mod, UNET_PINS), what


RF_MUTANTS = [
    ("carrier sign", "np.exp(-2j * np.pi * fc * (t0 + m / fs))", "np.exp(2j * np.pi * fc * (t0 + m / fs))"),
    ("carrier drops t0", "(t0 + m / fs))[None, None, :, None]", "(m / fs))[None, None, :, None]"),
    ("filter not centred", "c = (len(h) - 1) // 2", "c = 0"),
    ("decimation ignored", "idx = n * decim + k - c", "idx = n + k - c"),
    ("taps reversed", "out[:, :, ok, :] += h[k] * b[:, :, idx[ok], :]", "out[:, :, ok, :] += h[len(h) - 1 - k] * b[:, :, idx[ok], :]"),
    ("centre rounded up", "c = (len(h) - 1) // 2", "c = len(h) // 2"),
]
RF_PINS = [getattr(rf_pins, n) for n in dir(rf_pins) if n.startswith("test_")]


@pytest.mark.parametrize("what,old,new", RF_MUTANTS, ids=[m[0] for m in RF_MUTANTS])
def test_rf_oracle_pins_catch(what, old, new):
    mod = _mutant("oracle/rf_oracle.py", old, new, what.replace(" ", "_"))
    assert _caught(rf_pins, "rf_oracle", mod, RF_PINS), what
