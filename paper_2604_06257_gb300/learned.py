"""Learned compounding: turn a few-angle compounded DAS volume into the many-angle one.

Pipeline (every beamforming step runs in the library's DAS kernels, every network step in
its U-Net kernels):

* acquisitions: the 3D matrix-array set-up of the volumetric workload (32 x 32 elements,
  pitch 0.3 mm, fc 7.8 MHz, fs 31.2 MHz, F# 1.0 Gaussian window) with two transmit sets,
  FEW = 3 plane waves tilted -10, 0, +10 degrees in azimuth, and MANY = 21 plane waves,
  an azimuth/elevation cross (azimuth -10..10 degrees in 2-degree steps at elevation 0,
  elevation -10..10 degrees in 2-degree steps at azimuth 0, broadside counted once).
  FEW is a subset of MANY, so one simulated IQ block serves both;
* scenes: complex-weighted sums of seeded building blocks (speckle patches, point
  clusters, vessels).  DAS is linear in the scatterer amplitudes, so the DAS volume of a
  scene is the same weighted sum of its blocks' volumes: a bank of blocks is simulated
  and beamformed once, and every training scene is composed from it;
* training: mean squared error between the network's prediction from the FEW volume and
  the MANY volume (both divided by the FEW volume's RMS), Adam, batch 8;
* evaluation: normalised RMS error (dB) against the MANY volume on scenes composed of
  blocks never seen in training, for the network and for the plain FEW volume scaled by
  the least-squares gain (the method without the network).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time
from dataclasses import dataclass
from typing import Dict, List, Optional, Sequence

import numpy as np

FEW_DEG = ((-10.0, 0.0), (0.0, 0.0), (10.0, 0.0))
MANY_DEG = tuple((float(a), 0.0) for a in range(-10, 11, 2)) + tuple(
    (0.0, float(e)) for e in (-10, -8, -6, -4, -2, 2, 4, 6, 8, 10))
FEW_IN_MANY = tuple(MANY_DEG.index(p) for p in FEW_DEG)
WEIGHTS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights")
TEST_SEED0 = 1 << 40   # block seeds of held-out scenes start here; training blocks below


def angles(pairs) -> np.ndarray:
    return np.deg2rad(np.asarray(pairs, dtype=np.float64))


def acquisition(n: int = 128, frames: int = 8, which: str = "many", n_samples: int = 1536):
    """The matrix-array acquisition with the MANY (or FEW) transmit set and `frames`
    independent scenes on the frame axis."""
    import synth
    tx = angles(MANY_DEG if which == "many" else FEW_DEG)
    a = synth.acquisition.volume3d(n=n, n_frames=frames, n_samples=n_samples, tx_angles=tx)
    return a.replace(name=f"compounding3d_{n}^3_{which}{len(tx)}x{frames}")


def samples_for(n: int) -> int:
    """IQ samples that cover the round trip to the deepest voxel of an n^3 grid at 0.1 mm
    from 5 mm depth, with margin (1536 for the 128^3 grid)."""
    return 1536 if n >= 96 else 512


@dataclass
class Bank:
    """Beamformed blocks: few / many complex64 [V, M] CUDA tensors (block m in column m)."""
    few: "object"
    many: "object"
    seeds: List[int]
    n: int


def beamform_blocks(seeds: Sequence[int], n: int = 128, chunk: int = 32, device: str = "cuda",
                    n_samples: Optional[int] = None) -> Bank:
    """Simulate (noise-free) and beamform the blocks with both transmit sets."""
    import torch

    import synth
    from synth import phantoms
    from synth.iq import simulate_frames

    from . import Plan, plan_kwargs
    S = n_samples or samples_for(n)
    acq = acquisition(n, chunk, "many", S)
    few_acq = acquisition(n, chunk, "few", S)
    M, V = len(seeds), n ** 3
    few = torch.empty((V, M), dtype=torch.complex64, device=device)
    many = torch.empty((V, M), dtype=torch.complex64, device=device)
    idx = torch.tensor(FEW_IN_MANY, device=device)
    empty = phantoms.Phantom(np.zeros((0, 3)), np.zeros(0))
    with Plan(**plan_kwargs(acq)) as pm, Plan(**plan_kwargs(few_acq)) as pf:
        for m0 in range(0, M, chunk):
            blk = [phantoms.compounding_base(acq, int(s)) for s in seeds[m0:m0 + chunk]]
            k = len(blk)
            iq = simulate_frames(acq, blk + [empty] * (chunk - k), device)
            ym = pm.run(iq)
            yf = pf.run(iq.index_select(0, idx).contiguous())
            many[:, m0:m0 + k] = ym[:, :k]
            few[:, m0:m0 + k] = yf[:, :k]
            del iq
    return Bank(few, many, list(seeds), n)


def scene_weights(rng: np.random.Generator, M: int, count: int, k=(6, 16)) -> np.ndarray:
    """complex64 [M, count]: each scene uses k random blocks with weights a e^{j phi},
    a log-uniform in [0.3, 3], phi uniform."""
    W = np.zeros((M, count), dtype=np.complex64)
    for j in range(count):
        kk = int(rng.integers(k[0], k[1] + 1))
        sel = rng.choice(M, size=min(kk, M), replace=False)
        a = np.exp(rng.uniform(math.log(0.3), math.log(3.0), len(sel)))
        W[sel, j] = a * np.exp(1j * rng.uniform(0, 2 * math.pi, len(sel)))
    return W


def compose(bank: Bank, W):
    """(few, many) complex64 [V, B] volumes of the scenes with block weights W [M, B]
    (only the blocks some scene uses are read)."""
    used = (W != 0).any(dim=1).nonzero().flatten()
    if len(used) == 0:
        z = bank.few.new_zeros((bank.few.shape[0], W.shape[1]))
        return z, z.clone()
    Wu = W.index_select(0, used)
    return bank.few.index_select(1, used) @ Wu, bank.many.index_select(1, used) @ Wu


def flip(vol, n: int, fx: bool, fy: bool):
    """Mirror [V, B] volumes (v = ix + n (iy + n iz)) in x and/or y; both transmit sets
    are symmetric under these mirrors, so a mirrored pair is the pair of the mirrored scene."""
    if not (fx or fy):
        return vol
    B = vol.shape[1]
    v = vol.view(n, n, n, B)
    dims = [d for d, f in ((2, fx), (1, fy)) if f]
    return v.flip(dims).reshape(n ** 3, B).contiguous()


def ls_gain(bank: Bank) -> float:
    """Least-squares gain g minimising sum |g few - many|^2 over the bank."""
    num = (bank.few.conj() * bank.many).real.sum().item()
    den = (bank.few.abs() ** 2).sum().item()
    return float(num / den) if den > 0 else 1.0


def nrmse_db(pred, ref) -> float:
    return float(10.0 * math.log10(((pred - ref).abs() ** 2).sum().item() / (ref.abs() ** 2).sum().item()))


def evaluate(net, bank: Bank, W: np.ndarray, gain: float) -> Dict[str, float]:
    """Errors (dB) against the MANY volumes over the scenes W (columns), in batches of
    the network's batch size."""
    import torch
    B = net.batch
    num_net = num_base = den = 0.0
    for j in range(0, W.shape[1] - B + 1, B):
        Wj = torch.as_tensor(W[:, j:j + B]).to(bank.few.device)
        x, t = compose(bank, Wj)
        p = net.forward(x.contiguous())
        num_net += ((p - t).abs() ** 2).sum().item()
        num_base += ((gain * x - t).abs() ** 2).sum().item()
        den += (t.abs() ** 2).sum().item()
    return {"network_db": 10 * math.log10(num_net / den), "few_angle_db": 10 * math.log10(num_base / den)}


def train(n: int = 128, bank_size: int = 512, samples: int = 2000, epochs: int = 4, batch: int = 8,
          lr: float = 5e-4, seed: int = 0, test_blocks: int = 128, test_scenes: int = 64, levels: int = 4,
          base_ch: int = 16, warmup: int = 0, coords: bool = False, log=print):
    """Train a network from scratch; returns (net, report)."""
    import torch

    from .nn import UNet
    t0 = time.time()
    rng = np.random.default_rng(seed)
    bank = beamform_blocks(list(range(seed * 100003, seed * 100003 + bank_size)), n)
    test = beamform_blocks(list(range(TEST_SEED0, TEST_SEED0 + test_blocks)), n)
    torch.cuda.synchronize()
    t_data = time.time() - t0
    gain = ls_gain(bank)
    net = UNet(n, n, n, batch, levels=levels, base_ch=base_ch, seed=seed, coords=coords)
    net.set_gain(gain)
    Wtr = scene_weights(rng, bank_size, samples)
    Wte = scene_weights(np.random.default_rng(seed + 7), test_blocks, test_scenes)
    before = evaluate(net, test, Wte, gain)
    steps = epochs * (samples // batch)
    loss = torch.zeros(1, device="cuda")
    hist = []
    step = 0
    t1 = time.time()
    for ep in range(epochs):
        order = rng.permutation(samples)
        for j in range(0, samples - batch + 1, batch):
            Wj = torch.as_tensor(Wtr[:, order[j:j + batch]]).cuda()
            x, t = compose(bank, Wj)
            fx, fy = bool(rng.integers(2)), bool(rng.integers(2))
            x, t = flip(x, n, fx, fy), flip(t, n, fx, fy)
            lr_t = lr * (0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * step / steps)))
            if step < warmup:                                   # linear warm-up
                lr_t *= (step + 1) / warmup
            net.train_step(x.contiguous(), t.contiguous(), lr_t, loss)
            step += 1
            if step % 25 == 0 or step == steps:
                hist.append((step, float(loss.item())))
                log(f"step {step}/{steps} loss {hist[-1][1]:.4f}")
    torch.cuda.synchronize()
    t_train = time.time() - t1
    after = evaluate(net, test, Wte, gain)
    report = {"n": n, "levels": levels, "base_ch": base_ch, "warmup": warmup, "coords": coords,
              "bank_blocks": bank_size, "train_scenes": samples, "epochs": epochs, "batch": batch,
              "lr": lr, "steps": steps, "gain": gain, "data_s": t_data, "train_s": t_train,
              "ms_per_step": 1e3 * t_train / steps, "test_blocks": test_blocks, "test_scenes": test_scenes,
              "untrained": before, "trained": after, "loss_history": hist}
    return net, report


def save(net, gain: float, path: str) -> None:
    """Parameters as bfloat16 bit patterns (the precision the convolutions use) + gain."""
    import torch
    p = torch.as_tensor(net.params()).to(torch.bfloat16).view(torch.int16).numpy()
    d = net.desc
    np.savez(path, params_bf16=p, gain=np.float64(gain), levels=d.levels, base_ch=d.base_ch, coords=d.coords)


def load(path: str):
    """(params float32, gain, levels, base_ch, coords) from `save` (coords False for files
    written before the position channels existed)."""
    import torch
    z = np.load(path)
    p = torch.as_tensor(z["params_bf16"]).view(torch.bfloat16).to(torch.float32).numpy()
    coords = bool(int(z["coords"])) if "coords" in z.files else False
    return p, float(z["gain"]), int(z["levels"]), int(z["base_ch"]), coords


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--bank", type=int, default=1024)
    ap.add_argument("--samples", type=int, default=4000)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--levels", type=int, default=4)
    ap.add_argument("--base-ch", type=int, default=16)
    ap.add_argument("--warmup", type=int, default=0, help="steps of linear learning-rate warm-up")
    ap.add_argument("--coords", action="store_true", help="voxel position as three extra input channels")
    ap.add_argument("--out", default=os.path.join(WEIGHTS_DIR, "unet_few3_many21_128.npz"))
    ap.add_argument("--report", default=None)
    a = ap.parse_args(argv)
    net, rep = train(a.n, a.bank, a.samples, a.epochs, a.batch, a.lr, a.seed, levels=a.levels, base_ch=a.base_ch,
                     warmup=a.warmup, coords=a.coords)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    save(net, rep["gain"], a.out)
    rep["weights"] = os.path.basename(a.out)
    print(json.dumps({k: v for k, v in rep.items() if k != "loss_history"}))
    if a.report:
        json.dump(rep, open(a.report, "w"), indent=1)


if __name__ == "__main__":
    main()
