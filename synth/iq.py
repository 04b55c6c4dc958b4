"""Analytic baseband IQ channel data for plane-wave acquisitions (forward model).

Physical model (the readings the beamformer is checked against):
  * a plane wave with direction u = (sin az cos el, sin el, cos az cos el) passes the
    array origin at t = 0, so it reaches point p at (u . p) / c;
  * a point scatterer of amplitude A at p re-emits a spherical wave, reaching element
    e at |p - e| / c later: round-trip time tau = (u . p + |p - e|) / c;
  * the received RF echo is A g(t - tau) cos(2 pi fc (t - tau)) with a Gaussian
    envelope g of full width at half maximum 2 / fc (a 2-cycle pulse);
  * IQ demodulation (multiply by exp(-j 2 pi fc t), low-pass) leaves
    IQ(t) = (A / 2) g(t - tau) exp(-j 2 pi fc tau), sampled at t_n = t0 + n / fs;
  * no spreading loss and no element directivity.

The envelope is truncated to the 2K taps around tau (|n - s_tau| < K, K = ceil(4 sigma)).
Synthesis runs in torch on any device; its precision does not matter to the parity
tests because the oracle and the GPU library are fed the same stored array.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np
import torch

from .acquisition import Acquisition, pulse_sigma_samples
from .phantoms import Phantom


def plane_wave_directions(acq: Acquisition) -> np.ndarray:
    az, el = acq.tx_angles[:, 0], acq.tx_angles[:, 1]
    return np.stack([np.sin(az) * np.cos(el), np.sin(el), np.cos(az) * np.cos(el)], axis=1)


def envelope_taps(acq: Acquisition) -> int:
    return int(math.ceil(4.0 * pulse_sigma_samples(acq)))


def add_echoes(buf: torch.Tensor, acq: Acquisition, pos: np.ndarray, amp: np.ndarray,
               chunk_elems: int = 1 << 24) -> None:
    """Add the echoes of scatterers (pos [J,3], real amp [J]) into ``buf``
    (complex [T, C, S], any device), in place."""
    if len(pos) == 0:
        return
    dev = buf.device
    fdt = torch.float64 if buf.dtype == torch.complex128 else torch.float32
    T, C, S = buf.shape
    u = torch.as_tensor(plane_wave_directions(acq), dtype=fdt, device=dev)       # [T,3]
    el = torch.as_tensor(acq.elem_pos.astype(np.float64), dtype=fdt, device=dev)  # [C,3]
    K = envelope_taps(acq)
    sig = pulse_sigma_samples(acq)
    offs = torch.arange(-K + 1, K + 1, device=dev, dtype=torch.int64)           # [2K]
    flat = torch.view_as_real(buf).reshape(-1, 2)
    per = max(1, chunk_elems // (T * C * 2 * K))
    base_tc = (torch.arange(T, device=dev)[:, None] * C + torch.arange(C, device=dev)[None, :]) * S
    for j0 in range(0, len(pos), per):
        p = torch.as_tensor(pos[j0:j0 + per], dtype=fdt, device=dev)            # [J,3]
        a = torch.as_tensor(amp[j0:j0 + per], dtype=fdt, device=dev)            # [J]
        tau_tx = (u @ p.T) / acq.c                                               # [T,J]
        tau_rx = torch.linalg.norm(p[None, :, :] - el[:, None, :], dim=-1) / acq.c  # [C,J]
        tau = tau_tx[:, None, :] + tau_rx[None, :, :]                            # [T,C,J]
        s = (tau - acq.t0) * acq.fs
        n = torch.floor(s).to(torch.int64)[..., None] + offs                     # [T,C,J,2K]
        g = torch.exp(-((n.to(fdt) - s[..., None]) ** 2) / (2.0 * sig * sig))
        ph = -2.0 * math.pi * acq.fc * tau
        mag = 0.5 * a[None, None, :, None] * g
        vre = mag * torch.cos(ph)[..., None]
        vim = mag * torch.sin(ph)[..., None]
        ok = (n >= 0) & (n < S)
        idx = (base_tc[:, :, None, None] + n)[ok]
        flat.index_add_(0, idx, torch.stack([vre[ok], vim[ok]], dim=-1))


def simulate(acq: Acquisition, phantom: Phantom, seed: int = 0, snr_db: Optional[float] = None,
             device="cpu", accum=torch.complex128, static_frames: bool = False) -> torch.Tensor:
    """IQ tensor complex64 [T, C, S, F] (frames contiguous) for ``phantom``.

    ``snr_db``: if given, complex Gaussian noise of power 10^(-snr/10) * mean |IQ|^2
    (noise-free data, frame 0) is added independently to every frame, from a torch
    generator seeded with ``seed``.  ``static_frames``: the moving part is ignored and
    every frame is the static echo plus its own noise.
    """
    T, C, S, F = acq.iq_shape
    dev = torch.device(device)
    stat = torch.zeros((T, C, S), dtype=accum, device=dev)
    add_echoes(stat, acq, phantom.static_pos, phantom.static_amp)
    out = torch.empty((T, C, S, F), dtype=torch.complex64, device=dev)
    ref_power = None
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed) * 1000003 + 17)
    for f in range(F):
        if phantom.moving is not None and not static_frames:
            fr = stat.clone()
            mp, ma = phantom.moving(f)
            add_echoes(fr, acq, mp, ma)
        else:
            fr = stat
        if snr_db is not None:
            if ref_power is None:
                ref_power = float((fr.abs() ** 2).mean())
            sd = math.sqrt(ref_power * 10.0 ** (-snr_db / 10.0) / 2.0)
            noise = torch.randn((T, C, S, 2), generator=gen, device=dev, dtype=torch.float32) * sd
            out[..., f] = fr.to(torch.complex64) + torch.view_as_complex(noise)
        else:
            out[..., f] = fr.to(torch.complex64)
    return out


def to_f16x2(iq: torch.Tensor) -> torch.Tensor:
    """complex64 [T,C,S,F] -> float16 [T,C,S,F,2] (re, im interleaved), round to nearest."""
    return torch.view_as_real(iq).to(torch.float16).contiguous()


def from_f16x2(iq16: torch.Tensor) -> torch.Tensor:
    """float16 [...,2] -> complex64 (exact widening)."""
    return torch.view_as_complex(iq16.to(torch.float32).contiguous())


def to_bf16x2(iq: torch.Tensor) -> torch.Tensor:
    """complex64 [T,C,S,F] -> bfloat16 [T,C,S,F,2] (re, im interleaved), round to nearest even."""
    return torch.view_as_real(iq).to(torch.bfloat16).contiguous()


def to_c64split(iq: torch.Tensor) -> torch.Tensor:
    """complex64 [T,C,S,F] -> float32 [T,C,S,2,F]: per sample row the F real parts, then
    the F imaginary parts (exact)."""
    return torch.view_as_real(iq).permute(0, 1, 2, 4, 3).contiguous()


def to_storage(iq: torch.Tensor, dtype: str) -> torch.Tensor:
    return {"c64": lambda x: x.contiguous(), "f16x2": to_f16x2, "bf16x2": to_bf16x2,
            "c64split": to_c64split}[dtype](iq)


def from_storage(x: torch.Tensor) -> torch.Tensor:
    """Widen stored IQ (complex64, float16 / bfloat16 pairs, or split float32 rows
    [T,C,S,2,F]) to complex64 [T,C,S,F], exactly."""
    if x.dtype == torch.complex64:
        return x
    if x.dtype == torch.float32 and x.dim() == 5 and x.shape[3] == 2:
        return torch.view_as_complex(x.permute(0, 1, 2, 4, 3).contiguous())
    return torch.view_as_complex(x.to(torch.float32).contiguous())


def simulate_frames(acq: Acquisition, phantoms, device="cpu", chunk_elems: int = 1 << 26) -> torch.Tensor:
    """IQ complex64 [T, C, S, F] whose frame f holds the noise-free echoes of
    ``phantoms[f]`` (F = len(phantoms)): independent scenes carried on the frame axis."""
    T, C, S, _ = acq.iq_shape
    dev = torch.device(device)
    out = torch.empty((T, C, S, len(phantoms)), dtype=torch.complex64, device=dev)
    buf = torch.zeros((T, C, S), dtype=torch.complex64, device=dev)
    for f, ph in enumerate(phantoms):
        buf.zero_()
        add_echoes(buf, acq, ph.static_pos, ph.static_amp, chunk_elems=chunk_elems)
        out[..., f] = buf
    return out


def lowpass_taps(n_taps: int, cutoff: float, fs: float) -> np.ndarray:
    """Hann-windowed sinc low-pass (cutoff in Hz at sampling rate fs), unit DC gain."""
    k = np.arange(n_taps) - (n_taps - 1) / 2.0
    h = np.sinc(2.0 * cutoff / fs * k) * np.hanning(n_taps + 2)[1:-1]
    return (h / h.sum()).astype(np.float32)


def simulate_rf(acq: Acquisition, phantom: Phantom, decim: int, device="cpu") -> torch.Tensor:
    """Real RF [T, C, S_rf, F] float32 of the static scatterers of ``phantom``, sampled at
    fs_rf = decim * acq.fs from acq.t0 with S_rf = decim * (S - 1) + 1 samples, so that
    demodulating and decimating by ``decim`` lands on the acquisition's IQ sample times.
    Echo of a scatterer of amplitude A with round-trip time tau:
    A g(t - tau) cos(2 pi fc (t - tau)), g the Gaussian envelope of the IQ model; every frame
    holds the same echoes."""
    T, C, S, F = acq.iq_shape
    dev = torch.device(device)
    fs_rf = decim * acq.fs
    S_rf = decim * (S - 1) + 1
    u = torch.as_tensor(plane_wave_directions(acq), dtype=torch.float64, device=dev)
    el = torch.as_tensor(acq.elem_pos.astype(np.float64), dtype=torch.float64, device=dev)
    sig = pulse_sigma_samples(acq) * decim                   # envelope sigma in RF samples
    K = int(math.ceil(4.0 * sig))
    offs = torch.arange(-K + 1, K + 1, device=dev, dtype=torch.int64)
    out = torch.zeros((T, C, S_rf), dtype=torch.float64, device=dev)
    flat = out.view(-1)
    base = (torch.arange(T, device=dev)[:, None] * C + torch.arange(C, device=dev)[None, :]) * S_rf
    pos = torch.as_tensor(phantom.static_pos, dtype=torch.float64, device=dev)
    amp = torch.as_tensor(phantom.static_amp, dtype=torch.float64, device=dev)
    for j in range(len(pos)):
        tau = (u @ pos[j])[:, None] / acq.c + torch.linalg.norm(pos[j][None, :] - el, dim=1)[None, :] / acq.c  # [T, C]
        s = (tau - acq.t0) * fs_rf
        n = torch.floor(s).to(torch.int64)[..., None] + offs
        tn = acq.t0 + n.to(torch.float64) / fs_rf
        v = amp[j] * torch.exp(-((n.to(torch.float64) - s[..., None]) ** 2) / (2 * sig * sig)) * \
            torch.cos(2 * math.pi * acq.fc * (tn - tau[..., None]))
        ok = (n >= 0) & (n < S_rf)
        flat.index_add_(0, (base[..., None] + n)[ok], v[ok])
    return out.to(torch.float32)[..., None].expand(T, C, S_rf, F).contiguous()
