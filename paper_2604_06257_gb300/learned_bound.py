"""How close can any estimator get to the many-angle volume from a few-angle one?

For speckle -- scatterers at uniform random positions with independent N(0, 1)
amplitudes -- the few-angle (FEW) and many-angle (MANY) DAS volumes are two linear images
of the same Gaussian scatterer field, hence jointly Gaussian.  The estimator of MANY from
FEW with the least mean-squared error is then linear, and where the point-spread function
varies slowly with position it is a Wiener filter in the spatial-frequency domain.  With
H_F(k), H_M(k) the spectra of the FEW and MANY point-spread functions, a white scatterer
field and a noise-to-signal ratio lam per frequency, its relative error is

    E(lam) = sum_k |H_M(k)|^2 lam / (|H_F(k)|^2 + lam)  /  sum_k |H_M(k)|^2 ,

and as lam -> 0 it tends to the share of MANY's energy at frequencies FEW does not see.
No network trained on such scenes can beat E on them; E therefore bounds the learned
compounding error on speckle (point targets, which are not Gaussian, can do better).

The study beamforms one point scatterer per depth with every transmit of the MANY set
and of candidate FEW sets separately (mach_das_run_per_tx), on the grid spacing the
network sees (0.1 mm), and evaluates E for several 3-angle sets:

    python -m paper_2604_06257_gb300.learned_bound [--depths 8 11 15] [--out report.json]
"""
from __future__ import annotations

import argparse
import json
import math
from typing import Dict, List, Sequence, Tuple

import numpy as np

from .learned import FEW_DEG, MANY_DEG

# candidate 3-angle sets, (azimuth, elevation) in degrees
CANDIDATES: Dict[str, Tuple[Tuple[float, float], ...]] = {
    "az3 (-10,0) (0,0) (10,0)": FEW_DEG,
    "el3 (0,-10) (0,0) (0,10)": ((0.0, -10.0), (0.0, 0.0), (0.0, 10.0)),
    "corner (-10,0) (0,0) (0,10)": ((-10.0, 0.0), (0.0, 0.0), (0.0, 10.0)),
    "az2+el (-10,0) (10,0) (0,10)": ((-10.0, 0.0), (10.0, 0.0), (0.0, 10.0)),
    "triangle r=10 (10,0) (-5,8.7) (-5,-8.7)": ((10.0, 0.0), (-5.0, 8.660254), (-5.0, -8.660254)),
    "triangle r=7 (7,0) (-3.5,6.1) (-3.5,-6.1)": ((7.0, 0.0), (-3.5, 6.062178), (-3.5, -6.062178)),
    "diagonal (-7.1,-7.1) (0,0) (7.1,7.1)": ((-7.071068, -7.071068), (0.0, 0.0), (7.071068, 7.071068)),
}
LAMBDAS = (1e-2, 1e-3, 1e-4, 1e-6)


def point_spectra(z_mm: float, angles_deg: Sequence[Tuple[float, float]], n: int = 64):
    """|FFT|-domain point-spread spectra: complex128 [T, n, n, n] numpy, one per transmit,
    of a unit point at (0, 0, z) beamformed on an n^3 grid (0.1 mm) centred on it."""
    import torch

    import synth
    from synth.iq import simulate_frames
    from synth.phantoms import Phantom

    from . import Plan, mach_das_run_per_tx, plan_kwargs

    tx = np.deg2rad(np.asarray(angles_deg, dtype=np.float64))
    h = (n - 1) / 2 * 1e-4
    acq = synth.acquisition.volume3d(n=n, n_frames=1, n_samples=1536, tx_angles=tx).replace(
        grid_origin=(-h, -h, z_mm * 1e-3 - h), name=f"psf_z{z_mm}")
    iq = simulate_frames(acq, [Phantom(np.array([[0.0, 0.0, z_mm * 1e-3]]), np.array([1.0]))], "cuda")
    T = len(tx)
    with Plan(**plan_kwargs(acq)) as p:
        y = torch.empty((acq.n_vox, T, 1), dtype=torch.complex64, device="cuda")
        mach_das_run_per_tx(p.handle, iq, y)
    vol = y[:, :, 0].T.reshape(T, n, n, n).to(torch.complex128)   # [t, z, y, x]
    return torch.fft.fftn(vol, dim=(1, 2, 3)).cpu().numpy()


def floor_db(HF: np.ndarray, HM: np.ndarray, lams=LAMBDAS) -> Dict[str, float]:
    """E(lam) in dB for lam relative to max |H_F|^2."""
    pf, pm = np.abs(HF) ** 2, np.abs(HM) ** 2
    out = {}
    for lam in lams:
        L = lam * pf.max()
        out[f"{lam:g}"] = float(10 * math.log10(np.sum(pm * L / (pf + L)) / np.sum(pm)))
    return out


def study(depths=(8.0, 11.0, 15.0), n: int = 64) -> dict:
    extra: List[Tuple[float, float]] = []
    for s in CANDIDATES.values():
        for a in s:
            if a not in MANY_DEG and a not in extra:
                extra.append(a)
    angles = list(MANY_DEG) + extra
    rep = {"many": [list(a) for a in MANY_DEG], "grid": f"{n}^3 at 0.1 mm centred on the point",
           "lambda": "noise-to-signal ratio per frequency, relative to max |H_F|^2", "depths_mm": list(depths),
           "sets": {}}
    spectra = {z: point_spectra(z, angles, n) for z in depths}
    for name, s in CANDIDATES.items():
        idx = [angles.index(a) for a in s]
        per = {}
        for z, H in spectra.items():
            HM = H[: len(MANY_DEG)].sum(0)
            HF = H[idx].sum(0)
            per[f"{z:g} mm"] = floor_db(HF, HM)
        rep["sets"][name] = per
    return rep


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--depths", type=float, nargs="+", default=[8.0, 11.0, 15.0])
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    from . import build
    build.build()
    rep = study(tuple(a.depths), a.n)
    for name, per in rep["sets"].items():
        print(name, json.dumps(per))
    if a.out:
        json.dump(rep, open(a.out, "w"), indent=1)


if __name__ == "__main__":
    main()
