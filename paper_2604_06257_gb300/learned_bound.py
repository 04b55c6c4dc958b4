"""How close can any estimator get to the many-angle volume from a few-angle one?

For speckle -- scatterers at uniform random positions with independent N(0, 1)
amplitudes -- the few-angle (FEW) and many-angle (MANY) DAS volumes are two linear images
of the same Gaussian scatterer field, hence jointly Gaussian, and the estimator of MANY
from FEW with the least mean-squared error is linear.  On the voxel grid the speckle field
is stationary under whole-voxel shifts, so that estimator is a Wiener filter in the grid's
frequency domain built from the cross-spectral densities of the two images, averaged over
where a scatterer sits inside its voxel:

    S_FF(k) = E|F_p(k)|^2,  S_MM(k) = E|M_p(k)|^2,  S_MF(k) = E[M_p(k) F_p(k)*],

F_p, M_p the grid spectra of the FEW and MANY images of a unit point at sub-voxel position
p.  With a noise-to-signal ratio lam per frequency its relative error is

    E(lam) = sum_k [S_MM - |S_MF|^2 / (S_FF + lam)] / sum_k S_MM .

If every scatterer sat at the same sub-voxel position, |S_MF|^2 = S_MM S_FF and E would
vanish as lam -> 0.  It does not: the IQ images carry the axial carrier at twice the
centre frequency, close to the 0.1 mm grid's Nyquist limit, so the grid samples of a
point's image depend on where the point sits inside its voxel, and the FEW and MANY
images decorrelate differently.  No network trained on such scenes can beat E on them;
E therefore bounds the learned compounding error on speckle (point targets, which are
not Gaussian, can do better).

The study beamforms a point at K random sub-voxel positions (seeded) with every transmit
of the MANY set and of candidate FEW sets separately (mach_das_run_per_tx), on the grid
spacing the network sees (0.1 mm), and evaluates E for several 3-angle sets:

    python -m paper_2604_06257_gb300.learned_bound [--depths 8 11 15] [--positions 48] [--out report.json]
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


def point_spectra(pos_mm, angles_deg: Sequence[Tuple[float, float]], centre_mm, n: int = 64):
    """Grid spectra complex128 [T, n, n, n] numpy, one per transmit, of a unit point at
    pos_mm (x, y, z) beamformed on an n^3 grid (0.1 mm) centred on centre_mm."""
    import torch

    import synth
    from synth.iq import simulate_frames
    from synth.phantoms import Phantom

    from . import Plan, mach_das_run_per_tx, plan_kwargs

    tx = np.deg2rad(np.asarray(angles_deg, dtype=np.float64))
    h = (n - 1) / 2 * 1e-4
    cx, cy, cz = (c * 1e-3 for c in centre_mm)
    acq = synth.acquisition.volume3d(n=n, n_frames=1, n_samples=1536, tx_angles=tx).replace(
        grid_origin=(cx - h, cy - h, cz - h), name="psf")
    pos = np.asarray(pos_mm, dtype=np.float64)[None, :] * 1e-3
    iq = simulate_frames(acq, [Phantom(pos, np.array([1.0]))], "cuda")
    T = len(tx)
    with Plan(**plan_kwargs(acq)) as p:
        y = torch.empty((acq.n_vox, T, 1), dtype=torch.complex64, device="cuda")
        mach_das_run_per_tx(p.handle, iq, y)
    vol = y[:, :, 0].T.reshape(T, n, n, n).to(torch.complex128)   # [t, z, y, x]
    return torch.fft.fftn(vol, dim=(1, 2, 3)).cpu().numpy()


def floor_db(SFF: np.ndarray, SMM: np.ndarray, SMF: np.ndarray, lams=LAMBDAS) -> Dict[str, float]:
    """E(lam) in dB for lam relative to max S_FF."""
    out = {}
    for lam in lams:
        L = lam * SFF.max()
        out[f"{lam:g}"] = float(10 * math.log10(np.sum(SMM - np.abs(SMF) ** 2 / (SFF + L)) / np.sum(SMM)))
    return out


def study(depths=(8.0, 11.0, 15.0), n: int = 64, positions: int = 48, seed: int = 0) -> dict:
    extra: List[Tuple[float, float]] = []
    for s in CANDIDATES.values():
        for a in s:
            if a not in MANY_DEG and a not in extra:
                extra.append(a)
    angles = list(MANY_DEG) + extra
    nm = len(MANY_DEG)
    idx = {name: [angles.index(a) for a in s] for name, s in CANDIDATES.items()}
    rng = np.random.default_rng(seed)
    rep = {"many": [list(a) for a in MANY_DEG], "grid": f"{n}^3 at 0.1 mm", "positions": positions,
           "lambda": "noise-to-signal ratio per frequency, relative to max S_FF", "depths_mm": list(depths),
           "sets": {name: {} for name in CANDIDATES}, "single_position": {name: {} for name in CANDIDATES}}
    for z in depths:
        acc = {name: [0.0, 0.0, 0.0] for name in CANDIDATES}
        for k in range(positions):
            d = rng.uniform(-0.05, 0.05, 3)   # anywhere inside the voxel around (0, 0, z)
            H = point_spectra((d[0], d[1], z + d[2]), angles, (0.0, 0.0, z), n)
            HM = H[:nm].sum(0)
            for name in CANDIDATES:
                HF = H[idx[name]].sum(0)
                a = acc[name]
                a[0] = a[0] + np.abs(HF) ** 2
                a[1] = a[1] + np.abs(HM) ** 2
                a[2] = a[2] + HM * HF.conj()
                if k == 0:
                    rep["single_position"][name][f"{z:g} mm"] = floor_db(np.abs(HF) ** 2, np.abs(HM) ** 2,
                                                                         HM * HF.conj())
        for name, (sff, smm, smf) in acc.items():
            rep["sets"][name][f"{z:g} mm"] = floor_db(sff / positions, smm / positions, smf / positions)
    return rep


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--depths", type=float, nargs="+", default=[8.0, 11.0, 15.0])
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--positions", type=int, default=48)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    from . import build
    build.build()
    rep = study(tuple(a.depths), a.n, a.positions)
    for name, per in rep["sets"].items():
        print(name, json.dumps(per))
    if a.out:
        json.dump(rep, open(a.out, "w"), indent=1)


if __name__ == "__main__":
    main()
