"""Host logic of the learned-compounding pipeline (CPU): transmit sets, scene weights,
mirroring, the least-squares gain and the error measure."""
import math

import numpy as np
import pytest
import torch

from paper_2604_06257_gb300 import learned as Lc


def test_transmit_sets():
    assert len(Lc.MANY_DEG) == 21 and len(set(Lc.MANY_DEG)) == 21
    assert len(Lc.FEW_DEG) == 3
    assert [Lc.MANY_DEG[i] for i in Lc.FEW_IN_MANY] == list(Lc.FEW_DEG)
    for s in (Lc.FEW_DEG, Lc.MANY_DEG):     # mirror symmetry used by the augmentation
        assert {(-a, e) for a, e in s} == set(s) and {(a, -e) for a, e in s} == set(s)
    acq = Lc.acquisition(32, 4, "few", 512)
    assert acq.n_tx == 3 and acq.n_elem == 1024 and acq.grid_dims == (32, 32, 32)
    # the grid is centred on the array in x and y, so mirrored volumes stay on the grid
    assert acq.grid_origin[0] == pytest.approx(-(31) * 0.5e-4) and acq.grid_origin[1] == acq.grid_origin[0]


def test_scene_weights():
    W = Lc.scene_weights(np.random.default_rng(0), 40, 200, k=(3, 7))
    nnz = (W != 0).sum(0)
    assert nnz.min() >= 3 and nnz.max() <= 7
    a = np.abs(W[W != 0])
    assert a.min() >= 0.3 - 1e-6 and a.max() <= 3.0 + 1e-6


def test_flip_mirrors_the_grid_axes():
    n, B = 4, 2
    v = torch.arange(n ** 3 * B, dtype=torch.float32).reshape(n ** 3, B).to(torch.complex64)
    fx = Lc.flip(v, n, True, False)
    ix, iy, iz = 1, 2, 3
    src = ix + n * (iy + n * iz)
    dst = (n - 1 - ix) + n * (iy + n * iz)
    assert torch.equal(fx[dst], v[src])
    fy = Lc.flip(v, n, False, True)
    assert torch.equal(fy[ix + n * ((n - 1 - iy) + n * iz)], v[src])
    assert torch.equal(Lc.flip(Lc.flip(v, n, True, True), n, True, True), v)


def test_gain_and_error_measure():
    g = torch.Generator().manual_seed(0)
    few = torch.randn(50, 6, dtype=torch.complex64, generator=g)
    noise = torch.randn(50, 6, dtype=torch.complex64, generator=g)
    bank = Lc.Bank(few, 2.5 * few, [0] * 6, 4)
    assert Lc.ls_gain(bank) == pytest.approx(2.5, rel=1e-6)
    # least squares with noise orthogonal-in-expectation: still close to 2.5
    bank = Lc.Bank(few, 2.5 * few + 0.1 * noise, [0] * 6, 4)
    assert Lc.ls_gain(bank) == pytest.approx(2.5, abs=0.05)
    ref = torch.ones(10, 2, dtype=torch.complex64)
    assert Lc.nrmse_db(ref * 1.1, ref) == pytest.approx(20 * math.log10(0.1), abs=1e-4)
    x, t = Lc.compose(Lc.Bank(few, 2 * few, [], 4), torch.eye(6, 2, dtype=torch.complex64))
    assert torch.equal(x, few[:, :2]) and torch.equal(t, 2 * few[:, :2])


def test_wiener_bound_closed_forms():
    """The error floor of the bound study, E(lam) = sum_k [S_MM - |S_MF|^2 / (S_FF + lam max S_FF)]
    / sum_k S_MM, on cases with a closed form: identical images -> E = lam / (1 + lam) per
    frequency; uncorrelated images -> 0 dB; one frequency seen at two sub-voxel positions whose
    few/many phases differ by delta -> |S_MF|^2 = cos^2(delta / 2), E = sin^2(delta / 2) as
    lam -> 0; and the frequencies weigh in by their S_MM."""
    from paper_2604_06257_gb300 import learned_bound as B
    rng = np.random.default_rng(0)
    h = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    p = np.abs(h) ** 2
    same = B.floor_db(p, p, p, lams=(1e-2, 1e-4))
    s = np.sum(p * (1e-2 * p.max()) / (p + 1e-2 * p.max())) / p.sum()
    assert same["0.01"] == pytest.approx(10 * math.log10(s), abs=1e-9)
    assert same["0.0001"] < same["0.01"] - 15
    assert B.floor_db(p, p, np.zeros(50), lams=(1e-3,))["0.001"] == pytest.approx(0.0, abs=1e-12)
    for delta in (0.3, 1.0, 2.5):
        F = np.array([1.0, np.exp(1j * 0.7)])             # the FEW image at two positions
        M = np.array([1.0, np.exp(1j * (0.7 + delta))])   # the MANY image, phase moved by delta
        sff, smm, smf = np.mean(np.abs(F) ** 2), np.mean(np.abs(M) ** 2), np.mean(M * F.conj())
        e = B.floor_db(np.array([sff]), np.array([smm]), np.array([smf]), lams=(1e-12,))["1e-12"]
        assert e == pytest.approx(10 * math.log10(math.sin(delta / 2) ** 2), abs=1e-6)
    # two frequencies, one perfectly predictable (weight 3), one not (weight 1): E = 1/4
    e = B.floor_db(np.array([1.0, 1.0]), np.array([3.0, 1.0]), np.array([math.sqrt(3.0), 0.0]),
                   lams=(1e-12,))["1e-12"]
    assert e == pytest.approx(10 * math.log10(0.25), abs=1e-6)
