"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a wrong
sign or index, swapped operands) breaks at least one of them:
  * closed-form delays (broadside, steered, elevation tilt, element above voxel, t0);
  * mirror symmetry of the delay geometry;
  * hand-derivable single-element cases (constant and ramp IQ: lerp weights, phase
    sign, out-of-range rule R5 at both ends);
  * aperture windows at known points (centre, quarter, edge);
  * an analytic point scatterer from the forward model focusing to a real, known sum;
  * linearity, compounding = sum of single transmits, frame permutation, PD = |y|^2;
  * brute force against an independent numpy implementation on tiny random inputs;
  * contract-vs-exact delay error bound (float32 rounding of sample positions).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from synth.acquisition import Acquisition, linear_array, matrix_array, deg
import bruteforce_np


def one_element(z_list, S=64, F=1, apod="boxcar", f_number=1.0, t0=0.0, angles=None, x_list=None):
    """Single element at the origin, k = fs/c = 1000 samples/m (1 sample per mm),
    fc = fs/4, voxels given explicitly (float32)."""
    n = len(z_list)
    x = np.zeros(n) if x_list is None else np.asarray(x_list)
    vox = np.stack([x, np.zeros(n), np.asarray(z_list)], 1).astype(np.float32)
    ang = np.zeros((1, 2)) if angles is None else np.asarray(angles, dtype=np.float64)
    return Acquisition(name="one", ndim=2, elem_pos=np.zeros((1, 3), np.float32),
                       tx_angles=ang, fs=1.54e6, fc=0.385e6, c=1540.0, t0=t0,
                       f_number=f_number, apod=apod, n_samples=S, n_frames=F, vox_pos=vox)


def ramp_iq(acq):
    T, C, S, F = acq.iq_shape
    n = np.arange(S, dtype=np.float64)
    return np.broadcast_to(n[None, None, :, None], (T, C, S, F)).astype(np.complex64)


# ---------------------------------------------------------------- delays ----

@pytest.mark.parametrize("mode", ["exact", "contract"])
def test_broadside_tx_delay_is_depth(mode):
    acq = synth.bmode2d(nx=9, nz=7).replace(tx_angles=np.zeros((1, 2)), t0=1.3e-6)
    P = acq.voxel_positions()
    expect = (P[:, 2] / acq.c - acq.t0) * acq.fs
    got = oracle.tx_exact(acq)[0] if mode == "exact" else oracle.tx_table(acq)[0]
    tol = 1e-9 if mode == "exact" else 2e-4
    np.testing.assert_allclose(got, expect, rtol=0, atol=tol)


def test_steered_tx_delay_closed_form():
    th = deg(7.5)[0]
    acq = synth.bmode2d(nx=5, nz=5).replace(tx_angles=np.array([[th, 0.0]]))
    P = acq.voxel_positions()
    expect = (P[:, 0] * math.sin(th) + P[:, 2] * math.cos(th)) / acq.c * acq.fs
    np.testing.assert_allclose(oracle.tx_exact(acq)[0], expect, rtol=1e-13)


def test_elevation_tilt_closed_form_3d():
    el = deg(5.0)[0]
    acq = synth.volume3d(n=4, n_frames=1, n_side=4, n_samples=64).replace(
        tx_angles=np.array([[0.0, el]]))
    P = acq.voxel_positions()
    expect = (P[:, 1] * math.sin(el) + P[:, 2] * math.cos(el)) / acq.c * acq.fs
    np.testing.assert_allclose(oracle.tx_exact(acq)[0], expect, rtol=1e-13)
    # azimuth tilt of the same size must act on x, not y
    acq2 = acq.replace(tx_angles=np.array([[el, 0.0]]))
    expect2 = (P[:, 0] * math.sin(el) + P[:, 2] * math.cos(el)) / acq.c * acq.fs
    np.testing.assert_allclose(oracle.tx_exact(acq2)[0], expect2, rtol=1e-13)


def test_receive_delay_element_directly_above():
    """An element at the voxel's lateral position: s_rx = z fs / c."""
    acq = synth.bmode2d().replace(tx_angles=np.zeros((1, 2)))
    e = acq.elem_pos.astype(np.float64)
    zs = np.array([6e-3, 17e-3, 31e-3])
    vox = np.stack([e[[10, 64, 100], 0], np.zeros(3), zs], 1).astype(np.float32)
    a = acq.replace(grid_dims=None, vox_pos=vox)
    tr = oracle.terms(a, mode="exact")
    stx = oracle.tx_exact(a)[0]
    for j, c in enumerate([10, 64, 100]):
        srx = tr["s"][j, c, 0] - stx[j]
        assert abs(srx - float(vox[j, 2]) * a.fs / a.c) < 1e-9


def test_mirror_symmetry():
    """az -> -az with x -> -x leaves every delay unchanged (symmetric array)."""
    th = deg(5.0)[0]
    base = synth.bmode2d(nx=17, nz=9)
    P = base.voxel_positions()
    vox = P.astype(np.float32)
    mir = vox.copy(); mir[:, 0] *= -1
    a = base.replace(grid_dims=None, vox_pos=vox, tx_angles=np.array([[th, 0.0]]))
    b = base.replace(grid_dims=None, vox_pos=mir, tx_angles=np.array([[-th, 0.0]]))
    sa = oracle.terms(a, mode="exact")["s"]
    sb = oracle.terms(b, mode="exact")["s"][:, ::-1, :]    # element c <-> C-1-c
    np.testing.assert_allclose(sa, sb, rtol=1e-12)


def test_contract_delay_within_float_rounding_of_exact():
    acq = synth.make_acquisition("volume3d", "small")
    idx = np.arange(0, acq.n_vox, 37)
    se = oracle.terms(acq, idx, mode="exact")["s"]
    sc = oracle.terms(acq, idx, mode="contract")["s"]
    # float32 rounding of positions ~ 2^-24 * |s| per operand, a handful of operations
    assert np.max(np.abs(se - sc) / np.maximum(np.abs(se), 1.0)) < 8 * 2.0 ** -24 * 4


# ------------------------------------------------- hand-derivable cases ----

@pytest.mark.parametrize("mode", ["exact", "contract"])
def test_ramp_lerp_and_phase(mode):
    """One element at the origin, broadside wave, k = 1 sample/mm: s = 2 z [mm].
    Ramp IQ x[n] = n interpolates to exactly s, and the rotation is e^{j 2 pi s/4}."""
    zs = [10e-3, 10.3e-3, 12.125e-3, 7.77e-3]
    acq = one_element(zs)
    y, pd = oracle.das(acq, ramp_iq(acq), mode=mode)
    s = 2.0 * np.asarray(acq.vox_pos[:, 2], np.float64) * 1000.0
    expect = s * np.exp(2j * np.pi * 0.25 * s)
    np.testing.assert_allclose(y[:, 0], expect, rtol=2e-6, atol=1e-9)
    np.testing.assert_allclose(pd, np.abs(expect) ** 2, rtol=4e-6)
    assert abs(y[0, 0] - 20.0) < 1e-4   # z = 10 mm: s = 20, phase 10 pi -> real 20


def test_constant_iq_is_rotation_sum():
    """iq = 1: y = sum over valid terms of a * e^{j phi}.  Two transmits (0 and 30 deg)."""
    zs = [9.1e-3, 13.6e-3]
    acq = one_element(zs, angles=[[0.0, 0.0], [math.pi / 6, 0.0]])
    iq = np.ones(acq.iq_shape, np.complex64)
    y, _ = oracle.das(acq, iq, mode="exact")
    z = np.asarray(acq.vox_pos[:, 2], np.float64)
    expect = np.zeros(2, complex)
    for th in (0.0, math.pi / 6):
        s = (z * math.cos(th) + z) * 1000.0
        expect += np.exp(2j * np.pi * 0.25 * s)
    np.testing.assert_allclose(y[:, 0], expect, rtol=0, atol=1e-9)


def test_range_rule_both_ends():
    """R5: a term contributes iff 0 <= i0 and i0 + 1 <= S - 1, i.e. 0 <= s < S - 1.
    Geometry with fs/c = 1024 samples/m and z = m/2048 m, so s = 2 z fs/c = m exactly
    (binary fractions, no rounding in either mode)."""
    S = 22
    m = np.array([0.0, 0.5, 20.5, 21.0 - 2.0 ** -10, 21.0, 21.25, 30.0])
    zs = m / 2048.0
    for mode in ("exact", "contract"):
        acq = one_element(list(zs), S=S, apod="none").replace(fs=1540.0 * 1024, fc=1540.0 * 256)
        y, _ = oracle.das(acq, ramp_iq(acq), mode=mode)
        inside = (m >= 0) & (m < S - 1)
        assert np.all((y[:, 0] != 0)[1:] == inside[1:])
        np.testing.assert_allclose(np.abs(y[inside, 0]), m[inside], rtol=1e-6, atol=1e-12)
        # s = 0: i0 = 0, w = 0 -> x[0] = 0 for the ramp, so check with constant IQ
        yc, _ = oracle.das(acq, np.ones(acq.iq_shape, np.complex64), mode=mode)
        assert abs(abs(yc[0, 0]) - 1.0) < 1e-12
        assert np.all((yc[:, 0] != 0) == inside)
    # negative s (t0 after the echo) contributes nothing
    neg = one_element([5.0 / 2048.0], S=S).replace(fs=1540.0 * 1024, fc=1540.0 * 256,
                                                   t0=6.0 / (1540.0 * 1024))
    yn, _ = oracle.das(neg, np.ones(neg.iq_shape, np.complex64), mode="exact")
    assert np.all(yn == 0)


def test_large_t0_gives_zero_image():
    acq = synth.make_acquisition("bmode2d", "small").replace(t0=200e-6)
    iq = synth.random_iq(acq, 0)
    y, pd = oracle.das(acq, iq)
    assert np.all(y == 0) and np.all(pd == 0)


# ------------------------------------------------------------- windows ----

@pytest.mark.parametrize("mode", ["exact", "contract"])
def test_window_values(mode):
    """F# = 1: half-aperture h = z/2.  At lateral offset rho, t = rho/z.
    Hann: t=0 -> 1, t=1/4 -> 1/2, t=1/2 -> 0 (edge, included).  Gaussian at the edge
    e^{-2}.  Beyond the edge nothing contributes.  Boxcar: 1 inside."""
    z = 10e-3
    xs = [0.0, 2.5e-3, 5e-3, 5.2e-3]
    for apod, expect in [("hann", [1.0, 0.5, 0.0, None]),
                         ("gauss", [1.0, math.exp(-0.5), math.exp(-2.0), None]),
                         ("boxcar", [1.0, 1.0, 1.0, None])]:
        acq = one_element([z] * 4, x_list=xs, apod=apod, S=256)
        tr = oracle.terms(acq, mode=mode)
        for j, e in enumerate(expect):
            if e is None:
                assert not tr["valid"][j, 0, 0]
            else:
                assert tr["valid"][j, 0, 0]
                assert abs(tr["a"][j, 0, 0] - e) < 1e-6


def test_apod_none_has_no_mask():
    acq = one_element([10e-3, -1e-3], x_list=[30e-3, 0.0], apod="none", S=256)
    tr = oracle.terms(acq, mode="exact")
    assert tr["valid"][0, 0, 0] and tr["a"][0, 0, 0] == 1.0
    # a voxel behind the array is still summed when no aperture is applied
    assert tr["i0"][1, 0, 0] == -1 or tr["valid"][1, 0, 0] == (tr["s"][1, 0, 0] >= 0)


@pytest.mark.parametrize("mode", ["exact", "contract"])
def test_voxels_behind_the_array_get_no_terms(mode):
    """R6: an element contributes only to voxels in front of it (dz > 0), whatever the
    window.  t0 < 0 puts voxels behind the array plane inside the sample range, so only the
    aperture rule can drop them (on axis the squared test alone would keep them)."""
    for apod in ("boxcar", "hann", "gauss"):
        acq = one_element([-10e-3, -2e-3, -0.5e-3], x_list=[0.0, 0.5e-3, 0.0], apod=apod, S=256,
                          t0=-30e-6)
        tr = oracle.terms(acq, mode=mode)
        assert (tr["i0"] >= 0).all()                 # in range: the aperture decides
        assert not tr["valid"].any()


def test_contract_decisions_match_exact_in_3d():
    """On a 3D grid (matrix array, waves steered in azimuth and in elevation) the contract
    mode keeps the same terms as the exact mode, except within float rounding of the
    aperture edge or of the range ends, and its window values agree to float precision."""
    acq = synth.volume3d(n=12, n_frames=1, n_side=16, n_samples=512).replace(
        grid_origin=(-1.6137e-3, -1.6291e-3, 1.5173e-3), grid_step=(3e-4, 3e-4, 3e-4))
    # shallow, so the aperture cuts; the grid is off the element lattice, so few terms sit
    # exactly on an aperture edge (on the lattice, rho 2F# = dz happens exactly)
    idx = np.arange(0, acq.n_vox, 3)
    te = oracle.terms(acq, idx, mode="exact")
    tc = oracle.terms(acq, idx, mode="contract")
    p = acq.voxel_positions()[idx].astype(np.float64)
    e = acq.elem_pos.astype(np.float64)
    d = p[:, None, :] - e[None, :, :]
    rho = np.sqrt(d[..., 0] ** 2 + d[..., 1] ** 2)
    dz = d[..., 2]
    edge = np.abs(2.0 * acq.f_number * rho - dz) <= 1e-5 * np.abs(dz)      # [n, C]
    ends = np.minimum(np.abs(te["s"]), np.abs(te["s"] - (acq.n_samples - 1))) < 1e-3
    diff = te["valid"] != tc["valid"]
    assert te["valid"].sum() > 1000 and (~te["valid"]).sum() > 1000       # both kinds present
    assert not (diff & ~(edge[:, :, None] | ends)).any()
    assert diff.sum() <= 1e-3 * diff.size
    both = te["valid"] & tc["valid"]
    assert np.max(np.abs(te["a"][both] - tc["a"][both])) < 1e-5


# ------------------------------------------------- point scatterer ----

@pytest.mark.parametrize("apod", ["none", "hann"])
def test_point_scatterer_focuses_to_known_real_sum(apod):
    """Forward-model a single scatterer (synth.iq) and beamform at its position.
    Exact delays match the echo time, so y(p) = (A/2) sum_t sum_c a_c
    [(1-w) g(-w) + w g(1-w)]: real and positive; off-target voxels are weaker."""
    base = synth.bmode2d(nx=5, nz=5).replace(tx_angles=deg(-5, 0, 5)[:, None] * [1, 0],
                                             apod=apod, f_number=1.0)
    p = np.array([[1.3e-3, 0.0, 21.7e-3]], dtype=np.float32)
    off = p + np.array([[0.0, 0, 0.3e-3], [0.4e-3, 0, 0], [0.0, 0, -0.3e-3]], np.float32)
    acq = base.replace(grid_dims=None, vox_pos=np.concatenate([p, off]).astype(np.float32))
    A = 1.7
    ph = synth.phantoms.Phantom(p.astype(np.float64), np.array([A]))
    iq = synth.iqmod.simulate(acq, ph)
    y, _ = oracle.das(acq, iq, mode="exact")
    # closed form
    pp = p[0].astype(np.float64)
    E = acq.elem_pos.astype(np.float64)
    U = synth.iqmod.plane_wave_directions(acq)
    sig = synth.acquisition.pulse_sigma_samples(acq)
    g = lambda x: np.exp(-x ** 2 / (2 * sig * sig))
    total = 0.0
    for u in U:
        for e in E:
            tau = (u @ pp + np.linalg.norm(pp - e)) / acq.c
            s = tau * acq.fs
            w = s - math.floor(s)
            rho, dz = abs(pp[0] - e[0]), pp[2] - e[2]
            if apod == "none":
                a = 1.0
            else:
                if rho * 2 * acq.f_number > dz:
                    continue
                a = math.cos(math.pi * rho * acq.f_number / dz) ** 2
            total += a * (A / 2) * ((1 - w) * g(-w) + w * g(1 - w))
    assert abs(y[0, 0].imag) < 1e-5 * abs(total)
    assert abs(y[0, 0].real - total) < 1e-5 * abs(total)
    assert np.all(np.abs(y[1:, 0]) < 0.8 * abs(y[0, 0]))


# ------------------------------------------------------- invariants ----

def test_linearity():
    acq = synth.make_acquisition("doppler2d", "small").replace(n_frames=3)
    X = synth.random_iq(acq, 1).numpy()
    Y = synth.random_iq(acq, 2).numpy()
    al, be = 0.75 - 0.5j, -1.25 + 2.0j
    Z = (al * X.astype(np.complex128) + be * Y).astype(np.complex64)
    idx = np.arange(0, acq.n_vox, 11)
    yx, _ = oracle.das(acq, X, idx)
    yy, _ = oracle.das(acq, Y, idx)
    yz, _ = oracle.das(acq, Z, idx)
    ref = al * yx + be * yy
    assert np.linalg.norm(yz - ref) / np.linalg.norm(ref) < 1e-6   # complex64 rounding of Z


def test_compounding_is_sum_of_single_transmits():
    acq = synth.make_acquisition("bmode2d", "small")
    iq = synth.random_iq(acq, 3).numpy()
    y, _ = oracle.das(acq, iq)
    acc = np.zeros_like(y)
    for t in range(acq.n_tx):
        a1 = acq.replace(tx_angles=acq.tx_angles[t:t + 1])
        acc += oracle.das(a1, iq[t:t + 1])[0]
    np.testing.assert_allclose(y, acc, rtol=1e-12, atol=1e-12)


def test_frame_permutation_and_power_doppler():
    acq = synth.make_acquisition("doppler2d", "small").replace(n_frames=5)
    iq = synth.random_iq(acq, 4).numpy()
    perm = np.array([3, 0, 4, 1, 2])
    idx = np.arange(0, acq.n_vox, 7)
    y, pd = oracle.das(acq, iq, idx)
    yp, pdp = oracle.das(acq, np.ascontiguousarray(iq[..., perm]), idx)
    np.testing.assert_array_equal(yp, y[:, perm])
    np.testing.assert_allclose(pd, (np.abs(y) ** 2).sum(1), rtol=1e-12)
    np.testing.assert_allclose(pdp, pd, rtol=1e-12)
    a1 = acq.replace(n_frames=1)
    y1, pd1 = oracle.das(a1, np.ascontiguousarray(iq[..., :1]), idx)
    np.testing.assert_allclose(pd1, np.abs(y1[:, 0]) ** 2, rtol=1e-12)


# ------------------------------------------------------- brute force ----

@pytest.mark.parametrize("seed", range(6))
def test_brute_force_tiny_random(seed):
    rng = np.random.default_rng(100 + seed)
    ndim = 2 if seed % 2 == 0 else 3
    C, V, S = 2 + seed % 3, 3 + seed, 10 + 2 * (seed % 3)
    T, F = 1 + seed % 2, 1 + seed % 3
    # delays 2 z fs/c span roughly 2..14 samples: some terms fall past S - 1
    elem = np.zeros((C, 3)); elem[:, 0] = rng.uniform(-0.4e-3, 0.4e-3, C)
    vox = np.zeros((V, 3)); vox[:, 0] = rng.uniform(-0.4e-3, 0.4e-3, V)
    vox[:, 2] = rng.uniform(0.15e-3, 0.9e-3, V)
    if ndim == 3:
        elem[:, 1] = rng.uniform(-0.4e-3, 0.4e-3, C); vox[:, 1] = rng.uniform(-0.4e-3, 0.4e-3, V)
    ang = np.zeros((T, 2)); ang[:, 0] = rng.uniform(-0.2, 0.2, T)
    if ndim == 3:
        ang[:, 1] = rng.uniform(-0.2, 0.2, T)
    apod = ["none", "boxcar", "hann", "gauss"][seed % 4]
    acq = Acquisition(name="tiny", ndim=ndim, elem_pos=elem.astype(np.float32), tx_angles=ang,
                      fs=10e6, fc=2.5e6 + 1e5 * seed, c=1540.0, t0=rng.uniform(0, 0.3e-6),
                      f_number=0.7, apod=apod, n_samples=S, n_frames=F,
                      vox_pos=vox.astype(np.float32))
    iq = (rng.standard_normal(acq.iq_shape) + 1j * rng.standard_normal(acq.iq_shape)).astype(np.complex64)
    y, pd = oracle.das(acq, iq, mode="exact")
    yb, pdb = bruteforce_np.das(acq, iq)
    assert np.count_nonzero(yb) > 0
    np.testing.assert_allclose(y, yb, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(pd, pdb, rtol=1e-10, atol=1e-11)


def test_brute_force_small_workloads():
    for name in ("bmode2d", "volume3d"):
        acq = synth.make_acquisition(name, "small")
        acq = acq.replace(n_frames=2, grid_dims=(5, 4 if acq.ndim == 3 else 1, 6))
        iq = synth.random_iq(acq, 5).numpy()
        y, _ = oracle.das(acq, iq, mode="exact")
        yb, _ = bruteforce_np.das(acq, iq)
        np.testing.assert_allclose(y, yb, rtol=1e-10, atol=1e-10)


# ----------------------------------------------------- rotating disk ----

def test_rotating_disk_power_doppler_contrast():
    """Disk-only phantom: PD inside the rotating disk exceeds the empty background by
    more than 20 dB (qualitative; the paper's PD image itself is not available)."""
    acq = synth.doppler2d(nx=41, nz=61, n_frames=8).replace(
        grid_origin=(-14e-3, 0.0, 16e-3), grid_step=(0.5e-3, 0.0, 0.5e-3))
    ph = synth.phantoms.rotating_disk(acq, seed=9, per_cell=2.0, background=False)
    iq = synth.iqmod.simulate(acq, ph)
    _, pd = oracle.das(acq, iq)
    P = acq.voxel_positions()
    r = np.hypot(P[:, 0], P[:, 2] - 22.5e-3)
    inside = pd[r < 8e-3].mean()
    outside = pd[r > 12e-3].mean()
    assert 10 * np.log10(inside / outside) > 20
