"""The exact-frame staged kernels (split complex64 rows, F = 32 or F = 64 as a compile-time
constant) against the generic staged kernels they specialise and against the FP64 oracle.

Both kernels stage the same windows, evaluate the same terms with the same device
functions and give every frame the same FMA sequence in the same pair order, so their
outputs must be bitwise equal; the oracle bars are those of the other parity tests.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2604_06257_gb300 as m
from paper_2604_06257_gb300 import build as pkg_build
from metrics import nrmse_db

pytestmark = pytest.mark.gpu

# (default exact-frame variant, the generic variant it specialises), per frame count; 3D
# grids with 32 frames default to the exact kernel with 3D tiles of 112 voxels
PAIRS = {32: ("staged_c64p_x32_f8v1w7t14e", "staged_c64p_ft32_v4w7"), 64: ("staged_c64p_x64_v4", "staged_c64p_ft64_v4")}
PAIRS_3D = {32: ("staged_c64p_x32_f8v1w7_t8x7e", "staged_c64p_ft32_v4w7"), 64: PAIRS[64]}


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg_build.build()
    m.lib()


def forced(kw, name):
    m.mach_debug_force_variant(name)
    try:
        return m.Plan(**kw)
    finally:
        m.mach_debug_force_variant(None)


def same_bits(a, b):
    """Frames bitwise equal; Power Doppler bitwise equal when both kernels hold a voxel's
    frames on the same lanes (4 frames per lane), else within float32 summation order."""
    (y_x, pd_x, fpl_x), (y_g, pd_g, fpl_g) = a, b
    assert torch.equal(y_x, y_g)
    if fpl_x == fpl_g:
        assert torch.equal(pd_x, pd_g)
    else:
        assert nrmse_db(pd_x.cpu().numpy().astype(np.float64), pd_g.cpu().numpy().astype(np.float64)) < -120


def run_both(acq, iq_c64, **extra):
    """(exact, generic) outputs on the same split-row IQ; checks the variant names."""
    a = acq.replace(iq_dtype="c64split")
    kw = {**m.plan_kwargs(a), **extra}
    x = synth.iqmod.to_c64split(iq_c64.cuda())
    exact, generic = (PAIRS_3D if a.vox_pos is None and a.grid_dims[1] > 1 else PAIRS)[a.n_frames]
    with m.Plan(**kw) as pd_plan:
        assert pd_plan.info()["variant"] == exact           # the default choice
    out = []
    for name in (exact, generic):
        with forced(kw, name) as p:
            assert p.info()["variant"] == name
            pd, y = p.power_doppler(x, want_y=True)
            torch.cuda.synchronize()
            assert p.device_status() == m.MACH_OK
            out.append((y, pd, p.info()["frames_per_lane"]))
    same_bits(*out)
    return out


def check_oracle(acq, iq_c64, y, pd, idx=None, **kw):
    y_ref, pd_ref = oracle.das(acq, iq_c64.cpu(), idx, **kw)
    sel = slice(None) if idx is None else torch.from_numpy(np.asarray(idx)).cuda()
    e_y = nrmse_db(y[sel].cpu().numpy(), y_ref)
    e_p = nrmse_db(pd[sel].cpu().numpy().astype(np.float64), pd_ref)
    assert e_y <= -100.0 and e_p <= -60.0, (e_y, e_p)
    return e_y, e_p


@pytest.mark.parametrize("name", ["doppler2d", "volume3d"])
def test_exact_equals_generic_bitwise_small(name):
    acq, iq = synth.make(name, "small", device="cpu")
    (y_x, pd_x, _), _ = run_both(acq, iq)
    print(name, check_oracle(acq, iq, y_x, pd_x))


def test_exact_3d_32_frames_defaults_to_one_plane_tiles():
    """3D grid, 32 frames: the default is the exact kernel with one-plane 8 x 7 x 1 tiles
    (8 frames per lane), bitwise equal to the generic kernel and within the oracle bars."""
    acq = synth.make_acquisition("ulm3d", "small").replace(n_frames=32)
    iq = synth.random_iq(acq, 33)
    (y_x, pd_x, _), _ = run_both(acq, iq)
    print(check_oracle(acq, iq, y_x, pd_x))


ONE_PLANE = [("staged_c64p_x32_v4w7_t8x14", "staged_c64p_ft32_v4w7", [8, 14, 1], 32),
             ("staged_c64p_x32_f8v1w7_t8x7e", "staged_c64p_ft32_v4w7", [8, 7, 1], 32),
             ("staged_c64p_x64_v4_t8x8", "staged_c64p_ft64_v4", [8, 8, 1], 64),
             ("staged_c64p_x16_f4v2w7_t8x14", "staged_c64p_x16_f4v2w7", [8, 14, 1], 16),
             ("staged_c64p_x8_f4v1w7_t8x14", "staged_c64p_x8_f4v1w7", [8, 14, 1], 8)]


@pytest.mark.parametrize("name,base,tile,F", ONE_PLANE)
def test_exact_one_plane_3d_tiles(name, base, tile, F):
    """3D grids in one-plane tiles (ragged in x and y): each voxel's kept terms arrive in
    the same pair order as with any other tiling, so the frames are bitwise those of the
    same kernel on its own tiles (or of the generic kernel), and within the oracle bars."""
    acq = synth.make_acquisition("ulm3d", "small").replace(n_frames=F, iq_dtype="c64split")
    iq = synth.random_iq(acq, 35 + F)
    x = synth.iqmod.to_c64split(iq.cuda())
    kw = m.plan_kwargs(acq)
    out = []
    for v in (name, base):
        with forced(kw, v) as p:
            info = p.info()
            assert info["variant"] == v
            if v == name:
                assert info["tile"] == tile
            pd, y = p.power_doppler(x, want_y=True)
            torch.cuda.synchronize()
            assert p.device_status() == m.MACH_OK
            out.append((y, pd, info["frames_per_lane"]))
    same_bits(*out)
    print(name, check_oracle(acq, iq, out[0][0], out[0][1]))


@pytest.mark.parametrize("F,expect", [(8, "staged_c64p_x8_f4v1w7"), (16, "staged_c64p_x16_f4v2w7")])
def test_exact_3d_short_ensembles_keep_their_3d_tiles(F, expect):
    """3D grids with 8 or 16 frames keep 8 x 2 x 7 tiles (one-plane tiles measured no faster
    for these frame counts)."""
    acq = synth.make_acquisition("ulm3d", "small").replace(n_frames=F, iq_dtype="c64split")
    iq = synth.random_iq(acq, 45 + F)
    with m.Plan(**m.plan_kwargs(acq)) as p:
        info = p.info()
        assert info["variant"] == expect and info["tile"] == [8, 2, 7]
        pd, y = p.power_doppler(synth.iqmod.to_c64split(iq.cuda()), want_y=True)
        torch.cuda.synchronize()
        assert p.device_status() == m.MACH_OK
    print(F, check_oracle(acq, iq, y, pd))


def test_exact_2d_64_frames_shallow_tiles():
    """2D grid, 64 frames: the default takes 16 x 4 voxel tiles (whose windows fit the ring),
    against the oracle; per-pair slot release changes no bit."""
    acq = synth.make_acquisition("doppler2d", "small").replace(n_frames=64, iq_dtype="c64split")
    iq = synth.random_iq(acq, 64)
    x = synth.iqmod.to_c64split(iq.cuda())
    kw = m.plan_kwargs(acq)
    out = []
    with m.Plan(**kw) as p:
        info = p.info()
        assert info["variant"] == "staged_c64p_x64_v4t16" and info["tile"] == [16, 1, 4]
        out.append(p.power_doppler(x, want_y=True))
    with forced(kw, "staged_c64p_x64_v4t16e") as p:
        out.append(p.power_doppler(x, want_y=True))
        torch.cuda.synchronize()
        assert p.device_status() == m.MACH_OK
    (pd0, y0), (pd1, y1) = out
    assert torch.equal(y0, y1) and torch.equal(pd0, pd1)
    print(check_oracle(acq, iq, y0, pd0))


def test_exact_equals_generic_bitwise_doppler2d_full():
    """The benchmark workload in the benchmarked launch configuration."""
    acq, iq = synth.make("doppler2d", "full", device="cuda")
    (y_x, pd_x, _), _ = run_both(acq, iq)
    idx = np.sort(np.random.default_rng(21).choice(acq.n_vox, 2048, replace=False))
    print(check_oracle(acq, iq, y_x, pd_x, idx))


@pytest.mark.parametrize("F", [32, 64])
def test_exact_many_transmits_ragged_tiles_and_windows(F):
    """21 transmits (more than the shared-memory delay cache holds), a Hann window, t0 != 0,
    a grid whose sides leave ragged tiles, and random IQ (2D for 32 frames, 3D for 64)."""
    ang = np.linspace(-0.15, 0.15, 21)
    if F == 32:
        acq = synth.doppler2d(nx=29, nz=23, n_frames=F, n_elem=24, n_samples=400).replace(
            grid_origin=(-1.2e-3, 0.0, 4e-3), tx_angles=np.stack([ang, np.zeros(21)], 1))
    else:
        tx = np.stack([ang, np.zeros(21)], 1)
        tx[1::2] = tx[1::2, ::-1]                      # alternate azimuth / elevation tilts
        acq = synth.make_acquisition("volume3d", "small").replace(tx_angles=np.ascontiguousarray(tx))
    acq = acq.replace(apod="hann", t0=0.21e-6, f_number=1.3)
    iq = synth.random_iq(acq, 100 + F)
    (y_x, pd_x, _), _ = run_both(acq, iq)
    print(F, check_oracle(acq, iq, y_x, pd_x))


def test_exact_voxel_list_3d_and_user_arrivals():
    acq = synth.make_acquisition("volume3d", "small")
    rng = np.random.default_rng(6)
    # list tiles take 64 voxels in list order: list an 8 x 8 x 12 sub-box as 4^3 blocks so
    # that every tile stays compact (its sample windows then fit the staged ring)
    nx, ny, _ = acq.grid_dims
    ix, iy, iz = np.meshgrid(np.arange(4), np.arange(4), np.arange(4), indexing="ij")
    blk = [(ix + bx + 5) + nx * ((iy + by + 4) + ny * (iz + bz + 3))
           for bz in (0, 4, 8) for by in (0, 4) for bx in (0, 4)]
    P = acq.voxel_positions()[np.concatenate([b.transpose(2, 1, 0).ravel() for b in blk])].astype(np.float32)
    lst = acq.replace(grid_dims=None, vox_pos=P)
    iq = synth.random_iq(lst, 7)
    (y_x, pd_x, _), _ = run_both(lst, iq)
    check_oracle(lst, iq, y_x, pd_x)
    # arrival times: the plane waves' own delays plus a per-voxel jitter (a tile's delay
    # range then stays small enough for the staged windows)
    u = synth.iqmod.plane_wave_directions(lst)
    arr = ((u @ P.astype(np.float64).T) / lst.c + rng.uniform(0, 2e-8, (lst.n_tx, lst.n_vox))).astype(np.float32)
    (y_x, pd_x, _), _ = run_both(lst, iq, tx_table_dev=torch.from_numpy(arr).cuda(), tx_angles=None)
    check_oracle(lst, iq, y_x, pd_x, tx_arrival=arr)


def test_exact_per_transmit_output():
    acq = synth.make_acquisition("volume3d", "small").replace(iq_dtype="c64split")
    iq = synth.random_iq(acq, 3)
    x = synth.iqmod.to_c64split(iq.cuda())
    T, F = acq.n_tx, acq.n_frames
    with m.Plan(**m.plan_kwargs(acq)) as p:
        assert p.info()["variant"] == "staged_c64p_x64_v4"
        y = torch.empty((acq.n_vox, T, F), dtype=torch.complex64, device="cuda")
        m.mach_das_run_per_tx(p.handle, x, y)
        full = p.run(x)
        torch.cuda.synchronize()
    # compounding = the sum of the per-transmit volumes (up to float32 summation order)
    assert nrmse_db(y.sum(1).cpu().numpy(), full.cpu().numpy()) < -110
    t = T // 2
    y_ref, _ = oracle.das(acq.replace(tx_angles=acq.tx_angles[t:t + 1]), iq[t:t + 1].contiguous())
    assert nrmse_db(y[:, t].cpu().numpy(), y_ref) <= -100.0


def test_term_table_plans_keep_the_generic_kernel():
    acq, iq = synth.make("doppler2d", "small", device="cpu")
    a = acq.replace(iq_dtype="c64split")
    with m.Plan(**m.plan_kwargs(a), term_table=True) as p:
        assert p.info()["variant"] == "staged_c64p_ft32_v4w7"
        assert p.info()["term_table_bytes"] > 0
        pd, y = p.power_doppler(synth.iqmod.to_c64split(iq.cuda()), want_y=True)
        torch.cuda.synchronize()
    check_oracle(acq, iq, y, pd)


def test_exact_bounded_wait_reports_timeout():
    acq, iq = synth.make("doppler2d", "small", device="cpu")
    a = acq.replace(iq_dtype="c64split")
    x = synth.iqmod.to_c64split(iq.cuda())
    m.mach_debug_set_wait_limit(2000)
    m.mach_debug_stall_producer(True)
    try:
        with m.Plan(**m.plan_kwargs(a)) as p:
            assert p.info()["variant"] == PAIRS[32][0]
            p.power_doppler(x, want_y=True)
            assert p.device_status() == m.MACH_ERR_TIMEOUT
    finally:
        m.mach_debug_stall_producer(False)
        m.mach_debug_set_wait_limit(0)
    with m.Plan(**m.plan_kwargs(a)) as p:
        pd, y = p.power_doppler(x, want_y=True)
        assert p.device_status() == m.MACH_OK
    check_oracle(acq, iq, y, pd)


SHAPES = [("staged_c64p_x32_v4w7", 32), ("staged_c64p_x32_f4v2w7", 32), ("staged_c64p_x32_f8v1w7", 32),
          ("staged_c64p_x32_f4v2w15", 32), ("staged_c64p_x32_f8v1w15", 32), ("staged_c64p_x64_v4", 64),
          ("staged_c64p_x64_f8v2", 64), ("staged_c64p_x32_f8v1w15t24", 32), ("staged_c64p_x32_f8v1w15t40", 32),
          ("staged_c64p_x32_f8v1w15t24s", 32), ("staged_c64p_x64_v4s", 64), ("staged_c64p_x32_f8v1w7t14", 32),
          ("staged_c64p_x32_f8v1w7t14e", 32), ("staged_c64p_x32_f4v2w7t14", 32), ("staged_c64p_x32_f8v1w15t30r12", 32),
          ("staged_c64p_x32_f8v1w15t30r12e", 32), ("staged_c64p_x64_v4e", 64), ("staged_c64p_x64_v4t16", 64),
          ("staged_c64p_x64_v4t16e", 64), ("staged_c64p_x32_v4w7_t8x14", 32), ("staged_c64p_x32_f8v1w7_t8x7e", 32),
          ("staged_c64p_x64_v4_t8x8", 64)]


@pytest.mark.parametrize("name,F", SHAPES)
def test_every_exact_shape_against_the_generic_kernel(name, F):
    """Each voxel's kept terms arrive in the same pair order whatever the tiling (pairs no
    voxel of a tile uses add nothing), so the frames are bitwise those of the generic
    kernel for every lane shape; Power Doppler too when a voxel's frames sit on the same
    lanes (4 frames per lane), else within float32 summation-order error."""
    acq, iq = synth.make("doppler2d" if F == 32 else "volume3d", "small", device="cpu")
    a = acq.replace(iq_dtype="c64split")
    kw = m.plan_kwargs(a)
    x = synth.iqmod.to_c64split(iq.cuda())
    res = {}
    for v in (name, PAIRS[F][1]):
        try:
            plan = forced(kw, v)
        except m.MachError as e:    # a shape whose ring does not fit this workload's windows
            assert e.status == m.MACH_ERR_UNSUPPORTED and v != PAIRS[F][0]
            pytest.skip(f"{v}: ring does not fit")
        with plan as p:
            assert p.info()["variant"] == v
            pd, y = p.power_doppler(x, want_y=True)
            torch.cuda.synchronize()
            assert p.device_status() == m.MACH_OK
            res[v] = (y, pd, p.info())
    (y_x, pd_x, info), (y_g, pd_g, _) = res[name], res[PAIRS[F][1]]
    assert torch.equal(y_x, y_g)
    if info["frames_per_lane"] == 4:
        assert torch.equal(pd_x, pd_g)
    else:
        assert nrmse_db(pd_x.cpu().numpy().astype(np.float64), pd_g.cpu().numpy().astype(np.float64)) < -120
    print(name, info["tile"], info["ctas"], check_oracle(acq, iq, y_x, pd_x))


def small_2d(F, T=1, seed=0):
    """A small 2D acquisition (ragged tiles) with F frames and T plane waves, random IQ."""
    ang = np.linspace(-0.1, 0.1, T) if T > 1 else np.zeros(1)
    acq = synth.doppler2d(nx=45, nz=29, n_frames=F, n_elem=40, n_samples=600).replace(
        grid_origin=(-2.2e-3, 0.0, 5e-3), tx_angles=np.stack([ang, np.zeros(T)], 1))
    return acq, synth.random_iq(acq, 50 + F + seed)


@pytest.mark.parametrize("F,T,expect", [(8, 1, "staged_c64p_x8_f4v1w7"), (16, 1, "staged_c64p_x16_f4v2w7"),
                                        (16, 3, "staged_c64p_x16_f4v2w7"), (8, 5, "staged_c64p_x8_f4v1w7")])
def test_few_frames(F, T, expect):
    """8 and 16 frames (exact-frame kernels for short ensembles): the default plan's kernel
    against the L1-path kernel (same per-frame FMA sequence and, with 32 voxels per warp,
    the same term order: bitwise frames) and against the oracle."""
    acq, iq = small_2d(F, T)
    a = acq.replace(iq_dtype="c64split")
    kw = m.plan_kwargs(a)
    x = synth.iqmod.to_c64split(iq.cuda())
    with m.Plan(**kw) as p:
        info = p.info()
        assert info["variant"] == expect
        pd, y = p.power_doppler(x, want_y=True)
        y_only = p.run(x)
        torch.cuda.synchronize()
        assert p.device_status() == m.MACH_OK
    assert torch.equal(y, y_only)
    l1 = "frames_c64p_ft32" if F <= 32 else "frames_c64p_ft64"
    with forced(kw, l1) as pl:
        pd_l, y_l = pl.power_doppler(x, want_y=True)
        torch.cuda.synchronize()
        same_order = T == 1 or pl.info()["voxels_per_cta"] // 8 == 32
    if same_order:
        assert torch.equal(y, y_l)
    else:
        assert nrmse_db(y.cpu().numpy(), y_l.cpu().numpy()) < -120
    assert nrmse_db(pd.cpu().numpy().astype(np.float64), pd_l.cpu().numpy().astype(np.float64)) < -120
    print(F, T, info["tile"], info["frame_tiles"], check_oracle(acq, iq, y, pd))
