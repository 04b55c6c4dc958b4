"""Plan-time term table (mach_das_desc.term_table = 1): every run reads the terms the
plan stored instead of evaluating them, and must give the same bits as the on-the-fly
kernel -- same terms from the same device functions, accumulated in the same order --
for every storage type, 2D and 3D grids, voxel lists, ragged tiles and several
transmits; plus the FP64 oracle on one case, the bounded-wait path, and the cases
without a table form."""
import numpy as np
import pytest
import torch

import synth
import paper_2604_06257_gb300 as m
from paper_2604_06257_gb300 import build as pkg_build

from test_gpu_parity import compare, dev_iq, plan_for, small_random

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg_build.build()
    m.lib()


# with split rows and F = 32 or 64 the default on-the-fly plan runs an exact-frame kernel
# (tests/test_gpu_exact.py holds it to the generic kernel); a table plan keeps the generic
# kernel's record layout, so the table is compared with the generic on-the-fly kernel
GENERIC = {"staged_c64p_x32": "staged_c64p_ft32_v4w7", "staged_c64p_x64": "staged_c64p_ft64_v4"}


def on_the_fly_plan(acq):
    with plan_for(acq) as p:
        v = p.info()["variant"]
    g = GENERIC.get(v[:15])
    if g is None:
        return plan_for(acq)
    m.mach_debug_force_variant(g)
    try:
        return plan_for(acq)
    finally:
        m.mach_debug_force_variant(None)


def both_modes(acq, diq):
    with on_the_fly_plan(acq) as ph, plan_for(acq, term_table=True) as pt:
        ih, it = ph.info(), pt.info()
        pd_h, y_h = ph.power_doppler(diq, want_y=True)
        pd_t, y_t = pt.power_doppler(diq, want_y=True)
        y_only = pt.run(diq)
        torch.cuda.synchronize()
        assert pt.device_status() == m.MACH_OK
    assert ih["variant"] == it["variant"]
    assert ih["term_table_bytes"] == 0 and it["term_table_bytes"] > 0
    assert it["copy_pairs"] == ih["copy_pairs"]
    # pairs x voxel slots x 16 B of records + 16 B per pair + one 8-byte index per tile (+1)
    nrec = it["voxels_per_cta"]
    tiles = it["ctas"] // it["frame_tiles"]
    assert it["term_table_bytes"] == ih["copy_pairs"] * (16 * nrec + 16) + 8 * (tiles + 1)
    assert torch.equal(y_t, y_h) and torch.equal(pd_t, pd_h) and torch.equal(y_only, y_h)
    return it, y_t, pd_t


@pytest.mark.parametrize("F,dt", [(32, "c64split"), (32, "c64"), (24, "c64"), (64, "c64split"), (64, "c64"),
                                  (48, "c64"), (32, "f16x2"), (32, "bf16x2"), (64, "f16x2"), (64, "bf16x2"),
                                  (20, "c64split")])
def test_table_bitwise_equals_on_the_fly_2d(F, dt):
    # 64-frame tiles hold fewer rows per ring slot: a finer grid keeps their windows short
    step = 1e-4 if F <= 32 else 5e-5
    acq = small_random(F, C=19, T=3, S=400, iq_dtype=dt, grid=(29, 1, 23), grid_step=(step, 0.0, step))
    iq = synth.random_iq(acq, 11 * F, device="cuda")
    info, y, pd = both_modes(acq, dev_iq(acq, iq))
    assert info["variant"].startswith("staged")


def test_table_many_transmits():
    """More transmits than the on-the-fly kernel caches per warp (16): it then reads the
    transmit delays from global memory; the table must still give the same bits."""
    acq = small_random(32, C=9, T=21, S=400, iq_dtype="c64split", grid=(21, 1, 17))
    iq = synth.random_iq(acq, 21, device="cuda")
    diq = dev_iq(acq, iq)
    info, y, pd = both_modes(acq, diq)
    assert info["variant"].startswith("staged")
    compare(acq, synth.iqmod.from_storage(diq).cpu(), y, pd)


def test_table_unsupported_when_windows_exceed_the_ring():
    """Where the on-the-fly plan falls back to an L1-path kernel because the sample
    windows do not fit the ring, a table plan is refused (no table form)."""
    acq = small_random(64, C=19, T=3, S=400, iq_dtype="c64split", grid=(29, 1, 23), grid_step=(3e-4, 0.0, 3e-4))
    with plan_for(acq) as ph:
        assert not ph.info()["variant"].startswith("staged")
    with pytest.raises(m.MachError) as e:
        plan_for(acq, term_table=True)
    assert e.value.status == m.MACH_ERR_UNSUPPORTED


@pytest.mark.parametrize("name,dt", [("doppler2d", "c64split"), ("doppler2d", "c64"), ("volume3d", "c64split"),
                                     ("volume3d", "f16x2"), ("volume3d", "c64")])
def test_table_workloads_against_oracle(name, dt):
    acq, iq = synth.make(name, "small", device="cuda", iq_dtype=dt)
    diq = dev_iq(acq, iq)
    info, y, pd = both_modes(acq, diq)
    ref_iq = synth.iqmod.from_storage(diq).cpu()
    if dt in ("c64", "c64split"):
        compare(acq, ref_iq, y, pd)


def test_table_voxel_list_and_ragged_tiles():
    acq = small_random(32, C=13, T=2, S=350, iq_dtype="c64split", grid=(37, 1, 19))
    r = np.random.default_rng(5)
    # 333 scattered voxels, listed by depth so that a block's 112 consecutive voxels stay
    # within about a millimetre of depth (short sample windows); the last block is ragged
    vox = np.stack([r.uniform(-1.5e-3, 1.5e-3, 333), np.zeros(333), np.sort(r.uniform(3.5e-3, 7e-3, 333))], 1)
    acq = acq.replace(vox_pos=vox.astype(np.float32), grid_dims=None)
    iq = synth.random_iq(acq, 3, device="cuda")
    both_modes(acq, dev_iq(acq, iq))


def test_table_unsupported_without_staged_kernel():
    for F in (8, 1, 130):     # L1-path kernels: no table form
        acq = small_random(F)
        with pytest.raises(m.MachError) as e:
            plan_for(acq, term_table=True)
        assert e.value.status == m.MACH_ERR_UNSUPPORTED


def test_table_bounded_wait_reports_timeout():
    acq, iq = synth.make("doppler2d", "small", device="cuda", iq_dtype="c64split")
    diq = dev_iq(acq, iq)
    m.mach_debug_set_wait_limit(2000)
    m.mach_debug_stall_producer(True)
    try:
        with plan_for(acq, term_table=True) as p:
            p.power_doppler(diq, want_y=True)
            assert p.device_status() == m.MACH_ERR_TIMEOUT
            assert p.device_status() == m.MACH_OK
    finally:
        m.mach_debug_stall_producer(False)
        m.mach_debug_set_wait_limit(0)
    both_modes(acq, diq)
