"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars (reading R9): integer sample indices and interpolation weights bit-exact against
the oracle's float32 "contract" delays; complex frames (B-mode) NRMSE <= -100 dB and
Power Doppler NRMSE <= -60 dB for complex64 IQ; with float16 IQ storage, <= -100 dB
against the oracle run on the same (dequantised) samples and <= -60 dB against the
oracle on the unquantised complex64 samples.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2604_06257_gb300 as m
from paper_2604_06257_gb300 import build as pkg_build
from metrics import nrmse_db, peak_db

pytestmark = pytest.mark.gpu

FP32_BMODE_DB = -100.0
PD_DB = -60.0
FP16_DB = -60.0
# |y|^2 doubles the relative amplitude error of the stored samples: +6 dB over FP16_DB
FP16_PD_DB = FP16_DB + 6.0
# bfloat16 keeps 8 significand bits (unit roundoff 2^-8): the rms relative rounding error of
# a sample is about 2^-7/sqrt(12) x 0.72 (mean of 1/m over log-uniform mantissas m in [1, 2))
# ~ -56 dB; the gate leaves 6 dB of margin (PD: +6 dB as above)
BF16_DB = -50.0
BF16_PD_DB = BF16_DB + 6.0


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg_build.build()
    m.lib()


def plan_for(acq, **kw):
    return m.Plan(**{**m.plan_kwargs(acq), **kw})


def dev_iq(acq, iq):
    """Device IQ in the acquisition's storage type."""
    return synth.iqmod.to_storage(iq.cuda(), acq.iq_dtype)


def check_terms(acq, plan, idx):
    i0, w, cw = plan.terms(idx)
    i0, w, cw = i0.cpu().numpy(), w.cpu().numpy(), cw.cpu().numpy()
    tr = oracle.terms(acq, idx, mode="contract")
    ref_i0 = np.where(tr["valid"], tr["i0"], -1)
    np.testing.assert_array_equal(i0, ref_i0)
    v = tr["valid"]
    assert np.array_equal(w[v], tr["w"][v].astype(np.float32))       # exact value
    assert np.max(np.abs(cw[v] - tr["cw"][v]), initial=0.0) < 2e-6
    return int(v.sum())


# ------------------------------------------------------------------ tables ----

@pytest.mark.parametrize("name", ["bmode2d", "doppler2d", "volume3d", "ulm3d"])
@pytest.mark.parametrize("scale", ["small", "full"])
def test_tx_table_bit_identical(name, scale):
    acq = synth.make_acquisition(name, scale)
    with plan_for(acq) as p:
        got = p.tx_table().cpu().numpy()
    ref = oracle.tx_table(acq)
    assert got.shape == ref.shape
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_tx_table_voxel_list_and_user_arrivals():
    acq = synth.make_acquisition("volume3d", "small")
    rng = np.random.default_rng(0)
    P = acq.voxel_positions()[rng.permutation(acq.n_vox)[:500]].astype(np.float32)
    lst = acq.replace(grid_dims=None, vox_pos=P)
    with plan_for(lst) as p:
        got = p.tx_table().cpu().numpy()
    assert np.array_equal(got.view(np.uint32), oracle.tx_table(lst).view(np.uint32))
    # user-supplied arrival times in seconds (e.g. from a simulator)
    arr = (rng.uniform(5e-6, 20e-6, (3, lst.n_vox))).astype(np.float32)
    a3 = lst.replace(tx_angles=np.zeros((3, 2)))
    with plan_for(a3, tx_table_dev=torch.from_numpy(arr).cuda(), tx_angles=None) as p:
        got = p.tx_table().cpu().numpy()
    assert np.array_equal(got.view(np.uint32), oracle.tx_table(a3, tx_arrival=arr).view(np.uint32))


# ------------------------------------------------------------ index terms ----

@pytest.mark.parametrize("name", ["bmode2d", "doppler2d", "volume3d"])
def test_terms_bit_exact_small(name):
    acq = synth.make_acquisition(name, "small")
    with plan_for(acq) as p:
        n = check_terms(acq, p, np.arange(acq.n_vox))
    assert n > 0


@pytest.mark.parametrize("name", ["bmode2d", "doppler2d", "volume3d", "ulm3d"])
def test_terms_bit_exact_full_sampled(name):
    acq = synth.make_acquisition(name, "full")
    idx = np.sort(np.random.default_rng(11).choice(acq.n_vox, 1500, replace=False))
    with plan_for(acq) as p:
        assert check_terms(acq, p, idx) > 0


@pytest.mark.parametrize("apod", ["none", "boxcar", "hann", "gauss"])
def test_terms_all_windows_and_t0(apod):
    acq = synth.make_acquisition("volume3d", "small").replace(apod=apod, t0=0.37e-6, f_number=1.3)
    with plan_for(acq) as p:
        check_terms(acq, p, np.arange(0, acq.n_vox, 3))


# ------------------------------------------------------- beamformed output ----

def compare(acq, iq_host, y, pd, idx=None, bmode_db=FP32_BMODE_DB, iq_oracle=None, pd_db=PD_DB):
    y_ref, pd_ref = oracle.das(acq, iq_host if iq_oracle is None else iq_oracle, idx)
    out = {}
    if y is not None:
        yk = y.cpu().numpy()
        if idx is not None:
            yk = yk[idx]
        out["bmode_db"] = nrmse_db(yk, y_ref)
        out["bmode_peak_db"] = peak_db(yk, y_ref)
        assert out["bmode_db"] <= bmode_db, out
    if pd is not None:
        pk = pd.cpu().numpy().astype(np.float64)
        if idx is not None:
            pk = pk[idx]
        out["pd_db"] = nrmse_db(pk, pd_ref)
        out["pd_peak_db"] = peak_db(pk, pd_ref, power=True)
        assert out["pd_db"] <= pd_db, out
    return out


@pytest.mark.parametrize("name", ["bmode2d", "doppler2d", "volume3d", "ulm3d"])
def test_das_and_pd_small(name):
    acq, iq = synth.make(name, "small", device="cuda")
    with plan_for(acq) as p:
        y = p.run(iq)
        pd, y2 = p.power_doppler(iq, want_y=True)
        torch.cuda.synchronize()
    assert torch.equal(y, y2)
    r = compare(acq, iq.cpu(), y, pd)
    print(name, r)


def test_bmode2d_full_all_voxels():
    acq, iq = synth.make("bmode2d", "full", device="cuda")
    with plan_for(acq) as p:
        y = p.run(iq)
    print(compare(acq, iq.cpu(), y, None))


def test_doppler2d_full_all_voxels():
    """The benchmark workload, in the launch configuration the benchmark times."""
    acq, iq = synth.make("doppler2d", "full", device="cuda")
    with plan_for(acq) as p:
        assert p.info()["variant"].startswith("staged_c64_ft32")
        pd, y = p.power_doppler(iq, want_y=True)
    print(compare(acq, iq.cpu(), y, pd))


@pytest.mark.parametrize("iq_dtype", ["c64", "f16x2"])
def test_volume3d_full_sampled(iq_dtype):
    acq, iq = synth.make("volume3d", "full", device="cuda", iq_dtype=iq_dtype)
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(acq.n_vox, 384, replace=False))
    with plan_for(acq) as p:
        diq = dev_iq(acq, iq)
        pd, y = p.power_doppler(diq, want_y=True)
        torch.cuda.synchronize()
    if iq_dtype == "c64":
        print(compare(acq, iq.cpu(), y, pd, idx))
    else:
        q = synth.iqmod.from_f16x2(diq.cpu())
        print("vs dequantised", compare(acq, q, y, pd, idx))
        print("vs complex64", compare(acq, iq.cpu(), y, pd, idx, bmode_db=FP16_DB, pd_db=FP16_PD_DB))
    del iq


@pytest.mark.parametrize("name", ["doppler2d", "volume3d"])
def test_fp16_storage_small(name):
    acq, iq = synth.make(name, "small", device="cuda", iq_dtype="f16x2")
    diq = dev_iq(acq, iq)
    with plan_for(acq) as p:
        pd, y = p.power_doppler(diq, want_y=True)
    q = synth.iqmod.from_f16x2(diq.cpu())
    print(compare(acq, q, y, pd))
    print(compare(acq, iq.cpu(), y, pd, bmode_db=FP16_DB, pd_db=FP16_PD_DB))


# ------------------------------------------------------------- edge cases ----

def small_random(F, C=9, T=2, S=300, iq_dtype="c64", grid=(13, 1, 11), apod="hann", **kw):
    base = synth.doppler2d(nx=grid[0], nz=grid[2], n_frames=F, n_elem=C, n_samples=S,
                           iq_dtype=iq_dtype).replace(
        grid_origin=(-0.6e-3, 0.0, 4e-3), tx_angles=np.stack([np.linspace(-0.1, 0.1, T), np.zeros(T)], 1),
        apod=apod, **kw)
    return base


@pytest.mark.parametrize("F", [1, 2, 3, 4, 5, 7, 16, 17, 32, 33, 64, 65, 130])
def test_frame_counts_c64(F):
    acq = small_random(F)
    iq = synth.random_iq(acq, F, device="cuda")
    with plan_for(acq) as p:
        pd, y = p.power_doppler(iq, want_y=True)
        info = p.info()
    print(F, info["variant"], info["frame_tiles"], compare(acq, iq.cpu(), y, pd))


@pytest.mark.parametrize("name", ["channels_c64_cl8", "channels_c64_cl16", "channels_c64_cl32"])
@pytest.mark.parametrize("F,C", [(1, 9), (3, 33), (4, 128)])
def test_channel_lane_widths(name, F, C):
    """8, 16 or 32 lanes per voxel splitting its elements (shuffle-tree partial sums)."""
    acq = small_random(F, C=C, T=3)
    iq = synth.random_iq(acq, 40 + F + C, device="cuda")
    m.mach_debug_force_variant(name)
    try:
        p = plan_for(acq)
    finally:
        m.mach_debug_force_variant(None)
    with p:
        assert p.info()["variant"] == name
        pd, y = p.power_doppler(iq, want_y=True)
    compare(acq, iq.cpu(), y, pd)


@pytest.mark.parametrize("F,dt", [(512, "c64"), (512, "c64split"), (256, "f16x2")])
def test_largest_swept_frame_counts(F, dt):
    """The scaling sweep's longest ensembles (frame-tiled kernels) against the oracle."""
    acq = small_random(F, C=7, T=1, iq_dtype=dt, grid=(9, 1, 7))
    iq = synth.random_iq(acq, F + 3, device="cuda")
    diq = dev_iq(acq, iq)
    with plan_for(acq) as p:
        pd, y = p.power_doppler(diq, want_y=True)
        info = p.info()
    ref_iq = synth.iqmod.from_storage(diq.cpu()) if dt == "f16x2" else iq.cpu()
    print(F, dt, info["variant"], info["frame_tiles"], compare(acq, ref_iq, y, pd))


def test_largest_swept_channel_count():
    """8192 channels (the sweep's largest array) on the split-row default kernel, sampled voxels."""
    acq = small_random(32, C=8192, T=1, S=400, iq_dtype="c64split", grid=(33, 1, 17)).replace(
        elem_pos=synth.acquisition.linear_array(8192, pitch=0.3e-3 * 128 / 8192))
    iq = synth.random_iq(acq, 81, device="cuda")
    with plan_for(acq) as p:
        pd, y = p.power_doppler(dev_iq(acq, iq), want_y=True)
        info = p.info()
    idx = np.arange(0, acq.n_vox, 3)
    print(info["variant"], compare(acq, iq.cpu(), y, pd, idx=idx))


def test_largest_swept_voxel_count():
    """2510 x 2510 pixels (6.3 M voxels, the sweep's largest grid) in the benchmarked kernel,
    2048 sampled voxels against the oracle."""
    n, fov = 2510, 25.6e-3
    step = fov / n
    acq = synth.doppler2d().replace(grid_dims=(n, 1, n), grid_origin=(-(n - 1) * step / 2, 0.0, 10e-3),
                                    grid_step=(step, 0.0, step), iq_dtype="c64split")
    iq = synth.random_iq(acq, 25, device="cuda")
    with plan_for(acq) as p:
        pd, y = p.power_doppler(dev_iq(acq, iq), want_y=True)
        info = p.info()
    idx = np.sort(np.random.default_rng(25).choice(acq.n_vox, 2048, replace=False))
    print(info["variant"], compare(acq, iq.cpu(), y, pd, idx=idx))


@pytest.mark.parametrize("F", [1, 4, 6, 8, 12, 32, 36, 64, 68, 132])
def test_frame_counts_f16(F):
    acq = small_random(F, iq_dtype="f16x2")
    iq = synth.random_iq(acq, 100 + F, device="cuda")
    diq = dev_iq(acq, iq)
    with plan_for(acq) as p:
        pd, y = p.power_doppler(diq, want_y=True)
    compare(acq, synth.iqmod.from_f16x2(diq.cpu()), y, pd)


@pytest.mark.parametrize("C,T", [(1, 1), (3, 9), (17, 11), (33, 1)])
def test_channel_and_transmit_counts(C, T):
    for F in (3, 32, 64):
        acq = small_random(F, C=C, T=T)
        iq = synth.random_iq(acq, C * T + F, device="cuda")
        with plan_for(acq) as p:
            pd, y = p.power_doppler(iq, want_y=True)
        compare(acq, iq.cpu(), y, pd)


@pytest.mark.parametrize("apod", ["none", "boxcar", "gauss"])
def test_windows_end_to_end(apod):
    acq = small_random(32, apod=apod, t0=-0.2e-6)
    iq = synth.random_iq(acq, 7, device="cuda")
    with plan_for(acq) as p:
        y = p.run(iq)
    compare(acq, iq.cpu(), y, None)


def test_voxel_list_any_order_3d():
    acq = synth.make_acquisition("volume3d", "small").replace(n_frames=32)
    rng = np.random.default_rng(3)
    P = acq.voxel_positions()[rng.permutation(acq.n_vox)[:777]].astype(np.float32)
    lst = acq.replace(grid_dims=None, vox_pos=P)
    iq = synth.random_iq(lst, 8, device="cuda")
    with plan_for(lst) as p:
        pd, y = p.power_doppler(iq, want_y=True)
    compare(lst, iq.cpu(), y, pd)


def test_minimal_and_degenerate():
    # two samples per channel, one element, one voxel
    acq = synth.doppler2d(nx=1, nz=1, n_frames=1, n_elem=1, n_samples=2).replace(
        grid_origin=(0.0, 0.0, 0.5 * 1540 / 20.8e6 / 2), apod="none")
    iq = synth.random_iq(acq, 1, device="cuda")
    with plan_for(acq) as p:
        y = p.run(iq)
    y_ref, _ = oracle.das(acq, iq.cpu())
    assert abs(y.cpu().numpy()[0, 0] - y_ref[0, 0]) < 1e-5 * max(1.0, abs(y_ref[0, 0]))
    # every term past the end: exact zeros
    late = small_random(32, t0=-1e-3)
    iq = synth.random_iq(late, 2, device="cuda")
    with plan_for(late) as p:
        pd, y = p.power_doppler(iq, want_y=True)
    assert torch.count_nonzero(y).item() == 0 and torch.count_nonzero(pd).item() == 0


def test_large_sample_count():
    """S near the float-exact index limit region (2^20 samples)."""
    acq = small_random(2, C=2, T=1, S=1 << 20).replace(t0=-0.9 * (1 << 20) / 20.8e6)
    iq = synth.random_iq(acq, 3, device="cuda")
    with plan_for(acq) as p:
        y = p.run(iq)
        check_terms(acq, p, np.arange(acq.n_vox))
    compare(acq, iq.cpu(), y, None)


# --------------------------------------------------------- streams, graphs ----

def test_non_default_stream_and_graph_capture():
    acq, iq = synth.make("doppler2d", "small", device="cuda")
    with plan_for(acq) as p:
        ref_pd, ref_y = p.power_doppler(iq, want_y=True)
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        pd = torch.empty_like(ref_pd)
        y = torch.empty_like(ref_y)
        with torch.cuda.stream(s):
            m.mach_power_doppler(p.handle, iq, pd, y, stream=s)
        s.synchronize()
        assert torch.equal(pd, ref_pd) and torch.equal(y, ref_y)
        g = torch.cuda.CUDAGraph()
        pd2 = torch.zeros_like(ref_pd)
        y2 = torch.zeros_like(ref_y)
        with torch.cuda.graph(g):
            m.mach_power_doppler(p.handle, iq, pd2, y2)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(pd2, ref_pd) and torch.equal(y2, ref_y)


def test_errors_leave_outputs_untouched():
    acq, iq = synth.make("doppler2d", "small", device="cuda")
    with plan_for(acq) as p:
        y = torch.full((acq.n_vox, acq.n_frames), 7.0 + 0j, dtype=torch.complex64, device="cuda")
        import ctypes as C
        st = m.lib().mach_power_doppler(p.handle, iq.data_ptr(), None, y.data_ptr(), None)
        assert st == m.MACH_ERR_INVALID_ARG
        st = m.lib().mach_das_run(p.handle, None, y.data_ptr(), None)
        assert st == m.MACH_ERR_INVALID_ARG
        torch.cuda.synchronize()
        assert torch.all(y == 7.0)


def test_injected_allocation_failure_and_no_leak():
    acq = synth.make_acquisition("volume3d", "small").replace(n_frames=130)   # frame tiles -> 4 allocations
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in (1, 2, 3, 4):
        m.mach_debug_fail_alloc_after(k)
        with pytest.raises(m.MachError) as e:
            plan_for(acq)
        assert e.value.status == m.MACH_ERR_OOM
    m.mach_debug_fail_alloc_after(0)
    with plan_for(acq) as p:
        assert p.info()["frame_tiles"] > 1
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (64 << 20)


def test_oversize_plan_is_refused_before_allocating():
    acq = synth.doppler2d(nx=1 << 15, nz=1 << 15, n_frames=32)
    with pytest.raises(m.MachError) as e:
        plan_for(acq.replace(tx_angles=np.zeros((512, 2))))
    assert e.value.status == m.MACH_ERR_OOM


# ------------------------------------------------------ kernel variants ----

def forced(acq, name):
    m.mach_debug_force_variant(name)
    try:
        return plan_for(acq)
    finally:
        m.mach_debug_force_variant(None)


STAGED_CASES = [
    ("staged_c64_ft32", "frames_c64_ft32", "doppler2d", "c64"),
    ("staged_c64_ft32_v4", "frames_c64_ft32", "doppler2d", "c64"),
    ("staged_c64_ft64", "frames_c64_ft64", "volume3d", "c64"),
    ("staged_f16_ft32", "frames_f16_ft32", "doppler2d", "f16x2"),
    ("staged_f16_ft64", "frames_f16_ft64", "volume3d", "f16x2"),
    ("staged_c64_ft32_v4w4", "frames_c64_ft32", "doppler2d", "c64"),
    ("staged_c64_ft64_v4", "frames_c64_ft64", "volume3d", "c64"),
    ("staged_f16_ft64_v4", "frames_f16_ft64", "volume3d", "f16x2"),
    ("staged_b16_ft32", "frames_b16_ft32", "doppler2d", "bf16x2"),
    ("staged_b16_ft64_v4", "frames_b16_ft64", "volume3d", "bf16x2"),
    ("staged_c64p_ft32_v4", "frames_c64p_ft32", "doppler2d", "c64split"),
    ("staged_c64p_ft64_v4", "frames_c64p_ft64", "volume3d", "c64split"),
    ("staged_c64p_x32_v4w7", "frames_c64p_ft32", "doppler2d", "c64split"),
    ("staged_c64p_x64_v4", "frames_c64p_ft64", "volume3d", "c64split"),
    ("staged_f16_ft32_v4", "frames_f16_ft32", "doppler2d", "f16x2"),
    ("staged_b16_ft32_v4", "frames_b16_ft32", "doppler2d", "bf16x2"),
]


@pytest.mark.parametrize("staged,l1,name,dt", STAGED_CASES)
def test_staged_matches_oracle_and_l1_kernel_bitwise(staged, l1, name, dt):
    """The staged kernel reads the same taps from shared memory that the L1 kernel reads
    from global memory and accumulates the terms in the same order: identical bits."""
    acq, iq = synth.make(name, "small", device="cuda", iq_dtype=dt)
    diq = dev_iq(acq, iq)
    with forced(acq, staged) as ps, forced(acq, l1) as pl:
        assert ps.info()["variant"] == staged and pl.info()["variant"] == l1
        info = ps.info()
        same_order = pl.info()["voxels_per_cta"] // 8 == 32
        assert info["ring_rows"] >= 2 and info["copy_pairs"] > 0
        pd_s, y_s = ps.power_doppler(diq, want_y=True)
        pd_l, y_l = pl.power_doppler(diq, want_y=True)
        torch.cuda.synchronize()
        assert ps.device_status() == m.MACH_OK
    if same_order:
        # one element per round in both kernels: the same FMA sequence per accumulator
        assert torch.equal(y_s, y_l) and torch.equal(pd_s, pd_l)
    else:
        # the L1 kernel takes two elements per round (16 voxels per warp): other order
        assert nrmse_db(y_s.cpu().numpy(), y_l.cpu().numpy()) < -120
    ref_iq = synth.iqmod.from_storage(diq.cpu())
    print(staged, info["ring_rows"], info["copy_pairs"], compare(acq, ref_iq, y_s, pd_s))


@pytest.mark.parametrize("F", [18, 20, 30, 32, 34, 48, 62, 64])
def test_staged_partial_frame_tiles(F):
    acq = small_random(F, C=17, T=3)
    iq = synth.random_iq(acq, F, device="cuda")
    with plan_for(acq) as p:
        variant = p.info()["variant"]
        pd, y = p.power_doppler(iq, want_y=True)
    print(F, variant, compare(acq, iq.cpu(), y, pd))


def test_staged_full_doppler_bitwise_equal_to_l1():
    acq, iq = synth.make("doppler2d", "full", device="cuda")
    with forced(acq, "staged_c64_ft32") as ps, forced(acq, "frames_c64_ft32") as pl:
        pd_s, y_s = ps.power_doppler(iq, want_y=True)
        pd_l, y_l = pl.power_doppler(iq, want_y=True)
        torch.cuda.synchronize()
        print(ps.info())
    assert torch.equal(y_s, y_l) and torch.equal(pd_s, pd_l)


def test_forced_variant_rejections():
    acq = synth.make_acquisition("doppler2d", "small")
    with pytest.raises(m.MachError):
        m.mach_debug_force_variant("no_such_variant")
    m.mach_debug_force_variant("staged_f16_ft32")    # wrong storage type for this plan
    try:
        with pytest.raises(m.MachError) as e:
            plan_for(acq)
        assert e.value.status == m.MACH_ERR_UNSUPPORTED
    finally:
        m.mach_debug_force_variant(None)


def test_bounded_wait_reports_timeout_and_context_survives():
    """The producer announces its copies but never issues them: every consumer wait runs
    out (bounded), the kernel sets the error word and returns; the host reads
    MACH_ERR_TIMEOUT, and the same context then beamforms correctly."""
    acq, iq = synth.make("doppler2d", "small", device="cuda")
    m.mach_debug_set_wait_limit(2000)
    m.mach_debug_stall_producer(True)
    try:
        with plan_for(acq) as p:
            assert p.info()["variant"].startswith("staged")
            pd, y = p.power_doppler(iq, want_y=True)
            assert p.device_status() == m.MACH_ERR_TIMEOUT
            assert p.device_status() == m.MACH_OK          # cleared
    finally:
        m.mach_debug_stall_producer(False)
        m.mach_debug_set_wait_limit(0)
    with plan_for(acq) as p:
        pd, y = p.power_doppler(iq, want_y=True)
        assert p.device_status() == m.MACH_OK
    compare(acq, iq.cpu(), y, pd)


# ------------------------------------------------- K0 and bfloat16 storage ----

@pytest.mark.parametrize("dtype", ["c64", "f16x2", "bf16x2", "c64split"])
@pytest.mark.parametrize("order", ["ftcs", "tcsf"])
# odd T*C*S (8-byte tiles), even T*C*S with F % 4 == 2 (16-byte loads; 16-byte stores for
# complex64 only) and with F % 4 == 0 (16-byte loads and stores for every storage type)
@pytest.mark.parametrize("shape", [(3, 17, 129, 37), (2, 17, 130, 70), (2, 5, 66, 36)])
def test_iq_convert_bit_exact(order, dtype, shape):
    T, Cn, S, F = shape
    g = torch.Generator(device="cuda").manual_seed(5)
    src_tcsf = torch.view_as_complex(torch.randn((T, Cn, S, F, 2), generator=g, device="cuda") * 3)
    src = src_tcsf.permute(3, 0, 1, 2).contiguous() if order == "ftcs" else src_tcsf.contiguous()
    out = m.prepare_iq(src, order, dtype, shape=(T, Cn, S, F))
    ref = synth.iqmod.to_storage(src_tcsf.contiguous(), dtype)
    torch.cuda.synchronize()
    assert out.shape == ref.shape and out.dtype == ref.dtype
    assert torch.equal(out.view(torch.uint8) if dtype != "c64" else out, ref.view(torch.uint8) if dtype != "c64" else ref)


def test_iq_convert_rejects_bad_arguments():
    x = torch.zeros(64, dtype=torch.complex64, device="cuda")
    L = m.lib()
    assert L.mach_iq_convert(x.data_ptr(), 7, x.data_ptr() + 512, 0, 1, 1, 1, 1, None) == m.MACH_ERR_INVALID_ARG
    assert L.mach_iq_convert(x.data_ptr(), 0, x.data_ptr(), 0, 1, 1, 1, 1, None) == m.MACH_ERR_INVALID_ARG
    assert L.mach_iq_convert(x.data_ptr(), 0, x.data_ptr() + 512, 9, 1, 1, 1, 1, None) == m.MACH_ERR_INVALID_ARG
    assert L.mach_iq_convert(x.data_ptr(), 0, x.data_ptr() + 512, 0, 0, 1, 1, 1, None) == m.MACH_ERR_INVALID_ARG


@pytest.mark.parametrize("name", ["doppler2d", "volume3d"])
def test_bf16_storage_small(name):
    acq, iq = synth.make(name, "small", device="cuda", iq_dtype="bf16x2")
    diq = dev_iq(acq, iq)
    with plan_for(acq) as p:
        pd, y = p.power_doppler(diq, want_y=True)
    print(compare(acq, synth.iqmod.from_storage(diq.cpu()), y, pd))
    print(compare(acq, iq.cpu(), y, pd, bmode_db=BF16_DB, pd_db=BF16_PD_DB))


@pytest.mark.parametrize("F", [1, 4, 6, 8, 12, 32, 36, 64, 68])
def test_frame_counts_bf16(F):
    acq = small_random(F, iq_dtype="bf16x2")
    iq = synth.random_iq(acq, 200 + F, device="cuda")
    diq = dev_iq(acq, iq)
    with plan_for(acq) as p:
        pd, y = p.power_doppler(diq, want_y=True)
    compare(acq, synth.iqmod.from_storage(diq.cpu()), y, pd)


def test_prepare_then_beamform_from_acquisition_order():
    """K0 from scanner order followed by DAS equals DAS on the directly laid-out data."""
    acq, iq = synth.make("doppler2d", "small", device="cuda")
    scanner = iq.permute(3, 0, 1, 2).contiguous()        # [F][T][C][S]
    for dtype in ("c64", "f16x2", "bf16x2", "c64split"):
        a = acq.replace(iq_dtype=dtype)
        prepared = m.prepare_iq(scanner, "ftcs", dtype)
        with plan_for(a) as p:
            pd1, y1 = p.power_doppler(prepared, want_y=True)
            pd2, y2 = p.power_doppler(dev_iq(a, iq), want_y=True)
        assert torch.equal(y1, y2) and torch.equal(pd1, pd2)


@pytest.mark.parametrize("name,pair", [("doppler2d", ("staged_c64p_ft32_v4", "staged_c64_ft32_v4")),
                                       ("volume3d", ("staged_c64p_ft64_v4", "staged_c64_ft64_v4"))])
def test_split_rows_bitwise_equal_to_interleaved(name, pair):
    """Split complex64 rows (packed FP32x2 accumulation) perform the same FMA sequence per
    element as interleaved complex64: identical frames.  Power Doppler agrees to rounding
    only: the two layouts give a lane different frames, so the order of its partial
    sum of |y|^2 differs."""
    acq, iq = synth.make(name, "small", device="cuda")
    split = acq.replace(iq_dtype="c64split")
    with forced(split, pair[0]) as ps, forced(acq, pair[1]) as pi:
        pd_s, y_s = ps.power_doppler(synth.iqmod.to_c64split(iq), want_y=True)
        pd_i, y_i = pi.power_doppler(iq, want_y=True)
        torch.cuda.synchronize()
    assert torch.equal(y_s, y_i)
    assert torch.max(torch.abs(pd_s - pd_i) / pd_i.abs().clamp_min(1e-30)).item() < 1e-6


@pytest.mark.parametrize("F", [8, 12, 16, 20, 32, 36, 64, 68])
def test_frame_counts_split(F):
    acq = small_random(F, iq_dtype="c64split")
    iq = synth.random_iq(acq, 300 + F, device="cuda")
    with plan_for(acq) as p:
        pd, y = p.power_doppler(dev_iq(acq, iq), want_y=True)
    compare(acq, iq.cpu(), y, pd)


def test_split_rows_reject_unsupported_frame_counts():
    for F in (3, 4, 6):
        acq = small_random(F, iq_dtype="c64split")
        with pytest.raises(m.MachError) as e:
            plan_for(acq)
        assert e.value.status == m.MACH_ERR_UNSUPPORTED
