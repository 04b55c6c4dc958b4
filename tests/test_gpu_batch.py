"""Ragged batches: many instances in one persistent launch, against the FP64 oracle and
against single-instance plans; graph capture; the autotuner's choices."""
import numpy as np
import pytest
import torch

import oracle
import synth
from synth.ragged import ragged_instances
import paper_2604_06257_gb300 as m
from paper_2604_06257_gb300 import autotune, build as pkg_build
from metrics import nrmse_db

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg_build.build()
    m.lib()


def buffers(acqs, seed=0):
    iqs, ys, pds = [], [], []
    for i, a in enumerate(acqs):
        iq = synth.random_iq(a, seed + i, device="cuda")
        iqs.append(iq)
        ys.append(torch.zeros((a.n_vox, a.n_frames), dtype=torch.complex64, device="cuda"))
        pds.append(torch.zeros(a.n_vox, dtype=torch.float32, device="cuda"))
    return iqs, ys, pds


@pytest.mark.parametrize("dtype", ["c64", "f16x2"])
def test_ragged_batch_matches_oracle(dtype):
    # frame counts for every lane mapping and load width: channel lanes (F <= 4), two frame
    # lanes (5-8), single samples (odd F), 8-byte pairs (even F off the 16-byte grid: 10,
    # 18, 34), 16-byte vectors (F % 4 == 0), staged windows (F > 16 off the grid)
    acqs = ragged_instances(n=13, seed=11, iq_dtype=dtype, scale=0.12)
    acqs = [a.replace(n_frames=F) for a, F in zip(acqs, [1, 3, 4, 5, 7, 10, 12, 17, 18, 33, 34, 48, 64])]
    iqs, ys, pds = buffers(acqs)
    stored = [synth.iqmod.to_storage(x, dtype) for x in iqs]
    with m.Batch([m.plan_kwargs(a) for a in acqs]) as b:
        b.bind(stored, ys, pds)
        b.run()
        torch.cuda.synchronize()
        info = b.info()
    assert info["instances"] == 13 and info["items"] >= 13
    modes = [s[0] for s in info["shapes"]]
    # channel lanes for F <= 4; staged windows for F > 16 off the 16-byte grid (frame lanes
    # where a window exceeds the ring); frame lanes otherwise
    assert modes[:3] == [1, 1, 1] and all(x in (0, 2) for x in modes[3:]) and 2 in modes
    assert all(mo == 0 for a, mo in zip(acqs, modes) if 4 < a.n_frames and (a.n_frames <= 16 or a.n_frames % 4 == 0))
    for a, x, y, pd in zip(acqs, stored, ys, pds):
        idx = np.arange(0, a.n_vox, max(1, a.n_vox // 300))
        y_ref, pd_ref = oracle.das(a, synth.iqmod.from_storage(x.cpu()), idx)
        assert nrmse_db(y.cpu().numpy()[idx], y_ref) <= -100, a.name
        assert nrmse_db(pd.cpu().numpy()[idx].astype(np.float64), pd_ref) <= -60, a.name


def test_batch_equals_single_plans_and_replays_from_a_graph():
    acqs = ragged_instances(n=6, seed=5, iq_dtype="c64", scale=0.15)
    iqs, ys, pds = buffers(acqs, seed=50)
    kws = [m.plan_kwargs(a) for a in acqs]
    with m.Batch(kws) as b:
        b.bind(iqs, ys, pds)
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            b.run(stream=s)                     # warm-up outside capture
        s.synchronize()
        for y in ys:
            y.zero_()
        with torch.cuda.graph(g):
            b.run()
        g.replay()
        g.replay()                              # the work counter resets itself
        torch.cuda.synchronize()
    for a, iq, y, pd in zip(acqs, iqs, ys, pds):
        with m.Plan(**m.plan_kwargs(a)) as p:
            pd1, y1 = p.power_doppler(iq, want_y=True)
            torch.cuda.synchronize()
        assert nrmse_db(y.cpu().numpy(), y1.cpu().numpy()) <= -110, a.name
        assert nrmse_db(pd.cpu().numpy().astype(np.float64), pd1.cpu().numpy().astype(np.float64)) <= -100


def test_explicit_shapes_and_validation():
    acqs = ragged_instances(n=3, seed=8, iq_dtype="c64", scale=0.1)
    acqs = [a.replace(n_frames=F) for a, F in zip(acqs, [2, 20, 40])]
    kws = [m.plan_kwargs(a) for a in acqs]
    shapes = [(1, 0, None), (0, 8, None), (0, 16, (2, 2, 16) if acqs[2].ndim == 3 else (4, 1, 16))]
    iqs, ys, pds = buffers(acqs, seed=70)
    with m.Batch(kws, shapes=shapes) as b:
        b.bind(iqs, ys, pds)
        b.run()
        torch.cuda.synchronize()
        got = b.info()["shapes"]
    assert got[0][:2] == (1, 0) and got[1][:2] == (0, 8) and got[2][:2] == (0, 16)
    for a, iq, y in zip(acqs, iqs, ys):
        idx = np.arange(0, a.n_vox, max(1, a.n_vox // 200))
        y_ref, _ = oracle.das(a, iq.cpu(), idx)
        assert nrmse_db(y.cpu().numpy()[idx], y_ref) <= -100
    # staged windows with explicit frame lanes and boxes
    st = [(1, 0, None), (2, 8, (28, 1, 4) if acqs[1].ndim == 2 else (4, 4, 7)),
          (2, 16, (14, 1, 4) if acqs[2].ndim == 2 else (4, 2, 7))]
    with m.Batch(kws, shapes=st) as b:
        b.bind(iqs, ys, pds)
        b.run()
        torch.cuda.synchronize()
        got = b.info()["shapes"]
    assert [g[:2] for g in got] == [(1, 0), (2, 8), (2, 16)]
    for a, iq, y in zip(acqs, iqs, ys):
        idx = np.arange(0, a.n_vox, max(1, a.n_vox // 200))
        y_ref, _ = oracle.das(a, iq.cpu(), idx)
        assert nrmse_db(y.cpu().numpy()[idx], y_ref) <= -100
    bad = [[(1, 0, None), (0, 8, None), (0, 4, None)],          # 4 lanes x 4 frames < 40 frames
           [(0, 8, None), (0, 8, None), (0, 16, None)],         # channel lanes required for F <= 4? no: allowed
           [(1, 0, None), (0, 8, (3, 1, 3)), (0, 16, None)]]    # tile volume mismatch
    with pytest.raises(m.MachError):
        m.Batch(kws, shapes=bad[0])
    with pytest.raises(m.MachError):
        m.Batch(kws, shapes=bad[2])
    with pytest.raises(m.MachError):                          # 8 staged frame lanes hold 32 frames
        m.Batch(kws, shapes=[(1, 0, None), (0, 8, None), (2, 8, None)])


def test_two_frame_lanes_for_up_to_eight_frames():
    """5-8 frames: two lanes per voxel (4 frames each, 2 voxels per lane), by default and
    with explicit boxes, 2D and 3D, vector and scalar frame loads, against the oracle."""
    acqs = ragged_instances(n=4, seed=12, iq_dtype="f16x2", scale=0.12)
    acqs = [a.replace(n_frames=F) for a, F in zip(acqs, [8, 6, 5, 8])]
    kws = [m.plan_kwargs(a) for a in acqs]
    iqs, ys, pds = buffers(acqs, seed=90)
    stored = [synth.iqmod.to_storage(x, "f16x2") for x in iqs]
    boxes = [None, None, (16, 1, 16) if acqs[2].ndim == 2 else (8, 4, 8),
             (8, 1, 32) if acqs[3].ndim == 2 else (4, 4, 16)]
    for shapes in (None, [(0, 2, b) for b in boxes]):
        with m.Batch(kws, shapes=shapes) as b:
            b.bind(stored, ys, pds)
            b.run()
            torch.cuda.synchronize()
            assert [g[:2] for g in b.info()["shapes"]] == [(0, 2)] * 4
        for a, x, y, pd in zip(acqs, stored, ys, pds):
            idx = np.arange(0, a.n_vox, max(1, a.n_vox // 300))
            y_ref, pd_ref = oracle.das(a, synth.iqmod.from_storage(x.cpu()), idx)
            assert nrmse_db(y.cpu().numpy()[idx], y_ref) <= -100, a.name
            assert nrmse_db(pd.cpu().numpy()[idx].astype(np.float64), pd_ref) <= -60, a.name
    with pytest.raises(m.MachError):                          # 2 lanes x 4 frames < 9 frames
        m.Batch([m.plan_kwargs(acqs[0].replace(n_frames=9))], shapes=[(0, 2, None)])


def test_autotuner_picks_a_valid_and_fastest_candidate():
    acqs = ragged_instances(n=2, seed=9, iq_dtype="f16x2", scale=0.2)
    kws = [m.plan_kwargs(a) for a in acqs]
    iqs, ys, pds = buffers(acqs, seed=90)
    stored = [synth.iqmod.to_f16x2(x) for x in iqs]
    for kw, iq, y, pd in zip(kws, stored, ys, pds):
        best, times = autotune.tune_instance(kw, iq, y, pd)
        assert best in autotune.candidates(kw)
        if times:
            assert times[best] == min(times.values())


def test_ragged_batch_full_scale_bench_instances():
    """The benchmarked batch itself: the 64 seeded instances at full scale (up to 1024
    elements, 112^3 voxels, 48 frames, 15 transmits; 4.9 GB of float16 IQ) in one
    persistent launch, each instance against the oracle on 256 sampled voxels (first
    and last voxel included) of the dequantised samples.  Covers the 64-bit IQ offsets,
    the longest-first work list of the whole batch and the work counter's reset (the
    launch runs twice)."""
    acqs = ragged_instances(n=64, seed=4, iq_dtype="f16x2", scale=1.0)
    kws = [m.plan_kwargs(a) for a in acqs]
    iqs, ys, pds = [], [], []
    for i, a in enumerate(acqs):
        iqs.append(synth.iqmod.to_f16x2(synth.random_iq(a, 1000 + i, device="cuda")))
        ys.append(torch.zeros((a.n_vox, a.n_frames), dtype=torch.complex64, device="cuda"))
        pds.append(torch.zeros(a.n_vox, dtype=torch.float32, device="cuda"))
    with m.Batch(kws) as b:
        b.bind(iqs, ys, pds)
        b.run()
        for y in ys:
            y.zero_()
        b.run()
        torch.cuda.synchronize()
        info = b.info()
    assert info["instances"] == 64
    rng = np.random.default_rng(44)
    worst_y, worst_pd = -np.inf, -np.inf
    for a, x, y, pd in zip(acqs, iqs, ys, pds):
        idx = np.unique(np.concatenate([[0, a.n_vox - 1], rng.choice(a.n_vox, 254, replace=False)]))
        y_ref, pd_ref = oracle.das(a, x.cpu(), idx)
        ey = nrmse_db(y[torch.from_numpy(idx).cuda()].cpu().numpy(), y_ref)
        ep = nrmse_db(pd[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64), pd_ref)
        assert ey <= -100, (a.name, ey)
        assert ep <= -60, (a.name, ep)
        worst_y, worst_pd = max(worst_y, ey), max(worst_pd, ep)
    print(f"64 instances at full scale: worst frames NRMSE {worst_y:.1f} dB, worst Power Doppler {worst_pd:.1f} dB")
