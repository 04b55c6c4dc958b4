"""The allocation-free entry point, mach_das_run_noalloc, against the plan-based one and
the FP64 oracle.

Callers that cannot allocate device memory (host callbacks, real-time loops, host
frameworks that own all device memory) use mach_das_run_noalloc, which keeps its tables
in a fixed device array inside the library.  Two calls in a row on different workloads
(so the second overwrites the first one's tables) must each match mach_power_doppler on
a plan within the tolerances of the other GPU tests; so must a voxel list, user arrival
times and 16-bit IQ storage, which take other table paths.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2604_06257_gb300 as m
from paper_2604_06257_gb300 import build as pkg_build
from metrics import nrmse_db

pytestmark = pytest.mark.gpu


def noalloc(kw, iq, n_vox, F):
    """Frames and Power Doppler from mach_das_run_noalloc (outputs pre-filled with junk)."""
    L = m.lib()
    d, keep = m.make_desc(**kw)
    y = torch.full((n_vox, F), 3.0 + 0j, dtype=torch.complex64, device="cuda")
    pd = torch.full((n_vox,), 3.0, dtype=torch.float32, device="cuda")
    st = L.mach_das_run_noalloc(C.byref(d), iq.data_ptr(), y.data_ptr(), pd.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert st == m.MACH_OK, m.mach_status_string(st)
    return y, pd, keep


def plan_ref(kw, iq):
    with m.Plan(**kw) as p:
        pd, y = p.power_doppler(iq, want_y=True)
        torch.cuda.synchronize()
    return y, pd


def check(y, pd, y_ref, pd_ref, frames_db=-100.0, pd_db=-60.0):
    yk, yr = y.cpu().numpy(), np.asarray(y_ref)
    assert nrmse_db(yk, yr) <= frames_db, nrmse_db(yk, yr)
    pk, pr = pd.cpu().numpy().astype(np.float64), np.asarray(pd_ref, dtype=np.float64)
    assert nrmse_db(pk, pr) <= pd_db, nrmse_db(pk, pr)


def test_noalloc_matches_plan_on_two_calls_in_a_row():
    pkg_build.build()
    runs = []
    for name in ("doppler2d", "bmode2d"):
        acq, iq = synth.make(name, "small", device="cuda")
        kw = m.plan_kwargs(acq)
        y, pd, keep = noalloc(kw, iq, acq.n_vox, acq.n_frames)
        runs.append((acq, kw, iq, y, pd, keep))
    torch.cuda.synchronize()
    for acq, kw, iq, y, pd, _ in runs:
        y_ref, pd_ref = plan_ref(kw, iq)
        check(y, pd, y_ref.cpu().numpy(), pd_ref.cpu().numpy())
        y_o, pd_o = oracle.das(acq, iq.cpu())
        check(y, pd, y_o, pd_o)


def test_noalloc_voxel_list_and_user_arrival_times():
    """A voxel list (raw positions copied into the array) and arrival times given on the
    device (no plane-wave directions), each against the plan and the oracle."""
    pkg_build.build()
    acq, iq = synth.make("volume3d", "small", device="cuda")
    rng = np.random.default_rng(3)
    P = acq.voxel_positions()[rng.permutation(acq.n_vox)[:700]].astype(np.float32)
    lst = acq.replace(grid_dims=None, vox_pos=P)
    kw = m.plan_kwargs(lst)
    y, pd, _ = noalloc(kw, iq, lst.n_vox, lst.n_frames)
    torch.cuda.synchronize()
    y_ref, pd_ref = plan_ref(kw, iq)
    check(y, pd, y_ref.cpu().numpy(), pd_ref.cpu().numpy())
    check(y, pd, *oracle.das(lst, iq.cpu()))

    # arrival times in seconds per (transmit, voxel): here the plane waves' own delays
    # plus a per-voxel jitter, so the result differs from the plane-wave one
    T = lst.n_tx
    u = synth.iqmod.plane_wave_directions(lst)
    arr = ((u @ P.astype(np.float64).T) / lst.c + rng.uniform(0, 2e-8, (T, lst.n_vox))).astype(np.float32)
    arr_dev = torch.from_numpy(arr).cuda()
    kw_u = dict(kw, tx_table_dev=arr_dev, tx_angles=None)
    y, pd, _ = noalloc(kw_u, iq, lst.n_vox, lst.n_frames)
    torch.cuda.synchronize()
    y_ref, pd_ref = plan_ref(kw_u, iq)
    check(y, pd, y_ref.cpu().numpy(), pd_ref.cpu().numpy())
    check(y, pd, *oracle.das(lst, iq.cpu(), tx_arrival=arr))


def test_noalloc_bfloat16_storage():
    pkg_build.build()
    acq, iq = synth.make("doppler2d", "small", device="cuda", iq_dtype="bf16x2")
    q = synth.iqmod.to_bf16x2(iq)
    kw = m.plan_kwargs(acq)
    y, pd, _ = noalloc(kw, q, acq.n_vox, acq.n_frames)
    torch.cuda.synchronize()
    y_ref, pd_ref = plan_ref(kw, q)
    check(y, pd, y_ref.cpu().numpy(), pd_ref.cpu().numpy())
    deq = torch.view_as_complex(q.float().contiguous()).cpu()
    check(y, pd, *oracle.das(acq, deq))


def test_noalloc_rejects_tables_beyond_the_fixed_array():
    acq = synth.make_acquisition("volume3d", "full")          # 2M voxels x 11 transmits
    d, keep = m.make_desc(**m.plan_kwargs(acq))
    y = torch.zeros(8, dtype=torch.complex64, device="cuda")
    st = m.lib().mach_das_run_noalloc(C.byref(d), y.data_ptr(), y.data_ptr(), None,
                                      torch.cuda.current_stream().cuda_stream)
    assert st == m.MACH_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert torch.count_nonzero(y).item() == 0


def test_noalloc_refuses_a_capturing_stream():
    """Inside a CUDA-graph capture the call is refused before it enqueues anything (its
    host copies would be replayed from buffers that no longer exist)."""
    acq, iq = synth.make("doppler2d", "small", device="cuda")
    d, keep = m.make_desc(**m.plan_kwargs(acq))
    y = torch.zeros((acq.n_vox, acq.n_frames), dtype=torch.complex64, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        st = m.lib().mach_das_run_noalloc(C.byref(d), iq.data_ptr(), y.data_ptr(), None, s.cuda_stream)
    assert st == m.MACH_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert torch.count_nonzero(y).item() == 0
