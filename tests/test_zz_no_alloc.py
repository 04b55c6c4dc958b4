"""The allocation-free entry point, mach_das_run_noalloc, against the plan-based one.

Callers that cannot allocate device memory (host callbacks, real-time loops, host
frameworks that own all device memory) use mach_das_run_noalloc, which keeps its tables
in a fixed device array inside the library.  Two calls in a row on different workloads
(so the second overwrites the first one's tables) must each match mach_power_doppler on
a plan within the tolerances of the other GPU tests.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
import paper_2604_06257_gb300 as m
from paper_2604_06257_gb300 import build as pkg_build
from metrics import nrmse_db

pytestmark = pytest.mark.gpu


def test_noalloc_matches_plan_on_two_calls_in_a_row():
    pkg_build.build()
    L = m.lib()
    stream = torch.cuda.current_stream().cuda_stream
    runs = []
    for name in ("doppler2d", "bmode2d"):
        acq, iq = synth.make(name, "small", device="cuda")
        d, keep = m.make_desc(**m.plan_kwargs(acq))
        y = torch.full((acq.n_vox, acq.n_frames), 3.0 + 0j, dtype=torch.complex64, device="cuda")
        pd = torch.full((acq.n_vox,), 3.0, dtype=torch.float32, device="cuda")
        st = L.mach_das_run_noalloc(C.byref(d), iq.data_ptr(), y.data_ptr(), pd.data_ptr(), stream)
        assert st == m.MACH_OK, m.mach_status_string(st)
        runs.append((acq, iq, y, pd, keep))
    torch.cuda.synchronize()
    for acq, iq, y, pd, _ in runs:
        with m.Plan(**m.plan_kwargs(acq)) as p:
            pd_ref, y_ref = p.power_doppler(iq, want_y=True)
            torch.cuda.synchronize()
        yk, yr = y.cpu().numpy(), y_ref.cpu().numpy()
        assert nrmse_db(yk, yr) <= -100.0
        assert nrmse_db(pd.cpu().numpy().astype(np.float64), pd_ref.cpu().numpy().astype(np.float64)) <= -60.0


def test_noalloc_rejects_tables_beyond_the_fixed_array():
    acq = synth.make_acquisition("volume3d", "full")          # 2M voxels x 11 transmits
    d, keep = m.make_desc(**m.plan_kwargs(acq))
    y = torch.zeros(8, dtype=torch.complex64, device="cuda")
    st = m.lib().mach_das_run_noalloc(C.byref(d), y.data_ptr(), y.data_ptr(), None,
                                      torch.cuda.current_stream().cuda_stream)
    assert st == m.MACH_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert torch.count_nonzero(y).item() == 0
