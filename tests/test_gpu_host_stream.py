"""Pipelined host-memory entry point (mach_power_doppler_host_stream): for every
acquisition of a sequence, Power Doppler and frames equal bit for bit the one-acquisition
host path (K0 + mach_power_doppler, synchronised), whatever the sequence length (odd and
even, so both staging sets are reused), the source order and the storage type; the
frames also match the FP64 oracle."""
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


def host_seq(acq, n, order, seed0):
    """n distinct acquisitions as pinned host tensors in `order` (None: plan layout)."""
    out, raw = [], []
    for k in range(n):
        iq = synth.random_iq(acq, seed0 + k, device="cuda")      # complex64 [T, C, S, F]
        raw.append(iq)
        if order == "ftcs":
            h = iq.permute(3, 0, 1, 2).contiguous()
        elif order == "tcsf":
            h = iq
        else:
            h = dev_iq(acq, iq)
        out.append(h.cpu().pin_memory())
    return out, raw


@pytest.mark.parametrize("n,order,dt,F", [(1, "ftcs", "c64", 16), (5, "ftcs", "c64split", 32),
                                          (6, "tcsf", "c64", 8), (4, None, "c64", 17),
                                          (3, None, "bf16x2", 32), (7, "ftcs", "f16x2", 12)])
def test_stream_matches_single_calls(n, order, dt, F):
    acq = small_random(F, C=11, T=3, iq_dtype=dt)
    seq, raw = host_seq(acq, n, order, 100 * F)
    V = acq.n_vox
    pd = [torch.full((V,), float("nan")).pin_memory() for _ in range(n)]
    y = [torch.full((V, F), float("nan"), dtype=torch.complex64).pin_memory() for _ in range(n)]
    with plan_for(acq) as p:
        p.power_doppler_host_stream(seq, pd, y, order=order)
        pd1 = torch.empty(V).pin_memory()
        y1 = torch.empty((V, F), dtype=torch.complex64).pin_memory()
        for k in range(n):
            p.power_doppler_host(seq[k], pd1, y1, order=order)
            assert torch.equal(pd[k], pd1), k
            assert torch.equal(y[k], y1), k
        # without the frames: the same Power Doppler
        pd_only = [torch.empty(V).pin_memory() for _ in range(n)]
        p.power_doppler_host_stream(seq, pd_only, None, order=order)
        for k in range(n):
            assert torch.equal(pd_only[k], pd[k]), k
    # and against the FP64 oracle (first and last acquisition), on the values the kernels read
    for k in {0, n - 1}:
        ref_iq = synth.iqmod.from_storage(dev_iq(acq, raw[k])).cpu()
        compare(acq, ref_iq, y[k].cuda(), pd[k].cuda())


def test_stream_rejects_bad_arguments():
    acq = small_random(8)
    seq, _ = host_seq(acq, 2, "ftcs", 1)
    pd = [torch.empty(acq.n_vox).pin_memory() for _ in range(2)]
    with plan_for(acq) as p:
        with pytest.raises(ValueError):
            p.power_doppler_host_stream(seq, pd[:1], None, order="ftcs")
        with pytest.raises(ValueError):
            p.power_doppler_host_stream(seq, pd, None, order="tcsf")      # wrong shape for the order
        with pytest.raises(m.MachError):
            m.mach_power_doppler_host_stream(p.handle, seq, 7, pd)
        with pytest.raises(m.MachError):
            m.mach_power_doppler_host_stream(p.handle, [], "ftcs", [])
        # the plan is still usable
        p.power_doppler_host_stream(seq, pd, None, order="ftcs")
