"""Uncompounded (per-transmit) output: every transmit's volume equals the oracle's DAS of
that transmit alone, equals bit for bit a plan built for that transmit alone, and the
volumes sum to the compounded output."""
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


CASES = [(3, "c64"), (8, "c64"), (32, "c64"), (64, "c64"), (130, "c64"), (32, "f16x2"), (32, "c64split"),
         (64, "bf16x2")]


@pytest.mark.parametrize("F,dt", CASES)
def test_per_transmit_volumes(F, dt):
    T = 4
    acq = small_random(F, C=11, T=T, iq_dtype=dt)
    iq = synth.random_iq(acq, 7 * F + T, device="cuda")
    diq = dev_iq(acq, iq)
    ref_iq = synth.iqmod.from_storage(diq).cpu()          # the values the kernels read
    with plan_for(acq) as p:
        y_tx = p.run_per_tx(diq)
        y = p.run(diq)
        variant = p.info()["variant"]
    torch.cuda.synchronize()
    assert y_tx.shape == (acq.n_vox, T, F)
    # compounding the per-transmit volumes gives the compounded output (summation order
    # differs: float32 rounding only)
    tot = y_tx.sum(dim=1)
    assert float((tot - y).abs().max()) <= 1e-5 * float(y.abs().max())
    for t in range(T):
        one = acq.replace(tx_angles=acq.tx_angles[t:t + 1])
        iq_t = diq[t:t + 1].contiguous()
        yt = y_tx[:, t, :].contiguous()
        compare(one, ref_iq[t:t + 1].contiguous(), yt, None)
        with plan_for(one) as p1:
            assert p1.info()["variant"] == variant
            y1 = p1.run(iq_t)
        assert torch.equal(y1, yt), (t, variant)


def test_per_transmit_rejects_bad_arguments():
    acq = small_random(8, T=2)
    iq = synth.random_iq(acq, 1, device="cuda")
    with plan_for(acq) as p:
        y = torch.empty((acq.n_vox, 2, 8), dtype=torch.complex64, device="cuda")
        assert m.lib().mach_das_run_per_tx(p.handle, None, y.data_ptr(), None) == m.MACH_ERR_INVALID_ARG
        assert m.lib().mach_das_run_per_tx(p.handle, iq.data_ptr() + 8, y.data_ptr(), None) == \
            m.MACH_ERR_INVALID_ARG
        assert m.lib().mach_das_run_per_tx(None, iq.data_ptr(), y.data_ptr(), None) == m.MACH_ERR_INVALID_ARG
