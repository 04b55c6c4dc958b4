"""RF input on the GPU: demodulation against the FP64 oracle, and DAS of demodulated RF
against DAS of the analytic IQ of the same scatterer."""
import numpy as np
import pytest
import torch

import synth
from synth import iq as iqm
from synth import phantoms
from oracle import rf_oracle
import paper_2604_06257_gb300 as m
from paper_2604_06257_gb300 import build as pkg_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg_build.build()
    m.lib()


@pytest.mark.parametrize("shape,taps,decim", [((2, 5, 301, 3), 17, 2), ((1, 3, 1000, 1), 1, 1),
                                              ((3, 4, 257, 7), 64, 3), ((1, 2, 64, 32), 128, 1),
                                              ((1, 1, 10, 2), 33, 4)])
def test_rf_to_iq_matches_oracle(shape, taps, decim):
    r = np.random.default_rng(sum(shape) + taps)
    rf = r.standard_normal(shape).astype(np.float32)
    h = r.standard_normal(taps).astype(np.float32)
    fs, fc, t0 = 31.2e6, 7.8e6, 2.1e-6
    got = m.mach_rf_to_iq(torch.as_tensor(rf).cuda(), h, fs, fc, t0, decim).cpu().numpy()
    ref = rf_oracle.rf_to_iq(rf, h, fs, fc, t0, decim)
    # float32 products and sums, the fixed-point carrier phase (<= S 2^-33 turns) and the
    # sine/cosine (a few ulp) relative to sum |h| |rf|
    scale = rf_oracle.rf_to_iq(np.abs(rf), np.abs(h), fs, 0.0, 0.0, decim).real
    bound = ((taps + 2) * 2.0 ** -24 + 2 * np.pi * shape[2] * 2.0 ** -33 + 1e-6) * scale + 1e-30
    assert np.all(np.abs(got - ref) <= bound)


# Even ensembles of 16 frames or more with up to 16 taps per polyphase branch take the
# polyphase kernel: several branch counts (P = 1 ... 16), partial frame tiles, a signal
# shorter than one block's outputs, large decimations (10, 40), many blocks; an odd frame
# count and a source off the 8-byte grid fall back to the direct kernel.
@pytest.mark.parametrize("shape,taps,decim,offset", [((2, 3, 301, 32), 17, 2, 0), ((1, 2, 1000, 48), 32, 4, 0),
                                                     ((1, 1, 50, 16), 33, 4, 0), ((2, 2, 513, 20), 1, 1, 0),
                                                     ((1, 3, 700, 17), 24, 3, 0), ((1, 1, 4000, 16), 64, 10, 0),
                                                     ((1, 1, 4000, 16), 64, 40, 0), ((1, 2, 400, 32), 32, 4, 1),
                                                     ((4, 96, 1200, 32), 32, 4, 0)])
def test_rf_polyphase_matches_oracle(shape, taps, decim, offset):
    r = np.random.default_rng(sum(shape) + taps + decim)
    rf = r.standard_normal(shape).astype(np.float32)
    h = r.standard_normal(taps).astype(np.float32)
    fs, fc, t0 = 83.2e6, 5.2e6, 1.3e-6
    buf = torch.zeros(rf.size + offset, dtype=torch.float32, device="cuda")
    buf[offset:] = torch.as_tensor(rf.ravel()).cuda()
    src = buf[offset:].view(shape)
    got = m.mach_rf_to_iq(src, h, fs, fc, t0, decim).cpu().numpy()
    ref = rf_oracle.rf_to_iq(rf, h, fs, fc, t0, decim)
    scale = rf_oracle.rf_to_iq(np.abs(rf), np.abs(h), fs, 0.0, 0.0, decim).real
    bound = ((taps + 2) * 2.0 ** -24 + 2 * np.pi * shape[2] * 2.0 ** -33 + 1e-6) * scale + 1e-30
    assert np.all(np.abs(got - ref) <= bound)


def test_beamforming_demodulated_rf():
    acq = synth.make_acquisition("bmode2d", "small").replace(n_frames=2)
    ph = phantoms.Phantom(np.array([[0.5e-3, 0.0, 20e-3], [-1.2e-3, 0.0, 17e-3]]), np.array([1.0, 0.6]))
    rf = iqm.simulate_rf(acq, ph, 2, device="cuda")
    h = iqm.lowpass_taps(65, acq.fc, 2 * acq.fs)
    iq = m.mach_rf_to_iq(rf, h, 2 * acq.fs, acq.fc, acq.t0, 2)
    assert tuple(iq.shape) == acq.iq_shape
    model = iqm.simulate(acq, ph, seed=0, snr_db=None, device="cuda")
    with m.Plan(**m.plan_kwargs(acq)) as p:
        y_rf = p.run(iq)
        y_iq = p.run(model)
        torch.cuda.synchronize()
    err = float((y_rf - y_iq).abs().pow(2).sum() / y_iq.abs().pow(2).sum())
    assert 10 * np.log10(err) < -50.0
    # the brightest voxel is the same
    assert int(y_rf[:, 0].abs().argmax()) == int(y_iq[:, 0].abs().argmax())
