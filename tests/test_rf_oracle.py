"""Pins for the RF demodulation oracle (CPU): identity filter, a pure tone, decimation,
and the analytic echo, whose demodulated RF must be the IQ model (A/2) g e^{-j 2 pi fc tau}."""
import numpy as np
import pytest
import torch

import synth
from synth import iq as iqm
from synth import phantoms
from oracle import rf_oracle


def test_identity_filter_is_mixing_only():
    r = np.random.default_rng(0)
    rf = r.standard_normal((2, 3, 50, 4))
    fs, fc, t0 = 40e6, 5e6, 1.3e-6
    out = rf_oracle.rf_to_iq(rf, [1.0], fs, fc, t0, 1)
    m = np.arange(50)
    np.testing.assert_allclose(out, rf * np.exp(-2j * np.pi * fc * (t0 + m / fs))[None, None, :, None], rtol=1e-14)


def test_pure_tone_demodulates_to_its_phasor():
    fs, fc, t0, phi = 40e6, 5e6, 0.7e-6, 0.9
    m = np.arange(400)
    rf = np.cos(2 * np.pi * fc * (t0 + m / fs) + phi)[None, None, :, None]
    h = iqm.lowpass_taps(65, fc, fs)
    out = rf_oracle.rf_to_iq(rf, h, fs, fc, t0, 1)[0, 0, 40:-40, 0]
    assert np.max(np.abs(out - 0.5 * np.exp(1j * phi) * float(np.sum(h.astype(np.float64))))) < 2e-3


def test_decimation_subsamples():
    r = np.random.default_rng(1)
    rf = r.standard_normal((1, 2, 97, 3))
    h = r.standard_normal(9)
    full = rf_oracle.rf_to_iq(rf, h, 20e6, 3e6, 0.0, 1)
    for d in (2, 3, 5):
        np.testing.assert_array_equal(rf_oracle.rf_to_iq(rf, h, 20e6, 3e6, 0.0, d), full[:, :, ::d, :])


def test_analytic_echo_demodulates_to_the_iq_model():
    acq = synth.make_acquisition("bmode2d", "small").replace(n_frames=1)
    ph = phantoms.Phantom(np.array([[0.5e-3, 0.0, 20e-3]]), np.array([1.0]))
    rf = iqm.simulate_rf(acq, ph, 2)
    h = iqm.lowpass_taps(65, acq.fc, 2 * acq.fs)
    d = rf_oracle.rf_to_iq(rf.numpy(), h, 2 * acq.fs, acq.fc, acq.t0, 2)
    ref = iqm.simulate(acq, ph, seed=0, snr_db=None, accum=torch.complex128).numpy()
    err_db = 20 * np.log10(np.linalg.norm(d - ref) / np.linalg.norm(ref))
    assert err_db < -60.0, err_db


def test_carrier_factors_into_complex_taps_and_an_output_rotation():
    """The identity the polyphase RF kernel evaluates: with the carrier phase linear in the
    sample index, exp(-j phase(nD + k - c)) = exp(-j phase(nD - c)) exp(-j 2 pi fc k / fs), so
    filtering the real samples with complex taps h[k] exp(-j 2 pi fc k / fs) and rotating each
    output once gives the mixed-then-filtered result; and the polyphase split k = qD + r sums
    the same terms."""
    r = np.random.default_rng(3)
    rf = r.standard_normal((1, 2, 301, 3))
    h = r.standard_normal(23)
    fs, fc, t0, D = 83.2e6, 5.2e6, 0.9e-6, 4
    ref = rf_oracle.rf_to_iq(rf, h, fs, fc, t0, D)
    S, L = rf.shape[2], len(h)
    c = (L - 1) // 2
    n = np.arange((S - 1) // D + 1)
    g = h * np.exp(-2j * np.pi * fc * np.arange(L) / fs)
    P = -(-L // D)
    out = np.zeros_like(ref)
    for rr in range(D):                       # polyphase branches
        for q in range(P):
            k = q * D + rr
            if k >= L:
                continue
            m = n * D + k - c
            ok = (m >= 0) & (m < S)
            out[:, :, ok, :] += g[k] * rf[:, :, m[ok], :]
    out *= np.exp(-2j * np.pi * fc * (t0 + (n * D - c) / fs))[None, None, :, None]
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)



def test_centred_fir_equals_library_correlation():
    """The filter and decimation steps against numpy's correlation: with the mixed samples
    zero-padded by c = (L - 1) // 2 in front and L - 1 - c behind, the 'valid' correlation
    with the taps at index nD is the centred FIR output n (odd and even tap counts, one tap,
    several decimations)."""
    fs, fc, t0 = 31.2e6, 7.8e6, 0.4e-6
    m = np.arange(57)
    for L, D in ((7, 1), (8, 3), (1, 2), (12, 5)):
        r = np.random.default_rng(10 + L + D)
        rf = r.standard_normal((2, 3, 57, 2))
        h = r.standard_normal(L)
        out = rf_oracle.rf_to_iq(rf, h, fs, fc, t0, D)
        b = rf * np.exp(-2j * np.pi * fc * (t0 + m / fs))[None, None, :, None]
        c = (L - 1) // 2
        assert out.shape == (2, 3, (57 - 1) // D + 1, 2)
        for t in range(2):
            for ch in range(3):
                for f in range(2):
                    bp = np.concatenate([np.zeros(c), b[t, ch, :, f], np.zeros(L - 1 - c)])
                    ref = np.correlate(bp, h, mode="valid")[::D]
                    np.testing.assert_allclose(out[t, ch, :, f], ref, rtol=1e-12, atol=1e-12)
