"""The C ABI without a GPU: the library loads, exports every declared entry point, and
rejects bad arguments before touching CUDA."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2604_06257_gb300 as m
from paper_2604_06257_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg_build.build()


def declared_functions(header=None):
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)) if header is None else [header]:
        src = open(os.path.join(inc, h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(mach_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    L = m.lib()
    names = declared_functions()
    assert "mach_das_plan" in names and "mach_power_doppler" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(m.EXPORTS) >= set(declared_functions("mach.h"))
    from paper_2604_06257_gb300 import nn
    assert set(m.EXPORTS) | set(nn.NN_EXPORTS) == set(names)


def test_status_strings_and_version():
    assert m.mach_status_string(0) == "ok"
    assert "invalid" in m.mach_status_string(1)
    assert m.mach_status_string(99) == "unknown status"
    assert "sm_103a" in m.mach_version()


def good_kwargs(**over):
    kw = dict(ndim=2, elem_pos=np.stack([np.linspace(-1e-3, 1e-3, 8), np.zeros(8), np.zeros(8)], 1),
              tx_angles=np.zeros((1, 2)), fs=20e6, fc=5e6, c=1540.0, n_samples=64, n_frames=4,
              grid_dims=(4, 1, 4), grid_origin=(0.0, 0.0, 1e-3), grid_step=(1e-4, 0.0, 1e-4))
    kw.update(over)
    return kw


BAD = [
    dict(ndim=4),
    dict(fs=0.0),
    dict(fs=float("nan")),
    dict(c=-1.0),
    dict(fc=-1.0),
    dict(f_number=-0.5),
    dict(apod=7),
    dict(iq_dtype=5),
    dict(term_table=2),
    dict(n_samples=1),
    dict(n_samples=(1 << 24) + 1),
    dict(n_frames=0),
    dict(grid_dims=(0, 1, 4)),
    dict(grid_dims=(4, 2, 4)),                       # 2D grid must have ny = 1
    dict(grid_origin=(0.0, 1e-3, 1e-3)),             # 2D grid must lie in y = 0
    dict(tx_angles=np.array([[0.0, 0.1]])),          # 2D: no elevation tilt
    dict(elem_pos=np.ones((8, 3))),                  # 2D: elements at y = 0
    dict(elem_pos=np.full((2, 3), np.inf)),
    dict(grid_dims=None, vox_pos=np.zeros((0, 3))),
    dict(grid_dims=None, vox_pos=np.array([[0.0, 1e-3, 1e-3]])),
]


@pytest.mark.parametrize("over", BAD)
def test_invalid_descriptors_rejected_before_cuda(over):
    kw = good_kwargs(**over)
    if kw.get("grid_dims") is None:
        kw.pop("grid_dims"); kw.pop("grid_origin"); kw.pop("grid_step")
    d, keep = m.make_desc(**kw)
    h = C.c_void_p(1234)
    st = m.lib().mach_das_plan(C.byref(d), None, C.byref(h))
    assert st == m.MACH_ERR_INVALID_ARG
    assert h.value is None


def test_null_arguments():
    L = m.lib()
    h = C.c_void_p()
    assert L.mach_das_plan(None, None, C.byref(h)) == m.MACH_ERR_INVALID_ARG
    d, keep = m.make_desc(**good_kwargs())
    assert L.mach_das_plan(C.byref(d), None, None) == m.MACH_ERR_INVALID_ARG
    assert L.mach_das_run(None, None, None, None) == m.MACH_ERR_INVALID_ARG
    assert L.mach_power_doppler(None, None, None, None, None) == m.MACH_ERR_INVALID_ARG
    assert L.mach_power_doppler_host_stream(None, None, 0, None, None, 1) == m.MACH_ERR_INVALID_ARG
    assert L.mach_plan_destroy(None) == m.MACH_OK
    assert L.mach_plan_get_info(None, None) == m.MACH_ERR_INVALID_ARG
    assert L.mach_plan_tx_table(None, None, None) == m.MACH_ERR_INVALID_ARG
    assert L.mach_das_terms(None, None, 0, None, None, None, None) == m.MACH_ERR_INVALID_ARG


def test_unsupported_slab_size():
    d, keep = m.make_desc(**good_kwargs(n_samples=1 << 24, n_frames=256))
    h = C.c_void_p()
    assert m.lib().mach_das_plan(C.byref(d), None, C.byref(h)) == m.MACH_ERR_UNSUPPORTED


def test_valid_descriptor_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    d, keep = m.make_desc(**good_kwargs())
    h = C.c_void_p()
    assert m.lib().mach_das_plan(C.byref(d), None, C.byref(h)) == m.MACH_ERR_CUDA
    assert h.value is None


def test_network_entry_points_reject_bad_arguments_before_cuda():
    from paper_2604_06257_gb300 import nn
    L = nn._L()
    fake = C.c_void_p(256)   # never dereferenced: every call below fails validation first
    # channel counts must be multiples of 16
    assert L.mach_nn_conv3d(fake, fake, None, fake, None, 1, 4, 4, 4, 8, 16, 0, 0, None) == m.MACH_ERR_INVALID_ARG
    assert L.mach_nn_conv3d(fake, fake, None, None, None, 1, 4, 4, 4, 16, 16, 0, 0, None) == m.MACH_ERR_INVALID_ARG
    assert L.mach_nn_conv3d(C.c_void_p(258), fake, None, fake, None, 1, 4, 4, 4, 16, 16, 0, 0, None) == \
        m.MACH_ERR_INVALID_ARG   # misaligned input
    assert L.mach_nn_conv3d_wgrad(fake, fake, fake, 1, 4, 4, 4, 16, 24, None) == m.MACH_ERR_INVALID_ARG
    assert L.mach_nn_bias_grad(fake, fake, 10, 48, None) == m.MACH_ERR_INVALID_ARG
    assert L.mach_nn_pool2(fake, fake, 1, 3, 4, 4, 16, 0, 0, None) == m.MACH_ERR_INVALID_ARG   # odd side
    assert L.mach_nn_up2(fake, fake, 1, 2, 2, 2, 16, 16, 8, 0, None) == m.MACH_ERR_INVALID_ARG   # off + c > cy
    assert L.mach_nn_adam(fake, fake, fake, fake, 10, 1e-3, 0.9, 0.999, 1e-8, 0, None, None, 0, 0, None) == \
        m.MACH_ERR_INVALID_ARG   # step 0
    h = C.c_void_p()
    for d, want in [((0, 16, 1, 8, 8, 8), m.MACH_ERR_INVALID_ARG),      # no level
                    ((4, 8, 1, 8, 8, 8), m.MACH_ERR_INVALID_ARG),       # base channels not a multiple of 16
                    ((4, 16, 1, 12, 8, 8), m.MACH_ERR_INVALID_ARG),     # nx not a multiple of 8
                    ((4, 16, 0, 8, 8, 8), m.MACH_ERR_INVALID_ARG),      # empty batch
                    ((4, 48, 1, 8, 8, 8), m.MACH_ERR_UNSUPPORTED)]:     # 384 channels at the bottom
        assert L.mach_unet_create(C.byref(nn.mach_unet_desc(*d, 0)), 0, C.byref(h)) == want, d
        assert not h.value


def test_rf_to_iq_rejects_bad_arguments_before_cuda():
    L = m.lib()
    fake = C.c_void_p(256)
    h = np.ones(4, dtype=np.float32)
    hp = h.ctypes.data
    ok = dict(rf=fake, iq=fake, T=1, C=2, S=100, F=1, fs=20e6, fc=5e6, t0=0.0, taps=hp, L=4, D=1)
    cases = [dict(L=0), dict(L=129), dict(D=0), dict(D=101), dict(fs=0.0), dict(fs=float("nan")),
             dict(fc=-1.0), dict(t0=float("inf")), dict(S=0), dict(iq=None), dict(rf=C.c_void_p(258))]
    for over in cases:
        a = {**ok, **over}
        st = L.mach_rf_to_iq(a["rf"], a["iq"], a["T"], a["C"], a["S"], a["F"], a["fs"], a["fc"], a["t0"],
                             a["taps"], a["L"], a["D"], None)
        assert st == m.MACH_ERR_INVALID_ARG, over
    bad = np.array([1.0, np.nan], dtype=np.float32)
    assert L.mach_rf_to_iq(fake, fake, 1, 1, 10, 1, 20e6, 5e6, 0.0, bad.ctypes.data, 2, 1, None) == \
        m.MACH_ERR_INVALID_ARG


def test_term_table_is_plan_state_only():
    """The allocation-free entry point and ragged batches have no term table: a
    descriptor asking for one is refused before anything touches the device."""
    d, keep = m.make_desc(**good_kwargs(term_table=True))
    fake = C.c_void_p(256)
    L = m.lib()
    assert L.mach_das_run_noalloc(C.byref(d), fake, fake, None, None) == m.MACH_ERR_UNSUPPORTED
    arr = (m.mach_das_desc * 1)(d)
    h = C.c_void_p()
    assert L.mach_batch_plan(arr, 1, None, None, C.byref(h)) == m.MACH_ERR_UNSUPPORTED


def test_rf_to_iq_size_limits_refused_before_launch():
    """More than 65535 runs of 64 output samples (the grid's second axis), or a decimation
    whose phasor window exceeds 48 KB of shared memory, are refused before any launch."""
    L = m.lib()
    fake = C.c_void_p(256)
    h = np.ones(8, dtype=np.float32)
    # 65536 * 64 + 1 IQ samples per channel at decimation 1
    assert L.mach_rf_to_iq(fake, fake, 1, 1, 65536 * 64 + 1, 1, 20e6, 5e6, 0.0, h.ctypes.data, 8, 1,
                           None) == m.MACH_ERR_UNSUPPORTED
    # (63 * decim + taps) complex phasors over 48 KB
    assert L.mach_rf_to_iq(fake, fake, 1, 1, 100000, 1, 20e6, 5e6, 0.0, h.ctypes.data, 8, 100,
                           None) == m.MACH_ERR_UNSUPPORTED
    # more than 2^24 frames (a block's outputs are counted in 32 bits)
    assert L.mach_rf_to_iq(fake, fake, 1, 1, 100, (1 << 24) + 1, 20e6, 5e6, 0.0, h.ctypes.data, 8, 1,
                           None) == m.MACH_ERR_UNSUPPORTED


def test_every_variant_name_the_tests_force_is_known():
    """Each kernel variant the GPU tests, the benchmark or the autotuner name by string is
    one the library knows (the lookup needs no GPU); an unknown name is refused."""
    pat = re.compile(r"[\"']((?:staged|frames|channels)_(?:c64p|c64|f16|b16|h16)_[a-z0-9_]+)[\"']")
    names = set()
    for rel in ("tests", "paper_2604_06257_gb300"):
        d = os.path.join(ROOT, rel)
        for f in sorted(os.listdir(d)):
            if f.endswith(".py"):
                names |= set(pat.findall(open(os.path.join(d, f)).read()))
    names |= set(pat.findall(open(os.path.join(ROOT, "bench.py")).read()))
    assert len(names) > 30
    unknown = []
    try:
        for n in sorted(names):
            try:
                m.mach_debug_force_variant(n)
            except m.MachError:
                unknown.append(n)
        known = names - set(unknown)
        # the rest are families matched with startswith ("staged_c64p_x32")
        for n in unknown:
            assert any(k.startswith(n + "_") for k in known), n
        assert len(unknown) <= 2
        with pytest.raises(m.MachError) as e:
            m.mach_debug_force_variant("staged_no_such_variant")
        assert e.value.status == m.MACH_ERR_INVALID_ARG
    finally:
        m.mach_debug_force_variant(None)
