"""The learned-compounding workload at its full size (128^3 voxels, 1024 elements, 32
scenes per batch, split complex64 rows), in the launch configurations the benchmark
times: both DAS plans against the FP64 oracle on sampled voxels, and the network by
properties that hold at any size (the oracle cannot run it at 128^3 in test time)."""
import numpy as np
import pytest
import torch

import synth
import oracle
import paper_2604_06257_gb300 as m
from paper_2604_06257_gb300 import build as pkg_build, learned as Lc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg_build.build()
    m.lib()


def _nrmse_db(a, b):
    return 20 * np.log10(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("which", ["few", "many"])
def test_full_size_das_plans_match_oracle_on_sampled_voxels(which):
    acq = Lc.acquisition(128, 32, which).replace(iq_dtype="c64split")
    iq = synth.random_iq(acq.replace(iq_dtype="c64"), 77, device="cuda")        # complex64 [T, C, S, F]
    split = synth.iqmod.to_c64split(iq)
    with m.Plan(**m.plan_kwargs(acq)) as p:
        y = p.run(split)
        variant = p.info()["variant"]
        torch.cuda.synchronize()
    assert variant.startswith("staged_c64p_x32")
    idx = np.sort(np.random.default_rng(3).choice(acq.n_vox, 96, replace=False))
    y_ref, _ = oracle.das(acq.replace(iq_dtype="c64"), iq.cpu(), idx)
    err = _nrmse_db(y.cpu().numpy()[idx].astype(np.complex128), y_ref)
    assert err <= -100.0, err


def _random_net(batch, seed=4, biases=True):
    from oracle import unet_oracle
    from paper_2604_06257_gb300.nn import UNet
    p = unet_oracle.he_like(4, 16, np.random.default_rng(seed), scale=0.8)
    if not biases:
        for sp in unet_oracle.layout(4, 16):
            p[sp.b_off:sp.b_off + sp.co] = 0.0
    net = UNet(128, 128, 128, batch, levels=4, base_ch=16)
    net.set_params(p.astype(np.float32))
    net.set_gain(0.5)
    return net


def test_full_size_network_volumes_are_independent_of_the_batch():
    # every reduction is in a fixed order, so a volume's prediction is bit-identical alone
    # and inside a batch
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(128 ** 3, 4, dtype=torch.complex64, device="cuda", generator=g)
    with _random_net(4) as n4, _random_net(1) as n1:
        y4 = n4.forward(x)
        y1 = n1.forward(x[:, 2:3].contiguous())
        torch.cuda.synchronize()
    assert torch.equal(y4[:, 2:3], y1)


def test_network_commutes_with_eight_voxel_shifts_away_from_the_borders():
    # Three 2x poolings make the network equivariant to shifts by multiples of 8 voxels,
    # except within its receptive field of a border (zero padding there; about 67 voxels for
    # four levels).  A 256^3 volume and its copy rolled by 8 voxels per axis must give the
    # same prediction, shifted, at every voxel at least 72 voxels from a border and from the
    # rolled-in slab.  The two volumes hold the same values in another order, so their RMS
    # (the input normalisation) can differ in the last bit and move a few bfloat16
    # roundings: the gate is 1e-3 in relative L2 instead of bit equality.
    from oracle import unet_oracle
    from paper_2604_06257_gb300.nn import UNet
    n, s, r = 256, 8, 72
    g = torch.Generator(device="cuda").manual_seed(6)
    a = torch.randn(n, n, n, dtype=torch.complex64, device="cuda", generator=g)
    b = torch.roll(a, shifts=(s, s, s), dims=(0, 1, 2))
    x = torch.stack([a.reshape(-1), b.reshape(-1)], dim=1).contiguous()
    del a, b
    with UNet(n, n, n, 2, levels=4, base_ch=16) as net:
        net.set_params(unet_oracle.he_like(4, 16, np.random.default_rng(4), scale=0.8).astype(np.float32))
        net.set_gain(0.5)
        y = net.forward(x)
        torch.cuda.synchronize()
    c = slice(r, n - s - r)
    cs = slice(r + s, n - r)
    ya = y[:, 0].reshape(n, n, n)[c, c, c]
    yb = y[:, 1].reshape(n, n, n)[cs, cs, cs]
    rel = float((ya - yb).abs().pow(2).sum().sqrt() / ya.abs().pow(2).sum().sqrt())
    assert rel <= 1e-3, rel
