"""The one-call layers he_hconv2d and he_havgpool.

They plan with the library's own encoder, so their bits are defined by the library: each must
give exactly the limbs of the create / run path on the same input (which the other GPU tests
compare limb by limb with the oracle after importing the oracle's plaintexts), the output
layout the oracle plans, and a decryption within 2^-20 of the range of torch's conv2d /
avg_pool2d."""
import numpy as np
import pytest
import torch

from oracle import layers as Ly
from oracle.ckks import Context
from oracle.params import Params

pytestmark = pytest.mark.gpu

MID = Params(log_n=12, n_q=6, n_p=2, dnum=3, q0_bits=50, q_bits=40, p_bits=50,
             scale=2.0 ** 40, seed=5)


@pytest.fixture(scope="module")
def mid():
    from tests._hegpu_util import GpuCtx
    o = Context(MID)
    g = GpuCtx(MID)
    yield o, g
    g.close()


def _close(img, want):
    assert img.shape == want.shape
    assert np.abs(img - want).max() <= 2.0 ** -20 * (want.max() - want.min())


@pytest.mark.parametrize("c,co,m,k,stride,pad", [(8, 8, 28, 3, 1, 1), (3, 4, 32, 7, 2, 3), (4, 4, 16, 3, 1, 1)])
def test_hconv2d_equals_create_run_and_decrypts_to_conv2d(mid, c, co, m, k, stride, pad):
    from paper_2306_09189_gb300 import hegpu as H
    o, g = mid
    level = 5
    rng = np.random.default_rng(c * 13 + m + stride)
    x = rng.uniform(0, 1, (c, m, m))
    W = rng.uniform(-1, 1, (co, c, k, k)) / k
    b = rng.uniform(-1, 1, co)
    lin = Ly.image_layout(c, m, o.N)
    plan = Ly.conv_plan(lin, W, b, pad)
    lout = Ly.pool_plan(plan.lout, select_top_left=True).lout if stride == 2 else plan.lout
    lay = H.he_layout_image(c, m, o.N)
    ins = [g.upload(o.encrypt(s, level, nonce=2300 + u)) for u, s in enumerate(Ly.pack(lin, x))]
    want = (torch.nn.functional.conv2d(torch.tensor(x)[None], torch.tensor(W), stride=stride,
                                       padding=pad)[0].numpy() + b[:, None, None])
    out_level = level - (1 if stride == 1 else 3)
    conv = H.he_conv_create(g.h, lay, W, b, stride, pad, level, o.pr.scale)
    H.he_keygen_rotations(g.h, H.he_conv_rotations(conv))
    for mode in (H.HE_PLAIN, H.HE_BATCHED, H.HE_FUSED):
        outs = [g.ct(level) for _ in range(lout.n_shards)]
        lay_out = H.he_hconv2d(g.h, lay, ins, W, b, stride, pad, mode, outs)
        chan, row0 = lay_out.tables()
        assert np.array_equal(chan, lout.chan) and np.array_equal(row0, lout.row0)
        ref = [g.ct(out_level) for _ in range(lout.n_shards)]
        H.he_conv_run(g.h, conv, ins, ref, mode)
        for oc, rc in zip(outs, ref):
            assert H.he_ct_level(oc) == out_level and H.he_ct_scale(oc) == H.he_ct_scale(rc)
            assert np.array_equal(g.download(oc), g.download(rc))
        _close(Ly.unpack(lout, np.stack([H.he_decrypt(g.h, oc, o.N) for oc in outs])), want)
    H.he_conv_destroy(conv)


@pytest.mark.parametrize("c,m", [(8, 32), (2, 64), (3, 32)])
def test_havgpool_equals_create_run_and_decrypts_to_avg_pool(mid, c, m):
    from paper_2306_09189_gb300 import hegpu as H
    o, g = mid
    level = 4
    rng = np.random.default_rng(c + 7 * m)
    x = rng.uniform(0, 1, (c, m, m))
    lin = Ly.image_layout(c, m, o.N)
    lout = Ly.pool_plan(lin).lout
    lay = H.he_layout_image(c, m, o.N)
    ins = [g.upload(o.encrypt(s, level, nonce=2400 + u)) for u, s in enumerate(Ly.pack(lin, x))]
    want = torch.nn.functional.avg_pool2d(torch.tensor(x)[None], 2)[0].numpy()
    pool = H.he_pool_create(g.h, lay, level)
    H.he_keygen_rotations(g.h, H.he_pool_rotations(pool))
    for mode in (H.HE_PLAIN, H.HE_BATCHED, H.HE_FUSED):
        outs = [g.ct(level) for _ in range(lout.n_shards)]
        lay_out = H.he_havgpool(g.h, lay, ins, mode, outs)
        chan, row0 = lay_out.tables()
        assert np.array_equal(chan, lout.chan) and np.array_equal(row0, lout.row0)
        ref = [g.ct(level - 2) for _ in range(lout.n_shards)]
        H.he_pool_run(g.h, pool, ins, ref, mode)
        for oc, rc in zip(outs, ref):
            assert H.he_ct_level(oc) == level - 2
            assert np.array_equal(g.download(oc), g.download(rc))
        _close(Ly.unpack(lout, np.stack([H.he_decrypt(g.h, oc, o.N) for oc in outs])), want)
    H.he_pool_destroy(pool)
