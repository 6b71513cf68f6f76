"""The caller-provided device allocator (he_set_allocator) with PyTorch's caching allocator.

With torch's allocator installed, every device block of a context and its objects must come
from torch's pool (torch.cuda.memory_allocated grows by them and returns when they are freed),
the results must be the same bits as under cudaMalloc (here: a sharded convolution in every
mode against the oracle), and the allocator cannot be swapped while blocks are live.
"""
import numpy as np
import pytest

from oracle import layers as Ly
from oracle.ckks import Context
from oracle.encode import encode
from oracle.params import Params

pytestmark = pytest.mark.gpu

MID = Params(log_n=12, n_q=6, n_p=2, dnum=3, q0_bits=50, q_bits=40, p_bits=50,
             scale=2.0 ** 40, seed=5)


def test_torch_caching_allocator_backs_every_block():
    import torch
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import GpuCtx, assert_ct_equal
    torch.cuda.set_device(0)
    torch.cuda.synchronize()
    assert H.he_live_allocations() == 0
    o = Context(MID)
    c, co, m, level = 8, 8, 16, 3
    rng = np.random.default_rng(31)
    x = rng.uniform(0, 1, (c, m, m))
    W = rng.uniform(-1, 1, (co, c, 3, 3))
    lin = Ly.image_layout(c, m, o.N)
    plan = Ly.conv_plan(lin, W, None, 1)
    pts = Ly.conv_plaintexts(plan, o.n, float(o.q[level]))
    bias = {v: encode(plan.bias[v], o.n, o.pr.scale) for v in range(plan.lout.n_shards)}
    cts = [o.encrypt(s, level, nonce=2100 + u) for u, s in enumerate(Ly.pack(lin, x))]
    refs = {False: Ly.conv_he(o, plan, cts, pts, bias), True: Ly.conv_he_raised(o, plan, cts, pts, bias)}

    before = torch.cuda.memory_allocated()
    H.use_torch_allocator()
    try:
        g = GpuCtx(MID)
        try:
            in_pool = torch.cuda.memory_allocated() - before
            assert in_pool > 0 and H.he_live_allocations() > 0      # the context's tables and scratch
            with pytest.raises(H.HEError) as e:                       # blocks are live: no swap
                H.use_default_allocator()
            assert e.value.code == H.HE_ESTATE
            conv = H.he_conv_create(g.h, H.he_layout_image(c, m, o.N), W, None, 1, 1, level, o.pr.scale)
            H.he_keygen_rotations(g.h, H.he_conv_rotations(conv))
            keys = [(vv, uu, aa) for vv in sorted(plan.terms) for (uu, aa) in sorted(plan.terms[vv])]
            H.he_conv_import_plaintexts(conv, np.stack([pts[(uu, vv, aa)] for (vv, uu, aa) in keys]),
                                        np.stack([bias[v] for v in range(plan.lout.n_shards)]))
            ins = [g.upload(ct) for ct in cts]
            assert torch.cuda.memory_allocated() - before > in_pool  # keys, plaintexts, ciphertexts
            for mode, ks in ((H.HE_PLAIN, H.HE_KEY_STREAM_AUTO), (H.HE_BATCHED, H.HE_KEY_STREAM_AUTO),
                             (H.HE_FUSED, H.HE_KEY_STREAM_AUTO), (H.HE_FUSED, H.HE_KEY_STREAM_SPLIT)):
                H.he_ctx_set_option(g.h, H.HE_OPT_KEY_STREAM, ks)
                outs = [g.ct(level - 1) for _ in range(plan.lout.n_shards)]
                H.he_conv_run(g.h, conv, ins, outs, mode)
                H.he_ctx_check(g.h)
                for oc, rc in zip(outs, refs[mode == H.HE_FUSED]):
                    assert_ct_equal(g.download(oc), rc)
            H.he_conv_destroy(conv)
        finally:
            g.close()
        assert H.he_live_allocations() == 0
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before                # every block went back
    finally:
        if H.he_live_allocations() == 0:
            H.use_default_allocator()
    # and the default allocator is back: a context no longer draws on torch's pool
    g = GpuCtx(MID)
    try:
        assert torch.cuda.memory_allocated() == before and H.he_live_allocations() > 0
    finally:
        g.close()

