"""Mixed-level image batches through one convolution (GPU vs the oracle, bit for bit).

Three images at levels 5, 3 and 4 go through a conv planned at level 5: the plaintexts are
encoded once at scale q_5 and serve every lower level.  In HE_FUSED mode one fused-kernel
launch carries every image's groups; each image's output must equal the oracle's raised-basis
convolution at that image's level with the same integer plaintexts.  The per-rotation modes
must equal the oracle's per-rotation convolution."""
import numpy as np
import pytest

from oracle import layers as Ly
from oracle.params import Params
from oracle.ckks import Context
from oracle.encode import encode

pytestmark = pytest.mark.gpu

MID = Params(log_n=12, n_q=6, n_p=2, dnum=3, q0_bits=50, q_bits=40, p_bits=50,
             scale=2.0 ** 40, seed=5)


def test_mixed_level_batch_bit_exact():
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import GpuCtx, assert_ct_equal
    o = Context(MID)
    g = GpuCtx(MID)
    try:
        c, co, m, k, pad, top = 4, 4, 32, 3, 1, 5
        rng = np.random.default_rng(21)
        W = rng.uniform(-1, 1, (co, c, k, k))
        b = rng.uniform(-1, 1, co)
        lin = Ly.image_layout(c, m, o.N)
        plan = Ly.conv_plan(lin, W, b, pad)
        assert lin.n_shards == 2 and plan.lout.n_shards == 2
        S_pt = float(o.q[top])
        pts = Ly.conv_plaintexts(plan, o.n, S_pt)
        keys = [(vv, uu, aa) for vv in sorted(plan.terms) for (uu, aa) in sorted(plan.terms[vv])]
        lay = H.he_layout_image(c, m, o.N)
        conv = H.he_conv_create(g.h, lay, W, b, 1, pad, top, o.pr.scale)
        H.he_keygen_rotations(g.h, H.he_conv_rotations(conv))
        H.he_conv_import_plaintexts(conv, np.stack([pts[(uu, vv, aa)] for (vv, uu, aa) in keys]), None)
        levels = [5, 3, 4, 2, 5]                  # two image groups of the image-batched MAC
        imgs, cts, refs_f, refs_p, ins = [], [], [], [], []
        for i, lv in enumerate(levels):
            x = rng.uniform(0, 1, (c, m, m))
            slots = Ly.pack(lin, x)
            ci = [o.encrypt(slots[u], lv, nonce=700 + 10 * i + u) for u in range(lin.n_shards)]
            out_scale = o.pr.scale * S_pt / float(o.q[lv])
            bias = {v: encode(plan.bias[v], o.n, out_scale) for v in range(plan.lout.n_shards)}
            H.he_conv_import_bias(conv, lv, out_scale, np.stack([bias[v] for v in range(plan.lout.n_shards)]))
            refs_f.append(Ly.conv_he_raised(o, plan, ci, pts, bias, pt_scale=S_pt))
            refs_p.append(Ly.conv_he(o, plan, ci, pts, bias, pt_scale=S_pt))
            imgs.append(x)
            ins += [g.upload(ct) for ct in ci]
        runs = [(H.HE_FUSED, H.HE_KEY_STREAM_AUTO, refs_f), (H.HE_FUSED, H.HE_KEY_STREAM_LDG, refs_f),
                (H.HE_FUSED, H.HE_KEY_STREAM_TMA, refs_f), (H.HE_FUSED, H.HE_KEY_STREAM_SPLIT, refs_f),
                (H.HE_FUSED, H.HE_KEY_STREAM_CP, refs_f), (H.HE_FUSED, H.HE_KEY_STREAM_LDG1, refs_f),
                (H.HE_FUSED, H.HE_KEY_STREAM_PK, refs_f), (H.HE_FUSED, H.HE_KEY_STREAM_SPLITM, refs_f),
                (H.HE_PLAIN, H.HE_KEY_STREAM_AUTO, refs_p), (H.HE_BATCHED, H.HE_KEY_STREAM_AUTO, refs_p)]
        for mode, ks, refs in runs:
            H.he_ctx_set_option(g.h, H.HE_OPT_KEY_STREAM, ks)
            outs = [g.ct(top - 1) for _ in range(len(levels) * plan.lout.n_shards)]
            H.he_conv_run_batch(g.h, conv, ins, outs, len(levels), mode)
            H.he_ctx_check(g.h)
            for i, lv in enumerate(levels):
                for v in range(plan.lout.n_shards):
                    oc, rc = outs[i * plan.lout.n_shards + v], refs[i][v]
                    assert H.he_ct_level(oc) == lv - 1 and H.he_ct_scale(oc) == rc.scale
                    assert_ct_equal(g.download(oc), rc)
        # and the batch decrypts to the plaintext convolution for every image
        import torch
        for i, x in enumerate(imgs):
            want = (torch.nn.functional.conv2d(torch.tensor(x)[None], torch.tensor(W), padding=pad)[0].numpy()
                    + b[:, None, None])
            got = Ly.unpack(plan.lout, np.stack([o.decrypt(ct) for ct in refs_f[i]]))
            assert np.abs(got - want).max() <= 2.0 ** -20 * (want.max() - want.min())
        # a level outside 1..top is refused
        bad = [g.ct(0) for _ in range(lin.n_shards)]
        with pytest.raises(H.HEError) as e:
            H.he_conv_run_batch(g.h, conv, bad, outs[:plan.lout.n_shards], 1, H.HE_FUSED)
        assert e.value.code == H.HE_ELEVEL
        H.he_conv_destroy(conv)
    finally:
        g.close()
