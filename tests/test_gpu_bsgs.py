"""Baby-step giant-step convolution on the GPU against the oracle, bit for bit.

The oracle's BSGS plan (every diagonal amount a = g + t, baby steps rot_t of each input shard
weighted by rot_{-g} of the diagonal, giant steps rot_g of each partial sum) is imported as
integer plaintexts; the per-rotation modes must equal ``conv_he_bsgs(raised=False)`` and the
fused mode (every key-stream form) ``conv_he_bsgs(raised=True)``.  Image shards, duplicated
shards, a 5x5 kernel, channel shards (no giant steps), a mixed-level batch and stride 2."""
import numpy as np
import pytest
import torch

from oracle import layers as Ly
from oracle.params import Params
from oracle.ckks import Context
from oracle.encode import encode

pytestmark = pytest.mark.gpu

MID = Params(log_n=12, n_q=6, n_p=2, dnum=3, q0_bits=50, q_bits=40, p_bits=50,
             scale=2.0 ** 40, seed=5)

FORMS = ("LDG", "TMA", "CP", "LDG1", "SPLIT", "PK", "PK3", "PKP")


@pytest.fixture(scope="module")
def mid():
    from tests._hegpu_util import GpuCtx
    o = Context(MID)
    g = GpuCtx(MID)
    yield o, g
    g.close()


def _plan_order(bp, N):
    """(v, u, a) of every term in the library's BSGS order: v, then g, u, t."""
    out = []
    for (v, g) in bp.keys():
        for (u, t) in sorted(bp.baby[(v, g)]):
            out.append((v, u, (g + t) % N))
    return out


def _create(H, g, o, lin, W, b, level, pad, bp, stride=1):
    lay = H.he_layout_image(lin.c, lin.m, o.N)
    conv = H.he_conv_create_bsgs(g.h, lay, W, b, stride, pad, level, o.pr.scale, bp.k)
    assert H.he_conv_bsgs_giant(conv) == bp.k
    rots = set(int(r) for r in H.he_conv_rotations(conv))
    H.he_keygen_rotations(g.h, sorted(rots))
    if stride == 1:
        babies = {t for u in range(lin.n_shards) for t in bp.baby_amounts(u) if t != 0}
        giants = {gg for (_, gg) in bp.baby if gg != 0}
        assert rots == babies | giants
        assert H.he_conv_keyswitches(conv) == bp.n_rotations()
    return conv


@pytest.mark.parametrize("c,co,m,k,pad,gk", [(8, 8, 28, 3, 1, 1),    # 4 image shards of 2 channels
                                              (16, 24, 16, 3, 1, 1),  # 2 image shards of 8 channels
                                              (16, 24, 16, 3, 1, 4),  # the same, giant stride 4 blocks
                                              (2, 2, 16, 3, 1, 1),    # one shard, 4 copies
                                              (2, 2, 16, 3, 1, 2),    # the same, giant stride 2 blocks
                                              (4, 2, 16, 5, 2, 1),    # one shard, 2 copies, 5x5
                                              (2, 2, 56, 3, 1, 1)])   # channel shards: no giant step
def test_bsgs_conv_bit_exact(mid, c, co, m, k, pad, gk):
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = mid
    level = 3
    rng = np.random.default_rng(c * 7 + m)
    x = rng.uniform(0, 1, (c, m, m))
    W = rng.uniform(-1, 1, (co, c, k, k))
    b = rng.uniform(-1, 1, co)
    lin = Ly.image_layout(c, m, o.N)
    plan = Ly.conv_plan(lin, W, b, pad)
    bp = Ly.conv_plan_bsgs(plan, gk)
    slots = Ly.pack(lin, x)
    cts = [o.encrypt(slots[u], level, nonce=900 + u) for u in range(lin.n_shards)]
    pts = Ly.bsgs_plaintexts(bp, o.n, float(o.q[level]))
    bias_pts = {v: encode(plan.bias[v], o.n, o.pr.scale) for v in range(plan.lout.n_shards)}
    ref_rot = Ly.conv_he_bsgs(o, bp, cts, pts, bias_pts, raised=False)
    ref_raised = Ly.conv_he_bsgs(o, bp, cts, pts, bias_pts, raised=True)

    conv = _create(H, g, o, lin, W, b, level, pad, bp)
    u, v, a, d = H.he_conv_export_plan(conv, o.N, with_diag=True)
    order = _plan_order(bp, o.N)
    assert [(int(vv), int(uu), int(aa)) for uu, vv, aa in zip(u, v, a)] == order
    for i, (vv, uu, aa) in enumerate(order):
        assert np.array_equal(d[i], plan.terms[vv][(uu, aa)])
    H.he_conv_import_plaintexts(conv, np.stack([pts[(uu, vv, aa)] for (vv, uu, aa) in order]),
                                np.stack([bias_pts[vv] for vv in range(plan.lout.n_shards)]))
    ins = [g.upload(ct) for ct in cts]
    runs = [(H.HE_PLAIN, "LDG", ref_rot), (H.HE_BATCHED, "LDG", ref_rot)]
    runs += [(H.HE_FUSED, f, ref_raised) for f in FORMS + ("AUTO",)]
    for mode, form, ref in runs:
        H.he_ctx_set_option(g.h, H.HE_OPT_KEY_STREAM, getattr(H, "HE_KEY_STREAM_" + form))
        outs = [g.ct(level - 1) for _ in range(plan.lout.n_shards)]
        H.he_conv_run(g.h, conv, ins, outs, mode)
        H.he_ctx_check(g.h)
        for oc, rc in zip(outs, ref):
            assert H.he_ct_level(oc) == rc.level and H.he_ct_scale(oc) == rc.scale
            assert_ct_equal(g.download(oc), rc)
    H.he_ctx_set_option(g.h, H.HE_OPT_KEY_STREAM, H.HE_KEY_STREAM_AUTO)
    # and it decrypts to the FP64 convolution
    img = Ly.unpack(plan.lout, np.stack([o.decrypt(ct) for ct in ref_raised]))
    want = torch.nn.functional.conv2d(torch.tensor(x)[None], torch.tensor(W), padding=pad)[0].numpy() \
        + b[:, None, None]
    assert np.abs(img - want).max() <= 2.0 ** -20 * (want.max() - want.min())
    H.he_conv_destroy(conv)


def test_bsgs_mixed_level_batch_bit_exact(mid):
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = mid
    c, co, m, k, pad, top = 4, 4, 32, 3, 1, 5
    rng = np.random.default_rng(31)
    W = rng.uniform(-1, 1, (co, c, k, k))
    b = rng.uniform(-1, 1, co)
    lin = Ly.image_layout(c, m, o.N)
    plan = Ly.conv_plan(lin, W, b, pad)
    bp = Ly.conv_plan_bsgs(plan)
    assert lin.n_shards == 2 and any(gg != 0 for (_, gg) in bp.baby)
    S_pt = float(o.q[top])
    pts = Ly.bsgs_plaintexts(bp, o.n, S_pt)
    order = _plan_order(bp, o.N)
    conv = _create(H, g, o, lin, W, b, top, pad, bp)
    H.he_conv_import_plaintexts(conv, np.stack([pts[(uu, vv, aa)] for (vv, uu, aa) in order]), None)
    levels = [5, 3, 4]
    refs_f, refs_p, ins = [], [], []
    for i, lv in enumerate(levels):
        x = rng.uniform(0, 1, (c, m, m))
        ci = [o.encrypt(Ly.pack(lin, x)[u], lv, nonce=950 + 10 * i + u) for u in range(lin.n_shards)]
        out_scale = o.pr.scale * S_pt / float(o.q[lv])
        bias = {v: encode(plan.bias[v], o.n, out_scale) for v in range(plan.lout.n_shards)}
        H.he_conv_import_bias(conv, lv, out_scale, np.stack([bias[v] for v in range(plan.lout.n_shards)]))
        refs_f.append(Ly.conv_he_bsgs(o, bp, ci, pts, bias, pt_scale=S_pt, raised=True))
        refs_p.append(Ly.conv_he_bsgs(o, bp, ci, pts, bias, pt_scale=S_pt, raised=False))
        ins += [g.upload(ct) for ct in ci]
    runs = [(H.HE_FUSED, f, refs_f) for f in ("AUTO", "LDG", "TMA", "SPLIT", "SPLITM", "PK")]
    runs += [(H.HE_PLAIN, "AUTO", refs_p), (H.HE_BATCHED, "AUTO", refs_p)]
    no = plan.lout.n_shards
    for mode, form, refs in runs:
        H.he_ctx_set_option(g.h, H.HE_OPT_KEY_STREAM, getattr(H, "HE_KEY_STREAM_" + form))
        outs = [g.ct(top - 1) for _ in range(len(levels) * no)]
        H.he_conv_run_batch(g.h, conv, ins, outs, len(levels), mode)
        H.he_ctx_check(g.h)
        for i, lv in enumerate(levels):
            for v in range(no):
                oc, rc = outs[i * no + v], refs[i][v]
                assert H.he_ct_level(oc) == lv - 1 and H.he_ct_scale(oc) == rc.scale
                assert_ct_equal(g.download(oc), rc)
    H.he_ctx_set_option(g.h, H.HE_OPT_KEY_STREAM, H.HE_KEY_STREAM_AUTO)
    H.he_conv_destroy(conv)


def test_bsgs_giant_stride_choice_and_checks(mid):
    from paper_2306_09189_gb300 import hegpu as H
    o, g = mid
    rng = np.random.default_rng(5)
    W = rng.uniform(-1, 1, (2, 2, 3, 3))
    lay = H.he_layout_image(2, 16, o.N)          # one shard of 8 blocks (4 copies)
    conv = H.he_conv_create_bsgs(g.h, lay, W, None, 1, 1, 3, o.pr.scale, 0)
    k = H.he_conv_bsgs_giant(conv)
    assert k in (1, 2, 4, 8) and "bsgs giant stride" in H.he_ctx_tuning_log(g.h)
    H.he_conv_destroy(conv)
    for bad in (3, 16):                          # not a power of two / more than the 8 blocks
        with pytest.raises(H.HEError) as e:
            H.he_conv_create_bsgs(g.h, lay, W, None, 1, 1, 3, o.pr.scale, bad)
        assert e.value.code == H.HE_EINVAL
    conv = H.he_conv_create(g.h, lay, W, None, 1, 1, 3, o.pr.scale)
    assert H.he_conv_bsgs_giant(conv) == 0
    H.he_conv_destroy(conv)


def test_bsgs_stride2_conv_decrypts_to_torch(mid):
    from paper_2306_09189_gb300 import hegpu as H
    o, g = mid
    rng = np.random.default_rng(12)
    c, co, m, level = 4, 4, 32, 5
    x = rng.uniform(0, 1, (c, m, m))
    W = rng.normal(0, 0.1, (co, c, 3, 3))
    lin = Ly.image_layout(c, m, o.N)
    bp = Ly.conv_plan_bsgs(Ly.conv_plan(lin, W, None, 1))
    slots = Ly.pack(lin, x)
    ins = []
    for u in range(lin.n_shards):
        ct = g.ct(level)
        H.he_encrypt(g.h, slots[u], level, o.pr.scale, 60 + u, ct)
        ins.append(ct)
    conv = _create(H, g, o, lin, W, None, level, 1, bp, stride=2)
    lout = H.he_conv_out_layout(conv)
    chan, row0 = lout.tables()
    ol = Ly.Layout(lout.c, lout.m, lout.M, lout.N, lout.B, chan.astype(np.int64), row0.astype(np.int64))
    want = torch.nn.functional.conv2d(torch.tensor(x)[None], torch.tensor(W), stride=2, padding=1)[0].numpy()
    for mode in (H.HE_BATCHED, H.HE_FUSED):
        outs = [g.ct(level - 3) for _ in range(lout.n_shards)]
        H.he_conv_run(g.h, conv, ins, outs, mode)
        H.he_ctx_check(g.h)
        img = Ly.unpack(ol, np.stack([H.he_decrypt(g.h, oc, o.N) for oc in outs]))
        assert np.abs(img - want).max() <= 2.0 ** -20 * (want.max() - want.min())
    H.he_conv_destroy(conv)
