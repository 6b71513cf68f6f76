"""Stride 2 and the residual path on the GPU, word by word against the oracle.

Stride 2 (Sec. 4.1 "Strided convolutions"; the downsampling of Sec. 4.2 with weights (1,0,0,0),
Eqs. 10-11): the library's stride-2 convolution is the unstrided convolution followed by its
select stage.  The oracle runs the same two programs (conv_he / conv_he_raised, then pool_he /
pool_he_raised with pool_plan(select_top_left=True)); with the oracle's integer plaintexts
imported into both stages every output limb must agree, in every execution mode, for the
diagonal form on image shards and for the factored channel-shard form of the stem.

Residual and level alignment (the ResNet basic block of Sec. 5 adds its input to the second
convolution's output): he_add / he_sub of ciphertexts at different levels and he_ct_drop_level
must equal the oracle's add_ct / sub_ct after drop_to, limb for limb.
"""
import numpy as np
import pytest
import torch

from oracle import layers as Ly
from oracle.ckks import Context
from oracle.encode import encode
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


def _select_masks(o, pp, level):
    """The select stage's integer masks: horizontal at q_level, vertical at q_{level-1}."""
    ns = pp.lin.n_shards
    hm = np.stack([[encode(mk[u], o.n, float(o.q[level])) for u in range(ns)] for _, mk in pp.h_terms])
    vm = np.stack([[encode(mk[u], o.n, float(o.q[level - 1])) for u in range(ns)] for _, mk in pp.v_terms])
    return hm, vm


def _import_select(H, conv, pp, hm, vm):
    pool = H.he_conv_select_pool(conv)
    nh, nv = H.he_pool_n_masks(pool)
    assert nh == len(pp.h_terms) and nv == len(pp.v_terms)
    H.he_pool_import_plaintexts(pool, hm, vm)
    chan, row0 = H.he_conv_out_layout(conv).tables()
    assert np.array_equal(chan, pp.lout.chan) and np.array_equal(row0, pp.lout.row0)


def _run_modes(H, g, conv, ins, n_out, out_level, runs):
    from tests._hegpu_util import assert_ct_equal
    for mode, ks, refs in runs:
        H.he_ctx_set_option(g.h, H.HE_OPT_KEY_STREAM, ks)
        outs = [g.ct(out_level) for _ in range(n_out)]
        H.he_conv_run(g.h, conv, ins, outs, mode)
        H.he_ctx_check(g.h)
        for oc, rc in zip(outs, refs):
            assert H.he_ct_level(oc) == rc.level and H.he_ct_scale(oc) == rc.scale
            assert_ct_equal(g.download(oc), rc)
    H.he_ctx_set_option(g.h, H.HE_OPT_KEY_STREAM, H.HE_KEY_STREAM_AUTO)


@pytest.mark.parametrize("c,co,m,k,pad", [(3, 4, 32, 7, 3),      # image shards (2), 7x7 like a stem
                                           (4, 4, 16, 3, 1),      # one shard with duplication
                                           (2, 3, 32, 3, 1)])     # one full shard
def test_stride2_conv_bit_exact(mid, c, co, m, k, pad):
    from paper_2306_09189_gb300 import hegpu as H
    o, g = mid
    level = 5
    rng = np.random.default_rng(100 + c * 7 + m + k)
    x = rng.uniform(0, 1, (c, m, m))
    W = rng.normal(0, 0.05, (co, c, k, k)) if k == 7 else rng.uniform(-1, 1, (co, c, k, k))
    b = rng.uniform(-1, 1, co)
    lin = Ly.image_layout(c, m, o.N)
    plan = Ly.conv_plan(lin, W, b, pad)
    pts = Ly.conv_plaintexts(plan, o.n, float(o.q[level]))
    bias = {v: encode(plan.bias[v], o.n, o.pr.scale) for v in range(plan.lout.n_shards)}
    cts = [o.encrypt(s, level, nonce=1200 + u) for u, s in enumerate(Ly.pack(lin, x))]
    pp = Ly.pool_plan(plan.lout, select_top_left=True)
    hm, vm = _select_masks(o, pp, level - 1)
    ref_p = Ly.pool_he(o, pp, Ly.conv_he(o, plan, cts, pts, bias))
    ref_r = Ly.pool_he_raised(o, pp, Ly.conv_he_raised(o, plan, cts, pts, bias), list(hm), list(vm))

    conv = H.he_conv_create(g.h, H.he_layout_image(c, m, o.N), W, b, 2, pad, level, o.pr.scale)
    H.he_keygen_rotations(g.h, H.he_conv_rotations(conv))
    assert H.he_conv_out_level(conv) == level - 3 == ref_p[0].level
    keys = [(vv, uu, aa) for vv in sorted(plan.terms) for (uu, aa) in sorted(plan.terms[vv])]
    H.he_conv_import_plaintexts(conv, np.stack([pts[(uu, vv, aa)] for (vv, uu, aa) in keys]),
                                np.stack([bias[v] for v in range(plan.lout.n_shards)]))
    _import_select(H, conv, pp, hm, vm)
    ins = [g.upload(ct) for ct in cts]
    runs = [(H.HE_PLAIN, H.HE_KEY_STREAM_AUTO, ref_p), (H.HE_BATCHED, H.HE_KEY_STREAM_AUTO, ref_p),
            (H.HE_FUSED, H.HE_KEY_STREAM_AUTO, ref_r), (H.HE_FUSED, H.HE_KEY_STREAM_LDG, ref_r),
            (H.HE_FUSED, H.HE_KEY_STREAM_TMA, ref_r), (H.HE_FUSED, H.HE_KEY_STREAM_LDG1, ref_r),
            (H.HE_FUSED, H.HE_KEY_STREAM_SPLIT, ref_r), (H.HE_FUSED, H.HE_KEY_STREAM_PK3, ref_r)]
    _run_modes(H, g, conv, ins, len(ref_p), level - 3, runs)
    H.he_conv_destroy(conv)
    # and both oracle programs are conv2d(stride=2)
    want = (torch.nn.functional.conv2d(torch.tensor(x)[None], torch.tensor(W), stride=2, padding=pad)[0].numpy()
            + b[:, None, None])
    for ref in (ref_p, ref_r):
        img = Ly.unpack(pp.lout, np.stack([o.decrypt(ct) for ct in ref]))
        assert img.shape == want.shape
        assert np.abs(img - want).max() <= 2.0 ** -20 * (want.max() - want.min())


def test_factored_stride2_stem_bit_exact(mid):
    """The stem's form in small: channel shards, 7x7 stride 2, factored (masks, then integer
    scalars), then the select stage."""
    from paper_2306_09189_gb300 import hegpu as H
    o, g = mid
    c, co, m, level = 3, 4, 64, 5
    rng = np.random.default_rng(23)
    x = rng.uniform(0, 1, (c, m, m))
    W = rng.normal(0, 0.05, (co, c, 7, 7))
    lin = Ly.image_layout(c, m, o.N)
    assert lin.n_shards == 2 * c                       # two channel shards per channel
    plan = Ly.conv_plan_factored(lin, W, None, 3)
    mpts = Ly.mask_plaintexts(plan, o.n, float(o.q[level]))
    bias = {v: encode(plan.bias[v], o.n, o.pr.scale) for v in range(plan.lout.n_shards)}
    cts = [o.encrypt(s, level, nonce=1300 + u) for u, s in enumerate(Ly.pack(lin, x))]
    pp = Ly.pool_plan(plan.lout, select_top_left=True)
    hm, vm = _select_masks(o, pp, level - 2)
    ref_p = Ly.pool_he(o, pp, Ly.conv_he_factored(o, plan, cts, mpts, bias, raised=False))
    ref_r = Ly.pool_he_raised(o, pp, Ly.conv_he_factored(o, plan, cts, mpts, bias, raised=True),
                              list(hm), list(vm))

    conv = H.he_conv_create_factored(g.h, H.he_layout_image(c, m, o.N), W, None, 2, 3, level, o.pr.scale)
    H.he_keygen_rotations(g.h, H.he_conv_rotations(conv))
    assert H.he_conv_out_level(conv) == level - 4 == ref_p[0].level
    H.he_conv_import_plaintexts(conv, np.stack([mpts[key] for key in sorted(plan.masks)]),
                                np.stack([bias[v] for v in range(plan.lout.n_shards)]))
    _import_select(H, conv, pp, hm, vm)
    ins = [g.upload(ct) for ct in cts]
    runs = [(H.HE_PLAIN, H.HE_KEY_STREAM_AUTO, ref_p), (H.HE_BATCHED, H.HE_KEY_STREAM_AUTO, ref_p),
            (H.HE_FUSED, H.HE_KEY_STREAM_AUTO, ref_r), (H.HE_FUSED, H.HE_KEY_STREAM_LDG, ref_r),
            (H.HE_FUSED, H.HE_KEY_STREAM_SPLIT, ref_r)]
    _run_modes(H, g, conv, ins, len(ref_p), level - 4, runs)
    H.he_conv_destroy(conv)
    want = torch.nn.functional.conv2d(torch.tensor(x)[None], torch.tensor(W), stride=2, padding=3)[0].numpy()
    img = Ly.unpack(pp.lout, np.stack([o.decrypt(ct) for ct in ref_r]))
    assert np.abs(img - want).max() <= 2.0 ** -20 * (want.max() - want.min())


def test_stride2_select_pool_is_refused_for_stride_1(mid):
    from paper_2306_09189_gb300 import hegpu as H
    o, g = mid
    conv = H.he_conv_create(g.h, H.he_layout_image(2, 16, o.N), np.ones((2, 2, 3, 3)), None, 1, 1, 3, o.pr.scale)
    try:
        with pytest.raises(H.HEError) as e:
            H.he_conv_select_pool(conv)
        assert e.value.code == H.HE_EINVAL
    finally:
        H.he_conv_destroy(conv)


@pytest.mark.parametrize("la,lb", [(5, 5), (5, 3), (4, 1), (3, 0)])
def test_add_sub_drop_level_bit_exact(mid, la, lb):
    """acc (level lb) +/- b (level la >= lb) reads b's limbs q_0..q_lb: b dropped to acc's level."""
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = mid
    rng = np.random.default_rng(10 * la + lb)
    a = o.encrypt(rng.uniform(-1, 1, o.N), la, nonce=1400 + la)
    b = o.encrypt(rng.uniform(-1, 1, o.N), lb, nonce=1450 + lb)
    for fn, ofn in ((H.he_add, o.add_ct), (H.he_sub, o.sub_ct)):
        acc = g.upload(b)
        fn(g.h, acc, g.upload(a))
        ref = ofn(b, o.drop_to(a, lb))
        assert H.he_ct_level(acc) == lb and H.he_ct_scale(acc) == b.scale
        assert_ct_equal(g.download(acc), ref)
    # dropping limbs is exact: the top limbs are cut, the rest untouched
    d = g.upload(a)
    H.he_ct_drop_level(d, lb)
    assert H.he_ct_level(d) == lb and H.he_ct_scale(d) == a.scale
    assert_ct_equal(g.download(d), o.drop_to(a, lb))
    if la > lb:
        # the accumulator never takes a lower-level addend: that would need limbs it lacks
        hi = g.upload(a)
        for fn in (H.he_add, H.he_sub):
            with pytest.raises(H.HEError) as e:
                fn(g.h, hi, g.upload(b))
            assert e.value.code == H.HE_ELEVEL
        assert_ct_equal(g.download(hi), a)
