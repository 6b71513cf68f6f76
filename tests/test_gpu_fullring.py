"""Full-ring parity of the measured layers against the oracle, word by word.

The benchmarked layers run at n = 2^16 with 20 ciphertext primes and 5 special primes
(alpha = K = 5, four key-switching digits at the top level), where every other bit-exact test
uses rings of 2^12..2^13 with at most two special primes.  Here the GPU output limbs of

  * the CIFAR-shaped layer (16x32x32, conv3x3 16->16 with folded BatchNorm, Sec. 4.1 "With a
    Single Shard", Eqs. 1-5 with duplication; 143 hoisted rotations) in the fused raised-basis
    form the benchmark times (the autotuned pre-keyed kernel), in the register-fed form, and in
    the per-rotation plain and batched modes, followed by the degree-16 Chebyshev GELU by
    Paterson-Stockmeyer (Appendix, Chebyshev basis);
  * one convolution of the ResNet basic block (64x56x56 in 8 image shards, Eq. 6), planned at
    the top level and applied to an image at level 8 through the mixed-level batch entry in the
    fused form the benchmark uses (output shard 0, computed by the oracle for that shard alone;
    the per-rotation modes are compared at the full ring on the CIFAR layer)

must equal the oracle's limbs exactly, on the same seeded ciphertexts and the oracle's integer
plaintexts.  The oracle side costs a few minutes of host time (rotation keys and hoisted
rotations at the full ring).
"""
import numpy as np
import pytest

from oracle import layers as Ly
from oracle.ckks import Context
from oracle.encode import encode
from oracle.params import C20
import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def c20():
    from tests._hegpu_util import GpuCtx
    o = Context(C20)
    g = GpuCtx(C20)
    yield o, g
    g.close()


def _import_plan(H, conv, plan, pts_of, bias_rows):
    """Import integer plaintexts in the library's term order (v, then (u, a) ascending)."""
    u, v, a, _ = H.he_conv_export_plan(conv)
    order = list(zip(v.tolist(), u.tolist(), a.tolist()))
    want = [(vv, uu, aa) for vv in sorted(plan.terms) for (uu, aa) in sorted(plan.terms[vv])]
    assert order == want
    H.he_conv_import_plaintexts(conv, np.stack([pts_of(uu, vv, aa) for (vv, uu, aa) in order]),
                                None if bias_rows is None else np.stack(bias_rows))


def test_cifar_layer_full_ring_limbs_equal_oracle(c20):
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = c20
    level, scale = 19, C20.scale
    wl = workloads.cifar_conv_bn(0)
    lin = Ly.image_layout(16, 32, o.N)
    plan = Ly.conv_plan(lin, wl.W, wl.bias, 1)
    assert lin.n_shards == 1 and plan.n_rotations() == 143
    pts = Ly.conv_plaintexts(plan, o.n, float(o.q[level]))
    bias = [encode(plan.bias[0], o.n, scale)]
    ct = o.encrypt(Ly.pack(lin, wl.x)[0], level, nonce=1)

    conv = H.he_conv_create(g.h, H.he_layout_image(16, 32, o.N), wl.W, wl.bias, 1, 1, level, scale)
    H.he_keygen_rotations(g.h, H.he_conv_rotations(conv))
    _import_plan(H, conv, plan, lambda u, v, a: pts[(u, v, a)], bias)
    x = g.upload(ct)

    # the fused raised-basis form: autotuned (the benchmark's choice), pre-keyed at three
    # blocks per SM and with one coefficient per thread, and the register-fed kernel
    ref_f = Ly.conv_he_raised(o, plan, [ct], pts, {0: bias[0]})[0]
    fused = None
    for ks in (H.HE_KEY_STREAM_AUTO, H.HE_KEY_STREAM_PK3, H.HE_KEY_STREAM_PK1, H.HE_KEY_STREAM_PKT,
               H.HE_KEY_STREAM_PK3L, H.HE_KEY_STREAM_LDG):
        H.he_ctx_set_option(g.h, H.HE_OPT_KEY_STREAM, ks)
        y = g.ct(level - 1)
        H.he_conv_run(g.h, conv, [x], [y], H.HE_FUSED)
        H.he_ctx_check(g.h)
        assert H.he_ct_level(y) == ref_f.level and H.he_ct_scale(y) == ref_f.scale
        assert_ct_equal(g.download(y), ref_f)
        if fused is None:
            fused = y
    H.he_ctx_set_option(g.h, H.HE_OPT_KEY_STREAM, H.HE_KEY_STREAM_AUTO)

    # one ModDown per rotation (plain per-ciphertext launches, and batched launches)
    ref_p = Ly.conv_he(o, plan, [ct], pts, {0: bias[0]})[0]
    for mode in (H.HE_PLAIN, H.HE_BATCHED):
        y = g.ct(level - 1)
        H.he_conv_run(g.h, conv, [x], [y], mode)
        assert H.he_ct_scale(y) == ref_p.scale
        assert_ct_equal(g.download(y), ref_p)
    H.he_conv_destroy(conv)

    # the benchmark's activation on the fused output: degree-16 GELU by Paterson-Stockmeyer
    o.gen_relin_key()
    H.he_keygen_relin(g.h)
    cheb = Ly.cheb_nodes_coeffs(Ly.gelu, workloads.GELU_DEGREE, -8, 8)
    ref_a = Ly.cheb_ps_he(o, ref_f, cheb, target_scale=scale)
    H.he_poly_eval_ps(g.h, fused, cheb, scale)
    H.he_ctx_check(g.h)
    assert H.he_ct_level(fused) == ref_a.level == level - 1 - 5
    assert H.he_ct_scale(fused) == ref_a.scale
    assert_ct_equal(g.download(fused), ref_a)
    # and it is the polynomial of the convolution
    import torch
    pre = (torch.nn.functional.conv2d(torch.tensor(wl.x)[None], torch.tensor(wl.W), padding=1)[0].numpy()
           + wl.bias[:, None, None])
    want = Ly.cheb_eval(cheb, 8 * pre, -8, 8)
    got = Ly.unpack(lin, o.decrypt(ref_a)[None])
    assert np.abs(got - want).max() <= 2.0 ** -20 * (want.max() - want.min())


def test_block_conv_at_level_8_limbs_equal_oracle(c20):
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = c20
    top, lv, scale = 19, 8, C20.scale
    x0, (W1, b1), _ = workloads.resnet_block(0)
    lin = Ly.image_layout(64, 56, o.N)
    plan = Ly.conv_plan(lin, W1, b1, 1)
    assert lin.n_shards == 8 and plan.lout.n_shards == 8
    S_pt = float(o.q[top])                            # one plaintext set, planned at the top level
    pts0 = {(u, 0, a): encode(D, o.n, S_pt) for (u, a), D in plan.terms[0].items()}
    out_scale = scale * S_pt / float(o.q[lv])
    bias0 = encode(plan.bias[0], o.n, out_scale)
    cts = [o.encrypt(s, lv, nonce=4000 + u) for u, s in enumerate(Ly.pack(lin, x0))]

    conv = H.he_conv_create(g.h, H.he_layout_image(64, 56, o.N), W1, b1, 1, 1, top, scale)
    H.he_keygen_rotations(g.h, H.he_conv_rotations(conv))
    zero = np.zeros(o.n, dtype=np.int64)              # only output shard 0 is compared
    _import_plan(H, conv, plan, lambda u, v, a: pts0[(u, v, a)] if v == 0 else zero, None)
    H.he_conv_import_bias(conv, lv, out_scale, np.stack([bias0] + [zero] * 7))
    ins = [g.upload(c) for c in cts]

    ref_f = Ly.conv_he_raised(o, plan, cts, pts0, {0: bias0}, pt_scale=S_pt, outputs=[0])[0]
    outs = [g.ct(top - 1) for _ in range(8)]
    H.he_ctx_set_option(g.h, H.HE_OPT_KEY_STREAM, H.HE_KEY_STREAM_AUTO)
    H.he_conv_run_batch(g.h, conv, ins, outs, 1, H.HE_FUSED)
    H.he_ctx_check(g.h)
    assert H.he_ct_level(outs[0]) == lv - 1 and H.he_ct_scale(outs[0]) == ref_f.scale
    assert_ct_equal(g.download(outs[0]), ref_f)

    H.he_conv_destroy(conv)

    import torch
    want = (torch.nn.functional.conv2d(torch.tensor(x0)[None], torch.tensor(W1), padding=1)[0].numpy()
            + b1[:, None, None])
    got = Ly.unpack(plan.lout, np.stack([o.decrypt(ref_f)] + [np.zeros(o.N)] * 7))
    ch = plan.lout.chan[0][plan.lout.chan[0] >= 0]
    ref = want[np.unique(ch)]
    sel = got[np.unique(ch)]
    assert np.abs(sel - ref).max() <= 2.0 ** -20 * (ref.max() - ref.min())
