"""Paterson-Stockmeyer Chebyshev evaluation on the GPU, bit for bit against the oracle.

Degrees 16, 27 and 59 (the paper's GELU), several ciphertexts at two input levels in one call:
every output equals the oracle's cheb_ps_he on that ciphertext, at the paper's depth."""
import numpy as np
import pytest

from oracle import layers as Ly
from oracle.params import Params
from oracle.ckks import Context

pytestmark = pytest.mark.gpu

DEEP = Params(log_n=12, n_q=10, n_p=3, dnum=4, q0_bits=50, q_bits=40, p_bits=50, scale=2.0 ** 40, seed=9)


@pytest.fixture(scope="module")
def deep():
    from tests._hegpu_util import GpuCtx
    o = Context(DEEP)
    o.gen_relin_key()
    g = GpuCtx(DEEP)
    from paper_2306_09189_gb300 import hegpu as H
    H.he_keygen_relin(g.h)
    yield o, g
    g.close()


@pytest.mark.parametrize("deg,levels", [(16, [9, 8, 9]), (27, [9, 7]), (59, [9, 9])])
def test_ps_bit_exact(deep, deg, levels):
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = deep
    c = Ly.cheb_nodes_coeffs(Ly.gelu, deg, -8, 8)
    rng = np.random.default_rng(deg)
    cts = [o.encrypt(rng.uniform(-1, 1, o.N), lv, nonce=3000 + 10 * deg + i) for i, lv in enumerate(levels)]
    targets = [o.pr.scale, o.pr.scale * 0.75, o.pr.scale][:len(cts)]
    refs = [Ly.cheb_ps_he(o, ct, c, target_scale=t) for ct, t in zip(cts, targets)]
    gcs = [g.upload(ct) for ct in cts]
    H.he_poly_eval_ps_many(g.h, gcs, c, targets)
    H.he_ctx_check(g.h)
    for gc, ref in zip(gcs, refs):
        assert H.he_ct_level(gc) == ref.level and H.he_ct_scale(gc) == ref.scale
        assert_ct_equal(g.download(gc), ref)
    # the single-ciphertext entry gives the same bits
    one = g.upload(cts[0])
    H.he_poly_eval_ps(g.h, one, c, targets[0])
    assert_ct_equal(g.download(one), refs[0])
    # and the result is the polynomial
    z = o.decrypt(cts[0])
    want = Ly.cheb_eval(c, 8 * z, -8, 8)
    got = H.he_decrypt(g.h, gcs[0], o.N)
    assert np.abs(got - want).max() <= 2.0 ** -20 * (want.max() - want.min())


def test_ps_minimax_gelu_degree_59(deep):
    # the paper's degree-59 GELU on [-16, 16] in its minimax form (the oracle's Remez routine):
    # bit for bit against the oracle's evaluator, and within the minimax error of GELU itself
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = deep
    c, E = Ly.minimax_coeffs(Ly.gelu, 59, -16, 16)
    z = np.random.default_rng(59).uniform(-1, 1, o.N)
    ct = o.encrypt(z, 9, nonce=4059)
    ref = Ly.cheb_ps_he(o, ct, c, target_scale=o.pr.scale)
    gc = g.upload(ct)
    H.he_poly_eval_ps(g.h, gc, c, o.pr.scale)
    H.he_ctx_check(g.h)
    assert H.he_ct_level(gc) == ref.level == 9 - 6
    assert_ct_equal(g.download(gc), ref)
    got = H.he_decrypt(g.h, gc, o.N)
    want = np.array([Ly.gelu(16 * v) for v in z])
    assert np.abs(got - want).max() <= E + 2.0 ** -20 * (want.max() - want.min())


def test_ps_batches_independent_products(deep):
    # degree 16 (k = 4, giants 4, 8, 16) has eight products at five operand levels: T_2 | T_3, T_4
    # | T_8 | T_16 with the product inside the T_8 quotient | the two products of the T_8 and T_4
    # quotients of the remainder.  The scheduler issues one batched relinearisation per level
    # (five inner-product launches for one ciphertext), and the bits stay the oracle's.
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = deep
    c = Ly.cheb_nodes_coeffs(Ly.gelu, 16, -8, 8)
    ct = o.encrypt(np.random.default_rng(16).uniform(-1, 1, o.N), 9, nonce=4016)
    ref = Ly.cheb_ps_he(o, ct, c, target_scale=o.pr.scale)
    gc = g.upload(ct)
    H.he_poly_eval_ps(g.h, gc, c, o.pr.scale)          # warm (temporaries, scratch)
    gc = g.upload(ct)
    H.he_trace_start("ip")
    H.he_poly_eval_ps(g.h, gc, c, o.pr.scale)
    tr = H.he_trace_stop()
    H.he_ctx_check(g.h)
    assert tr["launches"] == 5
    assert H.he_ct_level(gc) == ref.level == 9 - 5
    assert_ct_equal(g.download(gc), ref)
