"""GPU parity: ciphertext limbs from the CUDA path equal the oracle's bit for bit.

Inputs are the oracle's own ciphertexts (imported in coefficient form), keys are generated
on both sides from the same seed, and every comparison is on exported coefficient-form limbs.
Sizes: a mid ring (n = 2^12, 6 primes, 3 digits with a partial last digit at some levels) that
spans several NTT tiles, the TOY ring, and the full 2^16 ring for single operations.
"""
import numpy as np
import pytest

from oracle.params import Params, TOY, C20
from oracle.ckks import Context
from oracle.encode import encode

pytestmark = pytest.mark.gpu

MID = Params(log_n=12, n_q=6, n_p=2, dnum=3, q0_bits=50, q_bits=40, p_bits=50,
             scale=2.0 ** 40, seed=5)


@pytest.fixture(scope="module")
def pair():
    from tests._hegpu_util import GpuCtx
    o = Context(MID)
    g = GpuCtx(MID)
    yield o, g
    g.close()


def _rand_ct(o, level, seed):
    z = np.random.default_rng(seed).uniform(-1, 1, o.N)
    return o.encrypt(z, level, nonce=seed), z


def test_context_primes(pair):
    o, g = pair
    assert [int(x) for x in g.info["q"]] == o.q and [int(x) for x in g.info["p"]] == o.p
    assert g.info["alpha"] == o.alpha


def test_import_export_roundtrip(pair):
    o, g = pair
    ct, _ = _rand_ct(o, 5, 1)
    from tests._hegpu_util import assert_ct_equal
    assert_ct_equal(g.download(g.upload(ct)), ct)


@pytest.mark.parametrize("level", [0, 3, 5])
def test_encrypt_coeffs_bit_exact(pair, level):
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = pair
    m = encode(np.random.default_rng(level).uniform(-1, 1, o.N), o.n, 2.0 ** 40)
    ref = o.encrypt_coeffs(m, level, 2.0 ** 40, 77 + level)
    c = g.ct(level)
    H.he_encrypt_coeffs(g.h, m, level, 2.0 ** 40, 77 + level, c)
    assert_ct_equal(g.download(c), ref)


def test_rotation_and_relin_keys_bit_exact(pair):
    from paper_2306_09189_gb300 import hegpu as H
    o, g = pair
    for r in (1, 77):
        gel = o.gen_rotation_key(r)
        H.he_keygen_rotations(g.h, [r])
        ref = o.export_key(gel)
        got = H.he_key_export(g.h, r, ref.shape)
        assert np.array_equal(got, ref)
    o.gen_relin_key()
    H.he_keygen_relin(g.h)
    ref = o.export_key(0)
    assert np.array_equal(H.he_key_export(g.h, H.HE_RELIN_KEY, ref.shape), ref)


@pytest.mark.parametrize("level,r", [(5, 1), (5, 77), (4, 3), (3, -5), (1, 1000), (0, 1)])
def test_rotate_bit_exact(pair, level, r):
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = pair
    ct, z = _rand_ct(o, level, 10 + level)
    o.gen_rotation_key(r)
    H.he_keygen_rotations(g.h, [r])
    out = g.ct(level)
    H.he_rotate(g.h, g.upload(ct), r, out)
    assert_ct_equal(g.download(out), o.rotate(ct, r))


def test_rotate_hoisted_bit_exact(pair):
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = pair
    rots = [0, 1, 5, 64, -3, 2047]
    for level in (5, 4):
        ct, z = _rand_ct(o, level, 30 + level)
        for r in rots:
            o.gen_rotation_key(r)
        H.he_keygen_rotations(g.h, rots)
        outs = [g.ct(level) for _ in rots]
        H.he_rotate_hoisted(g.h, g.upload(ct), rots, outs)
        D = o.hoist(ct)
        for r, c in zip(rots, outs):
            assert_ct_equal(g.download(c), o.rotate_hoisted(ct, D, r))


@pytest.mark.parametrize("level", [1, 3, 5])
def test_rescale_bit_exact(pair, level):
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = pair
    ct, _ = _rand_ct(o, level, 50 + level)
    c = g.upload(ct)
    H.he_rescale(g.h, c)
    ref = o.rescale(ct)
    assert H.he_ct_level(c) == level - 1 and H.he_ct_scale(c) == ref.scale
    assert_ct_equal(g.download(c), ref)


def test_mul_pt_acc_bit_exact(pair):
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = pair
    level = 4
    cts = [_rand_ct(o, level, 60 + i)[0] for i in range(3)]
    rng = np.random.default_rng(9)
    pts = [encode(rng.uniform(-1, 1, o.N), o.n, float(o.q[level])) for _ in range(3)]
    acc = g.ct(level)
    H.he_ct_zero(acc, level, 0.0)
    hp = []
    for ct, m in zip(cts, pts):
        p = H.he_pt_import_coeffs(g.h, m, level, float(o.q[level]))
        hp.append(p)
        H.he_mul_pt_acc(g.h, acc, g.upload(ct), p)
    ref = o.mul_plain(cts[0], pts[0], float(o.q[level]))
    for ct, m in zip(cts[1:], pts[1:]):
        ref = o.add_ct(ref, o.mul_plain(ct, m, float(o.q[level])))
    assert_ct_equal(g.download(acc), ref)
    H.he_rescale(g.h, acc)
    assert_ct_equal(g.download(acc), o.rescale(ref))
    for p in hp:
        H.he_pt_free(p)


def test_mul_relin_bit_exact(pair):
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = pair
    o.gen_relin_key()
    H.he_keygen_relin(g.h)
    for level in (5, 3):
        a, _ = _rand_ct(o, level, 70 + level)
        b, _ = _rand_ct(o, level, 80 + level)
        out = g.ct(level)
        H.he_mul_relin(g.h, g.upload(a), g.upload(b), out)
        ref = o.mul_relin(a, b)
        assert H.he_ct_scale(out) == ref.scale
        assert_ct_equal(g.download(out), ref)


def test_scalar_ops_bit_exact(pair):
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = pair
    ct, _ = _rand_ct(o, 5, 90)
    c = g.upload(ct)
    K = float(2 ** 70 + 2 ** 20)      # exact in a double
    H.he_mul_int(g.h, c, -K)
    H.he_add_const_int(g.h, c, 123456789.0)
    ref = o.add_const_int(o.mul_int(ct, -int(K)), 123456789)
    assert_ct_equal(g.download(c), ref)


def test_decrypt_matches_oracle(pair):
    from paper_2306_09189_gb300 import hegpu as H
    o, g = pair
    for level in (0, 5):
        ct, z = _rand_ct(o, level, 95 + level)
        got = H.he_decrypt(g.h, g.upload(ct), o.N)
        assert np.abs(got - o.decrypt(ct)).max() < 1e-9 and np.abs(got - z).max() < 1e-7


def test_encrypt_decrypt_on_device(pair):
    from paper_2306_09189_gb300 import hegpu as H
    o, g = pair
    z = np.random.default_rng(3).uniform(-2, 2, o.N)
    c = g.ct(4)
    H.he_encrypt(g.h, z, 4, 2.0 ** 40, 5, c)
    assert np.abs(H.he_decrypt(g.h, c, o.N) - z).max() < 1e-7


def test_library_encoder_within_one_of_oracle(pair):
    # the two FP64 encoders (independent FFTs) may round a coefficient differently by one
    from paper_2306_09189_gb300 import hegpu as H
    o, g = pair
    z = np.random.default_rng(4).uniform(-1, 1, o.N)
    p = H.he_pt_encode(g.h, z, 2, 2.0 ** 40)
    acc = g.ct(2)
    ct, w = _rand_ct(o, 2, 6)
    H.he_ct_zero(acc, 2, 0.0)
    H.he_mul_pt_acc(g.h, acc, g.upload(ct), p)
    H.he_rescale(g.h, acc)
    got = H.he_decrypt(g.h, acc, o.N)
    assert np.abs(got - z * w).max() < 1e-6
    H.he_pt_free(p)


# --------------------------------------------------------------------------- full ring
@pytest.fixture(scope="module")
def pair20():
    from tests._hegpu_util import GpuCtx
    o = Context(C20)
    g = GpuCtx(C20)
    yield o, g
    g.close()


@pytest.mark.parametrize("form", ["onepass", "onepass8", "twopass", "twopass-corrected", "twopass-shuffle"])
@pytest.mark.parametrize("level", [19, 12])
def test_full_ring_rotation_bit_exact(pair20, level, form):
    """At n = 2^16 every NTT form (one launch per limb on a CTA cluster, or two passes with or
    without the per-butterfly correction of the forward transform) gives the oracle's words
    through a key switch (INTT, ModUp, NTT, ModDown) and a rescale."""
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = pair20
    H.he_ctx_set_option(g.h, H.HE_OPT_NTT, {"onepass": H.HE_NTT_ONEPASS, "onepass8": H.HE_NTT_ONEPASS8,
                                            "twopass": H.HE_NTT_TWOPASS,
                                            "twopass-corrected": H.HE_NTT_TWOPASS_CORRECTED,
                                            "twopass-shuffle": H.HE_NTT_TWOPASS_SHUFFLE}[form])
    try:
        ct, z = _rand_ct(o, level, 200 + level)
        o.gen_rotation_key(33)
        H.he_keygen_rotations(g.h, [33])
        out = g.ct(level)
        c = g.upload(ct)
        H.he_rotate(g.h, c, 33, out)
        assert_ct_equal(g.download(out), o.rotate(ct, 33))
        assert np.abs(H.he_decrypt(g.h, out, o.N) - np.roll(z, -33)).max() < 2.0 ** -20
        H.he_rescale(g.h, c)
        assert_ct_equal(g.download(c), o.rescale(ct))
    finally:
        H.he_ctx_set_option(g.h, H.HE_OPT_NTT, H.HE_NTT_TWOPASS)


def test_full_ring_ntt_forms_give_the_same_words(pair20):
    """Forward in one form, inverse in the other, is the identity on random residues (so the two
    forward transforms agree word for word), and encryption matches the oracle in both forms."""
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = pair20
    level = 19
    rng = np.random.default_rng(1919)
    q = np.array([int(v) for v in o.q[:level + 1]], dtype=np.uint64)
    words = (rng.integers(0, 2 ** 63, (2, level + 1, o.n), dtype=np.uint64) % q[None, :, None])
    one, two, eight, corr = H.HE_NTT_ONEPASS, H.HE_NTT_TWOPASS, H.HE_NTT_ONEPASS8, H.HE_NTT_TWOPASS_CORRECTED
    shf = H.HE_NTT_TWOPASS_SHUFFLE
    try:
        for fwd, inv in ((one, two), (two, one), (one, one), (eight, two), (two, eight), (two, corr), (corr, two),
                         (shf, two), (two, shf), (shf, shf)):
            x = g.ct(level)
            H.he_ctx_set_option(g.h, H.HE_OPT_NTT, fwd)
            H.he_ct_import_coeffs(x, words, level, o.pr.scale)
            H.he_ctx_set_option(g.h, H.HE_OPT_NTT, inv)
            assert np.array_equal(g.download(x), words)
        m = rng.integers(-2 ** 40, 2 ** 40, o.n, dtype=np.int64)
        for form in (one, two, eight, corr, shf):
            H.he_ctx_set_option(g.h, H.HE_OPT_NTT, form)
            x = g.ct(level)
            H.he_encrypt_coeffs(g.h, m, level, o.pr.scale, 77, x)
            assert_ct_equal(g.download(x), o.encrypt_coeffs(m, level, o.pr.scale, 77))
    finally:
        H.he_ctx_set_option(g.h, H.HE_OPT_NTT, two)


@pytest.mark.parametrize("log_n", [10, 11, 13])
def test_small_ring_rotation_and_relin_bit_exact(log_n):
    """Rings below 2^12 take the shared-memory radix-2 NTT; 2^13 the radix-16 one."""
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import GpuCtx, assert_ct_equal
    pr = Params(log_n=log_n, n_q=4, n_p=2, dnum=2, q0_bits=50, q_bits=40, p_bits=50,
                scale=2.0 ** 40, seed=9)
    o = Context(pr)
    g = GpuCtx(pr)
    try:
        ct, z = _rand_ct(o, 3, 300 + log_n)
        ct2, _ = _rand_ct(o, 3, 400 + log_n)
        o.gen_rotation_key(7)
        o.gen_relin_key()
        H.he_keygen_rotations(g.h, [7])
        H.he_keygen_relin(g.h)
        out = g.ct(3)
        H.he_rotate(g.h, g.upload(ct), 7, out)
        assert_ct_equal(g.download(out), o.rotate(ct, 7))
        m = g.ct(3)
        H.he_mul_relin(g.h, g.upload(ct), g.upload(ct2), m)
        assert_ct_equal(g.download(m), o.mul_relin(ct, ct2))
    finally:
        g.close()


def test_wide_digits_and_many_special_primes_bit_exact():
    """alpha = 12 and K = 10 (the serving parameters have alpha = K = 11): the base conversions
    and the inner product run their general instantiations, bit for bit against the oracle."""
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import GpuCtx, assert_ct_equal
    from oracle import layers as Ly
    pr = Params(log_n=12, n_q=12, n_p=10, dnum=1, q0_bits=50, q_bits=40, p_bits=50,
                scale=2.0 ** 40, seed=13)
    o = Context(pr)
    g = GpuCtx(pr)
    try:
        assert o.alpha == 12 and len(o.p) == 10
        level = 11
        ct, z = _rand_ct(o, level, 500)
        ct2, _ = _rand_ct(o, level, 501)
        rots = [3, -40]
        for r in rots:
            o.gen_rotation_key(r)
        o.gen_relin_key()
        H.he_keygen_rotations(g.h, rots)
        H.he_keygen_relin(g.h)
        out = g.ct(level)
        H.he_rotate(g.h, g.upload(ct), rots[0], out)
        assert_ct_equal(g.download(out), o.rotate(ct, rots[0]))
        outs = [g.ct(level) for _ in rots]
        H.he_rotate_hoisted(g.h, g.upload(ct), rots, outs)
        D = o.hoist(ct)
        for r, c in zip(rots, outs):
            assert_ct_equal(g.download(c), o.rotate_hoisted(ct, D, r))
        m = g.ct(level)
        H.he_mul_relin(g.h, g.upload(ct), g.upload(ct2), m)
        assert_ct_equal(g.download(m), o.mul_relin(ct, ct2))
        c = Ly.cheb_nodes_coeffs(Ly.gelu, 8, -8, 8)
        ref = Ly.cheb_ps_he(o, ct, c, target_scale=o.pr.scale)
        gc = g.upload(ct)
        H.he_poly_eval_ps(g.h, gc, c, o.pr.scale)
        H.he_ctx_check(g.h)
        assert H.he_ct_level(gc) == ref.level
        assert_ct_equal(g.download(gc), ref)
    finally:
        g.close()
