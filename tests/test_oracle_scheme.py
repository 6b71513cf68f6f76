"""Pins for the oracle's encoder and scheme operations (no GPU)."""
import numpy as np
import pytest

from oracle.params import Params
from oracle.ckks import Context
from oracle.encode import encode, encode_real, encode_naive, decode, decode_naive

SMALL = Params(log_n=10, n_q=6, n_p=2, dnum=3, q0_bits=50, q_bits=40, p_bits=50,
               scale=2.0 ** 40, seed=11)


@pytest.fixture(scope="module")
def ctx():
    c = Context(SMALL)
    c.gen_relin_key()
    return c


@pytest.mark.parametrize("n", [16, 64, 256])
def test_fft_encoder_matches_closed_form(n):
    rng = np.random.default_rng(n)
    z = rng.uniform(-3, 3, n // 2)
    a = encode_real(z, n, 2.0 ** 30)
    b = encode_naive(z, n, 2.0 ** 30)
    assert np.abs(a - b).max() < 1e-6 * 2 ** 30 / n * n
    assert np.abs(decode(a, n, 2.0 ** 30) - decode_naive(a, n, 2.0 ** 30)).max() < 1e-9
    assert np.abs(decode(a, n, 2.0 ** 30) - z).max() < 1e-9


def test_constant_vector_encodes_to_constant_polynomial():
    n = 1024
    m = encode(np.full(n // 2, 0.75), n, 2.0 ** 40)
    assert m[0] == round(0.75 * 2 ** 40) and np.all(m[1:] == 0)


def test_embedding_is_multiplicative(ctx):
    # the canonical embedding maps the negacyclic product to the slot-wise product
    rng = np.random.default_rng(1)
    z, w = rng.uniform(-1, 1, ctx.N), rng.uniform(-1, 1, ctx.N)
    S = 2.0 ** 30
    mz, mw = encode(z, ctx.n, S), encode(w, ctx.n, S)
    prod = ctx.poly_mul(ctx.reduce_int(mz, ctx.mods(1)), ctx.reduce_int(mw, ctx.mods(1)), 1)
    from oracle.ckks import crt_centred
    coeffs = np.array([float(v) for v in crt_centred(prod, [int(x) for x in ctx.mods(1)])])
    assert np.abs(decode(coeffs, ctx.n, S * S) - z * w).max() < 1e-6


def test_encrypt_decrypt(ctx):
    rng = np.random.default_rng(2)
    z = rng.uniform(-1, 1, ctx.N)
    for level in (0, 3, 5):
        assert np.abs(ctx.decrypt(ctx.encrypt(z, level, nonce=level)) - z).max() < 1e-9


@pytest.mark.parametrize("r", [1, 5, 100, -1, -37])
def test_rotation_is_roll(ctx, r):
    rng = np.random.default_rng(3)
    z = rng.uniform(-1, 1, ctx.N)
    ct = ctx.encrypt(z, 5, nonce=9)
    ctx.gen_rotation_key(r)
    assert np.abs(ctx.decrypt(ctx.rotate(ct, r)) - np.roll(z, -r)).max() < 1e-7
    D = ctx.hoist(ct)
    assert np.abs(ctx.decrypt(ctx.rotate_hoisted(ct, D, r)) - np.roll(z, -r)).max() < 1e-7


def test_rotation_at_lower_level_partial_digit(ctx):
    # level 3: digits {0,1},{2,3}; level 4: {0,1},{2,3},{4} (partial last digit)
    rng = np.random.default_rng(4)
    z = rng.uniform(-1, 1, ctx.N)
    ctx.gen_rotation_key(3)
    for level in (1, 3, 4):
        ct = ctx.encrypt(z, level, nonce=20 + level)
        assert np.abs(ctx.decrypt(ctx.rotate(ct, 3)) - np.roll(z, -3)).max() < 1e-7


def test_relinearised_product_is_slotwise_product(ctx):
    rng = np.random.default_rng(5)
    z, w = rng.uniform(-1, 1, ctx.N), rng.uniform(-1, 1, ctx.N)
    a, b = ctx.encrypt(z, 5, nonce=1), ctx.encrypt(w, 5, nonce=2)
    m = ctx.mul_relin(a, b)
    assert m.level == 4
    assert abs(m.scale - 2.0 ** 80 / ctx.q[5]) < 1e-3
    assert np.abs(ctx.decrypt(m) - z * w).max() < 1e-7


def test_plaintext_product_keeps_scale_exact(ctx):
    rng = np.random.default_rng(6)
    z, w = rng.uniform(-1, 1, ctx.N), rng.uniform(-1, 1, ctx.N)
    ct = ctx.encrypt(z, 4, nonce=3)
    out = ctx.rescale(ctx.mul_plain(ct, encode(w, ctx.n, float(ctx.q[4])), float(ctx.q[4])))
    assert out.scale == 2.0 ** 40 and out.level == 3
    assert np.abs(ctx.decrypt(out) - z * w).max() < 1e-7


def test_key_switching_key_decrypts_to_gadget(ctx):
    # b_j + a_j s = e_j + P s' on C_j: the key (coefficient form) minus P s' is small
    g = ctx.gen_rotation_key(2)
    key = ctx.export_key(g)
    mods = ctx.mods(ctx.L, True)
    s = ctx.reduce_int(ctx.s_int, mods)
    sp = ctx.secret_int_automorph(g)
    P = 1
    for p in ctx.p:
        P *= p
    for j, dig in enumerate(ctx.digits(ctx.L)):
        v = ctx.add(key[j, 0], ctx.poly_mul(key[j, 1], s, ctx.L, True), mods)
        for i, m in enumerate(mods):
            m = int(m)
            gad = (P % m) * sp % m if i in dig else np.zeros(ctx.n, dtype=np.int64)
            e = (v[i].astype(object) - np.asarray(gad, dtype=object)) % m
            e = np.where(e > m // 2, e - m, e).astype(np.int64)
            assert np.abs(e).max() <= 21


def test_special_modulus_below_a_digit_is_rejected():
    # digits of 3 primes (~130 bits) against P of 2 primes (~100 bits): key switching would
    # not be correct, key generation refuses the set (the library refuses the context)
    ctx = Context(Params(log_n=10, n_q=5, n_p=2, dnum=2, q0_bits=50, q_bits=40, p_bits=50, scale=2.0 ** 40, seed=1))
    with pytest.raises(ValueError):
        ctx.gen_rotation_key(1)
    with pytest.raises(ValueError):
        ctx.gen_relin_key()
