"""Pins of the oracle's bootstrapping (oracle/bootstrap.py) against the mathematics it rests on.

* complex encoding: the closed form written as a literal sum, and decoding as the dense
  matrix U_ij = zeta^{g_i j} applied to m_lo + i m_hi;
* the special DFT: the merged butterfly levels against the dense U (SlotToCoeff gives U w from
  BR(w), CoeffToSlot gives N BR(U^-1 z)), the baby-step giant-step regrouping against the
  level it regroups, the diagonal counts a butterfly network must have;
* ModRaise: the raised ciphertext decrypts to the level-0 decryption plus q_0 I, exactly, with
  |I| <= (h + 1) / 2 for a weight-h secret;
* conjugation and monomials: decrypted slots conjugated / multiplied by i, X^n = -1 exactly;
* EvalMod: the interpolant against cos, the double angles against sin(2 pi x);
* the whole bootstrap: the decrypted output equals the input message within the precision the
  noise analysis gives, at the level the plan says.
"""
import math

import numpy as np
import pytest

from oracle import bootstrap as B
from oracle.ckks import Context
from oracle.encode import (encode, encode_real, encode_complex, encode_complex_real, encode_complex_naive,
                           decode_complex, decode_complex_naive)
from oracle.layers import cheb_eval, cheb_ps_slots
from oracle.params import Params, BOOT12

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

TINY = Params(log_n=10, n_q=17, n_p=4, dnum=6, q0_bits=50, q_bits=50, p_bits=50, scale=2.0 ** 50, seed=3,
              secret_hw=64)


@pytest.fixture(scope="module")
def tiny():
    ctx = Context(TINY)
    plan = B.BootPlan(ctx)
    B.gen_boot_keys(ctx, plan)
    return ctx, plan


# ------------------------------------------------------------------ complex encoding
def test_complex_encoding_closed_form():
    rng = np.random.default_rng(0)
    for n in (16, 256):
        z = rng.normal(size=n // 2) + 1j * rng.normal(size=n // 2)
        S = 2.0 ** 30
        a = encode_complex_real(z, n, S)
        b = encode_complex_naive(z, n, S)
        assert np.max(np.abs(a - b)) < 1e-6 * S / n * n
        m = rng.normal(size=n) * 1e6
        d = decode_complex(m, n, 1.0)
        tol = 1e-12 * np.max(np.abs(d))
        assert np.max(np.abs(d - decode_complex_naive(m, n, 1.0))) < tol
        # decoding is the dense U applied to m_lo + i m_hi (zeta^{g_i N} = i since g_i = 1 mod 4)
        U = B.dft_matrix(n)
        N = n // 2
        assert np.max(np.abs(d - U @ (m[:N] + 1j * m[N:]))) < tol
        # real slots: the same integers as the real encoder
        zr = rng.uniform(-1, 1, N)
        assert np.array_equal(encode_complex(zr, n, S), encode(zr, n, S))
        # round trip
        back = decode_complex(encode_complex_real(z, n, S), n, S)
        assert np.max(np.abs(back - z)) < 1e-9


# ------------------------------------------------------------------ the special DFT
@pytest.mark.parametrize("n,levels", [(16, 1), (64, 2), (256, 3), (1024, 3), (1024, 4)])
def test_merged_levels_are_the_encoding_dft(n, levels):
    rng = np.random.default_rng(n + levels)
    N = n // 2
    U = B.dft_matrix(n)
    br = B.bit_reverse(N)
    w = rng.normal(size=N) + 1j * rng.normal(size=N)
    v = w[br]
    for st, D in B.stc_levels(N, levels):
        v = B.apply_diagonals(D, v)
    assert np.max(np.abs(v - U @ w)) < 1e-9 * N
    z = rng.normal(size=N) + 1j * rng.normal(size=N)
    u = z.copy()
    for st, D in B.cts_levels(N, levels):
        u = B.apply_diagonals(D, u)
    winv = np.linalg.solve(U, z)
    assert np.max(np.abs(u - N * winv[br])) < 1e-9 * N


@pytest.mark.parametrize("n,levels", [(256, 3), (2048, 3), (4096, 3)])
def test_bsgs_regrouping_and_diagonal_counts(n, levels):
    rng = np.random.default_rng(7)
    N = n // 2
    logN = N.bit_length() - 1
    for which in (B.cts_levels, B.stc_levels):
        for st, D in which(N, levels):
            m = len(st)
            wraps = 2 * max(st) == N
            # a butterfly network of m stages reaches offsets sum e_k h_k, e_k in {-1, 0, 1}:
            # 2^(m+1) - 1 diagonals, or 2^m when the largest stage spans the whole vector
            assert len(D) == (2 ** m if wraps else 2 ** (m + 1) - 1)
            # unit-magnitude entries (every input-output pair joined by one path)
            for v in D.values():
                nz = v[v != 0]
                assert np.allclose(np.abs(nz), 1.0)
            L = B.bsgs_level(N, st, D, 1.0)
            x = rng.normal(size=N) + 1j * rng.normal(size=N)
            assert np.max(np.abs(B.bsgs_apply(L, x) - B.apply_diagonals(D, x))) < 1e-9
            assert sum(len(b) for b in L.baby.values()) == len(D)
    assert sum(B.level_groups(logN, levels)) == logN


# ------------------------------------------------------------------ sparse secret, ModRaise
def test_sparse_secret_weight_and_modraise_is_exact(tiny):
    ctx, plan = tiny
    s = ctx.s_int
    assert np.count_nonzero(s) == TINY.secret_hw
    assert set(np.unique(s).tolist()) <= {-1, 0, 1}
    assert not np.array_equal(s, Context(Params(**{**TINY.__dict__, "seed": 4})).s_int)
    rng = np.random.default_rng(1)
    z = rng.uniform(-1, 1, ctx.N)
    ct = ctx.encrypt(z, 0, 2.0 ** 40)
    base = ctx.decrypt_coeffs(ct)                 # centred mod q_0
    x = ctx.modraise(ct)
    assert x.level == ctx.L
    t = ctx.decrypt_coeffs(x)                     # centred mod Q_L: the integer c0 + c1 s
    q0 = ctx.q[0]
    bound = (TINY.secret_hw + 1) // 2
    for a, b in zip(t, base):
        assert (a - b) % q0 == 0
        assert abs((a - b) // q0) <= bound


# ------------------------------------------------------------------ conjugation, monomials
def test_conjugation_and_monomials(tiny):
    ctx, plan = tiny
    rng = np.random.default_rng(2)
    z = rng.uniform(-1, 1, ctx.N) + 1j * rng.uniform(-1, 1, ctx.N)
    S = 2.0 ** 45
    ct = ctx.encrypt_coeffs(encode_complex(z, ctx.n, S), 5, S, nonce=9)
    c = ctx.conjugate(ct)
    assert np.max(np.abs(ctx.decrypt_complex(c) - np.conj(z))) < 2 ** -25
    mi = ctx.mul_monomial(ct, ctx.n // 2)
    assert np.max(np.abs(ctx.decrypt_complex(mi) - 1j * z)) < 2 ** -25
    neg = ctx.mul_monomial(ct, ctx.n)
    assert np.array_equal(neg.c, np.stack([ctx.neg(ct.c[k], ctx.mods(5)) for k in range(2)]))
    twice = ctx.mul_monomial(ctx.mul_monomial(ct, 3), 2 * ctx.n - 3)
    assert np.array_equal(twice.c, ct.c)


# ------------------------------------------------------------------ one linear level
def test_one_merged_level_decrypts_to_its_slot_simulator(tiny):
    ctx, plan = tiny
    rng = np.random.default_rng(3)
    z = rng.uniform(-1, 1, ctx.N) + 1j * rng.uniform(-1, 1, ctx.N)
    S = 2.0 ** 45
    lvl = plan.cts_level[0]
    ct = ctx.encrypt_coeffs(encode_complex(z, ctx.n, S), lvl, S, nonce=11)
    lv = plan.cts[0]
    out = B.lintrans_he(ctx, ct, lv, plan.plaintexts(ctx, "cts", 0))
    assert out.level == lvl - 1
    want = B.bsgs_apply(lv, z) / lv.gain
    assert np.max(np.abs(ctx.decrypt_complex(out) - want)) < 2 ** -30


# ------------------------------------------------------------------ EvalMod
def test_evalmod_polynomial_and_double_angles():
    cfg = B.BootConfig()
    ctx = Context(TINY)
    plan = B.BootPlan(ctx, cfg)
    u = np.linspace(-1, 1, 4001)
    f = np.cos(2 * np.pi * (cfg.K * u - 0.25) / 2 ** cfg.r)
    assert np.max(np.abs(cheb_eval(plan.coeffs, u, -1.0, 1.0) - f)) < 2 ** -40
    y = cheb_ps_slots(plan.coeffs, u)
    for _ in range(cfg.r):
        y = 2 * y * y - 1
    assert np.max(np.abs(y - np.sin(2 * np.pi * cfg.K * u))) < 2 ** -34
    # near an integer x = I + e the sine is the reduction: sin(2 pi x) / 2 pi = e - O(e^3)
    e = 2.0 ** -10
    for I in (-12, 0, 7):
        x = I + e
        assert abs(math.sin(2 * math.pi * x) / (2 * math.pi) - e) < (2 * math.pi) ** 2 * e ** 3 / 6 * 1.01
    assert plan.ps_depth == 6
    assert plan.out_level == ctx.L - 15


# ------------------------------------------------------------------ the whole bootstrap
def _check_bootstrap(ctx, plan, seed, bits):
    rng = np.random.default_rng(seed)
    z = rng.uniform(-1, 1, ctx.N)
    ct = ctx.encrypt(z, 0, 2.0 ** 40, nonce=seed)
    out = B.bootstrap(ctx, ct, plan)
    assert out.level == plan.out_level
    err = np.max(np.abs(ctx.decrypt(out) - z))
    assert err < 2.0 ** -bits, err
    return err


def test_bootstrap_restores_levels_ring_2_10(tiny):
    ctx, plan = tiny
    _check_bootstrap(ctx, plan, 21, 17)


def test_bootstrap_restores_levels_ring_2_12():
    ctx = Context(BOOT12)
    plan = B.BootPlan(ctx)
    B.gen_boot_keys(ctx, plan)
    _check_bootstrap(ctx, plan, 22, 15)


def test_bootstrap_from_a_higher_level(tiny):
    ctx, plan = tiny
    rng = np.random.default_rng(23)
    z = rng.uniform(-1, 1, ctx.N)
    ct = ctx.encrypt(z, 4, TINY.scale, nonce=23)
    y = B.to_level0(ctx, ct)
    assert y.level == 0 and abs(y.scale / (ctx.q[0] / 1024.0) - 1) < 2.0 ** -20
    assert np.max(np.abs(ctx.decrypt(y) - z)) < 2.0 ** -25
    out = B.bootstrap(ctx, ct, plan)
    assert out.level == plan.out_level
    assert np.max(np.abs(ctx.decrypt(out) - z)) < 2.0 ** -17


def test_meta_bootstrap_removes_most_of_the_error(tiny):
    ctx, plan = tiny
    rng = np.random.default_rng(24)
    z = rng.uniform(-1, 1, ctx.N)
    ct = ctx.encrypt(z, 0, 2.0 ** 40, nonce=24)
    one = np.max(np.abs(ctx.decrypt(B.bootstrap(ctx, ct, plan)) - z))
    out = B.meta_bootstrap(ctx, ct, plan)
    assert out.level == plan.out_level - 1
    two = np.max(np.abs(ctx.decrypt(out) - z))
    assert two < one / 16, (one, two)
