"""Pins for the oracle's ring arithmetic (no GPU).

Each test checks the oracle against something other than itself: direct polynomial
evaluation, schoolbook products, exact big-integer CRT identities, primality by brute force.
"""
import numpy as np
import pytest

from oracle import _lib
from oracle.params import Params, gen_primes, is_prime, primitive_2n_root
from oracle.ckks import Context, crt_centred

L = _lib.lib()


def _rand_res(rng, q, n):
    return np.array([int(rng.integers(0, q)) for _ in range(n)], dtype=np.uint64)


def test_is_prime_matches_trial_division():
    def trial(n):
        if n < 2:
            return False
        d = 2
        while d * d <= n:
            if n % d == 0:
                return False
            d += 1
        return True
    for n in range(0, 5000):
        assert is_prime(n) == trial(n)
    # strong pseudoprimes to several small bases must be rejected
    for n in (3215031751, 2152302898747, 3474749660383, 341550071728321):
        assert not is_prime(n)


@pytest.mark.parametrize("log_n", [4, 13, 16])
def test_prime_chain_rule(log_n):
    pr = Params(log_n=log_n, n_q=6, n_p=3, dnum=2, q0_bits=50, q_bits=40, p_bits=50,
                scale=2.0 ** 40, seed=0)
    q, p = gen_primes(pr)
    two_n = 2 << (log_n - 1) if log_n > 0 else 2
    two_n = 2 * (1 << log_n)
    allp = q + p
    assert len(set(allp)) == len(allp)
    for x in allp:
        assert is_prime(x) and x % two_n == 1
    assert q[0] < 2 ** 50 and all(2 ** 39 < x < 2 ** 40 for x in q[1:])
    # q_0 is the largest 50-bit prime = 1 mod 2n, then p_0 > p_1 > ... come next
    big = [q[0]] + p
    assert big == sorted(big, reverse=True)
    assert q[1:] == sorted(q[1:], reverse=True)
    c = big[0] + two_n
    while c < 2 ** 50:
        assert not is_prime(c)
        c += two_n


def test_primitive_root_order():
    for q in gen_primes(Params(10, 3, 1, 1, 40, 40, 50, 1.0, 0))[0]:
        psi = primitive_2n_root(q, 1024)
        assert pow(psi, 1024, q) == q - 1 and pow(psi, 2048, q) == 1


@pytest.mark.parametrize("n", [8, 16, 64])
def test_ntt_is_evaluation_at_odd_powers(n):
    q = gen_primes(Params(n.bit_length() - 1, 1, 1, 1, 40, 40, 50, 1.0, 0))[0][0]
    psi = primitive_2n_root(q, n)
    rng = np.random.default_rng(n)
    a = _rand_res(rng, q, n)
    A = a.copy()
    L.orc_ntt(A, 1, n, np.array([q], dtype=np.uint64), np.array([psi], dtype=np.uint64))
    for k in range(n):
        x = pow(psi, 2 * k + 1, q)
        assert int(A[k]) == sum(int(a[j]) * pow(x, j, q) for j in range(n)) % q
    L.orc_intt(A, 1, n, np.array([q], dtype=np.uint64), np.array([psi], dtype=np.uint64))
    assert np.array_equal(A, a)


@pytest.mark.parametrize("log_n", [3, 5, 8, 10])
def test_negacyclic_product_matches_schoolbook(log_n):
    pr = Params(log_n, 3, 1, 1, 50, 40, 50, 1.0, 0)
    ctx = Context(pr)
    n = ctx.n
    rng = np.random.default_rng(log_n)
    a = np.stack([_rand_res(rng, int(m), n) for m in ctx.mods(2)])
    b = np.stack([_rand_res(rng, int(m), n) for m in ctx.mods(2)])
    c = ctx.poly_mul(a, b, 2)
    for i, m in enumerate(ctx.mods(2)):
        m = int(m)
        ref = [0] * n
        ai, bi = [int(v) for v in a[i]], [int(v) for v in b[i]]
        for x in range(n):
            for y in range(n):
                if x + y < n:
                    ref[x + y] += ai[x] * bi[y]
                else:
                    ref[x + y - n] -= ai[x] * bi[y]
        assert [int(v) for v in c[i]] == [r % m for r in ref]


def test_automorphism_eval_form_equals_coefficient_form():
    ctx = Context(Params(8, 2, 1, 1, 50, 40, 50, 1.0, 0))
    rng = np.random.default_rng(5)
    mods, psis = ctx.mods(1), ctx.psis(1)
    a = np.stack([_rand_res(rng, int(m), ctx.n) for m in mods])
    for r in (1, 3, 77, ctx.N - 1):
        g = ctx.galois(r)
        lhs = ctx.automorph_eval(ctx.ntt(a, mods, psis), g)
        rhs = ctx.ntt(ctx.automorph_coeff(a, g, mods), mods, psis)
        assert np.array_equal(lhs, rhs)


def test_automorphism_coeff_is_substitution():
    # a(X^g) mod X^n + 1, computed by reducing exponents with a python dict
    ctx = Context(Params(5, 1, 1, 1, 50, 40, 50, 1.0, 0))
    q = int(ctx.q[0])
    rng = np.random.default_rng(1)
    a = _rand_res(rng, q, ctx.n)[None]
    g = ctx.galois(3)
    out = ctx.automorph_coeff(a, g, ctx.mods(0))[0]
    ref = [0] * ctx.n
    for j in range(ctx.n):
        e = j * g
        sgn = -1 if (e // ctx.n) % 2 else 1
        ref[e % ctx.n] = (ref[e % ctx.n] + sgn * int(a[0, j])) % q
    assert [int(v) for v in out] == ref


def _tiny_ctx():
    return Context(Params(log_n=4, n_q=5, n_p=2, dnum=2, q0_bits=30, q_bits=25, p_bits=30,
                          scale=2.0 ** 20, seed=3))


def _crt(res, mods):
    Q = 1
    for m in mods:
        Q *= m
    x = 0
    for r, m in zip(res, mods):
        Qi = Q // m
        x += int(r) * Qi * pow(Qi, -1, m)
    return x % Q, Q


def test_fbc_is_x_plus_small_multiple_of_Q():
    ctx = _tiny_ctx()
    rng = np.random.default_rng(0)
    qC = [int(x) for x in ctx.q[:3]]
    qB = [int(x) for x in ctx.q[3:]] + [int(x) for x in ctx.p]
    x = np.stack([_rand_res(rng, m, ctx.n) for m in qC])
    out = np.empty((len(qB), ctx.n), dtype=np.uint64)
    L.orc_fbc(x, np.array(qC, dtype=np.uint64), 3, np.array(qB, dtype=np.uint64), len(qB), out, ctx.n)
    for j in range(ctx.n):
        X, Q = _crt([x[i, j] for i in range(3)], qC)
        us = set()
        for b, p in enumerate(qB):
            u = (int(out[b, j]) - X) * pow(Q, -1, p) % p
            us.add(u)
        assert len(us) == 1 and 0 <= us.pop() < len(qC)


def test_moddown_is_rounded_division_by_P():
    # ModDown(y) = (Y - X')/P with X' = Y mod P and |X'| < K P / 2: within K/2 of Y / P
    ctx = _tiny_ctx()
    level = 3
    rng = np.random.default_rng(1)
    mods = [int(m) for m in ctx.mods(level, True)]
    y = np.stack([_rand_res(rng, m, ctx.n) for m in mods])
    r = ctx.moddown(y, level)
    P = 1
    for p in ctx.p:
        P *= p
    deltas = []
    for j in range(ctx.n):
        Y, _ = _crt(y[:, j], mods)
        base = (2 * Y + P) // (2 * P)                      # round(Y / P)
        ds = set()
        for i in range(level + 1):
            q = mods[i]
            d = (base - int(r[i, j])) % q
            ds.add(d if d <= q // 2 else d - q)
        assert len(ds) == 1
        d = ds.pop()
        assert abs(d) <= ctx.K // 2 + 1
        deltas.append(d)
    assert min(deltas) < 0 < max(deltas) or all(d == 0 for d in deltas)


def test_rescale_is_exact_rounded_division():
    ctx = _tiny_ctx()
    from oracle.ckks import Ciphertext
    level = 4
    rng = np.random.default_rng(2)
    mods = [int(m) for m in ctx.mods(level)]
    c = np.stack([np.stack([_rand_res(rng, m, ctx.n) for m in mods]) for _ in range(2)])
    out = ctx.rescale(Ciphertext(c, level, 2.0 ** 40))
    ql = mods[level]
    for k in range(2):
        for j in range(ctx.n):
            X, _ = _crt(c[k, :, j], mods)
            want = (2 * X + ql) // (2 * ql)                # round(X / q_l), q_l odd
            for i in range(level):
                assert int(out.c[k, i, j]) == want % mods[i]


def test_crt_centred_roundtrip():
    mods = [1099511590913, 1099511560193, 1125899906826241]
    rng = np.random.default_rng(0)
    Q = mods[0] * mods[1] * mods[2]
    vals = [int(rng.integers(-2 ** 62, 2 ** 62)) * int(rng.integers(1, 2 ** 40)) for _ in range(50)]
    res = np.array([[v % m for v in vals] for m in mods], dtype=np.uint64)
    assert crt_centred(res, mods) == vals
    assert all(abs(v) < Q // 2 for v in vals)


def test_splitmix64_published_vectors():
    # SplitMix64 with state 0 and increment gamma: first outputs of the reference
    # generator (Vigna, splitmix64.c) are mix(gamma), mix(2 gamma), ...
    gamma = 0x9E3779B97F4A7C15
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    for k, e in enumerate(expect):
        assert L.orc_splitmix64_mix((gamma * (k + 1)) % 2 ** 64) == e


def test_samplers_ranges_and_moments():
    n = 1 << 14
    s = np.zeros(n, dtype=np.int64)
    L.orc_sample_ternary(7, 1, n, s)
    assert set(np.unique(s)) <= {-1, 0, 1}
    assert abs(np.mean(s == 0) - 1 / 3) < 0.02
    e = np.zeros(n, dtype=np.int64)
    L.orc_sample_cbd(7, 9, n, e)
    assert np.abs(e).max() <= 21 and abs(e.var() - 10.5) < 0.6 and abs(e.mean()) < 0.1
