"""Plain RNS-CKKS for the oracle (TEST INFRASTRUCTURE ONLY).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may use this.

Paper, Sec. 2 ("Homomorphic encryption"): ciphertexts live in R_Q^2 with
R_Q = Z_Q[X]/(X^{2N}+1); each multiplication consumes one level; the scheme supports slot-wise
addition, multiplication and cyclic rotation.  The paper runs these through OpenFHE and is
silent on the internals, so the oracle fixes the textbook hybrid-key-switching RNS-CKKS
construction, one convention per step:

  storage      coefficient form, limb-major [poly][limb][n], residues in [0, q)
  secret       uniform ternary (SplitMix64 word mod 3), or with secret_hw = h > 0 a sparse
               ternary secret: a partial Fisher-Yates shuffle of 0..n-1 whose step k swaps
               position k with k + (word 2k mod (n - k)) and gives the coefficient at the
               position it lands on the sign + (word 2k+1 even) or - (odd), k < h
  errors       centred binomial eta=21
  uniform a    128-bit word pair mod q, sampled in coefficient form per limb
  encrypt      (c0, c1) = (-a s + e + m, a)  over Q_l
  keys         digit j covers C_j = {q_{j alpha} .. q_{(j+1) alpha - 1}};
               ksk[j] = (b_j, a_j) over Q_L u P with
               b_j = -a_j s + e_j + [P]_{q_i} s'   on q_i in C_j,   -a_j s + e_j elsewhere
  ModUp        digit j of x at level l: x on C_j n Q_l, fast base conversion elsewhere
  ModDown      (y_q - FBC~_{P->Q_l}(y_P)) * P^{-1}, FBC~ with centred digits, so the
               result is round(y / P) up to a small zero-mean integer
  rotate by r  g = 5^(r mod N) mod 2n; slot i <- slot i+r (numpy roll by -r)
               non-hoisted: u = sum_j ModUp(phi_g(c1))_j * ksk_g[j]
               hoisted:     u = sum_j phi_g(ModUp(c1)_j) * ksk_g[j]
               out = (phi_g(c0) + ModDown(u0), ModDown(u1))
  rescale      c'_i = (c_i - [t]_{q_i}) * q_l^{-1} mod q_i with t the centred representative
               of c_l (c_l - q_l when 2 c_l > q_l), i.e. c' = round(c / q_l)

The two roundings are centred on purpose: a [0, q) (floor) choice adds a bias of about 1/2
(rescale) or K/2 (ModDown) to every coefficient, and a constant coefficient bias evaluates to
~ (2n/pi)|s(zeta)| at the slot whose root is nearest 1 -- about 4e-6 at n = 2^16, above the
2^-20 accuracy target.
  mult         (a0 b0, a0 b1 + a1 b0, a1 b1), relinearise with s' = s^2, rescale
"""
import math

import numpy as np

from . import _lib
from .params import Params, gen_primes, primitive_2n_root
from .encode import encode, decode, decode_complex

STREAM_SECRET = 1
STREAM_KEY_A = 2 << 56
STREAM_KEY_E = 3 << 56
STREAM_ENC_A = 4 << 56
STREAM_ENC_E = 5 << 56
STREAM_SECRET_SPARSE = 6 << 56


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def reduce_signed(v: np.ndarray, q: int) -> np.ndarray:
    """int64 array -> residues in [0, q)."""
    assert q < (1 << 62)
    return np.mod(np.asarray(v, dtype=np.int64), np.int64(q)).astype(np.uint64)


class Ciphertext:
    """Coefficient-form ciphertext: c has shape [k][l+1][n] (k = 2, or 3 before relin)."""

    def __init__(self, c, level, scale):
        self.c = c
        self.level = level
        self.scale = float(scale)

    def copy(self):
        return Ciphertext(self.c.copy(), self.level, self.scale)


class Context:
    def __init__(self, params: Params):
        self.pr = params
        self.n = params.n
        self.N = params.slots
        self.L = params.n_q - 1
        self.K = params.n_p
        self.alpha = params.alpha
        self.q, self.p = gen_primes(params)
        self.psi_q = [primitive_2n_root(x, self.n) for x in self.q]
        self.psi_p = [primitive_2n_root(x, self.n) for x in self.p]
        self.lib = _lib.lib()
        self.seed = params.seed
        # ternary secret in Z (int64 coefficients)
        if params.secret_hw > 0:
            s = self.sparse_secret(params.secret_hw)
        else:
            s = np.zeros(self.n, dtype=np.int64)
            self.lib.orc_sample_ternary(self.seed, STREAM_SECRET, self.n, s)
        self.s_int = s
        self.keys = {}          # key_id -> list over digits of (b, a) eval form over Q_L u P
        self._s_eval_cache = {}

    def sparse_secret(self, h):
        """Exactly h coefficients +-1 at distinct positions (partial Fisher-Yates, module doc)."""
        n = self.n
        assert 0 < h <= n
        perm = list(range(n))
        s = np.zeros(n, dtype=np.int64)
        for k in range(h):
            r = int(self.lib.orc_rng(self.seed, STREAM_SECRET_SPARSE, 2 * k)) % (n - k)
            perm[k], perm[k + r] = perm[k + r], perm[k]
            odd = int(self.lib.orc_rng(self.seed, STREAM_SECRET_SPARSE, 2 * k + 1)) & 1
            s[perm[k]] = -1 if odd else 1
        return s

    # ------------------------------------------------------------ prime bookkeeping
    def mods(self, level, ext=False):
        m = self.q[: level + 1] + (self.p if ext else [])
        return np.array(m, dtype=np.uint64)

    def psis(self, level, ext=False):
        m = self.psi_q[: level + 1] + (self.psi_p if ext else [])
        return np.array(m, dtype=np.uint64)

    def limb_ids(self, level, ext=False):
        ids = list(range(level + 1)) + ([self.L + 1 + k for k in range(self.K)] if ext else [])
        return np.array(ids, dtype=np.int32)

    def digits(self, level):
        """Index lists C_j n Q_level, j < ceil((level+1)/alpha)."""
        out = []
        for j in range(-(-(level + 1) // self.alpha)):
            lo = j * self.alpha
            out.append(list(range(lo, min(lo + self.alpha, level + 1))))
        return out

    # ------------------------------------------------------------ ring helpers
    def ntt(self, a, mods, psis):
        a = _u64(a).copy()
        nl = a.size // self.n
        self.lib.orc_ntt(a, nl, self.n, _u64(mods), _u64(psis))
        return a

    def intt(self, a, mods, psis):
        a = _u64(a).copy()
        nl = a.size // self.n
        self.lib.orc_intt(a, nl, self.n, _u64(mods), _u64(psis))
        return a

    def reduce_int(self, v, mods):
        """Integer polynomial (int64 [n]) -> residues [len(mods)][n]."""
        return np.stack([reduce_signed(v, int(m)) for m in mods])

    def poly_mul(self, a, b, level, ext=False):
        """Negacyclic product of two coefficient-form polynomials, limb by limb."""
        mods, psis = self.mods(level, ext), self.psis(level, ext)
        A = self.ntt(a, mods, psis)
        B = self.ntt(b, mods, psis)
        C = np.empty_like(A)
        self.lib.orc_mul(A, B, C, len(mods), self.n, mods)
        return self.intt(C, mods, psis).reshape(len(mods), self.n)

    @staticmethod
    def add(a, b, mods):
        m = mods[:, None]
        return (a + b) % m

    @staticmethod
    def sub(a, b, mods):
        m = mods[:, None]
        return (a + (m - b % m)) % m

    @staticmethod
    def neg(a, mods):
        m = mods[:, None]
        return (m - a % m) % m

    def mul_scalar(self, a, scal, mods):
        out = np.empty_like(_u64(a))
        self.lib.orc_mul_scalar(_u64(a), _u64(scal), out, len(mods), self.n, _u64(mods))
        return out

    def automorph_coeff(self, a, g, mods):
        a = _u64(a)
        out = np.empty_like(a)
        self.lib.orc_automorph_coeff(a, out, len(mods), self.n, _u64(mods), g)
        return out

    def automorph_eval(self, a, g):
        a = _u64(a)
        out = np.empty_like(a)
        self.lib.orc_automorph_eval(a, out, a.size // self.n, self.n, g)
        return out

    def galois(self, r):
        return pow(5, r % self.N, 2 * self.n)

    # ------------------------------------------------------------ sampling
    def sample_uniform(self, stream, level, ext):
        mods = self.mods(level, ext)
        ids = self.limb_ids(level, ext)
        out = np.empty((len(mods), self.n), dtype=np.uint64)
        self.lib.orc_sample_uniform(self.seed, stream, self.n, len(mods), ids, mods, out)
        return out

    def sample_cbd(self, stream):
        e = np.zeros(self.n, dtype=np.int64)
        self.lib.orc_sample_cbd(self.seed, stream, self.n, e)
        return e

    def secret_int_automorph(self, g):
        """phi_g(s) as an integer polynomial."""
        n = self.n
        t = (np.arange(n, dtype=np.int64) * g) % (2 * n)
        out = np.zeros(n, dtype=np.int64)
        lo = t < n
        out[t[lo]] = self.s_int[lo]
        out[t[~lo] - n] = -self.s_int[~lo]
        return out

    # ------------------------------------------------------------ keys
    def _gen_ksk(self, key_id, s_prime_int):
        """Hybrid key-switching key for s' (integer polynomial), eval form over Q_L u P."""
        # hybrid key switching needs P at least as large as every digit's modulus: the
        # inner product's error grows with the digit modulus and ModDown divides it by P
        P = math.prod(self.p)
        for dig in self.digits(self.L):
            if math.prod(self.q[i] for i in dig) > P:
                raise ValueError("special modulus P smaller than a digit modulus")
        L = self.L
        mods = self.mods(L, True)
        psis = self.psis(L, True)
        s_res = self.reduce_int(self.s_int, mods)
        sp_res = self.reduce_int(s_prime_int, mods)
        P_mod = [1] * len(mods)
        for i, m in enumerate(mods):
            v = 1
            for pj in self.p:
                v = v * pj % int(m)
            P_mod[i] = v
        s_eval = self.ntt(s_res, mods, psis).reshape(len(mods), self.n)
        out = []
        for j, dig in enumerate(self.digits(L)):
            a = self.sample_uniform(STREAM_KEY_A | (key_id << 8) | j, L, True)
            e = self.reduce_int(self.sample_cbd(STREAM_KEY_E | (key_id << 8) | j), mods)
            a_eval = self.ntt(a, mods, psis).reshape(len(mods), self.n)
            as_eval = np.empty_like(a_eval)
            self.lib.orc_mul(a_eval, s_eval, as_eval, len(mods), self.n, mods)
            as_coef = self.intt(as_eval, mods, psis).reshape(len(mods), self.n)
            b = self.sub(e, as_coef, mods)
            gadget = np.zeros((len(mods), self.n), dtype=np.uint64)
            for i in dig:
                gadget[i] = self.mul_scalar(sp_res[i:i + 1], np.array([P_mod[i]], dtype=np.uint64),
                                            mods[i:i + 1])[0]
            b = self.add(b, gadget, mods)
            out.append((self.ntt(b, mods, psis).reshape(len(mods), self.n), a_eval))
        return out

    def gen_rotation_key(self, r):
        g = self.galois(r)
        if g not in self.keys:
            self.keys[g] = self._gen_ksk(g, self.secret_int_automorph(g))
        return g

    def conj_galois(self):
        """Galois element of complex conjugation of the slots: X -> X^{2n-1} = X^{-1}."""
        return 2 * self.n - 1

    def gen_conj_key(self):
        g = self.conj_galois()
        if g not in self.keys:
            self.keys[g] = self._gen_ksk(g, self.secret_int_automorph(g))
        return g

    def gen_relin_key(self):
        if 0 not in self.keys:
            L = self.L
            # s^2 as an integer polynomial: every coefficient of the negacyclic square of a
            # ternary polynomial lies in [-n, n], far inside (-q_0/2, q_0/2), so the
            # product mod q_0, centred, is the exact integer square.
            q0 = self.q[0]
            s0 = self.reduce_int(self.s_int, self.mods(0))
            sq = self.poly_mul(s0, s0, 0)[0].astype(np.int64)
            sq = np.where(sq > q0 // 2, sq - q0, sq)
            assert np.all(np.abs(sq) <= self.n)
            self.keys[0] = self._gen_ksk(0, sq)
        return 0

    def export_key(self, key_id):
        """Key in coefficient form: array [digits][2][L+1+K][n] (b, a)."""
        L = self.L
        mods, psis = self.mods(L, True), self.psis(L, True)
        out = []
        for b, a in self.keys[key_id]:
            out.append(np.stack([self.intt(b, mods, psis).reshape(len(mods), self.n),
                                 self.intt(a, mods, psis).reshape(len(mods), self.n)]))
        return np.stack(out)

    # ------------------------------------------------------------ encrypt / decrypt
    def encrypt_coeffs(self, m_int, level, scale, nonce):
        """Encrypt an integer message polynomial (int64 [n])."""
        mods, psis = self.mods(level), self.psis(level)
        a = self.sample_uniform(STREAM_ENC_A | nonce, level, False)
        e = self.sample_cbd(STREAM_ENC_E | nonce)
        s_res = self.reduce_int(self.s_int, mods)
        as_ = self.poly_mul(a, s_res, level)
        c0 = self.add(self.sub(self.reduce_int(e, mods), as_, mods), self.reduce_int(m_int, mods), mods)
        return Ciphertext(np.stack([c0, a]), level, scale)

    def encrypt(self, z, level, scale=None, nonce=0):
        scale = self.pr.scale if scale is None else scale
        return self.encrypt_coeffs(encode(z, self.n, scale), level, scale, nonce)

    def decrypt_coeffs(self, ct):
        """Centred integer coefficients (python ints) of c0 + c1 s (+ c2 s^2) mod Q_l."""
        level = ct.level
        mods = self.mods(level)
        s_res = self.reduce_int(self.s_int, mods)
        m = ct.c[0].copy()
        spow = s_res
        for k in range(1, ct.c.shape[0]):
            m = self.add(m, self.poly_mul(ct.c[k], spow, level), mods)
            if k + 1 < ct.c.shape[0]:
                spow = self.poly_mul(spow, s_res, level)
        return crt_centred(m, [int(x) for x in mods])

    def decrypt(self, ct):
        coeffs = self.decrypt_coeffs(ct)
        return decode(np.array([float(c) for c in coeffs]), self.n, ct.scale)

    def decrypt_complex(self, ct):
        coeffs = self.decrypt_coeffs(ct)
        return decode_complex(np.array([float(c) for c in coeffs]), self.n, ct.scale)

    # ------------------------------------------------------------ basic ops
    def rescale(self, ct):
        l = ct.level
        assert l >= 1
        mods = self.mods(l - 1)
        ql = self.q[l]
        out = np.empty((ct.c.shape[0], l, self.n), dtype=np.uint64)
        inv = np.array([pow(ql, -1, int(m)) for m in mods], dtype=np.uint64)
        for k in range(ct.c.shape[0]):
            top = ct.c[k, l].astype(np.int64)        # in [0, q_l)
            t = np.where(2 * top > ql, top - ql, top)          # centred representative
            red = np.stack([reduce_signed(t, int(m)) for m in mods])
            diff = self.sub(ct.c[k, :l], red, mods)
            out[k] = self.mul_scalar(diff, inv, mods)
        return Ciphertext(out, l - 1, ct.scale / ql)

    def drop_to(self, ct, level):
        assert level <= ct.level
        return Ciphertext(ct.c[:, : level + 1].copy(), level, ct.scale)

    def add_ct(self, a, b):
        assert a.level == b.level
        mods = self.mods(a.level)
        return Ciphertext(np.stack([self.add(a.c[k], b.c[k], mods) for k in range(2)]),
                          a.level, a.scale)

    def sub_ct(self, a, b):
        assert a.level == b.level
        mods = self.mods(a.level)
        return Ciphertext(np.stack([self.sub(a.c[k], b.c[k], mods) for k in range(2)]),
                          a.level, a.scale)

    def mul_plain(self, ct, pt_coeffs, pt_scale):
        """ct * pt (no rescale); pt_coeffs is an int64 integer polynomial."""
        mods = self.mods(ct.level)
        p = self.reduce_int(pt_coeffs, mods)
        return Ciphertext(np.stack([self.poly_mul(ct.c[k], p, ct.level) for k in range(2)]),
                          ct.level, ct.scale * pt_scale)

    def mul_int(self, ct, c):
        """Multiply by a (signed python) integer constant; no level consumed."""
        mods = self.mods(ct.level)
        scal = np.array([c % int(m) for m in mods], dtype=np.uint64)
        return Ciphertext(np.stack([self.mul_scalar(ct.c[k], scal, mods) for k in range(2)]),
                          ct.level, ct.scale)

    def add_const_int(self, ct, c):
        """Add the constant polynomial c (python int) to c0."""
        mods = self.mods(ct.level)
        out = ct.c.copy()
        for i, m in enumerate(mods):
            out[0, i, 0] = (int(out[0, i, 0]) + c) % int(m)
        return Ciphertext(out, ct.level, ct.scale)

    # ------------------------------------------------------------ key switching
    def modup(self, x, level):
        """x: coefficient form [level+1][n].  Returns list of digits D_j [level+1+K][n]."""
        mods_ext = self.mods(level, True)
        out = []
        for dig in self.digits(level):
            D = np.empty((len(mods_ext), self.n), dtype=np.uint64)
            others = [t for t in range(len(mods_ext)) if t not in dig]
            qC = np.array([self.q[i] for i in dig], dtype=np.uint64)
            qB = mods_ext[others].copy()
            conv = np.empty((len(others), self.n), dtype=np.uint64)
            self.lib.orc_fbc(_u64(x[dig]), qC, len(dig), qB, len(others), conv, self.n)
            D[dig] = x[dig]
            D[others] = conv
            out.append(D)
        return out

    def moddown(self, y, level):
        """y: coefficient form over Q_level u P.  Returns [level+1][n]."""
        mods = self.mods(level)
        nq = level + 1
        conv = np.empty((nq, self.n), dtype=np.uint64)
        self.lib.orc_fbc_centred(_u64(y[nq:]), np.array(self.p, dtype=np.uint64), self.K, mods,
                                 nq, conv, self.n)
        diff = self.sub(y[:nq], conv, mods)
        Pinv = []
        for m in mods:
            v = 1
            for pj in self.p:
                v = v * pj % int(m)
            Pinv.append(pow(v, -1, int(m)))
        return self.mul_scalar(diff, np.array(Pinv, dtype=np.uint64), mods)

    def _key_limbs(self, key_id, level):
        """Restrict a key (eval form over Q_L u P) to the limbs of Q_level u P."""
        idx = list(range(level + 1)) + [self.L + 1 + k for k in range(self.K)]
        return [(b[idx], a[idx]) for (b, a) in self.keys[key_id]]

    def _inner_product(self, D_eval, key_id, level):
        """u_c = sum_j D_j * ksk[j]_c in eval form, returned in coefficient form."""
        mods, psis = self.mods(level, True), self.psis(level, True)
        keys = self._key_limbs(key_id, level)
        u = [np.zeros((len(mods), self.n), dtype=np.uint64) for _ in range(2)]
        for j, Dj in enumerate(D_eval):
            b, a = keys[j]
            self.lib.orc_mac(u[0], _u64(Dj), _u64(b), len(mods), self.n, mods)
            self.lib.orc_mac(u[1], _u64(Dj), _u64(a), len(mods), self.n, mods)
        return [self.intt(x, mods, psis).reshape(len(mods), self.n) for x in u]

    def key_switch(self, d, level, key_id):
        """Non-hoisted key switch of polynomial d (coeff form) -> (ModDown(u0), ModDown(u1))."""
        mods, psis = self.mods(level, True), self.psis(level, True)
        D = self.modup(d, level)
        D_eval = [self.ntt(Dj, mods, psis).reshape(len(mods), self.n) for Dj in D]
        u = self._inner_product(D_eval, key_id, level)
        return self.moddown(u[0], level), self.moddown(u[1], level)

    def rotate(self, ct, r):
        """Non-hoisted rotation (slot i <- slot i+r)."""
        g = self.galois(r)
        assert g in self.keys, "rotation key missing"
        mods = self.mods(ct.level)
        c0 = self.automorph_coeff(ct.c[0], g, mods)
        c1 = self.automorph_coeff(ct.c[1], g, mods)
        k0, k1 = self.key_switch(c1, ct.level, g)
        return Ciphertext(np.stack([self.add(c0, k0, mods), k1]), ct.level, ct.scale)

    def conjugate(self, ct):
        """Slot-wise complex conjugate: phi_g with g = 2n - 1 (zeta^{g_i} -> zeta^{-g_i}), then a
        non-hoisted key switch from phi_g(s) back to s."""
        g = self.conj_galois()
        assert g in self.keys, "conjugation key missing"
        mods = self.mods(ct.level)
        c0 = self.automorph_coeff(ct.c[0], g, mods)
        c1 = self.automorph_coeff(ct.c[1], g, mods)
        k0, k1 = self.key_switch(c1, ct.level, g)
        return Ciphertext(np.stack([self.add(c0, k0, mods), k1]), ct.level, ct.scale)

    def mul_monomial(self, ct, k):
        """Multiply both polynomials by X^k in Z_Q[X]/(X^n + 1) (exact; no level, no noise).
        Slot i is multiplied by zeta^{k g_i}; k = n/2 multiplies every slot by i, since
        g_i = 1 mod 4."""
        n = self.n
        k %= 2 * n
        sign = 1
        if k >= n:
            k -= n
            sign = -1
        mods = self.mods(ct.level)
        out = np.empty_like(ct.c)
        for p in range(ct.c.shape[0]):
            a = ct.c[p]
            hi = self.neg(a[:, n - k:], mods) if k else a[:, :0]
            rot = np.concatenate([hi, a[:, :n - k]], axis=1)    # X^k: j -> j + k, wrap negated
            out[p] = rot if sign > 0 else self.neg(rot, mods)
        return Ciphertext(out, ct.level, ct.scale)

    def modraise(self, ct, level=None):
        """A level-0 ciphertext read over Q_level (default L): every residue mod q_0 is lifted to
        its centred representative in (-q_0/2, q_0/2] and reduced mod q_0..q_level.  The result
        decrypts to t = [c0 + c1 s]_{q_0} + q_0 I for an integer polynomial I with
        |I| <= (||s||_1 + 1) / 2 (the centred c0 + c1 s over Z, divided by q_0)."""
        assert ct.level == 0
        level = self.L if level is None else level
        q0 = self.q[0]
        mods = self.mods(level)
        out = np.empty((ct.c.shape[0], level + 1, self.n), dtype=np.uint64)
        for p in range(ct.c.shape[0]):
            x = ct.c[p, 0].astype(np.int64)
            x = np.where(2 * x > q0, x - q0, x)
            out[p] = self.reduce_int(x, mods)
        return Ciphertext(out, level, ct.scale)

    def hoist(self, ct):
        """ModUp(c1) once per ciphertext, digits in eval form."""
        mods, psis = self.mods(ct.level, True), self.psis(ct.level, True)
        return [self.ntt(Dj, mods, psis).reshape(len(mods), self.n)
                for Dj in self.modup(ct.c[1], ct.level)]

    def rotate_hoisted(self, ct, D_eval, r):
        """Hoisted rotation: u = sum_j phi_g(D_j) * ksk_g[j]."""
        if r % self.N == 0:
            return ct.copy()
        g = self.galois(r)
        assert g in self.keys, "rotation key missing"
        mods = self.mods(ct.level)
        Dg = [self.automorph_eval(Dj, g).reshape(Dj.shape) for Dj in D_eval]
        u = self._inner_product(Dg, g, ct.level)
        c0 = self.automorph_coeff(ct.c[0], g, mods)
        out0 = self.add(c0, self.moddown(u[0], ct.level), mods)
        return Ciphertext(np.stack([out0, self.moddown(u[1], ct.level)]), ct.level, ct.scale)

    def mul_relin(self, a, b):
        """Tensor, relinearise, rescale."""
        assert a.level == b.level
        l = a.level
        mods = self.mods(l)
        d0 = self.poly_mul(a.c[0], b.c[0], l)
        d1 = self.add(self.poly_mul(a.c[0], b.c[1], l), self.poly_mul(a.c[1], b.c[0], l), mods)
        d2 = self.poly_mul(a.c[1], b.c[1], l)
        k0, k1 = self.key_switch(d2, l, 0)
        ct = Ciphertext(np.stack([self.add(d0, k0, mods), self.add(d1, k1, mods)]), l,
                        a.scale * b.scale)
        return self.rescale(ct)


def crt_centred(res, mods):
    """Residues [k][n] -> list of centred python ints in (-Q/2, Q/2]."""
    Q = 1
    for m in mods:
        Q *= m
    coef = []
    for m in mods:
        Qi = Q // m
        coef.append(Qi * pow(Qi, -1, m))
    n = res.shape[1]
    out = [0] * n
    cols = [res[i].tolist() for i in range(len(mods))]
    for j in range(n):
        x = 0
        for i in range(len(mods)):
            x += cols[i][j] * coef[i]
        x %= Q
        if x > Q // 2:
            x -= Q
        out[j] = x
    return out
