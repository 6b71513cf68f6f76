"""RNS-CKKS parameter sets and prime chains for the oracle (TEST INFRASTRUCTURE ONLY).

The paper (Sec. 2, "Homomorphic encryption"; Sec. 5.3 for its own sizes) works in
R_Q = Z_Q[X]/(X^{2N}+1) with N slots.  It does not say how the RNS primes are chosen, so
the oracle fixes one rule (a reading, listed in the design notes):

* every prime is = 1 mod 2n (n = 2N is the ring degree), so a primitive 2n-th root exists;
* primes of a given bit size b are the largest such primes below 2^b, in descending order;
* they are drawn in the order q_0 (q0_bits), p_0..p_{K-1} (p_bits), q_1..q_L (q_bits),
  each draw taking the next unused prime of its size, so all primes are distinct.

Primality is deterministic Miller-Rabin with the prime bases 2..37 (exact for n < 3.3e24).
"""
from dataclasses import dataclass


def is_prime(n: int) -> bool:
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for p in small:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def _prime_stream(bits: int, two_n: int):
    """Primes q < 2^bits with q = 1 mod two_n, largest first."""
    c = ((1 << bits) - 1) // two_n * two_n + 1
    if c >= (1 << bits):
        c -= two_n
    while c > two_n:
        if is_prime(c):
            yield c
        c -= two_n


@dataclass(frozen=True)
class Params:
    log_n: int          # ring degree n = 2^log_n  (the paper's 2N)
    n_q: int            # ciphertext primes q_0..q_L  (L = n_q - 1)
    n_p: int            # special primes p_0..p_{K-1}
    dnum: int           # key-switching digits
    q0_bits: int
    q_bits: int
    p_bits: int
    scale: float        # Delta
    seed: int
    secret_hw: int = 0  # 0: uniform ternary secret; h > 0: exactly h non-zero +-1 coefficients

    @property
    def n(self):
        return 1 << self.log_n

    @property
    def slots(self):
        return self.n // 2

    @property
    def alpha(self):
        return -(-self.n_q // self.dnum)


def gen_primes(pr: Params):
    """Return (q list, p list) following the module rule."""
    two_n = 2 * pr.n
    streams = {}

    def draw(bits):
        if bits not in streams:
            streams[bits] = _prime_stream(bits, two_n)
        return next(streams[bits])

    q0 = draw(pr.q0_bits)
    p = [draw(pr.p_bits) for _ in range(pr.n_p)]
    q = [q0] + [draw(pr.q_bits) for _ in range(pr.n_q - 1)]
    return q, p


def primitive_2n_root(q: int, n: int) -> int:
    """psi = x^((q-1)/2n) for the smallest quadratic non-residue x; then psi^n = -1."""
    x = 2
    while pow(x, (q - 1) // 2, q) != q - 1:
        x += 1
    psi = pow(x, (q - 1) // (2 * n), q)
    assert pow(psi, n, q) == q - 1
    return psi


# Parameter sets (a reading of the workload descriptions: 2^40 scale, ~40-bit ciphertext
# primes, ~50-bit first and special primes).
TOY = Params(log_n=13, n_q=4, n_p=1, dnum=4, q0_bits=40, q_bits=40, p_bits=50,
             scale=2.0 ** 40, seed=0)
C20 = Params(log_n=16, n_q=20, n_p=5, dnum=4, q0_bits=50, q_bits=40, p_bits=50,
             scale=2.0 ** 40, seed=0)
S33 = Params(log_n=16, n_q=33, n_p=11, dnum=3, q0_bits=50, q_bits=40, p_bits=50,
             scale=2.0 ** 40, seed=0)

# Bootstrapping sets.  The modular reduction of the raised ciphertext is approximated on
# [-K, K], K a bound on the integer I of t = m + q_0 I.  I is a sum of h + 1 terms in
# [-1/2, 1/2] (h = the secret's Hamming weight): |I| <= (h + 1) / 2 always, with standard
# deviation about sqrt((h + 1) / 12).  A uniform ternary secret at n = 2^16 would need K in the
# hundreds, so these sets use a sparse secret of weight 64 (deviation 2.3; K = 16 is 7 of them).
# Every prime has 50 bits and the scale is 2^50: the bootstrap's sine step runs at that scale,
# and a level-0 input at scale 2^40 keeps q_0 / scale = 2^10 for its small-angle reading.
# B24: ring 2^16, 23 levels (15 for the bootstrap, 8 for the network between bootstraps),
# log2(QP) = 1500.  BOOT12: ring 2^12 with the same 15-level bootstrap plus one level to spare,
# small enough for the oracle to run a whole bootstrap in seconds.
B24 = Params(log_n=16, n_q=24, n_p=6, dnum=4, q0_bits=50, q_bits=50, p_bits=50,
             scale=2.0 ** 50, seed=0, secret_hw=64)
BOOT12 = Params(log_n=12, n_q=17, n_p=4, dnum=6, q0_bits=50, q_bits=50, p_bits=50,
                scale=2.0 ** 50, seed=0, secret_hw=64)
