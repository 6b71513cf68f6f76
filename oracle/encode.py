"""CKKS canonical-embedding encoder/decoder for the oracle (TEST INFRASTRUCTURE ONLY).

Paper, Sec. 2 ("Homomorphic encryption"): a ciphertext over Z_Q[X]/(X^{2N}+1) has N slots,
each holding one real number.  With n = 2N, zeta = exp(i*pi/n) and g_i = 5^i mod 2n, slot i
is the evaluation of the plaintext polynomial at zeta^{g_i}.  For real slot values z the
unique real polynomial with m(zeta^{+-g_i}) = S z_i has coefficients

    m_j = (2 S / n) * sum_{i<N} z_i cos(pi g_i j / n)                           (closed form)

and decoding is z_i = (1/S) sum_j m_j cos(pi g_i j / n).  The integer plaintext rounds m_j
half away from zero.  `encode_naive`/`decode_naive` evaluate those sums literally; `encode`/
`decode` compute the same sums with one length-2n FFT (numpy), a library step.

Complex slots (needed by bootstrapping, whose linear transforms have complex diagonals): the
real polynomial with m(zeta^{g_i}) = S z_i and m(zeta^{-g_i}) = S conj(z_i) has coefficients

    m_j = (2 S / n) * sum_{i<N} Re(z_i zeta^{-g_i j}),                          (closed form)

which reduces to the cosine sum for real z; decoding is z_i = m(zeta^{g_i}) / S.
`encode_complex(_naive)` / `decode_complex(_naive)` implement these.
"""
import numpy as np


def slot_exponents(n: int) -> np.ndarray:
    """g_i = 5^i mod 2n for i < n/2."""
    N = n // 2
    g = np.empty(N, dtype=np.int64)
    v = 1
    for i in range(N):
        g[i] = v
        v = v * 5 % (2 * n)
    return g


def round_half_away(x: np.ndarray) -> np.ndarray:
    return np.where(x >= 0, np.floor(x + 0.5), np.ceil(x - 0.5))


def encode_real(z, n: int, S: float) -> np.ndarray:
    """Real (unrounded) coefficients (2S/n) sum_i z_i cos(pi g_i j/n), via one FFT.

    A[k] = z_i at k = g_i and k = 2n - g_i (the conjugate slots), 0 elsewhere; then
    sum_k A[k] exp(-2 pi i k j / 2n) = 2 sum_i z_i cos(pi g_i j / n).
    """
    z = np.asarray(z, dtype=np.float64)
    N = n // 2
    assert z.shape == (N,)
    g = slot_exponents(n)
    A = np.zeros(2 * n, dtype=np.float64)
    A[g] = z
    A[2 * n - g] = z
    F = np.fft.fft(A)
    return (S / n) * F.real[:n]


def encode(z, n: int, S: float) -> np.ndarray:
    """Integer plaintext coefficients (int64), rounded half away from zero."""
    m = round_half_away(encode_real(z, n, S))
    assert np.all(np.abs(m) < 2.0 ** 62), "plaintext coefficient overflow"
    return m.astype(np.int64)


def encode_naive(z, n: int, S: float) -> np.ndarray:
    """Literal double sum of the closed form (small n only)."""
    z = np.asarray(z, dtype=np.float64)
    g = slot_exponents(n)
    j = np.arange(n)
    C = np.cos(np.pi * np.outer(g, j) / n)       # [N][n]
    return (2.0 * S / n) * (z @ C)


def decode(m, n: int, S: float) -> np.ndarray:
    """Slots from real polynomial coefficients m (float64 array of length n)."""
    m = np.asarray(m, dtype=np.float64)
    g = slot_exponents(n)
    a = np.zeros(2 * n, dtype=np.float64)
    a[:n] = m
    F = np.fft.fft(a)             # F[k] = sum_j m_j exp(-2 pi i k j / 2n)
    return F.real[g] / S          # real part of m(zeta^{g}) (conjugate has equal real part)


def decode_naive(m, n: int, S: float) -> np.ndarray:
    m = np.asarray(m, dtype=np.float64)
    g = slot_exponents(n)
    j = np.arange(n)
    C = np.cos(np.pi * np.outer(g, j) / n)
    return (C @ m) / S


def encode_complex_real(z, n: int, S: float) -> np.ndarray:
    """Real (unrounded) coefficients (2S/n) sum_i Re(z_i zeta^{-g_i j}), via one FFT.

    A[g_i] = z_i and A[2n - g_i] = conj(z_i); sum_k A[k] exp(-2 pi i k j / 2n) is then real and
    equals 2 sum_i Re(z_i zeta^{-g_i j})."""
    z = np.asarray(z, dtype=np.complex128)
    N = n // 2
    assert z.shape == (N,)
    g = slot_exponents(n)
    A = np.zeros(2 * n, dtype=np.complex128)
    A[g] = z
    A[2 * n - g] = np.conj(z)
    F = np.fft.fft(A)
    return (S / n) * F.real[:n]


def encode_complex(z, n: int, S: float) -> np.ndarray:
    """Integer plaintext of complex slot values (int64), rounded half away from zero."""
    m = round_half_away(encode_complex_real(z, n, S))
    assert np.all(np.abs(m) < 2.0 ** 62), "plaintext coefficient overflow"
    return m.astype(np.int64)


def encode_complex_naive(z, n: int, S: float) -> np.ndarray:
    """Literal sum of the closed form (small n only)."""
    z = np.asarray(z, dtype=np.complex128)
    g = slot_exponents(n)
    j = np.arange(n)
    E = np.exp(-1j * np.pi * np.outer(g, j) / n)   # zeta^{-g_i j}
    return (2.0 * S / n) * np.real(z @ E)


def decode_complex(m, n: int, S: float) -> np.ndarray:
    """Complex slots m(zeta^{g_i}) / S from real coefficients (float64 array of length n)."""
    m = np.asarray(m, dtype=np.float64)
    g = slot_exponents(n)
    a = np.zeros(2 * n, dtype=np.float64)
    a[:n] = m
    F = np.fft.fft(a)             # F[k] = m(zeta^{-k}) = conj(m(zeta^{k})) for a real m
    return np.conj(F[g]) / S


def decode_complex_naive(m, n: int, S: float) -> np.ndarray:
    m = np.asarray(m, dtype=np.float64)
    g = slot_exponents(n)
    j = np.arange(n)
    E = np.exp(1j * np.pi * np.outer(g, j) / n)    # zeta^{g_i j}
    return (E @ m) / S
