"""Host-side helpers of the product path: parameter sets, image <-> slot packing from the
C-ABI layout tables, Chebyshev interpolation of an activation, and encrypted-image wrappers.

Packing follows the layout metadata of Sec. 4 ("Sharding and Encrypting an Image",
"Duplicating and Permuting Channels"): block b of shard u holds frame rows [row0, row0 + B/M)
of channel chan[u][b], row-major with row stride M.  The activation polynomial is the
Chebyshev interpolant at the deg+1 first-kind nodes (Appendix, "Chebyshev Basis").
"""
import math

import numpy as np

from . import hegpu as H


def params(log_n, n_q, n_p, dnum, q0_bits, q_bits, p_bits, scale=2.0 ** 40, seed=0):
    return H.he_params(log_n, n_q, n_p, dnum, q0_bits, q_bits, p_bits, scale, seed)


def toy_params(seed=0):
    """2N = 2^13, four ~40-bit ciphertext primes, one special prime, dnum 4 (test only)."""
    return params(13, 4, 1, 4, 40, 40, 50, seed=seed)


def cifar_params(seed=0):
    """2N = 2^16, q_0 of 50 bits + 19 primes of 40 bits, 5 special primes, dnum 4."""
    return params(16, 20, 5, 4, 50, 40, 50, seed=seed)


def serving_params(seed=0):
    """2N = 2^16, 33 ciphertext primes (depth ~ the paper's 34), 11 special primes, dnum 3."""
    return params(16, 33, 11, 3, 50, 40, 50, seed=seed)


# ----------------------------------------------------------------------------- packing
def _coords(lay, u):
    chan, row0 = lay.tables()
    i = np.arange(lay.N)
    b = i // lay.B
    ch = chan[u][b]
    y = row0[u][b] + (i % lay.B) // lay.M
    x = i % lay.M
    ok = (ch >= 0) & (y < lay.m) & (x < lay.m)
    return ch, y, x, ok


def pack(lay, img):
    """img [c][m][m] -> slot vectors [n_shards][N] (zeros outside the valid pixels)."""
    img = np.asarray(img, dtype=np.float64)
    out = np.zeros((lay.n_shards, lay.N))
    for u in range(lay.n_shards):
        ch, y, x, ok = _coords(lay, u)
        out[u, ok] = img[ch[ok], y[ok], x[ok]]
    return out


def unpack(lay, slots):
    """slot vectors -> img [c][m][m], reading every pixel from its first copy."""
    img = np.full((lay.c, lay.m, lay.m), np.nan)
    for u in range(lay.n_shards):
        ch, y, x, ok = _coords(lay, u)
        cur = img[ch[ok], y[ok], x[ok]]
        img[ch[ok], y[ok], x[ok]] = np.where(np.isnan(cur), slots[u][ok], cur)
    if np.isnan(img).any():
        raise ValueError("layout does not cover every pixel")
    return img


# ----------------------------------------------------------------------------- activation
def gelu(x):
    return 0.5 * x * (1.0 + math.erf(x / math.sqrt(2.0)))


def chebyshev_coeffs(f, deg, lo, hi):
    """c_0..c_deg with f(x) ~ sum_k c_k T_k((2x - lo - hi)/(hi - lo)), interpolating at the
    nodes t_j = cos(pi (j + 1/2) / (deg + 1)) (discrete orthogonality of T_k there)."""
    K = deg + 1
    j = np.arange(K)
    theta = np.pi * (j + 0.5) / K
    fv = np.array([f(0.5 * (hi - lo) * math.cos(t) + 0.5 * (hi + lo)) for t in theta])
    c = np.array([(2.0 / K) * np.dot(fv, np.cos(k * theta)) for k in range(K)])
    c[0] /= 2.0
    return c


def minimax_coeffs(fn, deg, lo, hi):
    """The minimax polynomial of an activation ("gelu", "relu", "silu", "softplus") by the
    library's Remez routine: (c_0..c_deg in the same Chebyshev form, levelled error)."""
    ids = {"gelu": H.HE_FN_GELU, "relu": H.HE_FN_RELU, "silu": H.HE_FN_SILU, "softplus": H.HE_FN_SOFTPLUS}
    return H.he_cheb_minimax(ids[fn], deg, lo, hi)


# ----------------------------------------------------------------------------- images
def encrypt_image(ctx, lay, img, level, scale, nonce0=0, stream=None):
    slots = pack(lay, img)
    cts = []
    for u in range(lay.n_shards):
        ct = H.he_ct_alloc(ctx, level)
        H.he_encrypt(ctx, slots[u], level, scale, nonce0 + u, ct, stream)
        cts.append(ct)
    return cts


def decrypt_image(ctx, lay, cts, stream=None):
    return unpack(lay, np.stack([H.he_decrypt(ctx, ct, lay.N, stream) for ct in cts]))


def ps_products(deg):
    """Relinearised products of the Paterson-Stockmeyer evaluation of a degree-deg polynomial:
    the baby steps T_2..T_k, the giant steps beyond T_k, and one per split with a non-constant
    quotient (the same recursion as the library's)."""
    k = 2
    while k * k < (deg + 1) // 2:
        k *= 2
    giants = []
    g = k
    while g <= deg:
        giants.append(g)
        g *= 2
    count = (k - 1) + max(0, len(giants) - 1)

    def splits(d):
        if d < k:
            return 0
        G = max(x for x in giants if x <= d)
        qd, rd = d - G, G - 1
        if qd == 0:
            return splits(rd) if rd >= k else 0
        return 1 + splits(qd) + splits(rd)
    return count + splits(deg)


def ps_depth(deg):
    """Levels the Paterson-Stockmeyer evaluation of a degree-deg polynomial consumes (the
    library's recursion: leaves cost one level above their deepest baby step, a split with a
    non-constant quotient one level above the quotient and the giant step)."""
    k = 2
    while k * k < (deg + 1) // 2:
        k *= 2
    giants = []
    g = k
    while g <= deg:
        giants.append(g)
        g *= 2
    depth = lambda i: (i - 1).bit_length()

    def need(d):
        if d < k:
            return 1 + max([depth(i) for i in range(1, d + 1)] + [0])
        G = max(x for x in giants if x <= d)
        qd, rd = d - G, G - 1
        if qd == 0 and rd < k:
            return 1 + max([depth(G)] + [depth(i) for i in range(1, G)])
        if qd == 0:
            return max(1 + depth(G), need(rd))
        return max(need(qd) + 1, depth(G) + 1, need(rd))
    return need(deg)
