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


def params(log_n, n_q, n_p, dnum, q0_bits, q_bits, p_bits, scale=2.0 ** 40, seed=0, secret_hw=0):
    return H.he_params(log_n, n_q, n_p, dnum, q0_bits, q_bits, p_bits, scale, seed, secret_hw)


def toy_params(seed=0):
    """2N = 2^13, four ~40-bit ciphertext primes, one special prime, dnum 4 (test only)."""
    return params(13, 4, 1, 4, 40, 40, 50, seed=seed)


def cifar_params(seed=0):
    """2N = 2^16, q_0 of 50 bits + 19 primes of 40 bits, 5 special primes, dnum 4."""
    return params(16, 20, 5, 4, 50, 40, 50, seed=seed)


def bootstrap_params(seed=0):
    """2N = 2^16, 24 ciphertext primes and 6 special primes of 50 bits, dnum 4, scale 2^50, a
    sparse secret of weight 64: 15 levels for the bootstrap (3 CoeffToSlot, 1 retarget, 6
    Paterson-Stockmeyer, 2 double angles, 3 SlotToCoeff) and 8 for the network between two
    bootstraps; log2(QP) = 1500."""
    return params(16, 24, 6, 4, 50, 50, 50, scale=2.0 ** 50, seed=seed, secret_hw=64)


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
def _fn_id(fn):
    ids = {"gelu": H.HE_FN_GELU, "relu": H.HE_FN_RELU, "silu": H.HE_FN_SILU, "softplus": H.HE_FN_SOFTPLUS}
    return ids[fn]


def chebyshev_coeffs(fn, deg, lo, hi):
    """c_0..c_deg with f(x) ~ sum_k c_k T_k((2x - lo - hi)/(hi - lo)): the library's interpolation
    at the deg + 1 first-kind Chebyshev nodes, for an activation "gelu", "relu", "silu" or
    "softplus"."""
    return H.he_cheb_interp(_fn_id(fn), deg, lo, hi)


def minimax_coeffs(fn, deg, lo, hi):
    """The minimax polynomial of an activation ("gelu", "relu", "silu", "softplus") by the
    library's Remez routine: (c_0..c_deg in the same Chebyshev form, levelled error)."""
    return H.he_cheb_minimax(_fn_id(fn), deg, lo, hi)


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
    """Relinearised products of the library's Paterson-Stockmeyer evaluation of a degree-deg
    polynomial."""
    return H.he_poly_ps_plan(deg)[0]


def ps_depth(deg):
    """Levels the library's Paterson-Stockmeyer evaluation of a degree-deg polynomial consumes."""
    return H.he_poly_ps_plan(deg)[1]
