"""The library's host Remez routine (he_cheb_minimax, no GPU) against the oracle's."""
import numpy as np
import pytest

from oracle import layers as Ly


@pytest.mark.parametrize("fn,deg,lo,hi", [("relu", 27, -16, 16), ("gelu", 27, -16, 16), ("relu", 59, -16, 16),
                                          ("gelu", 59, -16, 16), ("gelu", 16, -8, 8)])
def test_library_minimax_equals_oracle(fn, deg, lo, hi):
    from paper_2306_09189_gb300 import host
    c, E = host.minimax_coeffs(fn, deg, lo, hi)
    oc, oE = Ly.minimax_coeffs(getattr(Ly, fn), deg, lo, hi)
    assert abs(E - oE) <= 1e-9 * oE
    assert np.abs(c - oc).max() <= 1e-9 * max(1.0, np.abs(oc).max())


def test_library_minimax_other_activations_and_errors():
    from paper_2306_09189_gb300 import hegpu as H, host
    xs = np.linspace(-8, 8, 20001)
    for fn, f in (("silu", lambda x: x / (1 + np.exp(-x))), ("softplus", lambda x: np.log1p(np.exp(x)))):
        c, E = host.minimax_coeffs(fn, 20, -8, 8)
        r = f(xs) - Ly.cheb_eval(c, xs, -8, 8)
        assert np.abs(r).max() <= E * (1 + 1e-6) and E < 1e-2
    with pytest.raises(H.HEError):
        H.he_cheb_minimax(9, 10, -1, 1)
    with pytest.raises(H.HEError):
        H.he_cheb_minimax(H.HE_FN_GELU, 10, 1, -1)


@pytest.mark.parametrize("fn,deg,lo,hi", [("gelu", 16, -8, 8), ("gelu", 27, -16, 16), ("relu", 59, -16, 16),
                                          ("gelu", 59, -16, 16), ("relu", 3, -1, 1)])
def test_library_chebyshev_interpolation_equals_oracle(fn, deg, lo, hi):
    """The library's node interpolation (he_cheb_interp, host only) agrees with the oracle's to
    rounding, and reproduces the paper's interpolation rows through the oracle's evaluation."""
    from paper_2306_09189_gb300 import host
    c = host.chebyshev_coeffs(fn, deg, lo, hi)
    oc = Ly.cheb_nodes_coeffs(getattr(Ly, fn), deg, lo, hi)
    assert c.shape == oc.shape
    assert np.abs(c - oc).max() <= 1e-13 * max(1.0, np.abs(oc).max())
    # it interpolates: exact at the nodes
    t = np.cos(np.pi * (np.arange(deg + 1) + 0.5) / (deg + 1))
    x = 0.5 * (hi - lo) * t + 0.5 * (hi + lo)
    f = np.array([getattr(Ly, fn)(v) for v in x])
    assert np.abs(Ly.cheb_eval(c, x, lo, hi) - f).max() <= 1e-12 * max(1.0, np.abs(f).max())


def test_library_ps_plan_equals_the_oracle_evaluation():
    """he_poly_ps_plan (host only) gives the products and levels the oracle's Paterson-Stockmeyer
    evaluation actually takes: mul_relin calls counted and output level measured on a small ring."""
    from paper_2306_09189_gb300 import hegpu as H
    from oracle.ckks import Context
    from oracle.params import Params
    ctx = Context(Params(log_n=9, n_q=10, n_p=3, dnum=4, q0_bits=50, q_bits=40, p_bits=50,
                         scale=2.0 ** 40, seed=11))
    ctx.gen_relin_key()
    ct = ctx.encrypt(np.random.default_rng(1).uniform(-1, 1, ctx.N), 9, nonce=1)
    orig = ctx.mul_relin
    for deg in (2, 3, 4, 5, 7, 8, 9, 15, 16, 17, 27, 31, 32, 33, 59):
        count = [0]

        def counted(a, b):
            count[0] += 1
            return orig(a, b)
        ctx.mul_relin = counted
        try:
            out = Ly.cheb_ps_he(ctx, ct, Ly.cheb_nodes_coeffs(Ly.gelu, deg, -8, 8))
        finally:
            ctx.mul_relin = orig
        assert H.he_poly_ps_plan(deg) == (count[0], ct.level - out.level), deg
    assert [H.he_poly_ps_plan(d) for d in (16, 27, 59)] == [(8, 5), (11, 5), (16, 6)]
    with pytest.raises(H.HEError):
        H.he_poly_ps_plan(1)
