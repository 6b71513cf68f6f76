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
