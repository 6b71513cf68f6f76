"""he_rescale_noalloc: the rescale for callers that cannot allocate device memory.

It must give exactly what he_rescale gives (ciphertext limbs are integers, so the tolerance
is zero), on two calls in a row, and refuse sizes beyond its fixed scratch.  This file sorts
last so that a run stopping at the first failure has run every other test before it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ctx(log_n, n_q, n_p, dnum):
    from paper_2306_09189_gb300 import hegpu as H
    return H.he_ctx_create(H.he_params(log_n, n_q, n_p, dnum, 50, 40, 50, 2.0 ** 40, 21))


@pytest.mark.parametrize("log_n,n_q,n_p,dnum", [(12, 6, 2, 3), (16, 20, 5, 4)])
def test_noalloc_rescale_equals_rescale_twice(log_n, n_q, n_p, dnum):
    from paper_2306_09189_gb300 import hegpu as H
    ctx = _ctx(log_n, n_q, n_p, dnum)
    cts = []
    try:
        n = 1 << log_n
        level = n_q - 1
        z = np.random.default_rng(log_n).uniform(-1, 1, n // 2)
        a, b = H.he_ct_alloc(ctx, level), H.he_ct_alloc(ctx, level)
        cts += [a, b]
        q = H.he_ctx_info(ctx)["q"]
        H.he_encrypt(ctx, z, level, 2.0 ** 40, 5, a)
        H.he_ct_copy(b, a)
        for step in range(2):                       # two calls in a row
            lv = level - step
            for c in (a, b):                        # scale up by q_l so the rescale keeps z
                H.he_mul_int(ctx, c, float(q[lv]))
                H.he_ct_set_scale(c, H.he_ct_scale(c) * float(q[lv]))
            H.he_rescale(ctx, a)
            H.he_rescale_noalloc(ctx, b)
            assert H.he_ct_level(a) == H.he_ct_level(b) == level - 1 - step
            assert H.he_ct_scale(a) == H.he_ct_scale(b)
            ea, eb = H.he_ct_export_coeffs(ctx, a, n), H.he_ct_export_coeffs(ctx, b, n)
            assert np.array_equal(ea, eb)
            got = H.he_decrypt(ctx, b, n // 2)
            assert np.abs(got - z).max() < 1e-6
    finally:
        for c in cts:
            H.he_ct_free(c)
        H.he_ctx_destroy(ctx)


def test_noalloc_rescale_limit_is_exact():
    """2 * level * n words must fit in the 3 * 2^20-word scratch: at n = 2^16 level 24 fills it
    exactly and must give he_rescale's bits; level 25 is one limb pair too many and is refused."""
    from paper_2306_09189_gb300 import hegpu as H
    ctx = _ctx(16, 26, 8, 3)                        # levels 0..25 at n = 2^16
    cts = []
    try:
        n = 1 << 16
        q = H.he_ctx_info(ctx)["q"]
        z = np.random.default_rng(24).uniform(-1, 1, n // 2)
        a, b = H.he_ct_alloc(ctx, 24), H.he_ct_alloc(ctx, 24)
        cts += [a, b]
        H.he_encrypt(ctx, z, 24, 2.0 ** 40, 7, a)
        H.he_mul_int(ctx, a, float(q[24]))            # scale up by q_24 so the rescale keeps z
        H.he_ct_set_scale(a, H.he_ct_scale(a) * float(q[24]))
        H.he_ct_copy(b, a)
        H.he_rescale(ctx, a)
        H.he_rescale_noalloc(ctx, b)
        assert H.he_ct_level(b) == 23 and H.he_ct_scale(a) == H.he_ct_scale(b)
        assert np.array_equal(H.he_ct_export_coeffs(ctx, a, n), H.he_ct_export_coeffs(ctx, b, n))
        assert np.abs(H.he_decrypt(ctx, b, n // 2) - z).max() < 1e-6
        top = H.he_ct_alloc(ctx, 25)
        cts.append(top)
        H.he_encrypt(ctx, z, 25, 2.0 ** 40, 8, top)
        with pytest.raises(H.HEError) as e:
            H.he_rescale_noalloc(ctx, top)
        assert e.value.code == H.HE_EINVAL and "scratch" in str(e.value)
        assert H.he_ct_level(top) == 25                 # a refused call leaves the ciphertext as it was
    finally:
        for c in cts:
            H.he_ct_free(c)
        H.he_ctx_destroy(ctx)
