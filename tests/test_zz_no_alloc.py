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


def test_noalloc_rescale_rejects_too_large_a_ciphertext():
    from paper_2306_09189_gb300 import hegpu as H
    ctx = _ctx(16, 33, 11, 3)                       # level 32 at n = 2^16: 2*32*2^16 words
    try:
        ct = H.he_ct_alloc(ctx, 32)
        with pytest.raises(H.HEError) as e:
            H.he_rescale_noalloc(ctx, ct)
        assert e.value.code == H.HE_EINVAL and "scratch" in str(e.value)
        H.he_ct_free(ct)
    finally:
        H.he_ctx_destroy(ctx)
