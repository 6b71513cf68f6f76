"""Failure detection without a GPU fault: a bounded device wait that nothing satisfies gives up,
the host reads HE_ETIMEOUT from he_ctx_check, and the context keeps working afterwards."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_stays_usable():
    from paper_2306_09189_gb300 import hegpu as H, host
    pr = host.params(12, 6, 2, 3, 50, 40, 50, seed=3)
    ctx = H.he_ctx_create(pr)
    try:
        H.he_ctx_check(ctx)                       # clean to begin with
        t0 = time.perf_counter()
        H.he_selftest_bounded_wait(ctx)
        with pytest.raises(H.HEError) as e:
            H.he_ctx_check(ctx)
        assert e.value.code == H.HE_ETIMEOUT
        assert time.perf_counter() - t0 < 10.0   # the wait is bounded in time
        H.he_ctx_check(ctx)                       # the flag was cleared
        # the context still computes: a rotation decrypts to the rolled slots
        H.he_keygen_rotations(ctx, [3])
        z = np.random.default_rng(0).uniform(-1, 1, 2048)
        a, b = H.he_ct_alloc(ctx, 5), H.he_ct_alloc(ctx, 5)
        H.he_encrypt(ctx, z, 5, pr.scale, 1, a)
        H.he_rotate(ctx, a, 3, b)
        H.he_ctx_check(ctx)
        assert np.abs(H.he_decrypt(ctx, b, 2048) - np.roll(z, -3)).max() < 1e-6
        H.he_ct_free(a)
        H.he_ct_free(b)
    finally:
        H.he_ctx_destroy(ctx)
