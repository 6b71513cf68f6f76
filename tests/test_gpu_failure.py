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


def test_host_side_faults_return_codes_and_leave_the_context_usable():
    # simulated allocation failure, a missing rotation key, level exhaustion and a malformed
    # layout each come back as an error code; no GPU fault, and the context keeps computing
    import torch
    from paper_2306_09189_gb300 import hegpu as H, host
    pr = host.params(12, 6, 2, 3, 50, 40, 50, seed=3)
    ctx = H.he_ctx_create(pr)
    try:
        N = 2048
        # allocation failure: the very next device allocation, then one deep inside a plan
        H.he_debug_fail_alloc(0)
        with pytest.raises(H.HEError) as e:
            H.he_ct_alloc(ctx, 5)
        assert e.value.code == H.HE_ENOMEM
        ct = H.he_ct_alloc(ctx, 5)                        # the hook disarmed itself
        rng = np.random.default_rng(1)
        W = rng.uniform(-1, 1, (4, 4, 3, 3))
        lay = H.he_layout_image(4, 16, N)
        for after in (0, 1, 3):                          # plan tables, bias, run buffers
            H.he_debug_fail_alloc(after)
            with pytest.raises(H.HEError) as e:
                H.he_conv_create(ctx, lay, W, None, 1, 1, 3, pr.scale)
            assert e.value.code == H.HE_ENOMEM
        H.he_debug_fail_alloc(-1)
        conv = H.he_conv_create(ctx, lay, W, None, 1, 1, 3, pr.scale)
        # missing rotation key: the run refuses before launching anything
        x = host.encrypt_image(ctx, lay, rng.uniform(0, 1, (4, 16, 16)), 3, pr.scale)
        y = [H.he_ct_alloc(ctx, 2)]
        with pytest.raises(H.HEError) as e:
            H.he_conv_run(ctx, conv, x, y, H.HE_BATCHED)
        assert e.value.code == H.HE_EKEY
        H.he_keygen_rotations(ctx, H.he_conv_rotations(conv))
        H.he_conv_run(ctx, conv, x, y, H.HE_BATCHED)
        H.he_ctx_check(ctx)
        assert H.he_ct_check_range(ctx, y[0]) == 0
        # level exhaustion: a ciphertext at level 0 cannot be rescaled
        z = H.he_ct_alloc(ctx, 0)
        H.he_encrypt(ctx, rng.uniform(-1, 1, N), 0, pr.scale, 7, z)
        with pytest.raises(H.HEError) as e:
            H.he_rescale(ctx, z)
        assert e.value.code == H.HE_ELEVEL
        # malformed layout: a block pointing at a channel the image does not have
        bad = H.he_layout_image(4, 16, N)
        bad.chan[0] = 9
        with pytest.raises(H.HEError) as e:
            H.he_conv_create(ctx, bad, W, None, 1, 1, 3, pr.scale)
        assert e.value.code == H.HE_EINVAL
        H.he_conv_destroy(conv)
        for c in x + y + [ct, z]:
            H.he_ct_free(c)
    finally:
        H.he_debug_fail_alloc(-1)
        H.he_ctx_destroy(ctx)


def test_range_sanitizer_counts_out_of_range_words():
    import torch
    from paper_2306_09189_gb300 import hegpu as H, host
    pr = host.params(12, 6, 2, 3, 50, 40, 50, seed=3)
    ctx = H.he_ctx_create(pr)
    try:
        N, n = 2048, 4096
        a = H.he_ct_alloc(ctx, 3)
        H.he_encrypt(ctx, np.random.default_rng(2).uniform(-1, 1, N), 3, pr.scale, 5, a)
        assert H.he_ct_check_range(ctx, a) == 0
        # a buffer of all-ones words (2^64 - 1 is above every prime) wrapped as a ciphertext
        buf = torch.full((2 * 4 * n,), -1, dtype=torch.int64, device="cuda")
        w = H.he_ct_wrap(ctx, buf.data_ptr(), buf.numel() * 8, 3)
        assert H.he_ct_check_range(ctx, w) == 2 * 4 * n
        buf[: 4 * n] = 0                                  # poly 0 in range now
        assert H.he_ct_check_range(ctx, w) == 4 * n
        H.he_ct_free(w)
        H.he_ct_free(a)
    finally:
        H.he_ctx_destroy(ctx)
