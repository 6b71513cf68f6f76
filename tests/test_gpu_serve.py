"""Serving on the GPU: each request's result is the same alone and in a concurrent mix (bit for
bit), and decrypts to the FP64 network with the same polynomial."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_results_identical_alone_and_in_the_mix():
    from paper_2306_09189_gb300 import hegpu as H, host
    from paper_2306_09189_gb300.serve import (Stack, Server, Request, encrypt_request, decrypt_result,
                                              plaintext_stack, latency_stats)
    # ring 2^12, 17 primes: two layers of conv (1 level) + degree-16 GELU (5) + pool (2)
    pr = host.params(12, 17, 5, 4, 50, 40, 50, seed=7)
    root = H.he_ctx_create(pr)
    try:
        H.he_keygen_relin(root)
        layers = workloads.serving_stack(0, widths=(4, 8, 8), m=16)
        cheb = host.chebyshev_coeffs("gelu", 16, -8.0, 8.0)
        stacks = {m: Stack(root, m, layers, cheb, 16, pr.scale) for m in (8, 16)}
        rng = np.random.default_rng(1)
        imgs, reqs = [], []
        for i, m in enumerate([16, 8, 16, 8]):
            img = rng.uniform(0, 1, (4, m, m))
            img[3] = 0.0
            imgs.append(img)
            reqs.append(Request(i, 0.0, m, encrypt_request(root, stacks[m], img, 100 * i)))
        alone = Server(root, stacks, 1)
        solo = []
        for r in reqs:
            solo += alone.serve([Request(r.rid, 0.0, r.m, r.coeffs)])
        mix = Server(root, stacks, 3)
        both = mix.serve([Request(r.rid, 0.001 * r.rid, r.m, r.coeffs) for r in reqs])
        for a, b in zip(solo, both):
            assert a.rid == b.rid
            for x, y in zip(a.result, b.result):
                assert np.array_equal(x, y)
        for r, img in zip(both, imgs):
            got = decrypt_result(root, stacks[r.m], r.result)
            want = plaintext_stack(img, layers, cheb)
            assert got.shape == want.shape
            assert np.abs(got - want).max() <= 2.0 ** -20 * (want.max() - want.min())
        st = latency_stats(both)
        assert st["n"] == 4 and st["p99_ms"] >= st["p50_ms"] > 0
        alone.destroy()
        mix.destroy()
        for s in stacks.values():
            s.destroy()
    finally:
        H.he_ctx_destroy(root)


def test_parameters_with_too_small_special_modulus_are_rejected():
    from paper_2306_09189_gb300 import hegpu as H, host
    with pytest.raises(H.HEError) as e:
        H.he_ctx_create(host.params(12, 17, 3, 4, 50, 40, 50))      # P ~ 2^150 < digit ~ 2^210
    assert e.value.code == H.HE_EINVAL and "special primes" in str(e.value)


def test_forked_context_shares_keys_and_matches_parent():
    from paper_2306_09189_gb300 import hegpu as H, host
    pr = host.params(12, 6, 2, 3, 50, 40, 50, seed=3)
    root = H.he_ctx_create(pr)
    try:
        fork = H.he_ctx_fork(root)
        H.he_keygen_rotations(root, [5])          # generated after the fork: still shared
        z = np.random.default_rng(0).uniform(-1, 1, 2048)
        a, b, c = H.he_ct_alloc(root, 5), H.he_ct_alloc(root, 5), H.he_ct_alloc(fork, 5)
        H.he_encrypt(root, z, 5, 2.0 ** 40, 1, a)
        H.he_rotate(root, a, 5, b)
        H.he_rotate(fork, a, 5, c)
        assert np.array_equal(H.he_ct_export_coeffs(root, b, 4096), H.he_ct_export_coeffs(fork, c, 4096))
        assert H.he_key_bytes(fork) == H.he_key_bytes(root) > 0
        for x in (a, b, c):
            H.he_ct_free(x)
        H.he_ctx_destroy(fork)
    finally:
        H.he_ctx_destroy(root)


def _batched_vs_alone(pr, level, widths, sizes, order, max_batch):
    from paper_2306_09189_gb300 import hegpu as H, host
    from paper_2306_09189_gb300.serve import (Stack, Server, BatchServer, Request, encrypt_request,
                                              decrypt_result, plaintext_stack)
    root = H.he_ctx_create(pr)
    try:
        H.he_keygen_relin(root)
        layers = workloads.serving_stack(0, widths=widths, m=max(sizes))
        cheb = host.chebyshev_coeffs("gelu", 16, -8.0, 8.0)
        stacks = {m: Stack(root, m, layers, cheb, level, pr.scale) for m in sizes}
        rng = np.random.default_rng(5)
        imgs, reqs = [], []
        for i, m in enumerate(order):
            img = rng.uniform(0, 1, (4, m, m))
            img[3] = 0.0
            imgs.append(img)
            reqs.append(Request(i, 0.0, m, encrypt_request(root, stacks[m], img, 300 + 10 * i)))
        alone = Server(root, stacks, 1)
        solo = []
        for r in reqs:
            solo += alone.serve([Request(r.rid, 0.0, r.m, r.coeffs)])
        batch = BatchServer(root, stacks, max_batch=max_batch, slots_per_res=max_batch)
        # a burst, then a request arriving while the burst is on the GPU
        arrivals = [0.0] * (len(reqs) - 1) + [0.002]
        got = batch.serve([Request(r.rid, a, r.m, r.coeffs) for r, a in zip(reqs, arrivals)])
        assert max(size for _, _, size in batch.steps) > 1            # requests shared launches
        for a, b in zip(solo, got):
            assert a.rid == b.rid and b.finish >= b.start >= b.arrival
            for x, y in zip(a.result, b.result):
                assert np.array_equal(x, y)                          # the same bits as alone
        for r, img in zip(got, imgs):
            out = decrypt_result(root, stacks[r.m], r.result)
            want = plaintext_stack(img, layers, cheb)
            assert np.abs(out - want).max() <= 2.0 ** -20 * (want.max() - want.min())
        batch.destroy()
        alone.destroy()
        for s in stacks.values():
            s.destroy()
    finally:
        H.he_ctx_destroy(root)


def test_batched_server_gives_each_request_its_alone_bits():
    """Stage-granularity batching at ring 2^12: two layers, two resolutions, a burst of five."""
    from paper_2306_09189_gb300 import host
    _batched_vs_alone(host.params(12, 17, 5, 4, 50, 40, 50, seed=7), 16, (4, 8, 8), (8, 16),
                      [16, 8, 16, 16, 8], 4)


def test_batched_server_full_ring():
    """The same at n = 2^16 with the benchmark's parameters (20 + 5 primes): one layer on
    32 x 32 images, three requests batched."""
    from paper_2306_09189_gb300 import host
    _batched_vs_alone(host.cifar_params(seed=0), 19, (4, 8), (32,), [32, 32, 32], 2)
