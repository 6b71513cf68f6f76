"""CUDA-graph capture and the fused-stage autotuner on the GPU.

A captured layer step (fused conv + bias, then the Chebyshev GELU) replays to the same bits as
the eager step, and its kernel count per replay is what the eager step launched.  A capture
that would need a first-run allocation fails cleanly.  The autotuner's choice never changes
the bits."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _setup(H, host):
    pr = host.params(12, 10, 4, 3, 50, 40, 50, seed=4)
    ctx = H.he_ctx_create(pr)
    N = 2048
    rng = np.random.default_rng(2)
    c, m = 4, 16
    W = rng.uniform(-0.2, 0.2, (c, c, 3, 3))
    b = rng.uniform(-0.1, 0.1, c)
    lay = H.he_layout_image(c, m, N)
    conv = H.he_conv_create(ctx, lay, W, b, 1, 1, 9, pr.scale)
    H.he_keygen_rotations(ctx, H.he_conv_rotations(conv))
    H.he_keygen_relin(ctx)
    x = host.encrypt_image(ctx, lay, rng.uniform(0, 1, (c, m, m)), 9, pr.scale, nonce0=3)[0]
    y = H.he_ct_alloc(ctx, 8)
    cheb = host.chebyshev_coeffs("gelu", 8, -8.0, 8.0)
    return pr, ctx, conv, x, y, cheb


def test_graph_replay_is_bit_exact():
    from paper_2306_09189_gb300 import hegpu as H, host
    pr, ctx, conv, x, y, cheb = _setup(H, host)
    try:
        stream = torch.cuda.Stream()                # the default stream cannot be captured
        torch.cuda.synchronize()
        with pytest.raises(H.HEError):
            H.he_graph_begin(ctx, torch.cuda.default_stream())

        def step():
            H.he_conv_run(ctx, conv, [x], [y], H.HE_FUSED, stream)
            H.he_poly_eval(ctx, y, cheb, pr.scale, stream)

        # a capture before the first run would allocate: refused, stream left usable
        H.he_graph_begin(ctx, stream)
        try:
            with pytest.raises(H.HEError) as e:
                step()
            assert e.value.code == H.HE_ESTATE
        finally:
            with pytest.raises(H.HEError):          # the capture always ends; the graph is discarded
                H.he_graph_end(ctx, stream)
        step()
        torch.cuda.synchronize()
        want = H.he_ct_export_coeffs(ctx, y, 4096, stream)
        l0 = H.he_kernel_launches()
        step()
        torch.cuda.synchronize()
        eager = H.he_kernel_launches() - l0
        H.he_graph_begin(ctx, stream)
        try:
            step()
        finally:
            g = H.he_graph_end(ctx, stream)
        assert H.he_graph_kernels(g) == eager
        lv, sc = H.he_ct_level(y), H.he_ct_scale(y)
        for _ in range(2):
            H.he_ct_zero(y, lv, sc, stream)         # clobber the output between replays
            l0 = H.he_kernel_launches()
            H.he_graph_launch(g, stream)
            torch.cuda.synchronize()
            assert H.he_kernel_launches() - l0 == eager
            assert np.array_equal(H.he_ct_export_coeffs(ctx, y, 4096, stream), want)
        H.he_graph_destroy(g)
        # a graph captured while tracing times each traced launch inside it (the fused form,
        # chosen explicitly: the autotuner may prefer the split form at this size)
        H.he_ctx_set_option(ctx, H.HE_OPT_KEY_STREAM, H.HE_KEY_STREAM_LDG)
        step()                                    # builds the fused tables outside the capture
        torch.cuda.synchronize()
        H.he_trace_start("ipmac")
        H.he_graph_begin(ctx, stream)
        try:
            step()
            step()
        finally:
            g2 = H.he_graph_end(ctx, stream)
        H.he_graph_launch(g2, stream)
        tr = H.he_trace_stop()
        assert tr["launches"] == 2 and tr["ms"] > 0 and tr["bytes"] > 0
        assert np.array_equal(H.he_ct_export_coeffs(ctx, y, 4096, stream), want)
        H.he_graph_destroy(g2)
        H.he_ctx_check(ctx, stream)
    finally:
        H.he_conv_destroy(conv)
        H.he_ct_free(x)
        H.he_ct_free(y)
        H.he_ctx_destroy(ctx)


def test_autotuner_choice_keeps_bits():
    from paper_2306_09189_gb300 import hegpu as H, host
    pr, ctx, conv, x, y, cheb = _setup(H, host)
    try:
        outs = {}
        for ks in (H.HE_KEY_STREAM_AUTO, H.HE_KEY_STREAM_LDG, H.HE_KEY_STREAM_TMA, H.HE_KEY_STREAM_SPLIT,
                   H.HE_KEY_STREAM_CP, H.HE_KEY_STREAM_LDG1, H.HE_KEY_STREAM_PK, H.HE_KEY_STREAM_PK3,
                   H.HE_KEY_STREAM_PKP, H.HE_KEY_STREAM_SPLITM, H.HE_KEY_STREAM_PK1,
                   H.HE_KEY_STREAM_PKT, H.HE_KEY_STREAM_PK3L):
            H.he_ctx_set_option(ctx, H.HE_OPT_KEY_STREAM, ks)
            assert H.he_ctx_get_option(ctx, H.HE_OPT_KEY_STREAM) == ks
            H.he_conv_run(ctx, conv, [x], [y], H.HE_FUSED)
            H.he_ctx_check(ctx)
            outs[ks] = H.he_ct_export_coeffs(ctx, y, 4096)
        assert all(np.array_equal(outs[H.HE_KEY_STREAM_AUTO], v) for v in outs.values())
        log = H.he_ctx_tuning_log(ctx)
        assert "conv 4->4 16x16" in log and "->" in log
        with pytest.raises(H.HEError):
            H.he_ctx_set_option(ctx, H.HE_OPT_KEY_STREAM, 99)
    finally:
        H.he_conv_destroy(conv)
        H.he_ct_free(x)
        H.he_ct_free(y)
        H.he_ctx_destroy(ctx)
