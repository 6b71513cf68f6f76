"""Bootstrapping on the GPU against the oracle (oracle/bootstrap.py), word for word.

The oracle's plaintexts (complex diagonals of the merged special-DFT levels, encoded by the
oracle) and its Chebyshev coefficients are imported, so every step must give the oracle's bits:
ModRaise, conjugation, monomial products, each linear level, the whole bootstrap at ring 2^12,
and ModRaise plus the first CoeffToSlot level at the full ring.  With the library's own
encodings the bootstrap must decrypt to the message within the stated precision, at ring 2^12
and at the full ring 2^16 (23-level chain, 50-bit primes, weight-64 secret).
"""
import math

import numpy as np
import pytest

from oracle import bootstrap as B
from oracle.ckks import Context
from oracle.params import BOOT12, B24
from paper_2306_09189_gb300 import hegpu as H
from tests._hegpu_util import GpuCtx, assert_ct_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def boot12():
    o = Context(BOOT12)
    plan = B.BootPlan(o)
    B.gen_boot_keys(o, plan)
    g = GpuCtx(BOOT12)
    bt = H.he_boot_create(g.h)
    H.he_keygen_rotations(g.h, H.he_boot_rotations(bt))
    H.he_keygen_conjugation(g.h)
    H.he_keygen_relin(g.h)
    yield o, plan, g, bt
    H.he_boot_destroy(bt)
    g.close()


def _import_oracle(o, plan, bt):
    for st, name in ((0, "cts"), (1, "stc")):
        levels = plan.cts if st == 0 else plan.stc
        for i, lv in enumerate(levels):
            pts = plan.plaintexts(o, name, i)
            keys = [(gi, j) for gi in lv.giants for j in sorted(lv.baby[gi])]
            assert H.he_boot_n_plaintexts(bt, st, i) == len(keys)
            H.he_boot_import_plaintexts(bt, st, i, np.stack([pts[k] for k in keys]))
    H.he_boot_import_coeffs(bt, plan.coeffs)


def test_plan_matches_the_oracle(boot12):
    o, plan, g, bt = boot12
    assert sorted(H.he_boot_rotations(bt).tolist()) == plan.rotations()
    info = H.he_boot_info(bt)
    assert info["out_level"] == plan.out_level
    assert info["evalmod_level"] == plan.evalmod_level
    assert info["stc_level"] == plan.stc_level[0]
    for st, levels in ((0, plan.cts), (1, plan.stc)):
        for i, lv in enumerate(levels):
            assert H.he_boot_n_plaintexts(bt, st, i) == sum(len(b) for b in lv.baby.values())


def test_sparse_secret_keys_and_primitives_bit_exact(boot12):
    o, plan, g, bt = boot12
    n, L = o.n, o.L
    rng = np.random.default_rng(1)
    z = rng.uniform(-1, 1, o.N)
    ct = o.encrypt(z, 0, 2.0 ** 40, nonce=3)
    d = g.upload(ct)
    x = g.ct(L)
    H.he_modraise(g.h, d, L, x)
    assert_ct_equal(g.download(x), o.modraise(ct))
    y5 = o.encrypt(z, 5, 2.0 ** 45, nonce=4)
    d5 = g.upload(y5)
    c5 = g.ct(5)
    H.he_conjugate(g.h, d5, c5)
    assert_ct_equal(g.download(c5), o.conjugate(y5))
    for e in (n // 2, 3 * n // 2, 5, n + 3, -7):
        m = g.upload(y5)
        H.he_mul_monomial(g.h, m, e)
        assert_ct_equal(g.download(m), o.mul_monomial(y5, e))


def test_rotation_key_of_sparse_secret_bit_exact(boot12):
    o, plan, g, bt = boot12
    r = plan.rotations()[0]
    got = H.he_key_export(g.h, r, (BOOT12.dnum, 2, o.L + 1 + o.K, o.n))
    want = o.export_key(o.galois(r))
    assert np.array_equal(got, want)


def test_linear_levels_bit_exact(boot12):
    o, plan, g, bt = boot12
    _import_oracle(o, plan, bt)
    rng = np.random.default_rng(2)
    from oracle.encode import encode_complex
    for st, name, levels, lvls in ((0, "cts", plan.cts, plan.cts_level), (1, "stc", plan.stc, plan.stc_level)):
        for i, lv in enumerate(levels):
            z = rng.uniform(-1, 1, o.N) + 1j * rng.uniform(-1, 1, o.N)
            S = 2.0 ** 45
            ct = o.encrypt_coeffs(encode_complex(z, o.n, S), lvls[i], S, nonce=20 + i + 10 * st)
            want = B.lintrans_he(o, ct, lv, plan.plaintexts(o, name, i))
            d = g.upload(ct)
            out = g.ct(lvls[i])
            H.he_boot_lintrans(g.h, bt, st, i, d, out)
            assert_ct_equal(g.download(out), want)
            assert H.he_ct_scale(out) == want.scale


def test_bootstrap_bit_exact_ring_2_12(boot12):
    o, plan, g, bt = boot12
    _import_oracle(o, plan, bt)
    rng = np.random.default_rng(3)
    z = rng.uniform(-1, 1, o.N)
    ct = o.encrypt(z, 0, 2.0 ** 40, nonce=30)
    want = B.bootstrap(o, ct, plan)
    d = g.upload(ct)
    out = g.ct(plan.out_level)
    H.he_bootstrap(g.h, bt, d, out)
    assert H.he_ct_level(out) == plan.out_level
    assert H.he_ct_scale(out) == want.scale
    assert_ct_equal(g.download(out), want)
    err = np.max(np.abs(o.decrypt(want) - z))
    assert err < 2.0 ** -15


def test_bootstrap_bit_exact_from_level_3(boot12):
    # an input above level 0 goes to level 0 at scale q_0 / 2^10 first (exact retarget)
    o, plan, g, bt = boot12
    _import_oracle(o, plan, bt)
    rng = np.random.default_rng(6)
    z = rng.uniform(-1, 1, o.N)
    ct = o.encrypt(z, 3, BOOT12.scale, nonce=31)
    want = B.bootstrap(o, ct, plan)
    d = g.upload(ct)
    out = g.ct(plan.out_level)
    H.he_bootstrap(g.h, bt, d, out)
    assert H.he_ct_scale(out) == want.scale
    assert_ct_equal(g.download(out), want)
    assert np.max(np.abs(o.decrypt(want) - z)) < 2.0 ** -15


def test_meta_bootstrap_bit_exact_ring_2_12(boot12):
    o, plan, g, bt = boot12
    _import_oracle(o, plan, bt)
    rng = np.random.default_rng(7)
    z = rng.uniform(-1, 1, o.N)
    ct = o.encrypt(z, 0, 2.0 ** 40, nonce=32)
    want = B.meta_bootstrap(o, ct, plan)
    d = g.upload(ct)
    out = g.ct(plan.out_level)
    H.he_bootstrap_meta(g.h, bt, d, out, 10)
    assert H.he_ct_level(out) == plan.out_level - 1
    assert H.he_ct_scale(out) == want.scale
    assert_ct_equal(g.download(out), want)
    one = np.max(np.abs(o.decrypt(B.bootstrap(o, ct, plan)) - z))
    assert np.max(np.abs(o.decrypt(want) - z)) < one / 16


def test_bootstrap_own_encoding_precision_ring_2_12():
    o = Context(BOOT12)
    g = GpuCtx(BOOT12)
    try:
        bt = H.he_boot_create(g.h)
        H.he_keygen_rotations(g.h, H.he_boot_rotations(bt))
        H.he_keygen_conjugation(g.h)
        H.he_keygen_relin(g.h)
        rng = np.random.default_rng(4)
        z = rng.uniform(-1, 1, o.N)
        d = g.upload(o.encrypt(z, 0, 2.0 ** 40, nonce=40))
        lvl = H.he_boot_info(bt)["out_level"]
        out = g.ct(lvl)
        H.he_bootstrap(g.h, bt, d, out)
        got = H.he_decrypt(g.h, out, o.N)
        err = np.max(np.abs(got - z))
        assert err < 2.0 ** -15, err
        # twice in a row (the plan's buffers are reused): same words
        out2 = g.ct(lvl)
        H.he_bootstrap(g.h, bt, d, out2)
        assert np.array_equal(g.download(out), g.download(out2))
        H.he_boot_destroy(bt)
    finally:
        g.close()


def test_bootstrap_full_ring_precision_and_first_level_bit_exact():
    o = Context(B24)
    plan = B.BootPlan(o)
    g = GpuCtx(B24)
    try:
        bt = H.he_boot_create(g.h)
        rots = H.he_boot_rotations(bt)
        assert sorted(rots.tolist()) == plan.rotations()
        H.he_keygen_rotations(g.h, rots)
        H.he_keygen_conjugation(g.h)
        H.he_keygen_relin(g.h)
        rng = np.random.default_rng(5)
        z = rng.uniform(-1, 1, o.N)
        ct = o.encrypt(z, 0, 2.0 ** 40, nonce=50)
        d = g.upload(ct)
        out = g.ct(plan.out_level)
        H.he_bootstrap(g.h, bt, d, out)
        assert H.he_ct_level(out) == plan.out_level == B24.n_q - 1 - 15
        err = np.max(np.abs(H.he_decrypt(g.h, out, o.N) - z))
        assert err < 2.0 ** -12, err
        meta = g.ct(plan.out_level)
        H.he_bootstrap_meta(g.h, bt, d, meta, 10)
        err2 = np.max(np.abs(H.he_decrypt(g.h, meta, o.N) - z))
        assert err2 < err / 16, (err, err2)
        # ModRaise and the first CoeffToSlot level at the full ring, word for word
        x = g.ct(o.L)
        H.he_modraise(g.h, d, o.L, x)
        ox = o.modraise(ct)
        assert_ct_equal(g.download(x), ox)
        ox.scale = float(o.q[0]) * plan.cfg.K
        H.he_ct_set_scale(x, ox.scale)
        for a in plan.cts[0].rotations():
            o.gen_rotation_key(a)
        pts = plan.plaintexts(o, "cts", 0)
        lv = plan.cts[0]
        keys = [(gi, j) for gi in lv.giants for j in sorted(lv.baby[gi])]
        H.he_boot_import_plaintexts(bt, 0, 0, np.stack([pts[k] for k in keys]))
        y = g.ct(o.L)
        H.he_boot_lintrans(g.h, bt, 0, 0, x, y)
        assert_ct_equal(g.download(y), B.lintrans_he(o, ox, lv, pts))
        H.he_boot_destroy(bt)
    finally:
        g.close()


def test_network_deeper_than_the_chain():
    """conv3x3+BN -> GELU -> bootstrap -> conv3x3+BN -> GELU on a 4x32x32 image at ring 2^16:
    12 levels of layers on an 8-level budget, decrypted against the FP64 network with the same
    polynomial."""
    import workloads
    from paper_2306_09189_gb300 import host
    torch = pytest.importorskip("torch")
    pr = B24
    wl = workloads.cifar_conv_bn(0, c=4, m=32)
    cheb = host.chebyshev_coeffs("gelu", 16, -workloads.GELU_BOUND, workloads.GELU_BOUND)
    act = lambda v: np.polynomial.chebyshev.chebval(v, cheb)
    conv = lambda x, W, b: torch.nn.functional.conv2d(torch.tensor(x)[None], torch.tensor(W), padding=1)[0].numpy() + b[:, None, None]
    y1 = act(conv(wl.x, wl.W, wl.bias))
    rng = np.random.default_rng(11)
    W2 = rng.uniform(-1 / 6, 1 / 6, (4, 4, 3, 3))
    W2f, b2f = workloads.fold_bn(y1, W2, 1)
    y2 = act(conv(y1, W2f, b2f))
    g = GpuCtx(pr)
    try:
        ctx = g.h
        bt = H.he_boot_create(ctx)
        info = H.he_boot_info(bt)
        lay = H.he_layout_image(4, 32, g.N)
        level = 7
        xs = host.encrypt_image(ctx, lay, wl.x, level, pr.scale, nonce0=1)
        c1 = H.he_conv_create(ctx, lay, wl.W, wl.bias, 1, 1, level, pr.scale)
        lay1 = H.he_conv_out_layout(c1)
        H.he_keygen_rotations(ctx, sorted(set(H.he_boot_rotations(bt).tolist()) | set(H.he_conv_rotations(c1))))
        H.he_keygen_conjugation(ctx)
        H.he_keygen_relin(ctx)
        a1 = [H.he_ct_alloc(ctx, level - 1) for _ in range(lay1.n_shards)]
        H.he_conv_run(ctx, c1, xs, a1, H.HE_FUSED)
        for ct in a1:
            H.he_poly_eval_ps(ctx, ct, cheb, pr.scale)
        assert H.he_ct_level(a1[0]) == 1                 # the chain is spent
        b1 = [H.he_ct_alloc(ctx, info["out_level"]) for _ in a1]
        for src, dst in zip(a1, b1):
            H.he_bootstrap(ctx, bt, src, dst)
        lv2 = H.he_ct_level(b1[0])
        assert lv2 == info["out_level"]
        c2 = H.he_conv_create(ctx, lay1, W2f, b2f, 1, 1, lv2, H.he_ct_scale(b1[0]))
        H.he_keygen_rotations(ctx, H.he_conv_rotations(c2))
        lay2 = H.he_conv_out_layout(c2)
        a2 = [H.he_ct_alloc(ctx, lv2 - 1) for _ in range(lay2.n_shards)]
        H.he_conv_run(ctx, c2, b1, a2, H.HE_FUSED)
        for ct in a2:
            H.he_poly_eval_ps(ctx, ct, cheb, pr.scale)
        got = host.decrypt_image(ctx, lay2, a2)
        err = np.max(np.abs(got - y2))
        rng_y = np.max(y2) - np.min(y2)
        assert err < 2.0 ** -8 * rng_y, (err, rng_y)
        for ct in xs + a1 + b1 + a2:
            H.he_ct_free(ct)
        H.he_conv_destroy(c1)
        H.he_conv_destroy(c2)
        H.he_boot_destroy(bt)
    finally:
        g.close()


def test_bootstrap_errors_leave_the_context_usable(boot12):
    from oracle.params import TOY
    o, plan, g, bt = boot12
    # a chain too short for the 15 levels
    small = GpuCtx(TOY)
    try:
        with pytest.raises(H.HEError) as e:
            H.he_boot_create(small.h)
        assert e.value.code == H.HE_ELEVEL
    finally:
        small.close()
    ct = o.encrypt(np.zeros(o.N), 0, 2.0 ** 40, nonce=60)
    d = g.upload(ct)
    # an output below the bootstrap's output level
    low = g.ct(0)
    if plan.out_level > 0:
        with pytest.raises(H.HEError) as e:
            H.he_bootstrap(g.h, bt, d, low)
        assert e.value.code == H.HE_ELEVEL
    # a bad linear level index, a wrong coefficient count
    with pytest.raises(H.HEError):
        H.he_boot_n_plaintexts(bt, 0, 99)
    with pytest.raises(H.HEError):
        H.he_boot_import_coeffs(bt, np.zeros(5))
    # the plan still runs
    out = g.ct(plan.out_level)
    H.he_bootstrap(g.h, bt, d, out)
    assert H.he_ct_level(out) == plan.out_level


def test_full_ring_bootstrap_equals_the_oracle_word_for_word():
    """The whole bootstrap at ring 2^16 on the oracle's plaintexts and coefficients: every output
    word equals the oracle's (SHA-256 of the words against tests/golden/bootstrap_b24.json, which
    tests/golden/make_bootstrap_golden.py wrote from the oracle alone on the same input)."""
    import hashlib
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bootstrap_b24.json")) as f:
        gold = json.load(f)
    o = Context(B24)
    plan = B.BootPlan(o)
    h = hashlib.sha256()
    for name, levels in (("cts", plan.cts), ("stc", plan.stc)):
        for i, lv in enumerate(levels):
            pts = plan.plaintexts(o, name, i)
            for gi in lv.giants:
                for j in sorted(lv.baby[gi]):
                    h.update(np.ascontiguousarray(pts[(gi, j)], dtype="<i8").tobytes())
    assert h.hexdigest() == gold["sha256_plaintexts"], \
        "this machine's numpy encodes the diagonals differently from the one that wrote the golden file"
    z = np.random.default_rng(gold["seed_z"]).uniform(-1, 1, o.N)
    ct = o.encrypt(z, 0, gold["input_scale"], nonce=gold["nonce"])
    g = GpuCtx(B24)
    try:
        bt = H.he_boot_create(g.h)
        H.he_keygen_rotations(g.h, H.he_boot_rotations(bt))
        H.he_keygen_conjugation(g.h)
        H.he_keygen_relin(g.h)
        _import_oracle(o, plan, bt)
        out = g.ct(plan.out_level)
        H.he_bootstrap(g.h, bt, g.upload(ct), out)
        assert H.he_ct_level(out) == gold["out_level"]
        assert H.he_ct_scale(out) == gold["out_scale"]
        words = np.ascontiguousarray(g.download(out), dtype="<u8")
        assert words[:, :, :4].tolist() == gold["first_words"]
        assert hashlib.sha256(words.tobytes()).hexdigest() == gold["sha256_words"]
        # the bootstrap with its error bootstrapped and subtracted, word for word too
        meta = g.ct(plan.out_level)
        H.he_bootstrap_meta(g.h, bt, g.upload(ct), meta, gold["meta"]["kb"])
        assert H.he_ct_level(meta) == gold["meta"]["out_level"]
        assert H.he_ct_scale(meta) == gold["meta"]["out_scale"]
        mw = np.ascontiguousarray(g.download(meta), dtype="<u8")
        assert mw[:, :, :4].tolist() == gold["meta"]["first_words"]
        assert hashlib.sha256(mw.tobytes()).hexdigest() == gold["meta"]["sha256_words"]
        H.he_boot_destroy(bt)
    finally:
        g.close()
