"""Linear and pool-linear head on the GPU against the oracle, bit for bit.

The oracle's plan (row j of the weights on the first copy of every pixel, rotate-and-add over
all slots, one-hot masks) is imported as integer plaintexts; the GPU output must equal
``linear_head``'s ciphertext limb for limb and decrypt to the FP64 dot products."""
import numpy as np
import pytest
import torch

from oracle import layers as Ly
from oracle.params import Params
from oracle.ckks import Context
from oracle.encode import encode

pytestmark = pytest.mark.gpu

MID = Params(log_n=12, n_q=6, n_p=2, dnum=3, q0_bits=50, q_bits=40, p_bits=50,
             scale=2.0 ** 40, seed=5)


@pytest.fixture(scope="module")
def mid():
    from tests._hegpu_util import GpuCtx
    o = Context(MID)
    g = GpuCtx(MID)
    yield o, g
    g.close()


@pytest.mark.parametrize("c,m,n_out,pool,level", [(16, 8, 10, True, 4),    # ResNet tail: one shard, 2 copies
                                                  (8, 16, 4, True, 3),     # 4 channels per shard, 2 shards
                                                  (2, 64, 3, False, 2),    # channel shards, full weights
                                                  (3, 28, 5, False, 3)])   # padded frame, full weights
def test_linear_head_bit_exact(mid, c, m, n_out, pool, level):
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = mid
    rng = np.random.default_rng(c * 13 + m)
    x = rng.uniform(0, 1, (c, m, m))
    W = rng.uniform(-1, 1, (n_out, c) if pool else (n_out, c, m, m))
    b = rng.uniform(-1, 1, n_out)
    lin = Ly.image_layout(c, m, o.N)
    plan = (Ly.pool_linear_plan if pool else Ly.linear_plan)(lin, W, b)
    cts = [o.encrypt(Ly.pack(lin, x)[u], level, nonce=300 + u) for u in range(lin.n_shards)]
    w_pts, m_pts = Ly.linear_plaintexts(plan, o.n, *Ly.linear_scales(o, level))
    zb = np.zeros(o.N)
    zb[:n_out] = b
    b_pt = encode(zb, o.n, o.pr.scale)
    ref = Ly.linear_he(o, plan, cts, w_pts, m_pts, b_pt)

    lay = H.he_layout_image(c, m, o.N)
    create = H.he_pool_linear_create if pool else H.he_linear_create
    L = create(g.h, lay, W, b, level, o.pr.scale)
    rots = H.he_linear_rotations(L)
    assert list(rots) == plan.amounts()
    assert H.he_linear_out_level(L) == level - 2
    assert H.he_linear_keyswitches(L) == n_out * len(plan.amounts())
    H.he_keygen_rotations(g.h, rots)
    ins = [g.upload(ct) for ct in cts]
    out = g.ct(level)
    # the library's own encoding first: decrypts to the FP64 head
    H.he_linear_run(g.h, L, ins, out)
    H.he_ctx_check(g.h)
    if pool:
        want = W @ x.mean(axis=(1, 2)) + b
    else:
        want = W.reshape(n_out, -1) @ x.reshape(-1) + b
    got = H.he_decrypt(g.h, out, o.N)
    tol = 2.0 ** -20 * (want.max() - want.min())
    assert np.abs(got[:n_out] - want).max() <= tol and np.abs(got[n_out:]).max() <= tol
    # the oracle's integer plaintexts: bit for bit
    H.he_linear_import_plaintexts(L, np.stack([np.stack([w_pts[(j, u)] for u in range(lin.n_shards)])
                                               for j in range(n_out)]),
                                  np.stack([m_pts[j] for j in range(n_out)]), b_pt)
    for ks in (H.HE_KEY_STREAM_AUTO, H.HE_KEY_STREAM_AUTO, H.HE_KEY_STREAM_PK, H.HE_KEY_STREAM_PK3,
               H.HE_KEY_STREAM_PKP, H.HE_KEY_STREAM_LDG):
        H.he_ctx_set_option(g.h, H.HE_OPT_KEY_STREAM, ks)   # a second run reuses the built stages
        H.he_linear_run(g.h, L, ins, out)
        H.he_ctx_check(g.h)
        assert H.he_ct_level(out) == ref.level and H.he_ct_scale(out) == ref.scale
        assert_ct_equal(g.download(out), ref)
    H.he_ctx_set_option(g.h, H.HE_OPT_KEY_STREAM, H.HE_KEY_STREAM_AUTO)
    # a shard at another level is refused
    bad = [g.ct(level - 1) for _ in range(lin.n_shards)]
    with pytest.raises(H.HEError) as e:
        H.he_linear_run(g.h, L, bad, out)
    assert e.value.code == H.HE_ELEVEL
    H.he_linear_destroy(L)


def test_linear_head_refuses_bad_plans(mid):
    from paper_2306_09189_gb300 import hegpu as H
    o, g = mid
    lay = H.he_layout_image(4, 8, o.N)
    with pytest.raises(H.HEError) as e:                 # one level is not enough
        H.he_pool_linear_create(g.h, lay, np.ones((2, 4)), None, 1, o.pr.scale)
    assert e.value.code == H.HE_ELEVEL
    with pytest.raises(H.HEError) as e:                 # more outputs than slots
        H.he_pool_linear_create(g.h, lay, np.ones((o.N + 1, 4)), None, 3, o.pr.scale)
    assert e.value.code == H.HE_EINVAL


@pytest.mark.parametrize("c,m,n_out,pool,level", [(16, 8, 10, True, 4), (8, 16, 4, True, 3),
                                                  (2, 64, 3, False, 2), (3, 28, 5, False, 3)])
def test_packed_head_bit_exact(mid, c, m, n_out, pool, level):
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import assert_ct_equal
    o, g = mid
    rng = np.random.default_rng(c * 17 + m)
    x = rng.uniform(0, 1, (c, m, m))
    W = rng.uniform(-1, 1, (n_out, c) if pool else (n_out, c, m, m))
    b = rng.uniform(-1, 1, n_out)
    lin = Ly.image_layout(c, m, o.N)
    plan = (Ly.pool_linear_plan if pool else Ly.linear_plan)(lin, W, b)
    cts = [o.encrypt(Ly.pack(lin, x)[u], level, nonce=500 + u) for u in range(lin.n_shards)]
    w_pts, m_pt = Ly.linear_packed_plaintexts(plan, o.n, *Ly.linear_scales(o, level))
    zb = np.zeros(o.N)
    zb[:n_out] = b
    b_pt = encode(zb, o.n, o.pr.scale)
    ref = Ly.linear_packed_he(o, plan, cts, w_pts, m_pt, b_pt)
    lay = H.he_layout_image(c, m, o.N)
    create = H.he_pool_linear_create_packed if pool else H.he_linear_create_packed
    L = create(g.h, lay, W, b, level, o.pr.scale)
    npk = Ly.linear_packed_width(n_out)
    assert sorted(H.he_linear_rotations(L)) == sorted(list(range(1, npk)) + Ly.linear_packed_shifts(plan))
    assert H.he_linear_keyswitches(L) == lin.n_shards * (npk - 1) + len(Ly.linear_packed_shifts(plan))
    H.he_keygen_rotations(g.h, H.he_linear_rotations(L))
    ins = [g.upload(ct) for ct in cts]
    out = g.ct(level)
    H.he_linear_run(g.h, L, ins, out)                  # the library's own encoding
    H.he_ctx_check(g.h)
    want = W @ x.mean(axis=(1, 2)) + b if pool else W.reshape(n_out, -1) @ x.reshape(-1) + b
    got = H.he_decrypt(g.h, out, o.N)
    tol = 2.0 ** -20 * (want.max() - want.min())
    assert np.abs(got[:n_out] - want).max() <= tol and np.abs(got[n_out:]).max() <= tol
    H.he_linear_import_plaintexts(L, np.stack([np.stack([w_pts[(u, d)] for d in range(npk)])
                                               for u in range(lin.n_shards)]), m_pt[None], b_pt)
    for ks in (H.HE_KEY_STREAM_AUTO, H.HE_KEY_STREAM_LDG, H.HE_KEY_STREAM_PK3, H.HE_KEY_STREAM_SPLIT):
        H.he_ctx_set_option(g.h, H.HE_OPT_KEY_STREAM, ks)
        H.he_linear_run(g.h, L, ins, out)
        H.he_ctx_check(g.h)
        assert H.he_ct_level(out) == ref.level and H.he_ct_scale(out) == ref.scale
        assert_ct_equal(g.download(out), ref)
    H.he_ctx_set_option(g.h, H.HE_OPT_KEY_STREAM, H.HE_KEY_STREAM_AUTO)
    H.he_linear_destroy(L)
