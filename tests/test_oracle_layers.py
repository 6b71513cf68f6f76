"""Pins for the oracle's layer programs (Sec. 4) and polynomial routine (Appendix); no GPU."""
import os

import numpy as np
import pytest
import torch

from oracle import layers as Ly
from oracle.params import TOY, Params
from oracle.ckks import Context
import workloads

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _conv_ref(x, W, b, pad):
    return torch.nn.functional.conv2d(torch.tensor(x)[None], torch.tensor(W),
                                      None if b is None else torch.tensor(b), padding=pad)[0].numpy()


CASES = [  # (c_in, c_out, m, N, k, pad): single shard + dup, image shards, channel shards
    (4, 4, 32, 4096, 3, 1),
    (16, 16, 32, 32768, 3, 1),
    (8, 8, 28, 2048, 3, 1),
    (2, 3, 32, 512, 3, 1),
    (3, 4, 32, 512, 7, 3),
    (16, 8, 16, 1024, 3, 1),
    (4, 4, 8, 64, 1, 0),
]


@pytest.mark.parametrize("c,co,m,N,k,pad", CASES)
def test_conv_plan_equals_torch_conv2d(c, co, m, N, k, pad):
    rng = np.random.default_rng(c * 100 + m)
    x = rng.uniform(0, 1, (c, m, m))
    W = rng.uniform(-1, 1, (co, c, k, k))
    b = rng.uniform(-1, 1, co)
    lin = Ly.image_layout(c, m, N)
    plan = Ly.conv_plan(lin, W, b, pad)
    img = Ly.unpack(plan.lout, Ly.conv_slots(plan, Ly.pack(lin, x)), check_copies=True, atol=1e-12)
    assert np.abs(img - _conv_ref(x, W, b, pad)).max() < 1e-12


def test_rotation_counts_match_the_paper():
    # one full shard: c kappa^2 rotations including the identity (Sec. 4.1, Eqs. 4-5)
    rng = np.random.default_rng(0)
    p = Ly.conv_plan(Ly.image_layout(16, 32, 32768), rng.uniform(-1, 1, (16, 16, 3, 3)), None, 1)
    assert p.n_rotations() == 16 * 9 - 1
    # image shards: z kappa^2 amounts per input shard, shared by every output shard (Eq. 6)
    p = Ly.conv_plan(Ly.image_layout(16, 16, 1024), rng.uniform(-1, 1, (16, 16, 3, 3)), None, 1)
    assert [len(p.amounts(u)) for u in range(4)] == [4 * 9] * 4
    # channel shards: one amount per tap, shared by own and neighbour shard (Eq. 7)
    p = Ly.conv_plan(Ly.image_layout(2, 32, 512), rng.uniform(-1, 1, (2, 2, 3, 3)), None, 1)
    assert all(len(p.amounts(u)) == 9 for u in range(p.lin.n_shards))
    own_nbr = {(u, a) for v, t in p.terms.items() for (u, a) in t if u != v}
    assert own_nbr  # some output shards read neighbour shards


@pytest.mark.parametrize("c,co,m,N,k,pad", CASES)
def test_bsgs_plan_equals_torch_conv2d(c, co, m, N, k, pad):
    # the baby-step / giant-step regrouping is the same linear map as the diagonal plan
    rng = np.random.default_rng(c * 100 + m + 1)
    x = rng.uniform(0, 1, (c, m, m))
    W = rng.uniform(-1, 1, (co, c, k, k))
    b = rng.uniform(-1, 1, co)
    lin = Ly.image_layout(c, m, N)
    plan = Ly.conv_plan(lin, W, b, pad)
    bp = Ly.conv_plan_bsgs(plan)
    slots = Ly.pack(lin, x)
    out = Ly.bsgs_slots(bp, slots)
    assert np.abs(out - Ly.conv_slots(plan, slots)).max() < 1e-12
    img = Ly.unpack(plan.lout, out, check_copies=True, atol=1e-12)
    assert np.abs(img - _conv_ref(x, W, b, pad)).max() < 1e-12
    for (v, g), d in bp.baby.items():           # every split is g + t with g whole blocks
        assert g % lin.B == 0
        for (u, t) in d:
            assert (u, (g + t) % N) in plan.terms[v]
            assert min(t, N - t) <= lin.B // 2 or lin.B == N
    k = 2
    while k * lin.B <= N:                        # wider giant strides: the same linear map
        assert np.abs(Ly.bsgs_slots(Ly.conv_plan_bsgs(plan, k), slots) - out).max() < 1e-12
        k *= 2


def test_bsgs_rotation_counts():
    rng = np.random.default_rng(1)
    # one duplicated shard (c = 16): c kappa^2 - 1 = 143 diagonal rotations become
    # (kappa^2 - 1) baby + (c - 1) giant = 23
    p = Ly.conv_plan(Ly.image_layout(16, 32, 32768), rng.uniform(-1, 1, (16, 16, 3, 3)), None, 1)
    assert p.n_rotations() == 143 and Ly.conv_plan_bsgs(p).n_rotations() == 8 + 15
    # giant stride of k blocks: (k kappa^2 - 1) baby + (c/k - 1) giant; k = c is the diagonal form
    for k, want in ((2, 17 + 7), (4, 35 + 3), (8, 71 + 1), (16, 143), (32, 143)):
        assert Ly.conv_plan_bsgs(p, k).n_rotations() == want
    # image shards, z = 4 channels per shard, 4 in / 4 out: n_in (kappa^2 - 1) + n_out (z - 1)
    p = Ly.conv_plan(Ly.image_layout(16, 16, 1024), rng.uniform(-1, 1, (16, 16, 3, 3)), None, 1)
    assert p.n_rotations() == 4 * 35 and Ly.conv_plan_bsgs(p).n_rotations() == 4 * 8 + 4 * 3
    # channel shards: every amount is a tap shift, no giant steps
    p = Ly.conv_plan(Ly.image_layout(2, 32, 512), rng.uniform(-1, 1, (2, 2, 3, 3)), None, 1)
    bp = Ly.conv_plan_bsgs(p)
    assert all(g == 0 for (_, g) in bp.baby) and bp.n_rotations() == p.n_rotations()
    # the split itself: centred residue modulo the block
    assert Ly.bsgs_split(3 * 256 + 17, 256, 1024) == (768, 17)
    assert Ly.bsgs_split(3 * 256 - 17, 256, 1024) == (768, 1024 - 17)
    assert Ly.bsgs_split(1024 - 1, 256, 1024) == (0, 1023)
    assert Ly.bsgs_split(3 * 256 + 17, 256, 1024, 2) == (512, 256 + 17)
    assert Ly.bsgs_split(3 * 256 - 17, 256, 1024, 4) == (0, 3 * 256 - 17)


@pytest.mark.parametrize("c,m,N,sel", [(4, 32, 4096, False), (16, 32, 2048, False),
                                        (8, 32, 2048, False), (2, 32, 512, False),
                                        (2, 28, 512, False), (3, 32, 512, True),
                                        (64, 56, 32768, False),
                                        # 2 shards or 1 with an empty block: duplication (Eq. 13)
                                        # must leave the empty block's copies empty
                                        (3, 32, 2048, False), (3, 32, 2048, True),
                                        (5, 32, 4096, False), (3, 32, 4096, False)])
def test_pool_plan_equals_torch_avg_pool(c, m, N, sel):
    rng = np.random.default_rng(m + c)
    x = rng.uniform(0, 1, (c, m, m))
    lin = Ly.image_layout(c, m, N)
    plan = Ly.pool_plan(lin, select_top_left=sel)
    img = Ly.unpack(plan.lout, Ly.pool_slots(plan, Ly.pack(lin, x)), check_copies=True,
                    atol=1e-12)
    ref = x[:, ::2, ::2] if sel else torch.nn.functional.avg_pool2d(torch.tensor(x)[None], 2)[0].numpy()
    assert np.abs(img - ref).max() < 1e-12


def test_pool_permutes_image_shards_but_not_channel_shards():
    plan = Ly.pool_plan(Ly.image_layout(8, 32, 2048))
    order = [int(c) for c in plan.lout.chan[0] if c >= 0]
    assert sorted(order) == list(range(8)) and order != list(range(8))   # Fig. (consolidate)
    plan = Ly.pool_plan(Ly.image_layout(2, 32, 512))                      # channel shards
    ch = plan.lout.chan[0]
    assert list(ch) == sorted(ch)                                         # order kept


def test_strided_conv_is_conv_then_top_left_select():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (3, 32, 32))
    W = rng.normal(0, 0.05, (4, 3, 7, 7))
    lin = Ly.image_layout(3, 32, 512)
    cp = Ly.conv_plan(lin, W, None, 3)
    pp = Ly.pool_plan(cp.lout, select_top_left=True)
    out = Ly.pool_slots(pp, Ly.conv_slots(cp, Ly.pack(lin, x)))
    ref = torch.nn.functional.conv2d(torch.tensor(x)[None], torch.tensor(W), stride=2,
                                     padding=3)[0].numpy()
    assert np.abs(Ly.unpack(pp.lout, out) - ref).max() < 1e-12


def _table(method):
    return [l.split()[1:] for l in open(os.path.join(GOLD, "poly_approx_table.txt"))
            if l.strip() and not l.startswith("#") and l.split()[0] == method]


def test_chebyshev_nodes_table_from_the_paper():
    rows = _table("chebyshev")
    assert len(rows) == 2
    xs = np.linspace(-16, 16, 100001)
    for deg, relu_err, gelu_err in rows:
        for f, want in ((Ly.relu, relu_err), (Ly.gelu, gelu_err)):
            c = Ly.cheb_nodes_coeffs(f, int(deg), -16, 16)
            err = np.abs(Ly.cheb_eval(c, xs, -16, 16) - np.array([f(v) for v in xs])).max()
            assert round(err, 4) == float(want), (deg, f.__name__, err)


@pytest.fixture(scope="module")
def minimax16():
    return {(f.__name__, d): Ly.minimax_coeffs(f, d, -16, 16) for f in (Ly.relu, Ly.gelu) for d in (27, 59)}


def test_minimax_table_from_the_paper(minimax16):
    # GELU rows: the printed digits.  ReLU rows: the exact minimax error sits at most 2% below
    # the printed value (a minimax error cannot exceed any approximation's, and the paper's
    # routine stopped slightly short of the optimum); it is the Bernstein limit
    # E_{2k}(|x|) ~ beta / 2k with beta = 0.2801694990..., times 16 / 2 for ReLU = (x + |x|)/2
    rows = _table("minimax")
    assert len(rows) == 2
    for deg, relu_err, gelu_err in rows:
        d = int(deg)
        _, Eg = minimax16[("gelu", d)]
        _, Er = minimax16[("relu", d)]
        assert round(Eg, 4) == float(gelu_err), (d, Eg)
        assert 0.98 * float(relu_err) <= Er <= float(relu_err), (d, Er)
        assert abs(Er / 8.0 * (d - 1) / 0.2801694990 - 1.0) < 3e-3
        # optimality: below the Chebyshev-node interpolant of the same degree
        for f, E in ((Ly.relu, Er), (Ly.gelu, Eg)):
            xs = np.linspace(-16, 16, 20001)
            c = Ly.cheb_nodes_coeffs(f, d, -16, 16)
            assert E < np.abs(Ly.cheb_eval(c, xs, -16, 16) - np.array([f(v) for v in xs])).max()


def test_minimax_equioscillates(minimax16):
    # the characterisation theorem: the error reaches +-E alternately at deg + 2 points and
    # nowhere exceeds E
    for (name, d), (c, E) in minimax16.items():
        f = getattr(Ly, name)
        xs = np.linspace(-16, 16, 400001)
        r = np.array([f(v) for v in xs]) - Ly.cheb_eval(c, xs, -16, 16)
        assert np.abs(r).max() <= E * (1 + 1e-7)
        near = np.nonzero(np.abs(r) >= E * (1 - 1e-3))[0]
        signs = [np.sign(r[near[0]])]
        for i in near[1:]:
            if np.sign(r[i]) != signs[-1]:
                signs.append(np.sign(r[i]))
        assert len(signs) >= d + 2, (name, d, len(signs))


def test_minimax_wide_range_claims():
    # ReLU is homogeneous, so its minimax error scales with the range; on [-65, 65] GELU's
    # degree-59 minimax error is only about 1.2x below ReLU's (Appendix), against two orders of
    # magnitude on [-16, 16]
    _, Er16 = Ly.minimax_coeffs(Ly.relu, 59, -16, 16)
    _, Er65 = Ly.minimax_coeffs(Ly.relu, 59, -65, 65)
    _, Eg65 = Ly.minimax_coeffs(Ly.gelu, 59, -65, 65)
    assert abs(Er65 / Er16 - 65.0 / 16.0) < 1e-6
    assert 1.15 <= Er65 / Eg65 <= 1.35


def test_binary_tree_chebyshev_recursion_and_depth():
    t = np.linspace(-1, 1, 1001)
    c = np.random.default_rng(0).normal(size=60)
    assert np.abs(Ly.cheb_tree_slots(c, t) - Ly.cheb_eval(c, t, -1, 1)).max() < 1e-10

    # depth of T_k in the tree: T_1 = x at 0, T_k one level below its deeper operand
    def depths(d):
        dep = {1: 0}
        for k in range(2, d + 1):
            h = k // 2
            dep[k] = 1 + (dep[h] if k % 2 == 0 else max(dep[h], dep[h + 1]))
        return max(dep.values())
    assert depths(59) == 6 and depths(27) == 5        # Appendix, Chebyshev polynomials


@pytest.fixture(scope="module")
def toy():
    return Context(TOY)


def test_toy_conv_decrypts_to_fp64_conv(toy):
    wl = workloads.toy_conv(0)
    lin = Ly.image_layout(4, 32, toy.N)
    plan = Ly.conv_plan(lin, wl.W, wl.bias, wl.pad)
    slots = Ly.pack(lin, wl.x)
    cts = [toy.encrypt(slots[u], 3, nonce=u) for u in range(lin.n_shards)]
    out = Ly.conv_he(toy, plan, cts)
    img = Ly.unpack(plan.lout, np.stack([toy.decrypt(c) for c in out]))
    ref = _conv_ref(wl.x, wl.W, wl.bias, wl.pad)
    assert np.abs(img - ref).max() <= 2.0 ** -20 * (ref.max() - ref.min())
    assert plan.n_rotations() == 35


def test_toy_pool_decrypts_to_fp64_pool(toy):
    rng = np.random.default_rng(7)
    x = rng.uniform(0, 1, (4, 32, 32))
    lin = Ly.image_layout(4, 32, toy.N)
    plan = Ly.pool_plan(lin)
    cts = [toy.encrypt(Ly.pack(lin, x)[0], 3, nonce=5)]
    out = Ly.pool_he(toy, plan, cts)
    assert out[0].level == 1
    img = Ly.unpack(plan.lout, np.stack([toy.decrypt(c) for c in out]))
    ref = torch.nn.functional.avg_pool2d(torch.tensor(x)[None], 2)[0].numpy()
    assert np.abs(img - ref).max() <= 2.0 ** -20 * (ref.max() - ref.min())


def test_poly_gelu_he_matches_same_polynomial():
    ctx = Context(Params(log_n=10, n_q=8, n_p=2, dnum=4, q0_bits=50, q_bits=40, p_bits=50,
                         scale=2.0 ** 40, seed=1))
    ctx.gen_relin_key()
    z = np.random.default_rng(0).uniform(-1, 1, ctx.N)
    c = Ly.cheb_nodes_coeffs(Ly.gelu, 16, -8, 8)
    out = Ly.cheb_tree_he(ctx, ctx.encrypt(z, 7), c)
    assert out.level == 2 and out.scale == 2.0 ** 40
    ref = Ly.cheb_eval(c, 8 * z, -8, 8)
    assert np.abs(ctx.decrypt(out) - ref).max() <= 2.0 ** -20 * (ref.max() - ref.min())


def test_toy_conv_raised_basis_decrypts_to_fp64_conv(toy):
    # one ModDown per output shard: different bits from conv_he, same decryption
    wl = workloads.toy_conv(0)
    lin = Ly.image_layout(4, 32, toy.N)
    plan = Ly.conv_plan(lin, wl.W, np.linspace(-1, 1, 4), wl.pad)
    slots = Ly.pack(lin, wl.x)
    cts = [toy.encrypt(slots[u], 3, nonce=u) for u in range(lin.n_shards)]
    a = Ly.conv_he(toy, plan, cts)
    b = Ly.conv_he_raised(toy, plan, cts)
    assert not np.array_equal(a[0].c, b[0].c)
    ref = _conv_ref(wl.x, wl.W, np.linspace(-1, 1, 4), wl.pad)
    for out in (a, b):
        img = Ly.unpack(plan.lout, np.stack([toy.decrypt(c) for c in out]))
        assert np.abs(img - ref).max() <= 2.0 ** -20 * (ref.max() - ref.min())


def test_raised_basis_conv_on_image_shards():
    ctx = Context(Params(log_n=11, n_q=4, n_p=2, dnum=2, q0_bits=50, q_bits=40, p_bits=50,
                         scale=2.0 ** 40, seed=4))
    rng = np.random.default_rng(8)
    x = rng.uniform(0, 1, (8, 16, 16))
    W = rng.uniform(-1, 1, (4, 8, 3, 3))
    lin = Ly.image_layout(8, 16, ctx.N)
    assert lin.n_shards == 2
    plan = Ly.conv_plan(lin, W, None, 1)
    slots = Ly.pack(lin, x)
    cts = [ctx.encrypt(slots[u], 3, nonce=u) for u in range(2)]
    out = Ly.conv_he_raised(ctx, plan, cts)
    img = Ly.unpack(plan.lout, np.stack([ctx.decrypt(c) for c in out]))
    ref = _conv_ref(x, W, None, 1)
    assert np.abs(img - ref).max() <= 2.0 ** -20 * (ref.max() - ref.min())


def test_toy_pool_raised_basis_decrypts_to_fp64_pool(toy):
    rng = np.random.default_rng(7)
    x = rng.uniform(0, 1, (4, 32, 32))
    lin = Ly.image_layout(4, 32, toy.N)
    plan = Ly.pool_plan(lin)
    cts = [toy.encrypt(Ly.pack(lin, x)[0], 3, nonce=5)]
    out = Ly.pool_he_raised(toy, plan, cts)
    assert out[0].level == 1 and not np.array_equal(out[0].c, Ly.pool_he(toy, plan, cts)[0].c)
    img = Ly.unpack(plan.lout, np.stack([toy.decrypt(c) for c in out]))
    ref = torch.nn.functional.avg_pool2d(torch.tensor(x)[None], 2)[0].numpy()
    assert np.abs(img - ref).max() <= 2.0 ** -20 * (ref.max() - ref.min())


def _small_ctx():
    return Context(Params(log_n=10, n_q=4, n_p=2, dnum=2, q0_bits=50, q_bits=40, p_bits=50,
                          scale=2.0 ** 40, seed=11))


def test_raised_stage_single_rotation_is_the_hoisted_rotation():
    # one term, plaintext 1, amount a: (phi(c0), 0) + ModDown(u_a) is exactly the hoisted
    # rotation, which is pinned against np.roll elsewhere
    ctx = _small_ctx()
    z = np.random.default_rng(3).uniform(-1, 1, ctx.N)
    ct = ctx.encrypt(z, 3, nonce=9)
    for a in (1, 5, ctx.N - 3):
        ctx.gen_rotation_key(a)
        out = Ly.raised_stage(ctx, [ct], {0: [(0, a, None)]})[0]
        ref = ctx.rotate_hoisted(ct, ctx.hoist(ct), a)
        assert np.array_equal(out.c, ref.c)


def test_raised_stage_without_rotations_is_the_direct_mac():
    # only amount-0 terms: nothing is raised, the ModDown adds zero, the result is sum pt * ct
    ctx = _small_ctx()
    rng = np.random.default_rng(4)
    cts = [ctx.encrypt(rng.uniform(-1, 1, ctx.N), 3, nonce=20 + i) for i in range(2)]
    pts = [rng.integers(-2 ** 20, 2 ** 20, ctx.n) for _ in range(2)]
    out = Ly.raised_stage(ctx, cts, {0: [(0, 0, pts[0]), (1, 0, pts[1])]})[0]
    mods, psis = ctx.mods(3), ctx.psis(3)
    want = []
    for k in range(2):
        acc = np.zeros((4, ctx.n), dtype=np.uint64)
        for ct, pt in zip(cts, pts):
            P = ctx.ntt(ctx.reduce_int(pt, mods), mods, psis).reshape(4, ctx.n)
            X = ctx.ntt(ct.c[k], mods, psis).reshape(4, ctx.n)
            ctx.lib.orc_mac(acc, P, X, 4, ctx.n, mods)
        want.append(ctx.intt(acc, mods, psis).reshape(4, ctx.n))
    assert np.array_equal(out.c, np.stack(want))


def test_plaintexts_encoded_for_a_higher_level_serve_a_lower_one():
    # a conv planned at level 3 (plaintexts at scale q_3) applied to an input at level 2:
    # the output scale is scale * q_3 / q_2 and it still decrypts to the FP64 convolution
    ctx = _small_ctx()
    rng = np.random.default_rng(6)
    x = rng.uniform(0, 1, (2, 16, 16))
    W = rng.uniform(-1, 1, (2, 2, 3, 3))
    b = rng.uniform(-1, 1, 2)
    lin = Ly.image_layout(2, 16, ctx.N)
    plan = Ly.conv_plan(lin, W, b, 1)
    S = float(ctx.q[3])
    pts = Ly.conv_plaintexts(plan, ctx.n, S)
    cts = [ctx.encrypt(Ly.pack(lin, x)[u], 2, nonce=30 + u) for u in range(lin.n_shards)]
    ref = _conv_ref(x, W, b, 1)
    for f in (Ly.conv_he, Ly.conv_he_raised):
        out = f(ctx, plan, cts, pts, pt_scale=S)
        assert out[0].level == 1 and out[0].scale == ctx.pr.scale * S / float(ctx.q[2])
        img = Ly.unpack(plan.lout, np.stack([ctx.decrypt(c) for c in out]))
        assert np.abs(img - ref).max() <= 2.0 ** -20 * (ref.max() - ref.min())


@pytest.mark.parametrize("c,m,N", [(4, 8, 512), (16, 8, 512), (2, 32, 512), (3, 28, 1024)])
def test_linear_plan_is_the_dot_product(c, m, N):
    # one duplicated shard, image shards, channel shards, a padded frame: every pixel counted once
    rng = np.random.default_rng(c * 31 + m)
    x = rng.uniform(-1, 1, (c, m, m))
    W = rng.uniform(-1, 1, (5, c, m, m))
    b = rng.uniform(-1, 1, 5)
    lin = Ly.image_layout(c, m, N)
    plan = Ly.linear_plan(lin, W, b)
    out = Ly.linear_slots(plan, Ly.pack(lin, x))
    want = W.reshape(5, -1) @ x.reshape(-1) + b
    assert np.abs(out[:5] - want).max() < 1e-9 and np.abs(out[5:]).max() < 1e-9
    assert plan.amounts() == [N >> i for i in range(1, N.bit_length())]


def test_pool_linear_is_global_average_pool_then_linear():
    rng = np.random.default_rng(9)
    c, m, N = 16, 8, 512                         # a ResNet tail: 8 x 8 channels, one shard
    x = rng.uniform(0, 1, (c, m, m))
    W = rng.uniform(-1, 1, (10, c))
    b = rng.uniform(-1, 1, 10)
    lin = Ly.image_layout(c, m, N)
    out = Ly.linear_slots(Ly.pool_linear_plan(lin, W, b), Ly.pack(lin, x))
    pooled = torch.nn.functional.adaptive_avg_pool2d(torch.tensor(x)[None], 1).reshape(-1)
    want = torch.nn.functional.linear(pooled, torch.tensor(W), torch.tensor(b)).numpy()
    assert np.abs(out[:10] - want).max() < 1e-12


def test_linear_he_decrypts_to_fp64():
    ctx = _small_ctx()
    rng = np.random.default_rng(10)
    c, m = 8, 8
    x = rng.uniform(0, 1, (c, m, m))
    W = rng.uniform(-1, 1, (4, c))
    b = rng.uniform(-1, 1, 4)
    lin = Ly.image_layout(c, m, ctx.N)
    plan = Ly.pool_linear_plan(lin, W, b)
    cts = [ctx.encrypt(Ly.pack(lin, x)[u], 3, nonce=70 + u) for u in range(lin.n_shards)]
    out = Ly.linear_he(ctx, plan, cts)
    assert out.level == 1 and out.scale == ctx.pr.scale
    got = ctx.decrypt(out)
    want = W @ x.mean(axis=(1, 2)) + b
    assert np.abs(got[:4] - want).max() <= 2.0 ** -20 * (want.max() - want.min())
    assert np.abs(got[4:]).max() <= 2.0 ** -20 * (want.max() - want.min())


@pytest.mark.parametrize("c,m,N,n_out", [(4, 8, 512, 5), (16, 8, 512, 10), (2, 32, 512, 3), (3, 28, 1024, 16),
                                         (8, 16, 1024, 1)])
def test_packed_head_equals_the_per_output_head(c, m, N, n_out):
    # the packed regrouping computes the same dot products in slots 0..n_out-1 and zeros elsewhere
    rng = np.random.default_rng(c + m + n_out)
    x = rng.uniform(-1, 1, (c, m, m))
    W = rng.uniform(-1, 1, (n_out, c, m, m))
    b = rng.uniform(-1, 1, n_out)
    lin = Ly.image_layout(c, m, N)
    plan = Ly.linear_plan(lin, W, b)
    slots = Ly.pack(lin, x)
    got = Ly.linear_packed_slots(plan, slots)
    assert np.abs(got - Ly.linear_slots(plan, slots)).max() < 1e-9
    npk = Ly.linear_packed_width(n_out)
    assert npk >= n_out and npk & (npk - 1) == 0 and npk < 2 * max(n_out, 1)
    # rotations: n' - 1 hoisted per shard and log2(N / n') shifts, against n_out log2 N
    assert len(Ly.linear_packed_shifts(plan)) == (N // npk).bit_length() - 1


def test_packed_head_he_decrypts_to_fp64():
    ctx = _small_ctx()
    rng = np.random.default_rng(11)
    c, m = 8, 8
    x = rng.uniform(0, 1, (c, m, m))
    W = rng.uniform(-1, 1, (6, c))
    b = rng.uniform(-1, 1, 6)
    lin = Ly.image_layout(c, m, ctx.N)
    plan = Ly.pool_linear_plan(lin, W, b)
    cts = [ctx.encrypt(Ly.pack(lin, x)[u], 3, nonce=80 + u) for u in range(lin.n_shards)]
    out = Ly.linear_packed_he(ctx, plan, cts)
    ref = Ly.linear_he(ctx, plan, cts)
    assert out.level == ref.level == 1 and out.scale == ref.scale and not np.array_equal(out.c, ref.c)
    got = ctx.decrypt(out)
    want = W @ x.mean(axis=(1, 2)) + b
    tol = 2.0 ** -20 * (want.max() - want.min())
    assert np.abs(got[:6] - want).max() <= tol and np.abs(got[6:]).max() <= tol


def test_bsgs_he_without_giant_steps_is_the_diagonal_form():
    # channel shards: every giant amount is 0, so S_{v,0} is the diagonal MAC (per-rotation
    # form) or the diagonal raised stage, and the giant stage adds nothing: bit for bit
    ctx = _small_ctx()
    rng = np.random.default_rng(12)
    x = rng.uniform(0, 1, (2, 32, 32))
    W = rng.uniform(-1, 1, (2, 2, 3, 3))
    b = rng.uniform(-1, 1, 2)
    lin = Ly.image_layout(2, 32, ctx.N)
    plan = Ly.conv_plan(lin, W, b, 1)
    bp = Ly.conv_plan_bsgs(plan)
    assert all(g == 0 for (_, g) in bp.baby)
    cts = [ctx.encrypt(Ly.pack(lin, x)[u], 3, nonce=40 + u) for u in range(lin.n_shards)]
    for raised, diag in ((False, Ly.conv_he), (True, Ly.conv_he_raised)):
        got = Ly.conv_he_bsgs(ctx, bp, cts, raised=raised)
        want = diag(ctx, plan, cts)
        for g_, w_ in zip(got, want):
            assert g_.level == w_.level and g_.scale == w_.scale and np.array_equal(g_.c, w_.c)


def test_bsgs_he_with_full_giant_stride_is_the_diagonal_form():
    # G = N: every g = 0 and t = a, on a duplicated shard that has giant steps at G = B
    ctx = _small_ctx()
    rng = np.random.default_rng(13)
    x = rng.uniform(0, 1, (2, 8, 8))
    W = rng.uniform(-1, 1, (2, 2, 3, 3))
    lin = Ly.image_layout(2, 8, ctx.N)
    plan = Ly.conv_plan(lin, W, None, 1)
    assert any(g != 0 for (_, g) in Ly.conv_plan_bsgs(plan).baby)
    bp = Ly.conv_plan_bsgs(plan, lin.nb)
    assert all(g == 0 for (_, g) in bp.baby) and bp.n_rotations() == plan.n_rotations()
    cts = [ctx.encrypt(Ly.pack(lin, x)[0], 3, nonce=45)]
    for raised, diag in ((False, Ly.conv_he), (True, Ly.conv_he_raised)):
        got, want = Ly.conv_he_bsgs(ctx, bp, cts, raised=raised), diag(ctx, plan, cts)
        assert all(np.array_equal(a.c, b.c) for a, b in zip(got, want))


@pytest.mark.parametrize("c,co,m,log_n", [(8, 4, 16, 11), (2, 2, 8, 10)])
def test_bsgs_he_decrypts_to_fp64_conv(c, co, m, log_n):
    # image shards (8 channels in 2 shards) and a duplicated shard (2 channels x 4 copies)
    ctx = Context(Params(log_n=log_n, n_q=4, n_p=2, dnum=2, q0_bits=50, q_bits=40, p_bits=50,
                         scale=2.0 ** 40, seed=4))
    rng = np.random.default_rng(c + m)
    x = rng.uniform(0, 1, (c, m, m))
    W = rng.uniform(-1, 1, (co, c, 3, 3))
    b = rng.uniform(-1, 1, co)
    lin = Ly.image_layout(c, m, ctx.N)
    plan = Ly.conv_plan(lin, W, b, 1)
    bp = Ly.conv_plan_bsgs(plan)
    assert any(g != 0 for (_, g) in bp.baby) and bp.n_rotations() < plan.n_rotations()
    S = float(ctx.q[3])                          # plaintexts for level 3 serve level 2 too
    pts = Ly.bsgs_plaintexts(bp, ctx.n, S)
    ref = _conv_ref(x, W, b, 1)
    for level in (3, 2):
        cts = [ctx.encrypt(Ly.pack(lin, x)[u], level, nonce=50 + u) for u in range(lin.n_shards)]
        outs = [Ly.conv_he_bsgs(ctx, bp, cts, pts, pt_scale=S, raised=r) for r in (False, True)]
        assert not np.array_equal(outs[0][0].c, outs[1][0].c)
        for out in outs:
            assert out[0].level == level - 1 and out[0].scale == ctx.pr.scale * S / float(ctx.q[level])
            img = Ly.unpack(plan.lout, np.stack([ctx.decrypt(ct) for ct in out]))
            assert np.abs(img - ref).max() <= 2.0 ** -20 * (ref.max() - ref.min())


@pytest.mark.parametrize("c,co,m,N,k,pad", [(3, 4, 32, 512, 3, 1), (2, 2, 32, 256, 7, 3), (3, 2, 28, 256, 5, 2),
                                           (1, 3, 64, 1024, 3, 1)])
def test_factored_plan_equals_torch_conv2d(c, co, m, N, k, pad):
    rng = np.random.default_rng(c * 7 + m)
    x = rng.uniform(0, 1, (c, m, m))
    W = rng.uniform(-1, 1, (co, c, k, k))
    b = rng.uniform(-1, 1, co)
    lin = Ly.image_layout(c, m, N)
    plan = Ly.conv_plan_factored(lin, W, b, pad)
    img = Ly.unpack(plan.lout, Ly.factored_slots(plan, Ly.pack(lin, x)))
    assert np.abs(img - _conv_ref(x, W, b, pad)).max() < 1e-12
    # own shard plus at most one neighbour per (shard, tap): the masks number <= 2 H T, and a
    # tap whose rows stay inside one shard has only the own mask there
    assert len(plan.masks) <= 2 * plan.H * k * k
    assert set(plan.amounts) == {((kk - pad) * lin.M + (ll - pad)) % N for kk in range(k) for ll in range(k)}


def test_factored_scalars_round_half_away():
    assert Ly.round_half_away(2.5) == 3 and Ly.round_half_away(-2.5) == -3
    assert Ly.round_half_away(-0.49) == 0 and Ly.round_half_away(7.0) == 7


@pytest.mark.parametrize("raised", [False, True])
def test_factored_conv_he_decrypts_to_fp64(raised):
    ctx = Context(Params(log_n=10, n_q=5, n_p=2, dnum=3, q0_bits=50, q_bits=40, p_bits=50,
                         scale=2.0 ** 40, seed=12))
    rng = np.random.default_rng(13)
    c, co, m, k, pad = 2, 3, 32, 3, 1
    x = rng.uniform(0, 1, (c, m, m))
    W = rng.uniform(-1, 1, (co, c, k, k))
    b = rng.uniform(-1, 1, co)
    lin = Ly.image_layout(c, m, ctx.N)
    plan = Ly.conv_plan_factored(lin, W, b, pad)
    assert plan.H == 2
    cts = [ctx.encrypt(s, 4, nonce=40 + u) for u, s in enumerate(Ly.pack(lin, x))]
    out = Ly.conv_he_factored(ctx, plan, cts, raised=raised)
    assert out[0].level == 2
    img = Ly.unpack(plan.lout, np.stack([ctx.decrypt(ct) for ct in out]))
    ref = _conv_ref(x, W, b, pad)
    assert np.abs(img - ref).max() <= 2.0 ** -20 * (ref.max() - ref.min())


@pytest.mark.parametrize("deg", [5, 8, 16, 27, 59])
def test_paterson_stockmeyer_slots_equal_chebyshev_sum(deg):
    c = Ly.cheb_nodes_coeffs(Ly.gelu, deg, -8, 8)
    t = np.linspace(-1, 1, 513)
    assert np.abs(Ly.cheb_ps_slots(c, t) - Ly.cheb_eval(c, 8 * t, -8, 8)).max() < 1e-12


def test_chebyshev_division_identity():
    # p = q T_G + r exactly (T_G T_j = (T_{G+j} + T_{|G-j|}) / 2), deg r < G
    rng = np.random.default_rng(3)
    t = np.linspace(-1, 1, 257)
    for d, G in ((16, 16), (15, 8), (59, 32), (31, 16), (9, 8)):
        c = rng.normal(size=d + 1)
        q, r = Ly.cheb_divide(list(c), G)
        assert len(r) == G and len(q) == d - G + 1
        TG = np.cos(G * np.arccos(t))
        lhs = Ly.cheb_eval(c, t, -1, 1)
        rhs = Ly.cheb_eval(q, t, -1, 1) * TG + Ly.cheb_eval(r, t, -1, 1)
        assert np.abs(lhs - rhs).max() < 1e-11


@pytest.fixture(scope="module")
def deep():
    ctx = Context(Params(log_n=10, n_q=10, n_p=3, dnum=4, q0_bits=50, q_bits=40, p_bits=50,
                         scale=2.0 ** 40, seed=21))
    ctx.gen_relin_key()
    return ctx


@pytest.mark.parametrize("deg,depth", [(59, 6), (27, 5), (16, 5)])
def test_paterson_stockmeyer_he_depth_and_accuracy(deep, deg, depth):
    """The paper evaluates the degree-59 GELU at depth 6 and degree 27 at depth 5 (Appendix):
    the Paterson-Stockmeyer recursion reaches exactly those depths, with fewer products than
    the binary tree, and decrypts to the same polynomial."""
    ctx = deep
    c = Ly.cheb_nodes_coeffs(Ly.gelu, deg, -8, 8)
    z = np.random.default_rng(deg).uniform(-1, 1, ctx.N)
    ct = ctx.encrypt(z, 9, nonce=deg)
    count = [0]
    orig = ctx.mul_relin

    def counted(a, b):
        count[0] += 1
        return orig(a, b)
    ctx.mul_relin = counted
    try:
        out = Ly.cheb_ps_he(ctx, ct, c)
    finally:
        ctx.mul_relin = orig
    assert ct.level - out.level == depth
    assert count[0] < deg - 1
    ref = Ly.cheb_eval(c, 8 * z, -8, 8)
    assert np.abs(ctx.decrypt(out) - ref).max() <= 2.0 ** -20 * (ref.max() - ref.min())


def test_paterson_stockmeyer_degree_16_products_by_operand_level(deep):
    """Degree 16 (k = 4, giant steps 4, 8, 16): the evaluation takes 8 relinearised products
    whose operands sit at 5 distinct levels, two products at every level but the first and the
    third: T_2 | T_3, T_4 | T_8 | T_16 and the product inside the T_8 quotient | the two
    products of the remainder's quotients.  Products at one level are independent, so 5 is the
    fewest batches of equal-level products the evaluation can be issued in."""
    ctx = deep
    c = Ly.cheb_nodes_coeffs(Ly.gelu, 16, -8, 8)
    ct = ctx.encrypt(np.random.default_rng(16).uniform(-1, 1, ctx.N), 9, nonce=316)
    levels = []
    orig = ctx.mul_relin

    def recorded(a, b):
        assert a.level == b.level
        levels.append(a.level)
        return orig(a, b)
    ctx.mul_relin = recorded
    try:
        Ly.cheb_ps_he(ctx, ct, c)
    finally:
        ctx.mul_relin = orig
    from collections import Counter
    assert Counter(levels) == Counter({9: 1, 8: 2, 7: 1, 6: 2, 5: 2})
