"""The paper's sharded layer programs, for the oracle (TEST INFRASTRUCTURE ONLY).

Sec. 4 of the paper.  Every program here has two evaluators that share one plan:

* ``*_slots``: the plan applied to cleartext float64 slot vectors, with ``np.roll`` as the
  rotation (the slot simulator; it pins layouts, rotation sets and masks against plain
  ``torch.nn.functional.conv2d`` / ``avg_pool2d`` without any encryption noise);
* ``*_he``: the same plan on oracle ciphertexts (``oracle.ckks``).

Layout (Sec. 4 "Sharding and Encrypting an Image", "Duplicating and Permuting Channels").
Each channel's valid m x m pixels sit row-major in an M x M frame, M the next power of two
(the paper's zero-padding suggestion for non-power-of-two sizes, Sec. 4), row stride M.
A shard of N slots is cut into blocks of B = min(M^2, N) slots; block b of shard u holds the
rows [row0, row0 + B/M) of one channel (or nothing).  A table (chan[u][b], row0[u][b]) is the
metadata: it expresses image shards (B = M^2, z = N/M^2 channels per shard), channel shards
(B = N, consecutive rows of one channel per shard), the duplication factor d (a channel in
several blocks; tiled order c_0..c_{c-1} repeated d times) and the pooling permutation tau
(chan[] in any order).
"""
from dataclasses import dataclass, field
import math

import numpy as np

from .encode import encode


# ============================================================================ layout
@dataclass
class Layout:
    c: int                  # channels
    m: int                  # valid side
    M: int                  # frame side (row stride), power of two
    N: int                  # slots per shard
    B: int                  # slots per block
    chan: np.ndarray        # [n_shards][nb] int: channel or -1
    row0: np.ndarray        # [n_shards][nb] int: first frame row held by the block

    @property
    def n_shards(self):
        return self.chan.shape[0]

    @property
    def nb(self):
        return self.chan.shape[1]

    @property
    def rows_per_block(self):
        return self.B // self.M

    def copy(self):
        return Layout(self.c, self.m, self.M, self.N, self.B, self.chan.copy(), self.row0.copy())


def next_pow2(x):
    return 1 << (int(x) - 1).bit_length()


def image_layout(c, m, N):
    """Initial layout of a c x m x m image (no permutation)."""
    M = next_pow2(m)
    if M * M <= N:
        B = M * M
        nb = N // B
        if c * B <= N:                          # one shard, duplicated d = nb // c times
            chan = np.full((1, nb), -1, dtype=np.int64)
            d = nb // c
            for b in range(d * c):
                chan[0, b] = b % c
        else:                                   # image shards, z = nb channels each
            t = -(-c // nb)
            chan = np.full((t, nb), -1, dtype=np.int64)
            for f in range(c):
                chan[f // nb, f % nb] = f
        row0 = np.zeros_like(chan)
    else:                                       # channel shards: N/M rows per shard
        B = N
        R = N // M
        h = M // R                              # shards per channel
        chan = np.zeros((c * h, 1), dtype=np.int64)
        row0 = np.zeros((c * h, 1), dtype=np.int64)
        for f in range(c):
            for k in range(h):
                chan[f * h + k, 0] = f
                row0[f * h + k, 0] = k * R
    return Layout(c, m, M, N, B, chan, row0)


def slot_coords(lay: Layout, u: int):
    """For every slot of shard u: (channel or -1, frame row y, column x, valid pixel?)."""
    i = np.arange(lay.N)
    b = i // lay.B
    ch = lay.chan[u][b]
    y = lay.row0[u][b] + (i % lay.B) // lay.M
    x = i % lay.M
    valid = (ch >= 0) & (y < lay.m) & (x < lay.m)
    return ch, y, x, valid


def pack(lay: Layout, img):
    """img [c][m][m] -> slot vectors [n_shards][N]."""
    img = np.asarray(img, dtype=np.float64)
    out = np.zeros((lay.n_shards, lay.N))
    for u in range(lay.n_shards):
        ch, y, x, valid = slot_coords(lay, u)
        out[u, valid] = img[ch[valid], y[valid], x[valid]]
    return out


def unpack(lay: Layout, slots, check_copies=False, atol=0.0):
    """Slot vectors -> img [c][m][m] (first copy of every pixel)."""
    img = np.full((lay.c, lay.m, lay.m), np.nan)
    for u in range(lay.n_shards):
        ch, y, x, valid = slot_coords(lay, u)
        cur = img[ch[valid], y[valid], x[valid]]
        vals = slots[u][valid]
        if check_copies:
            seen = ~np.isnan(cur)
            assert np.all(np.abs(cur[seen] - vals[seen]) <= atol), "duplicate copies disagree"
        fill = np.where(np.isnan(cur), vals, cur)
        img[ch[valid], y[valid], x[valid]] = fill
    assert not np.isnan(img).any(), "layout does not cover the image"
    return img


# ============================================================================ convolution
@dataclass
class ConvPlan:
    lin: Layout
    lout: Layout
    terms: dict = field(default_factory=dict)    # v -> {(u, a): D float64 [N]}
    bias: np.ndarray = None                      # [n_out][N], bias on valid output pixels

    def amounts(self, u):
        s = set()
        for v in self.terms:
            for (uu, a) in self.terms[v]:
                if uu == u:
                    s.add(a)
        return sorted(s)

    def n_rotations(self):
        return sum(len([a for a in self.amounts(u) if a != 0]) for u in range(self.lin.n_shards))


def conv_plan(lin: Layout, W, bias, pad):
    """Stride-1 'same' convolution as sums of rotated, diagonal-weighted shards.

    Eq. 1 (shift operator), Eqs. 2-5 (partial convolutions, rotation by r m^2), Eq. 6
    (image shards), the duplication/permutation rule of Sec. 4 and Eq. 7 (channel shards),
    written in one general form: for output slot i of shard v (channel o, pixel y, x), input
    channel f and tap (k, l) the source pixel (y+k-pad, x+l-pad), if inside the image, is
    read from the copy (u, slot j) of channel f holding that row; the amount is
    a = (j - i) mod N and D_{u,v,a}[i] = W[o][f][k][l] (cross-correlation, as the paper's
    S_{k,l} shifts rows up and columns left).  Among duplicated copies the one with the
    smallest block offset (b_in - b_out) mod nb is used, which yields the paper's rotation
    set {r m^2 + shift : 0 <= r < c}.
    """
    W = np.asarray(W, dtype=np.float64)
    co, ci, kh, kw = W.shape
    assert ci == lin.c
    lout = image_layout(co, lin.m, lin.N)
    assert lout.M == lin.M
    plan = ConvPlan(lin, lout)
    N = lin.N
    # copies of each input channel: (u, b, row0)
    copies = {f: [] for f in range(ci)}
    for u in range(lin.n_shards):
        for b in range(lin.nb):
            f = lin.chan[u, b]
            if f >= 0:
                copies[f].append((u, b, lin.row0[u, b]))
    R = lin.rows_per_block
    for v in range(lout.n_shards):
        ch, y, x, valid = slot_coords(lout, v)
        i = np.arange(N)
        b_out = i // lout.B
        terms = {}
        for f in range(ci):
            for k in range(kh):
                for l in range(kw):
                    ys, xs = y + k - pad, x + l - pad
                    ok = valid & (ys >= 0) & (ys < lin.m) & (xs >= 0) & (xs < lin.m)
                    best_key = np.full(N, np.iinfo(np.int64).max)
                    best_u = np.full(N, -1)
                    best_j = np.full(N, -1)
                    for (u, b, r0) in copies[f]:
                        has = ok & (ys >= r0) & (ys < r0 + R)
                        key = ((b - b_out) % lin.nb) * (lin.n_shards + 1) + u
                        better = has & (key < best_key)
                        j = b * lin.B + (ys - r0) * lin.M + xs
                        best_key = np.where(better, key, best_key)
                        best_u = np.where(better, u, best_u)
                        best_j = np.where(better, j, best_j)
                    sel = ok & (best_u >= 0)
                    assert np.all(best_u[ok] >= 0), "source pixel missing from layout"
                    if not sel.any():
                        continue
                    a = (best_j - i) % N
                    wv = W[np.where(sel, ch, 0), f, k, l]
                    keys = best_u[sel] * N + a[sel]
                    idx = np.nonzero(sel)[0]
                    for key in np.unique(keys):
                        uu, aa = divmod(int(key), N)
                        D = terms.setdefault((uu, aa), np.zeros(N))
                        pos = idx[keys == key]
                        assert np.all(D[pos] == 0.0), "two taps hit one diagonal entry"
                        D[pos] = wv[pos]
        plan.terms[v] = terms
    bv = np.zeros((lout.n_shards, N))
    if bias is not None:
        bias = np.asarray(bias, dtype=np.float64)
        for v in range(lout.n_shards):
            ch, y, x, valid = slot_coords(lout, v)
            bv[v, valid] = bias[ch[valid]]
    plan.bias = bv
    return plan


def conv_slots(plan: ConvPlan, slots):
    """Slot simulator: out_v = sum_{(u,a)} D_{u,v,a} * roll(in_u, -a) + bias."""
    out = np.zeros((plan.lout.n_shards, plan.lin.N))
    for v, terms in plan.terms.items():
        for (u, a), D in terms.items():
            out[v] += D * np.roll(slots[u], -a)
        out[v] += plan.bias[v]
    return out


def conv_plaintexts(plan: ConvPlan, n, S):
    """Integer plaintexts of every diagonal, encoded at scale S: {(u, v, a): int64 [n]}."""
    return {(u, v, a): encode(D, n, S) for v, t in plan.terms.items() for (u, a), D in t.items()}


def rotate_all(ctx, cts, amounts_of):
    """Hoisted rotations {(u, a): ct} of every input shard by every amount it needs."""
    R = {}
    for u, ct in enumerate(cts):
        am = amounts_of(u)
        if not am:
            continue
        D = ctx.hoist(ct) if any(a != 0 for a in am) else None
        for a in am:
            if a != 0:
                ctx.gen_rotation_key(a)
            R[(u, a)] = ct.copy() if a == 0 else ctx.rotate_hoisted(ct, D, a)
    return R


def mac_rescale(ctx, R, terms, pts, level, scale_in, pt_scale=None):
    """Rescale(sum_{(u,a)} pt_{u,a} * R_{u,a}): the fused pt x ct MAC of one output shard.
    pt_scale: the plaintexts' encoding scale (default q_level, which keeps the scale exact)."""
    return ctx.rescale(mac(ctx, R, terms, pts, level, scale_in, pt_scale))


def mac(ctx, R, terms, pts, level, scale_in, pt_scale=None):
    """sum_{(u,a)} pt_{u,a} * R_{u,a}, unrescaled (scale scale_in * pt_scale)."""
    mods, psis = ctx.mods(level), ctx.psis(level)
    acc = [np.zeros((level + 1, ctx.n), dtype=np.uint64) for _ in range(2)]
    for (u, a), pt in zip(terms, pts):
        P = ctx.ntt(ctx.reduce_int(pt, mods), mods, psis).reshape(level + 1, ctx.n)
        for k in range(2):
            X = ctx.ntt(R[(u, a)].c[k], mods, psis).reshape(level + 1, ctx.n)
            ctx.lib.orc_mac(acc[k], P, X, level + 1, ctx.n, mods)
    from .ckks import Ciphertext
    c = np.stack([ctx.intt(x, mods, psis).reshape(level + 1, ctx.n) for x in acc])
    S = float(ctx.q[level]) if pt_scale is None else pt_scale
    return Ciphertext(c, level, scale_in * S)


def conv_he(ctx, plan: ConvPlan, cts, pts=None, bias_pts=None, pt_scale=None, outputs=None):
    """hconv2d on oracle ciphertexts (all inputs at one level and scale).

    pts: optional {(u, v, a): int64 plaintext} at scale q_level (else encoded here);
    bias_pts: optional {v: int64 plaintext} at the input scale (else encoded here).
    pt_scale: the scale pts were encoded at, when they were encoded for another (higher)
    level: an integer plaintext is the same at every level, only its residues are fewer.
    outputs: the output shards to compute (default: all of them), returned in ascending
    order; only the rotations those shards read are formed.
    """
    level, scale = cts[0].level, cts[0].scale
    assert all(c.level == level and c.scale == scale for c in cts)
    vs = list(range(plan.lout.n_shards)) if outputs is None else sorted(set(outputs))
    if pts is None:
        pts = conv_plaintexts(plan, ctx.n, float(ctx.q[level]))
    R = rotate_all(ctx, cts, lambda u: sorted({a for v in vs for (uu, a) in plan.terms[v] if uu == u}))
    out = []
    for v in vs:
        keys = sorted(plan.terms[v].keys())
        ct = mac_rescale(ctx, R, keys, [pts[(u, v, a)] for (u, a) in keys], level, scale, pt_scale)
        bpt = bias_pts[v] if bias_pts is not None else encode(plan.bias[v], ctx.n, ct.scale)
        ct.c[0] = ctx.add(ct.c[0], ctx.reduce_int(bpt, ctx.mods(ct.level)), ctx.mods(ct.level))
        out.append(ct)
    return out


def raised_stage(ctx, srcs, terms_by_v):
    """Weighted hoisted rotations with one ModDown per output ("double hoisting").

    out_v = (B0, B1) + ModDown( sum_{(s, a), a != 0} pt * u_{s,a} ),  where for source s
    rotated by a the hoisted inner product is u_{s,a} = sum_j phi_a(D_j(s)) * ksk_a[j] over
    Q u P, B0 = sum_{(s,a)} pt * phi_a(c0_s) and B1 = sum_{(s,0)} pt * c1_s.  pt is an integer
    plaintext reduced modulo every prime of Q u P, or None for the integer 1.  All sources share
    one level; outputs are returned unrescaled, scale = source scale (times the plaintext scale,
    applied by the caller).
    """
    from .ckks import Ciphertext
    level = srcs[0].level
    assert all(c.level == level for c in srcs)
    mq, pq = ctx.mods(level), ctx.psis(level)
    me, pe = ctx.mods(level, True), ctx.psis(level, True)
    nq, ne, n = level + 1, len(me), ctx.n
    one = np.zeros(n, dtype=np.int64)
    one[0] = 1
    rotated = {s for terms in terms_by_v.values() for (s, a, _) in terms if a % ctx.N != 0}
    D = {s: ctx.hoist(srcs[s]) for s in sorted(rotated)}
    c_eval = [[ctx.ntt(ct.c[k], mq, pq).reshape(nq, n) for k in range(2)] for ct in srcs]
    out = {}
    for v in sorted(terms_by_v):
        acc = [np.zeros((ne, n), dtype=np.uint64) for _ in range(2)]
        base = [np.zeros((nq, n), dtype=np.uint64) for _ in range(2)]
        for (s, a, pt) in terms_by_v[v]:
            pt = one if pt is None else pt
            Pq = ctx.ntt(ctx.reduce_int(pt, mq), mq, pq).reshape(nq, n)
            if a % ctx.N == 0:
                for k in range(2):
                    ctx.lib.orc_mac(base[k], Pq, c_eval[s][k], nq, n, mq)
                continue
            g = ctx.galois(a)
            ctx.gen_rotation_key(a)
            c0g = ctx.automorph_eval(c_eval[s][0], g).reshape(nq, n)
            ctx.lib.orc_mac(base[0], Pq, c0g, nq, n, mq)
            Pe = ctx.ntt(ctx.reduce_int(pt, me), me, pe).reshape(ne, n)
            keys = ctx._key_limbs(g, level)
            for k in range(2):
                uk = np.zeros((ne, n), dtype=np.uint64)
                for j, Dj in enumerate(D[s]):
                    ctx.lib.orc_mac(uk, ctx.automorph_eval(Dj, g).reshape(ne, n),
                                    np.ascontiguousarray(keys[j][k]), ne, n, me)
                ctx.lib.orc_mac(acc[k], Pe, uk, ne, n, me)
        c = []
        for k in range(2):
            y = ctx.moddown(ctx.intt(acc[k], me, pe).reshape(ne, n), level)
            c.append(ctx.add(ctx.intt(base[k], mq, pq).reshape(nq, n), y, mq))
        out[v] = Ciphertext(np.stack(c), level, srcs[0].scale)
    return [out[v] for v in sorted(out)]


def conv_he_raised(ctx, plan, cts, pts=None, bias_pts=None, pt_scale=None, outputs=None):
    """hconv2d with one ModDown per output shard (raised_stage), then rescale and bias.
    Same plan and plaintexts as conv_he; decrypts like it, different bits.  pt_scale and
    outputs as in conv_he."""
    level, scale = cts[0].level, cts[0].scale
    assert all(c.level == level and c.scale == scale for c in cts)
    vs = list(range(plan.lout.n_shards)) if outputs is None else sorted(set(outputs))
    if pts is None:
        pts = conv_plaintexts(plan, ctx.n, float(ctx.q[level]))
    terms = {v: [(u, a, pts[(u, v, a)]) for (u, a) in sorted(plan.terms[v].keys())] for v in vs}
    out = []
    for v, acc in zip(vs, raised_stage(ctx, cts, terms)):
        acc.scale = scale * (float(ctx.q[level]) if pt_scale is None else pt_scale)
        ct = ctx.rescale(acc)
        bpt = bias_pts[v] if bias_pts is not None else encode(plan.bias[v], ctx.n, ct.scale)
        ct.c[0] = ctx.add(ct.c[0], ctx.reduce_int(bpt, ctx.mods(ct.level)), ctx.mods(ct.level))
        out.append(ct)
    return out


# ============================================================================ BSGS convolution
def bsgs_split(a, B, N, k=1):
    """Amount a = g + t (mod N).  First a = r B + s with s the residue of a modulo the block
    length B taken in [-B/2, B/2) (the tap's row and column shift) and r = (a - s)/B mod N/B
    (the channel offset r m^2 of Eqs. 2-5); then with a giant stride of k blocks the baby step
    takes t = (r mod k) B + s and the giant step g = (r - r mod k) B.  k = 1: t is the tap
    shift; k = N/B: g = 0 (the diagonal form).  Both are returned as amounts in [0, N)."""
    s = a % B
    if 2 * s >= B:
        s -= B
    r = ((a - s) // B) % (N // B)
    return (r - r % k) * B % N, ((r % k) * B + s) % N


@dataclass
class BsgsPlan:
    """The diagonal plan regrouped baby-step / giant-step (double hoisting of the rotations of
    Eqs. 2-7): D_{u,v,a} (.) rot_a(X_u) = rot_g( rot_{-g}(D_{u,v,a}) (.) rot_t(X_u) ) with
    a = g + t, so

        S_{v,g} = sum_{(u,t)} rot_{-g}(D_{u,v,g+t}) (.) rot_t(X_u)     (baby steps, hoisted per u)
        out_v   = sum_g rot_g(S_{v,g}) + bias_v                       (giant steps)

    Rotations: the distinct non-zero t per input shard plus the distinct non-zero g per output
    shard, instead of the distinct non-zero a per input shard."""
    base: ConvPlan
    k: int = 1                                   # giant stride in blocks
    baby: dict = field(default_factory=dict)     # (v, g) -> {(u, t): rot_{-g}(D) float64 [N]}

    def keys(self):
        return sorted(self.baby)

    def baby_amounts(self, u):
        return sorted({t for d in self.baby.values() for (uu, t) in d if uu == u})

    def giants(self, v):
        return [g for (vv, g) in self.keys() if vv == v]

    def n_rotations(self):
        nb = sum(len([t for t in self.baby_amounts(u) if t != 0]) for u in range(self.base.lin.n_shards))
        ng = sum(len([g for g in self.giants(v) if g != 0]) for v in range(self.base.lout.n_shards))
        return nb + ng


def conv_plan_bsgs(plan: ConvPlan, giant_blocks=1):
    """Regroup a diagonal conv plan by (output shard, giant amount), every amount split with a
    giant stride of giant_blocks blocks of the input layout (bsgs_split).  giant_blocks = N/B
    leaves every g = 0: the diagonal form."""
    N, B = plan.lin.N, plan.lin.B
    assert giant_blocks >= 1 and (N // B) % giant_blocks == 0
    bp = BsgsPlan(plan, giant_blocks)
    for v, terms in plan.terms.items():
        for (u, a), D in terms.items():
            g, t = bsgs_split(a, B, N, giant_blocks)
            d = bp.baby.setdefault((v, g), {})
            assert (u, t) not in d
            d[(u, t)] = np.roll(D, g)               # rot_{-g}(D)
    return bp


def bsgs_slots(bp: BsgsPlan, slots):
    """Slot simulator of the BSGS form (np.roll as the rotation)."""
    out = np.zeros((bp.base.lout.n_shards, bp.base.lin.N))
    for (v, g), d in bp.baby.items():
        S = np.zeros(bp.base.lin.N)
        for (u, t), P in d.items():
            S += P * np.roll(slots[u], -t)
        out[v] += np.roll(S, -g)
    return out + bp.base.bias


def bsgs_plaintexts(bp: BsgsPlan, n, S):
    """Integer plaintexts of the rotated diagonals at scale S, keyed by the diagonal's own term
    (u, v, a = g + t)."""
    N = bp.base.lin.N
    return {(u, v, (g + t) % N): encode(P, n, S) for (v, g), d in bp.baby.items() for (u, t), P in d.items()}


def conv_he_bsgs(ctx, bp: BsgsPlan, cts, pts=None, bias_pts=None, pt_scale=None, raised=False):
    """hconv2d in the BSGS form, then rescale and bias.

    raised=False: baby steps are hoisted rotations of each input shard (one ModDown each), the
    S_{v,g} are plaintext MACs, and each S_{v,g} with g != 0 takes one hoisted rotation.
    raised=True: both steps are raised-basis stages (raised_stage): the baby step gives every
    S_{v,g} one ModDown, the giant step (plaintext 1) gives every output one ModDown.
    Rescaling once, after the giant step, leaves the output scale in * S_pt / q_level as in the
    diagonal form.  pts / bias_pts / pt_scale as in conv_he (pts keyed (u, v, a))."""
    level, scale = cts[0].level, cts[0].scale
    assert all(c.level == level and c.scale == scale for c in cts)
    N = bp.base.lin.N
    if pts is None:
        pts = bsgs_plaintexts(bp, ctx.n, float(ctx.q[level]))
    S_pt = float(ctx.q[level]) if pt_scale is None else pt_scale
    keys = bp.keys()
    nout = bp.base.lout.n_shards
    if raised:
        stage = {i: [(u, t, pts[(u, v, (g + t) % N)]) for (u, t) in sorted(bp.baby[(v, g)])]
                 for i, (v, g) in enumerate(keys)}
        S = raised_stage(ctx, cts, stage)
        for x in S:
            x.scale = scale * S_pt
        giant = {v: [(i, g, None) for i, (vv, g) in enumerate(keys) if vv == v] for v in range(nout)}
        accs = raised_stage(ctx, S, giant)
    else:
        R = rotate_all(ctx, cts, bp.baby_amounts)
        accs = [None] * nout
        for (v, g) in keys:
            terms = sorted(bp.baby[(v, g)])
            x = mac(ctx, R, terms, [pts[(u, v, (g + t) % N)] for (u, t) in terms], level, scale, pt_scale)
            if g != 0:
                ctx.gen_rotation_key(g)
                x = ctx.rotate_hoisted(x, ctx.hoist(x), g)
            accs[v] = x if accs[v] is None else ctx.add_ct(accs[v], x)
    out = []
    for v, acc in enumerate(accs):
        acc.scale = scale * S_pt
        ct = ctx.rescale(acc)
        bpt = bias_pts[v] if bias_pts is not None else encode(bp.base.bias[v], ctx.n, ct.scale)
        ct.c[0] = ctx.add(ct.c[0], ctx.reduce_int(bpt, ctx.mods(ct.level)), ctx.mods(ct.level))
        out.append(ct)
    return out


# ============================================================================ linear head
@dataclass
class LinearPlan:
    """Linear layer over a sharded image (Sec. 4 "Other Layers", Linear): output j is the dot
    product of the flattened feature map with row j of the weights.  w[(j, u)] holds row j on the
    first copy (shard, then block order) of every valid pixel of shard u, zero elsewhere, so
    duplicated channels are counted once."""
    lin: Layout
    n_out: int
    w: dict = field(default_factory=dict)        # (j, u) -> float64 [N]
    bias: np.ndarray = None                      # [n_out]

    def amounts(self):
        """The rotate-and-add shifts N/2, N/4, ..., 1."""
        out, s = [], self.lin.N // 2
        while s >= 1:
            out.append(s)
            s //= 2
        return out


def _first_copy_mask(lin: Layout):
    """[n_shards][N] bool: the slot is the first copy of its (channel, row, column)."""
    seen = set()
    masks = np.zeros((lin.n_shards, lin.N), dtype=bool)
    for u in range(lin.n_shards):
        ch, y, x, valid = slot_coords(lin, u)
        for i in np.nonzero(valid)[0]:
            key = (int(ch[i]), int(y[i]), int(x[i]))
            if key not in seen:
                seen.add(key)
                masks[u, i] = True
    return masks


def linear_plan(lin: Layout, W, bias=None):
    """W [n_out][c][m][m] (the flattened input's weights), bias [n_out] or None."""
    W = np.asarray(W, dtype=np.float64)
    n_out = W.shape[0]
    assert W.shape[1:] == (lin.c, lin.m, lin.m) and n_out <= lin.N
    first = _first_copy_mask(lin)
    plan = LinearPlan(lin, n_out, bias=np.zeros(n_out) if bias is None else np.asarray(bias, dtype=np.float64))
    for u in range(lin.n_shards):
        ch, y, x, valid = slot_coords(lin, u)
        sel = first[u]
        for j in range(n_out):
            v = np.zeros(lin.N)
            v[sel] = W[j, ch[sel], y[sel], x[sel]]
            plan.w[(j, u)] = v
    return plan


def pool_linear_plan(lin: Layout, W, bias=None):
    """Pool-linear (Sec. 4 "Other Layers"): every m x m channel averaged to one value, then a
    linear layer W [n_out][c]; the weights are spread over the channel's pixels and divided by
    the normalisation factor m^2."""
    W = np.asarray(W, dtype=np.float64)
    full = np.repeat(np.repeat(W[:, :, None, None], lin.m, 2), lin.m, 3) / float(lin.m * lin.m)
    return linear_plan(lin, full, bias)


def linear_slots(plan: LinearPlan, slots):
    """Slot simulator: T_j = sum_u w_{j,u} * x_u, summed over all slots by rotate-and-add
    (T += roll(T, -s) for s = N/2, ..., 1), masked to slot j and summed; plus the bias."""
    out = np.zeros(plan.lin.N)
    for j in range(plan.n_out):
        T = sum(plan.w[(j, u)] * slots[u] for u in range(plan.lin.n_shards))
        for s in plan.amounts():
            T = T + np.roll(T, -s)
        e = np.zeros(plan.lin.N)
        e[j] = 1.0
        out += e * T
    out[: plan.n_out] += plan.bias
    return out


def linear_plaintexts(plan: LinearPlan, n, S_w, S_mask):
    """Integer plaintexts: weights {(j, u)} at scale S_w, masks e_j {j} at scale S_mask."""
    w = {k: encode(v, n, S_w) for k, v in plan.w.items()}
    masks = {}
    for j in range(plan.n_out):
        e = np.zeros(plan.lin.N)
        e[j] = 1.0
        masks[j] = encode(e, n, S_mask)
    return w, masks


HEAD_BOOST_BITS = 12


def linear_scales(ctx, level):
    """(weight scale, mask scale) of the head at input level l: q_l 2^b and q_{l-1} / 2^b.

    The slot sum adds every slot of a partial sum, and each of its log2 steps doubles the noise
    of the key switches before it (up to N/2 times at the first one), so the sum runs at scale
    Delta 2^b; the masks take the 2^b back out, leaving the output at Delta exactly."""
    return float(ctx.q[level]) * 2.0 ** HEAD_BOOST_BITS, float(ctx.q[level - 1]) / 2.0 ** HEAD_BOOST_BITS


def linear_he(ctx, plan: LinearPlan, cts, w_pts=None, mask_pts=None, bias_pt=None):
    """The linear layer on oracle ciphertexts (all shards at one level l >= 2, one scale):
    T_j = Rescale(sum_u w_{j,u} * x_u) with weights at scale S_w; for s = N/2, ..., 1 the
    hoisted rotation T_j += rot_s(T_j); out = Rescale(sum_j e_j * T_j) with masks at scale
    S_mask; plus the bias (slots 0..n_out-1) at the output scale.  (S_w, S_mask) =
    linear_scales.  Output level l - 2, output scale the input scale."""
    level, scale = cts[0].level, cts[0].scale
    assert level >= 2 and all(c.level == level and c.scale == scale for c in cts)
    S_w, S_mask = linear_scales(ctx, level)
    if w_pts is None or mask_pts is None:
        w_pts, mask_pts = linear_plaintexts(plan, ctx.n, S_w, S_mask)
    R = {(u, 0): ct for u, ct in enumerate(cts)}
    terms = [(u, 0) for u in range(plan.lin.n_shards)]
    T = []
    for j in range(plan.n_out):
        t = ctx.rescale(mac(ctx, R, terms, [w_pts[(j, u)] for u in range(plan.lin.n_shards)], level, scale, S_w))
        for s in plan.amounts():
            ctx.gen_rotation_key(s)
            t = ctx.add_ct(t, ctx.rotate_hoisted(t, ctx.hoist(t), s))
        T.append(t)
    acc = mac(ctx, {(j, 0): t for j, t in enumerate(T)}, [(j, 0) for j in range(plan.n_out)],
              [mask_pts[j] for j in range(plan.n_out)], level - 1, T[0].scale, S_mask)
    out = ctx.rescale(acc)
    if bias_pt is None:
        b = np.zeros(plan.lin.N)
        b[: plan.n_out] = plan.bias
        bias_pt = encode(b, ctx.n, out.scale)
    out.c[0] = ctx.add(out.c[0], ctx.reduce_int(bias_pt, ctx.mods(out.level)), ctx.mods(out.level))
    return out


# ---------------------------------------------------------------------------- packed head
def linear_packed_width(n_out):
    """n' = the smallest power of two >= n_out: output j is gathered in slot j of n'-periodic sums."""
    return 1 << max(0, (int(n_out) - 1).bit_length())


def linear_packed_weights(plan: LinearPlan):
    """Q_{u,d}[i] = w_{i mod n', u}[(i + d) mod N] (zero where i mod n' >= n_out), d < n'.

    Sum_u Sum_d Q_{u,d} (.) rot_d(X_u) puts, in every slot i, the terms of output j = i mod n'
    at the slots i + d; summing the slots of one residue class mod n' (rotate-and-add by N/2,
    ..., n') then covers every slot of every shard exactly once: out_j in slot j.  The same
    dot products as the per-output form with n' hoisted rotations per shard and log2(N/n')
    shifts instead of n_out log2 N."""
    N = plan.lin.N
    npk = linear_packed_width(plan.n_out)
    i = np.arange(N)
    j = i % npk
    Q = {}
    for u in range(plan.lin.n_shards):
        W = np.stack([plan.w[(jj, u)] for jj in range(plan.n_out)] +
                     [np.zeros(N)] * (npk - plan.n_out))            # [n'][N]
        for d in range(npk):
            Q[(u, d)] = W[j, (i + d) % N]
    return Q


def linear_packed_shifts(plan: LinearPlan):
    npk, out, s = linear_packed_width(plan.n_out), [], plan.lin.N // 2
    while s >= npk:
        out.append(s)
        s //= 2
    return out


def linear_packed_slots(plan: LinearPlan, slots):
    """Slot simulator of the packed head."""
    N = plan.lin.N
    C = np.zeros(N)
    for (u, d), q in linear_packed_weights(plan).items():
        C += q * np.roll(slots[u], -d)
    for s in linear_packed_shifts(plan):
        C = C + np.roll(C, -s)
    e = np.zeros(N)
    e[: plan.n_out] = 1.0
    out = e * C
    out[: plan.n_out] += plan.bias
    return out


def linear_packed_plaintexts(plan: LinearPlan, n, S_w, S_mask):
    """Integer plaintexts: packed weights {(u, d)} at scale S_w, the first-n_out mask at S_mask."""
    e = np.zeros(plan.lin.N)
    e[: plan.n_out] = 1.0
    return {k: encode(v, n, S_w) for k, v in linear_packed_weights(plan).items()}, encode(e, n, S_mask)


def linear_packed_he(ctx, plan: LinearPlan, cts, w_pts=None, mask_pt=None, bias_pt=None):
    """The packed head on oracle ciphertexts: C = Rescale(raised stage sum_{(u,d)} Q_{u,d} (.)
    rot_d(X_u)) (one ModDown), C += hoisted rot_s(C) for s = N/2, ..., n', out =
    Rescale(mask (.) C) + bias.  Levels and scales as in linear_he; different bits."""
    level, scale = cts[0].level, cts[0].scale
    assert level >= 2 and all(c.level == level and c.scale == scale for c in cts)
    npk = linear_packed_width(plan.n_out)
    S_w, S_mask = linear_scales(ctx, level)
    if w_pts is None or mask_pt is None:
        w_pts, mask_pt = linear_packed_plaintexts(plan, ctx.n, S_w, S_mask)
    terms = {0: [(u, d, w_pts[(u, d)]) for u in range(plan.lin.n_shards) for d in range(npk)]}
    C = raised_stage(ctx, cts, terms)[0]
    C.scale = scale * S_w
    C = ctx.rescale(C)
    for s in linear_packed_shifts(plan):
        ctx.gen_rotation_key(s)
        C = ctx.add_ct(C, ctx.rotate_hoisted(C, ctx.hoist(C), s))
    out = ctx.rescale(mac(ctx, {(0, 0): C}, [(0, 0)], [mask_pt], level - 1, C.scale, S_mask))
    if bias_pt is None:
        b = np.zeros(plan.lin.N)
        b[: plan.n_out] = plan.bias
        bias_pt = encode(b, ctx.n, out.scale)
    out.c[0] = ctx.add(out.c[0], ctx.reduce_int(bias_pt, ctx.mods(out.level)), ctx.mods(out.level))
    return out


# ============================================================================ factored conv
@dataclass
class FactoredPlan:
    """Channel-shard convolution in two stages (Eq. 7 with the weights taken out of the masks).

    Every shard holds R = N/M consecutive rows of one channel, H = M/R shards per channel.  For
    tap t = (k, l) the source pixel of an output slot lies in the same shard or in a
    neighbouring one, always at the same rotation amount a_t = ((k - pad) M + (l - pad)) mod N
    (the shared amount of Eq. 7).  Stage 1 forms, per input channel f, shard h and tap t,
        Y_{f,h,t} = sum_{h'} B_{h,h',t} (.) rot_{a_t}(X_{f,h'})
    with binary masks B that depend on (h, h', t) only (every channel has the same geometry);
    stage 2 weights them with integer scalars:
        out_{o,h} = sum_{f,t} round(W[o][f][t] q) Y_{f,h,t} / q + bias.
    Two levels instead of one; mask plaintexts number 2 H T at most instead of co ci H T."""
    lin: Layout
    lout: Layout
    H: int                    # shards per channel
    pad: int
    taps: list                # [(k, l)]
    amounts: list             # a_t per tap
    masks: dict               # (h, h_src, t) -> float64 [N] in {0, 1}
    W: np.ndarray             # [co][ci][kh][kw]
    bias: np.ndarray          # [n_out][N]

    def sources(self, f, h, t):
        """[(input shard, mask key)] summed into Y_{f,h,t}."""
        return [(f * self.H + hs, key) for key in sorted(self.masks) if key[0] == h and key[2] == t
                for hs in [key[1]]]


def conv_plan_factored(lin: Layout, W, bias, pad):
    W = np.asarray(W, dtype=np.float64)
    co, ci, kh, kw = W.shape
    assert ci == lin.c and lin.nb == 1 and lin.B == lin.N, "channel shards only"
    M, N, R = lin.M, lin.N, lin.rows_per_block
    H = M // R
    assert lin.n_shards == ci * H
    lout = image_layout(co, lin.m, N)
    i = np.arange(N)
    taps = [(k, l) for k in range(kh) for l in range(kw)]
    amounts, masks = [], {}
    for t, (k, l) in enumerate(taps):
        a = ((k - pad) * M + (l - pad)) % N
        amounts.append(a)
        for h in range(H):
            ch, y, x, valid = slot_coords(lout, h)      # shard h of output channel 0
            ys, xs = y + k - pad, x + l - pad
            ok = valid & (ys >= 0) & (ys < lin.m) & (xs >= 0) & (xs < lin.m)
            hs = np.where(ok, ys // R, -1)
            j = (ys - hs * R) * M + xs
            assert np.all(((j - i) % N)[ok] == a), "own and neighbour reads share the amount"
            for h_src in np.unique(hs[ok]):
                masks[(h, int(h_src), t)] = (ok & (hs == h_src)).astype(np.float64)
    bv = np.zeros((lout.n_shards, N))
    if bias is not None:
        bias = np.asarray(bias, dtype=np.float64)
        for v in range(lout.n_shards):
            ch, y, x, valid = slot_coords(lout, v)
            bv[v, valid] = bias[ch[valid]]
    return FactoredPlan(lin, lout, H, pad, taps, amounts, masks, W, bv)


def factored_slots(plan: FactoredPlan, slots):
    """Slot simulator of both stages (float64 weights)."""
    co, ci = plan.W.shape[:2]
    H, N = plan.H, plan.lin.N
    out = np.zeros((plan.lout.n_shards, N))
    for f in range(ci):
        for h in range(H):
            for t, (k, l) in enumerate(plan.taps):
                Y = np.zeros(N)
                for (u, key) in plan.sources(f, h, t):
                    Y += plan.masks[key] * np.roll(slots[u], -plan.amounts[t])
                for o in range(co):
                    out[o * H + h] += plan.W[o, f, k, l] * Y
    return out + plan.bias


def round_half_away(x):
    return int(math.copysign(math.floor(abs(x) + 0.5), x))


def factored_scalars(plan: FactoredPlan, q):
    """Stage-2 integer weights round(W[o][f][t] q), [co][ci][T] python ints."""
    co, ci = plan.W.shape[:2]
    return [[[round_half_away(float(plan.W[o, f, k, l]) * float(q)) for (k, l) in plan.taps]
             for f in range(ci)] for o in range(co)]


def mask_plaintexts(plan: FactoredPlan, n, S):
    """Integer plaintexts of the masks at scale S: {(h, h_src, t): int64 [n]}."""
    return {key: encode(m, n, S) for key, m in plan.masks.items()}


def conv_he_factored(ctx, plan: FactoredPlan, cts, mask_pts=None, bias_pts=None, raised=False):
    """Both stages on oracle ciphertexts (inputs at one level l, scale s): stage 1 at level l
    (masks at scale q_l, rescale), stage 2 with integer scalars round(w q_{l-1}) (rescale),
    then the bias: output at level l - 2.  raised=True takes stage 1 with one ModDown per Y
    (raised_stage) instead of one per rotation; different bits, same decryption."""
    from .ckks import Ciphertext
    level, scale = cts[0].level, cts[0].scale
    assert all(c.level == level and c.scale == scale for c in cts)
    co, ci = plan.W.shape[:2]
    H, T = plan.H, len(plan.taps)
    if mask_pts is None:
        mask_pts = mask_plaintexts(plan, ctx.n, float(ctx.q[level]))
    ykeys = [(f, h, t) for f in range(ci) for h in range(H) for t in range(T)]
    Y = {}
    if raised:
        terms = {y: [(u, plan.amounts[t], mask_pts[key]) for (u, key) in plan.sources(f, h, t)]
                 for y, (f, h, t) in enumerate(ykeys)}
        outs = raised_stage(ctx, cts, terms)
        for y, key in enumerate(ykeys):
            outs[y].scale = scale * float(ctx.q[level])
            Y[key] = ctx.rescale(outs[y])
    else:
        R = rotate_all(ctx, cts, lambda u: sorted({plan.amounts[t] for t in range(T)}))
        for (f, h, t) in ykeys:
            src = plan.sources(f, h, t)
            Y[(f, h, t)] = mac_rescale(ctx, R, [(u, plan.amounts[t]) for (u, _) in src],
                                       [mask_pts[key] for (_, key) in src], level, scale)
    l1 = level - 1
    mods = ctx.mods(l1)
    Wt = factored_scalars(plan, ctx.q[l1])
    out = []
    for o in range(co):
        for h in range(H):
            acc = [np.zeros((l1 + 1, ctx.n), dtype=np.uint64) for _ in range(2)]
            for f in range(ci):
                for t in range(T):
                    w = np.array([Wt[o][f][t] % int(q) for q in mods], dtype=np.uint64)
                    y = Y[(f, h, t)]
                    for k in range(2):
                        acc[k] = ctx.add(acc[k], ctx.mul_scalar(y.c[k], w, mods), mods)
            ct = ctx.rescale(Ciphertext(np.stack(acc), l1, Y[(0, h, 0)].scale * float(ctx.q[l1])))
            v = o * H + h
            bpt = bias_pts[v] if bias_pts is not None else encode(plan.bias[v], ctx.n, ct.scale)
            ct.c[0] = ctx.add(ct.c[0], ctx.reduce_int(bpt, ctx.mods(ct.level)), ctx.mods(ct.level))
            out.append(ct)
    return out


# ============================================================================ pooling
@dataclass
class PoolPlan:
    lin: Layout
    lout: Layout
    pre: list            # amounts summed unmasked before downsampling (S stage)
    h_terms: list        # [(amount, mask float64 [N])] horizontal reduction
    v_terms: list        # [(amount, mask float64 [N])] vertical reduction
    groups: list         # consolidation: list over output shards of [(input shard, amount)]
    dup: list            # duplication amounts applied to the consolidated shard (incl. 0)


def pool_plan(lin: Layout, weights=(0.25, 0.25, 0.25, 0.25), select_top_left=False):
    """2x2 average pool (Sec. 4.2), or the stride-2 downsample when select_top_left.

    S: W = X + rot_1 X + rot_M X + rot_{M+1} X      (the 2x2 ones convolution, unmasked)
    H: Y = sum_{x'} mask_{x'} * rot_{x'}(W)          (Eq. 10, rotate-then-mask form)
    V: Z = sum_{y'} mask_{y'} * rot_{3 y' M/2}(Y)     (Eq. 11)
    C: consolidate 4 shards into one (Eq. 12), or duplicate when 1-2 shards remain (Eq. 13).
    With select_top_left the S stage is skipped and the masks carry weight 1 (the paper's
    strided convolution = unstrided convolution + downsampling, Sec. 4.1).
    """
    M, N, B, m = lin.M, lin.N, lin.B, lin.m
    assert m % 2 == 0 and M >= 2
    Mh = M // 2
    Rb = lin.rows_per_block
    assert Rb % 2 == 0 or Rb == 1
    w = 1.0 if select_top_left else 0.25
    pre = [] if select_top_left else [0, 1, M, M + 1]
    i = np.arange(N)
    loc = i % B
    lr = loc // M                 # local row within the block
    col = i % M
    blk = i // B
    h_terms = []
    for xp in range(m // 2):
        masks = np.zeros((lin.n_shards, N))
        for u in range(lin.n_shards):
            ch = lin.chan[u][blk]
            y = lin.row0[u][blk] + lr
            sel = (ch >= 0) & (y % 2 == 0) & (y < m) & (col == xp)
            masks[u, sel] = w
        h_terms.append((xp, masks))
    v_terms = []
    for yp in range(max(Rb // 2, 1)):
        amount = 3 * yp * M // 2
        masks = np.zeros((lin.n_shards, N))
        for u in range(lin.n_shards):
            ch = lin.chan[u][blk]
            ynew = lin.row0[u][blk] // 2 + yp
            sel = (ch >= 0) & (loc >= yp * Mh) & (loc < yp * Mh + m // 2) & (ynew < m // 2)
            masks[u, sel] = 1.0
        if masks.any():
            v_terms.append((amount, masks))
    # new layout: old block b of shard s -> new block 4b + q of output shard s // 4 (q = s % 4)
    Bn = B // 4
    nbn = N // Bn
    t = lin.n_shards
    n_out = -(-t // 4)
    chan = np.full((n_out, nbn), -1, dtype=np.int64)
    row0 = np.zeros((n_out, nbn), dtype=np.int64)
    groups = []
    for g in range(n_out):
        grp = []
        for q in range(4):
            s = 4 * g + q
            if s >= t:
                break
            grp.append((s, (-q * Bn) % N))
            for b in range(lin.nb):
                chan[g, 4 * b + q] = lin.chan[s, b]
                row0[g, 4 * b + q] = lin.row0[s, b] // 2
        groups.append(grp)
    dup = [0]
    if t in (1, 2):
        f = 4 // t
        step = t * Bn
        dup = [(-k * step) % N for k in range(f)]
        # Eq. 13: block b of the duplicated shard sums the consolidated blocks b - k t (k < f);
        # it holds the channel of whichever of them holds data, so the table before
        # duplication is the one read (an empty block stays empty)
        chan0, row00 = chan[0].copy(), row0[0].copy()
        for k in range(1, f):
            for b in range(nbn):
                src = b - k * (step // Bn)
                if src >= 0 and chan0[src] >= 0 and chan[0, b] < 0:
                    chan[0, b] = chan0[src]
                    row0[0, b] = row00[src]
    lout = Layout(lin.c, m // 2, Mh, N, Bn, chan, row0)
    return PoolPlan(lin, lout, pre, h_terms, v_terms, groups, dup)


def pool_slots(plan: PoolPlan, slots):
    out_sh = []
    Z = []
    for u in range(plan.lin.n_shards):
        x = slots[u]
        Wv = sum(np.roll(x, -a) for a in plan.pre) if plan.pre else x
        Y = sum(mk[u] * np.roll(Wv, -a) for a, mk in plan.h_terms)
        Z.append(sum(mk[u] * np.roll(Y, -a) for a, mk in plan.v_terms))
    for grp in plan.groups:
        S = sum(np.roll(Z[s], -a) for s, a in grp)
        out_sh.append(S)
    if len(plan.dup) > 1:
        out_sh = [sum(np.roll(out_sh[0], -a) for a in plan.dup)]
    return np.stack(out_sh)


def _masked_stage(ctx, cts, terms, level):
    """Rescale(sum_a Encode(mask_a, q_level) * rot_a(ct)) for every shard."""
    out = []
    for u, ct in enumerate(cts):
        R = rotate_all(ctx, [ct], lambda _u: [a for a, _ in terms])
        keys = [(0, a) for a, _ in terms]
        pts = [encode(mk[u], ctx.n, float(ctx.q[level])) for _, mk in terms]
        out.append(mac_rescale(ctx, R, keys, pts, level, ct.scale))
    return out


def pool_he_raised(ctx, plan: PoolPlan, cts, h_pts=None, v_pts=None):
    """havgpool with every stage (ones-sum, H, V, consolidate, duplicate) as a raised_stage:
    one ModDown per output shard per stage.  h_pts/v_pts: optional integer masks
    [amount][shard] (else encoded here at q_l and q_{l-1})."""
    level = cts[0].level
    ns = plan.lin.n_shards
    if h_pts is None:
        h_pts = [[encode(mk[u], ctx.n, float(ctx.q[level])) for u in range(ns)] for _, mk in plan.h_terms]
    if v_pts is None:
        v_pts = [[encode(mk[u], ctx.n, float(ctx.q[level - 1])) for u in range(ns)] for _, mk in plan.v_terms]
    W = cts
    if plan.pre:
        W = raised_stage(ctx, cts, {u: [(u, a, None) for a in plan.pre] for u in range(ns)})
    Y = raised_stage(ctx, W, {u: [(u, a, h_pts[i][u]) for i, (a, _) in enumerate(plan.h_terms)]
                              for u in range(ns)})
    Y2 = []
    for y in Y:
        y.scale = W[0].scale * ctx.q[level]
        Y2.append(ctx.rescale(y))
    Z = raised_stage(ctx, Y2, {u: [(u, a, v_pts[i][u]) for i, (a, _) in enumerate(plan.v_terms)]
                               for u in range(ns)})
    Z2 = []
    for z in Z:
        z.scale = Y2[0].scale * ctx.q[level - 1]
        Z2.append(ctx.rescale(z))
    S = raised_stage(ctx, Z2, {g: [(s, a, None) for s, a in grp] for g, grp in enumerate(plan.groups)})
    if len(plan.dup) > 1:
        S = raised_stage(ctx, [S[0]], {0: [(0, a, None) for a in plan.dup]})
    return S


def pool_he(ctx, plan: PoolPlan, cts):
    level = cts[0].level
    Ws = []
    for ct in cts:
        if plan.pre:
            R = rotate_all(ctx, [ct], lambda _u: plan.pre)
            acc = R[(0, plan.pre[0])]
            for a in plan.pre[1:]:
                acc = ctx.add_ct(acc, R[(0, a)])
            Ws.append(acc)
        else:
            Ws.append(ct)
    Ys = _masked_stage(ctx, Ws, plan.h_terms, level)
    Zs = _masked_stage(ctx, Ys, plan.v_terms, level - 1)
    outs = []
    for grp in plan.groups:
        acc = None
        for s, a in grp:
            r = rotate_all(ctx, [Zs[s]], lambda _u: [a])[(0, a)]
            acc = r if acc is None else ctx.add_ct(acc, r)
        outs.append(acc)
    if len(plan.dup) > 1:
        R = rotate_all(ctx, [outs[0]], lambda _u: plan.dup)
        acc = R[(0, plan.dup[0])]
        for a in plan.dup[1:]:
            acc = ctx.add_ct(acc, R[(0, a)])
        outs = [acc]
    return outs


# ============================================================================ polynomial
def cheb_nodes_coeffs(f, deg, lo, hi):
    """Chebyshev interpolant of f on [lo, hi] at the deg+1 first-kind nodes (Appendix,
    'Chebyshev Basis'): returns c_0..c_deg with p(x) = sum c_k T_k(t), t = (2x-lo-hi)/(hi-lo)."""
    K = deg + 1
    k = np.arange(K)
    t = np.cos(np.pi * (k + 0.5) / K)
    fx = np.array([f(0.5 * (hi - lo) * tt + 0.5 * (hi + lo)) for tt in t])
    c = np.zeros(K)
    for j in range(K):
        c[j] = 2.0 / K * np.sum(fx * np.cos(j * np.pi * (k + 0.5) / K))
    c[0] *= 0.5
    return c


def cheb_eval(c, x, lo, hi):
    """p(x) = sum c_k T_k(t) with T_k(t) = cos(k arccos t) by the three-term recurrence."""
    t = (2.0 * np.asarray(x, dtype=np.float64) - lo - hi) / (hi - lo)
    T0, T1 = np.ones_like(t), t
    acc = c[0] * T0 + (c[1] * T1 if len(c) > 1 else 0.0)
    for k in range(2, len(c)):
        T0, T1 = T1, 2.0 * t * T1 - T0
        acc = acc + c[k] * T1
    return acc


def minimax_coeffs(f, deg, lo, hi, iters=80, tol=1e-10):
    """Best uniform (minimax) approximation of degree deg to f on [lo, hi] by the Remez exchange
    algorithm (Appendix, 'Chebyshev Basis': the alternative to Chebyshev interpolation whose
    errors the approximation table also lists).  Chebyshev coefficients on [lo, hi] as in
    cheb_nodes_coeffs; returns (c, E) with E the levelled error.

    Start from the deg+2 Chebyshev extrema; each step solves p(x_i) + (-1)^i E = f(x_i) on the
    reference, then takes as the new reference one extremum of f - p per run of constant sign
    (scanned on a fine grid and refined by golden-section search), keeping deg+2 of them with
    alternating signs; stop when the largest error equals |E| to a relative tol."""
    n = deg + 2
    fv = np.vectorize(f, otypes=[np.float64])

    def X(t):
        return 0.5 * (hi - lo) * np.asarray(t) + 0.5 * (hi + lo)

    def err(t, c):
        return fv(X(t)) - cheb_eval(c, X(t), lo, hi)

    tg = np.unique(np.concatenate([np.cos(np.pi * np.arange(400 * n + 1) / (400 * n)), [0.0]]))
    fg = fv(X(tg))
    ref = np.cos(np.pi * np.arange(n) / (n - 1))[::-1].copy()
    for _ in range(iters):
        A = np.zeros((n, n))
        T0, T1 = np.ones(n), ref.copy()
        A[:, 0] = T0
        if deg >= 1:
            A[:, 1] = T1
        for k in range(2, deg + 1):
            T0, T1 = T1, 2.0 * ref * T1 - T0
            A[:, k] = T1
        A[:, deg + 1] = (-1.0) ** np.arange(n)
        sol = np.linalg.solve(A, fv(X(ref)))
        c, E = sol[: deg + 1], sol[deg + 1]
        r = fg - cheb_eval(c, X(tg), lo, hi)
        # one extremum per run of constant sign
        sg = np.sign(r)
        ext = []
        i = 0
        while i < len(tg):
            j = i
            while j + 1 < len(tg) and sg[j + 1] == sg[i]:
                j += 1
            k = i + int(np.argmax(np.abs(r[i:j + 1])))
            ext.append(k)
            i = j + 1
        # refine each by golden-section search between its grid neighbours
        pts, vals = [], []
        gr = (math.sqrt(5.0) - 1.0) / 2.0
        for k in ext:
            a, b = tg[max(k - 1, 0)], tg[min(k + 1, len(tg) - 1)]
            s_ = np.sign(r[k]) if r[k] != 0 else 1.0
            x1, x2 = b - gr * (b - a), a + gr * (b - a)
            f1, f2 = s_ * err(x1, c), s_ * err(x2, c)
            for _ in range(60):
                if f1 > f2:
                    b, x2, f2 = x2, x1, f1
                    x1 = b - gr * (b - a)
                    f1 = s_ * err(x1, c)
                else:
                    a, x1, f1 = x1, x2, f2
                    x2 = a + gr * (b - a)
                    f2 = s_ * err(x2, c)
            cand = [(s_ * r[k], tg[k]), (f1, x1), (f2, x2)]
            best = max(cand)
            pts.append(best[1])
            vals.append(s_ * best[0])
        pts, vals = list(pts), list(vals)
        while len(pts) > n:                      # keep n alternating extrema
            if len(pts) == n + 1:
                drop = 0 if abs(vals[0]) < abs(vals[-1]) else len(pts) - 1
                del pts[drop], vals[drop]
                continue
            k = int(np.argmin(np.abs(vals)))
            if k == 0 or k == len(pts) - 1:
                del pts[k], vals[k]
            else:
                kk = k - 1 if abs(vals[k - 1]) < abs(vals[k + 1]) else k + 1
                for d in sorted((k, kk), reverse=True):
                    del pts[d], vals[d]
        if len(pts) < n:
            raise RuntimeError("Remez: fewer alternation points than deg + 2")
        ref = np.array(pts)
        emax = max(abs(v) for v in vals)
        if emax - abs(E) <= tol * emax:
            break
    return c, abs(E)


def gelu(x):
    return 0.5 * x * (1.0 + math.erf(x / math.sqrt(2.0)))


def relu(x):
    return max(x, 0.0)


def cheb_tree_slots(c, t):
    """The paper's binary-tree recursion (Appendix, 'Chebyshev Polynomials'):
    T_{2k} = 2 T_k^2 - 1, T_{2k+1} = 2 T_k T_{k+1} - T_1, then sum c_k T_k, on cleartext."""
    T = {0: np.ones_like(t), 1: t}
    for k in range(2, len(c)):
        h = k // 2
        T[k] = 2 * T[h] * T[h] - 1 if k % 2 == 0 else 2 * T[h] * T[h + 1] - T[1]
    return sum(c[k] * T[k] for k in range(len(c)))


def cheb_ps_params(deg):
    """Paterson-Stockmeyer split for degree deg: baby steps T_1..T_k (k a power of two near
    sqrt((deg + 1) / 2)) and giant steps T_k, T_2k, T_4k, ... <= deg."""
    k = 2
    while k * k < (deg + 1) // 2:
        k *= 2
    giants = []
    g = k
    while g <= deg:
        giants.append(g)
        g *= 2
    return k, giants


def cheb_divide(c, G):
    """Chebyshev division p = q T_G + r (deg p < 2G): with T_G T_j = (T_{G+j} + T_{|G-j|}) / 2,
    q_0 = c_G, q_j = 2 c_{G+j} (j >= 1), r_i = c_i - c_{2G-i} for i < G (c beyond deg p is 0)."""
    d = len(c) - 1
    q = [c[G]] + [2.0 * c[G + j] for j in range(1, d - G + 1)]
    r = [c[i] - (c[2 * G - i] if 2 * G - i <= d and i >= 1 else 0.0) for i in range(G)]
    return q, r


def cheb_ps_slots(c, t):
    """Paterson-Stockmeyer evaluation of sum c_k T_k(t) on cleartext (same recursion as the HE form)."""
    deg = len(c) - 1
    k, giants = cheb_ps_params(deg)
    T = {0: np.ones_like(t), 1: t}
    for j in range(2, max([k] + giants) + 1):
        if j <= k or j in giants:
            h = j // 2
            T[j] = 2 * T[h] * T[h] - 1 if j % 2 == 0 else 2 * T[h] * T[h + 1] - T[1]

    def ev(cc):
        d = len(cc) - 1
        if d < k:
            return sum(cc[i] * T[i] for i in range(d + 1))
        G = max(g for g in giants if g <= d)
        q, r = cheb_divide(cc, G)
        return ev(q) * T[G] + ev(r)
    return ev(list(c))


def cheb_ps_need(cc, k, giants):
    """Levels the Paterson-Stockmeyer evaluation of sum cc_i T_i consumes below its input's
    level (cheb_ps_he's recursion; T_i of the binary tree costs bit_length(i - 1) levels)."""
    d = len(cc) - 1
    depth = lambda i: (i - 1).bit_length()
    if d < k:
        return 1 + max([depth(i) for i in range(1, d + 1)] + [0])
    G = max(g for g in giants if g <= d)
    q, r = cheb_divide(cc, G)
    if len(q) == 1 and G - 1 < k:
        return 1 + max([depth(G)] + [depth(i) for i in range(1, G)])
    if len(q) == 1:
        return max(1 + depth(G), cheb_ps_need(r, k, giants))
    return max(cheb_ps_need(q, k, giants) + 1, depth(G) + 1, cheb_ps_need(r, k, giants))


def cheb_ps_he(ctx, ct, c, target_scale=None):
    """Homomorphic Paterson-Stockmeyer evaluation of sum c_k T_k(ct) in the Chebyshev basis.

    Baby steps T_1..T_k and giant steps T_k, T_2k, ... come from the binary-tree recursion
    (the same products and exact-scale re-targeting as cheb_tree_he).  ev(p, l, s) returns p at
    level l and scale s (the scale of a product is s' = s_q s_G / q_{l+1}, within rounding of s):
      * deg p < k (or p = q_0 T_G + r with a constant quotient and deg r < k): one exact-scale
        linear combination sum round(c_i s q_{l+1} / s_i) T_i at level l + 1, then a rescale; a
        constant quotient with a larger remainder adds q_0 T_G (one combination) to ev(r, l, s);
      * otherwise p = q T_G + r: Q = ev(q, l + 1, s q_{l+1} / s_G), then mul_relin(Q, T_G) lands at
        level l with scale s', and r is evaluated to exactly (l, s') and added.
    The output level is the highest the recursion allows."""
    target_scale = ctx.pr.scale if target_scale is None else target_scale
    deg = len(c) - 1
    k, giants = cheb_ps_params(deg)
    T = {1: ct}

    def retarget(x, level, scale_t):
        y = ctx.drop_to(x, level + 1)
        K = int(round(scale_t * ctx.q[level + 1] / y.scale))
        y = ctx.mul_int(y, K)
        y = ctx.rescale(y)
        y.scale = scale_t
        return y

    for j in range(2, max([k] + giants) + 1):
        if not (j <= k or j in giants):
            continue
        h = j // 2
        if j % 2 == 0:
            p = ctx.mul_relin(T[h], T[h])
            p = ctx.mul_int(p, 2)
            p = ctx.add_const_int(p, -int(round(p.scale)))
        else:
            a, b = T[h], T[h + 1]
            lv = min(a.level, b.level)
            p = ctx.mul_relin(ctx.drop_to(a, lv), ctx.drop_to(b, lv))
            p = ctx.mul_int(p, 2)
            t1 = retarget(T[1], p.level, p.scale)
            p = ctx.sub_ct(p, t1)
        T[j] = p

    def lincomb(terms, c0, level, scale):
        """sum_(coef, T) round(coef scale q_{l+1} / s_T) T + round(c0 scale q_{l+1}), rescaled to (l, scale)."""
        acc = None
        for coef, x in terms:
            y = ctx.drop_to(x, level + 1)
            K = int(round(coef * scale * ctx.q[level + 1] / y.scale))
            y = ctx.mul_int(y, K)
            y.scale = scale * ctx.q[level + 1]
            acc = y if acc is None else ctx.add_ct(acc, y)
        acc = ctx.add_const_int(acc, int(round(c0 * scale * ctx.q[level + 1])))
        out = ctx.rescale(acc)
        out.scale = scale
        return out

    def need(cc):
        return cheb_ps_need(cc, k, giants)

    def ev(cc, level, scale):
        d = len(cc) - 1
        if d < k:
            return lincomb([(cc[i], T[i]) for i in range(1, d + 1)], cc[0], level, scale)
        G = max(g for g in giants if g <= d)
        q, r = cheb_divide(cc, G)
        if len(q) == 1 and G - 1 < k:          # q_0 T_G + r in one combination (r a leaf)
            return lincomb([(cc_i, T[i]) for i, cc_i in enumerate(r) if i >= 1] + [(q[0], T[G])], r[0],
                           level, scale)
        if len(q) == 1:                        # scalar q_0 T_G plus the recursion on r, same (l, s)
            return ctx.add_ct(ev(r, level, scale), lincomb([(q[0], T[G])], 0.0, level, scale))
        TG = ctx.drop_to(T[G], level + 1)
        Q = ev(q, level + 1, scale * ctx.q[level + 1] / TG.scale)
        prod = ctx.mul_relin(ctx.drop_to(Q, level + 1), TG)
        return ctx.add_ct(prod, ev(r, level, prod.scale))

    out_level = ct.level - need(list(c))
    assert out_level >= 0, "not enough levels"
    return ev(list(c), out_level, target_scale)


def cheb_tree_he(ctx, ct, c, target_scale=None):
    """Homomorphic sum c_k T_k(ct) with the binary-tree T_k and exact-scale constants.

    T_1 = ct.  Products run through mul_relin (tensor, relinearise, rescale).  Every
    subtraction of T_1 and the final linear combination re-target the scale exactly: a
    ciphertext at scale s is multiplied by the integer round(c * S_target * q_l / s) at
    level l and rescaled, so its scale becomes S_target (value error ~ 2^-40 relative).
    The constant term is added as round(c_0 * scale) on coefficient 0.
    """
    target_scale = ctx.pr.scale if target_scale is None else target_scale
    deg = len(c) - 1
    T = {1: ct}

    def retarget(x, level, scale_t):
        """x (any scale) -> level `level`, scale exactly scale_t, costs one level."""
        y = ctx.drop_to(x, level + 1)
        K = int(round(scale_t * ctx.q[level + 1] / y.scale))
        y = ctx.mul_int(y, K)
        y = ctx.rescale(y)
        y.scale = scale_t
        return y

    for k in range(2, deg + 1):
        h = k // 2
        if k % 2 == 0:
            p = ctx.mul_relin(T[h], T[h])
            p = ctx.mul_int(p, 2)
            p = ctx.add_const_int(p, -int(round(p.scale)))
        else:
            a, b = T[h], T[h + 1]
            lv = min(a.level, b.level)
            p = ctx.mul_relin(ctx.drop_to(a, lv), ctx.drop_to(b, lv))
            p = ctx.mul_int(p, 2)
            t1 = retarget(T[1], p.level, p.scale)
            p = ctx.sub_ct(p, t1)
        T[k] = p
    lmin = min(x.level for x in T.values())
    acc = None
    for k in range(1, deg + 1):
        x = ctx.drop_to(T[k], lmin)
        K = int(round(c[k] * target_scale * ctx.q[lmin] / x.scale))
        y = ctx.mul_int(x, K)
        y.scale = target_scale * ctx.q[lmin]
        acc = y if acc is None else ctx.add_ct(acc, y)
    acc = ctx.add_const_int(acc, int(round(c[0] * target_scale * ctx.q[lmin])))
    out = ctx.rescale(acc)
    out.scale = target_scale
    return out
