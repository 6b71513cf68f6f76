"""Bootstrapping of RNS-CKKS ciphertexts, for the oracle (TEST INFRASTRUCTURE ONLY).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may use this.

The paper runs its networks' bootstrapping through OpenFHE (Sec. 5, the Bootstrap rows of the
latency tables; Appendix "Precision and Bootstrapping Noise") and does not define it.  The
oracle fixes the standard CKKS construction, one convention per step (readings in the design
notes):

  ModRaise     a level-0 ciphertext read over Q_L (centred lift of its residues mod q_0): it
               decrypts to t = m + q_0 I with |I| <= K.  Its scale is set to q_0 K, so the
               slots hold the encoding of t / (q_0 K).
  CoeffToSlot  the inverse of the encoding map.  With w_j = t_j + i t_{j+N} (j < N) the slots of
               t are z = U w, U_ij = zeta^{g_i j} (zeta = exp(i pi / n), g_i = 5^i mod 2n).
               U = S_{N/2} ... S_2 S_1 BR: BR the bit-reversal permutation and S_h the radix-2
               butterfly stage of half-length h (the recursion z_i = E_i + zeta_M^{5^i} O_i,
               z_{i+M/2} = E_i - zeta_M^{5^i} O_i of the even/odd coefficient split, with
               zeta_M = exp(2 pi i / 4M) for sub-problems of size M).  CoeffToSlot applies
               2 S_h^{-1} for h = N/2 .. 1 (the 1/2 of each inverse stage goes into the scale),
               the stages merged into levels; each merged level is a matrix with few non-zero
               diagonals, evaluated baby-step giant-step with one ModDown per partial sum and
               per output (the raised-basis stage of the convolution), then one rescale.  The
               output slots hold BR(w) / (q_0 K): the bit reversal is never applied, since
               the next step is slot-wise and SlotToCoeff expects that order.
  retarget     multiply by the integer k = round((Delta / 2) q_l / s) and rescale: the scale
               becomes s k / q_l (exact bookkeeping, about Delta / 2), the integers shrink to
               that size.  The split below doubles it, so EvalMod's input sits at about Delta,
               near the primes: the Chebyshev products' scales then stay near the primes too
               (a product's scale is s_a s_b / q_l), which the exact-scale constants need.
  split        with c = conj(ct) (key switch for X -> X^{2n-1}): re = ct + c, im = (ct - c) X^{3n/2}
               (X^{n/2} multiplies every slot by i), both at twice the scale: the slots of re
               hold t_j / (q_0 K), those of im t_{j+N} / (q_0 K), both real.
  EvalMod      x = K u = t / q_0; cos(2 pi (x - 1/4) / 2^r) as a Chebyshev interpolant in u on
               [-1, 1] (Paterson-Stockmeyer), then r double angles y <- 2 y^2 - 1, giving
               sin(2 pi x) = sin(2 pi m / q_0) ~ 2 pi m / q_0.
  SlotToCoeff  re + i im, scale times 2 pi Delta_in / q_0 (the slots then hold m / Delta_in,
               m's coefficients in bit-reversed order); times the integer round(Delta / s)
               (no level) so the scale is about Delta again; then the forward stages
               S_1 .. S_{N/2} merged into levels as above: the slots hold the message again.

Levels: CoeffToSlot and SlotToCoeff one per merged level, retarget one, EvalMod the
Paterson-Stockmeyer depth plus r.
"""
from dataclasses import dataclass, field
import math

import numpy as np

from .encode import encode_complex
from .layers import raised_stage, cheb_nodes_coeffs, cheb_ps_he, cheb_ps_params, cheb_ps_need


# ============================================================================ the special DFT
def bit_reverse(N):
    """Index permutation of the bit reversal on log2 N bits."""
    b = N.bit_length() - 1
    return np.array([int(format(i, "0%db" % b)[::-1], 2) if b else 0 for i in range(N)], dtype=np.int64)


def dft_matrix(n):
    """U_ij = zeta^{g_i j}, i, j < N = n/2: slots = U (m_lo + i m_hi) / S (dense, small n only)."""
    N = n // 2
    g = [pow(5, i, 2 * n) for i in range(N)]
    j = np.arange(N)
    return np.exp(1j * np.pi * np.outer(np.array(g, dtype=np.float64), j) / n)


def twiddle(j, h):
    """zeta_M^{5^j mod 4M} for the sub-problem of size M = 2h: exp(2 pi i (5^j mod 8h) / 8h)."""
    return np.exp(2j * np.pi * (pow(5, j, 8 * h)) / (8 * h))


def stage_diagonals(N, h, inverse):
    """Non-zero diagonals {offset mod N: vector over rows} of the butterfly stage S_h
    (inverse: of 2 S_h^{-1}).  Row x sits at p = x mod 2h of its block; j = p mod h.
      S_h:       p < h: out = v[x] + tw v[x+h];        p >= h: out = v[x-h] - tw v[x]
      2 S_h^-1:  p < h: out = v[x] + v[x+h];           p >= h: out = conj(tw) (v[x-h] - v[x])"""
    x = np.arange(N)
    p = x % (2 * h)
    lower = p < h
    tw = np.array([twiddle(int(jj), h) for jj in (p % h)])
    d0 = np.where(lower, 1.0 + 0j, -(np.conj(tw) if inverse else tw))
    dp = np.where(lower, 1.0 + 0j if inverse else tw, 0j)
    dm = np.where(lower, 0j, np.conj(tw) if inverse else 1.0 + 0j)
    out = {}
    for off, v in ((0, d0), (h % N, dp), ((-h) % N, dm)):
        out[off] = out.get(off, 0) + v          # h = N/2: +h and -h are one diagonal
    return out


def diag_product(A, B, N):
    """Diagonals of the product A B (B applied first):
    diag_d(AB)[x] = sum_e diag_e(A)[x] diag_{d-e}(B)[x+e]."""
    out = {}
    x = np.arange(N)
    for e, a in A.items():
        for f, b in B.items():
            d = (e + f) % N
            out[d] = out.get(d, 0) + a * b[(x + e) % N]
    return {d: v for d, v in out.items() if np.any(v != 0)}


def apply_diagonals(D, v):
    """(M v)_x = sum_d diag_d[x] v[x+d]  (slot simulator; np.roll(v, -d)[x] = v[x+d])."""
    out = np.zeros(len(v), dtype=np.complex128)
    for d, dv in D.items():
        out += dv * np.roll(v, -d)
    return out


def level_groups(logN, levels):
    """Stage counts of the merged levels, larger first: logN stages into `levels` groups."""
    base, extra = divmod(logN, levels)
    return [base + (1 if i < extra else 0) for i in range(levels)]


def cts_levels(N, levels):
    """CoeffToSlot: 2 S_h^{-1} for h = N/2 down to 1, merged into levels (stage lists, diagonals)."""
    logN = N.bit_length() - 1
    hs = [1 << e for e in range(logN - 1, -1, -1)]
    out, i = [], 0
    for m in level_groups(logN, levels):
        grp = hs[i:i + m]
        i += m
        D = stage_diagonals(N, grp[0], True)
        for h in grp[1:]:
            D = diag_product(stage_diagonals(N, h, True), D, N)
        out.append((grp, D))
    return out


def stc_levels(N, levels):
    """SlotToCoeff: S_h for h = 1 up to N/2, merged into levels (the CoeffToSlot grouping reversed)."""
    logN = N.bit_length() - 1
    hs = [1 << e for e in range(logN)]
    out, i = [], 0
    for m in reversed(level_groups(logN, levels)):
        grp = hs[i:i + m]
        i += m
        D = stage_diagonals(N, grp[0], False)
        for h in grp[1:]:
            D = diag_product(stage_diagonals(N, h, False), D, N)
        out.append((grp, D))
    return out


# ============================================================================ baby-step giant-step
@dataclass
class BsgsLevel:
    """One merged level, regrouped: offset d = (i b1 + j) u (u = the level's smallest stage
    half-length, k = i b1 + j the offset in units, taken in [-N/2u, N/2u), j = k mod b1):

        M v = sum_i rot_{i b1 u}( sum_j rot_{-i b1 u}(diag_d) (.) rot_{j u}(v) )

    b1 = the smallest power of two >= (k_max - k_min + 1) / 2, so there are two giant steps:
    each giant partial sum costs a ModUp and a ModDown (a few hundred limb NTTs at the top
    level), a baby rotation only a key read in the raised-basis stage."""
    N: int
    stages: list
    gain: float                                   # scale factor of the level (2^stages for CoeffToSlot)
    unit: int = 1
    b1: int = 1
    giants: list = field(default_factory=list)    # giant indices i (ascending)
    baby: dict = field(default_factory=dict)      # i -> {j: rotated diagonal (complex [N])}

    def baby_amounts(self):
        return sorted({j * self.unit for d in self.baby.values() for j in d})

    def giant_amounts(self):
        return [(i * self.b1 * self.unit) % self.N for i in self.giants]

    def rotations(self):
        """Distinct non-zero rotation amounts (mod N) the level's key switches use."""
        s = {a % self.N for a in self.baby_amounts()} | set(self.giant_amounts())
        return sorted(a for a in s if a != 0)


def bsgs_level(N, stages, D, gain):
    u = min(stages)
    span = N // u
    ks = {}
    for d, v in D.items():
        assert d % u == 0
        k = d // u
        if 2 * k >= span:
            k -= span
        ks[k] = v
    kmin, kmax = min(ks), max(ks)
    b1 = 1
    while 2 * b1 < kmax - kmin + 1:
        b1 *= 2
    L = BsgsLevel(N, list(stages), gain, u, b1)
    for k, v in sorted(ks.items()):
        i, j = k // b1, k % b1
        L.baby.setdefault(i, {})[j] = np.roll(v, i * b1 * u)       # rot_{-i b1 u}(diag)
    L.giants = sorted(L.baby)
    return L


def bsgs_apply(L: BsgsLevel, v):
    """Slot simulator of the regrouped level (np.roll as the rotation)."""
    out = np.zeros(L.N, dtype=np.complex128)
    for i in L.giants:
        S = np.zeros(L.N, dtype=np.complex128)
        for j, P in L.baby[i].items():
            S += P * np.roll(v, -j * L.unit)
        out += np.roll(S, -i * L.b1 * L.unit)
    return out


# ============================================================================ plan
@dataclass
class BootConfig:
    K: int = 16                 # |I| bound: EvalMod's domain is x in [-K, K]
    r: int = 2                  # double-angle steps
    deg: int = 59               # Chebyshev degree of the cosine
    levels_cts: int = 3
    levels_stc: int = 3


class BootPlan:
    """Merged levels, their baby-step giant-step form, the EvalMod coefficients and the levels
    every step runs at, for one context (top level L)."""

    def __init__(self, ctx, cfg: BootConfig = BootConfig()):
        self.cfg = cfg
        N, n = ctx.N, ctx.n
        self.cts = [bsgs_level(N, st, D, float(2 ** len(st))) for st, D in cts_levels(N, cfg.levels_cts)]
        self.stc = [bsgs_level(N, st, D, 1.0) for st, D in stc_levels(N, cfg.levels_stc)]
        K, r = cfg.K, cfg.r
        self.coeffs = cheb_nodes_coeffs(lambda u: math.cos(2 * math.pi * (K * u - 0.25) / 2 ** r),
                                        cfg.deg, -1.0, 1.0)
        k, giants = cheb_ps_params(cfg.deg)
        self.ps_depth = cheb_ps_need(list(self.coeffs), k, giants)
        L = ctx.L
        self.cts_level = [L - i for i in range(cfg.levels_cts)]
        self.retarget_level = L - cfg.levels_cts
        self.evalmod_level = self.retarget_level - 1
        top_stc = self.evalmod_level - self.ps_depth - r
        self.stc_level = [top_stc - i for i in range(cfg.levels_stc)]
        self.out_level = top_stc - cfg.levels_stc
        assert self.out_level >= 0, "not enough levels for the bootstrap"
        self._pts = {}

    def rotations(self):
        return sorted({a for lv in self.cts + self.stc for a in lv.rotations()})

    def plaintexts(self, ctx, which, idx):
        """{(i, j): int64 plaintext} of level idx of 'cts' or 'stc', at scale q_level."""
        key = (which, idx)
        if key not in self._pts:
            lv = (self.cts if which == "cts" else self.stc)[idx]
            level = (self.cts_level if which == "cts" else self.stc_level)[idx]
            S = float(ctx.q[level])
            self._pts[key] = {(i, j): encode_complex(P, ctx.n, S)
                              for i in lv.giants for j, P in sorted(lv.baby[i].items())}
        return self._pts[key]


# ============================================================================ homomorphic steps
def lintrans_he(ctx, ct, lv: BsgsLevel, pts):
    """One merged level: baby stage (input rotated by j u, one ModDown per partial sum S_i),
    giant stage (S_i rotated by i b1 u, plaintext 1, one ModDown), rescale, scale times gain.
    pts: {(i, j): int64} at scale q_level."""
    level = ct.level
    S_pt = float(ctx.q[level])
    baby = {gi: [(0, j * lv.unit, pts[(i, j)]) for j in sorted(lv.baby[i])] for gi, i in enumerate(lv.giants)}
    S = raised_stage(ctx, [ct], baby)
    for x in S:
        x.scale = ct.scale * S_pt
    giant = {0: [(gi, i * lv.b1 * lv.unit, None) for gi, i in enumerate(lv.giants)]}
    acc = raised_stage(ctx, S, giant)[0]
    acc.scale = ct.scale * S_pt
    out = ctx.rescale(acc)
    out.scale = out.scale * lv.gain
    return out


def retarget_exact(ctx, ct, scale_t):
    """ct times the integer k = round(scale_t q_l / s), rescaled; scale s k / q_l."""
    k = int(round(scale_t * float(ctx.q[ct.level]) / ct.scale))
    y = ctx.mul_int(ct, k)
    y.scale = ct.scale * k
    return ctx.rescale(y)


def split_re_im(ctx, ct):
    """(re, im) with real slots Re(u), Im(u) of ct's slots u."""
    c = ctx.conjugate(ct)
    re = ctx.add_ct(ct, c)
    re.scale = ct.scale * 2.0
    im = ctx.mul_monomial(ctx.sub_ct(ct, c), 3 * ctx.n // 2)
    im.scale = ct.scale * 2.0
    return re, im


def evalmod_he(ctx, ct, plan: BootPlan):
    """cos(2 pi (K u - 1/4) / 2^r) by Paterson-Stockmeyer, then r double angles 2 y^2 - 1."""
    y = cheb_ps_he(ctx, ct, list(plan.coeffs), ctx.pr.scale)
    for _ in range(plan.cfg.r):
        y = ctx.mul_relin(y, y)
        y = ctx.mul_int(y, 2)
        y = ctx.add_const_int(y, -int(round(y.scale)))
    return y


def gen_boot_keys(ctx, plan: BootPlan):
    for a in plan.rotations():
        ctx.gen_rotation_key(a)
    ctx.gen_conj_key()
    ctx.gen_relin_key()


def to_level0(ctx, ct, ratio_bits=10):
    """A ciphertext above level 0 brought to level 0 at scale q_0 / 2^ratio_bits: dropped to
    level 1, multiplied by the integer round((q_0 / 2^ratio_bits) q_1 / s), rescaled (the scale
    bookkeeping exact: s k / q_1).  q_0 / scale = 2^ratio_bits is the small-angle margin the sine
    step of EvalMod reads the message with."""
    if ct.level == 0:
        return ct
    y = ctx.drop_to(ct, 1) if ct.level > 1 else ct
    return retarget_exact(ctx, y, float(ctx.q[0]) / 2.0 ** ratio_bits)


def bootstrap(ctx, ct, plan: BootPlan, trace=None):
    """The whole bootstrap; returns a ciphertext at plan.out_level with the same slot values.
    An input above level 0 first goes through to_level0.  trace (a dict) receives the
    intermediate ciphertexts by step name."""
    ct = to_level0(ctx, ct)
    K = plan.cfg.K
    q0 = float(ctx.q[0])
    in_scale = ct.scale
    x = ctx.modraise(ct)
    x.scale = q0 * K
    if trace is not None:
        trace["modraise"] = x
    for i, lv in enumerate(plan.cts):
        x = lintrans_he(ctx, x, lv, plan.plaintexts(ctx, "cts", i))
        if trace is not None:
            trace["cts%d" % i] = x
    x = retarget_exact(ctx, x, ctx.pr.scale / 2.0)
    if trace is not None:
        trace["retarget"] = x
    re, im = split_re_im(ctx, x)
    if trace is not None:
        trace["re"], trace["im"] = re, im
    re = evalmod_he(ctx, re, plan)
    im = evalmod_he(ctx, im, plan)
    if trace is not None:
        trace["evalmod_re"], trace["evalmod_im"] = re, im
    w = ctx.add_ct(re, ctx.mul_monomial(im, ctx.n // 2))
    w.scale = w.scale * (2.0 * math.pi * in_scale / q0)
    # back to about Delta without a level: times the integer k = round(Delta / s) (exact scale
    # s k), so the output can go straight into products whose scales must stay near the primes
    k = int(round(ctx.pr.scale / w.scale))
    if k > 1:
        w = ctx.mul_int(w, k)
        w.scale = w.scale * k
    if trace is not None:
        trace["combine"] = w
    for i, lv in enumerate(plan.stc):
        w = lintrans_he(ctx, w, lv, plan.plaintexts(ctx, "stc", i))
        if trace is not None:
            trace["stc%d" % i] = w
    return w


def meta_bootstrap(ctx, ct, plan: BootPlan, kb=10):
    """Bootstrapping with its own error removed once more (the paper's Appendix on precision
    and bootstrapping noise applies MetaBTS for about twice the bits, one level and a second
    bootstrap more): c1 = bootstrap(ct); the difference of c1 (brought back to level 0 at ct's
    scale) and ct encrypts the bootstrapping error E; it is bootstrapped at 2^kb times its size
    and subtracted: c1 - E, at one level below the bootstrap's output.

      y  = c1 dropped to level 1, times round(s0 q_1 / s), rescaled; read at scale s0 (exact to
           1/(2k) relative, k ~ 2^40)
      e  = (y - ct) 2^kb                 level 0, value E 2^kb
      f  = bootstrap(e), scale times 2^kb (value E plus its own error / 2^kb)
      g  = f times round(s1 q_lv / s_f), rescaled, read at c1's scale s1
      out = c1 dropped to lv - 1, minus g"""
    ct = to_level0(ctx, ct)
    s0 = ct.scale
    c1 = bootstrap(ctx, ct, plan)
    y = ctx.drop_to(c1, 1)
    k = int(round(s0 * float(ctx.q[1]) / y.scale))
    y = ctx.mul_int(y, k)
    y.scale = y.scale * k
    y = ctx.rescale(y)
    y.scale = s0
    e = ctx.mul_int(ctx.sub_ct(y, ct), 2 ** kb)
    f = bootstrap(ctx, e, plan)
    f.scale = f.scale * 2.0 ** kb
    lv = f.level
    kf = int(round(c1.scale * float(ctx.q[lv]) / f.scale))
    g = ctx.mul_int(f, kf)
    g.scale = f.scale * kf
    g = ctx.rescale(g)
    g.scale = c1.scale
    return ctx.sub_ct(ctx.drop_to(c1, lv - 1), g)
