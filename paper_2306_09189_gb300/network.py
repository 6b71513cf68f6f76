"""A whole encrypted ResNet on one GPU: sharded convolutions, GELU, residual connections, the
pool-linear head, and bootstrapping wherever the levels run out (the paper's networks, Sec. 5;
bootstrapping restores the level, Sec. 2).

Control flow only: every ciphertext operation is a call into libhegpu (hegpu.py).  The runner
keeps one plan per layer, made the first time the layer runs (at the level and scale the input
arrives with, which are the same on every run) together with the layer's rotation keys.  The
convolutions take the baby-step giant-step form by default: after a stride-2 stage the channels
sit in the pooling's permuted block order, where the diagonal form needs over a thousand
distinct rotation keys for one 3x3 convolution (134 GB at this chain).

Level policy (chain with a bootstrap output level B): before a convolution followed by its
activation, a ciphertext with fewer than conv + GELU + 1 levels is bootstrapped; an activation
whose output lands at level 0 targets the scale q_0 / 2^10 the bootstrap reads level-0 inputs
at (otherwise Delta).  A residual operand is brought to the other operand's level and scale by
an exact retarget (times the integer round(s q_(l+1) / s_x), rescale), after a bootstrap if it
has no level to spare; the identity shortcut enters as x / bound by its scale alone.  The
stride-2 shortcut (a 1x1 convolution) lands in the pooling's block order and is moved to the main
path's image order by an identity 1x1 convolution before the add.
"""
import time

import numpy as np

from . import hegpu as H
from . import host

GELU_LEVELS = None      # levels the Paterson-Stockmeyer activation consumes (from the library)


def same_layout(a, b):
    """Two layouts with the same shards, blocks and channel / row tables."""
    if (a.c, a.m, a.M, a.N, a.B, a.n_shards, a.nb) != (b.c, b.m, b.M, b.N, b.B, b.n_shards, b.nb):
        return False
    k = a.n_shards * a.nb
    return list(a.chan[:k]) == list(b.chan[:k]) and list(a.row0[:k]) == list(b.row0[:k])


class EncryptedResNet:
    def __init__(self, pr, net, cheb, bound=8.0, key_stream=H.HE_KEY_STREAM_LDG, conv_form="bsgs"):
        global GELU_LEVELS
        self.pr = pr
        self.net = net
        self.cheb = np.asarray(cheb, dtype=np.float64)
        self.bound = bound
        self.ctx = H.he_ctx_create(pr)
        H.he_ctx_set_option(self.ctx, H.HE_OPT_KEY_STREAM, key_stream)
        info = H.he_ctx_info(self.ctx)
        self.N, self.q = info["slots"], [int(v) for v in info["q"]]
        self.boot = H.he_boot_create(self.ctx)
        H.he_keygen_rotations(self.ctx, H.he_boot_rotations(self.boot))
        H.he_keygen_conjugation(self.ctx)
        H.he_keygen_relin(self.ctx)
        self.boot_level = H.he_boot_info(self.boot)["out_level"]
        GELU_LEVELS = H.he_poly_ps_plan(len(self.cheb) - 1)[1]
        self.conv_form = conv_form
        self.plans = {}
        self.timing = {}
        self.counts = {}
        self._cts = []

    # ------------------------------------------------------------------ bookkeeping
    def _ct(self, level):
        c = H.he_ct_alloc(self.ctx, level)
        self._cts.append(c)
        return c

    def _tick(self, what, t0):
        import torch
        torch.cuda.synchronize()
        self.timing[what] = self.timing.get(what, 0.0) + time.perf_counter() - t0
        self.counts[what] = self.counts.get(what, 0) + 1

    def release(self):
        for c in self._cts:
            H.he_ct_free(c)
        self._cts = []

    def close(self):
        self.release()
        for p in self.plans.values():
            if p[0] == "conv":
                H.he_conv_destroy(p[1])
            else:
                H.he_linear_destroy(p[1])
        H.he_boot_destroy(self.boot)
        H.he_ctx_destroy(self.ctx)

    # ------------------------------------------------------------------ steps
    def bootstrap(self, cts):
        t0 = time.perf_counter()
        out = []
        for c in cts:
            o = self._ct(self.boot_level)
            H.he_bootstrap(self.ctx, self.boot, c, o)
            out.append(o)
        self._tick("bootstrap", t0)
        return out

    def conv(self, key, lay, cts, W, b, stride, pad):
        t0 = time.perf_counter()
        level, scale = H.he_ct_level(cts[0]), H.he_ct_scale(cts[0])
        pk = (key, level, scale)
        if pk not in self.plans:
            make = H.he_conv_create_bsgs if self.conv_form == "bsgs" else H.he_conv_create
            cv = make(self.ctx, lay, W, b, stride, pad, level, scale)
            H.he_keygen_rotations(self.ctx, H.he_conv_rotations(cv))
            self.plans[pk] = ("conv", cv)
        cv = self.plans[pk][1]
        lo = H.he_conv_out_layout(cv)
        outs = [self._ct(H.he_conv_out_level(cv)) for _ in range(lo.n_shards)]
        H.he_conv_run(self.ctx, cv, cts, outs, H.HE_FUSED)
        self._tick("conv", t0)
        return lo, outs

    def gelu(self, cts):
        t0 = time.perf_counter()
        lv = H.he_ct_level(cts[0]) - GELU_LEVELS
        target = self.q[0] / 1024.0 if lv == 0 else self.pr.scale
        H.he_poly_eval_ps_many(self.ctx, cts, self.cheb, [target] * len(cts))
        self._tick("gelu", t0)
        return cts

    def align(self, x, level, scale):
        """x (level > `level`) at exactly (level, scale): drop, times round(scale q / s), rescale."""
        y = self._ct(H.he_ct_level(x))
        H.he_ct_copy(y, x)
        H.he_ct_drop_level(y, level + 1)
        k = round(scale * self.q[level + 1] / H.he_ct_scale(y))
        H.he_mul_int(self.ctx, y, float(k))
        H.he_ct_set_scale(y, H.he_ct_scale(y) * k)
        H.he_rescale(self.ctx, y)
        H.he_ct_set_scale(y, scale)
        return y

    def ensure(self, cts, need):
        """Bootstrap when fewer than need + 1 levels remain."""
        if H.he_ct_level(cts[0]) < need + 1:
            return self.bootstrap(cts)
        return cts

    # ------------------------------------------------------------------ the network
    def run(self, x_cts, lay):
        net, B = self.net, self.bound
        a = self.ensure(x_cts, 1 + GELU_LEVELS)
        lay, a = self.conv("stem", lay, a, net["stem"][0], net["stem"][1], 1, 1)
        a = self.gelu(a)
        for i, blk in enumerate(net["blocks"]):
            s = blk["stride"]
            conv_levels = 1 if s == 1 else 3
            a = self.ensure(a, conv_levels + GELU_LEVELS)
            lay_h, h = self.conv(("c1", i), lay, a, blk["W1"], blk["b1"], s, 1)
            h = self.gelu(h)
            h = self.ensure(h, 1 + GELU_LEVELS)
            lay_y, y = self.conv(("c2", i), lay_h, h, blk["W2"], blk["b2"], 1, 1)
            ly, sy = H.he_ct_level(y[0]), H.he_ct_scale(y[0])
            t0 = time.perf_counter()
            if blk["Ws"] is None:
                sc = a
                for c in sc:                             # the shortcut enters as x / bound
                    H.he_ct_set_scale(c, H.he_ct_scale(c) * B)
            else:
                sc = a if H.he_ct_level(a[0]) >= 3 + 1 + 1 else self.bootstrap(a)
                lay_s, sc = self.conv(("sc", i), lay, sc, blk["Ws"], blk["bs"], s, 0)
                if not same_layout(lay_s, lay_y):
                    # the stride-2 outputs sit in the pooling's block order, the stride-1
                    # convolution's output in image order: an identity 1x1 convolution moves the
                    # shortcut to the main path's layout
                    co = blk["Ws"].shape[0]
                    eye = np.eye(co)[:, :, None, None]
                    _, sc = self.conv(("re", i), lay_s, sc, eye, np.zeros(co), 1, 0)
            if H.he_ct_level(sc[0]) < ly + 1:
                sc = self.bootstrap(sc)
            for yc, c in zip(y, sc):
                H.he_add(self.ctx, yc, self.align(c, ly, sy))
            self._tick("residual", t0)
            if blk["Ws"] is None:
                for c in a:
                    H.he_ct_set_scale(c, H.he_ct_scale(c) / B)
            a = self.gelu(y)
            lay = lay_y
        # pool-linear head (two levels)
        a = self.ensure(a, 2 - 1)
        t0 = time.perf_counter()
        level, scale = H.he_ct_level(a[0]), H.he_ct_scale(a[0])
        pk = ("head", level, scale)
        if pk not in self.plans:
            W, b = net["head"]
            lin = H.he_pool_linear_create(self.ctx, lay, W, b, level, scale)
            H.he_keygen_rotations(self.ctx, H.he_linear_rotations(lin))
            self.plans[pk] = ("linear", lin)
        lin = self.plans[pk][1]
        out = self._ct(H.he_linear_out_level(lin))
        H.he_linear_run(self.ctx, lin, a, out)
        self._tick("head", t0)
        return out

    def infer(self, img, level=None, nonce0=1):
        """Encrypt one image (channels x m x m) at the top level, run, decrypt the 10 logits."""
        level = H.he_ctx_info(self.ctx)["L"] if level is None else level
        lay = H.he_layout_image(img.shape[0], img.shape[1], self.N)
        x = host.encrypt_image(self.ctx, lay, img, level, self.pr.scale, nonce0=nonce0)
        self._cts += x
        out = self.run(x, lay)
        logits = H.he_decrypt(self.ctx, out, self.N)[:10]
        self.release()
        return logits
