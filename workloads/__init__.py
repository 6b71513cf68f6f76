"""Seeded synthetic workloads shaped like the paper's CIFAR- and ImageNet-sized layers.

This module only draws inputs (images, weights, folded BatchNorm affines, request arrival
times).  It holds none of the homomorphic method's arithmetic, so both the CUDA path and the
CPU oracle can take their inputs from it.  The paper evaluates on CIFAR-10/100 (32x32x3) and
ImageNet-1k (224/128/256 pixels) with trained ResNets (Sec. 5.1-5.2); neither datasets nor
weights exist here, so these seeded draws stand in for them with the same shapes and value
ranges: pixels uniform in [0, 1], PyTorch's default conv initialisation, BatchNorm statistics
taken from the plaintext convolution output (so pre-activations stay inside the polynomial's
interval, the role the paper's kurtosis regularisation plays, Appendix).
"""
from dataclasses import dataclass
import math

import numpy as np

GELU_BOUND = 8.0      # polynomial interval [-8, 8]; BN output is divided by it (folded)
GELU_DEGREE = 16


@dataclass
class ConvLayer:
    x: np.ndarray          # [c][m][m]
    W: np.ndarray          # [co][ci][k][k], BN and 1/GELU_BOUND folded in when bn=True
    bias: np.ndarray       # [co]
    stride: int
    pad: int
    name: str


def image(c, m, seed):
    return np.random.default_rng(seed).uniform(0.0, 1.0, (c, m, m))


def _plain_conv(x, W, pad):
    import torch
    return torch.nn.functional.conv2d(torch.tensor(x)[None], torch.tensor(W),
                                      padding=pad)[0].numpy()


def fold_bn(x, W, pad, bound=GELU_BOUND, eps=1e-5):
    """gamma = 1, beta = 0, mu/sigma^2 from the plaintext conv output; divide by `bound`."""
    y = _plain_conv(x, W, pad)
    mu = y.mean(axis=(1, 2))
    sd = np.sqrt(y.var(axis=(1, 2)) + eps)
    Wf = W / (sd[:, None, None, None] * bound)
    bf = -mu / (sd * bound)
    return Wf, bf


def toy_conv(seed=0):
    """4x32x32 image, 3x3 conv 4->4, weights U[-1,1], bias 0, stride 1, pad 1."""
    rng = np.random.default_rng(seed + 1)
    return ConvLayer(image(4, 32, seed), rng.uniform(-1, 1, (4, 4, 3, 3)), np.zeros(4), 1, 1,
                     "toy 4x32x32 conv3x3 4->4")


def cifar_conv_bn(seed=0, c=16, m=32):
    """16x32x32 image, 3x3 conv 16->16 (PyTorch default init), BN folded, /8 for the GELU."""
    while True:
        rng = np.random.default_rng(seed + 1)
        x = image(c, m, seed)
        bound = 1.0 / math.sqrt(c * 9)
        W = rng.uniform(-bound, bound, (c, c, 3, 3))
        Wf, bf = fold_bn(x, W, 1)
        pre = _plain_conv(x, Wf, 1) + bf[:, None, None]
        if np.abs(pre).max() <= 1.0:
            return ConvLayer(x, Wf, bf, 1, 1, "cifar %dx%dx%d conv3x3+BN" % (c, m, m))
        seed += 1000


def imagenet_stem(seed=0):
    """224x224x3 image, 7x7 conv 3->64, stride 2, pad 3, weights N(0, 0.05^2)."""
    rng = np.random.default_rng(seed + 1)
    return ConvLayer(image(3, 224, seed), rng.normal(0.0, 0.05, (64, 3, 7, 7)), np.zeros(64), 2,
                     3, "imagenet stem 3x224x224 conv7x7/2 3->64")


def resnet_block(seed=0, c=64, m=56):
    """Basic block on 64x56x56: conv3x3-BN-GELU-conv3x3 (+ residual); BN folded per conv."""
    x = image(c, m, seed)
    rng = np.random.default_rng(seed + 1)
    bound = 1.0 / math.sqrt(c * 9)
    W1 = rng.uniform(-bound, bound, (c, c, 3, 3))
    W2 = rng.uniform(-bound, bound, (c, c, 3, 3))
    W1f, b1f = fold_bn(x, W1, 1)
    return x, (W1f, b1f), (W2 / 8.0, np.zeros(c))


def resnet_head(seed=0, c=64, m=8, n_out=10):
    """ResNet tail: a c x m x m feature map (post-GELU range), global average pool and a linear
    layer to n_out logits with PyTorch's default init U[+-1/sqrt(c)]."""
    rng = np.random.default_rng(seed + 3)
    x = rng.uniform(-0.2, 1.0, (c, m, m))
    bound = 1.0 / math.sqrt(c)
    return x, rng.uniform(-bound, bound, (n_out, c)), rng.uniform(-bound, bound, n_out)


def poisson_arrivals(n, rate, seed=0):
    """Arrival times (seconds) of n requests at `rate` requests/second."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))


def request_sizes(n, seed=0, sizes=(32, 64, 224), mix=(0.6, 0.3, 0.1)):
    rng = np.random.default_rng(seed + 7)
    return [int(s) for s in rng.choice(sizes, size=n, p=mix)]


def serving_stack(seed=0, widths=(4, 16, 32, 64, 64), m=32, bound=GELU_BOUND, deg=GELU_DEGREE):
    """Weights of the 4 x [conv3x3 + folded BN, GELU, 2x2 avg-pool] serving stack.

    PyTorch default conv init; BatchNorm statistics of every layer taken from a seeded m x m
    image pushed through the plaintext stack (conv, BN, exact GELU, avg-pool) and divided by
    `bound`, so the pre-activations of uniform images stay inside [-1, 1].  Returns
    [(W, b)] per layer."""
    import torch
    rng = np.random.default_rng(seed + 11)
    x = image(widths[0], m, seed + 5)
    x[3:] = 0.0                                  # 3 colour channels padded to 4
    layers = []
    for li in range(len(widths) - 1):
        ci, co = widths[li], widths[li + 1]
        lim = 1.0 / math.sqrt(ci * 9)
        W = rng.uniform(-lim, lim, (co, ci, 3, 3))
        Wf, bf = fold_bn(x, W, 1, bound=bound)
        layers.append((Wf, bf))
        y = torch.tensor(_plain_conv(x, Wf, 1) + bf[:, None, None])
        y = torch.nn.functional.gelu(y * bound)
        x = torch.nn.functional.avg_pool2d(y[None], 2)[0].numpy()
    return layers


def _gelu(v):
    from math import erf, sqrt
    return v * 0.5 * (1.0 + np.vectorize(erf)(v / sqrt(2.0)))


def resnet20(seed=0, m=32, bound=GELU_BOUND):
    """ResNet-20-shaped CIFAR network (the paper's smallest multiplexed ResNet, Sec. 5): a 3x3
    stem 3->16, three stages of three basic blocks at 16, 32 and 64 channels (the first block of
    stages 2 and 3 with stride 2 and a 1x1 stride-2 shortcut convolution), GELU activations,
    global average pool and a linear layer to 10 logits.  PyTorch's default initialisation;
    every BatchNorm folded into the convolution before it, its statistics taken from a seeded
    image pushed through the plaintext network (exact GELU) and divided by `bound`, so every
    activation input lies in [-1, 1] (the polynomial's interval [-bound, bound] folded in; the
    shortcut adds x / bound).  Reseeds until that holds.  Returns a dict: x [3][m][m], stem
    (W, b), blocks [{stride, W1, b1, W2, b2, Ws, bs}] (Ws None for the identity shortcut),
    head (W [10][64], b [10])."""
    import torch
    F = torch.nn.functional

    def conv(x, W, stride, pad):
        return F.conv2d(torch.tensor(x)[None], torch.tensor(W), stride=stride, padding=pad)[0].numpy()

    def fold(x, W, stride, pad, eps=1e-5):
        y = conv(x, W, stride, pad)
        mu = y.mean(axis=(1, 2))
        sd = np.sqrt(y.var(axis=(1, 2)) + eps)
        return W / (sd[:, None, None, None] * bound), -mu / (sd * bound)

    while True:
        rng = np.random.default_rng(seed + 11)
        x = image(3, m, seed)
        ok = True

        def init(co, ci, k):
            b = 1.0 / math.sqrt(ci * k * k)
            return rng.uniform(-b, b, (co, ci, k, k))

        W, b = fold(x, init(16, 3, 3), 1, 1)
        t = conv(x, W, 1, 1) + b[:, None, None]
        ok &= np.abs(t).max() <= 1.0
        a = _gelu(bound * t)
        stem = (W, b)
        blocks = []
        c = 16
        for stage, co in enumerate((16, 32, 64)):
            for i in range(3):
                stride = 2 if (stage > 0 and i == 0) else 1
                W1, b1 = fold(a, init(co, c, 3), stride, 1)
                h = _gelu(bound * (conv(a, W1, stride, 1) + b1[:, None, None]))
                W2, b2 = fold(h, init(co, co, 3), 1, 1)
                y = conv(h, W2, 1, 1) + b2[:, None, None]
                if stride == 2 or co != c:
                    Ws, bs = fold(a, init(co, c, 1), stride, 0)
                    sc = conv(a, Ws, stride, 0) + bs[:, None, None]
                else:
                    Ws, bs = None, None
                    sc = a / bound
                t = y + sc
                ok &= np.abs(t).max() <= 1.0
                a = _gelu(bound * t)
                blocks.append(dict(stride=stride, W1=W1, b1=b1, W2=W2, b2=b2, Ws=Ws, bs=bs))
                c = co
        hb = 1.0 / math.sqrt(64)
        head = (rng.uniform(-hb, hb, (10, 64)), rng.uniform(-hb, hb, 10))
        if ok:
            return dict(x=x, stem=stem, blocks=blocks, head=head)
        seed += 1000


def resnet20_forward(net, cheb, bound=GELU_BOUND):
    """The plaintext network in FP64 with the activation a given Chebyshev polynomial (the one
    the encrypted network evaluates): the reference its decrypted logits are checked against."""
    import torch
    F = torch.nn.functional
    act = lambda t: np.polynomial.chebyshev.chebval(t, cheb)

    def conv(x, W, b, stride, pad):
        return F.conv2d(torch.tensor(x)[None], torch.tensor(W), stride=stride, padding=pad)[0].numpy() + b[:, None, None]

    a = act(conv(net["x"], *net["stem"], 1, 1))
    for blk in net["blocks"]:
        s = blk["stride"]
        h = act(conv(a, blk["W1"], blk["b1"], s, 1))
        y = conv(h, blk["W2"], blk["b2"], 1, 1)
        sc = a / bound if blk["Ws"] is None else conv(a, blk["Ws"], blk["bs"], s, 0)
        a = act(y + sc)
    W, b = net["head"]
    return W @ a.mean(axis=(1, 2)) + b
