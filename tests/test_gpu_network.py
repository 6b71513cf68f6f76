"""A whole encrypted ResNet-20-shaped network on the GPU (the paper's smallest multiplexed ResNet,
Sec. 5): 19 convolutions with folded BatchNorm, 19 GELUs, 9 residual connections, two stride-2
stages, the pool-linear head, and a bootstrap wherever the levels run out.  The decrypted logits
must match the FP64 network with the same polynomial activation."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_resnet20_logits_match_the_fp64_network():
    import workloads
    from paper_2306_09189_gb300 import host
    from paper_2306_09189_gb300.network import EncryptedResNet
    net = workloads.resnet20(0)
    cheb = host.chebyshev_coeffs("gelu", workloads.GELU_DEGREE, -workloads.GELU_BOUND, workloads.GELU_BOUND)
    want = workloads.resnet20_forward(net, cheb)
    r = EncryptedResNet(host.bootstrap_params(0), net, cheb)
    try:
        got = r.infer(net["x"])
        err = np.max(np.abs(got - want))
        assert err < 2.0 ** -7 * (np.max(want) - np.min(want)), (err, want, got)
        assert r.counts.get("bootstrap", 0) >= 9          # the chain alone holds a few layers
        # a second image through the same plans gives the same logits as a fresh run would
        got2 = r.infer(net["x"], nonce0=101)
        assert np.max(np.abs(got2 - want)) < 2.0 ** -7 * (np.max(want) - np.min(want))
    finally:
        r.close()
