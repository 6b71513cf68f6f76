"""Helpers shared by the GPU tests: C-ABI contexts keyed like the oracle's, ct transfer."""
import numpy as np

from paper_2306_09189_gb300 import hegpu as H


def params_of(pr):
    return H.he_params(pr.log_n, pr.n_q, pr.n_p, pr.dnum, pr.q0_bits, pr.q_bits, pr.p_bits,
                       pr.scale, pr.seed, pr.secret_hw)


class GpuCtx:
    """A device context built from the same parameters (and seed) as an oracle context."""

    def __init__(self, pr):
        self.pr = pr
        self.h = H.he_ctx_create(params_of(pr))
        self.info = H.he_ctx_info(self.h)
        self.n = self.info["n"]
        self.N = self.info["slots"]
        self._cts = []

    def ct(self, level):
        c = H.he_ct_alloc(self.h, level)
        self._cts.append(c)
        return c

    def upload(self, oct_):
        """oracle Ciphertext -> device ciphertext"""
        c = self.ct(oct_.level)
        H.he_ct_import_coeffs(c, oct_.c, oct_.level, oct_.scale)
        return c

    def download(self, c):
        return H.he_ct_export_coeffs(self.h, c, self.n)

    def close(self):
        for c in self._cts:
            H.he_ct_free(c)
        self._cts = []
        H.he_ctx_destroy(self.h)


def assert_ct_equal(gpu_coeffs, oracle_ct):
    assert gpu_coeffs.shape == oracle_ct.c.shape, (gpu_coeffs.shape, oracle_ct.c.shape)
    bad = np.argwhere(gpu_coeffs != oracle_ct.c)
    assert bad.size == 0, "%d words differ, first at %s" % (len(bad), bad[:3].tolist())
