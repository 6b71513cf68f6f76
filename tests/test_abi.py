"""The C-ABI library builds, loads without a GPU and exports every declared entry point;
its host-only logic (prime chain, initial layouts) agrees with the oracle.  No GPU compute."""
import os
import re

import numpy as np
import pytest

from oracle import layers as Ly
from oracle.params import TOY, C20, S33, Params, gen_primes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hegpu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(he_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2306_09189_gb300 import hegpu as H
    lib = H.load()
    declared = _declared()
    assert len(declared) > 50
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(H.exported_symbols())
    assert b"sm_103a" in lib.he_version()


@pytest.mark.parametrize("pr", [TOY, C20, S33, Params(10, 6, 2, 3, 50, 40, 50, 1.0, 0)])
def test_prime_chain_matches_oracle(pr):
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import params_of
    q, p = H.he_params_primes(params_of(pr))
    oq, op = gen_primes(pr)
    assert [int(x) for x in q] == oq and [int(x) for x in p] == op


@pytest.mark.parametrize("c,m,N", [(4, 32, 4096), (16, 32, 32768), (64, 56, 32768),
                                    (3, 224, 32768), (64, 112, 32768), (3, 30, 512), (5, 8, 256)])
def test_initial_layout_matches_oracle(c, m, N):
    from paper_2306_09189_gb300 import hegpu as H
    lay = H.he_layout_image(c, m, N)
    ref = Ly.image_layout(c, m, N)
    chan, row0 = lay.tables()
    assert (lay.M, lay.B, lay.n_shards, lay.nb) == (ref.M, ref.B, ref.n_shards, ref.nb)
    assert np.array_equal(chan, ref.chan) and np.array_equal(row0, ref.row0)


def test_no_gpu_means_loud_failure():
    import torch
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import params_of
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(H.HEError):
        H.he_ctx_create(params_of(TOY))


def test_bad_parameters_are_rejected_on_host():
    from paper_2306_09189_gb300 import hegpu as H
    from tests._hegpu_util import params_of
    with pytest.raises(H.HEError):
        H.he_params_primes(params_of(Params(3, 4, 1, 1, 40, 40, 50, 1.0, 0)))   # log_n < 9
    with pytest.raises(H.HEError):
        H.he_params_primes(params_of(Params(12, 4, 1, 1, 70, 40, 50, 1.0, 0)))  # 70-bit prime
    with pytest.raises(H.HEError):
        H.he_layout_image(3, 30, 500)                                           # N not 2^k


def test_header_constants_match_the_binding():
    # every integer constant the header defines (error codes, modes, options, key-stream forms,
    # activation ids) exists in the Python binding with the same value
    from paper_2306_09189_gb300 import hegpu as H
    src = open(os.path.join(ROOT, "include", "hegpu.h")).read()
    defs = dict(re.findall(r"^#define\s+(HE_[A-Z0-9_]+)\s+(-?\d+)\b", src, flags=re.M))
    assert len(defs) >= 15 and "HE_KEY_STREAM_SPLITM" in defs
    for name, value in defs.items():
        assert getattr(H, name) == int(value), name


def test_allocator_hook_arguments_are_checked():
    """he_set_allocator (host only): both functions or neither."""
    from paper_2306_09189_gb300 import hegpu as H
    L = H.load()
    with pytest.raises(H.HEError) as e:
        H._check(L.he_set_allocator(H.HE_DEVICE_ALLOC_FN(lambda n, u: None), H.HE_DEVICE_FREE_FN(), None))
    assert e.value.code == H.HE_EINVAL
    assert H.he_live_allocations() == 0
    H.use_default_allocator()                     # nothing live: accepted
