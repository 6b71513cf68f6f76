"""Build and load the oracle's C core (TEST INFRASTRUCTURE ONLY).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may import the
``oracle`` package.  The product path never touches it.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ckks_ref.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libckks_ref.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile ckks_ref.c with gcc (OpenMP when available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    base = ["gcc", "-O2", "-shared", "-fPIC", "-ffp-contract=off", _SRC, "-o", tmp]
    try:
        subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base)
    os.replace(tmp, _SO)
    return _SO


U64P = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
I64P = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
I32P = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
u64 = ctypes.c_uint64
cint = ctypes.c_int


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            L = _lib
            L.orc_powmod.argtypes = [u64, u64, u64]
            L.orc_powmod.restype = u64
            L.orc_mulmod.argtypes = [u64, u64, u64]
            L.orc_mulmod.restype = u64
            L.orc_splitmix64_mix.argtypes = [u64]
            L.orc_splitmix64_mix.restype = u64
            L.orc_rng.argtypes = [u64, u64, u64]
            L.orc_rng.restype = u64
            L.orc_sample_ternary.argtypes = [u64, u64, cint, I64P]
            L.orc_sample_cbd.argtypes = [u64, u64, cint, I64P]
            L.orc_sample_uniform.argtypes = [u64, u64, cint, cint, I32P, U64P, U64P]
            L.orc_ntt.argtypes = [U64P, cint, cint, U64P, U64P]
            L.orc_intt.argtypes = [U64P, cint, cint, U64P, U64P]
            L.orc_mul.argtypes = [U64P, U64P, U64P, cint, cint, U64P]
            L.orc_mac.argtypes = [U64P, U64P, U64P, cint, cint, U64P]
            L.orc_mul_scalar.argtypes = [U64P, U64P, U64P, cint, cint, U64P]
            L.orc_fbc.argtypes = [U64P, U64P, cint, U64P, cint, U64P, cint]
            L.orc_fbc_centred.argtypes = [U64P, U64P, cint, U64P, cint, U64P, cint]
            L.orc_automorph_coeff.argtypes = [U64P, U64P, cint, cint, U64P, u64]
            L.orc_automorph_eval.argtypes = [U64P, U64P, cint, cint, u64]
            for f in ("orc_sample_ternary", "orc_sample_cbd", "orc_sample_uniform", "orc_ntt",
                      "orc_intt", "orc_mul", "orc_mac", "orc_mul_scalar", "orc_fbc", "orc_fbc_centred",
                      "orc_automorph_coeff", "orc_automorph_eval"):
                getattr(L, f).restype = None
    return _lib
