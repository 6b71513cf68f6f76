"""Thin ctypes binding of the hegpu C ABI (include/hegpu.h): argument marshalling only.

Every homomorphic operation runs in the CUDA kernels of libhegpu.so.  There is no CPU
fallback: if the library cannot be built or loaded, or no GPU is present, the calls raise.
Function names match the C entry points; each raises HEError on a negative status.
"""
import ctypes
import os

import numpy as np

from . import build as _build

HE_OK, HE_EINVAL, HE_ELEVEL, HE_EKEY, HE_ENOMEM, HE_ETIMEOUT, HE_ECUDA, HE_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
HE_PLAIN, HE_BATCHED, HE_FUSED = 0, 1, 2
HE_RELIN_KEY = 0x7FFFFFFF
HE_MAX_BLOCKS = 32768
HE_OPT_KEY_STREAM = 1
HE_KEY_STREAM_LDG, HE_KEY_STREAM_TMA, HE_KEY_STREAM_AUTO, HE_KEY_STREAM_SPLIT, HE_KEY_STREAM_CP = 0, 1, 2, 3, 4
HE_KEY_STREAM_LDG1 = 5
HE_KEY_STREAM_PK = 6
HE_OPT_PDL = 2
HE_OPT_NTT = 3
HE_NTT_ONEPASS, HE_NTT_TWOPASS, HE_NTT_ONEPASS8, HE_NTT_TWOPASS_CORRECTED, HE_NTT_TWOPASS_SHUFFLE = 0, 1, 2, 3, 4
HE_KEY_STREAM_PK3 = 7
HE_KEY_STREAM_PKP = 8
HE_KEY_STREAM_SPLITM = 9
HE_KEY_STREAM_PK1 = 10
HE_KEY_STREAM_PKT = 11
HE_KEY_STREAM_PK3L = 12

c_int, c_double, c_size_t, c_u64, c_i32, c_vp = (ctypes.c_int, ctypes.c_double, ctypes.c_size_t,
                                                 ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p)
U64P = ctypes.POINTER(ctypes.c_uint64)
I64P = ctypes.POINTER(ctypes.c_int64)
I32P = ctypes.POINTER(ctypes.c_int32)
F64P = ctypes.POINTER(ctypes.c_double)


class HEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("hegpu error %d: %s" % (code, msg))
        self.code = code


class he_params(ctypes.Structure):
    _fields_ = [("log_n", c_int), ("n_q", c_int), ("n_p", c_int), ("dnum", c_int),
                ("q0_bits", c_int), ("q_bits", c_int), ("p_bits", c_int),
                ("scale", c_double), ("seed", c_u64), ("secret_hw", c_int)]


class he_boot_config(ctypes.Structure):
    _fields_ = [("K", c_int), ("double_angle", c_int), ("deg", c_int), ("levels_cts", c_int),
                ("levels_stc", c_int)]


class he_layout(ctypes.Structure):
    _fields_ = [("c", c_int), ("m", c_int), ("M", c_int), ("N", c_int), ("B", c_int),
                ("n_shards", c_int), ("nb", c_int),
                ("chan", ctypes.c_int32 * HE_MAX_BLOCKS), ("row0", ctypes.c_int32 * HE_MAX_BLOCKS)]

    def tables(self):
        k = self.n_shards * self.nb
        chan = np.ctypeslib.as_array(self.chan)[:k].reshape(self.n_shards, self.nb).copy()
        row0 = np.ctypeslib.as_array(self.row0)[:k].reshape(self.n_shards, self.nb).copy()
        return chan, row0


HE_DEVICE_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
HE_DEVICE_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_SIGS = {
    "he_set_allocator": (c_int, [HE_DEVICE_ALLOC_FN, HE_DEVICE_FREE_FN, c_vp]),
    "he_live_allocations": (ctypes.c_int64, []),
    "he_last_error": (ctypes.c_char_p, []),
    "he_version": (ctypes.c_char_p, []),
    "he_kernel_launches": (c_u64, []),
    "he_params_primes": (c_int, [ctypes.POINTER(he_params), U64P, U64P]),
    "he_layout_image": (c_int, [c_int, c_int, c_int, ctypes.POINTER(he_layout)]),
    "he_ctx_create": (c_int, [ctypes.POINTER(he_params), ctypes.POINTER(c_vp)]),
    "he_ctx_destroy": (None, [c_vp]),
    "he_ctx_fork": (c_int, [c_vp, ctypes.POINTER(c_vp)]),
    "he_ctx_check": (c_int, [c_vp, c_vp]),
    "he_ctx_set_option": (c_int, [c_vp, c_int, c_int]),
    "he_ctx_get_option": (c_int, [c_vp, c_int, ctypes.POINTER(c_int)]),
    "he_ctx_tuning_log": (c_size_t, [c_vp, ctypes.c_char_p, c_size_t]),
    "he_selftest_bounded_wait": (c_int, [c_vp, c_vp]),
    "he_graph_begin": (c_int, [c_vp, c_vp]),
    "he_graph_end": (c_int, [c_vp, c_vp, ctypes.POINTER(c_vp)]),
    "he_graph_launch": (c_int, [c_vp, c_vp]),
    "he_graph_kernels": (c_u64, [c_vp]),
    "he_graph_destroy": (None, [c_vp]),
    "he_ctx_info": (c_int, [c_vp] + [ctypes.POINTER(c_int)] * 6 + [U64P, U64P]),
    "he_keygen_rotations": (c_int, [c_vp, I32P, c_size_t]),
    "he_keygen_relin": (c_int, [c_vp]),
    "he_has_rotation_key": (c_int, [c_vp, c_i32]),
    "he_key_export": (c_int, [c_vp, c_i32, U64P]),
    "he_key_bytes": (c_size_t, [c_vp]),
    "he_ct_alloc": (c_int, [c_vp, c_int, ctypes.POINTER(c_vp)]),
    "he_ct_wrap": (c_int, [c_vp, c_vp, c_size_t, c_int, ctypes.POINTER(c_vp)]),
    "he_ct_free": (None, [c_vp]),
    "he_ct_level": (c_int, [c_vp]),
    "he_ct_scale": (c_double, [c_vp]),
    "he_ct_set_scale": (c_int, [c_vp, c_double]),
    "he_ct_limb_ptr": (c_vp, [c_vp, c_int, c_int]),
    "he_ct_copy": (c_int, [c_vp, c_vp, c_vp]),
    "he_ct_drop_level": (c_int, [c_vp, c_int]),
    "he_ct_import_coeffs": (c_int, [c_vp, U64P, c_int, c_double, c_vp]),
    "he_ct_export_coeffs": (c_int, [c_vp, U64P, c_vp]),
    "he_encrypt_coeffs": (c_int, [c_vp, I64P, c_int, c_double, c_u64, c_vp, c_vp]),
    "he_encrypt": (c_int, [c_vp, F64P, c_size_t, c_int, c_double, c_u64, c_vp, c_vp]),
    "he_decrypt": (c_int, [c_vp, c_vp, F64P, c_size_t, c_vp]),
    "he_pt_import_coeffs": (c_int, [c_vp, I64P, c_int, c_double, ctypes.POINTER(c_vp)]),
    "he_pt_encode": (c_int, [c_vp, F64P, c_size_t, c_int, c_double, ctypes.POINTER(c_vp)]),
    "he_pt_free": (None, [c_vp]),
    "he_rotate": (c_int, [c_vp, c_vp, c_i32, c_vp, c_vp]),
    "he_rotate_hoisted": (c_int, [c_vp, c_vp, I32P, c_size_t, ctypes.POINTER(c_vp), c_vp]),
    "he_ct_zero": (c_int, [c_vp, c_int, c_double, c_vp]),
    "he_mul_pt_acc": (c_int, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "he_rescale": (c_int, [c_vp, c_vp, c_vp]),
    "he_add": (c_int, [c_vp, c_vp, c_vp, c_vp]),
    "he_sub": (c_int, [c_vp, c_vp, c_vp, c_vp]),
    "he_mul_int": (c_int, [c_vp, c_vp, c_double, c_vp]),
    "he_add_const_int": (c_int, [c_vp, c_vp, c_double, c_vp]),
    "he_mul_relin": (c_int, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "he_keygen_conjugation": (c_int, [c_vp]),
    "he_conjugate": (c_int, [c_vp, c_vp, c_vp, c_vp]),
    "he_mul_monomial": (c_int, [c_vp, c_vp, ctypes.c_int64, c_vp]),
    "he_modraise": (c_int, [c_vp, c_vp, c_int, c_vp, c_vp]),
    "he_boot_create": (c_int, [c_vp, ctypes.POINTER(he_boot_config), ctypes.POINTER(c_vp)]),
    "he_boot_destroy": (None, [c_vp]),
    "he_boot_rotations": (c_int, [c_vp, I32P, c_size_t]),
    "he_boot_info": (c_int, [c_vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                             ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "he_boot_n_plaintexts": (c_int, [c_vp, c_int, c_int]),
    "he_boot_import_plaintexts": (c_int, [c_vp, c_int, c_int, I64P]),
    "he_boot_import_coeffs": (c_int, [c_vp, F64P, c_int]),
    "he_boot_lintrans": (c_int, [c_vp, c_vp, c_int, c_int, c_vp, c_vp, c_vp]),
    "he_bootstrap": (c_int, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "he_bootstrap_meta": (c_int, [c_vp, c_vp, c_vp, c_int, c_vp, c_vp]),
    "he_conv_create": (c_int, [c_vp, ctypes.POINTER(he_layout), F64P, F64P, c_int, c_int, c_int, c_int,
                               c_int, c_int, c_int, c_double, ctypes.POINTER(c_vp)]),
    "he_conv_create_factored": (c_int, [c_vp, ctypes.POINTER(he_layout), F64P, F64P, c_int, c_int, c_int, c_int,
                                        c_int, c_int, c_int, c_double, ctypes.POINTER(c_vp)]),
    "he_conv_create_bsgs": (c_int, [c_vp, ctypes.POINTER(he_layout), F64P, F64P, c_int, c_int, c_int, c_int,
                                    c_int, c_int, c_int, c_double, c_int, ctypes.POINTER(c_vp)]),
    "he_conv_bsgs_giant": (c_int, [c_vp]),
    "he_conv_destroy": (None, [c_vp]),
    "he_conv_fork": (c_int, [c_vp, c_vp, ctypes.POINTER(c_vp)]),
    "he_conv_out_layout": (c_int, [c_vp, ctypes.POINTER(he_layout)]),
    "he_conv_out_level": (c_int, [c_vp]),
    "he_conv_select_pool": (c_int, [c_vp, ctypes.POINTER(c_vp)]),
    "he_conv_rotations": (c_int, [c_vp, I32P, c_size_t]),
    "he_conv_n_terms": (c_int, [c_vp]),
    "he_conv_export_plan": (c_int, [c_vp, I32P, I32P, I32P, F64P]),
    "he_conv_import_plaintexts": (c_int, [c_vp, I64P, I64P]),
    "he_conv_run": (c_int, [c_vp, c_vp, ctypes.POINTER(c_vp), ctypes.POINTER(c_vp), c_int, c_vp]),
    "he_conv_keyswitches": (ctypes.c_int64, [c_vp]),
    "he_pool_keyswitches": (ctypes.c_int64, [c_vp]),
    "he_conv_run_batch": (c_int, [c_vp, c_vp, ctypes.POINTER(c_vp), ctypes.POINTER(c_vp), c_int, c_int, c_vp]),
    "he_conv_import_bias": (c_int, [c_vp, c_int, c_double, I64P]),
    "he_pool_create": (c_int, [c_vp, ctypes.POINTER(he_layout), c_int, ctypes.POINTER(c_vp)]),
    "he_linear_create": (c_int, [c_vp, ctypes.POINTER(he_layout), F64P, F64P, c_int, c_int, c_double,
                                 ctypes.POINTER(c_vp)]),
    "he_pool_linear_create": (c_int, [c_vp, ctypes.POINTER(he_layout), F64P, F64P, c_int, c_int, c_double,
                                      ctypes.POINTER(c_vp)]),
    "he_linear_create_packed": (c_int, [c_vp, ctypes.POINTER(he_layout), F64P, F64P, c_int, c_int, c_double,
                                        ctypes.POINTER(c_vp)]),
    "he_pool_linear_create_packed": (c_int, [c_vp, ctypes.POINTER(he_layout), F64P, F64P, c_int, c_int, c_double,
                                             ctypes.POINTER(c_vp)]),
    "he_linear_destroy": (None, [c_vp]),
    "he_ct_check_range": (ctypes.c_longlong, [c_vp, c_vp, c_vp]),
    "he_debug_fail_alloc": (c_int, [ctypes.c_long]),
    "he_cheb_minimax": (c_int, [c_int, c_int, c_double, c_double, F64P, F64P]),
    "he_cheb_interp": (c_int, [c_int, c_int, c_double, c_double, F64P]),
    "he_poly_ps_plan": (c_int, [c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "he_linear_rotations": (c_int, [c_vp, I32P, c_size_t]),
    "he_linear_out_level": (c_int, [c_vp]),
    "he_linear_keyswitches": (ctypes.c_int64, [c_vp]),
    "he_linear_import_plaintexts": (c_int, [c_vp, I64P, I64P, I64P]),
    "he_linear_run": (c_int, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "he_pool_destroy": (None, [c_vp]),
    "he_pool_fork": (c_int, [c_vp, c_vp, ctypes.POINTER(c_vp)]),
    "he_pool_out_layout": (c_int, [c_vp, ctypes.POINTER(he_layout)]),
    "he_pool_rotations": (c_int, [c_vp, I32P, c_size_t]),
    "he_pool_n_masks": (c_int, [c_vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "he_pool_import_plaintexts": (c_int, [c_vp, I64P, I64P]),
    "he_pool_run": (c_int, [c_vp, c_vp, ctypes.POINTER(c_vp), ctypes.POINTER(c_vp), c_int, c_vp]),
    "he_poly_eval": (c_int, [c_vp, c_vp, F64P, c_int, c_double, c_vp]),
    "he_poly_eval_many": (c_int, [c_vp, ctypes.POINTER(c_vp), c_int, F64P, c_int, F64P, c_vp]),
    "he_poly_eval_ps": (c_int, [c_vp, c_vp, F64P, c_int, c_double, c_vp]),
    "he_poly_eval_ps_many": (c_int, [c_vp, ctypes.POINTER(c_vp), c_int, F64P, c_int, F64P, c_vp]),
    "he_hconv2d": (c_int, [c_vp, ctypes.POINTER(he_layout), ctypes.POINTER(c_vp), F64P, F64P, c_int, c_int,
                           c_int, c_int, c_int, c_int, c_int, ctypes.POINTER(he_layout),
                           ctypes.POINTER(c_vp), c_vp]),
    "he_havgpool": (c_int, [c_vp, ctypes.POINTER(he_layout), ctypes.POINTER(c_vp), ctypes.POINTER(he_layout),
                            ctypes.POINTER(c_vp), c_int, c_vp]),
    "he_bench_modmul": (c_int, [c_vp, c_int, c_int, ctypes.POINTER(c_double)]),
    "he_bench_mac": (c_int, [c_vp, c_int, c_int, ctypes.POINTER(c_double)]),
    "he_rescale_noalloc": (c_int, [c_vp, c_vp, c_vp]),
    "he_trace_start": (c_int, [ctypes.c_char_p]),
    "he_trace_stop": (c_int, [ctypes.POINTER(c_double), ctypes.POINTER(c_u64), ctypes.POINTER(c_double),
                              ctypes.POINTER(c_double)]),
}

_lib = None


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libhegpu.so (building it with nvcc when it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libhegpu.so is missing: build it with paper_2306_09189_gb300/build.py")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(rc):
    if isinstance(rc, int) and rc < 0:
        raise HEError(rc, load().he_last_error().decode())
    return rc


def _p(a, t):
    return a.ctypes.data_as(t)


def stream_ptr(stream=None):
    """cudaStream_t of a torch stream (None -> torch's current stream, if torch is present)."""
    if stream is not None:
        return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return None


def _vp_array(objs):
    arr = (c_vp * len(objs))()
    for i, o in enumerate(objs):
        arr[i] = o.value if isinstance(o, ctypes.c_void_p) else o
    return arr


# ----------------------------------------------------------------------------- host-only
def he_params_primes(params: he_params):
    q = np.zeros(params.n_q, dtype=np.uint64)
    p = np.zeros(params.n_p, dtype=np.uint64)
    _check(load().he_params_primes(ctypes.byref(params), _p(q, U64P), _p(p, U64P)))
    return q, p


def he_layout_image(c, m, N):
    lay = he_layout()
    _check(load().he_layout_image(c, m, N, ctypes.byref(lay)))
    return lay


def he_kernel_launches():
    return int(load().he_kernel_launches())


# ----------------------------------------------------------------------------- context
def he_ctx_create(params: he_params):
    h = c_vp()
    _check(load().he_ctx_create(ctypes.byref(params), ctypes.byref(h)))
    return h


def he_ctx_destroy(ctx):
    load().he_ctx_destroy(ctx)


def he_ctx_check(ctx, stream=None):
    _check(load().he_ctx_check(ctx, stream_ptr(stream)))


def he_ctx_set_option(ctx, option, value):
    _check(load().he_ctx_set_option(ctx, option, value))


def he_ctx_get_option(ctx, option):
    v = c_int()
    _check(load().he_ctx_get_option(ctx, option, ctypes.byref(v)))
    return v.value


def he_ctx_tuning_log(ctx):
    n = load().he_ctx_tuning_log(ctx, None, 0)
    buf = ctypes.create_string_buffer(n + 1)
    load().he_ctx_tuning_log(ctx, buf, n + 1)
    return buf.value.decode()


def he_selftest_bounded_wait(ctx, stream=None):
    _check(load().he_selftest_bounded_wait(ctx, stream_ptr(stream)))


def he_graph_begin(ctx, stream=None):
    _check(load().he_graph_begin(ctx, stream_ptr(stream)))


def he_graph_end(ctx, stream=None):
    g = c_vp()
    _check(load().he_graph_end(ctx, stream_ptr(stream), ctypes.byref(g)))
    return g


def he_graph_launch(graph, stream=None):
    _check(load().he_graph_launch(graph, stream_ptr(stream)))


def he_graph_kernels(graph):
    return int(load().he_graph_kernels(graph))


def he_graph_destroy(graph):
    load().he_graph_destroy(graph)


def he_ctx_fork(ctx):
    h = c_vp()
    _check(load().he_ctx_fork(ctx, ctypes.byref(h)))
    return h


def he_ctx_info(ctx):
    vals = [c_int() for _ in range(6)]
    _check(load().he_ctx_info(ctx, *[ctypes.byref(v) for v in vals], None, None))
    n, slots, L, K, dnum, alpha = [v.value for v in vals]
    q = np.zeros(L + 1, dtype=np.uint64)
    p = np.zeros(K, dtype=np.uint64)
    _check(load().he_ctx_info(ctx, *[ctypes.byref(v) for v in vals], _p(q, U64P), _p(p, U64P)))
    return dict(n=n, slots=slots, L=L, K=K, dnum=dnum, alpha=alpha, q=q, p=p)


def he_keygen_rotations(ctx, rots):
    r = np.ascontiguousarray(rots, dtype=np.int32)
    _check(load().he_keygen_rotations(ctx, _p(r, I32P), r.size))


def he_keygen_relin(ctx):
    _check(load().he_keygen_relin(ctx))


def he_key_export(ctx, rot, shape):
    out = np.zeros(shape, dtype=np.uint64)
    _check(load().he_key_export(ctx, rot, _p(out, U64P)))
    return out


def he_key_bytes(ctx):
    return int(load().he_key_bytes(ctx))


# ----------------------------------------------------------------------------- ciphertexts
def he_ct_alloc(ctx, level):
    h = c_vp()
    _check(load().he_ct_alloc(ctx, level, ctypes.byref(h)))
    return h


def he_ct_wrap(ctx, dev_ptr, nbytes, level):
    h = c_vp()
    _check(load().he_ct_wrap(ctx, dev_ptr, nbytes, level, ctypes.byref(h)))
    return h


def he_ct_free(ct):
    load().he_ct_free(ct)


def he_ct_level(ct):
    return _check(load().he_ct_level(ct))


def he_ct_scale(ct):
    return load().he_ct_scale(ct)


def he_ct_set_scale(ct, s):
    _check(load().he_ct_set_scale(ct, s))


def he_ct_copy(dst, src, stream=None):
    _check(load().he_ct_copy(dst, src, stream_ptr(stream)))


def he_ct_drop_level(ct, level):
    _check(load().he_ct_drop_level(ct, level))


def he_ct_import_coeffs(ct, coeffs, level, scale, stream=None):
    a = np.ascontiguousarray(coeffs, dtype=np.uint64)
    _check(load().he_ct_import_coeffs(ct, _p(a, U64P), level, scale, stream_ptr(stream)))


def he_ct_export_coeffs(ctx, ct, n, stream=None):
    level = he_ct_level(ct)
    out = np.zeros((2, level + 1, n), dtype=np.uint64)
    _check(load().he_ct_export_coeffs(ct, _p(out, U64P), stream_ptr(stream)))
    return out


def he_encrypt_coeffs(ctx, m, level, scale, nonce, out, stream=None):
    a = np.ascontiguousarray(m, dtype=np.int64)
    _check(load().he_encrypt_coeffs(ctx, _p(a, I64P), level, scale, nonce, out, stream_ptr(stream)))


def he_encrypt(ctx, slots, level, scale, nonce, out, stream=None):
    z = np.ascontiguousarray(slots, dtype=np.float64)
    _check(load().he_encrypt(ctx, _p(z, F64P), z.size, level, scale, nonce, out, stream_ptr(stream)))


def he_decrypt(ctx, ct, n_slots, stream=None):
    out = np.zeros(n_slots, dtype=np.float64)
    _check(load().he_decrypt(ctx, ct, _p(out, F64P), n_slots, stream_ptr(stream)))
    return out


def he_pt_import_coeffs(ctx, m, level, scale):
    a = np.ascontiguousarray(m, dtype=np.int64)
    h = c_vp()
    _check(load().he_pt_import_coeffs(ctx, _p(a, I64P), level, scale, ctypes.byref(h)))
    return h


def he_pt_encode(ctx, slots, level, scale):
    z = np.ascontiguousarray(slots, dtype=np.float64)
    h = c_vp()
    _check(load().he_pt_encode(ctx, _p(z, F64P), z.size, level, scale, ctypes.byref(h)))
    return h


def he_pt_free(pt):
    load().he_pt_free(pt)


# ----------------------------------------------------------------------------- primitives
def he_rotate(ctx, ct_in, r, ct_out, stream=None):
    _check(load().he_rotate(ctx, ct_in, r, ct_out, stream_ptr(stream)))


def he_rotate_hoisted(ctx, ct_in, rots, outs, stream=None):
    r = np.ascontiguousarray(rots, dtype=np.int32)
    arr = _vp_array(outs)
    _check(load().he_rotate_hoisted(ctx, ct_in, _p(r, I32P), r.size, arr, stream_ptr(stream)))


def he_ct_zero(ct, level, scale, stream=None):
    _check(load().he_ct_zero(ct, level, scale, stream_ptr(stream)))


def he_mul_pt_acc(ctx, acc, ct, pt, stream=None):
    _check(load().he_mul_pt_acc(ctx, acc, ct, pt, stream_ptr(stream)))


def he_rescale(ctx, ct, stream=None):
    _check(load().he_rescale(ctx, ct, stream_ptr(stream)))


def he_rescale_noalloc(ctx, ct, stream=None):
    _check(load().he_rescale_noalloc(ctx, ct, stream_ptr(stream)))


def he_add(ctx, acc, b, stream=None):
    _check(load().he_add(ctx, acc, b, stream_ptr(stream)))


def he_sub(ctx, acc, b, stream=None):
    _check(load().he_sub(ctx, acc, b, stream_ptr(stream)))


def he_mul_int(ctx, ct, c, stream=None):
    _check(load().he_mul_int(ctx, ct, float(c), stream_ptr(stream)))


def he_add_const_int(ctx, ct, c, stream=None):
    _check(load().he_add_const_int(ctx, ct, float(c), stream_ptr(stream)))


def he_mul_relin(ctx, a, b, out, stream=None):
    _check(load().he_mul_relin(ctx, a, b, out, stream_ptr(stream)))


def he_keygen_conjugation(ctx):
    _check(load().he_keygen_conjugation(ctx))


def he_conjugate(ctx, ct_in, ct_out, stream=None):
    _check(load().he_conjugate(ctx, ct_in, ct_out, stream_ptr(stream)))


def he_mul_monomial(ctx, ct, e, stream=None):
    _check(load().he_mul_monomial(ctx, ct, int(e), stream_ptr(stream)))


def he_modraise(ctx, ct_in, level, ct_out, stream=None):
    _check(load().he_modraise(ctx, ct_in, level, ct_out, stream_ptr(stream)))


# ----------------------------------------------------------------------------- bootstrapping
def he_boot_create(ctx, K=0, double_angle=0, deg=0, levels_cts=0, levels_stc=0):
    """Bootstrapping plan (zero fields take the library's defaults: K 16, r 2, degree 59, 3 + 3
    linear levels)."""
    cfg = he_boot_config(K, double_angle, deg, levels_cts, levels_stc)
    h = c_vp()
    _check(load().he_boot_create(ctx, ctypes.byref(cfg), ctypes.byref(h)))
    return h


def he_boot_destroy(bt):
    load().he_boot_destroy(bt)


def he_boot_rotations(bt):
    n = _check(load().he_boot_rotations(bt, None, 0))
    a = np.zeros(max(n, 1), dtype=np.int32)
    _check(load().he_boot_rotations(bt, _p(a, I32P), a.size))
    return a[:n]


def he_boot_info(bt):
    v = [c_int() for _ in range(5)]
    _check(load().he_boot_info(bt, *[ctypes.byref(x) for x in v]))
    return dict(zip(("out_level", "cts_level", "evalmod_level", "stc_level", "keyswitches"), [x.value for x in v]))


def he_boot_n_plaintexts(bt, stage, idx):
    return _check(load().he_boot_n_plaintexts(bt, stage, idx))


def he_boot_import_plaintexts(bt, stage, idx, pts):
    a = np.ascontiguousarray(pts, dtype=np.int64)
    _check(load().he_boot_import_plaintexts(bt, stage, idx, _p(a, I64P)))


def he_boot_import_coeffs(bt, cheb):
    c = np.ascontiguousarray(cheb, dtype=np.float64)
    _check(load().he_boot_import_coeffs(bt, _p(c, F64P), c.size - 1))


def he_boot_lintrans(ctx, bt, stage, idx, ct_in, ct_out, stream=None):
    _check(load().he_boot_lintrans(ctx, bt, stage, idx, ct_in, ct_out, stream_ptr(stream)))


def he_bootstrap(ctx, bt, ct_in, ct_out, stream=None):
    _check(load().he_bootstrap(ctx, bt, ct_in, ct_out, stream_ptr(stream)))


def he_bootstrap_meta(ctx, bt, ct_in, ct_out, kb=10, stream=None):
    _check(load().he_bootstrap_meta(ctx, bt, ct_in, kb, ct_out, stream_ptr(stream)))


# ----------------------------------------------------------------------------- layers
def he_conv_create(ctx, layout, W, bias, stride, pad, level, in_scale):
    W = np.ascontiguousarray(W, dtype=np.float64)
    co, ci, kh, kw = W.shape
    b = None if bias is None else np.ascontiguousarray(bias, dtype=np.float64)
    h = c_vp()
    _check(load().he_conv_create(ctx, ctypes.byref(layout), _p(W, F64P), None if b is None else _p(b, F64P),
                                 co, ci, kh, kw, stride, pad, level, in_scale, ctypes.byref(h)))
    return h


def he_conv_create_factored(ctx, layout, W, bias, stride, pad, level, in_scale):
    W = np.ascontiguousarray(W, dtype=np.float64)
    co, ci, kh, kw = W.shape
    b = None if bias is None else np.ascontiguousarray(bias, dtype=np.float64)
    h = c_vp()
    _check(load().he_conv_create_factored(ctx, ctypes.byref(layout), _p(W, F64P), None if b is None else _p(b, F64P),
                                          co, ci, kh, kw, stride, pad, level, in_scale, ctypes.byref(h)))
    return h


def he_conv_create_bsgs(ctx, layout, W, bias, stride, pad, level, in_scale, giant_blocks=0):
    W = np.ascontiguousarray(W, dtype=np.float64)
    co, ci, kh, kw = W.shape
    b = None if bias is None else np.ascontiguousarray(bias, dtype=np.float64)
    h = c_vp()
    _check(load().he_conv_create_bsgs(ctx, ctypes.byref(layout), _p(W, F64P), None if b is None else _p(b, F64P),
                                      co, ci, kh, kw, stride, pad, level, in_scale, giant_blocks, ctypes.byref(h)))
    return h


def he_conv_bsgs_giant(conv):
    return _check(load().he_conv_bsgs_giant(conv))


def he_conv_destroy(conv):
    load().he_conv_destroy(conv)


def he_conv_fork(conv, ctx):
    h = c_vp()
    _check(load().he_conv_fork(conv, ctx, ctypes.byref(h)))
    return h


def he_conv_out_layout(conv):
    lay = he_layout()
    _check(load().he_conv_out_layout(conv, ctypes.byref(lay)))
    return lay


def he_conv_out_level(conv):
    return _check(load().he_conv_out_level(conv))


def he_conv_select_pool(conv):
    """The stride-2 convolution's select stage (a pool handle owned by the convolution)."""
    p = c_vp()
    _check(load().he_conv_select_pool(conv, ctypes.byref(p)))
    return p


def he_conv_rotations(conv):
    n = _check(load().he_conv_rotations(conv, None, 0))
    out = np.zeros(n, dtype=np.int32)
    load().he_conv_rotations(conv, _p(out, I32P), n)
    return out


def he_conv_n_terms(conv):
    return _check(load().he_conv_n_terms(conv))


def he_conv_export_plan(conv, n_slots=None, with_diag=False):
    t = he_conv_n_terms(conv)
    u, v, a = (np.zeros(t, dtype=np.int32) for _ in range(3))
    d = np.zeros((t, n_slots), dtype=np.float64) if with_diag else None
    _check(load().he_conv_export_plan(conv, _p(u, I32P), _p(v, I32P), _p(a, I32P),
                                      None if d is None else _p(d, F64P)))
    return u, v, a, d


def he_conv_import_plaintexts(conv, terms=None, bias=None):
    t = None if terms is None else np.ascontiguousarray(terms, dtype=np.int64)
    b = None if bias is None else np.ascontiguousarray(bias, dtype=np.int64)
    _check(load().he_conv_import_plaintexts(conv, None if t is None else _p(t, I64P),
                                            None if b is None else _p(b, I64P)))


def he_conv_run(ctx, conv, ins, outs, mode=HE_PLAIN, stream=None):
    _check(load().he_conv_run(ctx, conv, _vp_array(ins), _vp_array(outs), mode, stream_ptr(stream)))


def he_hconv2d(ctx, layout, ins, W, bias, stride, pad, mode, outs, stream=None):
    """One-call convolution (plan, rotation keys, run, release); returns the output layout.
    outs: allocated output handles, one per output shard."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    co, ci, kh, kw = W.shape
    b = None if bias is None else np.ascontiguousarray(bias, dtype=np.float64)
    lay = he_layout()
    _check(load().he_hconv2d(ctx, ctypes.byref(layout), _vp_array(ins), _p(W, F64P),
                             None if b is None else _p(b, F64P), co, ci, kh, kw, stride, pad, mode,
                             ctypes.byref(lay), _vp_array(outs), stream_ptr(stream)))
    return lay


def he_havgpool(ctx, layout, ins, mode, outs, stream=None):
    """One-call 2x2 average pool; returns the output layout."""
    lay = he_layout()
    _check(load().he_havgpool(ctx, ctypes.byref(layout), _vp_array(ins), ctypes.byref(lay), _vp_array(outs),
                              mode, stream_ptr(stream)))
    return lay


def he_conv_keyswitches(conv):
    return int(_check(load().he_conv_keyswitches(conv)))


def he_pool_keyswitches(pool):
    return int(_check(load().he_pool_keyswitches(pool)))


def he_conv_run_batch(ctx, conv, ins, outs, n_img, mode=HE_FUSED, stream=None):
    """ins: n_img * n_in shards (image-major); outs: n_img * n_out."""
    _check(load().he_conv_run_batch(ctx, conv, _vp_array(ins), _vp_array(outs), n_img, mode, stream_ptr(stream)))


def he_conv_import_bias(conv, level, out_scale, bias):
    b = np.ascontiguousarray(bias, dtype=np.int64)
    _check(load().he_conv_import_bias(conv, level, out_scale, _p(b, I64P)))


def he_linear_create(ctx, layout, W, bias, level, in_scale):
    """W [n_out][c][m][m]: a linear layer over the flattened sharded image."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    b = None if bias is None else np.ascontiguousarray(bias, dtype=np.float64)
    h = c_vp()
    _check(load().he_linear_create(ctx, ctypes.byref(layout), _p(W, F64P), None if b is None else _p(b, F64P),
                                   W.shape[0], level, in_scale, ctypes.byref(h)))
    return h


def he_pool_linear_create(ctx, layout, W, bias, level, in_scale):
    """W [n_out][c]: global average pool of every channel fused with a linear layer."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    b = None if bias is None else np.ascontiguousarray(bias, dtype=np.float64)
    h = c_vp()
    _check(load().he_pool_linear_create(ctx, ctypes.byref(layout), _p(W, F64P), None if b is None else _p(b, F64P),
                                        W.shape[0], level, in_scale, ctypes.byref(h)))
    return h


def he_linear_create_packed(ctx, layout, W, bias, level, in_scale):
    W = np.ascontiguousarray(W, dtype=np.float64)
    b = None if bias is None else np.ascontiguousarray(bias, dtype=np.float64)
    h = c_vp()
    _check(load().he_linear_create_packed(ctx, ctypes.byref(layout), _p(W, F64P), None if b is None else _p(b, F64P),
                                          W.shape[0], level, in_scale, ctypes.byref(h)))
    return h


def he_pool_linear_create_packed(ctx, layout, W, bias, level, in_scale):
    W = np.ascontiguousarray(W, dtype=np.float64)
    b = None if bias is None else np.ascontiguousarray(bias, dtype=np.float64)
    h = c_vp()
    _check(load().he_pool_linear_create_packed(ctx, ctypes.byref(layout), _p(W, F64P),
                                               None if b is None else _p(b, F64P), W.shape[0], level, in_scale,
                                               ctypes.byref(h)))
    return h


def he_linear_destroy(lin):
    load().he_linear_destroy(lin)


def he_linear_rotations(lin):
    n = _check(load().he_linear_rotations(lin, None, 0))
    out = np.zeros(n, dtype=np.int32)
    load().he_linear_rotations(lin, _p(out, I32P), n)
    return out


def he_linear_out_level(lin):
    return _check(load().he_linear_out_level(lin))


def he_linear_keyswitches(lin):
    return int(_check(load().he_linear_keyswitches(lin)))


def he_linear_import_plaintexts(lin, weights=None, masks=None, bias=None):
    arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.int64) for a in (weights, masks, bias)]
    _check(load().he_linear_import_plaintexts(lin, *[None if a is None else _p(a, I64P) for a in arrs]))


def he_linear_run(ctx, lin, ins, out, stream=None):
    _check(load().he_linear_run(ctx, lin, _vp_array(ins), out, stream_ptr(stream)))


def he_ct_check_range(ctx, ct, stream=None):
    """Words of ct not below their prime (0: well formed)."""
    return int(_check(load().he_ct_check_range(ctx, ct, stream_ptr(stream))))


def he_debug_fail_alloc(after):
    _check(load().he_debug_fail_alloc(after))


HE_FN_GELU, HE_FN_RELU, HE_FN_SILU, HE_FN_SOFTPLUS = 0, 1, 2, 3


def he_cheb_minimax(fn, deg, lo, hi):
    """(coefficients [deg + 1], levelled error) of the minimax polynomial (Remez)."""
    c = np.zeros(deg + 1, dtype=np.float64)
    e = np.zeros(1, dtype=np.float64)
    _check(load().he_cheb_minimax(fn, deg, lo, hi, _p(c, F64P), _p(e, F64P)))
    return c, float(e[0])


def he_cheb_interp(fn, deg, lo, hi):
    """Coefficients [deg + 1] of the Chebyshev interpolant at the first-kind nodes."""
    c = np.zeros(deg + 1, dtype=np.float64)
    _check(load().he_cheb_interp(fn, deg, lo, hi, _p(c, F64P)))
    return c


def he_poly_ps_plan(deg):
    """(relinearised products, levels consumed) of the Paterson-Stockmeyer evaluation."""
    p, d = c_int(), c_int()
    _check(load().he_poly_ps_plan(deg, ctypes.byref(p), ctypes.byref(d)))
    return p.value, d.value


def he_pool_create(ctx, layout, level):
    h = c_vp()
    _check(load().he_pool_create(ctx, ctypes.byref(layout), level, ctypes.byref(h)))
    return h


def he_pool_destroy(pool):
    load().he_pool_destroy(pool)


def he_pool_fork(pool, ctx):
    h = c_vp()
    _check(load().he_pool_fork(pool, ctx, ctypes.byref(h)))
    return h


def he_pool_out_layout(pool):
    lay = he_layout()
    _check(load().he_pool_out_layout(pool, ctypes.byref(lay)))
    return lay


def he_pool_rotations(pool):
    n = _check(load().he_pool_rotations(pool, None, 0))
    out = np.zeros(n, dtype=np.int32)
    load().he_pool_rotations(pool, _p(out, I32P), n)
    return out


def he_pool_n_masks(pool):
    a, b = c_int(), c_int()
    _check(load().he_pool_n_masks(pool, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def he_pool_import_plaintexts(pool, h=None, v=None):
    hh = None if h is None else np.ascontiguousarray(h, dtype=np.int64)
    vv = None if v is None else np.ascontiguousarray(v, dtype=np.int64)
    _check(load().he_pool_import_plaintexts(pool, None if hh is None else _p(hh, I64P),
                                            None if vv is None else _p(vv, I64P)))


def he_pool_run(ctx, pool, ins, outs, mode=HE_PLAIN, stream=None):
    _check(load().he_pool_run(ctx, pool, _vp_array(ins), _vp_array(outs), mode, stream_ptr(stream)))


def he_poly_eval_many(ctx, cts, cheb, target_scales, stream=None):
    c = np.ascontiguousarray(cheb, dtype=np.float64)
    t = np.ascontiguousarray(target_scales, dtype=np.float64)
    _check(load().he_poly_eval_many(ctx, _vp_array(cts), len(cts), _p(c, F64P), c.size - 1, _p(t, F64P),
                                    stream_ptr(stream)))


def he_poly_eval_ps(ctx, ct, cheb, target_scale, stream=None):
    c = np.ascontiguousarray(cheb, dtype=np.float64)
    _check(load().he_poly_eval_ps(ctx, ct, _p(c, F64P), c.size - 1, target_scale, stream_ptr(stream)))


def he_poly_eval_ps_many(ctx, cts, cheb, target_scales, stream=None):
    c = np.ascontiguousarray(cheb, dtype=np.float64)
    t = np.ascontiguousarray(target_scales, dtype=np.float64)
    _check(load().he_poly_eval_ps_many(ctx, _vp_array(cts), len(cts), _p(c, F64P), c.size - 1, _p(t, F64P),
                                       stream_ptr(stream)))


def he_poly_eval(ctx, ct, cheb, target_scale, stream=None):
    c = np.ascontiguousarray(cheb, dtype=np.float64)
    _check(load().he_poly_eval(ctx, ct, _p(c, F64P), c.size - 1, target_scale, stream_ptr(stream)))


def he_bench_modmul(ctx, blocks, iters):
    r = c_double()
    _check(load().he_bench_modmul(ctx, blocks, iters, ctypes.byref(r)))
    return r.value


def he_bench_mac(ctx, blocks, iters):
    r = c_double()
    _check(load().he_bench_mac(ctx, blocks, iters, ctypes.byref(r)))
    return r.value


def he_trace_start(kernel):
    _check(load().he_trace_start(kernel.encode()))


def he_trace_stop():
    ms, n, b, m = c_double(), c_u64(), c_double(), c_double()
    _check(load().he_trace_stop(ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b), ctypes.byref(m)))
    return dict(ms=ms.value, launches=int(n.value), bytes=b.value, mulmods=m.value)


# ----------------------------------------------------------------------------- device memory
_allocator = None          # the installed callbacks, kept alive while the library may call them


def he_set_allocator(alloc=None, free=None):
    """Install Python callables alloc(nbytes) -> device pointer (int, 0 on failure) and
    free(ptr) as the library's device allocator; no arguments restores cudaMalloc / cudaFree."""
    global _allocator
    if alloc is None and free is None:
        _check(load().he_set_allocator(HE_DEVICE_ALLOC_FN(), HE_DEVICE_FREE_FN(), None))
        _allocator = None
        return

    def _a(nbytes, _user):
        try:
            return int(alloc(int(nbytes))) or None
        except Exception:                     # out of memory: the library reports HE_ENOMEM
            return None

    def _f(ptr, _user):
        free(int(ptr))
    cbs = (HE_DEVICE_ALLOC_FN(_a), HE_DEVICE_FREE_FN(_f))
    _check(load().he_set_allocator(cbs[0], cbs[1], None))
    _allocator = cbs


def he_live_allocations():
    return int(load().he_live_allocations())


def use_torch_allocator():
    """Take every device block the library needs from PyTorch's caching allocator (on the
    current device and stream), so that the library's memory is part of torch's pool."""
    import torch
    he_set_allocator(lambda nbytes: torch.cuda.caching_allocator_alloc(nbytes),
                     lambda ptr: torch.cuda.caching_allocator_delete(ptr))


def use_default_allocator():
    he_set_allocator()
