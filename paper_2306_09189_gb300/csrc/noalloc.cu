// Rescale that performs no device allocation at call time.
//
// he_rescale works in scratch buffers that the context allocates (cudaMalloc, or the allocator
// installed with he_set_allocator).  Some callers cannot rely on that: an embedding application
// whose device memory is entirely owned by its own allocator (a framework's caching pool holding
// all of HBM), or a process running under a memory cap or policy that forbids driver
// allocations once it is set up.
// This variant keeps its scratch in a fixed device array that is part of the library image,
// reserved on every GPU that loads the library until the process exits.  The caller still
// passes the ciphertext, which is rescaled in place exactly like he_rescale does.
//
// The array lives in this translation unit's module.  Under CUDA's lazy module loading that
// module (and with it the array's device memory) is loaded the first time its address is
// asked for, so the address is looked up when a context is created (he_ctx_create calls
// he_noalloc_setup with the context's device current): the reservation then happens during
// set-up, not on the first no-allocation call.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

// [2][level][n] words: the top limb of both polynomials reduced to every remaining prime.
#define HE_NOALLOC_SCRATCH_WORDS (3u << 20)   // 24 MiB: 2 * level * n <= 3 * 2^20 words

static __device__ __align__(256) u64 g_noalloc_scratch[HE_NOALLOC_SCRATCH_WORDS];

namespace {
std::mutex g_mu;
u64 *g_addr[64] = {};      // device address of g_noalloc_scratch, per device ordinal
}  // namespace

// Device address of the scratch array on the current device.  The host-side symbol
// g_noalloc_scratch is only a stand-in: kernels must be given this address instead.
static int scratch_address(u64 **out) {
    int dev = 0;
    HE_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        he_set_error("he_rescale_noalloc: device ordinal %d out of range", dev);
        return HE_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();   // do not leave the error for a later launch check
            he_set_error("he_rescale_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return HE_ECUDA;
        }
        g_addr[dev] = (u64 *)p;
    }
    *out = g_addr[dev];
    return HE_OK;
}

// Set-up: load this module on the current device and cache the scratch array's address.
int he_noalloc_setup() {
    u64 *t = nullptr;
    return scratch_address(&t);
}

extern "C" int he_rescale_noalloc(he_ctx *c, he_ct *ct, void *stream) {
    if (!c || !ct || ct->ctx != c) { he_set_error("he_rescale_noalloc: bad argument"); return HE_EINVAL; }
    const int l = ct->level;
    if (l < 1) { he_set_error("he_rescale_noalloc: no level left"); return HE_ELEVEL; }
    const size_t need = 2 * (size_t)l * c->n;
    if (need > HE_NOALLOC_SCRATCH_WORDS) {
        he_set_error("he_rescale_noalloc: level %d at n = %d needs %zu scratch words, more than the "
                     "fixed %u; use he_rescale", l, c->n, need, (unsigned)HE_NOALLOC_SCRATCH_WORDS);
        return HE_EINVAL;
    }
    u64 *t = nullptr;
    HE_TRY(scratch_address(&t));
    cudaStream_t s = (cudaStream_t)stream;
    // same steps as he_rescale: top limb to coefficient form, centred residues of it modulo
    // every remaining prime (every scratch word is written before it is read, nothing needs
    // zeroing), back to NTT form, then (c_i - t_i) * q_l^{-1}
    HE_TRY(k_rescale_many(c, ct->d, ct->pstride, 1, l, t, s));
    ct->level = l - 1;
    ct->scale = ct->scale / (double)c->primes[l];
    return HE_OK;
}
