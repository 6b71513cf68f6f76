// Context, keys, ciphertext I/O and the per-ciphertext primitives of the C ABI.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>

#include "internal.h"

// ================================================================================ errors
static thread_local char g_err[512] = "";
static std::atomic<uint64_t> g_launches{0};

void he_set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
static thread_local bool g_capturing = false;
static thread_local uint64_t g_captured = 0;    // kernels recorded by this thread's capture
void he_count_launch(int k) {
    if (g_capturing) g_captured += (uint64_t)k;  // recorded, not run: counted per replay
    else g_launches += (uint64_t)k;
}

bool he_capturing() { return g_capturing; }
static thread_local bool g_capture_failed = false;
// Fault injection for tests (host side only): after g_fail_after more successful device
// allocations, the next one fails with HE_ENOMEM and the injection disarms (-1: disarmed).
static std::atomic<long> g_fail_after{-1};
bool he_alloc_should_fail() {
    long v = g_fail_after.load();
    while (v >= 0) {
        if (g_fail_after.compare_exchange_weak(v, v - 1)) return v == 0;
    }
    return false;
}
extern "C" int he_debug_fail_alloc(long after) {
    g_fail_after.store(after < 0 ? -1 : after);
    return HE_OK;
}

// ================================================================================ allocator
namespace {
std::mutex g_alloc_mu;
he_device_alloc_fn g_alloc_fn = nullptr;
he_device_free_fn g_free_fn = nullptr;
void *g_alloc_user = nullptr;
std::atomic<long long> g_live{0};     // device blocks the library holds (either allocator)
}  // namespace

cudaError_t he_malloc(void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    he_device_alloc_fn fn;
    void *user;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        fn = g_alloc_fn;
        user = g_alloc_user;
    }
    if (fn) {
        void *q = fn(bytes, user);
        if (!q) return cudaErrorMemoryAllocation;
        *p = q;
        g_live++;
        return cudaSuccess;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess && *p) g_live++;
    return e;
}

cudaError_t he_free(void *p) {
    if (!p) return cudaSuccess;
    he_device_free_fn fn;
    void *user;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        fn = g_free_fn;
        user = g_alloc_user;
    }
    g_live--;
    if (fn) {
        // cudaFree waits for the device; a caller's allocator may hand the block to other work
        // on any stream at once, so the library's work on it must be finished first
        cudaError_t e = cudaDeviceSynchronize();
        fn(p, user);
        return e;
    }
    return cudaFree(p);
}

extern "C" int he_set_allocator(he_device_alloc_fn alloc, he_device_free_fn free_fn, void *user) {
    if ((alloc == nullptr) != (free_fn == nullptr)) {
        he_set_error("he_set_allocator: give both functions, or neither for cudaMalloc / cudaFree");
        return HE_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    const long long live = g_live.load();
    if (live != 0) {
        he_set_error("he_set_allocator: %lld device blocks of the library are still allocated; free every "
                     "context and object first", live);
        return HE_ESTATE;
    }
    g_alloc_fn = alloc;
    g_free_fn = free_fn;
    g_alloc_user = alloc ? user : nullptr;
    return HE_OK;
}

extern "C" int64_t he_live_allocations(void) { return (int64_t)g_live.load(); }

int he_capture_guard(const char *what) {
    if (!g_capturing) return HE_OK;
    g_capture_failed = true;                     // the graph would be incomplete: discard it
    he_set_error("%s during graph capture: run the step once before capturing it", what);
    return HE_ESTATE;
}

// ================================================================================ tracing
#include <mutex>
namespace {
struct Tracer {
    std::mutex mu;
    std::string name;
    bool on = false;
    struct Rec { cudaEvent_t b, e; };
    std::vector<Rec> recs;
    double bytes = 0, mulmods = 0;
} g_tr;
}  // namespace

// Inside a graph capture the two events become external event-record nodes of the graph, so
// a graph captured while tracing (launched once before he_trace_stop) is timed per kernel too.
static cudaError_t trace_record(cudaEvent_t e, cudaStream_t s) {
    return g_capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
}

TraceScope::TraceScope(const char *name, cudaStream_t st, double bytes_, double mulmods_)
    : s(st), bytes(bytes_), mulmods(mulmods_) {
    if (!g_tr.on) return;
    std::lock_guard<std::mutex> lk(g_tr.mu);
    if (!g_tr.on || g_tr.name != name) return;
    on = true;
    cudaEventCreate(&b);
    trace_record(b, s);
}
TraceScope::~TraceScope() {
    if (!on) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    trace_record(e, s);
    std::lock_guard<std::mutex> lk(g_tr.mu);
    g_tr.recs.push_back({b, e});
    g_tr.bytes += bytes;
    g_tr.mulmods += mulmods;
}

extern "C" int he_trace_start(const char *kernel) {
    if (!kernel) return HE_EINVAL;
    std::lock_guard<std::mutex> lk(g_tr.mu);
    for (auto &r : g_tr.recs) { cudaEventDestroy(r.b); cudaEventDestroy(r.e); }
    g_tr.recs.clear();
    g_tr.bytes = g_tr.mulmods = 0;
    g_tr.name = kernel;
    g_tr.on = true;
    return HE_OK;
}

extern "C" int he_trace_stop(double *total_ms, uint64_t *launches, double *bytes, double *mulmods) {
    std::lock_guard<std::mutex> lk(g_tr.mu);
    g_tr.on = false;
    double ms = 0;
    for (auto &r : g_tr.recs) {
        float t = 0;
        if (cudaEventSynchronize(r.e) != cudaSuccess || cudaEventElapsedTime(&t, r.b, r.e) != cudaSuccess) {
            he_set_error("trace: event timing failed");
            return HE_ECUDA;
        }
        ms += t;
        cudaEventDestroy(r.b);
        cudaEventDestroy(r.e);
    }
    if (total_ms) *total_ms = ms;
    if (launches) *launches = g_tr.recs.size();
    if (bytes) *bytes = g_tr.bytes;
    if (mulmods) *mulmods = g_tr.mulmods;
    g_tr.recs.clear();
    return HE_OK;
}

extern "C" const char *he_last_error(void) { return g_err; }
extern "C" const char *he_version(void) { return "hegpu 0.1 sm_103a"; }
extern "C" uint64_t he_kernel_launches(void) { return g_launches.load(); }

// ================================================================================ host math
u64 h_mulmod(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }
u64 h_powmod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    for (; e; e >>= 1) {
        if (e & 1) r = h_mulmod(r, a, q);
        a = h_mulmod(a, a, q);
    }
    return r;
}
u64 h_invmod(u64 a, u64 q) { return h_powmod(a, q - 2, q); }
u64 h_shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }
static u64 h_mont(u64 x, u64 q) { return (u64)(((u128)(x % q) << 64) % q); }

static bool is_prime64(u64 n) {
    static const u64 bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 b : bases)
        if (n % b == 0) return n == b;
    u64 d = n - 1;
    int r = 0;
    while (!(d & 1)) { d >>= 1; r++; }
    for (u64 a : bases) {
        u64 x = h_powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < r; i++) {
            x = h_mulmod(x, x, n);
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

// Largest primes below 2^bits that are 1 mod 2n, one bit size at a time, in descending order.
struct PrimeStream {
    u64 step, cur;
    PrimeStream(int bits, u64 two_n) : step(two_n) {
        u64 top = (bits >= 64) ? ~0ull : ((1ull << bits) - 1);
        cur = top / two_n * two_n + 1;
        if (cur > top) cur -= two_n;
        cur += two_n;   // next() steps down first
    }
    u64 next() {
        for (;;) {
            cur -= step;
            if (cur <= step) return 0;
            if (is_prime64(cur)) return cur;
        }
    }
};

static int chain(const he_params *pr, std::vector<u64> &q, std::vector<u64> &p) {
    if (!pr || pr->log_n < 9 || pr->log_n > 17 || pr->n_q < 1 || pr->n_p < 1 || pr->dnum < 1 ||
        pr->n_q > 64 || pr->n_p > 16) {
        he_set_error("invalid parameters (log_n 9..17, 1<=n_q<=64, 1<=n_p<=16, dnum>=1)");
        return HE_EINVAL;
    }
    for (int b : {pr->q0_bits, pr->q_bits, pr->p_bits})
        if (b < 20 || b > 61) {
            he_set_error("prime bit sizes must lie in [20, 61]");
            return HE_EINVAL;
        }
    const u64 two_n = 2ull << (pr->log_n - 1) << 0;
    std::map<int, PrimeStream> st;
    auto draw = [&](int bits) -> u64 {
        auto it = st.find(bits);
        if (it == st.end()) it = st.emplace(bits, PrimeStream(bits, 2 * (1ull << pr->log_n))).first;
        return it->second.next();
    };
    (void)two_n;
    q.assign(1, draw(pr->q0_bits));
    p.clear();
    for (int k = 0; k < pr->n_p; k++) p.push_back(draw(pr->p_bits));
    for (int i = 1; i < pr->n_q; i++) q.push_back(draw(pr->q_bits));
    for (u64 x : q)
        if (!x) { he_set_error("ran out of primes"); return HE_EINVAL; }
    for (u64 x : p)
        if (!x) { he_set_error("ran out of primes"); return HE_EINVAL; }
    return HE_OK;
}

extern "C" int he_params_primes(const he_params *params, uint64_t *q, uint64_t *p) {
    std::vector<u64> vq, vp;
    HE_TRY(chain(params, vq, vp));
    if (q) memcpy(q, vq.data(), vq.size() * 8);
    if (p) memcpy(p, vp.data(), vp.size() * 8);
    return HE_OK;
}

static unsigned brev_bits(unsigned x, int bits) {
    unsigned r = 0;
    for (int b = 0; b < bits; b++)
        if (x >> b & 1) r |= 1u << (bits - 1 - b);
    return r;
}

// A primitive 2n-th root: for the smallest x with x^((q-1)/2) = -1, psi0 = x^((q-1)/2n)
// has order 2n; this library uses psi = psi0^3 (any odd power has the same order).
static u64 root_2n(u64 q, u64 n) {
    u64 x = 2;
    while (h_powmod(x, (q - 1) / 2, q) != q - 1) x++;
    u64 psi = h_powmod(h_powmod(x, (q - 1) / (2 * n), q), 3, q);
    return psi;
}

int prime_index(const he_ctx *ctx, int limb, int nq) {
    return limb < nq ? limb : ctx->L + 1 + (limb - nq);
}

u64 h_galois(const he_ctx *ctx, int32_t r) {
    long long rr = ((long long)r % ctx->N + ctx->N) % ctx->N;
    return h_powmod(5, (u64)rr, 2ull * ctx->n);
}

// ================================================================================ scratch
int Scratch::ensure(size_t w) {
    if (w <= words) return HE_OK;
    HE_TRY(he_capture_guard("scratch allocation"));
    if (p) he_free(p);
    p = nullptr;
    words = 0;
    if (he_alloc_should_fail() || he_malloc(&p, w * 8) != cudaSuccess) {
        cudaGetLastError();
        he_set_error("scratch allocation of %zu bytes failed", w * 8);
        return HE_ENOMEM;
    }
    words = w;
    return HE_OK;
}
Scratch::~Scratch() {
    if (p) he_free(p);
}

int upload_async(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    HE_CHECK_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
    return HE_OK;
}

// ================================================================================ context
static int build_fbc(he_ctx *c, const std::vector<int> &src, const std::vector<int> &dst,
                     FbcTable &t) {
    const int ns = (int)src.size(), nd = (int)dst.size();
    std::vector<u64> h(2 * ns + 2 * (size_t)nd * ns);
    for (int i = 0; i < ns; i++) {
        u64 qi = c->primes[src[i]];
        u64 prod = 1;
        for (int k = 0; k < ns; k++)
            if (k != i) prod = h_mulmod(prod, c->primes[src[k]] % qi, qi);
        h[i] = h_invmod(prod, qi);
        h[ns + i] = h_shoup(h[i], qi);
    }
    for (int d = 0; d < nd; d++) {
        u64 pd = c->primes[dst[d]];
        for (int i = 0; i < ns; i++) {
            u64 prod = 1 % pd;
            for (int k = 0; k < ns; k++)
                if (k != i) prod = h_mulmod(prod, c->primes[src[k]] % pd, pd);
            h[2 * ns + (size_t)d * ns + i] = h_mont(prod, pd);
            h[2 * ns + (size_t)nd * ns + (size_t)d * ns + i] = h_mont((pd - prod) % pd, pd);
        }
    }
    t.n_src = ns;
    t.n_dst = nd;
    t.src_prime = src;
    t.dst_prime = dst;
    HE_CHECK_CUDA(he_malloc(&t.d, h.size() * 8));
    HE_CHECK_CUDA(cudaMemcpy(t.d, h.data(), h.size() * 8, cudaMemcpyHostToDevice));
    return HE_OK;
}

static void free_ctx(he_ctx *c) {
    if (!c) return;
    for (he_ct *t : c->poly_tmp) he_ct_free(t);
    if (c->poly_block) he_free(c->poly_block);
    if (c->d_err) he_free(c->d_err);
    if (c->parent) {                       // a fork owns only its scratch
        delete c;
        return;
    }
    for (auto &lv : c->modup)
        for (auto &t : lv)
            if (t.d) he_free(t.d);
    for (auto &t : c->moddown)
        if (t.d) he_free(t.d);
    for (auto &kv : c->keys)
        if (kv.second.d) he_free(kv.second.d);
    for (auto &kv : c->pk_cache) { he_free(kv.second.Kp); he_free(kv.second.Ppt); }
    if (c->d_tables) he_free(c->d_tables);
    if (c->d_consts) he_free(c->d_consts);
    if (c->d_s) he_free(c->d_s);
    delete c;
}

static int ntt_poly(he_ctx *c, u64 *base, size_t pstride, int l0, int nl, int nq, int npoly,
                    bool inverse, cudaStream_t s) {
    ntt_job j{base, pstride, l0, nl, nq, 0, npoly};
    return k_ntt(c, j, inverse, s);
}

static int create(const he_params *pr, he_ctx **out) {
    std::vector<u64> q, p;
    HE_TRY(chain(pr, q, p));
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
        cudaGetLastError();
        he_set_error("no CUDA device: this library has no CPU fallback");
        return HE_ECUDA;
    }
    {
        // hybrid key switching divides by P = prod p_k; P must exceed every digit's modulus
        // (a product of alpha ciphertext primes) or the switching noise swamps the message
        const int alpha = (pr->n_q + pr->dnum - 1) / pr->dnum;
        double bits_P = 0, worst = 0;
        for (u64 x : p) bits_P += std::log2((double)x);
        for (int j = 0; j * alpha < pr->n_q; j++) {
            double b = 0;
            for (int i = j * alpha; i < std::min(pr->n_q, (j + 1) * alpha); i++) b += std::log2((double)q[i]);
            worst = std::max(worst, b);
        }
        if (bits_P < worst) {
            he_set_error("parameters: the special primes give %.0f bits, below the largest key-switching "
                         "digit (%.0f bits); raise n_p or dnum", bits_P, worst);
            return HE_EINVAL;
        }
    }
    if (pr->secret_hw < 0 || pr->secret_hw > (1 << pr->log_n)) {
        he_set_error("parameters: secret_hw must lie in [0, n]");
        return HE_EINVAL;
    }
    he_ctx *c = new he_ctx();
    c->pr = *pr;
    c->small_primes = true;
    for (u64 x : q) c->small_primes = c->small_primes && x < (1ull << 57);
    for (u64 x : p) c->small_primes = c->small_primes && x < (1ull << 57);
    c->logn = pr->log_n;
    c->n = 1 << pr->log_n;
    c->N = c->n / 2;
    c->L = pr->n_q - 1;
    c->K = pr->n_p;
    c->alpha = (pr->n_q + pr->dnum - 1) / pr->dnum;
    c->dnum = (pr->n_q + c->alpha - 1) / c->alpha;   // non-empty digits
    c->np = pr->n_q + pr->n_p;
    c->primes = q;
    c->primes.insert(c->primes.end(), p.begin(), p.end());
    const int n = c->n, np = c->np;
    // ---- per-prime tables
    c->psi.resize(np);
    c->h_qinv.resize(np);
    c->h_mu.resize(np);
    c->h_r2.resize(np);
    std::vector<u64> tw((size_t)np * n), tws(tw.size()), itw(tw.size()), itws(tw.size());
    std::vector<u64> ninv(np), ninvs(np);
    for (int t = 0; t < np; t++) {
        u64 qq = c->primes[t];
        u64 inv = qq;                              // Newton: q^-1 mod 2^64
        for (int it = 0; it < 6; it++) inv *= 2 - qq * inv;
        c->h_qinv[t] = inv;
        c->h_mu[t] = (u64)(((u128)1 << 64) / qq);
        u64 r1 = (u64)(((u128)1 << 64) % qq);
        c->h_r2[t] = h_mulmod(r1, r1, qq);
        u64 psi = root_2n(qq, n);
        c->psi[t] = psi;
        u64 ipsi = h_invmod(psi, qq);
        for (int k = 0; k < n; k++) {
            unsigned e = brev_bits((unsigned)k, c->logn);
            size_t o = (size_t)t * n + k;
            tw[o] = h_powmod(psi, e, qq);
            tws[o] = h_shoup(tw[o], qq);
            itw[o] = h_powmod(ipsi, e, qq);
            itws[o] = h_shoup(itw[o], qq);
        }
        ninv[t] = h_invmod((u64)n % qq, qq);
        ninvs[t] = h_shoup(ninv[t], qq);
    }
    std::vector<u64> tw2(2 * tw.size()), itw2(2 * tw.size());
    for (size_t k = 0; k < tw.size(); k++) {
        tw2[2 * k] = tw[k];
        tw2[2 * k + 1] = tws[k];
        itw2[2 * k] = itw[k];
        itw2[2 * k + 1] = itws[k];
    }
    size_t words = 4 * (size_t)np + 8 * (size_t)np * n + 2 * (size_t)np;
    if (he_malloc(&c->d_tables, words * 8) != cudaSuccess) {
        cudaGetLastError();
        free_ctx(c);
        he_set_error("table allocation failed");
        return HE_ENOMEM;
    }
    u64 *d = c->d_tables;
    auto put = [&](const u64 *src, size_t w) {
        cudaMemcpy(d, src, w * 8, cudaMemcpyHostToDevice);
        u64 *r = d;
        d += w;
        return r;
    };
    c->kp.n = n;
    c->kp.logn = c->logn;
    c->kp.L = c->L;
    c->kp.K = c->K;
    c->kp.q = put(c->primes.data(), np);
    c->kp.qinv = put(c->h_qinv.data(), np);
    c->kp.r2 = put(c->h_r2.data(), np);
    c->kp.mu = put(c->h_mu.data(), np);
    c->kp.tw = put(tw.data(), tw.size());
    c->kp.tws = put(tws.data(), tws.size());
    c->kp.itw = put(itw.data(), itw.size());
    c->kp.itws = put(itws.data(), itws.size());
    c->kp.ninv = put(ninv.data(), np);
    c->kp.ninvs = put(ninvs.data(), np);
    c->kp.tw2 = put(tw2.data(), tw2.size());
    c->kp.itw2 = put(itw2.data(), itw2.size());
    // ---- base conversion tables
    c->modup.resize(c->L + 1);
    c->moddown.resize(c->L + 1);
    for (int l = 0; l <= c->L; l++) {
        const int nq = l + 1;
        const int beta = (nq + c->alpha - 1) / c->alpha;
        c->modup[l].resize(beta);
        for (int j = 0; j < beta; j++) {
            std::vector<int> src, dst;
            int lo = j * c->alpha, hi = std::min(lo + c->alpha, nq);
            for (int i = lo; i < hi; i++) src.push_back(i);
            for (int limb = 0; limb < nq + c->K; limb++)
                if (limb < lo || limb >= hi) dst.push_back(prime_index(c, limb, nq));
            if (build_fbc(c, src, dst, c->modup[l][j]) != HE_OK) { free_ctx(c); return HE_ECUDA; }
        }
        std::vector<int> src, dst;
        for (int k = 0; k < c->K; k++) src.push_back(c->L + 1 + k);
        for (int i = 0; i < nq; i++) dst.push_back(i);
        if (build_fbc(c, src, dst, c->moddown[l]) != HE_OK) { free_ctx(c); return HE_ECUDA; }
    }
    // ---- small constants: pmod[np] | pinv[L+1] | pinvs[L+1] | per level l: inv[L+1], invs[L+1]
    const int Q = c->L + 1;
    std::vector<u64> cst(np + 2 * Q + (size_t)Q * 2 * Q, 0);
    c->pmod.assign(Q, 0);
    for (int t = 0; t < np; t++) {
        u64 v = 1;
        for (int k = 0; k < c->K; k++) v = h_mulmod(v, c->primes[Q + k] % c->primes[t], c->primes[t]);
        cst[t] = t < Q ? v : 0;
        if (t < Q) c->pmod[t] = v;
    }
    for (int i = 0; i < Q; i++) {
        cst[np + i] = h_invmod(c->pmod[i], c->primes[i]);
        cst[np + Q + i] = h_shoup(cst[np + i], c->primes[i]);
    }
    for (int l = 1; l < Q; l++)
        for (int i = 0; i < l; i++) {
            u64 qi = c->primes[i];
            u64 v = h_invmod(c->primes[l] % qi, qi);
            cst[np + 2 * Q + (size_t)l * 2 * Q + i] = v;
            cst[np + 2 * Q + (size_t)l * 2 * Q + Q + i] = h_shoup(v, qi);
        }
    if (he_malloc(&c->d_consts, cst.size() * 8) != cudaSuccess) {
        cudaGetLastError();
        free_ctx(c);
        he_set_error("constant allocation failed");
        return HE_ENOMEM;
    }
    cudaMemcpy(c->d_consts, cst.data(), cst.size() * 8, cudaMemcpyHostToDevice);
    // ---- scratch
    const size_t ext = (size_t)(Q + c->K) * n;
    int rc = HE_OK;
    if (rc == HE_OK) rc = c->sc_digits.ensure((size_t)c->dnum * ext);
    if (rc == HE_OK) rc = c->sc_u.ensure(2 * ext);
    if (rc == HE_OK) rc = c->sc_conv.ensure(2 * (size_t)Q * n);
    if (rc == HE_OK) rc = c->sc_tmp.ensure(3 * ext);
    if (rc == HE_OK) rc = c->sc_tmp2.ensure(ext);
    if (rc != HE_OK) { free_ctx(c); return rc; }
    // ---- secret key: ternary s (uniform, or sparse of a given weight), NTT form over every prime
    int64_t *s_int = nullptr;
    if (he_malloc(&c->d_s, (size_t)np * n * 8) != cudaSuccess ||
        he_malloc(&s_int, (size_t)n * 8) != cudaSuccess) {
        cudaGetLastError();
        if (s_int) he_free(s_int);
        free_ctx(c);
        he_set_error("secret allocation failed");
        return HE_ENOMEM;
    }
    if (he_malloc(&c->d_err, sizeof(int)) != cudaSuccess || cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        he_free(s_int);
        free_ctx(c);
        he_set_error("error-word allocation failed");
        return HE_ENOMEM;
    }
    // uniform ternary, or sparse of weight secret_hw (stream 6 << 56; the permutation in sc_tmp)
    if (pr->secret_hw > 0) rc = k_sample_sparse(c, pr->seed, 6ull << 56, pr->secret_hw, (int32_t *)c->sc_tmp.p, s_int, 0);
    else rc = k_sample_ternary(c, pr->seed, 1, s_int, 0);
    if (rc == HE_OK) rc = k_reduce_int(c, s_int, c->d_s, np, Q, false, 0);
    if (rc == HE_OK) rc = ntt_poly(c, c->d_s, 0, 0, np, Q, 1, false, 0);
    cudaDeviceSynchronize();
    he_free(s_int);
    cudaError_t e = cudaGetLastError();
    if (rc != HE_OK || e != cudaSuccess) {
        if (e != cudaSuccess) he_set_error("context setup: %s", cudaGetErrorString(e));
        free_ctx(c);
        return HE_ECUDA;
    }
    *out = c;
    return HE_OK;
}

extern "C" int he_ctx_create(const he_params *params, he_ctx **out) {
    if (!out) { he_set_error("null output"); return HE_EINVAL; }
    *out = nullptr;
    int rc = create(params, out);
    if (rc != HE_OK) return rc;
    // reserve the no-allocation rescale's fixed scratch now, during set-up (see noalloc.cu)
    rc = he_noalloc_setup();
    if (rc != HE_OK) {
        he_ctx_destroy(*out);
        *out = nullptr;
    }
    return rc;
}
extern "C" void he_ctx_destroy(he_ctx *ctx) {
    if (ctx) cudaDeviceSynchronize();
    free_ctx(ctx);
}
extern "C" int he_ctx_info(const he_ctx *c, int *n, int *slots, int *L, int *K, int *dnum,
                           int *alpha, uint64_t *q, uint64_t *p) {
    if (!c) { he_set_error("null context"); return HE_EINVAL; }
    if (n) *n = c->n;
    if (slots) *slots = c->N;
    if (L) *L = c->L;
    if (K) *K = c->K;
    if (dnum) *dnum = c->dnum;
    if (alpha) *alpha = c->alpha;
    if (q) memcpy(q, c->primes.data(), (c->L + 1) * 8);
    if (p) memcpy(p, c->primes.data() + c->L + 1, c->K * 8);
    return HE_OK;
}

// ================================================================================ keys
static int gen_key(he_ctx *c, int id, const u64 *sp_eval, cudaStream_t s) {
    const int np = c->np, n = c->n, Q = c->L + 1;
    const size_t limbs = (size_t)np * n;
    DeviceKey key;
    key.id = id;
    HE_TRY(he_capture_guard("key generation"));
    if (he_malloc(&key.d, (size_t)c->dnum * 2 * limbs * 8) != cudaSuccess) {
        cudaGetLastError();
        he_set_error("key allocation failed (%zu bytes)", (size_t)c->dnum * 2 * limbs * 8);
        return HE_ENOMEM;
    }
    u64 *e_eval = c->sc_tmp.p;                       // [np][n]
    int64_t *e_int = (int64_t *)(c->sc_tmp.p + limbs);
    int rc = HE_OK;
    for (int j = 0; j < c->dnum && rc == HE_OK; j++) {
        u64 *b = key.d + (size_t)(2 * j) * limbs;
        u64 *a = b + limbs;
        const u64 sa = (2ull << 56) | ((u64)id << 8) | (u64)j;
        const u64 se = (3ull << 56) | ((u64)id << 8) | (u64)j;
        rc = k_sample_uniform(c, c->pr.seed, sa, a, np, Q, s);
        if (rc == HE_OK) rc = ntt_poly(c, a, 0, 0, np, Q, 1, false, s);
        if (rc == HE_OK) rc = k_sample_cbd(c, c->pr.seed, se, e_int, s);
        if (rc == HE_OK) rc = k_reduce_int(c, e_int, e_eval, np, Q, false, s);
        if (rc == HE_OK) rc = ntt_poly(c, e_eval, 0, 0, np, Q, 1, false, s);
        if (rc == HE_OK) rc = k_keygen_combine(c, b, a, e_eval, c->d_s, sp_eval, j, s);
    }
    if (rc != HE_OK) {
        he_free(key.d);
        return rc;
    }
    c->root()->keys[id] = key;
    c->root()->key_bytes += (size_t)c->dnum * 2 * limbs * 8;
    return HE_OK;
}

extern "C" int he_keygen_rotations(he_ctx *c, const int32_t *rot, size_t n_rot) {
    if (!c || (!rot && n_rot)) { he_set_error("null argument"); return HE_EINVAL; }
    cudaStream_t s = 0;
    u64 *sp = c->sc_tmp2.p;      // [np][n]
    for (size_t i = 0; i < n_rot; i++) {
        u64 g = h_galois(c, rot[i]);
        if (g == 1 || c->root()->keys.count((int)g)) continue;
        HE_TRY(k_permute(c, c->d_s, sp, c->np, g, s));
        HE_TRY(gen_key(c, (int)g, sp, s));
    }
    HE_CHECK_CUDA(cudaStreamSynchronize(s));
    return HE_OK;
}

extern "C" int he_keygen_relin(he_ctx *c) {
    if (!c) { he_set_error("null context"); return HE_EINVAL; }
    if (c->root()->keys.count(0)) return HE_OK;
    u64 *sp = c->sc_tmp2.p;
    HE_TRY(k_mul_pointwise(c, c->d_s, c->d_s, sp, c->np, 0));
    HE_TRY(gen_key(c, 0, sp, 0));
    HE_CHECK_CUDA(cudaStreamSynchronize(0));
    return HE_OK;
}

extern "C" int he_keygen_conjugation(he_ctx *c) {
    if (!c) { he_set_error("null context"); return HE_EINVAL; }
    const u64 g = 2ull * c->n - 1;
    if (c->root()->keys.count((int)g)) return HE_OK;
    u64 *sp = c->sc_tmp2.p;
    HE_TRY(k_permute(c, c->d_s, sp, c->np, g, 0));
    HE_TRY(gen_key(c, (int)g, sp, 0));
    HE_CHECK_CUDA(cudaStreamSynchronize(0));
    return HE_OK;
}

extern "C" int he_has_rotation_key(const he_ctx *c, int32_t rot) {
    if (!c) return 0;
    u64 g = h_galois(c, rot);
    return g == 1 || c->root()->keys.count((int)g) ? 1 : 0;
}

int get_key(he_ctx *c, int id, const DeviceKey **out) {
    auto &keys = c->root()->keys;
    auto it = keys.find(id);
    if (it == keys.end()) {
        he_set_error(id == 0 ? "relinearisation key missing" : "rotation key for Galois element %d missing", id);
        return HE_EKEY;
    }
    *out = &it->second;
    return HE_OK;
}

extern "C" int he_key_export(he_ctx *c, int32_t rot, uint64_t *host) {
    if (!c || !host) { he_set_error("null argument"); return HE_EINVAL; }
    int id = rot == HE_RELIN_KEY ? 0 : (int)h_galois(c, rot);
    const DeviceKey *k;
    HE_TRY(get_key(c, id, &k));
    const size_t limbs = (size_t)c->np * c->n;
    u64 *tmp = c->sc_tmp.p;
    for (int j = 0; j < c->dnum; j++)
        for (int h = 0; h < 2; h++) {
            HE_CHECK_CUDA(cudaMemcpy(tmp, k->d + (size_t)(2 * j + h) * limbs, limbs * 8,
                                     cudaMemcpyDeviceToDevice));
            HE_TRY(k_from_mont(c, tmp, c->np, c->L + 1, 1, 0, 0));
            HE_TRY(ntt_poly(c, tmp, 0, 0, c->np, c->L + 1, 1, true, 0));
            HE_CHECK_CUDA(cudaMemcpy(host + (size_t)(2 * j + h) * limbs, tmp, limbs * 8,
                                     cudaMemcpyDeviceToHost));
        }
    return HE_OK;
}

extern "C" size_t he_key_bytes(const he_ctx *c) { return c ? c->root()->key_bytes : 0; }

extern "C" int he_ctx_fork(he_ctx *parent, he_ctx **out) {
    if (!parent || !out) { he_set_error("he_ctx_fork: null argument"); return HE_EINVAL; }
    he_ctx *r = parent->root();
    he_ctx *c = new he_ctx();
    c->pr = r->pr;
    c->n = r->n; c->logn = r->logn; c->N = r->N; c->L = r->L; c->K = r->K;
    c->dnum = r->dnum; c->alpha = r->alpha; c->np = r->np;
    c->primes = r->primes; c->psi = r->psi; c->kp = r->kp;
    c->d_tables = r->d_tables;
    c->h_qinv = r->h_qinv; c->h_mu = r->h_mu; c->h_r2 = r->h_r2;
    c->modup = r->modup; c->moddown = r->moddown;
    c->pinv = r->pinv; c->pinv_s = r->pinv_s; c->pmod = r->pmod;
    c->d_consts = r->d_consts;
    c->d_s = r->d_s;
    c->key_stream = parent->key_stream;
    c->ntt_form = parent->ntt_form;
    c->small_primes = parent->small_primes;
    c->parent = r;
    const size_t ext = (size_t)(c->L + 1 + c->K) * c->n;
    int rc = c->sc_digits.ensure((size_t)c->dnum * ext);
    if (rc == HE_OK) rc = c->sc_u.ensure(2 * ext);
    if (rc == HE_OK) rc = c->sc_conv.ensure(2 * (size_t)(c->L + 1) * c->n);
    if (rc == HE_OK) rc = c->sc_tmp.ensure(3 * ext);
    if (rc == HE_OK) rc = c->sc_tmp2.ensure(ext);
    if (rc == HE_OK && (he_malloc(&c->d_err, sizeof(int)) != cudaSuccess ||
                        cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess)) {
        cudaGetLastError();
        c->d_err = nullptr;
        rc = HE_ENOMEM;
    }
    if (rc != HE_OK) { free_ctx(c); return rc; }
    *out = c;
    return HE_OK;
}

extern "C" int he_ctx_check(he_ctx *c, void *stream) {
    if (!c) { he_set_error("null context"); return HE_EINVAL; }
    HE_CHECK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    HE_CHECK_CUDA(cudaGetLastError());
    int e = 0;
    HE_CHECK_CUDA(cudaMemcpy(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        cudaMemset(c->d_err, 0, sizeof(int));
        he_set_error("a bounded device wait gave up (key-tile pipeline); results of the work since "
                     "the last check are invalid");
        return HE_ETIMEOUT;
    }
    return HE_OK;
}

extern "C" int he_selftest_bounded_wait(he_ctx *c, void *stream) {
    if (!c) { he_set_error("null context"); return HE_EINVAL; }
    return k_selftest_bounded_wait(c, (cudaStream_t)stream);
}

extern "C" int he_ctx_set_option(he_ctx *c, int option, int value) {
    if (!c) { he_set_error("null context"); return HE_EINVAL; }
    if (option == HE_OPT_PDL && (value == 0 || value == 1)) {
        he_set_pdl(value);
        return HE_OK;
    }
    if (option == HE_OPT_KEY_STREAM &&
        (value == HE_KEY_STREAM_LDG || value == HE_KEY_STREAM_TMA || value == HE_KEY_STREAM_AUTO ||
         value == HE_KEY_STREAM_SPLIT || value == HE_KEY_STREAM_CP || value == HE_KEY_STREAM_LDG1 ||
         value == HE_KEY_STREAM_PK || value == HE_KEY_STREAM_PK3 || value == HE_KEY_STREAM_PKP ||
         value == HE_KEY_STREAM_SPLITM || value == HE_KEY_STREAM_PK1 ||
         value == HE_KEY_STREAM_PKT || value == HE_KEY_STREAM_PK3L)) {
        c->key_stream = value;
        return HE_OK;
    }
    if (option == HE_OPT_NTT && (value == HE_NTT_ONEPASS || value == HE_NTT_TWOPASS || value == HE_NTT_ONEPASS8 ||
                                 value == HE_NTT_TWOPASS_CORRECTED || value == HE_NTT_TWOPASS_SHUFFLE)) {
        c->ntt_form = value;
        return HE_OK;
    }
    he_set_error("he_ctx_set_option: unknown option %d or value %d", option, value);
    return HE_EINVAL;
}

extern "C" int he_ctx_get_option(const he_ctx *c, int option, int *value) {
    if (!c || !value) { he_set_error("he_ctx_get_option: null argument"); return HE_EINVAL; }
    if (option == HE_OPT_KEY_STREAM) { *value = c->key_stream; return HE_OK; }
    if (option == HE_OPT_PDL) { *value = he_get_pdl(); return HE_OK; }
    if (option == HE_OPT_NTT) { *value = c->ntt_form; return HE_OK; }
    he_set_error("he_ctx_get_option: unknown option %d", option);
    return HE_EINVAL;
}

void he_tune_note(he_ctx *c, const std::string &line) {
    he_ctx *r = c->root();
    std::lock_guard<std::mutex> lk(r->tune_mu);
    r->tune_log.push_back(line);
}

extern "C" size_t he_ctx_tuning_log(const he_ctx *cc, char *buf, size_t cap) {
    if (!cc) return 0;
    he_ctx *r = const_cast<he_ctx *>(cc)->root();
    std::lock_guard<std::mutex> lk(r->tune_mu);
    std::string all;
    for (auto &l : r->tune_log) all += l + "\n";
    if (buf && cap) {
        const size_t m = std::min(cap - 1, all.size());
        memcpy(buf, all.data(), m);
        buf[m] = 0;
    }
    return all.size();
}

// ================================================================================ graphs
struct he_graph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t e = nullptr;
    uint64_t kernels = 0;
};

extern "C" int he_graph_begin(he_ctx *c, void *stream) {
    if (!c) { he_set_error("null context"); return HE_EINVAL; }
    if (g_capturing) { he_set_error("he_graph_begin: already capturing"); return HE_ESTATE; }
    if (!stream || stream == (void *)cudaStreamLegacy || stream == (void *)cudaStreamPerThread) {
        he_set_error("he_graph_begin: the default stream cannot be captured; use a created stream");
        return HE_EINVAL;
    }
    HE_CHECK_CUDA(cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeThreadLocal));
    g_capturing = true;
    g_captured = 0;
    g_capture_failed = false;
    return HE_OK;
}

extern "C" int he_graph_end(he_ctx *c, void *stream, he_graph **out) {
    if (!c || !out) { he_set_error("he_graph_end: null argument"); return HE_EINVAL; }
    if (!g_capturing) { he_set_error("he_graph_end: not capturing"); return HE_ESTATE; }
    g_capturing = false;
    const uint64_t captured = g_captured;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture((cudaStream_t)stream, &g);
    if (e != cudaSuccess || !g) {
        cudaGetLastError();
        he_set_error("he_graph_end: capture failed (%s); a call inside it was not capturable",
                     cudaGetErrorString(e));
        if (g) cudaGraphDestroy(g);
        return HE_ECUDA;
    }
    if (g_capture_failed) {
        cudaGraphDestroy(g);
        he_set_error("he_graph_end: a call during the capture failed (see its error); graph discarded");
        return HE_ESTATE;
    }
    he_graph *h = new he_graph();
    h->g = g;
    h->kernels = captured;
    if (cudaGraphInstantiate(&h->e, g, 0) != cudaSuccess ||
        cudaGraphUpload(h->e, (cudaStream_t)stream) != cudaSuccess) {   // first launch pays no upload
        cudaGetLastError();
        if (h->e) cudaGraphExecDestroy(h->e);
        cudaGraphDestroy(g);
        delete h;
        he_set_error("he_graph_end: instantiation failed");
        return HE_ECUDA;
    }
    *out = h;
    return HE_OK;
}

extern "C" int he_graph_launch(he_graph *h, void *stream) {
    if (!h) { he_set_error("null graph"); return HE_EINVAL; }
    HE_CHECK_CUDA(cudaGraphLaunch(h->e, (cudaStream_t)stream));
    g_launches += h->kernels;
    return HE_OK;
}

extern "C" uint64_t he_graph_kernels(const he_graph *h) { return h ? h->kernels : 0; }

extern "C" void he_graph_destroy(he_graph *h) {
    if (!h) return;
    if (h->e) cudaGraphExecDestroy(h->e);
    if (h->g) cudaGraphDestroy(h->g);
    delete h;
}

// ================================================================================ ciphertexts
extern "C" int he_ct_alloc(he_ctx *c, int level, he_ct **out) {
    if (!c || !out || level < 0 || level > c->L) { he_set_error("he_ct_alloc: bad argument"); return HE_EINVAL; }
    he_ct *ct = new he_ct();
    ct->ctx = c;
    ct->cap = ct->level = level;
    ct->pstride = (size_t)(level + 1) * c->n;
    if (he_capturing()) { delete ct; return he_capture_guard("ciphertext allocation"); }
    if (he_alloc_should_fail() || he_malloc(&ct->d, 2 * ct->pstride * 8) != cudaSuccess) {
        cudaGetLastError();
        delete ct;
        he_set_error("ciphertext allocation failed");
        return HE_ENOMEM;
    }
    ct->scale = c->pr.scale;
    *out = ct;
    return HE_OK;
}

extern "C" long long he_ct_check_range(he_ctx *c, const he_ct *ct, void *stream) {
    if (!c || !ct || ct->ctx != c || !ct->d) { he_set_error("he_ct_check_range: bad argument"); return HE_EINVAL; }
    HE_TRY(he_capture_guard("a range check"));
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *bad = (unsigned long long *)c->sc_tmp.p;   // one word of scratch
    HE_CHECK_CUDA(cudaMemsetAsync(bad, 0, 8, s));
    HE_TRY(k_range_check(c, ct->d, ct->pstride, ct->level, bad, s));
    unsigned long long h = 0;
    HE_CHECK_CUDA(cudaMemcpyAsync(&h, bad, 8, cudaMemcpyDeviceToHost, s));
    HE_CHECK_CUDA(cudaStreamSynchronize(s));
    return (long long)h;
}

extern "C" int he_ct_wrap(he_ctx *c, void *dev_ptr, size_t bytes, int level, he_ct **out) {
    if (!c || !out || !dev_ptr || level < 0 || level > c->L ||
        bytes < 2 * (size_t)(level + 1) * c->n * 8) {
        he_set_error("he_ct_wrap: bad argument");
        return HE_EINVAL;
    }
    he_ct *ct = new he_ct();
    ct->ctx = c;
    ct->cap = ct->level = level;
    ct->pstride = (size_t)(level + 1) * c->n;
    ct->d = (u64 *)dev_ptr;
    ct->owned = false;
    ct->scale = c->pr.scale;
    *out = ct;
    return HE_OK;
}

extern "C" void he_ct_free(he_ct *ct) {
    if (!ct) return;
    if (ct->owned && ct->d) he_free(ct->d);
    delete ct;
}
extern "C" int he_ct_level(const he_ct *ct) { return ct ? ct->level : HE_EINVAL; }
extern "C" double he_ct_scale(const he_ct *ct) { return ct ? ct->scale : 0.0; }
extern "C" int he_ct_set_scale(he_ct *ct, double s) {
    if (!ct) return HE_EINVAL;
    ct->scale = s;
    return HE_OK;
}
extern "C" void *he_ct_limb_ptr(const he_ct *ct, int k, int i) {
    if (!ct || k < 0 || k > 1 || i < 0 || i > ct->level) return nullptr;
    return ct->d + k * ct->pstride + (size_t)i * ct->ctx->n;
}

int ensure_ct(he_ctx *c, he_ct *ct, int level) {
    if (!ct || ct->ctx != c) { he_set_error("ciphertext from another context"); return HE_ESTATE; }
    if (level > ct->cap) { he_set_error("ciphertext capacity %d < level %d", ct->cap, level); return HE_ELEVEL; }
    ct->level = level;
    return HE_OK;
}

extern "C" int he_ct_copy(he_ct *dst, const he_ct *src, void *stream) {
    if (!dst || !src) { he_set_error("null argument"); return HE_EINVAL; }
    he_ctx *c = src->ctx;
    HE_TRY(ensure_ct(c, dst, src->level));
    HE_TRY(k_copy_limbs(dst->d, dst->pstride, src->d, src->pstride, (size_t)(src->level + 1) * c->n, 2,
                        (cudaStream_t)stream));
    dst->scale = src->scale;
    return HE_OK;
}

extern "C" int he_ct_drop_level(he_ct *ct, int level) {
    if (!ct || level < 0 || level > ct->level) { he_set_error("he_ct_drop_level: bad level"); return HE_ELEVEL; }
    ct->level = level;
    return HE_OK;
}

extern "C" int he_ct_import_coeffs(he_ct *ct, const uint64_t *host, int level, double scale,
                                   void *stream) {
    if (!ct || !host) { he_set_error("null argument"); return HE_EINVAL; }
    he_ctx *c = ct->ctx;
    HE_TRY(ensure_ct(c, ct, level));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t w = (size_t)(level + 1) * c->n;
    for (int k = 0; k < 2; k++)
        HE_CHECK_CUDA(cudaMemcpyAsync(ct->d + k * ct->pstride, host + k * w, w * 8, cudaMemcpyHostToDevice, s));
    HE_TRY(ntt_poly(c, ct->d, ct->pstride, 0, level + 1, level + 1, 2, false, s));
    ct->scale = scale;
    return HE_OK;
}

extern "C" int he_ct_export_coeffs(const he_ct *ct, uint64_t *host, void *stream) {
    if (!ct || !host) { he_set_error("null argument"); return HE_EINVAL; }
    he_ctx *c = ct->ctx;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t w = (size_t)(ct->level + 1) * c->n;
    u64 *tmp = c->sc_tmp.p;
    HE_TRY(k_copy_limbs(tmp, w, ct->d, ct->pstride, w, 2, s));
    HE_TRY(ntt_poly(c, tmp, w, 0, ct->level + 1, ct->level + 1, 2, true, s));
    HE_CHECK_CUDA(cudaMemcpyAsync(host, tmp, 2 * w * 8, cudaMemcpyDeviceToHost, s));
    HE_CHECK_CUDA(cudaStreamSynchronize(s));
    return HE_OK;
}

extern "C" int he_encrypt_coeffs(he_ctx *c, const int64_t *m, int level, double scale,
                                 uint64_t nonce, he_ct *out, void *stream) {
    if (!c || !m || !out) { he_set_error("null argument"); return HE_EINVAL; }
    HE_TRY(ensure_ct(c, out, level));
    cudaStream_t s = (cudaStream_t)stream;
    const int nq = level + 1;
    const size_t w = (size_t)nq * c->n;
    u64 *mres = c->sc_tmp.p, *e = mres + w;
    int64_t *tmp_i = (int64_t *)(e + w);
    HE_CHECK_CUDA(cudaMemcpyAsync(tmp_i, m, (size_t)c->n * 8, cudaMemcpyHostToDevice, s));
    HE_TRY(k_reduce_int(c, tmp_i, mres, nq, nq, false, s));
    HE_TRY(ntt_poly(c, mres, 0, 0, nq, nq, 1, false, s));
    u64 *a = out->d + out->pstride;
    HE_TRY(k_sample_uniform(c, c->pr.seed, (4ull << 56) | nonce, a, nq, nq, s));
    HE_TRY(ntt_poly(c, a, 0, 0, nq, nq, 1, false, s));
    HE_TRY(k_sample_cbd(c, c->pr.seed, (5ull << 56) | nonce, tmp_i, s));
    HE_TRY(k_reduce_int(c, tmp_i, e, nq, nq, false, s));
    HE_TRY(ntt_poly(c, e, 0, 0, nq, nq, 1, false, s));
    HE_TRY(k_encrypt_combine(c, out->d, a, e, mres, level, s));
    out->scale = scale;
    HE_CHECK_CUDA(cudaStreamSynchronize(s));
    return HE_OK;
}

extern "C" int he_encrypt(he_ctx *c, const double *slots, size_t n_slots, int level, double scale,
                          uint64_t nonce, he_ct *out, void *stream) {
    if (!c || !slots || n_slots != (size_t)c->N) { he_set_error("he_encrypt: need N slots"); return HE_EINVAL; }
    std::vector<int64_t> m(c->n);
    encode_slots(slots, c->n, scale, m.data());
    return he_encrypt_coeffs(c, m.data(), level, scale, nonce, out, stream);
}

extern "C" int he_decrypt(he_ctx *c, const he_ct *ct, double *slots, size_t n_slots, void *stream) {
    if (!c || !ct || !slots || n_slots != (size_t)c->N) { he_set_error("he_decrypt: need N slots"); return HE_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const int nl = ct->level >= 1 ? 2 : 1;
    u64 *tmp = c->sc_tmp.p;
    HE_TRY(k_decrypt_dot(c, ct, tmp, nl, s));
    HE_TRY(ntt_poly(c, tmp, 0, 0, nl, ct->level + 1, 1, true, s));
    std::vector<u64> h((size_t)nl * c->n);
    HE_CHECK_CUDA(cudaMemcpyAsync(h.data(), tmp, h.size() * 8, cudaMemcpyDeviceToHost, s));
    HE_CHECK_CUDA(cudaStreamSynchronize(s));
    std::vector<double> m(c->n);
    const u64 q0 = c->primes[0];
    if (nl == 1) {
        for (int j = 0; j < c->n; j++) {
            u64 v = h[j];
            m[j] = 2 * v > q0 ? -(double)(q0 - v) : (double)v;
        }
    } else {
        const u64 q1 = c->primes[1];
        const u64 q0inv = h_invmod(q0 % q1, q1);
        const u128 Q = (u128)q0 * q1;
        for (int j = 0; j < c->n; j++) {
            u64 a0 = h[j], a1 = h[c->n + j];
            u64 t = h_mulmod((a1 + q1 - a0 % q1) % q1, q0inv, q1);
            u128 x = (u128)a0 + (u128)q0 * t;               // in [0, q0 q1)
            m[j] = 2 * x > Q ? -(double)(Q - x) : (double)x;
        }
    }
    decode_coeffs(m.data(), c->n, ct->scale, slots);
    return HE_OK;
}

// ================================================================================ plaintexts
extern "C" int he_pt_import_coeffs(he_ctx *c, const int64_t *m, int level, double scale, he_pt **out) {
    if (!c || !m || !out || level < 0 || level > c->L) { he_set_error("he_pt_import_coeffs: bad argument"); return HE_EINVAL; }
    he_pt *pt = new he_pt();
    pt->ctx = c;
    pt->level = level;
    pt->scale = scale;
    const size_t w = (size_t)(level + 1) * c->n;
    if (he_malloc(&pt->d, w * 8) != cudaSuccess) {
        cudaGetLastError();
        delete pt;
        he_set_error("plaintext allocation failed");
        return HE_ENOMEM;
    }
    int64_t *tmp_i = (int64_t *)c->sc_tmp.p;
    int rc = upload_async(tmp_i, m, (size_t)c->n * 8, 0);
    if (rc == HE_OK) rc = k_reduce_int(c, tmp_i, pt->d, level + 1, level + 1, false, 0);
    if (rc == HE_OK) rc = ntt_poly(c, pt->d, 0, 0, level + 1, level + 1, 1, false, 0);
    if (rc == HE_OK) rc = k_to_mont(c, pt->d, level + 1, level + 1, 1, 0, 0);
    if (rc == HE_OK && cudaStreamSynchronize(0) != cudaSuccess) rc = HE_ECUDA;
    if (rc != HE_OK) {
        he_free(pt->d);
        delete pt;
        return rc;
    }
    *out = pt;
    return HE_OK;
}

extern "C" int he_pt_encode(he_ctx *c, const double *slots, size_t n_slots, int level, double scale,
                            he_pt **out) {
    if (!c || !slots || n_slots != (size_t)c->N) { he_set_error("he_pt_encode: need N slots"); return HE_EINVAL; }
    std::vector<int64_t> m(c->n);
    encode_slots(slots, c->n, scale, m.data());
    return he_pt_import_coeffs(c, m.data(), level, scale, out);
}

extern "C" void he_pt_free(he_pt *pt) {
    if (!pt) return;
    if (pt->d) he_free(pt->d);
    delete pt;
}

// ================================================================================ key switching
// x (NTT form, level l) -> D = ModUp(x): [beta][l+1+K][n] NTT form, own limbs copied.
static int modup_ntt(he_ctx *c, const u64 *x_ntt, int level, u64 *D, cudaStream_t s) {
    const int nq = level + 1;
    const size_t ext = (size_t)(nq + c->K) * c->n;
    u64 *xc = c->sc_tmp2.p;
    HE_TRY(k_copy_limbs(xc, 0, x_ntt, 0, (size_t)nq * c->n, 1, s));
    HE_TRY(ntt_poly(c, xc, 0, 0, nq, nq, 1, true, s));
    HE_TRY(k_modup(c, xc, x_ntt, D, level, s));
    const int beta = (nq + c->alpha - 1) / c->alpha;
    ntt_job j{D, ext, 0, nq + c->K, nq, c->alpha, beta};
    return k_ntt(c, j, false, s);
}

int hoist_modup(he_ctx *c, const he_ct *in, u64 *D, cudaStream_t s) {
    return modup_ntt(c, in->d + in->pstride, in->level, D, s);
}

// u = sum_j phi_g(D_j) ksk[j]; out = base[phi_gb] + ModDown(u)   (per-ciphertext launches)
int ks_tail(he_ctx *c, const u64 *D, int level, const DeviceKey &key, u64 g_apply,
                   const u64 *base, size_t base_pstride, int base_polys, u64 g_base, u64 *out,
                   size_t out_pstride, cudaStream_t s) {
    const int nq = level + 1;
    const size_t ext = (size_t)(nq + c->K) * c->n;
    ip_item it{D, key.d, c->sc_u.p, g_apply, (nq + c->alpha - 1) / c->alpha};
    md_item md{c->sc_u.p, c->sc_conv.p, base, base_pstride, base_polys, g_base, out, out_pstride};
    HE_TRY(k_inner_product_one(c, it, level, s));
    ntt_job jp{c->sc_u.p, ext, nq, c->K, nq, 0, 2};
    HE_TRY(k_ntt(c, jp, true, s));
    HE_TRY(k_moddown_fbc(c, c->sc_u.p, c->sc_conv.p, level, 2, s));
    ntt_job jc{c->sc_conv.p, (size_t)nq * c->n, 0, nq, nq, 0, 2};
    HE_TRY(k_ntt(c, jc, false, s));
    return k_moddown_combine_one(c, md, level, s);
}

int keyswitch_core(he_ctx *c, const u64 *d_ntt, int level, const DeviceKey &key, u64 g_apply,
                   const u64 *base, size_t base_pstride, int base_polys, u64 g_base, he_ct *out,
                   cudaStream_t s) {
    HE_TRY(modup_ntt(c, d_ntt, level, c->sc_digits.p, s));
    return ks_tail(c, c->sc_digits.p, level, key, g_apply, base, base_pstride, base_polys, g_base,
                   out->d, out->pstride, s);
}

extern "C" int he_rotate(he_ctx *c, const he_ct *in, int32_t r, he_ct *out, void *stream) {
    if (!c || !in || !out || in == out) { he_set_error("he_rotate: bad argument"); return HE_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    u64 g = h_galois(c, r);
    HE_TRY(ensure_ct(c, out, in->level));
    out->scale = in->scale;
    if (g == 1) return he_ct_copy(out, in, stream);
    const DeviceKey *key;
    HE_TRY(get_key(c, (int)g, &key));
    u64 *d = c->sc_tmp.p;
    HE_TRY(k_permute(c, in->d + in->pstride, d, in->level + 1, g, s));
    // non-hoisted: d = phi_g(c1) is raised; c0 enters the combine through phi_g
    return keyswitch_core(c, d, in->level, *key, 1, in->d, in->pstride, 1, g, out, s);
}

extern "C" int he_conjugate(he_ctx *c, const he_ct *in, he_ct *out, void *stream) {
    if (!c || !in || !out || in == out) { he_set_error("he_conjugate: bad argument"); return HE_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const u64 g = 2ull * c->n - 1;
    const DeviceKey *key;
    HE_TRY(get_key(c, (int)g, &key));
    HE_TRY(ensure_ct(c, out, in->level));
    out->scale = in->scale;
    u64 *d = c->sc_tmp.p;
    HE_TRY(k_permute(c, in->d + in->pstride, d, in->level + 1, g, s));
    return keyswitch_core(c, d, in->level, *key, 1, in->d, in->pstride, 1, g, out, s);
}

extern "C" int he_mul_monomial(he_ctx *c, he_ct *ct, int64_t e, void *stream) {
    if (!c || !ct || ct->ctx != c) { he_set_error("he_mul_monomial: bad argument"); return HE_EINVAL; }
    const int64_t two_n = 2 * (int64_t)c->n;
    const u64 ee = (u64)(((e % two_n) + two_n) % two_n);
    if (ee == 0) return HE_OK;
    return k_monomial(c, ct->d, ct->pstride, ct->level + 1, ee, (cudaStream_t)stream);
}

extern "C" int he_modraise(he_ctx *c, const he_ct *in, int level, he_ct *out, void *stream) {
    if (!c || !in || !out || in == out || in->ctx != c) { he_set_error("he_modraise: bad argument"); return HE_EINVAL; }
    if (in->level != 0 || level < 0 || level > c->L) {
        he_set_error("he_modraise: input at level %d (needs 0), target level %d", in->level, level);
        return HE_ELEVEL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    HE_TRY(ensure_ct(c, out, level));
    const size_t n = c->n;
    u64 *t = c->sc_tmp.p;                                   // [2][n]: c0, c1 mod q_0, coefficient form
    HE_TRY(k_copy_limbs(t, n, in->d, in->pstride, n, 2, s));
    ntt_job ji{t, n, 0, 1, 1, 0, 2};
    HE_TRY(k_ntt(c, ji, true, s));
    HE_TRY(k_modraise(c, t, out->d, out->pstride, level + 1, s));
    ntt_job jf{out->d, out->pstride, 0, level + 1, level + 1, 0, 2};
    HE_TRY(k_ntt(c, jf, false, s));
    out->scale = in->scale;
    return HE_OK;
}

extern "C" int he_rotate_hoisted(he_ctx *c, const he_ct *in, const int32_t *r, size_t n_r,
                                 he_ct **out, void *stream) {
    if (!c || !in || (!r && n_r) || (!out && n_r)) { he_set_error("he_rotate_hoisted: bad argument"); return HE_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    bool need = false;
    for (size_t i = 0; i < n_r; i++) {
        u64 g = h_galois(c, r[i]);
        if (g != 1) {
            const DeviceKey *k;
            HE_TRY(get_key(c, (int)g, &k));
            need = true;
        }
        if (out[i] == in) { he_set_error("he_rotate_hoisted: output aliases input"); return HE_EINVAL; }
    }
    if (need) HE_TRY(hoist_modup(c, in, c->sc_digits.p, s));
    for (size_t i = 0; i < n_r; i++) {
        u64 g = h_galois(c, r[i]);
        HE_TRY(ensure_ct(c, out[i], in->level));
        out[i]->scale = in->scale;
        if (g == 1) {
            HE_TRY(he_ct_copy(out[i], in, stream));
            continue;
        }
        const DeviceKey *key;
        HE_TRY(get_key(c, (int)g, &key));
        HE_TRY(ks_tail(c, c->sc_digits.p, in->level, *key, g, in->d, in->pstride, 1, g, out[i]->d,
                       out[i]->pstride, s));
    }
    return HE_OK;
}

// ================================================================================ arithmetic
extern "C" int he_ct_zero(he_ct *acc, int level, double scale, void *stream) {
    if (!acc) { he_set_error("null argument"); return HE_EINVAL; }
    HE_TRY(ensure_ct(acc->ctx, acc, level));
    acc->scale = scale;
    const size_t w = (size_t)(level + 1) * acc->ctx->n;
    HE_TRY(k_zero(acc->d, w, (cudaStream_t)stream));
    return k_zero(acc->d + acc->pstride, w, (cudaStream_t)stream);
}

extern "C" int he_mul_pt_acc(he_ctx *c, he_ct *acc, const he_ct *ct, const he_pt *pt, void *stream) {
    if (!c || !acc || !ct || !pt) { he_set_error("null argument"); return HE_EINVAL; }
    if (acc->level != ct->level || pt->level < ct->level) { he_set_error("he_mul_pt_acc: level mismatch"); return HE_ELEVEL; }
    mac_term t{pt->d, ct->d, ct->pstride};
    HE_TRY(k_mac_one(c, t, acc->d, acc->pstride, ct->level, true, (cudaStream_t)stream));
    acc->scale = ct->scale * pt->scale;
    return HE_OK;
}

extern "C" int he_rescale(he_ctx *c, he_ct *ct, void *stream) {
    if (!c || !ct) { he_set_error("null argument"); return HE_EINVAL; }
    const int l = ct->level;
    if (l < 1) { he_set_error("he_rescale: no level left"); return HE_ELEVEL; }
    cudaStream_t s = (cudaStream_t)stream;
    // top limb to coefficient form, its centred residues mod q_0..q_{l-1} to NTT form, then
    // c_i = (c_i - t_i) q_l^-1 (both polynomials, pstride apart)
    HE_TRY(k_rescale_many(c, ct->d, ct->pstride, 1, l, c->sc_tmp.p, s));
    ct->level = l - 1;
    ct->scale = ct->scale / (double)c->primes[l];
    return HE_OK;
}

int rescale_batch(he_ctx *c, he_ct *const *cts, int m, cudaStream_t s) {
    if (m <= 0) return HE_OK;
    const int l = cts[0]->level;
    for (int j = 0; j < m; j++)
        if (!cts[j] || cts[j]->ctx != c || cts[j]->level != l || l < 1) {
            he_set_error("rescale batch: ciphertexts at different levels or no level left");
            return HE_ELEVEL;
        }
    const int per = HE_NTT_TAB / 2;
    HE_TRY(c->sc_rs.ensure((size_t)2 * std::min(m, per) * l * c->n));
    for (int j0 = 0; j0 < m; j0 += per) {
        const int cnt = std::min(per, m - j0);
        u64 *polys[HE_NTT_TAB];
        for (int j = 0; j < cnt; j++) {
            polys[2 * j] = cts[j0 + j]->d;
            polys[2 * j + 1] = cts[j0 + j]->d + cts[j0 + j]->pstride;
        }
        HE_TRY(k_rescale_tab(c, polys, cnt, l, c->sc_rs.p, s));
    }
    for (int j = 0; j < m; j++) {
        cts[j]->level = l - 1;
        cts[j]->scale = cts[j]->scale / (double)c->primes[l];
    }
    return HE_OK;
}

// b may sit above acc's level: its limbs q_0..q_l are b at level l (dropping limbs is exact)
extern "C" int he_add(he_ctx *c, he_ct *acc, const he_ct *b, void *stream) {
    if (!c || !acc || !b || acc->level > b->level) { he_set_error("he_add: addend below the accumulator's level"); return HE_ELEVEL; }
    return k_add(c, acc, b, false, (cudaStream_t)stream);
}
extern "C" int he_sub(he_ctx *c, he_ct *acc, const he_ct *b, void *stream) {
    if (!c || !acc || !b || acc->level > b->level) { he_set_error("he_sub: operand below the accumulator's level"); return HE_ELEVEL; }
    return k_add(c, acc, b, true, (cudaStream_t)stream);
}

// exact integer held by a double -> residue mod q
bool int_residue(double v, u64 q, u64 *out) {
    if (!(std::fabs(v) < 1.7e38) || v != std::nearbyint(v)) return false;
    bool neg = v < 0;
    double a = neg ? -v : v;
    u128 x = (u128)a;
    u64 r = (u64)(x % q);
    *out = (neg && r) ? q - r : r;
    return true;
}

extern "C" int he_mul_int(he_ctx *c, he_ct *ct, double v, void *stream) {
    if (!c || !ct) { he_set_error("null argument"); return HE_EINVAL; }
    u64 res[64], sh[64];
    for (int i = 0; i <= ct->level; i++) {
        if (!int_residue(v, c->primes[i], &res[i])) { he_set_error("he_mul_int: not an exact integer"); return HE_EINVAL; }
        sh[i] = h_shoup(res[i], c->primes[i]);
    }
    return k_mul_scalar_v(c, ct, res, sh, 2, (cudaStream_t)stream);
}

extern "C" int he_add_const_int(he_ctx *c, he_ct *ct, double v, void *stream) {
    if (!c || !ct) { he_set_error("null argument"); return HE_EINVAL; }
    u64 res[64];
    for (int i = 0; i <= ct->level; i++)
        if (!int_residue(v, c->primes[i], &res[i])) { he_set_error("he_add_const_int: not an exact integer"); return HE_EINVAL; }
    return k_add_const_v(c, ct, res, (cudaStream_t)stream);
}

extern "C" int he_mul_relin(he_ctx *c, const he_ct *a, const he_ct *b, he_ct *out, void *stream) {
    if (!c || !a || !b || !out || a->level != b->level) { he_set_error("he_mul_relin: level mismatch"); return HE_ELEVEL; }
    if (a->level < 1) { he_set_error("he_mul_relin: no level left"); return HE_ELEVEL; }
    const DeviceKey *key;
    HE_TRY(get_key(c, 0, &key));
    cudaStream_t s = (cudaStream_t)stream;
    const int l = a->level;
    const size_t w = (size_t)(l + 1) * c->n;
    u64 *d = c->sc_tmp.p;                        // [3][l+1][n]
    HE_TRY(k_tensor(c, a, b, d, s));
    double sc = a->scale * b->scale;
    HE_TRY(ensure_ct(c, out, l));
    HE_TRY(keyswitch_core(c, d + 2 * w, l, *key, 1, d, w, 2, 1, out, s));
    out->scale = sc;
    return he_rescale(c, out, stream);
}

extern "C" int he_bench_mac(he_ctx *c, int blocks, int iters, double *rate) {
    if (!c || !rate || blocks <= 0 || iters <= 0) { he_set_error("bad argument"); return HE_EINVAL; }
    *rate = k_bench_mac(blocks, iters, 0);
    return *rate > 0 ? HE_OK : HE_ECUDA;
}

extern "C" int he_bench_modmul(he_ctx *c, int blocks, int iters, double *rate) {
    if (!c || !rate || blocks <= 0 || iters <= 0) { he_set_error("bad argument"); return HE_EINVAL; }
    *rate = k_bench_modmul(c, blocks, iters, 0);
    return *rate > 0 ? HE_OK : HE_ECUDA;
}
