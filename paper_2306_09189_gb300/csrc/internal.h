// Internal declarations shared by the hegpu translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <array>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/hegpu.h"

typedef uint64_t u64;
typedef unsigned __int128 u128;

// ----------------------------------------------------------------------------- errors
void he_set_error(const char *fmt, ...);
#define HE_CHECK_CUDA(expr)                                                        \
    do {                                                                           \
        cudaError_t _e = (expr);                                                   \
        if (_e != cudaSuccess) {                                                   \
            cudaGetLastError();  /* do not leave the error for a later launch check */ \
            he_set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr,                \
                         cudaGetErrorString(_e));                                  \
            return HE_ECUDA;                                                       \
        }                                                                          \
    } while (0)
#define HE_TRY(expr)                \
    do {                            \
        int _rc = (expr);           \
        if (_rc != HE_OK) return _rc; \
    } while (0)

void he_count_launch(int k = 1);
bool he_alloc_should_fail();             // test fault injection (he_debug_fail_alloc)
// Every device allocation of the library goes through these: the caller's allocator when one
// is installed (he_set_allocator), else cudaMalloc / cudaFree.  he_free(nullptr) is a no-op.
cudaError_t he_malloc(void **p, size_t bytes);
cudaError_t he_free(void *p);
template <class T>
inline cudaError_t he_malloc(T **p, size_t bytes) { return he_malloc((void **)p, bytes); }
void he_set_pdl(int on);                 // programmatic dependent launch of every kernel (process-wide)
int he_get_pdl();
// True while this thread is capturing a CUDA graph (he_graph_begin .. he_graph_end): no device
// allocation, synchronous copy or event timing may happen then.
bool he_capturing();
int he_capture_guard(const char *what);    // HE_ESTATE with a message when capturing

// Per-kernel tracing: while a kernel name is selected, every launch of that kernel is
// bracketed by CUDA events on its own stream and its algorithmic work is accumulated.
struct TraceScope {
    bool on = false;
    cudaStream_t s = 0;
    cudaEvent_t b = nullptr;
    double bytes = 0, mulmods = 0;
    TraceScope(const char *name, cudaStream_t st, double bytes_, double mulmods_);
    ~TraceScope();
};

// ----------------------------------------------------------------------------- tables
// Every table is indexed by the global prime index: q_0..q_L are 0..L, p_k is L+1+k.
struct KP {                  // kernel parameters passed by value
    int n, logn, L, K;
    const u64 *q;            // primes
    const u64 *qinv;         // q^{-1} mod 2^64 (Montgomery)
    const u64 *r2;           // 2^128 mod q (to Montgomery form)
    const u64 *mu;           // floor(2^64 / q) (64-bit Barrett)
    const u64 *tw, *tws;     // [np][n] psi^{brev(k)} and its Shoup companion
    const u64 *itw, *itws;   // [np][n] psi^{-brev(k)} and Shoup
    const u64 *ninv, *ninvs; // [np] n^{-1} and Shoup
    const u64 *tw2, *itw2;   // [np][n] interleaved {w, w'} pairs of tw/tws and itw/itws
};

// Fast-base-conversion table for one (source set -> target set) conversion.
struct FbcTable {
    int n_src, n_dst;
    u64 *d;                  // device: [n_src] inv_hat, [n_src] inv_hat_shoup,
                             //         [n_dst][n_src] hat (Montgomery), [n_dst][n_src] -hat (Mont)
    std::vector<int> src_prime, dst_prime;   // global prime indices
};

struct DeviceKey {           // hybrid key-switching key, Montgomery NTT form
    u64 *d = nullptr;        // [dnum][2][L+1+K][n]
    int id = 0;
};

struct Scratch {             // grow-only device scratch owned by the context
    u64 *p = nullptr;
    size_t words = 0;
    int ensure(size_t w);
    ~Scratch();
};

// ----------------------------------------------------------------------------- objects
struct he_ct {
    he_ctx *ctx = nullptr;
    u64 *d = nullptr;        // poly k, limb i at d + k*pstride + i*n   (NTT form)
    size_t pstride = 0;      // words between the two polynomials
    int cap = 0;             // allocated level
    int level = 0;
    double scale = 1.0;
    bool owned = true;
};

struct he_pt {
    he_ctx *ctx = nullptr;
    u64 *d = nullptr;        // [level+1][n], Montgomery NTT form
    int level = 0;
    double scale = 1.0;
};

struct he_ctx {
    he_params pr;
    int n, logn, N, L, K, dnum, alpha, np;
    std::vector<u64> primes;             // global order
    std::vector<u64> psi;                // primitive 2n-th roots
    KP kp;
    u64 *d_tables = nullptr;
    std::vector<u64> h_qinv, h_mu, h_r2;
    // ModUp tables: [level][digit]; ModDown tables: [level]
    std::vector<std::vector<FbcTable>> modup;
    std::vector<FbcTable> moddown;
    std::vector<u64> pinv, pinv_s;       // [L+1] P^{-1} mod q_i and Shoup
    std::vector<u64> pmod;               // [L+1] P mod q_i
    u64 *d_consts = nullptr;             // device copies of small per-level constant arrays
    // secret key (this library also plays the client, for tests and benchmarks)
    u64 *d_s = nullptr;                  // [L+1+K][n] NTT form, normal
    std::map<int, DeviceKey> keys;       // key id (Galois element; 0 = relin) -> key
    Scratch sc_digits, sc_u, sc_conv, sc_tmp, sc_tmp2;
    size_t key_bytes = 0;
    int *d_err = nullptr;                // set by a bounded device wait that gave up
    int key_stream = HE_KEY_STREAM_AUTO; // HE_OPT_KEY_STREAM
    int ntt_form = HE_NTT_TWOPASS;       // HE_OPT_NTT
    bool small_primes = false;           // every prime below 2^57 (forward NTT without corrections)
    std::mutex tune_mu;                  // root only: the autotuner's log
    // root only: pre-keyed tables (key (.) plaintext and [P]_q plaintext), shared by every
    // fork and stage that uses the same key and plaintext at the same levels; refcounted
    struct PkEntry { u64 *Kp = nullptr, *Ppt = nullptr; int refs = 0; };
    std::mutex pk_mu;
    std::map<std::array<uintptr_t, 4>, PkEntry> pk_cache;   // (key, plaintext, level, pt_level)
    std::vector<std::string> tune_log;
    he_ctx *parent = nullptr;            // forks share tables, secret and keys with their root
    he_ctx *root() { return parent ? parent : this; }
    const he_ctx *root() const { return parent ? parent : this; }
    std::vector<he_ct *> poly_tmp;       // reusable temporaries of he_poly_eval (level L), views
    u64 *poly_block = nullptr;           // one allocation holding them at a uniform stride
    Scratch sc_relin;                    // batched relinearisation buffers
    Scratch sc_rs;                       // batched rescales: the correction terms
};

#define HE_NTT_TAB 16
struct ntt_job {
    u64 *base;               // poly p, limb l at base + p*poly_stride + l*n
    size_t poly_stride;
    int l0, nl;              // limbs [l0, l0+nl) of each poly
    int nq;                  // limbs < nq use prime q_limb, limbs >= nq use p_(limb-nq)
    int skip_alpha;          // if > 0: in poly p skip limbs [j*skip_alpha, min((j+1)*skip_alpha, nq)),
                             // j = p mod skip_mod (j = p when skip_mod is 0)
    int npoly;
    int skip_mod;
    // optional: when tab[0] is set, poly p starts at tab[p] instead of base + p*poly_stride
    // (npoly <= HE_NTT_TAB): polynomials of ciphertexts at unrelated addresses in one launch
    u64 *tab[HE_NTT_TAB];
};

// ----------------------------------------------------------------------------- kernels
int k_ntt(const he_ctx *ctx, const ntt_job &job, bool inverse, cudaStream_t s);
int k_reduce_int(const he_ctx *ctx, const int64_t *m, u64 *out, int nlimbs, int nq, bool mont,
                 cudaStream_t s);
int k_to_mont(const he_ctx *ctx, u64 *x, int nlimbs, int nq, int npoly, size_t pstride,
              cudaStream_t s);
int k_from_mont(const he_ctx *ctx, u64 *x, int nlimbs, int nq, int npoly, size_t pstride,
                cudaStream_t s);
int k_sample_uniform(const he_ctx *ctx, u64 seed, u64 stream, u64 *out, int nlimbs, int nq,
                     cudaStream_t s);
int k_sample_cbd(const he_ctx *ctx, u64 seed, u64 stream, int64_t *out, cudaStream_t s);
int k_sample_ternary(const he_ctx *ctx, u64 seed, u64 stream, int64_t *out, cudaStream_t s);
int k_permute(const he_ctx *ctx, const u64 *in, u64 *out, int nlimbs, u64 g, cudaStream_t s);
// sparse ternary secret of weight h (perm: n words of scratch)
int k_sample_sparse(const he_ctx *ctx, u64 seed, u64 stream, int h, int32_t *perm, int64_t *out, cudaStream_t s);
// ModRaise: in_coef [2][n] coefficient form mod q_0 -> out [2][nlimbs][n] (poly stride pstride),
// coefficient form mod q_0..q_{nlimbs-1}
int k_modraise(const he_ctx *ctx, const u64 *in_coef, u64 *out, size_t pstride, int nlimbs, cudaStream_t s);
// both polynomials (NTT form, q-limbs 0..nlimbs-1) times X^e, 0 <= e < 2n
int k_monomial(const he_ctx *ctx, u64 *d, size_t pstride, int nlimbs, u64 e, cudaStream_t s);
int k_keygen_combine(const he_ctx *ctx, u64 *b, u64 *a, const u64 *e, const u64 *s_eval,
                     const u64 *sp_eval, int digit, cudaStream_t s);
int k_encrypt_combine(const he_ctx *ctx, u64 *c0, const u64 *a, const u64 *e, const u64 *m,
                      int level, cudaStream_t s);
int k_decrypt_dot(const he_ctx *ctx, const he_ct *ct, u64 *out, int nlimbs, cudaStream_t s);
int k_add(const he_ctx *ctx, he_ct *acc, const he_ct *b, bool sub, cudaStream_t s);
int k_mul_scalar(const he_ctx *ctx, he_ct *ct, const u64 *res /*device [l+1]*/, const u64 *shoup,
                 cudaStream_t s);
int k_add_const(const he_ctx *ctx, he_ct *ct, const u64 *res_dev, cudaStream_t s);
int k_zero(u64 *p, size_t words, cudaStream_t s);
int k_copy_limbs(u64 *dst, size_t dst_pstride, const u64 *src, size_t src_pstride,
                 size_t words_per_poly, int npoly, cudaStream_t s);

// Key switching.  D: [beta][level+1+K][n]; u: [2][level+1+K][n]; conv: [2][level+1][n].
int k_modup(const he_ctx *ctx, const u64 *x_coef, const u64 *x_ntt, u64 *D, int level,
            cudaStream_t s);
// ModUp of several sources at one level in three launch sets: gather every c1 (NTT form) into
// tmp [n_src][level+1][n], one INTT, one base-conversion launch writing each source's digits
// at its D ([beta][level+1+K][n], coefficient form except the digit's own limbs); the digits'
// forward NTT is the caller's (one job over all of them)
struct modup_src {
    const u64 *c1;          // source c1, NTT form, [level+1][n]
    u64 *D;                 // its raised digits
};
// the pre-keyed kernel's variants (public key-stream values)
#define HE_FORM_PK3 HE_KEY_STREAM_PK3
#define HE_FORM_PKP HE_KEY_STREAM_PKP
// K' = key (.) pt on the limbs of Q_level u P (key layout) and Ppt = [P]_q (.) pt on the q-limbs
int k_prekey(const he_ctx *ctx, const u64 *key, const u64 *pt, int level, int pt_level, int beta, u64 *Kp, u64 *Ppt,
             cudaStream_t s);
int k_modup_batch(const he_ctx *ctx, const modup_src *d_tab, int n_src, u64 *tmp, int level, cudaStream_t s);
// ModUp of m sources at fixed strides (coefficient form x_coef + i xs, NTT form x_ntt + i ns,
// digits D + i ds): one launch, no table
int k_modup_strided(const he_ctx *ctx, const u64 *x_coef, size_t xs, const u64 *x_ntt, size_t ns, u64 *D, size_t ds,
                    int m, int level, cudaStream_t s);
// tensor products (d0, d1, d2) of m pairs at one level into d + i dstride
int k_tensor_batch(const he_ctx *ctx, const he_ct *const *a, const he_ct *const *b, int m, u64 *d, size_t dstride,
                   int level, cudaStream_t s);
struct ip_item {            // one key-switching inner product
    const u64 *D;           // raised digits
    const u64 *key;         // key [dnum][2][L+1+K][n]
    u64 *u;                 // output [2][level+1+K][n]
    u64 g;                  // automorphism applied to D on the fly (1 = none)
    int beta;               // digits used at this level, ceil((level+1)/alpha)
};
int k_inner_product(const he_ctx *ctx, const ip_item *items_dev, int n_items, int level,
                    cudaStream_t s);
int k_moddown_fbc(const he_ctx *ctx, const u64 *u, u64 *conv, int level, int npoly,
                  cudaStream_t s);
struct md_item {            // out_c = base_c[phi_g] + (u_c - conv_c) * P^{-1}
    const u64 *u;           // [2][level+1+K][n]
    const u64 *conv;        // [2][level+1][n]
    const u64 *base;        // NULL or ct (poly 0 at base, poly 1 at base + base_pstride)
    size_t base_pstride;
    int base_polys;         // 1: add base to out0 only; 2: add to both
    u64 g;                  // automorphism on base reads (1 = none)
    u64 *out;               // ct data
    size_t out_pstride;
};
int k_moddown_combine(const he_ctx *ctx, const md_item *items_dev, int n_items, int level,
                      cudaStream_t s);
// ModDown fused with the rescale that follows it (m relinearised products, see kernels.cu)
int k_moddown_rescale(const he_ctx *ctx, u64 *u, const u64 *base, size_t b_is, size_t b_ps, u64 *w,
                      u64 *const *out, const size_t *out_ps, int m, int level, cudaStream_t s);
int k_range_check(const he_ctx *ctx, const u64 *d, size_t ps, int level, unsigned long long *bad, cudaStream_t s);
struct mac_term {
    const u64 *pt;          // [level+1][n] Montgomery
    const u64 *ct;          // ct data
    size_t ct_pstride;
};
int k_mac(const he_ctx *ctx, const mac_term *terms_dev, int n_terms, u64 *out, size_t out_pstride,
          int level, bool accumulate, cudaStream_t s);
int k_tensor(const he_ctx *ctx, const he_ct *a, const he_ct *b, u64 *d /*[3][l+1][n]*/,
             cudaStream_t s);
int k_inner_product_one(const he_ctx *ctx, const ip_item &it, int level, cudaStream_t s);
int k_moddown_combine_one(const he_ctx *ctx, const md_item &it, int level, cudaStream_t s);
// up to HE_INLINE_ITEMS items passed by value (no device table, no upload)
#define HE_INLINE_ITEMS 8
int k_inner_product_inline(const he_ctx *ctx, const ip_item *items, int n, int level, cudaStream_t s);
int k_moddown_combine_inline(const he_ctx *ctx, const md_item *items, int n, int level, cudaStream_t s);
int k_mac_one(const he_ctx *ctx, const mac_term &t, u64 *out, size_t out_pstride, int level,
              bool accumulate, cudaStream_t s);
int k_mul_scalar_v(const he_ctx *ctx, he_ct *ct, const u64 *res, const u64 *shoup, int polys,
                   cudaStream_t s);
int k_add_const_v(const he_ctx *ctx, he_ct *ct, const u64 *res, cudaStream_t s);
int k_mul_pointwise(const he_ctx *ctx, const u64 *a, const u64 *b, u64 *out, int nlimbs,
                    cudaStream_t s);
// Fused inner product + MAC in the raised basis (one ModDown per output afterwards).
// Amount-major form: every rotation key is read once and applied to every source shard that
// uses that amount.  A plaintext pointer equal to HE_PT_ONE stands for the integer 1.
#define HE_PT_ONE ((const u64 *)1)
struct famt {
    const u64 *key;         // null for amount 0
    u64 g;
    int e0, e1;             // entries [e0, e1)
};
struct fent {
    const u64 *D;           // the source's raised digits [beta][l+1+K][n], or null
    const u64 *src;         // the source's ciphertext data (c0, c1 at src + ps), level l
    size_t ps;
    const u64 *pt[2];       // per output of the group (V <= 2): plaintext, HE_PT_ONE or null
    int s;                  // source index (host bookkeeping)
};
// One group of a fused launch: V outputs of one item (an image's layer stage at level l).
// Plaintexts hold pt_level + 1 q-limbs then the K p-limbs, pt_level >= l, so one plaintext
// set encoded for the top level also serves items at every lower level.
struct fgrp {
    const famt *amts;
    const fent *ents;
    int n_amt, level, beta, pt_level;
    int nv;                 // outputs present in this group (<= V); only these are stored
    u64 *acc;               // [2V][l+1+K][n]  raised-basis (folded) inner products x plaintexts
};
// One launch over n_grp groups (any mix of levels): the grid walks global primes, and the
// groups sharing a (coefficient tile, prime) are adjacent in launch order, so each key and
// plaintext word is fetched from DRAM once and served to the other groups from L2.
// form: HE_KEY_STREAM_LDG or HE_KEY_STREAM_TMA (TMA needs beta <= 4 in every group).
int k_ipmac(const he_ctx *ctx, const fgrp *grps_dev, int n_grp, int V, int max_beta, double bytes,
            double mulmods, int form, int gb, cudaStream_t s);       // gb: groups per batch (0: all)   // acc only: the base folds in (see kernels.cu)
// Split form of a fused stage (same bits): (1) the raised inner product of every (source,
// amount), with [P]_q phi_a(c0) folded into its first polynomial (and [P]_q (c0, c1) for
// amount 0), is written to HBM once (amount-major: each key read once per launch); then
// (2) a raised-basis MAC forms sum pt (.) U over Q u P for HE_RV outputs per pass.  Cheaper
// than the fused kernel when many output groups would each recompute the inner products.
#define HE_RV 8
struct uent {
    const u64 *D;           // the source's raised digits (keyed amounts)
    u64 *U;                 // output [2][l+1+K][n]
    const u64 *src;         // the source ciphertext (c0, c1 at src + ps)
    size_t ps;
    u64 g;                  // Galois element of the entry's amount (1 for amount 0)
};
struct ugrp {               // inner products of one stage (one image at one level)
    const famt *amts;       // amounts (key null for amount 0); entries index uent, in order
    const uent *ents;
    int n_amt, n_ent, level, beta;
};
struct rterm {
    const u64 *U;           // folded raised inner product of (s, a)
    const u64 *pt[HE_RV];   // per output of the group: plaintext, HE_PT_ONE or null
};
struct rgrp {               // HE_RV outputs of one stage
    const rterm *terms;
    int n_terms, level, pt_level;
    int nv;                 // outputs present in this group (<= HE_RV); only these are stored
    int accumulate;         // add to acc (mod q) instead of overwriting: later amount chunks
    u64 *acc;               // [2 HE_RV][l+1+K][n]
};
// Image-batched raised MAC: HE_RNI stages (images of one batch, same plan, any levels) and
// HE_RVM outputs per pass, so each plaintext word is read once for every image.
#define HE_RVM 4
#define HE_RNI 4
struct rterm_m {
    const u64 *U[HE_RNI];   // the term's inner product in each image (null: image absent)
    const u64 *pt[HE_RVM];  // per output: plaintext, HE_PT_ONE or null
};
struct rgrp_m {
    const rterm_m *terms;
    int n_terms, ni, pt_level, nv, accumulate;
    int level[HE_RNI];
    u64 *acc[HE_RNI];       // per image: [2 HE_RVM][level+1+K][n] at the group's first output
};
int k_rmac_m(const he_ctx *ctx, const rgrp_m *grps, int n_grp, double bytes, double mulmods, cudaStream_t s);
int k_ip_amounts(const he_ctx *ctx, const ugrp *grps_dev, int n_grp, int max_beta, double bytes, cudaStream_t s);
int k_rmac(const he_ctx *ctx, const rgrp *grps_dev, int n_grp, double bytes, double mulmods, cudaStream_t s);
void he_tune_note(he_ctx *ctx, const std::string &line);
// factored channel-shard conv, stage 2 (see kernels.cu); Y ct j at Y + j ystride, poly c at + c yps
int k_smac(const he_ctx *ctx, const u64 *Y, size_t ystride, size_t yps, const u64 *Wm, int co, int ci, int H, int T,
           int level, u64 *out, size_t ostride, size_t ops, cudaStream_t s);
int k_selftest_bounded_wait(const he_ctx *ctx, cudaStream_t s);
#define HE_LC_MAX 20        // terms of one k_lincomb launch
#define HE_LC_LIMBS 24      // limbs of one k_lincomb launch (residue table row length)
int k_lincomb(const he_ctx *ctx, const u64 *const *x, const size_t *ps, const u64 *res, int n,
              const u64 *cst, int level, u64 *out, size_t out_ps, cudaStream_t s);
// Rescale of m ciphertexts at one level, poly p of ciphertext i at base + (2i + p) ps, in place;
// t is scratch of 2 m level n words.  Every rescale goes through here (he_rescale with m = 1).
int k_rescale_many(const he_ctx *ctx, u64 *base, size_t ps, int m, int level, u64 *t, cudaStream_t s);
int k_rescale_tab(const he_ctx *ctx, u64 *const *polys, int m, int level, u64 *t, cudaStream_t s);
// Rescales m ciphertexts of one level as he_rescale does each (same words, same scales), with one
// launch set per HE_NTT_TAB / 2 of them.
int rescale_batch(he_ctx *c, he_ct *const *cts, int m, cudaStream_t s);
// Loads the no-allocation rescale's module on the current device and caches its scratch address.
int he_noalloc_setup();
double k_bench_mac(int blocks, int iters, cudaStream_t s);
double k_bench_modmul(const he_ctx *ctx, int blocks, int iters, cudaStream_t s);

// ----------------------------------------------------------------------------- host helpers
u64 h_mulmod(u64 a, u64 b, u64 q);
u64 h_powmod(u64 a, u64 e, u64 q);
u64 h_invmod(u64 a, u64 q);
u64 h_shoup(u64 w, u64 q);
u64 h_galois(const he_ctx *ctx, int32_t r);
int prime_index(const he_ctx *ctx, int limb, int nq);   // limb of a Q_l u P polynomial -> prime
void encode_slots(const double *z, int n, double S, int64_t *m_out);
void encode_slots_complex(const double *re, const double *im, int n, double S, int64_t *m_out);
void decode_coeffs(const double *m, int n, double S, double *z_out);
int ensure_ct(he_ctx *ctx, he_ct *ct, int level);
bool int_residue(double v, u64 q, u64 *out);   // exact-integer double -> residue mod q
int keyswitch_core(he_ctx *ctx, const u64 *d_ntt, int level, const DeviceKey &key, u64 g_apply,
                   const u64 *base, size_t base_pstride, int base_polys, u64 g_base, he_ct *out,
                   cudaStream_t s);
int get_key(he_ctx *ctx, int key_id, const DeviceKey **out);
// IP + ModDown + combine for one rotation of the raised digits D (see context.cu)
int ks_tail(he_ctx *c, const u64 *D, int level, const DeviceKey &key, u64 g_apply,
            const u64 *base, size_t base_pstride, int base_polys, u64 g_base, u64 *out,
            size_t out_pstride, cudaStream_t s);
int k_add_raw(const he_ctx *ctx, u64 *a, size_t pa, const u64 *b, size_t pb, int nlimbs, int npoly,
              bool sub, cudaStream_t s);
int hoist_modup(he_ctx *ctx, const he_ct *in, u64 *D, cudaStream_t s);
int upload_async(void *dst, const void *src, size_t bytes, cudaStream_t s);
