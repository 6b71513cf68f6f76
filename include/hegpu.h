/*
 * hegpu -- homomorphic convolution and average pooling over RNS-CKKS ciphertexts that hold a
 * row-major packed image sharded across several ciphertexts, on one GB300 (sm_103a).
 *
 * Paper: "High-Resolution Convolutional Neural Networks on Homomorphically Encrypted Data via
 * Sharding Ciphertexts" (arXiv 2306.09189).  Sec. 2 fixes the scheme: RNS-CKKS over
 * R_Q = Z_Q[X]/(X^{2N}+1), N real slots per ciphertext, levels consumed by multiplications,
 * slot rotations.  Sec. 4 gives the layer algorithms (shift operator Eq. 1, partial
 * convolutions Eqs. 2-5, image shards Eq. 6, duplication/permutation metadata, channel
 * shards Eq. 7, pooling Eqs. 10-13); the Appendix the Chebyshev-basis activation.
 *
 * Conventions for every entry point
 *   - Return value: HE_OK (0) or a negative HE_E* code; he_last_error() gives a message
 *     (thread-local).  No C++ exception crosses this boundary.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Work is
 *     enqueued on it; host-pointer outputs are complete when the call returns.
 *   - Ring degree n = 2^log_n (the paper's 2N), N = n/2 slots.  Level l means primes
 *     q_0..q_l are live.  Ciphertexts live on the device in NTT form; the host exchange
 *     format is coefficient form, residues in [0, q_i), layout [2][l+1][n] uint64.
 *   - All ciphertext arithmetic is exact integer arithmetic mod the RNS primes (uint64
 *     limbs); floating point appears only in encoding and in scale bookkeeping.
 *   - One context is driven from one host thread and one stream at a time: the context owns
 *     the scratch buffers that key switching uses.
 *   - Device memory: the library allocates with cudaMalloc, or through the caller's allocator
 *     once he_set_allocator has installed one (for instance PyTorch's caching allocator);
 *     he_ct_wrap lets a caller hand in its own device buffer (a torch tensor's storage).
 */
#ifndef HEGPU_H
#define HEGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    HE_OK = 0,
    HE_EINVAL = -1,    /* bad argument, shape or layout */
    HE_ELEVEL = -2,    /* not enough levels left for the operation */
    HE_EKEY = -3,      /* a rotation or relinearisation key is missing */
    HE_ENOMEM = -4,    /* device or host allocation failed */
    HE_ETIMEOUT = -5,  /* a bounded device wait gave up */
    HE_ECUDA = -6,     /* CUDA runtime error */
    HE_ESTATE = -7     /* object used in the wrong state (e.g. wrong context) */
};

/* Execution modes of the layer programs.  HE_PLAIN and HE_BATCHED give identical bits (one
 * ModDown per rotation).  HE_FUSED moves the weighted sum of each output shard inside the
 * ModDown (inner product and plaintext MAC fused over Q u P, one ModDown per output shard);
 * it decrypts to the same layer with different bits. */
enum { HE_PLAIN = 0, HE_BATCHED = 1, HE_FUSED = 2 };
enum { HE_RELIN_KEY = 0x7fffffff };   /* key id of the relinearisation key in he_key_export */

typedef struct he_ctx he_ctx;
typedef struct he_ct he_ct;
typedef struct he_pt he_pt;
typedef struct he_conv he_conv;
typedef struct he_pool he_pool;
typedef struct he_linear he_linear;
typedef struct he_poly he_poly;

/* Scheme parameters (Sec. 2; the paper uses ring 2^16 and 59-bit scales, Sec. 5.3).
 * Prime rule: every prime = 1 mod 2n; primes of b bits are the largest such primes below
 * 2^b in descending order, drawn in the order q_0 (q0_bits), p_0..p_{n_p-1} (p_bits),
 * q_1..q_{n_q-1} (q_bits), each the next unused prime of its size.
 * Key switching is hybrid with dnum digits of alpha = ceil(n_q/dnum) primes; he_ctx_create
 * rejects sets whose special-prime product P is smaller than the largest digit modulus.
 * seed keys the counter-based SplitMix64 generator that draws the secret, key and
 * encryption randomness (stream ids in the design notes).  A sparse secret (secret_hw = h)
 * takes, for k < h, word 2k of stream 6 << 56 modulo n - k as the swap offset of step k and
 * word 2k + 1's low bit as its sign (1: -1). */
typedef struct {
    int log_n;       /* 9..17 */
    int n_q;         /* ciphertext primes, L = n_q - 1 */
    int n_p;         /* special primes K */
    int dnum;        /* key-switching digits */
    int q0_bits, q_bits, p_bits;   /* each in [20, 61] */
    double scale;    /* Delta */
    uint64_t seed;
    int secret_hw;   /* 0: uniform ternary secret; h in 1..n: sparse ternary secret with exactly
                        h coefficients +-1 (bootstrapping's modular reduction needs the small
                        |I| a sparse secret gives); drawn by a partial Fisher-Yates shuffle */
} he_params;

/* Image layout metadata (Sec. 4 "Sharding and Encrypting an Image", "Duplicating and
 * Permuting Channels").  Each channel's valid m x m pixels sit row-major in an M x M frame
 * (M = next power of two of m, row stride M).  A shard of N slots is cut into nb blocks of
 * B = min(M*M, N) slots; block b of shard u holds the frame rows [row0, row0 + B/M) of
 * channel chan[u*nb + b] (-1 = empty).  This single table expresses image shards, channel
 * shards, the duplication factor d and the pooling permutation tau. */
#define HE_MAX_BLOCKS 32768   /* N / 1 for N = 2^15 slots: any frame of a 2^16 ring */
typedef struct {
    int c, m, M, N, B;
    int n_shards, nb;
    int32_t chan[HE_MAX_BLOCKS];
    int32_t row0[HE_MAX_BLOCKS];
} he_layout;

const char *he_last_error(void);

/* Library build id and the number of kernels it launched so far (all contexts). */
const char *he_version(void);
uint64_t he_kernel_launches(void);

/* Host only, no GPU needed: the prime chain the rule above gives, q[n_q] and p[n_p]. */
int he_params_primes(const he_params *params, uint64_t *q, uint64_t *p);

/* Host only: the initial layout of a c x m x m image over shards of N slots (no
 * permutation; one shard with tiled duplication when c M^2 <= N, image shards when
 * M^2 <= N < c M^2, channel shards of N/M rows when M^2 > N). */
int he_layout_image(int c, int m, int N, he_layout *out);

/* ------------------------------------------------------------------ device memory */
/* Caller-provided device allocator (the paper has no counterpart: this is how a host framework
 * that owns the GPU's memory, such as PyTorch's caching allocator, lends it to the library).
 * Once installed, every device block the library needs (tables, keys, ciphertexts, plaintexts,
 * scratch) comes from alloc(bytes, user), which returns a device pointer of the current device
 * aligned to at least 256 bytes, or NULL when it cannot (the library then reports HE_ENOMEM);
 * every block goes back through free_fn(ptr, user), after the library has synchronised the
 * device (the allocator may reuse the block on any stream at once).  Process-wide; both NULL
 * restores cudaMalloc / cudaFree.  HE_EINVAL if exactly one function is NULL; HE_ESTATE while
 * any block the library allocated is still live (destroy every context and object first), so
 * that a block is always returned to the allocator that made it.  Not during graph capture
 * (no allocation happens there).  The fixed scratch of he_rescale_noalloc is not affected. */
typedef void *(*he_device_alloc_fn)(size_t bytes, void *user);
typedef void (*he_device_free_fn)(void *ptr, void *user);
int he_set_allocator(he_device_alloc_fn alloc, he_device_free_fn free_fn, void *user);
/* Device blocks the library currently holds (from either allocator). */
int64_t he_live_allocations(void);

/* ------------------------------------------------------------------ context and keys */
int he_ctx_create(const he_params *params, he_ctx **out);
void he_ctx_destroy(he_ctx *ctx);
/* A context that shares everything read-only with `parent` (tables, secret, every key,
 * including keys generated later) but owns its own key-switching scratch, so that work on
 * several streams can proceed at once: one fork per concurrent stream.  Destroy forks
 * before their parent. */
int he_ctx_fork(he_ctx *parent, he_ctx **out);
/* Synchronise `stream` and report whether any bounded device wait of this context gave up
 * since the last check (HE_ETIMEOUT; the work since then is invalid) or a CUDA error
 * occurred (HE_ECUDA).  Clears the timeout flag. */
int he_ctx_check(he_ctx *ctx, void *stream);
/* Per-context tuning options (values are ints; a fork starts with its parent's values).
 * HE_OPT_KEY_STREAM selects how the fused key-switch + MAC kernel brings key words on chip:
 *   HE_KEY_STREAM_LDG (0): 16-byte vector loads straight into registers;
 *   HE_KEY_STREAM_TMA (1): cp.async.bulk copies into a double-buffered shared-memory tile,
 *     signalled by mbarriers with bounded waits (a wait that gives up is reported by
 *     he_ctx_check as HE_ETIMEOUT).  Used for up to 4 digits; otherwise the LDG form runs;
 *   HE_KEY_STREAM_LDG1 (5): vector loads with one coefficient per thread: fewer registers per
 *     thread, three blocks per SM;
 *   HE_KEY_STREAM_CP (4): every word of an (amount, source) item (key words, gathered digits,
 *     plaintexts, source words) copied by each thread with cp.async into its own shared-memory
 *     slots, two items ahead of the one it computes (no block barrier).  Up to 4 digits;
 *   HE_KEY_STREAM_PK (6): pre-keyed: for stages where every output takes at most one source
 *     per rotation amount, each amount's key is multiplied by the output's plaintext once
 *     (K (.) pt, built on first use; the key itself when the plaintext is 1), and the kernel
 *     accumulates sum_j D_j (K (.) pt)_j without per-amount reductions or a plaintext stream.
 *     Other stages fall back to the LDG form.  HE_KEY_STREAM_PK3 (7): the same kernel at three
 *     blocks per SM; HE_KEY_STREAM_PKP (8): at two blocks per SM with the next amount's key words
 *     requested before the current amount computes;
 *   HE_KEY_STREAM_PK1 (10): pre-keyed with one coefficient per thread (half the registers of
 *     the pair form, four blocks per SM);
 *   HE_KEY_STREAM_PKT (11): pre-keyed with the key tiles brought in by a producer warp through
 *     cp.async.bulk into a 3-stage ring; consumer warps release each stage on an mbarrier as
 *     soon as they hold its words (no block barrier); bounded waits as for HE_KEY_STREAM_TMA.
 *     Up to 4 digits, else the pair form runs.  Explicit selection only (measured slower);
 *   HE_KEY_STREAM_PK3L (12): HE_KEY_STREAM_PK3 with the key tiles of the amount two ahead
 *     requested into L2 by cp.async.bulk.prefetch (up to 4 digits); explicit selection only
 *     (measured slower);
 *   HE_KEY_STREAM_SPLITM (9): the split form with the raised MAC batched over the images of a
 *     mixed-level batch (he_conv_run_batch): each plaintext word is read once for up to 4 images
 *     x 4 outputs; a single image falls back to HE_KEY_STREAM_SPLIT;
 *   HE_KEY_STREAM_SPLIT (3): the split form: the raised inner product of every (source,
 *     amount) is written to HBM once (each key read once), then a raised-basis MAC forms the
 *     plaintext-weighted sums of 4 outputs per pass; amounts go in chunks of at most 2 GB of
 *     inner products.  Cheaper than the fused kernel when a stage has many output shards;
 *   HE_KEY_STREAM_AUTO (2, default): on the first run of each fused launch an autotuner times
 *     the eligible candidates (fused kernel: the LDG, TMA and LDG1 key streams x outputs per
 *     key pass; the pre-keyed forms and the split form, when device memory allows) and keeps the
 *     fastest (he_ctx_tuning_log lists them).  HE_KEY_STREAM_CP and HE_KEY_STREAM_SPLITM run
 *     only when selected explicitly.
 * Every choice gives the same bits.  Returns HE_EINVAL for an unknown option or value. */
#define HE_OPT_KEY_STREAM 1
#define HE_KEY_STREAM_LDG 0
#define HE_KEY_STREAM_TMA 1
#define HE_KEY_STREAM_AUTO 2
#define HE_KEY_STREAM_SPLIT 3
#define HE_KEY_STREAM_CP 4
#define HE_KEY_STREAM_LDG1 5
#define HE_KEY_STREAM_PK 6
#define HE_KEY_STREAM_PK3 7
#define HE_KEY_STREAM_PKP 8
#define HE_KEY_STREAM_SPLITM 9
#define HE_KEY_STREAM_PK1 10
#define HE_KEY_STREAM_PKT 11
#define HE_KEY_STREAM_PK3L 12
/* HE_OPT_PDL (0 default, or 1; process-wide, whichever context sets it): launch every kernel
 * with programmatic dependent launch, so each grid is set up while its predecessor on the
 * stream finishes (every kernel waits for the predecessor's writes before it reads).  Same
 * bits either way; on the graph-launched CIFAR-layer step it measured neutral. */
#define HE_OPT_PDL 2
/* HE_OPT_NTT selects the negacyclic NTT at n = 2^16: HE_NTT_ONEPASS (0) transforms each limb in
 * one launch on a cluster of 16 CTAs of 256 threads that exchange the limb's blocks through
 * distributed shared memory (the limb is read and written once); HE_NTT_ONEPASS8 (2) the same on
 * a cluster of 8 CTAs of 512 threads; HE_NTT_TWOPASS (1) runs a column pass and a row pass as
 * two launches with the limb going through memory in between (the default).  When every prime
 * of the context is below 2^57 the two-pass forward transform skips the per-butterfly
 * correction (values grow by at most 2q per stage and are reduced once at the end);
 * HE_NTT_TWOPASS_CORRECTED (3) keeps the correction in every butterfly; HE_NTT_TWOPASS_SHUFFLE
 * (4) does the row pass's two in-row transposes with warp shuffles instead of shared memory
 * (rings 2^12..2^16).  Same words in every form; smaller rings always take a two-pass form. */
#define HE_OPT_NTT 3
#define HE_NTT_ONEPASS 0
#define HE_NTT_TWOPASS 1
#define HE_NTT_ONEPASS8 2
#define HE_NTT_TWOPASS_CORRECTED 3
#define HE_NTT_TWOPASS_SHUFFLE 4
int he_ctx_set_option(he_ctx *ctx, int option, int value);
int he_ctx_get_option(const he_ctx *ctx, int option, int *value);
/* The autotuner's decisions so far (one line per tuned stage: the candidates' times and the
 * choice), NUL-terminated into buf[cap]; returns the length needed (excluding the NUL). */
size_t he_ctx_tuning_log(const he_ctx *ctx, char *buf, size_t cap);

/* CUDA graphs.  he_graph_begin starts capturing `stream` (thread-local capture mode); every
 * library call made on that stream by this thread until he_graph_end is recorded instead of
 * run.  Calls that would allocate device memory or synchronise (the first run of a layer,
 * encryption, export) fail with HE_ESTATE while capturing: run the step once before
 * capturing it.  Host-side ciphertext metadata (level, scale) is updated at capture time
 * exactly as a real run would, and a replay reproduces the captured device work bit for bit.
 * The stream must be a created stream (the default stream cannot be captured: HE_EINVAL).
 * he_graph_end returns the instantiated graph (caller owns it; he_graph_destroy frees it). */
typedef struct he_graph he_graph;
int he_graph_begin(he_ctx *ctx, void *stream);
int he_graph_end(he_ctx *ctx, void *stream, he_graph **out);
int he_graph_launch(he_graph *graph, void *stream);
/* Kernels one launch of the graph runs. */
uint64_t he_graph_kernels(const he_graph *graph);
void he_graph_destroy(he_graph *graph);

/* Failure-path self-test (no fault involved): launches one warp that waits, with the same
 * bound as the key-tile pipeline, on an mbarrier nothing arrives on.  The wait gives up after
 * 250 ms of wall time, records the timeout in the context's error word and returns; the next
 * he_ctx_check reports HE_ETIMEOUT and clears it, and the context stays usable. */
int he_selftest_bounded_wait(he_ctx *ctx, void *stream);

/* n, N, L, K, dnum, alpha; q[L+1] and p[K] when the pointers are non-NULL. */
int he_ctx_info(const he_ctx *ctx, int *n, int *slots, int *L, int *K, int *dnum, int *alpha,
                uint64_t *q, uint64_t *p);

/* Rotation keys for the left rotations rot[i] (slot j <- slot j + r; Galois element
 * 5^(r mod N) mod 2n).  Keys already present are skipped.  Device resident, Montgomery
 * NTT form, layout [dnum][2][L+1+K][n]. */
int he_keygen_rotations(he_ctx *ctx, const int32_t *rot, size_t n_rot);
/* Relinearisation key (switches s^2 to s). */
int he_keygen_relin(he_ctx *ctx);
/* Conjugation key: Galois element 2n - 1 (X -> X^-1 maps every slot to its complex
 * conjugate), the key bootstrapping's real/imaginary split needs. */
int he_keygen_conjugation(he_ctx *ctx);
int he_has_rotation_key(const he_ctx *ctx, int32_t rot);
/* Key in coefficient form, host layout [dnum][2][L+1+K][n]; rot = HE_RELIN_KEY for relin. */
int he_key_export(he_ctx *ctx, int32_t rot, uint64_t *host);
/* Total bytes of device-resident keys. */
size_t he_key_bytes(const he_ctx *ctx);

/* ------------------------------------------------------------------ ciphertexts */
int he_ct_alloc(he_ctx *ctx, int level, he_ct **out);
/* Device-side range sanitizer: the number of words of ct (both polynomials, limbs 0..level)
 * that are not below their prime (0 for a well-formed ciphertext); counts instead of
 * trapping.  Synchronises the stream; refused inside a graph capture (HE_ESTATE). */
long long he_ct_check_range(he_ctx *ctx, const he_ct *ct, void *stream);
/* Test hook, host side only: after `after` more successful device allocations the next one
 * fails with HE_ENOMEM (the hook then disarms); a negative value disarms it.  Lets tests drive
 * allocation failures without exhausting a shared GPU. */
int he_debug_fail_alloc(long after);
/* Wrap caller-owned device memory of at least 2*(level+1)*n*8 bytes (not freed by us). */
int he_ct_wrap(he_ctx *ctx, void *dev_ptr, size_t bytes, int level, he_ct **out);
void he_ct_free(he_ct *ct);
int he_ct_level(const he_ct *ct);
double he_ct_scale(const he_ct *ct);
int he_ct_set_scale(he_ct *ct, double scale);
/* Device pointer of limb i of polynomial k (k in {0,1}). */
void *he_ct_limb_ptr(const he_ct *ct, int k, int i);
int he_ct_copy(he_ct *dst, const he_ct *src, void *stream);
/* Drop the top limbs down to `level` (exact, no rescale). */
int he_ct_drop_level(he_ct *ct, int level);

/* Host coefficient form [2][level+1][n], residues in [0, q_i) -> device NTT form. */
int he_ct_import_coeffs(he_ct *ct, const uint64_t *host, int level, double scale, void *stream);
/* Device -> host coefficient form [2][level+1][n]. */
int he_ct_export_coeffs(const he_ct *ct, uint64_t *host, void *stream);

/* Secret-key encryption (test and client side; no security claim) of the integer message
 * polynomial m[n]: (c0, c1) = (-a s + e + m, a) over Q_level, randomness keyed by nonce. */
int he_encrypt_coeffs(he_ctx *ctx, const int64_t *m, int level, double scale, uint64_t nonce,
                      he_ct *out, void *stream);
/* Encode slots (canonical embedding, Sec. 2) at `scale`, then he_encrypt_coeffs. */
int he_encrypt(he_ctx *ctx, const double *slots, size_t n_slots, int level, double scale,
               uint64_t nonce, he_ct *out, void *stream);
/* Decrypt and decode N slots.  Exact while |c0 + c1 s| < q_0 q_1 / 2 coefficient-wise. */
int he_decrypt(he_ctx *ctx, const he_ct *ct, double *slots, size_t n_slots, void *stream);

/* ------------------------------------------------------------------ plaintexts */
/* Integer plaintext m[n] (coefficients) at `level`, stored for multiplication. */
int he_pt_import_coeffs(he_ctx *ctx, const int64_t *m, int level, double scale, he_pt **out);
int he_pt_encode(he_ctx *ctx, const double *slots, size_t n_slots, int level, double scale,
                 he_pt **out);
void he_pt_free(he_pt *pt);

/* ------------------------------------------------------------------ primitives */
/* Non-hoisted rotation by r (Sec. 4.1: a column shift is a rotation by 1, a row shift a
 * rotation by m): out = (phi_g(c0) + ModDown(u0), ModDown(u1)),
 * u = sum_j ModUp(phi_g(c1))_j * ksk_g[j].  out may not alias in. */
int he_rotate(he_ctx *ctx, const he_ct *in, int32_t r, he_ct *out, void *stream);
/* Hoisted rotations of one ciphertext by r[0..n_r-1]: ModUp(c1) once, then
 * u = sum_j phi_g(ModUp(c1)_j) * ksk_g[j] per amount ("computed once and cached", Sec. 4.1).
 * r = 0 copies.  out[i] must be allocated at in's level. */
int he_rotate_hoisted(he_ctx *ctx, const he_ct *in, const int32_t *r, size_t n_r, he_ct **out,
                      void *stream);
/* acc = 0 at `level` with the given scale. */
int he_ct_zero(he_ct *acc, int level, double scale, void *stream);
/* acc += ct (.) pt  (plaintext x ciphertext multiply-accumulate, Sec. 4.1: mask and kernel
 * weight merged on the plaintext side).  acc's scale becomes ct.scale * pt.scale. */
int he_mul_pt_acc(he_ctx *ctx, he_ct *acc, const he_ct *ct, const he_pt *pt, void *stream);
/* Drop q_l: c' = round(c / q_l) (centred representative of the top limb); scale /= q_l. */
int he_rescale(he_ctx *ctx, he_ct *ct, void *stream);
/* acc += b (he_sub: acc -= b) limb-wise.  b may sit at a higher level than acc: only its limbs
 * q_0..q_l are read, which is b dropped to acc's level (exact; the residual connection of a
 * ResNet block adds its input this way).  acc keeps its scale. */
int he_add(he_ctx *ctx, he_ct *acc, const he_ct *b, void *stream);
int he_sub(he_ctx *ctx, he_ct *acc, const he_ct *b, void *stream);
/* ct *= c for an integer c given as a double holding an exact integer (|c| < 2^127). */
int he_mul_int(he_ctx *ctx, he_ct *ct, double c, void *stream);
/* c0 += c (constant polynomial) for an exact-integer double c. */
int he_add_const_int(he_ctx *ctx, he_ct *ct, double c, void *stream);
/* Tensor, relinearise, rescale (levels must match; Appendix, Chebyshev evaluation). */
int he_mul_relin(he_ctx *ctx, const he_ct *a, const he_ct *b, he_ct *out, void *stream);
/* Slot-wise complex conjugate: phi_g with g = 2n - 1, then a non-hoisted key switch (needs
 * he_keygen_conjugation).  out may not alias in. */
int he_conjugate(he_ctx *ctx, const he_ct *in, he_ct *out, void *stream);
/* Both polynomials times X^e in Z_Q[X]/(X^n + 1), in place (any integer e, taken mod 2n;
 * X^n = -1).  Exact: no level, no noise.  Slot i is multiplied by zeta^(e g_i); e = n/2
 * multiplies every slot by the imaginary unit (g_i = 1 mod 4). */
int he_mul_monomial(he_ctx *ctx, he_ct *ct, int64_t e, void *stream);
/* ModRaise (bootstrapping's first step): a level-0 ciphertext read over Q_level, every
 * residue mod q_0 lifted to its centred representative in (-q_0/2, q_0/2].  The result
 * decrypts to t = m + q_0 I with |I| <= (||s||_1 + 1) / 2; scale unchanged.  out may not
 * alias in and must be allocated at `level` or above (HE_ELEVEL otherwise). */
int he_modraise(he_ctx *ctx, const he_ct *in, int level, he_ct *out, void *stream);

/* ------------------------------------------------------------------ layers (Sec. 4) */
/* Plan a stride-1 'same' convolution (cross-correlation, W[co][ci][kh][kw], bias[co] or
 * NULL) for an input image with layout `in` at `level`: the rotation set and the diagonal
 * plaintexts D_{u,v,a} that merge shift masks and kernel weights (Sec. 4.1 "combined
 * non-homomorphically"), encoded at scale q_level, plus the bias encoded at the output
 * scale in_scale.  stride 2 is the unstrided convolution followed by the top-left select
 * of the pooling program (Sec. 4.1, last paragraph of "With a Single Shard").
 * Rotation keys are not generated here: see he_conv_rotations. */
int he_conv_create(he_ctx *ctx, const he_layout *in, const double *W, const double *bias,
                   int co, int ci, int kh, int kw, int stride, int pad, int level,
                   double in_scale, he_conv **out);
/* The same convolution in the factored two-stage form for an input in channel shards (each
 * shard holds consecutive rows of one channel, channels in order; Sec. 4.1 "With Channel
 * Shards", Eq. 7): stage 1 forms Y_{f,h,t} = sum_{h'} B_{h,h',t} (.) rot_{a_t}(X_{f,h'}) with
 * binary masks B (own and neighbouring shard of tap t share the amount a_t) encoded at scale
 * q_level, and rescales; stage 2 weights them with the integer scalars round(w q_{level-1})
 * (round half away from zero), rescales, and adds the bias.  Two levels (four with stride 2)
 * instead of one, and at most 2 H T mask plaintexts (H shards per channel, T taps) instead of
 * co ci H T diagonals, which is what makes high-resolution channel-shard layers fit in HBM.
 * For this form he_conv_n_terms counts the masks and he_conv_export_plan returns, per mask,
 * u = source shard h', v = shard h, a = a_t and the mask; he_conv_import_plaintexts takes the
 * masks [n_masks][n] and the bias [n_out][n] (at level - 2).  Not available for batches and forks. */
int he_conv_create_factored(he_ctx *ctx, const he_layout *in, const double *W, const double *bias,
                            int co, int ci, int kh, int kw, int stride, int pad, int level,
                            double in_scale, he_conv **out);
/* The same convolution in baby-step giant-step form (double hoisting of the rotations of
 * Eqs. 2-7).  Every diagonal amount splits as a = r B + s: s the residue of a modulo the input
 * layout's block length B taken in [-B/2, B/2) (the tap's row/column shift), r the channel
 * offset in blocks (r m^2).  With a giant stride of k = giant_blocks blocks the baby amount is
 * t = (r mod k) B + s and the giant amount g = (r - r mod k) B.  Baby steps: S_{v,g} =
 * sum_{(u,t)} rot_{-g}(D_{u,v,a}) (.) rot_t(X_u), hoisted per input shard; giant steps:
 * out_v = sum_g rot_g(S_{v,g}), then one rescale and the bias.  Rotations drop from the
 * distinct a per input shard to the distinct t per input shard plus the distinct g per output
 * shard (16 duplicated channels, 3x3: 143 -> 23 at k = 1, 38 at k = 4); k = blocks per shard
 * gives every g = 0 (the diagonal rotation set).  giant_blocks = 0 picks k by a cost model of
 * key and digit streaming against the extra ModUps and ModDowns (logged in
 * he_ctx_tuning_log); otherwise it must be a power of two dividing the blocks per shard
 * (HE_EINVAL).  Same levels, plaintext count and output scale as he_conv_create; different
 * bits.  In HE_FUSED mode both steps are raised-basis stages (one ModDown per partial sum, one
 * per output); HE_PLAIN and HE_BATCHED give one hoisted rotation per partial sum.  Terms are
 * ordered by v, then g, u, t; he_conv_export_plan returns each term's (u, v, a = g + t) and
 * the unrotated diagonal D_{u,v,a}; he_conv_import_plaintexts takes the rotated diagonals
 * rot_{-g}(D) in that order. */
int he_conv_create_bsgs(he_ctx *ctx, const he_layout *in, const double *W, const double *bias,
                        int co, int ci, int kh, int kw, int stride, int pad, int level,
                        double in_scale, int giant_blocks, he_conv **out);
/* The giant stride (blocks) of a baby-step giant-step convolution; 0 for the other forms. */
int he_conv_bsgs_giant(const he_conv *conv);
void he_conv_destroy(he_conv *conv);
int he_conv_out_layout(const he_conv *conv, he_layout *out);
int he_conv_out_level(const he_conv *conv);
/* The select stage of a stride-2 convolution (Sec. 4.1 "Strided convolutions": the unstrided
 * convolution, then the pooling program of Sec. 4.2 with weights (1, 0, 0, 0) and no ones-
 * convolution, keeping the top-left pixel of every 2x2 window; masks of Eqs. 10-11 at weight
 * 1).  *out is borrowed: it belongs to `conv` and is destroyed with it.  Its masks can be read
 * with he_pool_n_masks and replaced with he_pool_import_plaintexts (horizontal masks at the
 * conv's output level, vertical one level lower), for instance by another encoder's integers.
 * HE_EINVAL for a stride-1 convolution. */
int he_conv_select_pool(const he_conv *conv, he_pool **out);
/* Distinct non-zero rotation amounts the plan needs (all stages); returns the count,
 * writes up to cap of them. */
int he_conv_rotations(const he_conv *conv, int32_t *amounts, size_t cap);
/* Key switches one run performs (distinct (input shard, nonzero amount) pairs of every stage,
 * including the stride-2 select); he_pool_keyswitches the same for a pooling layer. */
int64_t he_conv_keyswitches(const he_conv *conv);
/* Number of diagonal terms of the stride-1 stage and their (u, v, a) in plan order
 * (v, then u, then a ascending; BSGS form: v, then g, u, t); diag (optional) receives
 * [n_terms][N] doubles. */
int he_conv_n_terms(const he_conv *conv);
int he_conv_export_plan(const he_conv *conv, int32_t *u, int32_t *v, int32_t *a, double *diag);
/* Replace the plan's encoded plaintexts by caller-given integer polynomials (plan order,
 * [n_terms][n]) and bias plaintexts ([n_out][n]); used to run on plaintexts encoded
 * elsewhere, e.g. for bit-exact comparison.  The plan's pre-keyed tables (key x plaintext,
 * HE_KEY_STREAM_PK*) are rebuilt on its next run; forks share the plaintext memory but not
 * those tables, so import before forking (a fork made earlier keeps the old tables). */
int he_conv_import_plaintexts(he_conv *conv, const int64_t *terms, const int64_t *bias);
/* Run: out[v] (allocated by the caller at he_conv_out_level) for v < out layout n_shards.
 * mode HE_PLAIN = per-ciphertext launches; HE_BATCHED = every rotation of a stage in one
 * launch per kernel; these two give the same bits.  HE_FUSED = for each group of output
 * shards one kernel streams every rotation key once, forms the inner products and their
 * plaintext-weighted sums over Q u P in registers, then one ModDown per output shard. */
int he_conv_run(he_ctx *ctx, he_conv *conv, he_ct *const *in, he_ct **out, int mode,
                void *stream);
/* A batch of n_img images through one stride-1 convolution (Sec. 4.1 applied per image):
 * in[i * n_in + u] is shard u of image i, out[i * n_out + v] receives output shard v.  Each
 * image may sit at its own level l_i in 1..the layer's level (all its shards at one level and
 * scale): the plaintexts encoded for the layer's level serve every lower level, so image i's
 * output has scale in_scale_i * q_L' / q_{l_i} (L' = the layer's level) at level l_i - 1, and
 * its bias is encoded at that scale on first use (or imported, he_conv_import_bias).  In
 * HE_FUSED mode every image's key switches and MACs run in one fused-kernel launch (groups of
 * all images and levels side by side, each key read from DRAM once for the batch); HE_PLAIN
 * and HE_BATCHED run image by image.  Buffers are kept for the last level signature; a new
 * signature allocates (not allowed inside a graph capture). */
int he_conv_run_batch(he_ctx *ctx, he_conv *conv, he_ct *const *in, he_ct **out, int n_img, int mode,
                      void *stream);
/* Bias plaintexts ([n_out][n] integers) for images at `level` whose output scale is out_scale
 * (bit-exact comparison against another encoder). */
int he_conv_import_bias(he_conv *conv, int level, double out_scale, const int64_t *bias);

/* A copy of a convolution plan for another context of the same root (he_ctx_fork): it shares
 * the plan and the resident plaintexts, and owns its run buffers, so forks run concurrently
 * on their own streams.  Destroy forks before the original. */
int he_conv_fork(const he_conv *conv, he_ctx *ctx, he_conv **out);

/* ------------------------------------------------------------------ bootstrapping */
/* Restores the level of a level-0 ciphertext (Sec. 2: the level is restored through
 * bootstrapping; Sec. 5 tables: the Bootstrap rows, the largest cost of the paper's networks;
 * the paper runs OpenFHE's and does not define it).  This library's construction, in order:
 *   ModRaise (he_modraise to level L; scale set to q_0 K: slots hold t / (q_0 K));
 *   CoeffToSlot: the inverse of the encoding map U_ij = zeta^(g_i j) (slots z = U w for the
 *     complex coefficient vector w_j = t_j + i t_(j+N)), factored as the radix-2 butterfly
 *     stages 2 S_h^-1, h = N/2 .. 1 (twiddle exp(2 pi i (5^j mod 8h) / 8h)), merged into
 *     levels_cts levels; each level a baby-step giant-step product with its non-zero
 *     diagonals: a raised-basis stage with one ModDown per partial sum, a giant stage with
 *     one ModDown, one rescale (scale times 2^stages); output BR(w) / (q_0 K);
 *   retarget: times the integer round((Delta / 2) q_l / s), rescale (scale s k / q_l);
 *   split: c = conj(x); re = x + c, im = (x - c) X^(3n/2), both at twice the scale;
 *   EvalMod on re and im: cos(2 pi (K u - 1/4) / 2^r) as a degree-deg Chebyshev interpolant
 *     in u on [-1, 1] (Paterson-Stockmeyer, target scale Delta), then r double angles
 *     y <- 2 y^2 - 1: sin(2 pi t / q_0) ~ 2 pi m / q_0;
 *   re + im X^(n/2), scale times 2 pi Delta_in / q_0 (Delta_in: the input's scale), then
 *     times the integer round(Delta / s) (no level: the scale is about Delta again);
 *   SlotToCoeff: S_h, h = 1 .. N/2, merged into levels_stc levels the same way.
 * Levels used: levels_cts + 1 + (Paterson-Stockmeyer depth of deg) + r + levels_stc
 * (15 with the defaults); the output sits at L minus that, same slot values, scale within a
 * fraction of a percent of Delta (tracked exactly).
 * Needs K >= max |I| (|I| <= (h + 1) / 2 for a weight-h secret: he_params.secret_hw), and
 * q_0 / Delta_in large enough for sin(x) ~ x (2^10 gives about 2^-17 relative). */
typedef struct he_boot he_boot;
typedef struct {
    int K;            /* EvalMod domain [-K, K] (default 16) */
    int double_angle; /* r (default 2) */
    int deg;          /* Chebyshev degree of the cosine, 2..255 (default 59) */
    int levels_cts;   /* merged CoeffToSlot levels (default 3) */
    int levels_stc;   /* merged SlotToCoeff levels (default 3) */
} he_boot_config;
/* Plans the levels (diagonals, baby-step giant-step split), encodes the diagonals at scale
 * q_level over Q_level u P, and the cosine's coefficients.  cfg NULL or zero fields take the
 * defaults.  Keys are not generated: he_boot_rotations, he_keygen_conjugation, relin.  A plan
 * owns its temporaries: one bootstrap at a time per plan (and per context's scratch); the
 * first run also tunes the fused stages, so it allocates and must come before a graph
 * capture. */
int he_boot_create(he_ctx *ctx, const he_boot_config *cfg, he_boot **out);
void he_boot_destroy(he_boot *bt);
/* Distinct non-zero rotation amounts the linear levels use (count returned; amounts filled
 * up to cap). */
int he_boot_rotations(const he_boot *bt, int32_t *amounts, size_t cap);
/* Levels: the output level, the top level of CoeffToSlot / EvalMod input / SlotToCoeff, and
 * the key switches of one bootstrap (rotations, conjugation, relinearisations). */
int he_boot_info(const he_boot *bt, int *out_level, int *cts_level, int *evalmod_level, int *stc_level,
                 int *keyswitches);
/* Plaintexts of linear level idx of stage 0 (CoeffToSlot) or 1 (SlotToCoeff): their count,
 * and a replacement by caller-given integer polynomials ([count][n], giant index ascending,
 * then baby index ascending, at scale q_level) for a bit-exact comparison with another
 * encoder; he_boot_import_coeffs replaces the cosine's Chebyshev coefficients likewise. */
int he_boot_n_plaintexts(const he_boot *bt, int stage, int idx);
int he_boot_import_plaintexts(he_boot *bt, int stage, int idx, const int64_t *pts);
int he_boot_import_coeffs(he_boot *bt, const double *cheb, int deg);
/* One linear level on its own (for tests): in at the level's level, out one level lower. */
int he_boot_lintrans(he_ctx *ctx, he_boot *bt, int stage, int idx, const he_ct *in, he_ct *out, void *stream);
/* The whole bootstrap; out allocated at the output level or above (HE_ELEVEL otherwise).  A
 * level-0 input is taken at its scale; an input above level 0 is first brought to level 0 at
 * scale q_0 / 2^10 (dropped to level 1, times the integer round((q_0 / 2^10) q_1 / s),
 * rescaled), so a network can bootstrap wherever its levels run out. */
int he_bootstrap(he_ctx *ctx, he_boot *bt, const he_ct *in, he_ct *out, void *stream);
/* The bootstrap with its own error removed once more (the paper's Appendix, "Precision and
 * Bootstrapping Noise": MetaBTS, about twice the bits for one level and a second bootstrap):
 * c1 = bootstrap(in); the difference of c1 (brought back to level 0 at the input's scale) and
 * the input encrypts the bootstrap's error E; it is bootstrapped at 2^kb times its size
 * (kb in 0..30, 10 suits 2^-13 errors) and subtracted.  out (allocated at the bootstrap's
 * output level or above) receives c1 - E at one level below the bootstrap's output, c1's
 * scale. */
int he_bootstrap_meta(he_ctx *ctx, he_boot *bt, const he_ct *in, int kb, he_ct *out, void *stream);

/* ------------------------------------------------------------------ polynomial approximation (Appendix) */
/* Activation functions: GELU x Phi(x) (exact erf), ReLU, SiLU x / (1 + e^-x), Softplus. */
#define HE_FN_GELU 0
#define HE_FN_RELU 1
#define HE_FN_SILU 2
#define HE_FN_SOFTPLUS 3
/* Minimax (best uniform) polynomial of degree deg to activation fn on [lo, hi] by the Remez
 * exchange algorithm (the alternative to Chebyshev interpolation in the approximation table of
 * the Appendix): coeffs[0..deg] (caller-owned) receive c_k with p(x) = sum c_k T_k(t),
 * t = (2x - lo - hi)/(hi - lo), the form he_poly_eval / he_poly_eval_ps take; err (optional)
 * the levelled maximum error.  Host only (no device, no context).  HE_EINVAL for a bad
 * function id, deg outside 0..200 or hi <= lo; HE_ESTATE if the exchange degenerates. */
int he_cheb_minimax(int fn, int deg, double lo, double hi, double *coeffs, double *err);
/* Chebyshev interpolant of activation fn on [lo, hi] at the deg + 1 first-kind nodes (Appendix,
 * "Chebyshev Basis"; the interpolation rows of the approximation table): coeffs[0..deg]
 * (caller-owned) in the same form as he_cheb_minimax.  Host only.  HE_EINVAL for a bad function
 * id, deg outside 0..1000 or hi <= lo. */
int he_cheb_interp(int fn, int deg, double lo, double hi, double *coeffs);

/* ------------------------------------------------------------------ linear head (Sec. 4, Other Layers) */
/* Linear layer over a sharded image: output j = sum over the flattened (channel, row, column)
 * features of W[j][c][m][m] x feature, + bias[j] (bias NULL: 0).  Row j is placed on the first
 * copy (shard, then block order) of every valid pixel, so duplicated channels count once.
 * Evaluation: T_j = Rescale(sum_u w_{j,u} (.) X_u) with the weights at scale q_level 2^12; the
 * slot sum by rotate-and-add, T_j += rot_s(T_j) for s = N/2, ..., 1 (log2 N hoisted rotations per
 * output, every output's rotation by s in one fused launch); out = Rescale(sum_j e_j (.) T_j)
 * with one-hot masks e_j at scale q_{level-1} / 2^12, plus the bias in slots 0..n_out-1 (the
 * sum runs 2^12 above the input scale because each of its steps doubles the key-switch noise
 * before it; the output is at in_scale exactly).  The output
 * is one ciphertext at level - 2 (he_linear_out_level) and scale in_scale, out_j in slot j.
 * n_out <= N; level >= 2 (HE_ELEVEL).  Rotation keys: he_linear_rotations (the log2 N shifts). */
int he_linear_create(he_ctx *ctx, const he_layout *in, const double *W, const double *bias, int n_out,
                     int level, double in_scale, he_linear **out);
/* Pool-linear: every m x m channel averaged to one value and a linear layer W[n_out][c] applied,
 * fused as a linear layer whose weights are W[j][f] / m^2 on every pixel of channel f. */
int he_pool_linear_create(he_ctx *ctx, const he_layout *in, const double *W, const double *bias, int n_out,
                          int level, double in_scale, he_linear **out);
/* The same heads in packed form: with n' the smallest power of two >= n_out, the plaintexts
 * Q_{u,d}[i] = w_{i mod n', u}[(i + d) mod N] (d < n') make C = sum_{(u,d)} Q_{u,d} (.) rot_d(X_u)
 * (one raised-basis stage: n' - 1 hoisted rotations per shard, one ModDown) hold the terms of
 * output j = i mod n' around slot i; C += rot_s(C) for s = N/2, ..., n' sums each residue class
 * mod n', leaving out_j in slot j; then the first-n_out mask, rescale and bias as above.  Same
 * levels, scale and outputs; n_in (n' - 1) + log2(N/n') key switches instead of n_out log2 N;
 * different bits.  he_linear_import_plaintexts takes weights [n_in][n'][n] (the Q_{u,d}) and
 * one mask [n]. */
int he_linear_create_packed(he_ctx *ctx, const he_layout *in, const double *W, const double *bias, int n_out,
                            int level, double in_scale, he_linear **out);
int he_pool_linear_create_packed(he_ctx *ctx, const he_layout *in, const double *W, const double *bias,
                                 int n_out, int level, double in_scale, he_linear **out);
void he_linear_destroy(he_linear *lin);
int he_linear_rotations(const he_linear *lin, int32_t *amounts, size_t cap);
int he_linear_out_level(const he_linear *lin);
/* Key switches one run performs: n_out x log2 N. */
int64_t he_linear_keyswitches(const he_linear *lin);
/* Replace the encoded plaintexts by integer polynomials: weights [n_out][n_in_shards][n] at
 * scale q_level 2^12, masks [n_out][n] at scale q_{level-1} / 2^12, bias [n] at the output scale (each
 * optional, NULL keeps the encoded one). */
int he_linear_import_plaintexts(he_linear *lin, const int64_t *weights, const int64_t *masks,
                                const int64_t *bias);
/* Run on the input shards (level and scale as planned, else HE_ELEVEL); out is allocated by
 * the caller (any level; resized to level - 2). */
int he_linear_run(he_ctx *ctx, he_linear *lin, he_ct *const *in, he_ct *out, void *stream);

/* 2x2 average pool (Sec. 4.2): downsample (2x2 ones convolution, horizontal reduction
 * Eq. 10, vertical reduction Eq. 11), consolidate 4 shards into one (Eq. 12, channel order
 * permuted for image shards) or duplicate when 1-2 shards remain (Eq. 13).  Two levels. */
int he_pool_create(he_ctx *ctx, const he_layout *in, int level, he_pool **out);
void he_pool_destroy(he_pool *pool);
int he_pool_out_layout(const he_pool *pool, he_layout *out);
/* Fork of a pooling plan for another context of the same root (shares the mask plaintexts). */
int he_pool_fork(const he_pool *pool, he_ctx *ctx, he_pool **out);
int he_pool_rotations(const he_pool *pool, int32_t *amounts, size_t cap);
int64_t he_pool_keyswitches(const he_pool *pool);
/* Replace the mask plaintexts by caller-given integer polynomials: h [n_h][n_shards][n] for
 * the horizontal stage (column x' = 0, 1, ...) and v [n_v][n_shards][n] for the vertical
 * stage (rows y' whose mask is not empty), the order the plan uses. */
int he_pool_n_masks(const he_pool *pool, int *n_h, int *n_v);
int he_pool_import_plaintexts(he_pool *pool, const int64_t *h, const int64_t *v);
int he_pool_run(he_ctx *ctx, he_pool *pool, he_ct *const *in, he_ct **out, int mode,
                void *stream);

/* Chebyshev-basis polynomial sum_k c_k T_k(x) on a ciphertext holding x in [-1, 1]
 * (Appendix: T_{2k} = 2 T_k^2 - 1, T_{2k+1} = 2 T_k T_{k+1} - T_1, exact-scale constants).
 * Depth ceil(log2 deg) + 1; needs the relinearisation key.  io is replaced by the result
 * (scale `target_scale`, level lowered by the depth). */
int he_poly_eval(he_ctx *ctx, he_ct *io, const double *cheb, int deg, double target_scale,
                 void *stream);
/* The same polynomial on m ciphertexts (any levels; target_scales[m]): the ones at one level go
 * through the tree together, each tree depth one batched relinearisation for all of them.  Each
 * ciphertext gets exactly the bits he_poly_eval gives it. */
int he_poly_eval_many(he_ctx *ctx, he_ct *const *io, int m, const double *cheb, int deg,
                      const double *target_scales, void *stream);
/* The same polynomial by Paterson-Stockmeyer in the Chebyshev basis: baby steps T_1..T_k and
 * giant steps T_k, T_2k, ... (the binary-tree recursion), the division p = q T_G + r with
 * T_G T_j = (T_{G+j} + T_{|G-j|}) / 2, each node evaluated to a given level and scale (leaves as
 * exact-scale integer combinations).  Far fewer relinearised products than the tree (degree
 * 59: 16 instead of 58) and the paper's depths (degree 59 at 6, 27 at 5; Appendix).  The
 * output scale is target_scale up to the rounding of its own bookkeeping (a product node's
 * scale s_q s_G / q).  deg in 2..255.  Different bits from he_poly_eval, same polynomial. */
int he_poly_eval_ps(he_ctx *ctx, he_ct *io, const double *cheb, int deg, double target_scale, void *stream);
int he_poly_eval_ps_many(he_ctx *ctx, he_ct *const *io, int m, const double *cheb, int deg,
                         const double *target_scales, void *stream);
/* What he_poly_eval_ps costs for a degree-deg polynomial (the plan depends on the degree only):
 * *products = relinearised products (baby steps T_2..T_k, giant steps beyond T_k, one per
 * division with a non-constant quotient), *depth = levels consumed (degree 59: 16 products at
 * depth 6; 27: 11 at 5; 16: 8 at 5).  Host only.  HE_EINVAL for deg outside 2..255. */
int he_poly_ps_plan(int deg, int *products, int *depth);

/* One-call layers: plan, generate the missing rotation keys, run, synchronise the stream and
 * release the plan.  he_hconv2d is the paper's hconv2d (Sec. 4.1: shift operator Eq. 1, partial
 * convolutions Eqs. 2-5, image shards Eq. 6, channel shards Eq. 7; stride 2 as the unstrided
 * convolution plus the downsampling of Sec. 4.2) on the ciphertexts in_cts (all at one level and
 * scale; the plan is made at that level); he_havgpool is havgpool (Sec. 4.2, Eqs. 10-13: the 2x2
 * ones-convolution, horizontal and vertical reductions, consolidation or duplication).  W is
 * [co][ci][kh][kw], bias [co] or NULL.  out_cts: caller-allocated handles, one per output shard
 * of the output layout, allocated at the output level or above; out_layout (optional) receives that
 * layout.  The plaintexts are encoded by the library (within one integer per coefficient of any
 * other encoder of the same values), so the result decrypts to the layer; for bit-level control
 * of the plaintexts use he_conv_create / he_pool_create and their import calls. */
int he_hconv2d(he_ctx *ctx, const he_layout *in, he_ct *const *in_cts, const double *W,
               const double *bias, int co, int ci, int kh, int kw, int stride, int pad,
               int mode, he_layout *out_layout, he_ct **out_cts, void *stream);
int he_havgpool(he_ctx *ctx, const he_layout *in, he_ct *const *in_cts, he_layout *out_layout,
                he_ct **out_cts, int mode, void *stream);

/* Rescale without allocating anything: the same result as he_rescale, bit for bit, for
 * callers that must not allocate device memory after set-up (their device memory is owned
 * entirely by another allocator, or a memory cap forbids driver allocations).  The paper
 * has no counterpart; this is a property of this library's memory handling.
 * Its scratch is a fixed device array inside the library (24 MiB, 3 * 2^20 words), held on
 * every GPU that loads the library until the process exits; it rejects a ciphertext whose
 * 2 * level * n exceeds that with HE_EINVAL.  The array belongs to a module that CUDA may load
 * lazily; he_ctx_create loads it and looks up the array's device address (cudaGetSymbolAddress)
 * with the context's device current, so the array is reserved while the context is set up and
 * a later call allocates nothing.  (A call on a device that has no context yet does that look-up
 * itself: make it during set-up, before any stream capture.)  All calls share the one array and every call overwrites
 * it completely before reading it; calls whose work overlaps on the GPU (different streams,
 * or different host threads) race on it and must be serialised by the caller. */
int he_rescale_noalloc(he_ctx *ctx, he_ct *ct, void *stream);

/* ------------------------------------------------------------------ measurement */
/* Per-kernel tracing.  he_trace_start(name) selects one kernel (e.g. "ipmac", "ip", "ntt", "mac",
 * "modup", "moddown_fbc", "moddown_combine", "rescale"); every later launch of it is bracketed
 * by CUDA events recorded on the stream it is launched on.  he_trace_stop synchronises those
 * events and returns the summed device time, the launch count and the launches' algorithmic
 * work: minimal bytes (inputs + keys + outputs, intermediates excluded) and modular products.
 * Launches recorded into a CUDA graph while tracing get their events as external event-record
 * nodes: launch such a graph once before he_trace_stop (a later launch re-records them). */
int he_trace_start(const char *kernel);
int he_trace_stop(double *total_ms, uint64_t *launches, double *bytes, double *mulmods);

/* Time the integer pipe: `iters` dependent 64-bit Montgomery products per thread over
 * `blocks` x 256 threads; returns modular products per second (device-timed). */
int he_bench_modmul(he_ctx *ctx, int blocks, int iters, double *mulmods_per_s);
/* The integer pipe's throughput on the fused key-switch kernels' inner operation: `iters`
 * 64 x 64 -> 128-bit multiply-accumulates in each of 8 independent chains per thread over
 * `blocks` x 256 threads (on a 32-bit multiplier each is four 32 x 32 -> 64-bit partial
 * products and their carries); returns multiply-accumulates per second (device-timed). */
int he_bench_mac(he_ctx *ctx, int blocks, int iters, double *macs_per_s);

#ifdef __cplusplus
}
#endif
#endif
