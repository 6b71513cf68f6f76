/*
 * Plain CPU oracle for RNS-CKKS ring arithmetic (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load this
 * library.  It shares no code with the CUDA path.
 *
 * Every modular product is the literal definition (a*b) mod q through a 128-bit
 * integer and the C `%` operator; there is no Montgomery, Barrett or Shoup trick.
 * Polynomials are arrays of n uint64 words per RNS limb, limb-major.
 *
 * What each routine follows (the paper, Sec. 2 "Homomorphic encryption", states the
 * ring R_Q = Z_Q[X]/(X^{2N}+1); the internals below are the textbook RNS-CKKS
 * construction the paper relies on through OpenFHE):
 *   - orc_ntt / orc_intt: evaluation of a(X) at the odd powers psi^(2k+1) of a
 *     primitive 2n-th root psi, i.e. the negacyclic transform; written as
 *     "twist by psi^j, then a radix-2 cyclic transform with omega = psi^2".
 *   - orc_fbc: fast base conversion sum_i [x_i * (C/q_i)^-1]_{q_i} * (C/q_i) mod p.
 *   - orc_automorph_*: the Galois map X -> X^g used for slot rotation.
 *   - orc_rng: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used as a counter-based
 *     generator: output = mix(mix(seed ^ stream*gamma) + (idx+1)*gamma).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef unsigned __int128 u128;

static inline u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static inline u64 addmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + b) % q); }
static inline u64 submod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + q - (b % q)) % q); }

static u64 powmod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}
/* q prime: Fermat inverse */
static u64 invmod(u64 a, u64 q) { return powmod(a, q - 2, q); }

u64 orc_powmod(u64 a, u64 e, u64 q) { return powmod(a, e, q); }
u64 orc_mulmod(u64 a, u64 b, u64 q) { return mulmod(a, b, q); }

/* ---------------------------------------------------------------- PRNG */
static const u64 GAMMA = 0x9E3779B97F4A7C15ULL;

u64 orc_splitmix64_mix(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

u64 orc_rng(u64 seed, u64 stream, u64 idx) {
    u64 key = orc_splitmix64_mix(seed ^ (stream * GAMMA));
    return orc_splitmix64_mix(key + (idx + 1) * GAMMA);
}

/* ternary secret: word mod 3 -> {0, 1, -1} */
void orc_sample_ternary(u64 seed, u64 stream, int n, int64_t *out) {
    for (int j = 0; j < n; j++) {
        u64 r = orc_rng(seed, stream, (u64)j) % 3;
        out[j] = (r == 0) ? 0 : (r == 1 ? 1 : -1);
    }
}

/* centred binomial, eta = 21: popcount(low 21 bits) - popcount(next 21 bits) */
void orc_sample_cbd(u64 seed, u64 stream, int n, int64_t *out) {
    for (int j = 0; j < n; j++) {
        u64 r = orc_rng(seed, stream, (u64)j);
        int a = __builtin_popcountll(r & 0x1FFFFFULL);
        int b = __builtin_popcountll((r >> 21) & 0x1FFFFFULL);
        out[j] = (int64_t)a - (int64_t)b;
    }
}

/* uniform residue mod q for (limb_id, coefficient j): the 128-bit value hi*2^64+lo mod q,
   with lo = word 2*(limb_id*n+j), hi = word 2*(limb_id*n+j)+1 */
void orc_sample_uniform(u64 seed, u64 stream, int n, int nlimbs, const int *limb_id,
                        const u64 *q, u64 *out) {
    for (int l = 0; l < nlimbs; l++) {
        for (int j = 0; j < n; j++) {
            u64 base = 2 * ((u64)limb_id[l] * (u64)n + (u64)j);
            u64 lo = orc_rng(seed, stream, base);
            u64 hi = orc_rng(seed, stream, base + 1);
            u128 v = ((u128)hi << 64) | lo;
            out[(size_t)l * n + j] = (u64)(v % q[l]);
        }
    }
}

/* ---------------------------------------------------------------- NTT */
static void bitrev_permute(u64 *a, int n) {
    int logn = 0;
    while ((1 << logn) < n) logn++;
    for (int i = 0; i < n; i++) {
        int r = 0;
        for (int b = 0; b < logn; b++)
            if (i & (1 << b)) r |= 1 << (logn - 1 - b);
        if (i < r) { u64 t = a[i]; a[i] = a[r]; a[r] = t; }
    }
}

/* cyclic DFT over Z_q with primitive n-th root w, natural order in and out */
static void cyclic_ntt(u64 *a, int n, u64 q, u64 w) {
    bitrev_permute(a, n);
    for (int len = 2; len <= n; len <<= 1) {
        u64 wl = powmod(w, (u64)(n / len), q);
        for (int i = 0; i < n; i += len) {
            u64 wj = 1;
            for (int j = 0; j < len / 2; j++) {
                u64 u = a[i + j];
                u64 v = mulmod(a[i + j + len / 2], wj, q);
                a[i + j] = addmod(u, v, q);
                a[i + j + len / 2] = submod(u, v, q);
                wj = mulmod(wj, wl, q);
            }
        }
    }
}

/* out[k] = sum_j a[j] psi^((2k+1) j)  (evaluation at the odd powers of psi) */
static void ntt1(u64 *a, int n, u64 q, u64 psi) {
    u64 pj = 1;
    for (int j = 0; j < n; j++) { a[j] = mulmod(a[j], pj, q); pj = mulmod(pj, psi, q); }
    cyclic_ntt(a, n, q, mulmod(psi, psi, q));
}

/* inverse of ntt1 */
static void intt1(u64 *a, int n, u64 q, u64 psi) {
    u64 psi_inv = invmod(psi, q);
    cyclic_ntt(a, n, q, mulmod(psi_inv, psi_inv, q));
    u64 ninv = invmod((u64)n, q);
    u64 pj = ninv;
    for (int j = 0; j < n; j++) { a[j] = mulmod(a[j], pj, q); pj = mulmod(pj, psi_inv, q); }
}

void orc_ntt(u64 *a, int nlimbs, int n, const u64 *q, const u64 *psi) {
#pragma omp parallel for schedule(dynamic)
    for (int l = 0; l < nlimbs; l++) ntt1(a + (size_t)l * n, n, q[l], psi[l]);
}

void orc_intt(u64 *a, int nlimbs, int n, const u64 *q, const u64 *psi) {
#pragma omp parallel for schedule(dynamic)
    for (int l = 0; l < nlimbs; l++) intt1(a + (size_t)l * n, n, q[l], psi[l]);
}

/* ------------------------------------------------------- limb-wise arithmetic */
void orc_mul(const u64 *a, const u64 *b, u64 *out, int nlimbs, int n, const u64 *q) {
#pragma omp parallel for
    for (int l = 0; l < nlimbs; l++)
        for (int j = 0; j < n; j++) {
            size_t k = (size_t)l * n + j;
            out[k] = mulmod(a[k], b[k], q[l]);
        }
}

/* acc += a*b */
void orc_mac(u64 *acc, const u64 *a, const u64 *b, int nlimbs, int n, const u64 *q) {
#pragma omp parallel for
    for (int l = 0; l < nlimbs; l++)
        for (int j = 0; j < n; j++) {
            size_t k = (size_t)l * n + j;
            acc[k] = addmod(acc[k], mulmod(a[k], b[k], q[l]), q[l]);
        }
}

/* out = a * s_l for a per-limb scalar s_l */
void orc_mul_scalar(const u64 *a, const u64 *s, u64 *out, int nlimbs, int n, const u64 *q) {
#pragma omp parallel for
    for (int l = 0; l < nlimbs; l++)
        for (int j = 0; j < n; j++) {
            size_t k = (size_t)l * n + j;
            out[k] = mulmod(a[k], s[l] % q[l], q[l]);
        }
}

/* ------------------------------------------------------------------ FBC */
/* out[b] = sum_{i in C} [x_i * (C/q_i)^-1 mod q_i] * ((C/q_i) mod p_b) mod p_b,
   with every x_i a representative in [0, q_i).  C = prod qC, B = {qB}. */
void orc_fbc(const u64 *x, const u64 *qC, int nC, const u64 *qB, int nB, u64 *out, int n) {
    u64 *inv_hat = (u64 *)malloc(sizeof(u64) * nC);
    u64 *hat_mod_b = (u64 *)malloc(sizeof(u64) * nC * nB);
    for (int i = 0; i < nC; i++) {
        u64 h = 1;
        for (int k = 0; k < nC; k++) if (k != i) h = mulmod(h, qC[k] % qC[i], qC[i]);
        inv_hat[i] = invmod(h, qC[i]);
        for (int b = 0; b < nB; b++) {
            u64 hb = 1 % qB[b];
            for (int k = 0; k < nC; k++) if (k != i) hb = mulmod(hb, qC[k] % qB[b], qB[b]);
            hat_mod_b[i * nB + b] = hb;
        }
    }
#pragma omp parallel for
    for (int j = 0; j < n; j++) {
        for (int b = 0; b < nB; b++) {
            u64 acc = 0;
            for (int i = 0; i < nC; i++) {
                u64 y = mulmod(x[(size_t)i * n + j] % qC[i], inv_hat[i], qC[i]);
                acc = addmod(acc, mulmod(y % qB[b], hat_mod_b[i * nB + b], qB[b]), qB[b]);
            }
            out[(size_t)b * n + j] = acc;
        }
    }
    free(inv_hat);
    free(hat_mod_b);
}

/* ---------------------------------------------------------- automorphisms */
/* coefficient form: X^j -> X^(j*g mod 2n), with X^n = -1 */
void orc_automorph_coeff(const u64 *in, u64 *out, int nlimbs, int n, const u64 *q, u64 g) {
    u64 two_n = 2 * (u64)n;
    for (int l = 0; l < nlimbs; l++)
        for (int j = 0; j < n; j++) {
            u64 t = ((u64)j * g) % two_n;
            u64 v = in[(size_t)l * n + j];
            if (t < (u64)n) out[(size_t)l * n + t] = v;
            else out[(size_t)l * n + (t - n)] = (v == 0) ? 0 : q[l] - v;
        }
}

/* evaluation form of orc_ntt (slot k holds a(psi^(2k+1))):
   (a o X^g)(psi^e) = a(psi^(e g)), so out[k] = in[k'] with 2k'+1 = (2k+1) g mod 2n */
void orc_automorph_eval(const u64 *in, u64 *out, int nlimbs, int n, u64 g) {
    u64 two_n = 2 * (u64)n;
    for (int l = 0; l < nlimbs; l++)
        for (int k = 0; k < n; k++) {
            u64 e = ((2 * (u64)k + 1) * g) % two_n;
            out[(size_t)l * n + k] = in[(size_t)l * n + (e - 1) / 2];
        }
}

/* ------------------------------------------------------- centred FBC (ModDown) */
/* Like orc_fbc, but y_i = [x_i (C/q_i)^-1]_{q_i} is taken as its centred representative
   (y_i - q_i when 2 y_i > q_i), so the integer sum_i y_i (C/q_i) lies in (-|C| C/2, |C| C/2)
   and the result is free of the positive bias of the [0, q) choice. */
void orc_fbc_centred(const u64 *x, const u64 *qC, int nC, const u64 *qB, int nB, u64 *out,
                     int n) {
    u64 *inv_hat = (u64 *)malloc(sizeof(u64) * nC);
    u64 *hat_mod_b = (u64 *)malloc(sizeof(u64) * nC * nB);
    for (int i = 0; i < nC; i++) {
        u64 h = 1;
        for (int k = 0; k < nC; k++) if (k != i) h = mulmod(h, qC[k] % qC[i], qC[i]);
        inv_hat[i] = invmod(h, qC[i]);
        for (int b = 0; b < nB; b++) {
            u64 hb = 1 % qB[b];
            for (int k = 0; k < nC; k++) if (k != i) hb = mulmod(hb, qC[k] % qB[b], qB[b]);
            hat_mod_b[i * nB + b] = hb;
        }
    }
#pragma omp parallel for
    for (int j = 0; j < n; j++) {
        for (int b = 0; b < nB; b++) {
            u64 acc = 0;
            for (int i = 0; i < nC; i++) {
                u64 y = mulmod(x[(size_t)i * n + j] % qC[i], inv_hat[i], qC[i]);
                if (2 * (u128)y > qC[i]) {            /* negative representative y - q_i */
                    u64 mag = (qC[i] - y) % qB[b];
                    acc = submod(acc, mulmod(mag, hat_mod_b[i * nB + b], qB[b]), qB[b]);
                } else {
                    acc = addmod(acc, mulmod(y % qB[b], hat_mod_b[i * nB + b], qB[b]), qB[b]);
                }
            }
            out[(size_t)b * n + j] = acc;
        }
    }
    free(inv_hat);
    free(hat_mod_b);
}
