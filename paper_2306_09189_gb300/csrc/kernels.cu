// Device kernels: negacyclic NTT/INTT, fast base conversion (ModUp / ModDown), key-switching
// inner product, automorphism, rescale, plaintext x ciphertext MAC, tensor product, sampling.
// Ciphertexts are limb-major [poly][limb][n] uint64 in NTT form; one thread owns one
// coefficient index of one limb, so every global access is a coalesced 8-byte stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <string.h>

#include "internal.h"
#include "modarith.cuh"

namespace {

constexpr int TB = 256;         // threads per block for elementwise kernels
constexpr int NTT_TC = 8;       // columns per phase-A tile
constexpr int ROW = 256;        // phase-B row length (n = R * ROW)

__device__ __forceinline__ int prime_of(const KP &kp, int limb, int nq) {
    return limb < nq ? limb : kp.L + 1 + (limb - nq);
}

__device__ __forceinline__ int job_limb(const ntt_job &j, int y, int p) {
    int s0 = 0, s1 = 0;
    if (j.skip_alpha > 0) {
        if (j.skip_mod > 0) p %= j.skip_mod;
        s0 = p * j.skip_alpha;
        s1 = min(s0 + j.skip_alpha, j.nq);
        if (s0 >= j.nq) s0 = s1 = 0;
    }
    int count = j.nl - (s1 - s0);
    if (y >= count) return -1;
    int limb = j.l0 + y;
    if (s1 > s0 && limb >= s0) limb += s1 - s0;
    return limb;
}

// ------------------------------------------------------------------------------ NTT
// Forward: Cooley-Tukey with twiddles psi^{brev(k)}, natural order in, bit-reversed out.
// Inverse: Gentleman-Sande with psi^{-brev(k)}, bit-reversed in, natural out, times n^-1.
// n = R * 256: phase A runs the log2(R) stages whose butterfly distance is a multiple of 256
// on a tile of R rows x NTT_TC columns in shared memory; phase B runs the last 8 stages on
// 256-word rows, one warp per row.
template <bool INV>
__global__ void __launch_bounds__(256) ntt_cols(KP kp, ntt_job job) {
    extern __shared__ u64 sm[];
    const int p = blockIdx.z;
    const int limb = job_limb(job, blockIdx.y, p);
    if (limb < 0) return;
    const int pr = prime_of(kp, limb, job.nq);
    const u64 q = kp.q[pr];
    u64 *a = job.base + (size_t)p * job.poly_stride + (size_t)limb * kp.n;
    const int R = kp.n / ROW;
    const int c0 = blockIdx.x * NTT_TC;
    const u64 *W = (INV ? kp.itw : kp.tw) + (size_t)pr * kp.n;
    const u64 *Ws = (INV ? kp.itws : kp.tws) + (size_t)pr * kp.n;
    for (int e = threadIdx.x; e < R * NTT_TC; e += blockDim.x) {
        int r = e / NTT_TC, cc = e % NTT_TC;
        sm[e] = a[(size_t)r * ROW + c0 + cc];
    }
    __syncthreads();
    const int nb = (R / 2) * NTT_TC;
    if (!INV) {
        for (int m = 1; m < R; m <<= 1) {
            const int tr = R / (2 * m);
            for (int b = threadIdx.x; b < nb; b += blockDim.x) {
                int cc = b % NTT_TC, bb = b / NTT_TC;
                int i = bb / tr, jr = i * 2 * tr + (bb % tr);
                u64 U = sm[jr * NTT_TC + cc];
                u64 V = mul_shoup(sm[(jr + tr) * NTT_TC + cc], W[m + i], Ws[m + i], q);
                sm[jr * NTT_TC + cc] = add_mod(U, V, q);
                sm[(jr + tr) * NTT_TC + cc] = sub_mod(U, V, q);
            }
            __syncthreads();
        }
    } else {
        for (int tr = 1; tr < R; tr <<= 1) {
            const int m = R / (2 * tr);
            for (int b = threadIdx.x; b < nb; b += blockDim.x) {
                int cc = b % NTT_TC, bb = b / NTT_TC;
                int i = bb / tr, jr = i * 2 * tr + (bb % tr);
                u64 U = sm[jr * NTT_TC + cc];
                u64 V = sm[(jr + tr) * NTT_TC + cc];
                sm[jr * NTT_TC + cc] = add_mod(U, V, q);
                sm[(jr + tr) * NTT_TC + cc] = mul_shoup(sub_mod(U, V, q), W[m + i], Ws[m + i], q);
            }
            __syncthreads();
        }
    }
    const u64 ni = kp.ninv[pr], nis = kp.ninvs[pr];
    for (int e = threadIdx.x; e < R * NTT_TC; e += blockDim.x) {
        int r = e / NTT_TC, cc = e % NTT_TC;
        u64 v = sm[e];
        if (INV) v = mul_shoup(v, ni, nis, q);
        a[(size_t)r * ROW + c0 + cc] = v;
    }
}

template <bool INV>
__global__ void __launch_bounds__(256) ntt_rows(KP kp, ntt_job job) {
    __shared__ u64 sm[8][ROW];
    const int p = blockIdx.z;
    const int limb = job_limb(job, blockIdx.y, p);
    if (limb < 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int R = kp.n / ROW;
    const int row = blockIdx.x * 8 + warp;
    if (row >= R) return;                       // warp-uniform; only __syncwarp below
    const int pr = prime_of(kp, limb, job.nq);
    const u64 q = kp.q[pr];
    u64 *a = job.base + (size_t)p * job.poly_stride + (size_t)limb * kp.n + (size_t)row * ROW;
    const u64 *W = (INV ? kp.itw : kp.tw) + (size_t)pr * kp.n;
    const u64 *Ws = (INV ? kp.itws : kp.tws) + (size_t)pr * kp.n;
    u64 *s = sm[warp];
#pragma unroll
    for (int k = 0; k < 8; k++) s[lane + 32 * k] = a[lane + 32 * k];
    __syncwarp();
    if (!INV) {
        for (int m = R; m < kp.n; m <<= 1) {
            const int t = kp.n / (2 * m);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                int b = lane + 32 * k;
                int ig = b / t, jc = ig * 2 * t + (b % t);
                int i = (row * ROW + jc) / (2 * t);
                u64 U = s[jc];
                u64 V = mul_shoup(s[jc + t], W[m + i], Ws[m + i], q);
                s[jc] = add_mod(U, V, q);
                s[jc + t] = sub_mod(U, V, q);
            }
            __syncwarp();
        }
    } else {
        for (int t = 1; t < ROW; t <<= 1) {
            const int m = kp.n / (2 * t);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                int b = lane + 32 * k;
                int ig = b / t, jc = ig * 2 * t + (b % t);
                int i = (row * ROW + jc) / (2 * t);
                u64 U = s[jc], V = s[jc + t];
                s[jc] = add_mod(U, V, q);
                s[jc + t] = mul_shoup(sub_mod(U, V, q), W[m + i], Ws[m + i], q);
            }
            __syncwarp();
        }
    }
#pragma unroll
    for (int k = 0; k < 8; k++) a[lane + 32 * k] = s[lane + 32 * k];
}

// ------------------------------------------------------------------------------ NTT, radix 16
// Register-blocked form for 2^12 <= n <= 2^16 (R = n/256 rows of 256): every thread holds 16
// words and runs four butterfly stages in registers per pass; the two passes of a phase
// exchange through one shared-memory transpose.  Phase A (the log2 R stages whose distance is
// a multiple of 256): pass 1 on rows r + (R/16) j, pass 2 on rows 16 r + e.  Phase B (the last
// 8 stages, along 256-word rows): pass 1 on words l + 16 j, pass 2 on words 16 l + e.
// Butterflies are lazy (Harvey): forward values stay in [0, 4q), inverse values in [0, 2q);
// twiddles are read as {w, floor(w 2^64 / q)} pairs, one load per group of butterflies
// sharing a twiddle.
__device__ __forceinline__ void ct_lazy(u64 &X, u64 &Y, u64 w, u64 ws, u64 q, u64 q2) {
    u64 x = X >= q2 ? X - q2 : X;
    u64 t = Y * w - __umul64hi(Y, ws) * q;          // [0, 2q)
    X = x + t;
    Y = x - t + q2;
}
__device__ __forceinline__ void gs_lazy(u64 &X, u64 &Y, u64 w, u64 ws, u64 q, u64 q2) {
    u64 s = X + Y;
    s = s >= q2 ? s - q2 : s;
    u64 d = X - Y + q2;
    Y = d * w - __umul64hi(d, ws) * q;              // [0, 2q)
    X = s;
}

// stage with butterfly distance `half` words inside x[16]; element j has NTT index
// base + (j << ls); all butterflies of a group of 2*half consecutive j share one twiddle.
template <bool INV, int H>
__device__ __forceinline__ void reg_stage(u64 (&x)[16], int base, int ls, int logn,
                                          const ulonglong2 *__restrict__ W, u64 q, u64 q2) {
    constexpr int half = 1 << H;
    const int sh = ls + H + 1;
    const int m = (1 << logn) >> sh;
    const int i0 = base >> sh;
#pragma unroll
    for (int g = 0; g < (8 >> H); g++) {
        const ulonglong2 w = W[m + i0 + g];
#pragma unroll
        for (int k = 0; k < half; k++) {
            const int j = g * 2 * half + k;
            if (INV) gs_lazy(x[j], x[j + half], w.x, w.y, q, q2);
            else ct_lazy(x[j], x[j + half], w.x, w.y, q, q2);
        }
    }
}

// CT stages H = 3..lo (forward) or GS stages lo..3 (inverse), lo in [0, 4]
template <bool INV>
__device__ __forceinline__ void reg_pass(u64 (&x)[16], int base, int ls, int logn, int nstages,
                                         const ulonglong2 *__restrict__ W, u64 q, u64 q2) {
    if (!INV) {
        if (nstages >= 4) reg_stage<false, 3>(x, base, ls, logn, W, q, q2);
        if (nstages >= 3) reg_stage<false, 2>(x, base, ls, logn, W, q, q2);
        if (nstages >= 2) reg_stage<false, 1>(x, base, ls, logn, W, q, q2);
        if (nstages >= 1) reg_stage<false, 0>(x, base, ls, logn, W, q, q2);
    } else {
        if (nstages >= 1) reg_stage<true, 0>(x, base, ls, logn, W, q, q2);
        if (nstages >= 2) reg_stage<true, 1>(x, base, ls, logn, W, q, q2);
        if (nstages >= 3) reg_stage<true, 2>(x, base, ls, logn, W, q, q2);
        if (nstages >= 4) reg_stage<true, 3>(x, base, ls, logn, W, q, q2);
    }
}

template <bool INV>
__global__ void __launch_bounds__(256, 3) ntt16_cols(KP kp, ntt_job job) {
    __shared__ u64 sm[4096];
    const int p = blockIdx.z;
    const int limb = job_limb(job, blockIdx.y, p);
    if (limb < 0) return;
    const int pr = prime_of(kp, limb, job.nq);
    const u64 q = kp.q[pr], q2 = 2 * q;
    const int lr = kp.logn - 8;                      // R = 2^lr rows, 4 <= lr <= 8
    const int R16 = 1 << (lr - 4);
    const int ltc = 12 - lr, TC = 1 << ltc;           // columns per block
    const int t = threadIdx.x, tc = t & (TC - 1), r = t >> ltc;
    const int c = blockIdx.x * TC + tc;
    u64 *a = job.base + (size_t)p * job.poly_stride + (size_t)limb * kp.n;
    const ulonglong2 *W = (const ulonglong2 *)(INV ? kp.itw2 : kp.tw2) + (size_t)pr * kp.n;
    const int n2 = lr - 4;                           // pass-2 stages
    u64 x[16];
    if (!INV) {
#pragma unroll
        for (int j = 0; j < 16; j++) x[j] = a[(size_t)(r + R16 * j) * ROW + c];
        reg_pass<false>(x, r * ROW + c, lr + 4, kp.logn, 4, W, q, q2);
#pragma unroll
        for (int j = 0; j < 16; j++) sm[(r + R16 * j) * TC + tc] = x[j];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 16; e++) x[e] = sm[(16 * r + e) * TC + tc];
        reg_pass<false>(x, 16 * r * ROW + c, 8, kp.logn, n2, W, q, q2);
#pragma unroll
        for (int e = 0; e < 16; e++) a[(size_t)(16 * r + e) * ROW + c] = x[e];
    } else {
#pragma unroll
        for (int e = 0; e < 16; e++) x[e] = a[(size_t)(16 * r + e) * ROW + c];
        reg_pass<true>(x, 16 * r * ROW + c, 8, kp.logn, n2, W, q, q2);
#pragma unroll
        for (int e = 0; e < 16; e++) sm[(16 * r + e) * TC + tc] = x[e];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 16; j++) x[j] = sm[(r + R16 * j) * TC + tc];
        reg_pass<true>(x, r * ROW + c, lr + 4, kp.logn, 4, W, q, q2);
        const u64 ni = kp.ninv[pr], nis = kp.ninvs[pr];
#pragma unroll
        for (int j = 0; j < 16; j++) {
            u64 v = x[j] * ni - __umul64hi(x[j], nis) * q;
            a[(size_t)(r + R16 * j) * ROW + c] = v >= q ? v - q : v;
        }
    }
}

__device__ __forceinline__ int pad17(int k) { return k + (k >> 4); }

template <bool INV>
__global__ void __launch_bounds__(256, 3) ntt16_rows(KP kp, ntt_job job) {
    __shared__ u64 sm[16][272];
    const int p = blockIdx.z;
    const int limb = job_limb(job, blockIdx.y, p);
    if (limb < 0) return;
    const int pr = prime_of(kp, limb, job.nq);
    const u64 q = kp.q[pr], q2 = 2 * q;
    const int t = threadIdx.x, rl = t >> 4, l = t & 15;
    const int row = blockIdx.x * 16 + rl;
    u64 *a = job.base + (size_t)p * job.poly_stride + (size_t)limb * kp.n + (size_t)row * ROW;
    const ulonglong2 *W = (const ulonglong2 *)(INV ? kp.itw2 : kp.tw2) + (size_t)pr * kp.n;
    u64 *s = sm[rl];
    u64 x[16];
    if (!INV) {
#pragma unroll
        for (int j = 0; j < 16; j++) x[j] = a[l + 16 * j];
        reg_pass<false>(x, row * ROW + l, 4, kp.logn, 4, W, q, q2);
#pragma unroll
        for (int j = 0; j < 16; j++) s[pad17(l + 16 * j)] = x[j];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 16; e++) x[e] = s[pad17(16 * l + e)];
        reg_pass<false>(x, row * ROW + 16 * l, 0, kp.logn, 4, W, q, q2);
#pragma unroll
        for (int e = 0; e < 16; e++) {
            u64 v = x[e] >= q2 ? x[e] - q2 : x[e];
            s[pad17(16 * l + e)] = v >= q ? v - q : v;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 16; j++) a[l + 16 * j] = s[pad17(l + 16 * j)];
    } else {
#pragma unroll
        for (int j = 0; j < 16; j++) s[pad17(l + 16 * j)] = a[l + 16 * j];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 16; e++) x[e] = s[pad17(16 * l + e)];
        reg_pass<true>(x, row * ROW + 16 * l, 0, kp.logn, 4, W, q, q2);
#pragma unroll
        for (int e = 0; e < 16; e++) s[pad17(16 * l + e)] = x[e];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 16; j++) x[j] = s[pad17(l + 16 * j)];
        reg_pass<true>(x, row * ROW + l, 4, kp.logn, 4, W, q, q2);
#pragma unroll
        for (int j = 0; j < 16; j++) a[l + 16 * j] = x[j];
    }
}

// ------------------------------------------------------------------------------ sampling
__global__ void sample_uniform_kernel(KP kp, u64 seed, u64 stream, u64 *out, int nq) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int l = blockIdx.y;
    const int pr = prime_of(kp, l, nq);
    const u64 q = kp.q[pr];
    u64 base = 2 * ((u64)pr * kp.n + k);
    u64 lo = sm64_word(seed, stream, base);
    u64 hi = sm64_word(seed, stream, base + 1);
    // (hi 2^64 + lo) mod q = [hi]_q 2^64 + [lo]_q ; [hi]_q 2^64 = REDC([hi]_q * 2^128)
    u64 h = to_mont(reduce64(hi, q, kp.mu[pr]), q, kp.qinv[pr], kp.r2[pr]);
    out[(size_t)l * kp.n + k] = add_mod(h, reduce64(lo, q, kp.mu[pr]), q);
}

__global__ void sample_cbd_kernel(int n, u64 seed, u64 stream, int64_t *out) {
    const int k = blockIdx.x * TB + threadIdx.x;
    if (k >= n) return;
    u64 r = sm64_word(seed, stream, k);
    out[k] = (int64_t)__popcll(r & 0x1FFFFFull) - (int64_t)__popcll((r >> 21) & 0x1FFFFFull);
}

__global__ void sample_ternary_kernel(int n, u64 seed, u64 stream, int64_t *out) {
    const int k = blockIdx.x * TB + threadIdx.x;
    if (k >= n) return;
    u64 r = sm64_word(seed, stream, k) % 3;
    out[k] = r == 0 ? 0 : (r == 1 ? 1 : -1);
}

__global__ void reduce_int_kernel(KP kp, const int64_t *m, u64 *out, int nq, int mont) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int l = blockIdx.y;
    const int pr = prime_of(kp, l, nq);
    const u64 q = kp.q[pr];
    int64_t v = m[k];
    u64 r;
    if (v >= 0) {
        r = reduce64((u64)v, q, kp.mu[pr]);
    } else {
        u64 t = reduce64((u64)(-v), q, kp.mu[pr]);
        r = t == 0 ? 0 : q - t;
    }
    if (mont) r = to_mont(r, q, kp.qinv[pr], kp.r2[pr]);
    out[(size_t)l * kp.n + k] = r;
}

__global__ void mont_kernel(KP kp, u64 *x, int nq, size_t pstride, int to) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int l = blockIdx.y;
    const int pr = prime_of(kp, l, nq);
    const u64 q = kp.q[pr], qi = kp.qinv[pr];
    u64 *p = x + blockIdx.z * pstride + (size_t)l * kp.n + k;
    *p = to ? to_mont(*p, q, qi, kp.r2[pr]) : redc((u128)*p, q, qi);
}

__global__ void permute_kernel(KP kp, const u64 *in, u64 *out, u64 g) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const size_t off = (size_t)blockIdx.y * kp.n;
    out[off + k] = in[off + autom_index(k, g, kp.logn)];
}

// b = e - a s + [P]_{q_t} s'  on the limbs of digit `digit`, -a s + e elsewhere;
// then (b, a) go to Montgomery form.  All inputs NTT form over Q_L u P (global order).
__global__ void keygen_combine_kernel(KP kp, u64 *b, u64 *a, const u64 *e, const u64 *s,
                                      const u64 *sp, const u64 *pmod, int lo, int hi) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y;
    const u64 q = kp.q[t], qi = kp.qinv[t], r2 = kp.r2[t];
    const size_t i = (size_t)t * kp.n + k;
    u64 as = mul_mod(a[i], s[i], q, qi, r2);
    u64 v = sub_mod(e[i], as, q);
    if (t >= lo && t < hi) v = add_mod(v, mul_mod(pmod[t], sp[i], q, qi, r2), q);
    b[i] = to_mont(v, q, qi, r2);
    a[i] = to_mont(a[i], q, qi, r2);
}

// c0 = e - a s + m over Q_l (NTT form)
__global__ void encrypt_combine_kernel(KP kp, u64 *c0, const u64 *a, const u64 *e, const u64 *m,
                                       const u64 *s) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y;
    const u64 q = kp.q[t], qi = kp.qinv[t], r2 = kp.r2[t];
    const size_t i = (size_t)t * kp.n + k;
    u64 v = sub_mod(e[i], mul_mod(a[i], s[i], q, qi, r2), q);
    c0[i] = add_mod(v, m[i], q);
}

__global__ void decrypt_dot_kernel(KP kp, const u64 *c, size_t pstride, const u64 *s, u64 *out) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y;
    const u64 q = kp.q[t], qi = kp.qinv[t], r2 = kp.r2[t];
    const size_t i = (size_t)t * kp.n + k;
    out[i] = add_mod(c[i], mul_mod(c[pstride + i], s[i], q, qi, r2), q);
}

__global__ void addsub_kernel(KP kp, u64 *a, size_t pa, const u64 *b, size_t pb, int sub) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y;
    const u64 q = kp.q[t];
    u64 *x = a + blockIdx.z * pa + (size_t)t * kp.n + k;
    u64 y = b[blockIdx.z * pb + (size_t)t * kp.n + k];
    *x = sub ? sub_mod(*x, y, q) : add_mod(*x, y, q);
}

__global__ void mul_scalar_kernel(KP kp, u64 *a, size_t pa, const u64 *res, const u64 *sh) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y;
    u64 *x = a + blockIdx.z * pa + (size_t)t * kp.n + k;
    *x = mul_shoup(*x, res[t], sh[t], kp.q[t]);
}

struct Res64 {
    u64 v[64], s[64];
};

__global__ void mul_scalar_v_kernel(KP kp, u64 *a, size_t pa, Res64 r) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y;
    u64 *x = a + blockIdx.z * pa + (size_t)t * kp.n + k;
    *x = mul_shoup(*x, r.v[t], r.s[t], kp.q[t]);
}

__global__ void add_const_v_kernel(KP kp, u64 *a, Res64 r) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y;
    u64 *x = a + (size_t)t * kp.n + k;
    *x = add_mod(*x, r.v[t], kp.q[t]);
}

__global__ void mul_pointwise_kernel(KP kp, const u64 *a, const u64 *b, u64 *out) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y;
    const size_t i = (size_t)t * kp.n + k;
    out[i] = mul_mod(a[i], b[i], kp.q[t], kp.qinv[t], kp.r2[t]);
}

__global__ void add_const_kernel(KP kp, u64 *a, const u64 *res) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y;
    u64 *x = a + (size_t)t * kp.n + k;
    *x = add_mod(*x, res[t], kp.q[t]);
}

__global__ void zero_kernel(u64 *p, size_t words) {
    size_t i = (size_t)blockIdx.x * TB + threadIdx.x;
    if (i < words) p[i] = 0;
}

// ------------------------------------------------------------------------------ ModUp
// Digit j of x at level l: x itself on its own primes C_j n Q_l (copied from the NTT-form
// input), and on every other prime of Q_l u P the fast base conversion
//   sum_{i in C_j} [x_i (C/q_i)^-1]_{q_i} (C/q_i)  mod p     (x_i coefficient form, [0, q_i))
// The Montgomery table hat = (C/q_i) 2^64 mod p turns the whole sum into one 128-bit
// accumulation and one REDC.
struct ModupArgs {
    const u64 *x_coef, *x_ntt;
    u64 *D;
    int level, alpha;
    const u64 *tab[16];
};
__global__ void __launch_bounds__(TB) modup_kernel(KP kp, ModupArgs A) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int j = blockIdx.y;
    const int nq = A.level + 1;
    const int ext = nq + kp.K;
    const int lo = j * A.alpha;
    const int ns = min(A.alpha, nq - lo);
    const u64 *tab = A.tab[j];
    u64 *Dj = A.D + (size_t)j * ext * kp.n;
    u64 y[16];
#pragma unroll
    for (int i = 0; i < 16; i++) {
        if (i < ns) {
            const int pr = lo + i;
            u64 xv = A.x_coef[(size_t)pr * kp.n + k];
            y[i] = mul_shoup(xv, tab[i], tab[ns + i], kp.q[pr]);
            Dj[(size_t)pr * kp.n + k] = A.x_ntt[(size_t)pr * kp.n + k];
        }
    }
    const u64 *hat = tab + 2 * ns;
    const int nd = ext - ns;
    for (int d = 0; d < nd; d++) {
        const int limb = d < lo ? d : d + ns;
        const int pr = prime_of(kp, limb, nq);
        const u64 *h = hat + (size_t)d * ns;
        u128 acc = 0;
#pragma unroll
        for (int i = 0; i < 16; i++)
            if (i < ns) acc += (u128)y[i] * h[i];
        Dj[(size_t)limb * kp.n + k] = redc(acc, kp.q[pr], kp.qinv[pr]);
    }
}

// ------------------------------------------------------------------------------ inner product
// u_c[t][k] = sum_j D_j[t][phi_g(k)] * ksk[j][c][t'][k]   (key in Montgomery form -> normal)
struct IpInline {
    ip_item it[HE_INLINE_ITEMS];
};
struct MdInline {
    md_item it[HE_INLINE_ITEMS];
};

__global__ void __launch_bounds__(TB) ip_kernel(KP kp, const ip_item *items, IpInline inl, int level) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y;
    const ip_item it = items ? items[blockIdx.z] : inl.it[blockIdx.z];
    const int nq = level + 1;
    const int ext = nq + kp.K;
    const int kl = t < nq ? t : kp.L + 1 + (t - nq);     // key limb = global prime index
    const u64 q = kp.q[kl], qi = kp.qinv[kl];
    const int ks = it.g == 1 ? k : autom_index(k, it.g, kp.logn);
    const size_t kstride = (size_t)(kp.L + 1 + kp.K) * kp.n;
    u128 a0 = 0, a1 = 0;
    for (int j = 0; j < it.beta; j++) {
        u64 d = it.D[((size_t)j * ext + t) * kp.n + ks];
        const u64 *key = it.key + (size_t)(2 * j) * kstride + (size_t)kl * kp.n + k;
        a0 += (u128)d * key[0];
        a1 += (u128)d * key[kstride];
    }
    it.u[(size_t)t * kp.n + k] = redc(a0, q, qi);
    it.u[((size_t)ext + t) * kp.n + k] = redc(a1, q, qi);
}

// ------------------------------------------------------------------------------ ModDown
// conv[c][i][k] = sum_k' y~_k' (P/p_k') mod q_i with y_k' = [u_P,k' (P/p_k')^-1]_{p_k'} taken
// centred (y - p when 2y > p), so (u - conv) / P rounds instead of flooring.
__global__ void __launch_bounds__(TB) moddown_fbc_kernel(KP kp, const u64 *u, u64 *conv,
                                                         int level, const u64 *tab) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int c = blockIdx.y;
    const int nq = level + 1;
    const int ext = nq + kp.K;
    const int K = kp.K;
    const u64 *uc = u + (size_t)c * ext * kp.n;
    u64 v[16];
    bool neg[16];
#pragma unroll
    for (int i = 0; i < 16; i++) {
        if (i < K) {
            const int pr = kp.L + 1 + i;
            const u64 p = kp.q[pr];
            u64 y = mul_shoup(uc[(size_t)(nq + i) * kp.n + k], tab[i], tab[K + i], p);
            neg[i] = 2 * y > p;
            v[i] = neg[i] ? p - y : y;
        }
    }
    const u64 *hat = tab + 2 * K;
    const u64 *nhat = hat + (size_t)nq * K;
    for (int t = 0; t < nq; t++) {
        u128 acc = 0;
#pragma unroll
        for (int i = 0; i < 16; i++)
            if (i < K) acc += (u128)v[i] * (neg[i] ? nhat[t * K + i] : hat[t * K + i]);
        conv[((size_t)c * nq + t) * kp.n + k] = redc(acc, kp.q[t], kp.qinv[t]);
    }
}

// out_c[i][k] = base_c[i][phi_g(k)] + (u_c[i][k] - conv_c[i][k]) * P^-1
__global__ void __launch_bounds__(TB) moddown_combine_kernel(KP kp, const md_item *items, MdInline inl,
                                                             int level, const u64 *pinv,
                                                             const u64 *pinvs) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int i = blockIdx.y;
    const md_item it = items ? items[blockIdx.z] : inl.it[blockIdx.z];
    const int nq = level + 1;
    const int ext = nq + kp.K;
    const u64 q = kp.q[i];
    const int ks = it.g == 1 ? k : autom_index(k, it.g, kp.logn);
#pragma unroll
    for (int c = 0; c < 2; c++) {
        u64 d = sub_mod(it.u[((size_t)c * ext + i) * kp.n + k], it.conv[((size_t)c * nq + i) * kp.n + k], q);
        u64 v = mul_shoup(d, pinv[i], pinvs[i], q);
        if (it.base && c < it.base_polys) v = add_mod(v, it.base[c * it.base_pstride + (size_t)i * kp.n + ks], q);
        it.out[c * it.out_pstride + (size_t)i * kp.n + k] = v;
    }
}

// ------------------------------------------------------------------------------ rescale
// t[c][i][k] = [centred c_l]_{q_i}, from the coefficient-form top limb of poly c
__global__ void rescale_prep_kernel(KP kp, const u64 *top, size_t top_pstride, u64 *t, int level) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int i = blockIdx.y;
    const int c = blockIdx.z;
    const u64 ql = kp.q[level];
    const u64 q = kp.q[i];
    u64 v = top[c * top_pstride + k];
    u64 r;
    if (2 * v > ql) {
        u64 m = reduce64(ql - v, q, kp.mu[i]);
        r = m == 0 ? 0 : q - m;
    } else {
        r = reduce64(v, q, kp.mu[i]);
    }
    t[((size_t)c * level + i) * kp.n + k] = r;
}

__global__ void rescale_combine_kernel(KP kp, u64 *c, size_t pstride, const u64 *t, int level,
                                       const u64 *inv, const u64 *invs) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int i = blockIdx.y;
    const int p = blockIdx.z;
    const u64 q = kp.q[i];
    u64 *x = c + p * pstride + (size_t)i * kp.n + k;
    *x = mul_shoup(sub_mod(*x, t[((size_t)p * level + i) * kp.n + k], q), inv[i], invs[i], q);
}

// ------------------------------------------------------------------------------ MAC
// out_c[i][k] (+)= sum_terms pt[i][k] * ct_c[i][k]: one 128-bit accumulation per output
// word (plaintexts are in Montgomery form, so a single REDC finishes the sum).
__global__ void __launch_bounds__(TB) mac_kernel(KP kp, const mac_term *terms, mac_term one,
                                                 int n_terms, u64 *out, size_t out_pstride,
                                                 int accumulate) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int i = blockIdx.y;
    const u64 q = kp.q[i], qi = kp.qinv[i];
    const size_t off = (size_t)i * kp.n + k;
    u128 a0 = 0, a1 = 0;
    for (int t = 0; t < n_terms; t++) {
        const mac_term tm = terms ? terms[t] : one;
        u64 p = tm.pt[off];
        a0 += (u128)p * tm.ct[off];
        a1 += (u128)p * tm.ct[tm.ct_pstride + off];
    }
    u64 r0 = redc(a0, q, qi), r1 = redc(a1, q, qi);
    if (accumulate) {
        r0 = add_mod(r0, out[off], q);
        r1 = add_mod(r1, out[out_pstride + off], q);
    }
    out[off] = r0;
    out[out_pstride + off] = r1;
}

// ------------------------------------------------------------------------------ fused IP + MAC
// Two coefficients per thread: for Galois elements g = 1 mod 4 the NTT-domain automorphism
// maps the aligned pair (k, k^1) onto an aligned pair (phi(k), phi(k)^1), so every gather is a
// full 16-byte load and every key / plaintext / output access a 16-byte vector access.
__device__ __forceinline__ ulonglong2 ld2(const u64 *p) { return *(const ulonglong2 *)p; }
__device__ __forceinline__ void st2(u64 *p, u64 a, u64 b) { *(ulonglong2 *)p = make_ulonglong2(a, b); }

// Amount-major fused inner product + MAC.  For each amount the thread loads its key words
// once (two coefficients, beta digits, both polynomials) and applies them to every source
// shard that uses the amount; V <= 2 outputs per group.
template <int V, int B>
__global__ void __launch_bounds__(TB) ipmac2_kernel(KP kp, const fsrc *srcs, const famt *amts, int n_amt,
                                                    const fent *ents, int level, int beta,
                                                    u64 *acc, u64 *base) {
    const int k = 2 * (blockIdx.x * TB + threadIdx.x);
    const int t = blockIdx.y;
    const int nq = level + 1;
    const int ext = nq + kp.K;
    const int kl = t < nq ? t : kp.L + 1 + (t - nq);
    const u64 q = kp.q[kl], qi = kp.qinv[kl], r2 = kp.r2[kl];
    const u64 one = to_mont(1, q, qi, r2);
    const size_t kstride = (size_t)(kp.L + 1 + kp.K) * kp.n;
    const size_t off = (size_t)t * kp.n + k;
    u128 a0[V][2], a1[V][2], b0[V][2], b1[V][2];
#pragma unroll
    for (int v = 0; v < V; v++)
#pragma unroll
        for (int e = 0; e < 2; e++) a0[v][e] = a1[v][e] = b0[v][e] = b1[v][e] = 0;
    for (int i = 0; i < n_amt; i++) {
        const famt A = amts[i];
        const int ks = A.g == 1 ? k : autom_index(k, A.g, kp.logn);
        const int sw = ks & 1, kb = ks & ~1;
        ulonglong2 kk0[B], kk1[B];
        if (A.key) {
#pragma unroll
            for (int j = 0; j < B; j++)
                if (j < beta) {
                    const u64 *kp0 = A.key + (size_t)(2 * j) * kstride + (size_t)kl * kp.n + k;
                    kk0[j] = ld2(kp0);
                    kk1[j] = ld2(kp0 + kstride);
                }
        }
        for (int e = A.e0; e < A.e1; e++) {
            const fent E = ents[e];
            const fsrc S{E.D, E.src, E.ps};
            ulonglong2 p[V];
#pragma unroll
            for (int v = 0; v < V; v++) {
                const u64 *pp = E.pt[v];
                p[v] = pp == HE_PT_ONE ? make_ulonglong2(one, one) : (pp ? ld2(pp + off) : make_ulonglong2(0, 0));
            }
            if (A.key) {
                u128 s0[2] = {0, 0}, s1[2] = {0, 0};
#pragma unroll
                for (int j = 0; j < B; j++)
                    if (j < beta) {
                        const ulonglong2 d = ld2(S.D + ((size_t)j * ext + t) * kp.n + kb);
                        const u64 d0 = sw ? d.y : d.x, d1 = sw ? d.x : d.y;
                        s0[0] += (u128)d0 * kk0[j].x;
                        s0[1] += (u128)d1 * kk0[j].y;
                        s1[0] += (u128)d0 * kk1[j].x;
                        s1[1] += (u128)d1 * kk1[j].y;
                    }
                const u64 u00 = redc(s0[0], q, qi), u01 = redc(s0[1], q, qi);
                const u64 u10 = redc(s1[0], q, qi), u11 = redc(s1[1], q, qi);
#pragma unroll
                for (int v = 0; v < V; v++) {
                    a0[v][0] += (u128)p[v].x * u00;
                    a0[v][1] += (u128)p[v].y * u01;
                    a1[v][0] += (u128)p[v].x * u10;
                    a1[v][1] += (u128)p[v].y * u11;
                }
            }
            if (t < nq) {
                const ulonglong2 cc = ld2(S.src + (size_t)t * kp.n + kb);
                const u64 c00 = sw ? cc.y : cc.x, c01 = sw ? cc.x : cc.y;
                ulonglong2 c1 = make_ulonglong2(0, 0);
                if (!A.key) c1 = ld2(S.src + S.ps + off);
#pragma unroll
                for (int v = 0; v < V; v++) {
                    b0[v][0] += (u128)p[v].x * c00;
                    b0[v][1] += (u128)p[v].y * c01;
                    b1[v][0] += (u128)p[v].x * c1.x;
                    b1[v][1] += (u128)p[v].y * c1.y;
                }
            }
        }
    }
#pragma unroll
    for (int v = 0; v < V; v++) {
        st2(acc + ((size_t)(2 * v) * ext) * kp.n + off, redc(a0[v][0], q, qi), redc(a0[v][1], q, qi));
        st2(acc + ((size_t)(2 * v + 1) * ext) * kp.n + off, redc(a1[v][0], q, qi), redc(a1[v][1], q, qi));
        if (t < nq) {
            st2(base + ((size_t)(2 * v) * nq) * kp.n + off, redc(b0[v][0], q, qi), redc(b0[v][1], q, qi));
            st2(base + ((size_t)(2 * v + 1) * nq) * kp.n + off, redc(b1[v][0], q, qi), redc(b1[v][1], q, qi));
        }
    }
}

// acc = sum_terms K_term * x_term (+ c on poly 0) over limbs 0..level, x of any higher level
// (the drop is implicit); per-limb residues of the integer constants are passed by value.
#define HE_LC_MAX 20
#define HE_LC_LIMBS 24
struct LincombArgs {
    const u64 *x[HE_LC_MAX];
    size_t ps[HE_LC_MAX];
    u64 res[HE_LC_MAX][HE_LC_LIMBS];
    u64 cst[HE_LC_LIMBS];
    int n_terms;
};
__global__ void lincomb_kernel(KP kp, LincombArgs A, u64 *out, size_t out_ps) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int i = blockIdx.y;
    const int c = blockIdx.z;
    const u64 q = kp.q[i], qi = kp.qinv[i], r2 = kp.r2[i];
    u128 acc = 0;
    for (int t = 0; t < A.n_terms; t++) {
        const u64 x = A.x[t][c * A.ps[t] + (size_t)i * kp.n + k];
        acc += (u128)x * to_mont(A.res[t][i], q, qi, r2);
    }
    u64 r = redc(acc, q, qi);
    if (c == 0) r = add_mod(r, A.cst[i], q);
    out[c * out_ps + (size_t)i * kp.n + k] = r;
}

__global__ void tensor_kernel(KP kp, const u64 *a, size_t pa, const u64 *b, size_t pb, u64 *d,
                              int level) {
    const int k = blockIdx.x * TB + threadIdx.x;
    const int i = blockIdx.y;
    const u64 q = kp.q[i], qi = kp.qinv[i], r2 = kp.r2[i];
    const size_t off = (size_t)i * kp.n + k;
    const size_t ps = (size_t)(level + 1) * kp.n;
    u64 a0 = a[off], a1 = a[pa + off];
    u64 b0 = to_mont(b[off], q, qi, r2), b1 = to_mont(b[pb + off], q, qi, r2);
    d[off] = redc((u128)a0 * b0, q, qi);
    d[ps + off] = redc((u128)a0 * b1 + (u128)a1 * b0, q, qi);
    d[2 * ps + off] = redc((u128)a1 * b1, q, qi);
}

__global__ void copy_kernel(u64 *dst, size_t dps, const u64 *src, size_t sps, size_t words) {
    size_t i = (size_t)blockIdx.x * TB + threadIdx.x;
    if (i >= words) return;
    dst[blockIdx.y * dps + i] = src[blockIdx.y * sps + i];
}

__global__ void bench_modmul_kernel(u64 q, u64 qinv, int iters, u64 *sink) {
    u64 x = threadIdx.x + 12345, y = blockIdx.x + 777;
    for (int it = 0; it < iters; it++) {
        x = redc((u128)x * y, q, qinv);
        y = redc((u128)y * x, q, qinv);
    }
    if (x == 0xdeadbeef) sink[0] = y;
}

}  // namespace

// ================================================================================= launchers
#define LAUNCH_CHECK()                                        \
    do {                                                      \
        he_count_launch();                                    \
        cudaError_t _e = cudaGetLastError();                  \
        if (_e != cudaSuccess) {                              \
            he_set_error("kernel launch: %s", cudaGetErrorString(_e)); \
            return HE_ECUDA;                                  \
        }                                                     \
    } while (0)

int k_ntt(const he_ctx *ctx, const ntt_job &job, bool inverse, cudaStream_t s) {
    if (job.nl <= 0 || job.npoly <= 0) return HE_OK;
    const int R = ctx->n / ROW;
    if (ctx->logn >= 12 && ctx->logn <= 16) {
        const double limbs = (double)job.nl * job.npoly;
        TraceScope tr("ntt", s, limbs * 2.0 * ctx->n * 8, limbs * (ctx->n / 2) * ctx->logn);
        const int TC = 4096 / R;
        dim3 gA(ROW / TC, job.nl, job.npoly), gB(R / 16, job.nl, job.npoly);
        if (!inverse) {
            ntt16_cols<false><<<gA, 256, 0, s>>>(ctx->kp, job);
            LAUNCH_CHECK();
            ntt16_rows<false><<<gB, 256, 0, s>>>(ctx->kp, job);
            LAUNCH_CHECK();
        } else {
            ntt16_rows<true><<<gB, 256, 0, s>>>(ctx->kp, job);
            LAUNCH_CHECK();
            ntt16_cols<true><<<gA, 256, 0, s>>>(ctx->kp, job);
            LAUNCH_CHECK();
        }
        return HE_OK;
    }
    dim3 gA(ROW / NTT_TC, job.nl, job.npoly), gB((R + 7) / 8, job.nl, job.npoly);
    size_t smA = (size_t)R * NTT_TC * sizeof(u64);
    const double limbs = (double)job.nl * job.npoly;
    TraceScope tr("ntt", s, limbs * 2.0 * ctx->n * 8, limbs * (ctx->n / 2) * ctx->logn);
    if (!inverse) {
        ntt_cols<false><<<gA, 256, smA, s>>>(ctx->kp, job);
        LAUNCH_CHECK();
        ntt_rows<false><<<gB, 256, 0, s>>>(ctx->kp, job);
        LAUNCH_CHECK();
    } else {
        ntt_rows<true><<<gB, 256, 0, s>>>(ctx->kp, job);
        LAUNCH_CHECK();
        ntt_cols<true><<<gA, 256, smA, s>>>(ctx->kp, job);
        LAUNCH_CHECK();
    }
    return HE_OK;
}

int k_reduce_int(const he_ctx *ctx, const int64_t *m, u64 *out, int nlimbs, int nq, bool mont,
                 cudaStream_t s) {
    reduce_int_kernel<<<dim3(ctx->n / TB, nlimbs), TB, 0, s>>>(ctx->kp, m, out, nq, mont ? 1 : 0);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_to_mont(const he_ctx *ctx, u64 *x, int nlimbs, int nq, int npoly, size_t pstride,
              cudaStream_t s) {
    mont_kernel<<<dim3(ctx->n / TB, nlimbs, npoly), TB, 0, s>>>(ctx->kp, x, nq, pstride, 1);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_from_mont(const he_ctx *ctx, u64 *x, int nlimbs, int nq, int npoly, size_t pstride,
                cudaStream_t s) {
    mont_kernel<<<dim3(ctx->n / TB, nlimbs, npoly), TB, 0, s>>>(ctx->kp, x, nq, pstride, 0);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_sample_uniform(const he_ctx *ctx, u64 seed, u64 stream, u64 *out, int nlimbs, int nq,
                     cudaStream_t s) {
    sample_uniform_kernel<<<dim3(ctx->n / TB, nlimbs), TB, 0, s>>>(ctx->kp, seed, stream, out, nq);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_sample_cbd(const he_ctx *ctx, u64 seed, u64 stream, int64_t *out, cudaStream_t s) {
    sample_cbd_kernel<<<ctx->n / TB, TB, 0, s>>>(ctx->n, seed, stream, out);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_sample_ternary(const he_ctx *ctx, u64 seed, u64 stream, int64_t *out, cudaStream_t s) {
    sample_ternary_kernel<<<ctx->n / TB, TB, 0, s>>>(ctx->n, seed, stream, out);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_permute(const he_ctx *ctx, const u64 *in, u64 *out, int nlimbs, u64 g, cudaStream_t s) {
    permute_kernel<<<dim3(ctx->n / TB, nlimbs), TB, 0, s>>>(ctx->kp, in, out, g);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_keygen_combine(const he_ctx *ctx, u64 *b, u64 *a, const u64 *e, const u64 *s_eval,
                     const u64 *sp_eval, int digit, cudaStream_t s) {
    int lo = digit * ctx->alpha, hi = std::min(lo + ctx->alpha, ctx->L + 1);
    keygen_combine_kernel<<<dim3(ctx->n / TB, ctx->np), TB, 0, s>>>(
        ctx->kp, b, a, e, s_eval, sp_eval, ctx->d_consts, lo, hi);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_encrypt_combine(const he_ctx *ctx, u64 *c0, const u64 *a, const u64 *e, const u64 *m,
                      int level, cudaStream_t s) {
    encrypt_combine_kernel<<<dim3(ctx->n / TB, level + 1), TB, 0, s>>>(ctx->kp, c0, a, e, m, ctx->d_s);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_decrypt_dot(const he_ctx *ctx, const he_ct *ct, u64 *out, int nlimbs, cudaStream_t s) {
    decrypt_dot_kernel<<<dim3(ctx->n / TB, nlimbs), TB, 0, s>>>(ctx->kp, ct->d, ct->pstride, ctx->d_s, out);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_add(const he_ctx *ctx, he_ct *acc, const he_ct *b, bool sub, cudaStream_t s) {
    addsub_kernel<<<dim3(ctx->n / TB, acc->level + 1, 2), TB, 0, s>>>(
        ctx->kp, acc->d, acc->pstride, b->d, b->pstride, sub ? 1 : 0);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_add_raw(const he_ctx *ctx, u64 *a, size_t pa, const u64 *b, size_t pb, int nlimbs, int npoly,
              bool sub, cudaStream_t s) {
    addsub_kernel<<<dim3(ctx->n / TB, nlimbs, npoly), TB, 0, s>>>(ctx->kp, a, pa, b, pb, sub ? 1 : 0);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_mul_scalar(const he_ctx *ctx, he_ct *ct, const u64 *res, const u64 *shoup, cudaStream_t s) {
    mul_scalar_kernel<<<dim3(ctx->n / TB, ct->level + 1, 2), TB, 0, s>>>(ctx->kp, ct->d, ct->pstride, res, shoup);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_add_const(const he_ctx *ctx, he_ct *ct, const u64 *res_dev, cudaStream_t s) {
    add_const_kernel<<<dim3(ctx->n / TB, ct->level + 1), TB, 0, s>>>(ctx->kp, ct->d, res_dev);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_zero(u64 *p, size_t words, cudaStream_t s) {
    if (!words) return HE_OK;
    zero_kernel<<<(unsigned)((words + TB - 1) / TB), TB, 0, s>>>(p, words);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_copy_limbs(u64 *dst, size_t dps, const u64 *src, size_t sps, size_t words, int npoly,
                 cudaStream_t s) {
    copy_kernel<<<dim3((unsigned)((words + TB - 1) / TB), npoly), TB, 0, s>>>(dst, dps, src, sps, words);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_modup(const he_ctx *ctx, const u64 *x_coef, const u64 *x_ntt, u64 *D, int level,
            cudaStream_t s) {
    ModupArgs A;
    A.x_coef = x_coef;
    A.x_ntt = x_ntt;
    A.D = D;
    A.level = level;
    A.alpha = ctx->alpha;
    const int beta = (level + ctx->alpha) / ctx->alpha;
    if (beta > 16 || ctx->alpha > 16) {
        he_set_error("modup: at most 16 digits of at most 16 primes");
        return HE_EINVAL;
    }
    for (int j = 0; j < beta; j++) A.tab[j] = ctx->modup[level][j].d;
    const double nq = level + 1, ext = nq + ctx->K;
    TraceScope tr("modup", s, (nq + beta * ext) * ctx->n * 8, (nq + (double)beta * (ext - ctx->alpha) * ctx->alpha) * ctx->n);
    modup_kernel<<<dim3(ctx->n / TB, beta), TB, 0, s>>>(ctx->kp, A);
    LAUNCH_CHECK();
    return HE_OK;
}

static double ip_bytes(const he_ctx *ctx, int level, int items) {
    const double ext = level + 1 + ctx->K, beta = (level + ctx->alpha) / ctx->alpha;
    return (double)items * ext * ctx->n * 8 * (3 * beta + 2);
}
static double ip_mulmods(const he_ctx *ctx, int level, int items) {
    const double ext = level + 1 + ctx->K, beta = (level + ctx->alpha) / ctx->alpha;
    return (double)items * ext * ctx->n * 2 * beta;
}

int k_inner_product(const he_ctx *ctx, const ip_item *items_dev, int n_items, int level,
                    cudaStream_t s) {
    TraceScope tr("ip", s, ip_bytes(ctx, level, n_items), ip_mulmods(ctx, level, n_items));
    ip_kernel<<<dim3(ctx->n / TB, level + 1 + ctx->K, n_items), TB, 0, s>>>(ctx->kp, items_dev, IpInline{},
                                                                             level);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_inner_product_inline(const he_ctx *ctx, const ip_item *items, int n, int level, cudaStream_t s) {
    for (int i0 = 0; i0 < n; i0 += HE_INLINE_ITEMS) {
        const int cnt = std::min(HE_INLINE_ITEMS, n - i0);
        IpInline inl;
        for (int i = 0; i < cnt; i++) inl.it[i] = items[i0 + i];
        TraceScope tr("ip", s, ip_bytes(ctx, level, cnt), ip_mulmods(ctx, level, cnt));
        ip_kernel<<<dim3(ctx->n / TB, level + 1 + ctx->K, cnt), TB, 0, s>>>(ctx->kp, nullptr, inl, level);
        LAUNCH_CHECK();
    }
    return HE_OK;
}

int k_inner_product_one(const he_ctx *ctx, const ip_item &it, int level, cudaStream_t s) {
    return k_inner_product_inline(ctx, &it, 1, level, s);
}

int k_moddown_fbc(const he_ctx *ctx, const u64 *u, u64 *conv, int level, int npoly,
                  cudaStream_t s) {
    if (ctx->K > 16) {
        he_set_error("moddown: at most 16 special primes");
        return HE_EINVAL;
    }
    const double nq = level + 1;
    TraceScope tr("moddown_fbc", s, (double)npoly * (ctx->K + nq) * ctx->n * 8, (double)npoly * (ctx->K + nq * ctx->K) * ctx->n);
    moddown_fbc_kernel<<<dim3(ctx->n / TB, npoly), TB, 0, s>>>(ctx->kp, u, conv, level,
                                                              ctx->moddown[level].d);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_moddown_combine(const he_ctx *ctx, const md_item *items_dev, int n_items, int level,
                      cudaStream_t s) {
    const u64 *pinv = ctx->d_consts + ctx->np;
    const u64 *pinvs = pinv + (ctx->L + 1);
    TraceScope tr("moddown_combine", s, (double)n_items * (level + 1) * ctx->n * 8 * 7, (double)n_items * (level + 1) * ctx->n * 2);
    moddown_combine_kernel<<<dim3(ctx->n / TB, level + 1, n_items), TB, 0, s>>>(
        ctx->kp, items_dev, MdInline{}, level, pinv, pinvs);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_moddown_combine_inline(const he_ctx *ctx, const md_item *items, int n, int level, cudaStream_t s) {
    const u64 *pinv = ctx->d_consts + ctx->np;
    const u64 *pinvs = pinv + (ctx->L + 1);
    for (int i0 = 0; i0 < n; i0 += HE_INLINE_ITEMS) {
        const int cnt = std::min(HE_INLINE_ITEMS, n - i0);
        MdInline inl;
        for (int i = 0; i < cnt; i++) inl.it[i] = items[i0 + i];
        TraceScope tr("moddown_combine", s, (double)cnt * (level + 1) * ctx->n * 8 * 7,
                      (double)cnt * (level + 1) * ctx->n * 2);
        moddown_combine_kernel<<<dim3(ctx->n / TB, level + 1, cnt), TB, 0, s>>>(ctx->kp, nullptr, inl, level,
                                                                               pinv, pinvs);
        LAUNCH_CHECK();
    }
    return HE_OK;
}

int k_moddown_combine_one(const he_ctx *ctx, const md_item &it, int level, cudaStream_t s) {
    return k_moddown_combine_inline(ctx, &it, 1, level, s);
}

int k_rescale_prep(const he_ctx *ctx, const u64 *top, size_t top_pstride, u64 *t, int level,
                   cudaStream_t s) {
    rescale_prep_kernel<<<dim3(ctx->n / TB, level, 2), TB, 0, s>>>(ctx->kp, top, top_pstride, t, level);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_rescale_combine(const he_ctx *ctx, he_ct *ct, const u64 *t, cudaStream_t s) {
    const int l = ct->level;   // level before the drop
    const u64 *base = ctx->d_consts + ctx->np + 2 * (ctx->L + 1);
    const u64 *inv = base + (size_t)l * 2 * (ctx->L + 1);
    const u64 *invs = inv + (ctx->L + 1);
    TraceScope tr("rescale", s, (double)l * ctx->n * 8 * 6, (double)l * ctx->n * 2);
    rescale_combine_kernel<<<dim3(ctx->n / TB, l, 2), TB, 0, s>>>(ctx->kp, ct->d, ct->pstride, t, l, inv, invs);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_mac(const he_ctx *ctx, const mac_term *terms_dev, int n_terms, u64 *out, size_t out_pstride,
          int level, bool accumulate, cudaStream_t s) {
    TraceScope tr("mac", s, (double)(level + 1) * ctx->n * 8 * (3.0 * n_terms + 2), (double)(level + 1) * ctx->n * 2.0 * n_terms);
    mac_kernel<<<dim3(ctx->n / TB, level + 1), TB, 0, s>>>(ctx->kp, terms_dev, mac_term{}, n_terms, out,
                                                          out_pstride, accumulate ? 1 : 0);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_mac_one(const he_ctx *ctx, const mac_term &t, u64 *out, size_t out_pstride, int level,
              bool accumulate, cudaStream_t s) {
    mac_kernel<<<dim3(ctx->n / TB, level + 1), TB, 0, s>>>(ctx->kp, nullptr, t, 1, out, out_pstride,
                                                          accumulate ? 1 : 0);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_mul_scalar_v(const he_ctx *ctx, he_ct *ct, const u64 *res, const u64 *shoup, int polys,
                   cudaStream_t s) {
    Res64 r;
    for (int i = 0; i <= ct->level; i++) { r.v[i] = res[i]; r.s[i] = shoup[i]; }
    mul_scalar_v_kernel<<<dim3(ctx->n / TB, ct->level + 1, polys), TB, 0, s>>>(ctx->kp, ct->d, ct->pstride, r);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_add_const_v(const he_ctx *ctx, he_ct *ct, const u64 *res, cudaStream_t s) {
    Res64 r;
    for (int i = 0; i <= ct->level; i++) { r.v[i] = res[i]; r.s[i] = 0; }
    add_const_v_kernel<<<dim3(ctx->n / TB, ct->level + 1), TB, 0, s>>>(ctx->kp, ct->d, r);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_mul_pointwise(const he_ctx *ctx, const u64 *a, const u64 *b, u64 *out, int nlimbs,
                    cudaStream_t s) {
    mul_pointwise_kernel<<<dim3(ctx->n / TB, nlimbs), TB, 0, s>>>(ctx->kp, a, b, out);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_tensor(const he_ctx *ctx, const he_ct *a, const he_ct *b, u64 *d, cudaStream_t s) {
    tensor_kernel<<<dim3(ctx->n / TB, a->level + 1), TB, 0, s>>>(ctx->kp, a->d, a->pstride, b->d, b->pstride, d,
                                                                a->level);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_ipmac2(const he_ctx *ctx, const fsrc *srcs, const famt *amts, int n_amt, const fent *ents, int V,
             int level, u64 *acc, u64 *base, double bytes, double mulmods, cudaStream_t s) {
    const int ext = level + 1 + ctx->K;
    const int beta = (level + ctx->alpha) / ctx->alpha;
    if (beta > 8) { he_set_error("fused key switching: at most 8 digits"); return HE_EINVAL; }
    dim3 g(ctx->n / (2 * TB), ext);
    TraceScope tr("ipmac", s, bytes, mulmods);
#define IPM2(VV, BB) ipmac2_kernel<VV, BB><<<g, TB, 0, s>>>(ctx->kp, srcs, amts, n_amt, ents, level, beta, acc, base)
    if (V == 1) { if (beta <= 4) IPM2(1, 4); else IPM2(1, 8); }
    else if (V == 2) { if (beta <= 4) IPM2(2, 4); else IPM2(2, 8); }
    else { he_set_error("k_ipmac2: V must be 1 or 2"); return HE_EINVAL; }
#undef IPM2
    LAUNCH_CHECK();
    return HE_OK;
}

int k_lincomb(const he_ctx *ctx, const u64 *const *x, const size_t *ps, const u64 *res /*[n][24]*/, int n,
              const u64 *cst /*[24]*/, int level, u64 *out, size_t out_ps, cudaStream_t s) {
    if (n < 1 || n > HE_LC_MAX || level + 1 > HE_LC_LIMBS) {
        he_set_error("lincomb: at most %d terms of at most %d limbs", HE_LC_MAX, HE_LC_LIMBS);
        return HE_EINVAL;
    }
    LincombArgs A;
    memset(&A, 0, sizeof(A));
    for (int t = 0; t < n; t++) {
        A.x[t] = x[t];
        A.ps[t] = ps[t];
        for (int i = 0; i <= level; i++) A.res[t][i] = res[t * HE_LC_LIMBS + i];
    }
    for (int i = 0; i <= level; i++) A.cst[i] = cst[i];
    A.n_terms = n;
    lincomb_kernel<<<dim3(ctx->n / TB, level + 1, 2), TB, 0, s>>>(ctx->kp, A, out, out_ps);
    LAUNCH_CHECK();
    return HE_OK;
}

// rescale of m ciphertexts laid out at a uniform stride (poly p of ct i at base + (2i + p) ps)
int k_rescale_many(const he_ctx *ctx, u64 *base, size_t ps, int m, int level, u64 *t, cudaStream_t s) {
    ntt_job top{base, ps, level, 1, level + 1, 0, 2 * m, 0};
    HE_TRY(k_ntt(ctx, top, true, s));
    rescale_prep_kernel<<<dim3(ctx->n / TB, level, 2 * m), TB, 0, s>>>(ctx->kp, base + (size_t)level * ctx->n, ps, t, level);
    LAUNCH_CHECK();
    ntt_job tj{t, (size_t)level * ctx->n, 0, level, level, 0, 2 * m, 0};
    HE_TRY(k_ntt(ctx, tj, false, s));
    const u64 *cb = ctx->d_consts + ctx->np + 2 * (ctx->L + 1);
    const u64 *inv = cb + (size_t)level * 2 * (ctx->L + 1);
    const u64 *invs = inv + (ctx->L + 1);
    TraceScope tr("rescale", s, (double)m * level * ctx->n * 8 * 6, (double)m * level * ctx->n * 2);
    rescale_combine_kernel<<<dim3(ctx->n / TB, level, 2 * m), TB, 0, s>>>(ctx->kp, base, ps, t, level, inv, invs);
    LAUNCH_CHECK();
    return HE_OK;
}

double k_bench_modmul(const he_ctx *ctx, int blocks, int iters, cudaStream_t s) {
    u64 *sink;
    if (cudaMalloc(&sink, 8) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const u64 q = ctx->primes[0];
    bench_modmul_kernel<<<blocks, 256, 0, s>>>(q, ctx->h_qinv[0], 16, sink);   // warm-up
    cudaEventRecord(e0, s);
    bench_modmul_kernel<<<blocks, 256, 0, s>>>(q, ctx->h_qinv[0], iters, sink);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    he_count_launch(2);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return (double)blocks * 256.0 * 2.0 * iters / (ms * 1e-3);
}
