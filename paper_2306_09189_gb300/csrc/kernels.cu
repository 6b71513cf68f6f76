// Device kernels: negacyclic NTT/INTT, fast base conversion (ModUp / ModDown), key-switching
// inner product, automorphism, rescale, plaintext x ciphertext MAC, tensor product, sampling.
// Ciphertexts are limb-major [poly][limb][n] uint64 in NTT form; one thread owns one
// coefficient index of one limb, so every global access is a coalesced 8-byte stream.
#include <cuda_runtime.h>

#include <atomic>
#include <utility>

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

__device__ __forceinline__ u64 *job_poly(const ntt_job &j, int p) {
    return j.tab[0] ? j.tab[p] : j.base + (size_t)p * j.poly_stride;
}

// Programmatic dependent launch: every kernel is launched with the programmatic-serialisation
// attribute (when enabled), so its grid is set up while the predecessor on the stream
// finishes; each kernel's first statement, griddepcontrol.wait, holds it until the predecessor
// has completed and its writes are visible (a no-op for a normal launch).  The predecessor
// never waits for the dependent, so no launch can deadlock; results are unchanged.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ------------------------------------------------------------------------------ NTT
// Forward: Cooley-Tukey with twiddles psi^{brev(k)}, natural order in, bit-reversed out.
// Inverse: Gentleman-Sande with psi^{-brev(k)}, bit-reversed in, natural out, times n^-1.
// n = R * 256: phase A runs the log2(R) stages whose butterfly distance is a multiple of 256
// on a tile of R rows x NTT_TC columns in shared memory; phase B runs the last 8 stages on
// 256-word rows, one warp per row.

template <bool INV>
__global__ void __launch_bounds__(256) ntt_cols(KP kp, ntt_job job) {
    pdl_wait();
    extern __shared__ u64 sm[];
    const int p = blockIdx.z;
    const int limb = job_limb(job, blockIdx.y, p);
    if (limb < 0) return;
    const int pr = prime_of(kp, limb, job.nq);
    const u64 q = kp.q[pr];
    u64 *a = job_poly(job, p) + (size_t)limb * kp.n;
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
    pdl_wait();
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
    u64 *a = job_poly(job, p) + (size_t)limb * kp.n + (size_t)row * ROW;
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
// Forward butterfly without the correction of X (NC, "no correction"): with every prime below
// 2^57 the values may grow by 2q per stage instead: from [0, 4q) they stay below 36q < 2^63
// after the 16 stages of n = 2^16 (the Shoup product accepts any 64-bit word), and the last
// pass reduces them once (Barrett) instead of once per butterfly.
__device__ __forceinline__ void ct_lazy_nc(u64 &X, u64 &Y, u64 w, u64 ws, u64 q, u64 q2) {
    const u64 x = X;
    const u64 t = Y * w - __umul64hi(Y, ws) * q;    // [0, 2q)
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
template <bool INV, int H, bool NC = false>
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
            else if (NC) ct_lazy_nc(x[j], x[j + half], w.x, w.y, q, q2);
            else ct_lazy(x[j], x[j + half], w.x, w.y, q, q2);
        }
    }
}

// CT stages H = 3..lo (forward) or GS stages lo..3 (inverse), lo in [0, 4]
template <bool INV, bool NC = false>
__device__ __forceinline__ void reg_pass(u64 (&x)[16], int base, int ls, int logn, int nstages,
                                         const ulonglong2 *__restrict__ W, u64 q, u64 q2) {
    if (!INV) {
        if (nstages >= 4) reg_stage<false, 3, NC>(x, base, ls, logn, W, q, q2);
        if (nstages >= 3) reg_stage<false, 2, NC>(x, base, ls, logn, W, q, q2);
        if (nstages >= 2) reg_stage<false, 1, NC>(x, base, ls, logn, W, q, q2);
        if (nstages >= 1) reg_stage<false, 0, NC>(x, base, ls, logn, W, q, q2);
    } else {
        if (nstages >= 1) reg_stage<true, 0>(x, base, ls, logn, W, q, q2);
        if (nstages >= 2) reg_stage<true, 1>(x, base, ls, logn, W, q, q2);
        if (nstages >= 3) reg_stage<true, 2>(x, base, ls, logn, W, q, q2);
        if (nstages >= 4) reg_stage<true, 3>(x, base, ls, logn, W, q, q2);
    }
}

// A rescale fused into the forward NTT of its correction term t: RS in the column pass loads
// t[i] = [centred c_l]_{q_i} straight from the coefficient-form top limb of poly p (at
// c + p ps + level n); RS in the row pass stores c_i = (c_i - NTT(t)_i) q_l^-1 into the
// ciphertext instead of NTT(t).  Same words as rescale_prep / rescale_combine around the NTT.
struct RescaleFuse {
    u64 *c;
    size_t ps;
    int level;
    const u64 *inv, *invs;
    u64 *ctab[HE_NTT_TAB];   // when ctab[0] is set: poly p of the ciphertexts at ctab[p]
};
__device__ __forceinline__ u64 *fuse_poly(const RescaleFuse &F, int p) {
    return F.ctab[0] ? F.ctab[p] : F.c + (size_t)p * F.ps;
}
__device__ __forceinline__ u64 centred_mod(u64 v, u64 ql, u64 q, u64 mu) {
    if (2 * v > ql) {
        const u64 m = reduce64(ql - v, q, mu);
        return m == 0 ? 0 : q - m;
    }
    return reduce64(v, q, mu);
}

template <bool INV, bool RS = false, bool NC = false>
__global__ void __launch_bounds__(256, 3) ntt16_cols(KP kp, ntt_job job, RescaleFuse F) {
    pdl_wait();
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
    u64 *a = job_poly(job, p) + (size_t)limb * kp.n;
    const ulonglong2 *W = (const ulonglong2 *)(INV ? kp.itw2 : kp.tw2) + (size_t)pr * kp.n;
    const int n2 = lr - 4;                           // pass-2 stages
    u64 x[16];
    if (!INV) {
        if (RS) {
            const u64 *top = fuse_poly(F, p) + (size_t)F.level * kp.n;
            const u64 ql = kp.q[F.level], mu = kp.mu[pr];
#pragma unroll
            for (int j = 0; j < 16; j++) x[j] = centred_mod(top[(size_t)(r + R16 * j) * ROW + c], ql, q, mu);
        } else {
#pragma unroll
            for (int j = 0; j < 16; j++) x[j] = a[(size_t)(r + R16 * j) * ROW + c];
        }
        reg_pass<false, NC>(x, r * ROW + c, lr + 4, kp.logn, 4, W, q, q2);
#pragma unroll
        for (int j = 0; j < 16; j++) sm[(r + R16 * j) * TC + tc] = x[j];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 16; e++) x[e] = sm[(16 * r + e) * TC + tc];
        reg_pass<false, NC>(x, 16 * r * ROW + c, 8, kp.logn, n2, W, q, q2);
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

template <bool INV, bool RS = false, bool NC = false>
__global__ void __launch_bounds__(256, 3) ntt16_rows(KP kp, ntt_job job, RescaleFuse F) {
    pdl_wait();
    __shared__ u64 sm[16][272];
    const int p = blockIdx.z;
    const int limb = job_limb(job, blockIdx.y, p);
    if (limb < 0) return;
    const int pr = prime_of(kp, limb, job.nq);
    const u64 q = kp.q[pr], q2 = 2 * q;
    const int t = threadIdx.x, rl = t >> 4, l = t & 15;
    const int row = blockIdx.x * 16 + rl;
    u64 *a = job_poly(job, p) + (size_t)limb * kp.n + (size_t)row * ROW;
    const ulonglong2 *W = (const ulonglong2 *)(INV ? kp.itw2 : kp.tw2) + (size_t)pr * kp.n;
    u64 *s = sm[rl];
    u64 x[16];
    if (!INV) {
#pragma unroll
        for (int j = 0; j < 16; j++) x[j] = a[l + 16 * j];
        reg_pass<false, NC>(x, row * ROW + l, 4, kp.logn, 4, W, q, q2);
#pragma unroll
        for (int j = 0; j < 16; j++) s[pad17(l + 16 * j)] = x[j];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 16; e++) x[e] = s[pad17(16 * l + e)];
        reg_pass<false, NC>(x, row * ROW + 16 * l, 0, kp.logn, 4, W, q, q2);
        if (NC) {
            const u64 mu = kp.mu[pr];
#pragma unroll
            for (int e = 0; e < 16; e++) s[pad17(16 * l + e)] = reduce64(x[e], q, mu);
        } else {
#pragma unroll
            for (int e = 0; e < 16; e++) {
                u64 v = x[e] >= q2 ? x[e] - q2 : x[e];
                s[pad17(16 * l + e)] = v >= q ? v - q : v;
            }
        }
        __syncthreads();
        if (RS) {
            u64 *cr = fuse_poly(F, p) + (size_t)limb * kp.n + (size_t)row * ROW;
            const u64 iv = F.inv[pr], ivs = F.invs[pr];
#pragma unroll
            for (int j = 0; j < 16; j++) {
                u64 *xp = cr + l + 16 * j;
                *xp = mul_shoup(sub_mod(*xp, s[pad17(l + 16 * j)], q), iv, ivs, q);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 16; j++) a[l + 16 * j] = s[pad17(l + 16 * j)];
        }
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

// The row pass with the in-row transposes done by warp shuffles instead of shared memory
// (HE_NTT_TWOPASS_SHUFFLE): the 16 threads of a row are half a warp, so element (lane l,
// register j) moves to (lane j, register l) in four rounds of xor-shuffles, each swapping the
// off-diagonal halves of the 2m x 2m blocks (m = 8, 4, 2, 1).  No shared memory and no block
// barrier; 32 64-bit shuffles and their selects per transpose.  Same words as ntt16_rows.
__device__ __forceinline__ u64 shfl_xor64(u64 v, int m) {
    const unsigned lo = __shfl_xor_sync(0xffffffffu, (unsigned)v, m);
    const unsigned hi = __shfl_xor_sync(0xffffffffu, (unsigned)(v >> 32), m);
    return ((u64)hi << 32) | lo;
}
__device__ __forceinline__ void lane_transpose16(u64 (&x)[16], int l) {
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int m = 8 >> r;
        const bool b = (l & m) != 0;
#pragma unroll
        for (int j = 0; j < 16; j++)
            if (!(j & m)) {
                const u64 recv = shfl_xor64(b ? x[j] : x[j + m], m);
                if (b) x[j] = recv;
                else x[j + m] = recv;
            }
    }
}

template <bool INV, bool RS = false, bool NC = false>
__global__ void __launch_bounds__(256, 3) ntt16_rows_shfl(KP kp, ntt_job job, RescaleFuse F) {
    pdl_wait();
    const int p = blockIdx.z;
    const int limb = job_limb(job, blockIdx.y, p);
    if (limb < 0) return;
    const int pr = prime_of(kp, limb, job.nq);
    const u64 q = kp.q[pr], q2 = 2 * q;
    const int t = threadIdx.x, rl = t >> 4, l = t & 15;
    const int row = blockIdx.x * 16 + rl;
    u64 *a = job_poly(job, p) + (size_t)limb * kp.n + (size_t)row * ROW;
    const ulonglong2 *W = (const ulonglong2 *)(INV ? kp.itw2 : kp.tw2) + (size_t)pr * kp.n;
    u64 x[16];
#pragma unroll
    for (int j = 0; j < 16; j++) x[j] = a[l + 16 * j];
    if (!INV) {
        reg_pass<false, NC>(x, row * ROW + l, 4, kp.logn, 4, W, q, q2);
        lane_transpose16(x, l);
        reg_pass<false, NC>(x, row * ROW + 16 * l, 0, kp.logn, 4, W, q, q2);
        if (NC) {
            const u64 mu = kp.mu[pr];
#pragma unroll
            for (int e = 0; e < 16; e++) x[e] = reduce64(x[e], q, mu);
        } else {
#pragma unroll
            for (int e = 0; e < 16; e++) {
                const u64 v = x[e] >= q2 ? x[e] - q2 : x[e];
                x[e] = v >= q ? v - q : v;
            }
        }
        lane_transpose16(x, l);
        if (RS) {
            u64 *cr = fuse_poly(F, p) + (size_t)limb * kp.n + (size_t)row * ROW;
            const u64 iv = F.inv[pr], ivs = F.invs[pr];
#pragma unroll
            for (int j = 0; j < 16; j++) {
                u64 *xp = cr + l + 16 * j;
                *xp = mul_shoup(sub_mod(*xp, x[j], q), iv, ivs, q);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 16; j++) a[l + 16 * j] = x[j];
        }
    } else {
        lane_transpose16(x, l);
        reg_pass<true>(x, row * ROW + 16 * l, 0, kp.logn, 4, W, q, q2);
        lane_transpose16(x, l);
        reg_pass<true>(x, row * ROW + l, 4, kp.logn, 4, W, q, q2);
#pragma unroll
        for (int j = 0; j < 16; j++) a[l + 16 * j] = x[j];
    }
}

// ------------------------------------------------------------------------------ one-pass NTT
// n = 2^16 in ONE launch: each limb is transformed by a cluster of CL CTAs (CL = 8 or 16, 16 words
// per thread), so the data crosses HBM/L2 once each way instead of twice.  View the limb as CL
// blocks of BLK = 2^16 / CL words, one per CTA.  Forward (Cooley-Tukey, butterfly distances
// 2^15 .. 1, four stages per radix-16 round):
//   A  CTA r, thread t holds the 16 words b0 + k 2^12 (b0 = r T + t, T = BLK / 16 threads): the
//      four stages of distance >= 4096, which mix the blocks, run in registers;
//   -> every word is stored into the shared memory of the CTA owning its block (distributed
//      shared memory across the cluster), then one cluster barrier;
//   B  offsets (t >> 8) 4096 + (t & 255) + 256 k     distances 2048 .. 256
//   C  offsets (t >> 4) 256 + (t & 15) + 16 k        distances 128 .. 16
//   D  offsets 16 t + k                              distances 8 .. 1, then stored contiguously
// with a shared-memory transpose between rounds (padded one word in 16: conflict-free).  The
// inverse (Gentleman-Sande) runs D, C, B on the CTA's own block, scatters into the layout of A
// on the destination CTAs, and finishes with A and the factor n^-1.  Same words as the two-pass
// ntt16_cols / ntt16_rows pair.
template <int CL> struct NcShape {
    static constexpr int BLK = 65536 / CL;       // words per CTA
    static constexpr int T = BLK / 16;           // threads per CTA
    static constexpr int SMEM = BLK + BLK / 16;  // padded block (also holds round A's [16][T] layout)
    static constexpr int PER = BLK / 4096;       // 4096-word halves per block (2 or 1)
    static constexpr int MINB = CL == 8 ? 1 : 3; // resident CTAs per SM the register budget targets
};

__device__ __forceinline__ int pad16(int b) { return b + (b >> 4); }
__device__ __forceinline__ void cluster_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// shared::cluster address of `local` (this CTA's shared memory) in the CTA of cluster rank `rank`
__device__ __forceinline__ unsigned dsmem_addr(const void *local, unsigned rank) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(local);
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void dsmem_st(unsigned addr, u64 v) {
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}

// one radix-16 round on the CTA's block: 16 words at sm[pad16(b + (k << ls))]
template <bool INV>
__device__ __forceinline__ void nc_round(u64 (&x)[16], u64 *sm, int b, int ls, int gbase,
                                         const ulonglong2 *__restrict__ W, u64 q, u64 q2) {
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = sm[pad16(b + (k << ls))];
    reg_pass<INV>(x, gbase + b, ls, 16, 4, W, q, q2);
#pragma unroll
    for (int k = 0; k < 16; k++) sm[pad16(b + (k << ls))] = x[k];
}

template <bool INV, bool RS, int CL>
__global__ void __launch_bounds__(NcShape<CL>::T, NcShape<CL>::MINB)
    ntt16_cluster(KP kp, ntt_job job, RescaleFuse F) {
    using S = NcShape<CL>;
    pdl_wait();
    extern __shared__ u64 sm[];
    const int p = blockIdx.z;
    const int limb = job_limb(job, blockIdx.y, p);   // one limb per cluster: all its CTAs agree
    if (limb < 0) return;
    const int pr = prime_of(kp, limb, job.nq);
    const u64 q = kp.q[pr], q2 = 2 * q;
    const int t = threadIdx.x;
    const int r = blockIdx.x;                         // cluster rank: the grid is one cluster wide
    const int blk = r * S::BLK;                       // this CTA's block in rounds B, C, D
    const int b0 = r * S::T + t;                      // round A: words b0 + (k << 12), b0 < 4096
    u64 *a = job_poly(job, p) + (size_t)limb * kp.n;
    const ulonglong2 *W = (const ulonglong2 *)(INV ? kp.itw2 : kp.tw2) + (size_t)pr * kp.n;
    u64 x[16];
    if (!INV) {
        cluster_arrive_relaxed();                     // this CTA has started
        if (RS) {
            const u64 *top = fuse_poly(F, p) + (size_t)F.level * kp.n;
            const u64 ql = kp.q[F.level], mu = kp.mu[pr];
#pragma unroll
            for (int k = 0; k < 16; k++) x[k] = centred_mod(top[b0 + (k << 12)], ql, q, mu);
        } else {
#pragma unroll
            for (int k = 0; k < 16; k++) x[k] = a[b0 + (k << 12)];
        }
        reg_pass<false>(x, b0, 12, 16, 4, W, q, q2);
        cluster_wait();                               // every CTA has started: remote stores are safe
        // word b0 + (k << 12) lies in block k / PER at offset b0 + (k mod PER) 4096
#pragma unroll
        for (int k = 0; k < 16; k++)
            dsmem_st(dsmem_addr(&sm[pad16(b0 + ((k % S::PER) << 12))], k / S::PER), x[k]);
        cluster_arrive();
        cluster_wait();                               // the block is complete in this CTA
        nc_round<false>(x, sm, ((t >> 8) << 12) + (t & 255), 8, blk, W, q, q2);
        __syncthreads();
        nc_round<false>(x, sm, ((t >> 4) << 8) + (t & 15), 4, blk, W, q, q2);
        __syncthreads();
        const int bD = t << 4;
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = sm[pad16(bD + k)];
        reg_pass<false>(x, blk + bD, 0, 16, 4, W, q, q2);
#pragma unroll
        for (int k = 0; k < 16; k++) {
            const u64 v = x[k] >= q2 ? x[k] - q2 : x[k];
            x[k] = v >= q ? v - q : v;
        }
        if (RS) {
            ulonglong2 *cr = (ulonglong2 *)(fuse_poly(F, p) + (size_t)limb * kp.n + blk + bD);
            const u64 iv = F.inv[pr], ivs = F.invs[pr];
#pragma unroll
            for (int k = 0; k < 8; k++) {
                ulonglong2 v = cr[k];
                v.x = mul_shoup(sub_mod(v.x, x[2 * k], q), iv, ivs, q);
                v.y = mul_shoup(sub_mod(v.y, x[2 * k + 1], q), iv, ivs, q);
                cr[k] = v;
            }
        } else {
            ulonglong2 *o = (ulonglong2 *)(a + blk + bD);
#pragma unroll
            for (int k = 0; k < 8; k++) o[k] = make_ulonglong2(x[2 * k], x[2 * k + 1]);
        }
    } else {
        const int bD = t << 4;
        const ulonglong2 *in = (const ulonglong2 *)(a + blk + bD);
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const ulonglong2 v = in[k];
            x[2 * k] = v.x;
            x[2 * k + 1] = v.y;
        }
        reg_pass<true>(x, blk + bD, 0, 16, 4, W, q, q2);
#pragma unroll
        for (int k = 0; k < 16; k++) sm[pad16(bD + k)] = x[k];
        __syncthreads();
        nc_round<true>(x, sm, ((t >> 4) << 8) + (t & 15), 4, blk, W, q, q2);
        __syncthreads();
        const int bB = ((t >> 8) << 12) + (t & 255);
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = sm[pad16(bB + (k << 8))];
        cluster_arrive();                             // this CTA's block is read: it may be overwritten
        reg_pass<true>(x, blk + bB, 8, 16, 4, W, q, q2);
        cluster_wait();
        // word blk + bB + 256 k is word w + (j << 12) of round A's layout, w = (t & 255) + 256 k
        // and j = r PER + (t >> 8): thread w mod T of CTA w / T, slot j
        const int j = r * S::PER + (t >> 8);
#pragma unroll
        for (int k = 0; k < 16; k++) {
            const int w = (t & 255) + (k << 8);
            dsmem_st(dsmem_addr(&sm[j * S::T + w % S::T], w / S::T), x[k]);
        }
        cluster_arrive();
        cluster_wait();
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = sm[k * S::T + t];
        reg_pass<true>(x, b0, 12, 16, 4, W, q, q2);
        const u64 ni = kp.ninv[pr], nis = kp.ninvs[pr];
#pragma unroll
        for (int k = 0; k < 16; k++) {
            const u64 v = x[k] * ni - __umul64hi(x[k], nis) * q;
            a[b0 + (k << 12)] = v >= q ? v - q : v;
        }
    }
}

// ------------------------------------------------------------------------------ range check
// counts the words of a ciphertext (both polynomials, limbs 0..level) that are not below their
// prime: a device-side sanitizer that records instead of trapping
__global__ void range_check_kernel(KP kp, const u64 *d, size_t ps, unsigned long long *bad) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int i = blockIdx.y, c = blockIdx.z;
    const u64 v = d[c * ps + (size_t)i * kp.n + k];
    const unsigned m = __ballot_sync(0xffffffffu, v >= kp.q[i]);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(bad, (unsigned long long)__popc(m));
}

// ------------------------------------------------------------------------------ sampling
__global__ void sample_uniform_kernel(KP kp, u64 seed, u64 stream, u64 *out, int nq) {
    pdl_wait();
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
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    if (k >= n) return;
    u64 r = sm64_word(seed, stream, k);
    out[k] = (int64_t)__popcll(r & 0x1FFFFFull) - (int64_t)__popcll((r >> 21) & 0x1FFFFFull);
}

__global__ void sample_ternary_kernel(int n, u64 seed, u64 stream, int64_t *out) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    if (k >= n) return;
    u64 r = sm64_word(seed, stream, k) % 3;
    out[k] = r == 0 ? 0 : (r == 1 ? 1 : -1);
}

__global__ void reduce_int_kernel(KP kp, const int64_t *m, u64 *out, int nq, int mont) {
    pdl_wait();
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
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int l = blockIdx.y;
    const int pr = prime_of(kp, l, nq);
    const u64 q = kp.q[pr], qi = kp.qinv[pr];
    u64 *p = x + blockIdx.z * pstride + (size_t)l * kp.n + k;
    *p = to ? to_mont(*p, q, qi, kp.r2[pr]) : redc((u128)*p, q, qi);
}

__global__ void permute_kernel(KP kp, const u64 *in, u64 *out, u64 g) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const size_t off = (size_t)blockIdx.y * kp.n;
    out[off + k] = in[off + autom_index(k, g, kp.logn)];
}

// b = e - a s + [P]_{q_t} s'  on the limbs of digit `digit`, -a s + e elsewhere;
// then (b, a) go to Montgomery form.  All inputs NTT form over Q_L u P (global order).
__global__ void keygen_combine_kernel(KP kp, u64 *b, u64 *a, const u64 *e, const u64 *s,
                                      const u64 *sp, const u64 *pmod, int lo, int hi) {
    pdl_wait();
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
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y;
    const u64 q = kp.q[t], qi = kp.qinv[t], r2 = kp.r2[t];
    const size_t i = (size_t)t * kp.n + k;
    u64 v = sub_mod(e[i], mul_mod(a[i], s[i], q, qi, r2), q);
    c0[i] = add_mod(v, m[i], q);
}

__global__ void decrypt_dot_kernel(KP kp, const u64 *c, size_t pstride, const u64 *s, u64 *out) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y;
    const u64 q = kp.q[t], qi = kp.qinv[t], r2 = kp.r2[t];
    const size_t i = (size_t)t * kp.n + k;
    out[i] = add_mod(c[i], mul_mod(c[pstride + i], s[i], q, qi, r2), q);
}

__global__ void addsub_kernel(KP kp, u64 *a, size_t pa, const u64 *b, size_t pb, int sub) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y;
    const u64 q = kp.q[t];
    u64 *x = a + blockIdx.z * pa + (size_t)t * kp.n + k;
    u64 y = b[blockIdx.z * pb + (size_t)t * kp.n + k];
    *x = sub ? sub_mod(*x, y, q) : add_mod(*x, y, q);
}

__global__ void mul_scalar_kernel(KP kp, u64 *a, size_t pa, const u64 *res, const u64 *sh) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y;
    u64 *x = a + blockIdx.z * pa + (size_t)t * kp.n + k;
    *x = mul_shoup(*x, res[t], sh[t], kp.q[t]);
}

struct Res64 {
    u64 v[64], s[64];
};

__global__ void mul_scalar_v_kernel(KP kp, u64 *a, size_t pa, Res64 r) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y;
    u64 *x = a + blockIdx.z * pa + (size_t)t * kp.n + k;
    *x = mul_shoup(*x, r.v[t], r.s[t], kp.q[t]);
}

__global__ void add_const_v_kernel(KP kp, u64 *a, Res64 r) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y;
    u64 *x = a + (size_t)t * kp.n + k;
    *x = add_mod(*x, r.v[t], kp.q[t]);
}

__global__ void mul_pointwise_kernel(KP kp, const u64 *a, const u64 *b, u64 *out) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y;
    const size_t i = (size_t)t * kp.n + k;
    out[i] = mul_mod(a[i], b[i], kp.q[t], kp.qinv[t], kp.r2[t]);
}

// Sparse ternary secret of weight h: a partial Fisher-Yates shuffle of 0..n-1.  Step k swaps
// position k with k + (word 2k mod (n - k)) and gives the coefficient at the position it lands
// on the sign + (word 2k + 1 even) or - (odd).  One block: the threads clear the output and
// lay out the identity permutation, then one thread walks the h steps (h <= n, no waits).
__global__ void sample_sparse_kernel(int n, u64 seed, u64 stream, int h, int32_t *perm, int64_t *out) {
    pdl_wait();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        perm[i] = i;
        out[i] = 0;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int k = 0; k < h; k++) {
        const int r = (int)(sm64_word(seed, stream, 2 * (u64)k) % (u64)(n - k));
        const int32_t t = perm[k];
        perm[k] = perm[k + r];
        perm[k + r] = t;
        const bool odd = sm64_word(seed, stream, 2 * (u64)k + 1) & 1;
        out[perm[k]] = odd ? -1 : 1;
    }
}

// Coefficient-form residues mod q_0 (poly p at in + p n) lifted to their centred
// representatives in (-q_0/2, q_0/2] and reduced mod q_l, l < nl (ModRaise).
__global__ void modraise_kernel(KP kp, const u64 *in, u64 *out, size_t pstride) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int l = blockIdx.y;
    const int p = blockIdx.z;
    const u64 q0 = kp.q[0], q = kp.q[l], mu = kp.mu[l];
    const u64 x = in[(size_t)p * kp.n + k];
    u64 r;
    if (x > q0 - x) {                           // 2x > q_0: the representative x - q_0 < 0
        const u64 m = reduce64(q0 - x, q, mu);
        r = m ? q - m : 0;
    } else {
        r = reduce64(x, q, mu);
    }
    out[(size_t)p * pstride + (size_t)l * kp.n + k] = r;
}

// Both polynomials times the monomial X^e (0 <= e < 2n) in NTT form: slot k holds
// a(psi^(2 brev(k) + 1)), so it is multiplied by psi^(e (2 brev(k) + 1) mod 2n), read from the
// forward twiddle table (psi^j at position brev(j), j < n; psi^(j + n) = -psi^j).
__global__ void monomial_kernel(KP kp, u64 *d, size_t pstride, u64 e) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int l = blockIdx.y;
    const u64 q = kp.q[l];
    const unsigned bk = __brev((unsigned)k) >> (32 - kp.logn);
    const u64 ex = (e * (2 * (u64)bk + 1)) & ((2ull << kp.logn) - 1);
    const bool neg = ex >= (u64)kp.n;
    const unsigned j = (unsigned)(neg ? ex - kp.n : ex);
    const size_t w = (size_t)l * kp.n + (__brev(j) >> (32 - kp.logn));
    u64 *x = d + (size_t)blockIdx.z * pstride + (size_t)l * kp.n + k;
    const u64 v = mul_shoup(*x, kp.tw[w], kp.tws[w], q);
    *x = neg && v ? q - v : v;
}

__global__ void add_const_kernel(KP kp, u64 *a, const u64 *res) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y;
    u64 *x = a + (size_t)t * kp.n + k;
    *x = add_mod(*x, res[t], kp.q[t]);
}

__global__ void zero_kernel(u64 *p, size_t words) {
    pdl_wait();
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
// digit j of one source: x_coef = c1 in coefficient form, x_ntt = c1 in NTT form, D its digits.
// CAP >= the digit's prime count ns (alpha, or fewer for the last digit): the launchers pick
// CAP = alpha for alpha <= 8, so the loops unroll to the digit size instead of a fixed 16.
template <int CAP>
__device__ __forceinline__ void modup_digit(const KP &kp, const ModupArgs &A, const u64 *x_coef, const u64 *x_ntt,
                                            u64 *D, int k, int j) {
    const int nq = A.level + 1;
    const int ext = nq + kp.K;
    const int lo = j * A.alpha;
    const int ns = min(A.alpha, nq - lo);
    const u64 *tab = A.tab[j];
    u64 *Dj = D + (size_t)j * ext * kp.n;
    u64 y[CAP];
#pragma unroll
    for (int i = 0; i < CAP; i++) {
        if (i < ns) {
            const int pr = lo + i;
            u64 xv = x_coef[(size_t)pr * kp.n + k];
            y[i] = mul_shoup(xv, tab[i], tab[ns + i], kp.q[pr]);
            Dj[(size_t)pr * kp.n + k] = x_ntt[(size_t)pr * kp.n + k];
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
        for (int i = 0; i < CAP; i++)
            if (i < ns) acc += (u128)y[i] * h[i];
        Dj[(size_t)limb * kp.n + k] = redc(acc, kp.q[pr], kp.qinv[pr]);
    }
}

template <int CAP>
__global__ void __launch_bounds__(TB) modup_kernel(KP kp, ModupArgs A) {
    pdl_wait();
    modup_digit<CAP>(kp, A, A.x_coef, A.x_ntt, A.D, blockIdx.x * TB + threadIdx.x, blockIdx.y);
}

// several sources in one launch (blockIdx.z): coefficient-form c1 at x_coef + z nq n
template <int CAP>
__global__ void __launch_bounds__(TB) modup_batch_kernel(KP kp, ModupArgs A, const modup_src *tab) {
    pdl_wait();
    const int z = blockIdx.z;
    const size_t nqn = (size_t)(A.level + 1) * kp.n;
    modup_digit<CAP>(kp, A, A.x_coef + z * nqn, tab[z].c1, tab[z].D, blockIdx.x * TB + threadIdx.x, blockIdx.y);
}

// several sources at fixed strides in one launch (blockIdx.z): no table, so it is safe to
// capture in a graph
template <int CAP>
__global__ void __launch_bounds__(TB) modup_strided_kernel(KP kp, ModupArgs A, size_t xs, size_t ns, size_t ds) {
    pdl_wait();
    const size_t z = blockIdx.z;
    modup_digit<CAP>(kp, A, A.x_coef + z * xs, A.x_ntt + z * ns, A.D + z * ds, blockIdx.x * TB + threadIdx.x,
                     blockIdx.y);
}

// instantiation for a prime count n <= 16: exact for n <= 8, else 16
#define CAP_SWITCH(n, GO)                                                                         \
    switch (n) {                                                                                  \
        case 1: GO(1); break;                                                                     \
        case 2: GO(2); break;                                                                     \
        case 3: GO(3); break;                                                                     \
        case 4: GO(4); break;                                                                     \
        case 5: GO(5); break;                                                                     \
        case 6: GO(6); break;                                                                     \
        case 7: GO(7); break;                                                                     \
        case 8: GO(8); break;                                                                     \
        default: GO(16);                                                                          \
    }

// c1 (NTT form) of every source into one contiguous [n_src][words] buffer
__global__ void gather_c1_kernel(const modup_src *tab, u64 *dst, size_t words) {
    pdl_wait();
    const size_t k = (size_t)blockIdx.x * TB + threadIdx.x;
    if (k < words) dst[(size_t)blockIdx.y * words + k] = tab[blockIdx.y].c1[k];
}

// ------------------------------------------------------------------------------ inner product
// u_c[t][k] = sum_j D_j[t][phi_g(k)] * ksk[j][c][t'][k]   (key in Montgomery form -> normal)
struct IpInline {
    ip_item it[HE_INLINE_ITEMS];
};
struct MdInline {
    md_item it[HE_INLINE_ITEMS];
};

// CAP >= beta (the launchers pick CAP = beta for beta <= 8): every digit's loads issue together
template <int CAP>
__global__ void __launch_bounds__(TB) ip_kernel(KP kp, const ip_item *items, IpInline inl, int level) {
    pdl_wait();
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
#pragma unroll
    for (int j = 0; j < CAP; j++)
        if (j < it.beta) {
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
// centred y_k' of the K special primes for one coefficient; CAP >= K (the launchers pick
// CAP = K for K <= 8)
template <int CAP>
__device__ __forceinline__ void fbc_centred(const KP &kp, const u64 *uc, int nq, int k, const u64 *tab, u64 (&v)[CAP],
                                            bool (&neg)[CAP]) {
    const int K = kp.K;
#pragma unroll
    for (int i = 0; i < CAP; i++) {
        if (i < K) {
            const int pr = kp.L + 1 + i;
            const u64 p = kp.q[pr];
            u64 y = mul_shoup(uc[(size_t)(nq + i) * kp.n + k], tab[i], tab[K + i], p);
            neg[i] = 2 * y > p;
            v[i] = neg[i] ? p - y : y;
        }
    }
}
template <int CAP>
__device__ __forceinline__ u64 fbc_sum(const KP &kp, int t, const u64 (&v)[CAP], const bool (&neg)[CAP],
                                       const u64 *hat, const u64 *nhat) {
    const int K = kp.K;
    u128 acc = 0;
#pragma unroll
    for (int i = 0; i < CAP; i++)
        if (i < K) acc += (u128)v[i] * (neg[i] ? nhat[t * K + i] : hat[t * K + i]);
    return redc(acc, kp.q[t], kp.qinv[t]);
}

template <int CAP>
__global__ void __launch_bounds__(TB) moddown_fbc_kernel(KP kp, const u64 *u, u64 *conv, int level, const u64 *tab) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int c = blockIdx.y;
    const int nq = level + 1;
    const int ext = nq + kp.K;
    const int K = kp.K;
    const u64 *uc = u + (size_t)c * ext * kp.n;
    u64 v[CAP];
    bool neg[CAP];
    fbc_centred<CAP>(kp, uc, nq, k, tab, v, neg);
    const u64 *hat = tab + 2 * K;
    const u64 *nhat = hat + (size_t)nq * K;
    for (int t = 0; t < nq; t++) conv[((size_t)c * nq + t) * kp.n + k] = fbc_sum<CAP>(kp, t, v, neg, hat, nhat);
}

// out_c[i][k] = base_c[i][phi_g(k)] + (u_c[i][k] - conv_c[i][k]) * P^-1
__global__ void __launch_bounds__(TB) moddown_combine_kernel(KP kp, const md_item *items, MdInline inl,
                                                             int level, const u64 *pinv,
                                                             const u64 *pinvs) {
    pdl_wait();
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

// ------------------------------------------------------------------------------ ModDown + rescale
// A key switch whose output is rescaled at once (a relinearised product): with y = ModDown(u)
// + base and c' = Rescale(y), the top limb y_l is formed in coefficient form directly,
// y_l = (INTT(u_l + P base_l) - conv_l) P^-1 mod q_l (INTT is linear, so folding P base_l into
// u_l before its INTT adds base_l after it), and for i < l
//   c'_i = (u_i P^-1 + base_i - NTT(conv_i P^-1 + [y_l]_{q_i})) q_l^-1,
// one forward NTT of l limbs instead of the ModDown's l+1 and the rescale's l, and no INTT of
// y_l.  Every step is exact mod q_i: the bits of ModDown then rescale.

// u[i][c][l] += P base[i][c][l]  (NTT form, c = 0, 1; item i = blockIdx.z)
__global__ void fold_top_kernel(KP kp, u64 *u, size_t u_is, size_t u_ps, const u64 *base, size_t b_is, size_t b_ps,
                                int level, const u64 *pmod) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int c = blockIdx.y, i = blockIdx.z;
    const u64 q = kp.q[level], qi = kp.qinv[level], r2 = kp.r2[level];
    const u64 Pm = to_mont(pmod[level], q, qi, r2);
    u64 *x = u + (size_t)i * u_is + (size_t)c * u_ps + (size_t)level * kp.n + k;
    const u64 b = base[(size_t)i * b_is + (size_t)c * b_ps + (size_t)level * kp.n + k];
    *x = add_mod(*x, mul_mont(b, Pm, q, qi), q);
}

// per poly (blockIdx.y): u = [ext][n] with limbs l..l+K in coefficient form; w = [l][n]
template <int CAP>
__global__ void __launch_bounds__(TB) moddown_rescale_fbc_kernel(KP kp, const u64 *u, u64 *w, int level,
                                                                 const u64 *tab, const u64 *pinv, const u64 *pinvs) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int c = blockIdx.y;
    const int nq = level + 1;
    const int ext = nq + kp.K;
    const int K = kp.K;
    const u64 *uc = u + (size_t)c * ext * kp.n;
    u64 v[CAP];
    bool neg[CAP];
    fbc_centred<CAP>(kp, uc, nq, k, tab, v, neg);
    const u64 *hat = tab + 2 * K;
    const u64 *nhat = hat + (size_t)nq * K;
    // y_l in coefficient form, then its centred representative reduced mod every lower prime
    const u64 ql = kp.q[level];
    const u64 yl = mul_shoup(sub_mod(uc[(size_t)level * kp.n + k], fbc_sum<CAP>(kp, level, v, neg, hat, nhat), ql),
                             pinv[level], pinvs[level], ql);
    const bool yneg = 2 * yl > ql;
    // blockIdx.z of gridDim.z: this block's share of the target primes (small batches split the
    // targets so the launch fills the GPU; y_l is recomputed per share, K + 1 products)
    const int per = (level + gridDim.z - 1) / gridDim.z;
    const int t0 = blockIdx.z * per, t1 = min(level, t0 + per);
    for (int t = t0; t < t1; t++) {
        const u64 q = kp.q[t];
        u64 r;
        if (yneg) {
            const u64 m = reduce64(ql - yl, q, kp.mu[t]);
            r = m == 0 ? 0 : q - m;
        } else {
            r = reduce64(yl, q, kp.mu[t]);
        }
        w[((size_t)c * level + t) * kp.n + k] =
            add_mod(mul_shoup(fbc_sum<CAP>(kp, t, v, neg, hat, nhat), pinv[t], pinvs[t], q), r, q);
    }
}

struct mdr_item {            // one key switch of a fused ModDown + rescale
    const u64 *u;            // [2][l+1+K][n]
    const u64 *base;         // base polys (NTT form), poly c at base + c base_ps
    size_t base_ps;
    const u64 *w;            // [2][l][n], NTT form
    u64 *out;                // output at level l-1, poly c at out + c out_ps
    size_t out_ps;
};
struct MdrInline {
    mdr_item it[HE_INLINE_ITEMS];
};

__global__ void __launch_bounds__(TB) moddown_rescale_combine_kernel(KP kp, MdrInline inl, int level,
                                                                     const u64 *pinv, const u64 *pinvs,
                                                                     const u64 *linv, const u64 *linvs) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int i = blockIdx.y;
    const mdr_item it = inl.it[blockIdx.z];
    const int ext = level + 1 + kp.K;
    const u64 q = kp.q[i];
#pragma unroll
    for (int c = 0; c < 2; c++) {
        u64 x = mul_shoup(it.u[((size_t)c * ext + i) * kp.n + k], pinv[i], pinvs[i], q);
        x = add_mod(x, it.base[c * it.base_ps + (size_t)i * kp.n + k], q);
        x = sub_mod(x, it.w[((size_t)c * level + i) * kp.n + k], q);
        it.out[c * it.out_ps + (size_t)i * kp.n + k] = mul_shoup(x, linv[i], linvs[i], q);
    }
}

// ------------------------------------------------------------------------------ rescale
// t[c][i][k] = [centred c_l]_{q_i}, from the coefficient-form top limb of poly c
__global__ void rescale_prep_kernel(KP kp, const u64 *top, size_t top_pstride, u64 *t, int level) {
    pdl_wait();
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
    pdl_wait();
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
    pdl_wait();
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
// ==== fused key-switch + MAC kernels: begin (the profiles record a checksum of this region)
__device__ __forceinline__ ulonglong2 ld2(const u64 *p) { return *(const ulonglong2 *)p; }
__device__ __forceinline__ void st2(u64 *p, u64 a, u64 b) { *(ulonglong2 *)p = make_ulonglong2(a, b); }

// L2 residency: the key and plaintext streams are read once per launch, while the raised
// digits and the source ciphertext are gathered again for every rotation amount.  Streaming
// loads carry an evict-first policy and gathers an evict-last one, so the gathered working set
// (one source: beta (l+1+K) n words, 52 MB at n = 2^16, l = 19) stays in the 126 MB L2
// instead of being flushed by gigabytes of keys.
__device__ __forceinline__ u64 policy_evict_first() {
    u64 p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ u64 policy_evict_last() {
    u64 p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ u64 ld_hint(const u64 *p, u64 pol) {
    u64 r;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(pol));
    return r;
}

__device__ __forceinline__ ulonglong2 ld2_hint(const u64 *p, u64 pol) {
    ulonglong2 r;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
                 : "=l"(r.x), "=l"(r.y) : "l"(p), "l"(pol));
    return r;
}

// Block -> (group, coefficient tile, limb).  Groups go in batches of gb: blockIdx.x walks the
// batch's groups fastest, then the coefficient tiles, then the batches, so the groups sharing a
// (tile, prime) run side by side (each key and plaintext word comes from DRAM once per batch)
// while a batch's raised digits stay in L2 across all tiles (gb = n_grp: every group side by
// side; a smaller gb keeps the gathered working set small).  blockIdx.y is the global prime.
// Returns false for a q-prime above the group's level or a padding block past the last group.
// t is the limb's index in the group's Q_l u P layout, ptl its index in the plaintexts' layout.
__device__ __forceinline__ bool grp_pos(const KP &kp, const fgrp *grps, int n_grp, int gb, fgrp &P, int &tile,
                                        int &t, int &ptl, int tile_coeffs = 512) {
    const int n_tiles = kp.n / tile_coeffs;
    const int g_in = blockIdx.x % gb, rest = blockIdx.x / gb;
    tile = rest % n_tiles;
    const int g = (rest / n_tiles) * gb + g_in;
    if (g >= n_grp) return false;
    P = grps[g];
    const int kl = blockIdx.y;
    if (kl <= kp.L) {
        if (kl > P.level) return false;
        t = ptl = kl;
    } else {
        t = P.level + 1 + (kl - kp.L - 1);
        ptl = P.pt_level + 1 + (kl - kp.L - 1);
    }
    return true;
}

// Amount-major fused inner product + MAC.  For each amount the thread loads its key words
// once (two coefficients, beta digits, both polynomials) and applies them to every source
// shard that uses the amount; V <= 2 outputs per group.  The next amount's descriptors are
// fetched while the current one computes, so each amount costs one memory round trip.
//
// The unrotated part folds into the raised sum: on a q-limb, u_0 += [P]_q phi(c0) and, for
// amount 0, u = [P]_q (c0, c1).  ModDown(acc + P b) = ModDown(acc) + b exactly (P b vanishes
// mod every p), so the outputs need no separate base sums and the ModDown adds nothing else.
template <int V, int B>
__global__ void __launch_bounds__(TB, (V == 1 && B == 4) ? 2 : 1) ipmac_kernel(KP kp, const fgrp *grps, int n_grp,
                                                                               int gb, const u64 *pmod) {
    pdl_wait();
    fgrp P;
    int tile, t, ptl;
    if (!grp_pos(kp, grps, n_grp, gb, P, tile, t, ptl)) return;
    const int k = 2 * (tile * TB + threadIdx.x);
    const int kl = blockIdx.y;
    const int nq = P.level + 1;
    const int ext = nq + kp.K;
    const int beta = P.beta;
    const bool isq = t < nq;
    const u64 q = kp.q[kl], qi = kp.qinv[kl], r2 = kp.r2[kl];
    const u64 one = to_mont(1, q, qi, r2);
    const u64 Pm = isq ? to_mont(pmod[kl], q, qi, r2) : 0;     // [P]_q in Montgomery form
    const size_t kstride = (size_t)(kp.L + 1 + kp.K) * kp.n;
    const size_t off = (size_t)t * kp.n + k, ptoff = (size_t)ptl * kp.n + k;
    const u64 stream = policy_evict_first(), keep = policy_evict_last();
    u128 a0[V][2], a1[V][2];
#pragma unroll
    for (int v = 0; v < V; v++)
#pragma unroll
        for (int e = 0; e < 2; e++) a0[v][e] = a1[v][e] = 0;
    const int n_amt = P.n_amt;
    famt A = n_amt > 0 ? P.amts[0] : famt{};
    fent E = (n_amt > 0 && A.e0 < A.e1) ? P.ents[A.e0] : fent{};
    for (int i = 0; i < n_amt; i++) {
        famt An{};
        fent En{};
        if (i + 1 < n_amt) {
            An = P.amts[i + 1];
            if (An.e0 < An.e1) En = P.ents[An.e0];
        }
        const int ks = A.g == 1 ? k : autom_index(k, A.g, kp.logn);
        const int sw = ks & 1, kb = ks & ~1;
        ulonglong2 kk0[B], kk1[B];
        if (A.key) {
#pragma unroll
            for (int j = 0; j < B; j++)
                if (j < beta) {
                    const u64 *kp0 = A.key + (size_t)(2 * j) * kstride + (size_t)kl * kp.n + k;
                    kk0[j] = ld2_hint(kp0, stream);
                    kk1[j] = ld2_hint(kp0 + kstride, stream);
                }
        }
        for (int e = A.e0; e < A.e1; e++) {
            if (e > A.e0) E = P.ents[e];
            ulonglong2 p[V];
#pragma unroll
            for (int v = 0; v < V; v++) {
                const u64 *pp = E.pt[v];
                p[v] = pp == HE_PT_ONE ? make_ulonglong2(one, one) : (pp ? ld2_hint(pp + ptoff, stream) : make_ulonglong2(0, 0));
            }
            ulonglong2 cc = make_ulonglong2(0, 0), c1 = make_ulonglong2(0, 0);
            if (isq) {
                cc = ld2_hint(E.src + (size_t)t * kp.n + kb, keep);
                if (!A.key) c1 = ld2_hint(E.src + E.ps + off, keep);
            }
            u64 u00 = 0, u01 = 0, u10 = 0, u11 = 0;
            if (A.key) {
                u128 s0[2] = {0, 0}, s1[2] = {0, 0};
#pragma unroll
                for (int j = 0; j < B; j++)
                    if (j < beta) {
                        const ulonglong2 d = ld2_hint(E.D + ((size_t)j * ext + t) * kp.n + kb, keep);
                        const u64 d0 = sw ? d.y : d.x, d1 = sw ? d.x : d.y;
                        s0[0] += (u128)d0 * kk0[j].x;
                        s0[1] += (u128)d1 * kk0[j].y;
                        s1[0] += (u128)d0 * kk1[j].x;
                        s1[1] += (u128)d1 * kk1[j].y;
                    }
                u00 = redc(s0[0], q, qi);
                u01 = redc(s0[1], q, qi);
                u10 = redc(s1[0], q, qi);
                u11 = redc(s1[1], q, qi);
            }
            if (isq) {
                const u64 c00 = sw ? cc.y : cc.x, c01 = sw ? cc.x : cc.y;
                u00 = add_mod(u00, mul_mont(c00, Pm, q, qi), q);
                u01 = add_mod(u01, mul_mont(c01, Pm, q, qi), q);
                if (!A.key) {
                    u10 = mul_mont(c1.x, Pm, q, qi);
                    u11 = mul_mont(c1.y, Pm, q, qi);
                }
            }
#pragma unroll
            for (int v = 0; v < V; v++) {
                a0[v][0] += (u128)p[v].x * u00;
                a0[v][1] += (u128)p[v].y * u01;
                a1[v][0] += (u128)p[v].x * u10;
                a1[v][1] += (u128)p[v].y * u11;
            }
        }
        A = An;
        E = En;
    }
#pragma unroll
    for (int v = 0; v < V; v++)
        if (v < P.nv) {
            st2(P.acc + ((size_t)(2 * v) * ext) * kp.n + off, redc(a0[v][0], q, qi), redc(a0[v][1], q, qi));
            st2(P.acc + ((size_t)(2 * v + 1) * ext) * kp.n + off, redc(a1[v][0], q, qi), redc(a1[v][1], q, qi));
        }
}

// ---- TMA-pipelined form: each keyed amount's key tile (2 beta limb segments of 512 words)
// is copied by cp.async.bulk into a ring of TMA_STAGES shared-memory stages, each signalled
// by its own mbarrier; thread 0 keeps TMA_STAGES - 1 tiles in flight ahead of the block, so
// the key stream's latency is covered without holding key words in registers.  Every wait
// is bounded: on timeout the kernel sets *err, waits (bounded) for its copies in flight and
// returns.
constexpr int TMA_TILE = 512;                 // coefficients per block (two per thread)
constexpr int TMA_STAGES = 3;                 // ring depth (3 x 32 KB at beta = 4: 2 blocks per SM)
constexpr long long WAIT_LIMIT = 1ll << 24;   // try_wait polls before giving up, at most
constexpr unsigned long long WAIT_NS = 250000000ull;   // and at most 250 ms of wall time

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned phase) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(bar), "r"(phase) : "memory");
    return done != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Gives up after WAIT_NS of wall time (checked every 64 polls) or WAIT_LIMIT polls.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned phase) {
    const unsigned long long t0 = global_ns();
    for (long long it = 0; it < WAIT_LIMIT; it++) {
        if (mbar_try(bar, phase)) return true;
        if ((it & 63) == 63 && global_ns() - t0 > WAIT_NS) return false;
    }
    return false;
}
__device__ __forceinline__ void tma_load(unsigned dst, const void *src, unsigned bytes, unsigned bar, u64 pol) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar), "l"(pol) : "memory");
}

template <int V>
__global__ void __launch_bounds__(TB) ipmac_tma_kernel(KP kp, const fgrp *grps, int n_grp, int gb, int *err,
                                                       const u64 *pmod) {
    pdl_wait();
    constexpr int NS = TMA_STAGES;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    fgrp P;
    int tile, t, ptl;
    if (!grp_pos(kp, grps, n_grp, gb, P, tile, t, ptl)) return;   // block-uniform
    const int beta = P.beta, n_amt = P.n_amt;
    const famt *amts = P.amts;
    const fent *ents = P.ents;
    u64 *kbuf = (u64 *)smem_raw;                               // [NS stages][2 beta][TMA_TILE]
    const int seg = 2 * beta;
    uint64_t *bars = (uint64_t *)(kbuf + (size_t)NS * seg * TMA_TILE);
    const int k0 = tile * TMA_TILE;
    const int k = k0 + 2 * threadIdx.x;
    const int kl = blockIdx.y;
    const int nq = P.level + 1;
    const int ext = nq + kp.K;
    const u64 q = kp.q[kl], qi = kp.qinv[kl], r2 = kp.r2[kl];
    const u64 one = to_mont(1, q, qi, r2);
    const bool isq = t < nq;
    const u64 Pm = isq ? to_mont(pmod[kl], q, qi, r2) : 0;     // [P]_q in Montgomery form
    const size_t kstride = (size_t)(kp.L + 1 + kp.K) * kp.n;
    const size_t off = (size_t)t * kp.n + k, ptoff = (size_t)ptl * kp.n + k;
    const unsigned tile_bytes = TMA_TILE * 8;
    const u64 stream = policy_evict_first(), keep = policy_evict_last();
    if (*(volatile int *)err) return;              // an earlier block already gave up: results invalid
    if (threadIdx.x == 0) {
        for (int st = 0; st < NS; st++) mbar_init(smem_u32(&bars[st]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // producer (thread 0): copy the key tile of amount i into stage st
    auto issue = [&](int i, int st) {
        const unsigned bar = smem_u32(&bars[st]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, (unsigned)seg * tile_bytes);
        const u64 *kb = amts[i].key + (size_t)kl * kp.n + k0;
        for (int sgi = 0; sgi < seg; sgi++)
            tma_load(smem_u32(kbuf + ((size_t)st * seg + sgi) * TMA_TILE), kb + (size_t)sgi * kstride, tile_bytes, bar,
                     stream);
    };
    int next = 0, issued = 0, used = 0;            // next keyed amount to issue; counts of keyed amounts
    while (next < n_amt && !amts[next].key) next++;
    while (issued < NS - 1 && next < n_amt) {      // prologue: NS - 1 tiles in flight
        if (threadIdx.x == 0) issue(next, issued % NS);
        issued++;
        next++;
        while (next < n_amt && !amts[next].key) next++;
    }
    u128 a0[V][2], a1[V][2];
#pragma unroll
    for (int v = 0; v < V; v++)
#pragma unroll
        for (int e = 0; e < 2; e++) a0[v][e] = a1[v][e] = 0;
    bool failed = false;
    for (int i = 0; i < n_amt; i++) {
        const famt A = amts[i];
        const int ks = A.g == 1 ? k : autom_index(k, A.g, kp.logn);
        const int sw = ks & 1, kb = ks & ~1;
        const u64 *kt = nullptr;
        bool ok = true;
        if (A.key) {
            const int st = used % NS;
            // refill the stage the block released at the end of the previous keyed amount
            if (next < n_amt) {
                if (threadIdx.x == 0) issue(next, issued % NS);
                issued++;
                next++;
                while (next < n_amt && !amts[next].key) next++;
            }
            ok = mbar_wait_bounded(smem_u32(&bars[st]), (used / NS) & 1);
            kt = kbuf + (size_t)st * seg * TMA_TILE + 2 * threadIdx.x;
        }
        for (int e = A.e0; e < A.e1; e++) {
            const fent E = ents[e];
            ulonglong2 p[V];
#pragma unroll
            for (int v = 0; v < V; v++) {
                const u64 *pp = E.pt[v];
                p[v] = pp == HE_PT_ONE ? make_ulonglong2(one, one) : (pp ? ld2_hint(pp + ptoff, stream) : make_ulonglong2(0, 0));
            }
            ulonglong2 cc = make_ulonglong2(0, 0), c1 = make_ulonglong2(0, 0);
            if (isq) {
                cc = ld2_hint(E.src + (size_t)t * kp.n + kb, keep);
                if (!A.key) c1 = ld2_hint(E.src + E.ps + off, keep);
            }
            u64 u00 = 0, u01 = 0, u10 = 0, u11 = 0;
            if (A.key) {
                u128 s0[2] = {0, 0}, s1[2] = {0, 0};
#pragma unroll
                for (int j = 0; j < 4; j++)
                    if (j < beta) {
                        const ulonglong2 d = ld2_hint(E.D + ((size_t)j * ext + t) * kp.n + kb, keep);
                        const u64 d0 = sw ? d.y : d.x, d1 = sw ? d.x : d.y;
                        const ulonglong2 k0v = *(const ulonglong2 *)(kt + (size_t)(2 * j) * TMA_TILE);
                        const ulonglong2 k1v = *(const ulonglong2 *)(kt + (size_t)(2 * j + 1) * TMA_TILE);
                        s0[0] += (u128)d0 * k0v.x;
                        s0[1] += (u128)d1 * k0v.y;
                        s1[0] += (u128)d0 * k1v.x;
                        s1[1] += (u128)d1 * k1v.y;
                    }
                u00 = redc(s0[0], q, qi);
                u01 = redc(s0[1], q, qi);
                u10 = redc(s1[0], q, qi);
                u11 = redc(s1[1], q, qi);
            }
            if (isq) {                             // fold [P]_q phi(c0) (and [P]_q c1 at amount 0)
                const u64 c00 = sw ? cc.y : cc.x, c01 = sw ? cc.x : cc.y;
                u00 = add_mod(u00, mul_mont(c00, Pm, q, qi), q);
                u01 = add_mod(u01, mul_mont(c01, Pm, q, qi), q);
                if (!A.key) {
                    u10 = mul_mont(c1.x, Pm, q, qi);
                    u11 = mul_mont(c1.y, Pm, q, qi);
                }
            }
#pragma unroll
            for (int v = 0; v < V; v++) {
                a0[v][0] += (u128)p[v].x * u00;
                a0[v][1] += (u128)p[v].y * u01;
                a1[v][0] += (u128)p[v].x * u10;
                a1[v][1] += (u128)p[v].y * u11;
            }
        }
        if (A.key) {
            used++;
            // one barrier per keyed amount: it releases the stage for the refill issued next
            // round and makes the timeout decision block-uniform (a thread whose wait gave up
            // computed on stale words; the vote discards the block's results)
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
        }
    }
    if (failed) {
        // record it, then let the copies still in flight land (bounded) before the block's
        // shared memory goes away
        if (threadIdx.x == 0) atomicExch(err, 1);
        for (int u = used - 1; u < issued; u++) mbar_wait_bounded(smem_u32(&bars[u % NS]), (u / NS) & 1);
        return;
    }
#pragma unroll
    for (int v = 0; v < V; v++)
        if (v < P.nv) {
            st2(P.acc + ((size_t)(2 * v) * ext) * kp.n + off, redc(a0[v][0], q, qi), redc(a0[v][1], q, qi));
            st2(P.acc + ((size_t)(2 * v + 1) * ext) * kp.n + off, redc(a1[v][0], q, qi), redc(a1[v][1], q, qi));
        }
}

// ---- cp.async form: every word an (amount, entry) item needs (its amount's key words at the
// amount's first entry, the gathered digit pairs, plaintext pairs, c0 and c1) is copied by the
// thread itself, 16 bytes at a time, into its own shared-memory slots, CP_STAGES - 1 items ahead
// of the one it computes: no block barrier, no register holds a word in flight.
constexpr int CP_STAGES = 3;

__device__ __forceinline__ void cp_async16(unsigned dst, const void *src, u64 pol) {
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int V>
__global__ void __launch_bounds__(TB) ipmac_cp_kernel(KP kp, const fgrp *grps, int n_grp, int gb, const u64 *pmod) {
    pdl_wait();
    constexpr int RS = CP_STAGES, B = 4;
    constexpr int NW = 2 * B + B + V + 2;            // 16-byte words per item: keys, D, pt, c0, c1
    extern __shared__ ulonglong2 csm[];              // [RS][NW][TB]
    fgrp P;
    int tile, t, ptl;
    if (!grp_pos(kp, grps, n_grp, gb, P, tile, t, ptl)) return;
    const int k = 2 * (tile * TB + threadIdx.x);
    const int kl = blockIdx.y;
    const int nq = P.level + 1;
    const int ext = nq + kp.K;
    const int beta = P.beta;
    const bool isq = t < nq;
    const u64 q = kp.q[kl], qi = kp.qinv[kl], r2 = kp.r2[kl];
    const u64 one = to_mont(1, q, qi, r2);
    const u64 Pm = isq ? to_mont(pmod[kl], q, qi, r2) : 0;
    const size_t kstride = (size_t)(kp.L + 1 + kp.K) * kp.n;
    const size_t off = (size_t)t * kp.n + k, ptoff = (size_t)ptl * kp.n + k;
    const u64 stream = policy_evict_first(), keep = policy_evict_last();
    const unsigned sbase = smem_u32(csm);
    auto slot = [&](int st, int w) -> int { return (st * NW + w) * TB + threadIdx.x; };
    // items are (amount, entry) pairs in order; item e belongs to amount am[e]
    const int n_amt = P.n_amt;
    const int n_item = n_amt > 0 ? P.amts[n_amt - 1].e1 : 0;
    // producer state: the item to issue next and its amount
    int pi = 0, pa = 0;
    auto issue = [&](int st) {
        while (pa < n_amt && pi >= P.amts[pa].e1) pa++;
        const famt A = P.amts[pa];
        const fent E = P.ents[pi];
        const int ks = A.g == 1 ? k : autom_index(k, A.g, kp.logn);
        const int kb = ks & ~1;
        if (A.key) {
            if (pi == A.e0) {
#pragma unroll
                for (int j = 0; j < B; j++)
                    if (j < beta) {
                        const u64 *kp0 = A.key + (size_t)(2 * j) * kstride + (size_t)kl * kp.n + k;
                        cp_async16(sbase + 16u * slot(st, 2 * j), kp0, stream);
                        cp_async16(sbase + 16u * slot(st, 2 * j + 1), kp0 + kstride, stream);
                    }
            }
#pragma unroll
            for (int j = 0; j < B; j++)
                if (j < beta) cp_async16(sbase + 16u * slot(st, 2 * B + j), E.D + ((size_t)j * ext + t) * kp.n + kb, keep);
        }
#pragma unroll
        for (int v = 0; v < V; v++)
            if (E.pt[v] && E.pt[v] != HE_PT_ONE) cp_async16(sbase + 16u * slot(st, 3 * B + v), E.pt[v] + ptoff, stream);
        if (isq) {
            cp_async16(sbase + 16u * slot(st, 3 * B + V), E.src + (size_t)t * kp.n + kb, keep);
            if (!A.key) cp_async16(sbase + 16u * slot(st, 3 * B + V + 1), E.src + E.ps + off, keep);
        }
        pi++;
    };
    u128 a0[V][2], a1[V][2];
#pragma unroll
    for (int v = 0; v < V; v++)
#pragma unroll
        for (int e = 0; e < 2; e++) a0[v][e] = a1[v][e] = 0;
#pragma unroll
    for (int i = 0; i < RS - 1; i++) {
        if (pi < n_item) issue(i);
        cp_commit();
    }
    ulonglong2 kk0[B], kk1[B];
    int e = 0;
    for (int i = 0; i < n_amt; i++) {
        const famt A = P.amts[i];
        const int ks = A.g == 1 ? k : autom_index(k, A.g, kp.logn);
        const int sw = ks & 1;
        for (; e < A.e1; e++) {
            if (pi < n_item) issue((e + RS - 1) % RS);
            cp_commit();
            cp_wait<RS - 1>();
            const int st = e % RS;
            const fent E = P.ents[e];
            if (A.key && e == A.e0) {
#pragma unroll
                for (int j = 0; j < B; j++)
                    if (j < beta) {
                        kk0[j] = csm[slot(st, 2 * j)];
                        kk1[j] = csm[slot(st, 2 * j + 1)];
                    }
            }
            ulonglong2 p[V];
#pragma unroll
            for (int v = 0; v < V; v++) {
                const u64 *pp = E.pt[v];
                p[v] = pp == HE_PT_ONE ? make_ulonglong2(one, one) : (pp ? csm[slot(st, 3 * B + v)] : make_ulonglong2(0, 0));
            }
            u64 u00 = 0, u01 = 0, u10 = 0, u11 = 0;
            if (A.key) {
                u128 s0[2] = {0, 0}, s1[2] = {0, 0};
#pragma unroll
                for (int j = 0; j < B; j++)
                    if (j < beta) {
                        const ulonglong2 d = csm[slot(st, 2 * B + j)];
                        const u64 d0 = sw ? d.y : d.x, d1 = sw ? d.x : d.y;
                        s0[0] += (u128)d0 * kk0[j].x;
                        s0[1] += (u128)d1 * kk0[j].y;
                        s1[0] += (u128)d0 * kk1[j].x;
                        s1[1] += (u128)d1 * kk1[j].y;
                    }
                u00 = redc(s0[0], q, qi);
                u01 = redc(s0[1], q, qi);
                u10 = redc(s1[0], q, qi);
                u11 = redc(s1[1], q, qi);
            }
            if (isq) {                               // fold [P]_q phi(c0) (and [P]_q c1 at amount 0)
                const ulonglong2 cc = csm[slot(st, 3 * B + V)];
                const u64 c00 = sw ? cc.y : cc.x, c01 = sw ? cc.x : cc.y;
                u00 = add_mod(u00, mul_mont(c00, Pm, q, qi), q);
                u01 = add_mod(u01, mul_mont(c01, Pm, q, qi), q);
                if (!A.key) {
                    const ulonglong2 c1 = csm[slot(st, 3 * B + V + 1)];
                    u10 = mul_mont(c1.x, Pm, q, qi);
                    u11 = mul_mont(c1.y, Pm, q, qi);
                }
            }
#pragma unroll
            for (int v = 0; v < V; v++) {
                a0[v][0] += (u128)p[v].x * u00;
                a0[v][1] += (u128)p[v].y * u01;
                a1[v][0] += (u128)p[v].x * u10;
                a1[v][1] += (u128)p[v].y * u11;
            }
        }
    }
    cp_wait<0>();
#pragma unroll
    for (int v = 0; v < V; v++)
        if (v < P.nv) {
            st2(P.acc + ((size_t)(2 * v) * ext) * kp.n + off, redc(a0[v][0], q, qi), redc(a0[v][1], q, qi));
            st2(P.acc + ((size_t)(2 * v + 1) * ext) * kp.n + off, redc(a1[v][0], q, qi), redc(a1[v][1], q, qi));
        }
}

// ---- one-coefficient form: each thread handles one coefficient (8-byte loads), so a thread
// holds half the key, digit and accumulator words of the pair form and three blocks fit on an
// SM (24 warps to cover the key stream's latency).  Same arithmetic, same bits.
template <int V, int B>
__global__ void __launch_bounds__(TB, 3) ipmac1_kernel(KP kp, const fgrp *grps, int n_grp, int gb, const u64 *pmod) {
    pdl_wait();
    fgrp P;
    int tile, t, ptl;
    if (!grp_pos(kp, grps, n_grp, gb, P, tile, t, ptl, TB)) return;
    const int k = tile * TB + threadIdx.x;
    const int kl = blockIdx.y;
    const int nq = P.level + 1;
    const int ext = nq + kp.K;
    const int beta = P.beta;
    const bool isq = t < nq;
    const u64 q = kp.q[kl], qi = kp.qinv[kl], r2 = kp.r2[kl];
    const u64 one = to_mont(1, q, qi, r2);
    const u64 Pm = isq ? to_mont(pmod[kl], q, qi, r2) : 0;
    const size_t kstride = (size_t)(kp.L + 1 + kp.K) * kp.n;
    const size_t off = (size_t)t * kp.n + k, ptoff = (size_t)ptl * kp.n + k;
    const u64 stream = policy_evict_first(), keep = policy_evict_last();
    u128 a0[V], a1[V];
#pragma unroll
    for (int v = 0; v < V; v++) a0[v] = a1[v] = 0;
    const int n_amt = P.n_amt;
    famt A = n_amt > 0 ? P.amts[0] : famt{};
    fent E = (n_amt > 0 && A.e0 < A.e1) ? P.ents[A.e0] : fent{};
    for (int i = 0; i < n_amt; i++) {
        famt An{};
        fent En{};
        if (i + 1 < n_amt) {
            An = P.amts[i + 1];
            if (An.e0 < An.e1) En = P.ents[An.e0];
        }
        const int ks = A.g == 1 ? k : autom_index(k, A.g, kp.logn);
        u64 k0[B], k1[B];
        if (A.key) {
#pragma unroll
            for (int j = 0; j < B; j++)
                if (j < beta) {
                    const u64 *kp0 = A.key + (size_t)(2 * j) * kstride + (size_t)kl * kp.n + k;
                    k0[j] = ld_hint(kp0, stream);
                    k1[j] = ld_hint(kp0 + kstride, stream);
                }
        }
        for (int e = A.e0; e < A.e1; e++) {
            if (e > A.e0) E = P.ents[e];
            u64 p[V];
#pragma unroll
            for (int v = 0; v < V; v++) {
                const u64 *pp = E.pt[v];
                p[v] = pp == HE_PT_ONE ? one : (pp ? ld_hint(pp + ptoff, stream) : 0);
            }
            u64 c0 = 0, c1 = 0;
            if (isq) {
                c0 = ld_hint(E.src + (size_t)t * kp.n + ks, keep);
                if (!A.key) c1 = ld_hint(E.src + E.ps + off, keep);
            }
            u64 u0 = 0, u1 = 0;
            if (A.key) {
                u128 s0 = 0, s1 = 0;
#pragma unroll
                for (int j = 0; j < B; j++)
                    if (j < beta) {
                        const u64 d = ld_hint(E.D + ((size_t)j * ext + t) * kp.n + ks, keep);
                        s0 += (u128)d * k0[j];
                        s1 += (u128)d * k1[j];
                    }
                u0 = redc(s0, q, qi);
                u1 = redc(s1, q, qi);
            }
            if (isq) {                               // fold [P]_q phi(c0) (and [P]_q c1 at amount 0)
                u0 = add_mod(u0, mul_mont(c0, Pm, q, qi), q);
                if (!A.key) u1 = mul_mont(c1, Pm, q, qi);
            }
#pragma unroll
            for (int v = 0; v < V; v++) {
                a0[v] += (u128)p[v] * u0;
                a1[v] += (u128)p[v] * u1;
            }
        }
        A = An;
        E = En;
    }
#pragma unroll
    for (int v = 0; v < V; v++)
        if (v < P.nv) {
            P.acc[((size_t)(2 * v) * ext) * kp.n + off] = redc(a0[v], q, qi);
            P.acc[((size_t)(2 * v + 1) * ext) * kp.n + off] = redc(a1[v], q, qi);
        }
}
// ---- pre-keyed form: for a group whose every amount has one (source, output) term, the
// plaintext is folded into the key once (K' = K (.) pt, Montgomery) and into the unrotated part
// (P pt on the q-limbs), so per amount and coefficient the thread forms sum_j D_j K'_j plus
// c0 P pt directly into its 128-bit accumulators: no per-amount Montgomery reduction and no
// plaintext stream.  Terms are below p^2 < 2^100; a launch adds at most (beta + 1) per
// amount, far below 2^28 terms, so the 128-bit sums cannot wrap.  fent.pt[0] holds P pt
// ([l+1][n], Montgomery) or HE_PT_ONE for the integer 1 (then K' is the key itself).
// PF > 0: the K' tile (2 beta segments of 512 words, 4 KB each) of the amount PF ahead is
// requested into L2 by cp.async.bulk.prefetch (one thread per segment; a hint, no completion),
// so the amount's loads hit L2 without holding the words in registers.
template <int B, int MINB, bool PIPE, int PF = 0>
__global__ void __launch_bounds__(TB, MINB) ipmac_pk_kernel(KP kp, const fgrp *grps, int n_grp, int gb,
                                                            const u64 *pmod) {
    pdl_wait();
    fgrp P;
    int tile, t, ptl;
    if (!grp_pos(kp, grps, n_grp, gb, P, tile, t, ptl)) return;
    const int k = 2 * (tile * TB + threadIdx.x);
    const int kl = blockIdx.y;
    const int nq = P.level + 1;
    const int ext = nq + kp.K;
    const int beta = P.beta;
    const bool isq = t < nq;
    const u64 q = kp.q[kl], qi = kp.qinv[kl], r2 = kp.r2[kl];
    const u64 Pm = isq ? to_mont(pmod[kl], q, qi, r2) : 0;
    const size_t kstride = (size_t)(kp.L + 1 + kp.K) * kp.n;
    const size_t off = (size_t)t * kp.n + k;
    const u64 stream = policy_evict_first(), keep = policy_evict_last();
    u128 a00 = 0, a01 = 0, a10 = 0, a11 = 0;
    const int n_amt = P.n_amt;
    famt A = n_amt > 0 ? P.amts[0] : famt{};
    fent E = (n_amt > 0 && A.e0 < A.e1) ? P.ents[A.e0] : fent{};
    // PIPE: the next amount's key words are requested before this amount computes
    ulonglong2 kk0[B], kk1[B];
    auto load_key = [&](const famt &X, ulonglong2 (&k0)[B], ulonglong2 (&k1)[B]) {
        if (X.key) {
#pragma unroll
            for (int j = 0; j < B; j++)
                if (j < beta) {
                    const u64 *kp0 = X.key + (size_t)(2 * j) * kstride + (size_t)kl * kp.n + k;
                    k0[j] = ld2_hint(kp0, stream);
                    k1[j] = ld2_hint(kp0 + kstride, stream);
                }
        }
    };
    if (PIPE && n_amt > 0) load_key(A, kk0, kk1);
    for (int i = 0; i < n_amt; i++) {
        if (PF > 0 && (int)threadIdx.x < 2 * beta && i + PF < n_amt) {
            const u64 *kf = P.amts[i + PF].key;
            if (kf) {
                const u64 *src = kf + (size_t)threadIdx.x * kstride + (size_t)kl * kp.n + (size_t)tile * (2 * TB);
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(2u * TB * 8u) : "memory");
            }
        }
        famt An{};
        fent En{};
        if (i + 1 < n_amt) {
            An = P.amts[i + 1];
            if (An.e0 < An.e1) En = P.ents[An.e0];
        }
        ulonglong2 kn0[B], kn1[B];
        if (PIPE) load_key(An, kn0, kn1);
        else load_key(A, kk0, kk1);
        if (A.e0 < A.e1) {
            const int ks = A.g == 1 ? k : autom_index(k, A.g, kp.logn);
            const int sw = ks & 1, kb = ks & ~1;
            if (A.key) {
#pragma unroll
                for (int j = 0; j < B; j++)
                    if (j < beta) {
                        const ulonglong2 d = ld2_hint(E.D + ((size_t)j * ext + t) * kp.n + kb, keep);
                        const u64 d0 = sw ? d.y : d.x, d1 = sw ? d.x : d.y;
                        a00 += (u128)d0 * kk0[j].x;
                        a01 += (u128)d1 * kk0[j].y;
                        a10 += (u128)d0 * kk1[j].x;
                        a11 += (u128)d1 * kk1[j].y;
                    }
            }
            if (isq) {
                const ulonglong2 pp = E.pt[0] == HE_PT_ONE ? make_ulonglong2(Pm, Pm)
                                                           : ld2_hint(E.pt[0] + (size_t)t * kp.n + k, stream);
                const ulonglong2 cc = ld2_hint(E.src + (size_t)t * kp.n + kb, keep);
                a00 += (u128)(sw ? cc.y : cc.x) * pp.x;
                a01 += (u128)(sw ? cc.x : cc.y) * pp.y;
                if (!A.key) {
                    const ulonglong2 c1 = ld2_hint(E.src + E.ps + off, keep);
                    a10 += (u128)c1.x * pp.x;
                    a11 += (u128)c1.y * pp.y;
                }
            }
        }
        if (PIPE) {
#pragma unroll
            for (int j = 0; j < B; j++) { kk0[j] = kn0[j]; kk1[j] = kn1[j]; }
        }
        A = An;
        E = En;
    }
    st2(P.acc + off, redc(a00, q, qi), redc(a01, q, qi));
    st2(P.acc + (size_t)ext * kp.n + off, redc(a10, q, qi), redc(a11, q, qi));
}

// ---- pre-keyed form fed by a TMA ring with per-stage release: a producer warp copies each
// keyed amount's K' tile (2 beta segments of 512 words) by cp.async.bulk into one of PKT_STAGES
// shared-memory stages; the eight consumer warps wait on the stage's "full" mbarrier, take their
// key words into registers and release the stage on its "empty" mbarrier (one arrival per warp)
// before they compute, so warps run up to PKT_STAGES amounts apart and no block barrier paces
// the stream.  The producer waits on "empty" before refilling a stage.  Every wait is bounded:
// a consumer whose wait gives up sets *err and a shared abort flag that stops every warp; the
// block then waits (bounded) for the copies it issued before its shared memory goes away.
constexpr int PKT_STAGES = 3;                       // 3 x 32 KB at beta = 4: two blocks per SM
constexpr int PKT_THREADS = TB + 32;                // eight consumer warps and the producer warp

__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__global__ void __launch_bounds__(PKT_THREADS, 2) ipmac_pkt_kernel(KP kp, const fgrp *grps, int n_grp, int gb,
                                                                   int *err, const u64 *pmod) {
    pdl_wait();
    constexpr int NS = PKT_STAGES, B = 4;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_abort;
    __shared__ int s_issued;
    fgrp P;
    int tile, t, ptl;
    if (!grp_pos(kp, grps, n_grp, gb, P, tile, t, ptl)) return;   // block-uniform
    const int beta = P.beta, n_amt = P.n_amt, seg = 2 * beta;
    const famt *amts = P.amts;
    u64 *kbuf = (u64 *)smem_raw;                                // [NS][2 beta][TMA_TILE]
    uint64_t *full = (uint64_t *)(kbuf + (size_t)NS * 2 * B * TMA_TILE);
    uint64_t *empty = full + NS;
    const int k0 = tile * TMA_TILE;
    const int kl = blockIdx.y;
    const int nq = P.level + 1;
    const int ext = nq + kp.K;
    const size_t kstride = (size_t)(kp.L + 1 + kp.K) * kp.n;
    const u64 stream = policy_evict_first(), keep = policy_evict_last();
    const bool producer = threadIdx.x >= TB;
    if (threadIdx.x == 0) {
        s_abort = *(volatile int *)err;            // an earlier block already gave up: skip the work
        s_issued = 0;
        for (int st = 0; st < NS; st++) {
            mbar_init(smem_u32(&full[st]), 1);
            mbar_init(smem_u32(&empty[st]), TB / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (s_abort) return;                           // block-uniform after the barrier
    if (producer) {
        if (threadIdx.x == TB) {                   // one lane issues; the rest of the warp idles
            const unsigned bytes = (unsigned)seg * TMA_TILE * 8;
            int u = 0;
            for (int i = 0; i < n_amt; i++) {
                if (!amts[i].key) continue;
                const int st = u % NS;
                if (u >= NS && !mbar_wait_bounded(smem_u32(&empty[st]), ((u / NS) - 1) & 1)) break;
                if (*(volatile int *)&s_abort) break;
                const unsigned bar = smem_u32(&full[st]);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(bar, bytes);
                const u64 *kb = amts[i].key + (size_t)kl * kp.n + k0;
                for (int sgi = 0; sgi < seg; sgi++)
                    tma_load(smem_u32(kbuf + ((size_t)st * 2 * B + sgi) * TMA_TILE), kb + (size_t)sgi * kstride,
                             TMA_TILE * 8, bar, stream);
                u++;
                *(volatile int *)&s_issued = u;
            }
        }
    } else {
        const int k = k0 + 2 * threadIdx.x;
        const bool isq = t < nq;
        const u64 q = kp.q[kl], qi = kp.qinv[kl], r2 = kp.r2[kl];
        const u64 Pm = isq ? to_mont(pmod[kl], q, qi, r2) : 0;
        const size_t off = (size_t)t * kp.n + k;
        u128 a00 = 0, a01 = 0, a10 = 0, a11 = 0;
        int u = 0;
        for (int i = 0; i < n_amt; i++) {
            const famt A = amts[i];
            const bool has = A.e0 < A.e1;
            if (!A.key && !has) continue;
            const fent E = has ? P.ents[A.e0] : fent{};
            const int ks = A.g == 1 ? k : autom_index(k, A.g, kp.logn);
            const int sw = ks & 1, kb = ks & ~1;
            if (A.key) {
                const int st = u % NS;
                // warp-uniform decisions: every lane waits (each takes the barrier's acquire),
                // then the warp votes, so no lane leaves the loop alone
                if (__any_sync(0xffffffffu, *(volatile int *)&s_abort)) break;
                const bool ok = mbar_wait_bounded(smem_u32(&full[st]), (u / NS) & 1);
                if (!__all_sync(0xffffffffu, ok)) {
                    if ((threadIdx.x & 31) == 0) {
                        atomicExch(err, 1);
                        *(volatile int *)&s_abort = 1;
                    }
                    break;
                }
                ulonglong2 kk0[B], kk1[B];
                const u64 *kt = kbuf + (size_t)st * 2 * B * TMA_TILE + 2 * threadIdx.x;
#pragma unroll
                for (int j = 0; j < B; j++)
                    if (j < beta) {
                        kk0[j] = *(const ulonglong2 *)(kt + (size_t)(2 * j) * TMA_TILE);
                        kk1[j] = *(const ulonglong2 *)(kt + (size_t)(2 * j + 1) * TMA_TILE);
                    }
                __syncwarp();
                if ((threadIdx.x & 31) == 0) mbar_arrive(smem_u32(&empty[st]));   // stage released
                u++;
                if (has) {
#pragma unroll
                    for (int j = 0; j < B; j++)
                        if (j < beta) {
                            const ulonglong2 d = ld2_hint(E.D + ((size_t)j * ext + t) * kp.n + kb, keep);
                            const u64 d0 = sw ? d.y : d.x, d1 = sw ? d.x : d.y;
                            a00 += (u128)d0 * kk0[j].x;
                            a01 += (u128)d1 * kk0[j].y;
                            a10 += (u128)d0 * kk1[j].x;
                            a11 += (u128)d1 * kk1[j].y;
                        }
                }
            }
            if (isq && has) {
                const ulonglong2 pp = E.pt[0] == HE_PT_ONE ? make_ulonglong2(Pm, Pm)
                                                           : ld2_hint(E.pt[0] + (size_t)t * kp.n + k, stream);
                const ulonglong2 cc = ld2_hint(E.src + (size_t)t * kp.n + kb, keep);
                a00 += (u128)(sw ? cc.y : cc.x) * pp.x;
                a01 += (u128)(sw ? cc.x : cc.y) * pp.y;
                if (!A.key) {
                    const ulonglong2 c1 = ld2_hint(E.src + E.ps + off, keep);
                    a10 += (u128)c1.x * pp.x;
                    a11 += (u128)c1.y * pp.y;
                }
            }
        }
        if (!*(volatile int *)&s_abort) {
            st2(P.acc + off, redc(a00, q, qi), redc(a01, q, qi));
            st2(P.acc + (size_t)ext * kp.n + off, redc(a10, q, qi), redc(a11, q, qi));
        }
    }
    __syncthreads();
    if (s_abort && threadIdx.x == 0) {
        // the last copy issued into each stage lands (bounded) before the shared memory goes away
        const int issued = s_issued;
        for (int u = issued - NS < 0 ? 0 : issued - NS; u < issued; u++)
            mbar_wait_bounded(smem_u32(&full[u % NS]), (u / NS) & 1);
    }
}

// ---- pre-keyed, one coefficient per thread: the pair form's arithmetic with half its registers
// per thread, so more blocks per SM keep more key words in flight (8-byte loads; a warp still
// reads 256 contiguous bytes of every key word).  Same terms, same 128-bit sums, same bits.
template <int B, int MINB>
__global__ void __launch_bounds__(TB, MINB) ipmac_pk1_kernel(KP kp, const fgrp *grps, int n_grp, int gb,
                                                             const u64 *pmod) {
    pdl_wait();
    fgrp P;
    int tile, t, ptl;
    if (!grp_pos(kp, grps, n_grp, gb, P, tile, t, ptl, TB)) return;
    const int k = tile * TB + threadIdx.x;
    const int kl = blockIdx.y;
    const int nq = P.level + 1;
    const int ext = nq + kp.K;
    const int beta = P.beta;
    const bool isq = t < nq;
    const u64 q = kp.q[kl], qi = kp.qinv[kl], r2 = kp.r2[kl];
    const u64 Pm = isq ? to_mont(pmod[kl], q, qi, r2) : 0;
    const size_t kstride = (size_t)(kp.L + 1 + kp.K) * kp.n;
    const size_t off = (size_t)t * kp.n + k;
    const u64 stream = policy_evict_first(), keep = policy_evict_last();
    u128 a0 = 0, a1 = 0;
    const int n_amt = P.n_amt;
    famt A = n_amt > 0 ? P.amts[0] : famt{};
    fent E = (n_amt > 0 && A.e0 < A.e1) ? P.ents[A.e0] : fent{};
    for (int i = 0; i < n_amt; i++) {
        famt An{};
        fent En{};
        if (i + 1 < n_amt) {
            An = P.amts[i + 1];
            if (An.e0 < An.e1) En = P.ents[An.e0];
        }
        if (A.e0 < A.e1) {
            const int ks = A.g == 1 ? k : autom_index(k, A.g, kp.logn);
            if (A.key) {
                u64 k0[B], k1[B], d[B];
#pragma unroll
                for (int j = 0; j < B; j++)
                    if (j < beta) {
                        const u64 *kp0 = A.key + (size_t)(2 * j) * kstride + (size_t)kl * kp.n + k;
                        k0[j] = ld_hint(kp0, stream);
                        k1[j] = ld_hint(kp0 + kstride, stream);
                        d[j] = ld_hint(E.D + ((size_t)j * ext + t) * kp.n + ks, keep);
                    }
#pragma unroll
                for (int j = 0; j < B; j++)
                    if (j < beta) {
                        a0 += (u128)d[j] * k0[j];
                        a1 += (u128)d[j] * k1[j];
                    }
            }
            if (isq) {
                const u64 pp = E.pt[0] == HE_PT_ONE ? Pm : ld_hint(E.pt[0] + (size_t)t * kp.n + k, stream);
                a0 += (u128)ld_hint(E.src + (size_t)t * kp.n + ks, keep) * pp;
                if (!A.key) a1 += (u128)ld_hint(E.src + E.ps + off, keep) * pp;
            }
        }
        A = An;
        E = En;
    }
    P.acc[off] = redc(a0, q, qi);
    P.acc[(size_t)ext * kp.n + off] = redc(a1, q, qi);
}

// K'[2j + c] = K[2j + c] (.) pt on the limbs of Q_l u P (key layout: global prime index) and
// Ppt = [P]_q (.) pt on the q-limbs ([l+1][n]); pt holds pt_level + 1 q-limbs then the p-limbs.
__global__ void prekey_kernel(KP kp, const u64 *key, const u64 *pt, int level, int pt_level, int beta, u64 *Kp,
                              u64 *Ppt, const u64 *pmod) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int t = blockIdx.y, z = blockIdx.z;
    const int nq = level + 1;
    const int kl = t < nq ? t : kp.L + 1 + (t - nq);
    const int ptl = t < nq ? t : pt_level + 1 + (t - nq);
    const u64 q = kp.q[kl], qi = kp.qinv[kl], r2 = kp.r2[kl];
    const u64 p = pt[(size_t)ptl * kp.n + k];
    const size_t kstride = (size_t)(kp.L + 1 + kp.K) * kp.n;
    if (z < 2 * beta) {
        const size_t i = (size_t)z * kstride + (size_t)kl * kp.n + k;
        Kp[i] = mul_mont(key[i], p, q, qi);
    } else if (t < nq) {
        Ppt[(size_t)t * kp.n + k] = mul_mont(to_mont(pmod[kl], q, qi, r2), p, q, qi);
    }
}

// ==== fused key-switch + MAC kernels: end

// acc = sum_terms K_term * x_term (+ c on poly 0) over limbs 0..level, x of any higher level
// (the drop is implicit); per-limb residues of the integer constants are passed by value, already
// in Montgomery form, so one REDC of the 128-bit sum finishes it.
struct LincombArgs {
    const u64 *x[HE_LC_MAX];
    size_t ps[HE_LC_MAX];
    u64 res[HE_LC_MAX][HE_LC_LIMBS];
    u64 cst[HE_LC_LIMBS];
    int n_terms;
};
__global__ void lincomb_kernel(KP kp, LincombArgs A, u64 *out, size_t out_ps) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int i = blockIdx.y;
    const int c = blockIdx.z;
    const u64 q = kp.q[i], qi = kp.qinv[i];
    u128 acc = 0;
    for (int t = 0; t < A.n_terms; t++) {
        const u64 x = A.x[t][c * A.ps[t] + (size_t)i * kp.n + k];
        acc += (u128)x * A.res[t][i];
    }
    u64 r = redc(acc, q, qi);
    if (c == 0) r = add_mod(r, A.cst[i], q);
    out[c * out_ps + (size_t)i * kp.n + k] = r;
}

// tensor products of several pairs at one level (blockIdx.z), operands passed by value
struct TensorInline {
    const u64 *a[HE_INLINE_ITEMS], *b[HE_INLINE_ITEMS];
    size_t pa[HE_INLINE_ITEMS], pb[HE_INLINE_ITEMS];
};
__global__ void tensor_batch_kernel(KP kp, TensorInline T, u64 *d, size_t dstride, int level) {
    pdl_wait();
    const int k = blockIdx.x * TB + threadIdx.x;
    const int i = blockIdx.y, z = blockIdx.z;
    const u64 q = kp.q[i], qi = kp.qinv[i], r2 = kp.r2[i];
    const size_t off = (size_t)i * kp.n + k;
    const size_t ps = (size_t)(level + 1) * kp.n;
    const u64 *a = T.a[z], *b = T.b[z];
    u64 *dz = d + z * dstride;
    u64 a0 = a[off], a1 = a[T.pa[z] + off];
    u64 b0 = to_mont(b[off], q, qi, r2), b1 = to_mont(b[T.pb[z] + off], q, qi, r2);
    dz[off] = redc((u128)a0 * b0, q, qi);
    dz[ps + off] = redc((u128)a0 * b1 + (u128)a1 * b0, q, qi);
    dz[2 * ps + off] = redc((u128)a1 * b1, q, qi);
}

__global__ void tensor_kernel(KP kp, const u64 *a, size_t pa, const u64 *b, size_t pb, u64 *d,
                              int level) {
    pdl_wait();
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
    pdl_wait();
    size_t i = (size_t)blockIdx.x * TB + threadIdx.x;
    if (i >= words) return;
    dst[blockIdx.y * dps + i] = src[blockIdx.y * sps + i];
}

__global__ void bench_modmul_kernel(u64 q, u64 qinv, int iters, u64 *sink) {
    pdl_wait();
    u64 x = threadIdx.x + 12345, y = blockIdx.x + 777;
    for (int it = 0; it < iters; it++) {
        x = redc((u128)x * y, q, qinv);
        y = redc((u128)y * x, q, qinv);
    }
    if (x == 0xdeadbeef) sink[0] = y;
}

// Throughput of 64 x 64 -> 128-bit multiply-accumulates (the fused key-switch kernels' inner
// operation): eight independent chains per thread, acc_c += a_c b with a_c taken from the low
// word of the chain's last sum, so every chain is a true dependency and nothing can be hoisted.
__global__ void bench_mac_kernel(u64 b, int iters, u64 *sink) {
    pdl_wait();
    u64 a[8];
    u128 acc[8];
#pragma unroll
    for (int c = 0; c < 8; c++) {
        a[c] = (u64)threadIdx.x * 0x9E3779B97F4A7C15ull + c + blockIdx.x;
        acc[c] = a[c];
    }
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < 8; c++) {
            acc[c] += (u128)a[c] * b;
            a[c] = (u64)acc[c] | 1;
        }
    }
    u64 x = 0;
#pragma unroll
    for (int c = 0; c < 8; c++) x ^= (u64)acc[c] ^ (u64)(acc[c] >> 64);
    if (x == 0x0123456789abcdefull) sink[0] = x;
}

}  // namespace

// ================================================================================= launchers
// Every launch goes through cudaLaunchKernelEx with the programmatic-serialisation attribute
// (process-wide switch, HE_OPT_PDL); errors surface through cudaGetLastError as for <<<>>>.
static std::atomic<int> g_pdl{0};
void he_set_pdl(int on) { g_pdl.store(on ? 1 : 0); }
int he_get_pdl() { return g_pdl.load(); }
template <typename... KArgs, typename... Args>
static cudaError_t pdl_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = g_pdl.load();
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

#define LAUNCH_CHECK()                                        \
    do {                                                      \
        he_count_launch();                                    \
        cudaError_t _e = cudaGetLastError();                  \
        if (_e != cudaSuccess) {                              \
            he_set_error("kernel launch: %s", cudaGetErrorString(_e)); \
            return HE_ECUDA;                                  \
        }                                                     \
    } while (0)

// the one-pass cluster NTT of a 2^16 ring: cluster dimension at launch (16 is a non-portable
// size the kernel opts in to), dynamic shared memory opted in once per device
template <bool INV, bool RS, int CL>
static int ntt_cluster(const he_ctx *ctx, const ntt_job &job, const RescaleFuse &F, cudaStream_t s) {
    using S = NcShape<CL>;
    static std::mutex mu;
    static bool ready[64] = {};
    int dev = 0;
    HE_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { he_set_error("device ordinal %d out of range", dev); return HE_EINVAL; }
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!ready[dev]) {
            HE_CHECK_CUDA(cudaFuncSetAttribute(ntt16_cluster<INV, RS, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               S::SMEM * (int)sizeof(u64)));
            if (CL > 8)
                HE_CHECK_CUDA(cudaFuncSetAttribute(ntt16_cluster<INV, RS, CL>,
                                                   cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
            ready[dev] = true;
        }
    }
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = g_pdl.load();
    at[1].id = cudaLaunchAttributeClusterDimension;
    at[1].val.clusterDim.x = CL;
    at[1].val.clusterDim.y = 1;
    at[1].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(CL, job.nl, job.npoly);
    cfg.blockDim = dim3(S::T);
    cfg.dynamicSmemBytes = S::SMEM * sizeof(u64);
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    cudaLaunchKernelEx(&cfg, ntt16_cluster<INV, RS, CL>, ctx->kp, job, F);
    LAUNCH_CHECK();
    return HE_OK;
}

template <bool INV, bool RS>
static int ntt_onepass_launch(const he_ctx *ctx, const ntt_job &job, const RescaleFuse &F, cudaStream_t s) {
    return ctx->ntt_form == HE_NTT_ONEPASS8 ? ntt_cluster<INV, RS, 8>(ctx, job, F, s)
                                            : ntt_cluster<INV, RS, 16>(ctx, job, F, s);
}

static bool ntt_onepass(const he_ctx *ctx) {
    return ctx->logn == 16 && (ctx->ntt_form == HE_NTT_ONEPASS || ctx->ntt_form == HE_NTT_ONEPASS8);
}
// the two-pass forward transform without per-butterfly corrections (every prime below 2^57)
static bool ntt_nc(const he_ctx *ctx) {
    return ctx->small_primes && (ctx->ntt_form == HE_NTT_TWOPASS || ctx->ntt_form == HE_NTT_TWOPASS_SHUFFLE);
}
// the row pass with its transposes by warp shuffles
static bool ntt_shfl(const he_ctx *ctx) { return ctx->ntt_form == HE_NTT_TWOPASS_SHUFFLE; }

int k_ntt(const he_ctx *ctx, const ntt_job &job, bool inverse, cudaStream_t s) {
    if (job.nl <= 0 || job.npoly <= 0) return HE_OK;
    const int R = ctx->n / ROW;
    if (ntt_onepass(ctx)) {
        const double limbs = (double)job.nl * job.npoly;
        TraceScope tr("ntt", s, limbs * 2.0 * ctx->n * 8, limbs * (ctx->n / 2) * ctx->logn);
        return inverse ? ntt_onepass_launch<true, false>(ctx, job, RescaleFuse{}, s)
                       : ntt_onepass_launch<false, false>(ctx, job, RescaleFuse{}, s);
    }
    if (ctx->logn >= 12 && ctx->logn <= 16) {
        const double limbs = (double)job.nl * job.npoly;
        TraceScope tr("ntt", s, limbs * 2.0 * ctx->n * 8, limbs * (ctx->n / 2) * ctx->logn);
        const int TC = 4096 / R;
        dim3 gA(ROW / TC, job.nl, job.npoly), gB(R / 16, job.nl, job.npoly);
        if (ntt_shfl(ctx)) {
            if (!inverse) {
                if (ntt_nc(ctx)) {
                    pdl_launch(ntt16_cols<false, false, true>, gA, 256, 0, s, ctx->kp, job, RescaleFuse{});
                    LAUNCH_CHECK();
                    pdl_launch(ntt16_rows_shfl<false, false, true>, gB, 256, 0, s, ctx->kp, job, RescaleFuse{});
                } else {
                    pdl_launch(ntt16_cols<false>, gA, 256, 0, s, ctx->kp, job, RescaleFuse{});
                    LAUNCH_CHECK();
                    pdl_launch(ntt16_rows_shfl<false>, gB, 256, 0, s, ctx->kp, job, RescaleFuse{});
                }
                LAUNCH_CHECK();
            } else {
                pdl_launch(ntt16_rows_shfl<true>, gB, 256, 0, s, ctx->kp, job, RescaleFuse{});
                LAUNCH_CHECK();
                pdl_launch(ntt16_cols<true>, gA, 256, 0, s, ctx->kp, job, RescaleFuse{});
                LAUNCH_CHECK();
            }
        } else if (!inverse && ntt_nc(ctx)) {
            pdl_launch(ntt16_cols<false, false, true>, gA, 256, 0, s, ctx->kp, job, RescaleFuse{});
            LAUNCH_CHECK();
            pdl_launch(ntt16_rows<false, false, true>, gB, 256, 0, s, ctx->kp, job, RescaleFuse{});
            LAUNCH_CHECK();
        } else if (!inverse) {
            pdl_launch(ntt16_cols<false>, gA, 256, 0, s, ctx->kp, job, RescaleFuse{});
            LAUNCH_CHECK();
            pdl_launch(ntt16_rows<false>, gB, 256, 0, s, ctx->kp, job, RescaleFuse{});
            LAUNCH_CHECK();
        } else {
            pdl_launch(ntt16_rows<true>, gB, 256, 0, s, ctx->kp, job, RescaleFuse{});
            LAUNCH_CHECK();
            pdl_launch(ntt16_cols<true>, gA, 256, 0, s, ctx->kp, job, RescaleFuse{});
            LAUNCH_CHECK();
        }
        return HE_OK;
    }
    dim3 gA(ROW / NTT_TC, job.nl, job.npoly), gB((R + 7) / 8, job.nl, job.npoly);
    size_t smA = (size_t)R * NTT_TC * sizeof(u64);
    const double limbs = (double)job.nl * job.npoly;
    TraceScope tr("ntt", s, limbs * 2.0 * ctx->n * 8, limbs * (ctx->n / 2) * ctx->logn);
    if (!inverse) {
        pdl_launch(ntt_cols<false>, gA, 256, smA, s, ctx->kp, job);
        LAUNCH_CHECK();
        pdl_launch(ntt_rows<false>, gB, 256, 0, s, ctx->kp, job);
        LAUNCH_CHECK();
    } else {
        pdl_launch(ntt_rows<true>, gB, 256, 0, s, ctx->kp, job);
        LAUNCH_CHECK();
        pdl_launch(ntt_cols<true>, gA, 256, smA, s, ctx->kp, job);
        LAUNCH_CHECK();
    }
    return HE_OK;
}

int k_reduce_int(const he_ctx *ctx, const int64_t *m, u64 *out, int nlimbs, int nq, bool mont,
                 cudaStream_t s) {
    pdl_launch(reduce_int_kernel, dim3(ctx->n / TB, nlimbs), TB, 0, s, ctx->kp, m, out, nq, mont ? 1 : 0);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_to_mont(const he_ctx *ctx, u64 *x, int nlimbs, int nq, int npoly, size_t pstride,
              cudaStream_t s) {
    pdl_launch(mont_kernel, dim3(ctx->n / TB, nlimbs, npoly), TB, 0, s, ctx->kp, x, nq, pstride, 1);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_from_mont(const he_ctx *ctx, u64 *x, int nlimbs, int nq, int npoly, size_t pstride,
                cudaStream_t s) {
    pdl_launch(mont_kernel, dim3(ctx->n / TB, nlimbs, npoly), TB, 0, s, ctx->kp, x, nq, pstride, 0);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_sample_uniform(const he_ctx *ctx, u64 seed, u64 stream, u64 *out, int nlimbs, int nq,
                     cudaStream_t s) {
    pdl_launch(sample_uniform_kernel, dim3(ctx->n / TB, nlimbs), TB, 0, s, ctx->kp, seed, stream, out, nq);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_sample_cbd(const he_ctx *ctx, u64 seed, u64 stream, int64_t *out, cudaStream_t s) {
    pdl_launch(sample_cbd_kernel, ctx->n / TB, TB, 0, s, ctx->n, seed, stream, out);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_sample_ternary(const he_ctx *ctx, u64 seed, u64 stream, int64_t *out, cudaStream_t s) {
    pdl_launch(sample_ternary_kernel, ctx->n / TB, TB, 0, s, ctx->n, seed, stream, out);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_permute(const he_ctx *ctx, const u64 *in, u64 *out, int nlimbs, u64 g, cudaStream_t s) {
    pdl_launch(permute_kernel, dim3(ctx->n / TB, nlimbs), TB, 0, s, ctx->kp, in, out, g);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_keygen_combine(const he_ctx *ctx, u64 *b, u64 *a, const u64 *e, const u64 *s_eval,
                     const u64 *sp_eval, int digit, cudaStream_t s) {
    int lo = digit * ctx->alpha, hi = std::min(lo + ctx->alpha, ctx->L + 1);
    pdl_launch(keygen_combine_kernel, dim3(ctx->n / TB, ctx->np), TB, 0, s, 
        ctx->kp, b, a, e, s_eval, sp_eval, ctx->d_consts, lo, hi);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_encrypt_combine(const he_ctx *ctx, u64 *c0, const u64 *a, const u64 *e, const u64 *m,
                      int level, cudaStream_t s) {
    pdl_launch(encrypt_combine_kernel, dim3(ctx->n / TB, level + 1), TB, 0, s, ctx->kp, c0, a, e, m, ctx->d_s);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_decrypt_dot(const he_ctx *ctx, const he_ct *ct, u64 *out, int nlimbs, cudaStream_t s) {
    pdl_launch(decrypt_dot_kernel, dim3(ctx->n / TB, nlimbs), TB, 0, s, ctx->kp, ct->d, ct->pstride, ctx->d_s, out);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_add(const he_ctx *ctx, he_ct *acc, const he_ct *b, bool sub, cudaStream_t s) {
    pdl_launch(addsub_kernel, dim3(ctx->n / TB, acc->level + 1, 2), TB, 0, s, 
        ctx->kp, acc->d, acc->pstride, b->d, b->pstride, sub ? 1 : 0);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_add_raw(const he_ctx *ctx, u64 *a, size_t pa, const u64 *b, size_t pb, int nlimbs, int npoly,
              bool sub, cudaStream_t s) {
    pdl_launch(addsub_kernel, dim3(ctx->n / TB, nlimbs, npoly), TB, 0, s, ctx->kp, a, pa, b, pb, sub ? 1 : 0);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_mul_scalar(const he_ctx *ctx, he_ct *ct, const u64 *res, const u64 *shoup, cudaStream_t s) {
    pdl_launch(mul_scalar_kernel, dim3(ctx->n / TB, ct->level + 1, 2), TB, 0, s, ctx->kp, ct->d, ct->pstride, res, shoup);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_sample_sparse(const he_ctx *ctx, u64 seed, u64 stream, int h, int32_t *perm, int64_t *out, cudaStream_t s) {
    pdl_launch(sample_sparse_kernel, 1, 1024, 0, s, ctx->n, seed, stream, h, perm, out);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_modraise(const he_ctx *ctx, const u64 *in_coef, u64 *out, size_t pstride, int nlimbs, cudaStream_t s) {
    pdl_launch(modraise_kernel, dim3(ctx->n / TB, nlimbs, 2), TB, 0, s, ctx->kp, in_coef, out, pstride);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_monomial(const he_ctx *ctx, u64 *d, size_t pstride, int nlimbs, u64 e, cudaStream_t s) {
    pdl_launch(monomial_kernel, dim3(ctx->n / TB, nlimbs, 2), TB, 0, s, ctx->kp, d, pstride, e);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_add_const(const he_ctx *ctx, he_ct *ct, const u64 *res_dev, cudaStream_t s) {
    pdl_launch(add_const_kernel, dim3(ctx->n / TB, ct->level + 1), TB, 0, s, ctx->kp, ct->d, res_dev);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_zero(u64 *p, size_t words, cudaStream_t s) {
    if (!words) return HE_OK;
    pdl_launch(zero_kernel, (unsigned)((words + TB - 1) / TB), TB, 0, s, p, words);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_copy_limbs(u64 *dst, size_t dps, const u64 *src, size_t sps, size_t words, int npoly,
                 cudaStream_t s) {
    pdl_launch(copy_kernel, dim3((unsigned)((words + TB - 1) / TB), npoly), TB, 0, s, dst, dps, src, sps, words);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_modup_batch(const he_ctx *ctx, const modup_src *d_tab, int n_src, u64 *tmp, int level, cudaStream_t s) {
    if (n_src <= 0) return HE_OK;
    const int nq = level + 1, ext = nq + ctx->K;
    const int beta = (level + ctx->alpha) / ctx->alpha;
    if (beta > 16 || ctx->alpha > 16 || n_src > 65535) {
        he_set_error("modup: at most 16 digits of at most 16 primes, 65535 sources");
        return HE_EINVAL;
    }
    const size_t words = (size_t)nq * ctx->n;
    pdl_launch(gather_c1_kernel, dim3((unsigned)((words + TB - 1) / TB), n_src), TB, 0, s, d_tab, tmp, words);
    LAUNCH_CHECK();
    ntt_job ji{tmp, words, 0, nq, nq, 0, n_src, 0};
    HE_TRY(k_ntt(ctx, ji, true, s));
    ModupArgs A;
    A.x_coef = tmp;
    A.x_ntt = nullptr;
    A.D = nullptr;
    A.level = level;
    A.alpha = ctx->alpha;
    for (int j = 0; j < beta; j++) A.tab[j] = ctx->modup[level][j].d;
    {
        TraceScope tr("modup", s, (double)n_src * (nq + beta * ext) * ctx->n * 8,
                      (double)n_src * (nq + (double)beta * (ext - ctx->alpha) * ctx->alpha) * ctx->n);
#define GO(C) pdl_launch(modup_batch_kernel<C>, dim3(ctx->n / TB, beta, n_src), TB, 0, s, ctx->kp, A, d_tab)
        CAP_SWITCH(ctx->alpha, GO)
#undef GO
        LAUNCH_CHECK();
    }
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
#define GO(C) pdl_launch(modup_kernel<C>, dim3(ctx->n / TB, beta), TB, 0, s, ctx->kp, A)
    CAP_SWITCH(ctx->alpha, GO)
#undef GO
    LAUNCH_CHECK();
    return HE_OK;
}

int k_modup_strided(const he_ctx *ctx, const u64 *x_coef, size_t xs, const u64 *x_ntt, size_t ns, u64 *D, size_t ds,
                    int m, int level, cudaStream_t s) {
    if (m <= 0) return HE_OK;
    ModupArgs A;
    A.x_coef = x_coef;
    A.x_ntt = x_ntt;
    A.D = D;
    A.level = level;
    A.alpha = ctx->alpha;
    const int beta = (level + ctx->alpha) / ctx->alpha;
    if (beta > 16 || ctx->alpha > 16 || m > 65535) {
        he_set_error("modup: at most 16 digits of at most 16 primes, 65535 sources");
        return HE_EINVAL;
    }
    for (int j = 0; j < beta; j++) A.tab[j] = ctx->modup[level][j].d;
    const double nq = level + 1, ext = nq + ctx->K;
    TraceScope tr("modup", s, (double)m * (nq + beta * ext) * ctx->n * 8,
                  (double)m * (nq + (double)beta * (ext - ctx->alpha) * ctx->alpha) * ctx->n);
#define GO(C) pdl_launch(modup_strided_kernel<C>, dim3(ctx->n / TB, beta, m), TB, 0, s, ctx->kp, A, xs, ns, ds)
    CAP_SWITCH(ctx->alpha, GO)
#undef GO
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
    const int beta = (level + ctx->alpha) / ctx->alpha;
#define GO(C) pdl_launch(ip_kernel<C>, dim3(ctx->n / TB, level + 1 + ctx->K, n_items), TB, 0, s, ctx->kp, items_dev, \
                         IpInline{}, level)
    CAP_SWITCH(beta, GO)
#undef GO
    LAUNCH_CHECK();
    return HE_OK;
}

int k_inner_product_inline(const he_ctx *ctx, const ip_item *items, int n, int level, cudaStream_t s) {
    for (int i0 = 0; i0 < n; i0 += HE_INLINE_ITEMS) {
        const int cnt = std::min(HE_INLINE_ITEMS, n - i0);
        IpInline inl;
        for (int i = 0; i < cnt; i++) inl.it[i] = items[i0 + i];
        TraceScope tr("ip", s, ip_bytes(ctx, level, cnt), ip_mulmods(ctx, level, cnt));
        int beta = 0;
        for (int i = 0; i < cnt; i++) beta = std::max(beta, inl.it[i].beta);
#define GO(C) pdl_launch(ip_kernel<C>, dim3(ctx->n / TB, level + 1 + ctx->K, cnt), TB, 0, s, ctx->kp, nullptr, inl, level)
        CAP_SWITCH(beta, GO)
#undef GO
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
#define GO(C) pdl_launch(moddown_fbc_kernel<C>, dim3(ctx->n / TB, npoly), TB, 0, s, ctx->kp, u, conv, level, \
                         ctx->moddown[level].d)
    CAP_SWITCH(ctx->K, GO)
#undef GO
    LAUNCH_CHECK();
    return HE_OK;
}

int k_moddown_combine(const he_ctx *ctx, const md_item *items_dev, int n_items, int level,
                      cudaStream_t s) {
    const u64 *pinv = ctx->d_consts + ctx->np;
    const u64 *pinvs = pinv + (ctx->L + 1);
    TraceScope tr("moddown_combine", s, (double)n_items * (level + 1) * ctx->n * 8 * 7, (double)n_items * (level + 1) * ctx->n * 2);
    pdl_launch(moddown_combine_kernel, dim3(ctx->n / TB, level + 1, n_items), TB, 0, s, 
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
        pdl_launch(moddown_combine_kernel, dim3(ctx->n / TB, level + 1, cnt), TB, 0, s, ctx->kp, nullptr, inl, level,
                                                                               pinv, pinvs);
        LAUNCH_CHECK();
    }
    return HE_OK;
}

int k_moddown_combine_one(const he_ctx *ctx, const md_item &it, int level, cudaStream_t s) {
    return k_moddown_combine_inline(ctx, &it, 1, level, s);
}

// Relinearisation tail of m products at level l, fused with their rescale: u [m][2][l+1+K][n]
// (inner products, NTT form), base [m] polys 0, 1 at base + i b_is + c b_ps, w scratch
// [m][2][l][n]; outputs out[i] at level l - 1 (poly c at out[i] + c out_ps[i]).
int k_moddown_rescale(const he_ctx *ctx, u64 *u, const u64 *base, size_t b_is, size_t b_ps, u64 *w,
                      u64 *const *out, const size_t *out_ps, int m, int level, cudaStream_t s) {
    if (m <= 0) return HE_OK;
    if (ctx->K > 16 || level < 1) { he_set_error("moddown-rescale: bad level or special primes"); return HE_EINVAL; }
    const int nq = level + 1, ext = nq + ctx->K;
    const size_t we = (size_t)ext * ctx->n;
    pdl_launch(fold_top_kernel, dim3(ctx->n / TB, 2, m), TB, 0, s, ctx->kp, u, 2 * we, we, base, b_is, b_ps, level,
                                                           ctx->d_consts);
    LAUNCH_CHECK();
    ntt_job ju{u, we, level, ctx->K + 1, nq, 0, 2 * m, 0};
    HE_TRY(k_ntt(ctx, ju, true, s));
    const u64 *pinv = ctx->d_consts + ctx->np;
    const u64 *pinvs = pinv + (ctx->L + 1);
    {
        TraceScope tr("moddown_fbc", s, (double)2 * m * (ctx->K + 1 + level) * ctx->n * 8,
                      (double)2 * m * (ctx->K + nq * ctx->K + level) * ctx->n);
        // target-prime shares: enough blocks for about two per SM slot of a 152-SM GPU
        const int blocks = (ctx->n / TB) * 2 * m;
        const int shares = std::max(1, std::min(level, std::min(4, (2048 + blocks - 1) / blocks)));
#define GO(C) pdl_launch(moddown_rescale_fbc_kernel<C>, dim3(ctx->n / TB, 2 * m, shares), TB, 0, s, ctx->kp, u, w, \
                         level, ctx->moddown[level].d, pinv, pinvs)
        CAP_SWITCH(ctx->K, GO)
#undef GO
        LAUNCH_CHECK();
    }
    ntt_job jw{w, (size_t)level * ctx->n, 0, level, nq, 0, 2 * m, 0};
    HE_TRY(k_ntt(ctx, jw, false, s));
    const u64 *cb = ctx->d_consts + ctx->np + 2 * (ctx->L + 1);
    const u64 *linv = cb + (size_t)level * 2 * (ctx->L + 1);
    const u64 *linvs = linv + (ctx->L + 1);
    for (int i0 = 0; i0 < m; i0 += HE_INLINE_ITEMS) {
        const int cnt = std::min(HE_INLINE_ITEMS, m - i0);
        MdrInline inl;
        for (int i = 0; i < cnt; i++) {
            const int j = i0 + i;
            inl.it[i] = mdr_item{u + (size_t)j * 2 * we, base + (size_t)j * b_is, b_ps, w + (size_t)j * 2 * level * ctx->n,
                                 out[j], out_ps[j]};
        }
        TraceScope tr("moddown_combine", s, (double)cnt * level * ctx->n * 8 * 9, (double)cnt * level * ctx->n * 4);
        pdl_launch(moddown_rescale_combine_kernel, dim3(ctx->n / TB, level, cnt), TB, 0, s, ctx->kp, inl, level, pinv, pinvs,
                                                                                   linv, linvs);
        LAUNCH_CHECK();
    }
    return HE_OK;
}

int k_range_check(const he_ctx *ctx, const u64 *d, size_t ps, int level, unsigned long long *bad, cudaStream_t s) {
    pdl_launch(range_check_kernel, dim3(ctx->n / TB, level + 1, 2), TB, 0, s, ctx->kp, d, ps, bad);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_mac(const he_ctx *ctx, const mac_term *terms_dev, int n_terms, u64 *out, size_t out_pstride,
          int level, bool accumulate, cudaStream_t s) {
    TraceScope tr("mac", s, (double)(level + 1) * ctx->n * 8 * (3.0 * n_terms + 2), (double)(level + 1) * ctx->n * 2.0 * n_terms);
    pdl_launch(mac_kernel, dim3(ctx->n / TB, level + 1), TB, 0, s, ctx->kp, terms_dev, mac_term{}, n_terms, out,
                                                          out_pstride, accumulate ? 1 : 0);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_mac_one(const he_ctx *ctx, const mac_term &t, u64 *out, size_t out_pstride, int level,
              bool accumulate, cudaStream_t s) {
    pdl_launch(mac_kernel, dim3(ctx->n / TB, level + 1), TB, 0, s, ctx->kp, nullptr, t, 1, out, out_pstride,
                                                          accumulate ? 1 : 0);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_mul_scalar_v(const he_ctx *ctx, he_ct *ct, const u64 *res, const u64 *shoup, int polys,
                   cudaStream_t s) {
    Res64 r;
    for (int i = 0; i <= ct->level; i++) { r.v[i] = res[i]; r.s[i] = shoup[i]; }
    pdl_launch(mul_scalar_v_kernel, dim3(ctx->n / TB, ct->level + 1, polys), TB, 0, s, ctx->kp, ct->d, ct->pstride, r);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_add_const_v(const he_ctx *ctx, he_ct *ct, const u64 *res, cudaStream_t s) {
    Res64 r;
    for (int i = 0; i <= ct->level; i++) { r.v[i] = res[i]; r.s[i] = 0; }
    pdl_launch(add_const_v_kernel, dim3(ctx->n / TB, ct->level + 1), TB, 0, s, ctx->kp, ct->d, r);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_mul_pointwise(const he_ctx *ctx, const u64 *a, const u64 *b, u64 *out, int nlimbs,
                    cudaStream_t s) {
    pdl_launch(mul_pointwise_kernel, dim3(ctx->n / TB, nlimbs), TB, 0, s, ctx->kp, a, b, out);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_tensor_batch(const he_ctx *ctx, const he_ct *const *a, const he_ct *const *b, int m, u64 *d, size_t dstride,
                   int level, cudaStream_t s) {
    for (int i0 = 0; i0 < m; i0 += HE_INLINE_ITEMS) {
        const int cnt = std::min(HE_INLINE_ITEMS, m - i0);
        TensorInline T;
        for (int i = 0; i < cnt; i++) {
            T.a[i] = a[i0 + i]->d;
            T.b[i] = b[i0 + i]->d;
            T.pa[i] = a[i0 + i]->pstride;
            T.pb[i] = b[i0 + i]->pstride;
        }
        pdl_launch(tensor_batch_kernel, dim3(ctx->n / TB, level + 1, cnt), TB, 0, s, ctx->kp, T, d + (size_t)i0 * dstride,
                   dstride, level);
        LAUNCH_CHECK();
    }
    return HE_OK;
}

int k_tensor(const he_ctx *ctx, const he_ct *a, const he_ct *b, u64 *d, cudaStream_t s) {
    pdl_launch(tensor_kernel, dim3(ctx->n / TB, a->level + 1), TB, 0, s, ctx->kp, a->d, a->pstride, b->d, b->pstride, d,
                                                                a->level);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_prekey(const he_ctx *ctx, const u64 *key, const u64 *pt, int level, int pt_level, int beta, u64 *Kp, u64 *Ppt,
             cudaStream_t s) {
    dim3 g(ctx->n / TB, level + 1 + ctx->K, 2 * beta + 1);
    pdl_launch(prekey_kernel, g, TB, 0, s, ctx->kp, key, pt, level, pt_level, beta, Kp, Ppt, ctx->d_consts);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_ipmac(const he_ctx *ctx, const fgrp *grps, int n_grp, int V, int max_beta, double bytes, double mulmods,
            int form, int gb, cudaStream_t s) {
    if (n_grp <= 0) return HE_OK;
    if (gb <= 0 || gb > n_grp) gb = n_grp;
    const unsigned gx = (unsigned)((n_grp + gb - 1) / gb) * gb * (ctx->n / 512);
    if (max_beta > 8) { he_set_error("fused key switching: at most 8 digits"); return HE_EINVAL; }
    if (V != 1 && V != 2) { he_set_error("k_ipmac: V must be 1 or 2"); return HE_EINVAL; }
    const int primes = ctx->L + 1 + ctx->K;
    TraceScope tr("ipmac", s, bytes, mulmods);
    if (form == HE_KEY_STREAM_TMA && max_beta <= 4 && ctx->d_err) {
        // TMA-pipelined form: TMA_STAGES stages of 2*beta key segments of TMA_TILE words + mbarriers
        const size_t smem = TMA_STAGES * ((size_t)(2 * max_beta) * TMA_TILE * 8 + 8);
        const int smem_max = TMA_STAGES * (2 * 4 * TMA_TILE * 8 + 8);
        static const bool attr_ok =                       // thread-safe one-time opt-in
            cudaFuncSetAttribute(ipmac_tma_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max) ==
                cudaSuccess &&
            cudaFuncSetAttribute(ipmac_tma_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max) ==
                cudaSuccess;
        if (!attr_ok) { he_set_error("fused kernel: shared-memory opt-in failed"); return HE_ECUDA; }
        dim3 gt(gx, primes);
        if (V == 1)
            pdl_launch(ipmac_tma_kernel<1>, gt, TB, smem, s, ctx->kp, grps, n_grp, gb, ctx->d_err, ctx->d_consts);
        else
            pdl_launch(ipmac_tma_kernel<2>, gt, TB, smem, s, ctx->kp, grps, n_grp, gb, ctx->d_err, ctx->d_consts);
        LAUNCH_CHECK();
        return HE_OK;
    }
    if (form == HE_KEY_STREAM_PKT && !(max_beta <= 4 && ctx->d_err)) form = HE_KEY_STREAM_PK;   // pair form
    if (form == HE_KEY_STREAM_PKT) {
        if (V != 1) { he_set_error("k_ipmac: the pre-keyed form takes one output per group"); return HE_EINVAL; }
        const int smem = PKT_STAGES * (2 * 4 * TMA_TILE * 8) + 2 * PKT_STAGES * 8;
        static const bool attr_ok =
            cudaFuncSetAttribute(ipmac_pkt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess;
        if (!attr_ok) { he_set_error("fused kernel: shared-memory opt-in failed"); return HE_ECUDA; }
        pdl_launch(ipmac_pkt_kernel, dim3(gx, primes), PKT_THREADS, smem, s, ctx->kp, grps, n_grp, gb, ctx->d_err,
                   ctx->d_consts);
        LAUNCH_CHECK();
        return HE_OK;
    }
    if (form == HE_KEY_STREAM_PK1) {
        if (V != 1) { he_set_error("k_ipmac: the pre-keyed form takes one output per group"); return HE_EINVAL; }
        dim3 g1((unsigned)((n_grp + gb - 1) / gb) * gb * (ctx->n / TB), primes);
        if (max_beta <= 4) pdl_launch(ipmac_pk1_kernel<4, 4>, g1, TB, 0, s, ctx->kp, grps, n_grp, gb, ctx->d_consts);
        else pdl_launch(ipmac_pk1_kernel<8, 2>, g1, TB, 0, s, ctx->kp, grps, n_grp, gb, ctx->d_consts);
        LAUNCH_CHECK();
        return HE_OK;
    }
    if (form == HE_KEY_STREAM_PK || form == HE_FORM_PK3 || form == HE_FORM_PKP || form == HE_KEY_STREAM_PK3L) {
        if (V != 1) { he_set_error("k_ipmac: the pre-keyed form takes one output per group"); return HE_EINVAL; }
        dim3 gp(gx, primes);
        if (form == HE_FORM_PK3 && max_beta <= 4)
            pdl_launch(ipmac_pk_kernel<4, 3, false>, gp, TB, 0, s, ctx->kp, grps, n_grp, gb, ctx->d_consts);
        else if (form == HE_KEY_STREAM_PK3L && max_beta <= 4)
            pdl_launch(ipmac_pk_kernel<4, 3, false, 2>, gp, TB, 0, s, ctx->kp, grps, n_grp, gb, ctx->d_consts);
        else if (form == HE_FORM_PKP && max_beta <= 4)
            pdl_launch(ipmac_pk_kernel<4, 2, true>, gp, TB, 0, s, ctx->kp, grps, n_grp, gb, ctx->d_consts);
        else if (max_beta <= 4) pdl_launch(ipmac_pk_kernel<4, 2, false>, gp, TB, 0, s, ctx->kp, grps, n_grp, gb, ctx->d_consts);
        else pdl_launch(ipmac_pk_kernel<8, 2, false>, gp, TB, 0, s, ctx->kp, grps, n_grp, gb, ctx->d_consts);
        LAUNCH_CHECK();
        return HE_OK;
    }
    if (form == HE_KEY_STREAM_LDG1) {
        dim3 g1((unsigned)((n_grp + gb - 1) / gb) * gb * (ctx->n / TB), primes);
#define IPM1(VV, BB) pdl_launch(ipmac1_kernel<VV, BB>, g1, TB, 0, s, ctx->kp, grps, n_grp, gb, ctx->d_consts)
        if (V == 1) { if (max_beta <= 4) IPM1(1, 4); else IPM1(1, 8); }
        else { if (max_beta <= 4) IPM1(2, 4); else IPM1(2, 8); }
#undef IPM1
        LAUNCH_CHECK();
        return HE_OK;
    }
    if (form == HE_KEY_STREAM_CP && max_beta <= 4) {
        const size_t smem1 = (size_t)CP_STAGES * (2 * 4 + 4 + 1 + 2) * TB * 16;
        const size_t smem2 = (size_t)CP_STAGES * (2 * 4 + 4 + 2 + 2) * TB * 16;
        static const bool attr_ok =
            cudaFuncSetAttribute(ipmac_cp_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1) ==
                cudaSuccess &&
            cudaFuncSetAttribute(ipmac_cp_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2) ==
                cudaSuccess;
        if (!attr_ok) { he_set_error("fused kernel: shared-memory opt-in failed"); return HE_ECUDA; }
        dim3 gc(gx, primes);
        if (V == 1) pdl_launch(ipmac_cp_kernel<1>, gc, TB, smem1, s, ctx->kp, grps, n_grp, gb, ctx->d_consts);
        else pdl_launch(ipmac_cp_kernel<2>, gc, TB, smem2, s, ctx->kp, grps, n_grp, gb, ctx->d_consts);
        LAUNCH_CHECK();
        return HE_OK;
    }
    dim3 g(gx, primes);
#define IPM(VV, BB) pdl_launch(ipmac_kernel<VV, BB>, g, TB, 0, s, ctx->kp, grps, n_grp, gb, ctx->d_consts)
    if (V == 1) { if (max_beta <= 4) IPM(1, 4); else IPM(1, 8); }
    else { if (max_beta <= 4) IPM(2, 4); else IPM(2, 8); }
#undef IPM
    LAUNCH_CHECK();
    return HE_OK;
}

// ---- split form: amount-major inner products, then the raised-basis MAC
// One coefficient per thread.  Block -> (group, tile, prime) as in grp_pos.
__device__ __forceinline__ bool lvl_pos(const KP &kp, int level, int &t) {
    const int kl = blockIdx.y;
    if (kl <= kp.L) {
        if (kl > level) return false;
        t = kl;
    } else {
        t = level + 1 + (kl - kp.L - 1);
    }
    return true;
}

__device__ __forceinline__ void cp_async8(unsigned dst, const void *src, u64 pol) {
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Amount-major inner products of the split form.  Keys sit in registers for the entries of
// their amount; each thread keeps IPA_STAGES - 1 entries' gathered words (digits, c0, c1) in
// flight through cp.async into its own shared-memory slots.
constexpr int IPA_STAGES = 4;

template <int B>
__global__ void __launch_bounds__(TB) ip_amounts_kernel(KP kp, const ugrp *grps, int n_grp, const u64 *pmod) {
    pdl_wait();
    constexpr int RS = IPA_STAGES, NW = B + 2;        // words per entry: D[B], c0, c1
    extern __shared__ u64 ism[];                      // [RS][NW][TB]
    const ugrp P = grps[blockIdx.x % n_grp];
    const int tile = blockIdx.x / n_grp;
    int t;
    if (!lvl_pos(kp, P.level, t)) return;
    const int k = tile * TB + threadIdx.x;
    const int kl = blockIdx.y;
    const int nq = P.level + 1, ext = nq + kp.K;
    const int beta = P.beta;
    const bool isq = t < nq;
    const u64 q = kp.q[kl], qi = kp.qinv[kl], r2 = kp.r2[kl];
    const u64 Pm = isq ? to_mont(pmod[kl], q, qi, r2) : 0;
    const size_t kstride = (size_t)(kp.L + 1 + kp.K) * kp.n;
    const size_t off = (size_t)t * kp.n + k;
    const u64 stream = policy_evict_first(), keep = policy_evict_last();
    const unsigned sbase = smem_u32(ism);
    auto slot = [&](int st, int w) -> int { return (st * NW + w) * TB + threadIdx.x; };
    auto issue = [&](int e, int st) {
        const uent E = P.ents[e];
        const int ks = E.g == 1 ? k : autom_index(k, E.g, kp.logn);
        if (E.D) {
#pragma unroll
            for (int j = 0; j < B; j++)
                if (j < beta) cp_async8(sbase + 8u * slot(st, j), E.D + ((size_t)j * ext + t) * kp.n + ks, keep);
        }
        if (isq) {
            cp_async8(sbase + 8u * slot(st, B), E.src + (size_t)t * kp.n + ks, keep);
            if (E.g == 1) cp_async8(sbase + 8u * slot(st, B + 1), E.src + E.ps + off, keep);
        }
    };
    const int ne = P.n_ent;
#pragma unroll
    for (int e = 0; e < RS - 1; e++) {
        if (e < ne) issue(e, e);
        cp_async_commit();
    }
    for (int i = 0; i < P.n_amt; i++) {
        const famt A = P.amts[i];
        u64 k0[B], k1[B];
        if (A.key) {
#pragma unroll
            for (int j = 0; j < B; j++)
                if (j < beta) {
                    const u64 *kp0 = A.key + (size_t)(2 * j) * kstride + (size_t)kl * kp.n + k;
                    k0[j] = ld_hint(kp0, keep);
                    k1[j] = ld_hint(kp0 + kstride, keep);
                }
        }
        for (int e = A.e0; e < A.e1; e++) {
            if (e + RS - 1 < ne) issue(e + RS - 1, (e + RS - 1) % RS);
            cp_async_commit();
            cp_async_wait<RS - 1>();
            const int st = e % RS;
            const uent E = P.ents[e];
            u64 u0 = 0, u1 = 0;
            if (A.key) {
                u128 a0 = 0, a1 = 0;
#pragma unroll
                for (int j = 0; j < B; j++)
                    if (j < beta) {
                        const u64 d = ism[slot(st, j)];
                        a0 += (u128)d * k0[j];
                        a1 += (u128)d * k1[j];
                    }
                u0 = redc(a0, q, qi);
                u1 = redc(a1, q, qi);
            }
            if (isq) {                              // fold [P]_q phi(c0) (and [P]_q c1 at amount 0)
                u0 = add_mod(u0, mul_mont(ism[slot(st, B)], Pm, q, qi), q);
                if (!A.key) u1 = mul_mont(ism[slot(st, B + 1)], Pm, q, qi);
            }
            E.U[off] = u0;
            E.U[(size_t)ext * kp.n + off] = u1;
        }
    }
    cp_async_wait<0>();
}

// acc_v = sum_terms pt_v (.) U over Q u P for HE_RV outputs per thread (one coefficient); absent
// outputs are skipped (block-uniform).  Each thread keeps RMAC_STAGES - 1 terms in flight: it
// copies its own words of the coming terms into its own shared-memory slots with cp.async
// (8 bytes each), so no block barrier is needed and no register holds a word in flight.
constexpr int RMAC_STAGES = 4;
constexpr int RMAC_WORDS = 2 + HE_RV;               // u0, u1, pt[HE_RV]

__global__ void __launch_bounds__(TB, 2) rmac_kernel(KP kp, const rgrp *grps, int n_grp) {
    pdl_wait();
    constexpr int RV = HE_RV, RS = RMAC_STAGES;
    extern __shared__ u64 rsm[];                     // [RS][RMAC_WORDS][TB]
    const rgrp P = grps[blockIdx.x % n_grp];
    const int tile = blockIdx.x / n_grp;
    int t;
    if (!lvl_pos(kp, P.level, t)) return;
    const int k = tile * TB + threadIdx.x;
    const int kl = blockIdx.y;
    const int nq = P.level + 1, ext = nq + kp.K;
    const int ptl = kl <= kp.L ? kl : P.pt_level + 1 + (kl - kp.L - 1);
    const u64 q = kp.q[kl], qi = kp.qinv[kl], r2 = kp.r2[kl];
    const u64 one = to_mont(1, q, qi, r2);
    const size_t off = (size_t)t * kp.n + k, ptoff = (size_t)ptl * kp.n + k;
    const u64 stream = policy_evict_first();
    const unsigned sbase = smem_u32(rsm);
    auto slot = [&](int st, int w) -> int { return (st * RMAC_WORDS + w) * TB + threadIdx.x; };
    auto issue = [&](int i, int st) {
        const rterm T = P.terms[i];
        cp_async8(sbase + 8u * slot(st, 0), T.U + off, stream);
        cp_async8(sbase + 8u * slot(st, 1), T.U + (size_t)ext * kp.n + off, stream);
#pragma unroll
        for (int v = 0; v < RV; v++)
            if (T.pt[v] && T.pt[v] != HE_PT_ONE) cp_async8(sbase + 8u * slot(st, 2 + v), T.pt[v] + ptoff, stream);
    };
    u128 a0[RV], a1[RV];
#pragma unroll
    for (int v = 0; v < RV; v++) a0[v] = a1[v] = 0;
    const int nt = P.n_terms;
#pragma unroll
    for (int i = 0; i < RS - 1; i++) {
        if (i < nt) issue(i, i);
        cp_async_commit();
    }
    for (int i = 0; i < nt; i++) {
        if (i + RS - 1 < nt) issue(i + RS - 1, (i + RS - 1) % RS);
        cp_async_commit();                           // one group per iteration, empty or not
        cp_async_wait<RS - 1>();                     // term i's words have landed
        const int st = i % RS;
        const u64 u0 = rsm[slot(st, 0)], u1 = rsm[slot(st, 1)];
        const rterm T = P.terms[i];
#pragma unroll
        for (int v = 0; v < RV; v++)
            if (T.pt[v]) {                           // block-uniform
                const u64 p = T.pt[v] == HE_PT_ONE ? one : rsm[slot(st, 2 + v)];
                a0[v] += (u128)p * u0;
                a1[v] += (u128)p * u1;
            }
    }
    cp_async_wait<0>();
    // a later chunk of amounts adds its partial sums modulo q: same residues as one pass
    auto put = [&](u64 *dst, u128 acc) {
        u64 r = redc(acc, q, qi);
        if (P.accumulate) {
            r += *dst;
            if (r >= q) r -= q;
        }
        *dst = r;
    };
#pragma unroll
    for (int v = 0; v < RV; v++)
        if (v < P.nv) {
            put(P.acc + ((size_t)(2 * v) * ext) * kp.n + off, a0[v]);
            put(P.acc + ((size_t)(2 * v + 1) * ext) * kp.n + off, a1[v]);
        }
}

int k_ip_amounts(const he_ctx *ctx, const ugrp *grps, int n_grp, int max_beta, double bytes, cudaStream_t s) {
    if (n_grp <= 0) return HE_OK;
    if (max_beta > 8) { he_set_error("inner products: at most 8 digits"); return HE_EINVAL; }
    TraceScope tr("ip_amounts", s, bytes, 0);
    dim3 g((unsigned)(ctx->n / TB) * n_grp, ctx->L + 1 + ctx->K);
    const int smem4 = IPA_STAGES * (4 + 2) * TB * 8, smem8 = IPA_STAGES * (8 + 2) * TB * 8;
    static const bool attr_ok =
        cudaFuncSetAttribute(ip_amounts_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem4) == cudaSuccess &&
        cudaFuncSetAttribute(ip_amounts_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem8) == cudaSuccess;
    if (!attr_ok) { he_set_error("ip_amounts: shared-memory opt-in failed"); return HE_ECUDA; }
    if (max_beta <= 4) pdl_launch(ip_amounts_kernel<4>, g, TB, smem4, s, ctx->kp, grps, n_grp, ctx->d_consts);
    else pdl_launch(ip_amounts_kernel<8>, g, TB, smem8, s, ctx->kp, grps, n_grp, ctx->d_consts);
    LAUNCH_CHECK();
    return HE_OK;
}

// Image-batched form: per term, HE_RVM plaintext words (read once) meet the inner products of up
// to HE_RNI images, each at its own level (an image without the block's q-prime sits out); the
// same cp.async ring as rmac_kernel, HE_RVM + 2 HE_RNI words per term per thread.
constexpr int RMACM_WORDS = HE_RVM + 2 * HE_RNI;

__global__ void __launch_bounds__(TB, 1) rmac_m_kernel(KP kp, const rgrp_m *grps, int n_grp) {
    pdl_wait();
    constexpr int RV = HE_RVM, NI = HE_RNI, RS = RMAC_STAGES;
    extern __shared__ u64 rsm[];                     // [RS][RMACM_WORDS][TB]
    const rgrp_m P = grps[blockIdx.x % n_grp];
    const int tile = blockIdx.x / n_grp;
    const int kl = blockIdx.y;
    int t[NI];
    bool in[NI];
    bool any = false;
#pragma unroll
    for (int i = 0; i < NI; i++) {
        in[i] = i < P.ni && (kl > kp.L || kl <= P.level[i]);
        t[i] = kl <= kp.L ? kl : P.level[i] + 1 + (kl - kp.L - 1);
        any = any || in[i];
    }
    if (!any) return;
    const int k = tile * TB + threadIdx.x;
    const int ptl = kl <= kp.L ? kl : P.pt_level + 1 + (kl - kp.L - 1);
    const u64 q = kp.q[kl], qi = kp.qinv[kl], r2 = kp.r2[kl];
    const u64 one = to_mont(1, q, qi, r2);
    const size_t ptoff = (size_t)ptl * kp.n + k;
    const u64 stream = policy_evict_first();
    const unsigned sbase = smem_u32(rsm);
    auto slot = [&](int st, int w) -> int { return (st * RMACM_WORDS + w) * TB + threadIdx.x; };
    auto issue = [&](int e, int st) {
        const rterm_m T = P.terms[e];
#pragma unroll
        for (int v = 0; v < RV; v++)
            if (T.pt[v] && T.pt[v] != HE_PT_ONE) cp_async8(sbase + 8u * slot(st, v), T.pt[v] + ptoff, stream);
#pragma unroll
        for (int i = 0; i < NI; i++)
            if (in[i] && T.U[i]) {
                const size_t ext = (size_t)(P.level[i] + 1 + kp.K) * kp.n;
                cp_async8(sbase + 8u * slot(st, RV + 2 * i), T.U[i] + (size_t)t[i] * kp.n + k, stream);
                cp_async8(sbase + 8u * slot(st, RV + 2 * i + 1), T.U[i] + ext + (size_t)t[i] * kp.n + k, stream);
            }
    };
    u128 a0[RV][NI], a1[RV][NI];
#pragma unroll
    for (int v = 0; v < RV; v++)
#pragma unroll
        for (int i = 0; i < NI; i++) a0[v][i] = a1[v][i] = 0;
    const int nt = P.n_terms;
#pragma unroll
    for (int e = 0; e < RS - 1; e++) {
        if (e < nt) issue(e, e);
        cp_async_commit();
    }
    for (int e = 0; e < nt; e++) {
        if (e + RS - 1 < nt) issue(e + RS - 1, (e + RS - 1) % RS);
        cp_async_commit();
        cp_async_wait<RS - 1>();
        const int st = e % RS;
        const rterm_m T = P.terms[e];
#pragma unroll
        for (int v = 0; v < RV; v++)
            if (T.pt[v]) {                           // block-uniform
                const u64 p = T.pt[v] == HE_PT_ONE ? one : rsm[slot(st, v)];
#pragma unroll
                for (int i = 0; i < NI; i++)
                    if (in[i] && T.U[i]) {
                        a0[v][i] += (u128)p * rsm[slot(st, RV + 2 * i)];
                        a1[v][i] += (u128)p * rsm[slot(st, RV + 2 * i + 1)];
                    }
            }
    }
    cp_async_wait<0>();
    auto put = [&](u64 *dst, u128 acc) {
        u64 r = redc(acc, q, qi);
        if (P.accumulate) {
            r += *dst;
            if (r >= q) r -= q;
        }
        *dst = r;
    };
#pragma unroll
    for (int i = 0; i < NI; i++)
        if (in[i]) {
            const size_t ext = (size_t)(P.level[i] + 1 + kp.K) * kp.n;
            const size_t off = (size_t)t[i] * kp.n + k;
#pragma unroll
            for (int v = 0; v < RV; v++)
                if (v < P.nv) {
                    put(P.acc[i] + (size_t)(2 * v) * ext + off, a0[v][i]);
                    put(P.acc[i] + (size_t)(2 * v + 1) * ext + off, a1[v][i]);
                }
        }
}

int k_rmac_m(const he_ctx *ctx, const rgrp_m *grps, int n_grp, double bytes, double mulmods, cudaStream_t s) {
    if (n_grp <= 0) return HE_OK;
    TraceScope tr("rmac", s, bytes, mulmods);
    dim3 g((unsigned)(ctx->n / TB) * n_grp, ctx->L + 1 + ctx->K);
    const int smem = RMAC_STAGES * RMACM_WORDS * TB * 8;
    static const bool attr_ok =
        cudaFuncSetAttribute(rmac_m_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess;
    if (!attr_ok) { he_set_error("rmac_m: shared-memory opt-in failed"); return HE_ECUDA; }
    pdl_launch(rmac_m_kernel, g, TB, smem, s, ctx->kp, grps, n_grp);
    LAUNCH_CHECK();
    return HE_OK;
}

int k_rmac(const he_ctx *ctx, const rgrp *grps, int n_grp, double bytes, double mulmods, cudaStream_t s) {
    if (n_grp <= 0) return HE_OK;
    TraceScope tr("rmac", s, bytes, mulmods);
    dim3 g((unsigned)(ctx->n / TB) * n_grp, ctx->L + 1 + ctx->K);
    const int smem = RMAC_STAGES * RMAC_WORDS * TB * 8;
    static const bool attr_ok =
        cudaFuncSetAttribute(rmac_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess;
    if (!attr_ok) { he_set_error("rmac: shared-memory opt-in failed"); return HE_ECUDA; }
    pdl_launch(rmac_kernel, g, TB, smem, s, ctx->kp, grps, n_grp);
    LAUNCH_CHECK();
    return HE_OK;
}

// ---- factored channel-shard conv, stage 2: integer-scalar weighting of the masked rotations
// out[o H + h][c][i][k] = sum_{f, t} Wm[i][o][f T + t] * Y[(f H + h) T + t][c][i][k]   (mod q_i)
// Wm holds the scalars' residues in Montgomery form, so one REDC of the 128-bit sum gives the
// result.  SM_OB outputs per thread (one coefficient); the block's weights sit in shared memory.
constexpr int SM_OB = 16;

__global__ void __launch_bounds__(TB) smac_kernel(KP kp, const u64 *Y, size_t ystride, size_t yps, const u64 *Wm,
                                                  int co, int ci, int H, int T, u64 *out, size_t ostride,
                                                  size_t ops) {
    pdl_wait();
    extern __shared__ u64 wsm[];                                   // [SM_OB][nin]
    const int nin = ci * T;
    const int k = blockIdx.x * TB + threadIdx.x;
    const int i = blockIdx.y >> 1, c = blockIdx.y & 1;             // limb, polynomial
    const int h = blockIdx.z % H, o0 = (blockIdx.z / H) * SM_OB;
    const u64 q = kp.q[i], qi = kp.qinv[i];
    const int nob = min(SM_OB, co - o0);
    for (int x = threadIdx.x; x < nob * nin; x += TB) {
        const int ob = x / nin, kk = x % nin;
        wsm[x] = Wm[((size_t)i * co + o0 + ob) * nin + kk];
    }
    __syncthreads();
    u128 acc[SM_OB];
#pragma unroll
    for (int ob = 0; ob < SM_OB; ob++) acc[ob] = 0;
    const u64 stream = policy_evict_first();
    constexpr int U = 4;                                           // inputs in flight per thread
    for (int f = 0; f < ci; f++) {
        const u64 *yb = Y + (size_t)(f * H + h) * T * ystride + c * yps + (size_t)i * kp.n + k;
        const u64 *wf = wsm + f * T;
        for (int t = 0; t < T; t += U) {
            u64 y[U];
#pragma unroll
            for (int u = 0; u < U; u++) y[u] = t + u < T ? ld_hint(yb + (size_t)(t + u) * ystride, stream) : 0;
#pragma unroll
            for (int u = 0; u < U; u++)
                if (t + u < T) {
#pragma unroll
                    for (int ob = 0; ob < SM_OB; ob++)
                        if (ob < nob) acc[ob] += (u128)y[u] * wf[ob * nin + t + u];
                }
        }
    }
#pragma unroll
    for (int ob = 0; ob < SM_OB; ob++)
        if (ob < nob) out[(size_t)((o0 + ob) * H + h) * ostride + c * ops + (size_t)i * kp.n + k] = redc(acc[ob], q, qi);
}

int k_smac(const he_ctx *ctx, const u64 *Y, size_t ystride, size_t yps, const u64 *Wm, int co, int ci, int H, int T,
           int level, u64 *out, size_t ostride, size_t ops, cudaStream_t s) {
    const int nin = ci * T;
    const size_t smem = (size_t)SM_OB * nin * 8;
    if (smem > 200 * 1024) { he_set_error("factored conv: %d inputs per output exceed shared memory", nin); return HE_EINVAL; }
    if (smem > 48 * 1024) {
        static const bool ok = cudaFuncSetAttribute(smac_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    200 * 1024) == cudaSuccess;
        if (!ok) { he_set_error("factored conv: shared-memory opt-in failed"); return HE_ECUDA; }
    }
    const double nl = level + 1;
    TraceScope tr("smac", s, (double)(H * ci * T) * 2 * nl * ctx->n * 8 * ((co + SM_OB - 1) / SM_OB) +
                                 (double)co * H * 2 * nl * ctx->n * 8,
                  (double)co * H * ci * T * 2 * nl * ctx->n);
    dim3 g(ctx->n / TB, 2 * (level + 1), H * ((co + SM_OB - 1) / SM_OB));
    pdl_launch(smac_kernel, g, TB, smem, s, ctx->kp, Y, ystride, yps, Wm, co, ci, H, T, out, ostride, ops);
    LAUNCH_CHECK();
    return HE_OK;
}

// Failure-path self-test: one warp waits (bounded, like the key-tile pipeline) on an mbarrier
// that nothing will ever arrive on; the wait gives up, the kernel records the timeout in the
// context's error word and returns, leaving the context usable.
__global__ void bounded_wait_selftest_kernel(int *err) {
    pdl_wait();
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(smem_u32(&bar), 0);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(err, 1);
}

int k_selftest_bounded_wait(const he_ctx *ctx, cudaStream_t s) {
    if (!ctx->d_err) { he_set_error("context has no error word"); return HE_ESTATE; }
    pdl_launch(bounded_wait_selftest_kernel, 1, 32, 0, s, ctx->d_err);
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
        for (int i = 0; i <= level; i++) {                   // Montgomery form, once on the host
            // x R mod q as the device forms it: REDC(x (R^2 mod q)), three products
            const u64 q = ctx->primes[i], qinv = ctx->h_qinv[i];
            const u128 T = (u128)res[t * HE_LC_LIMBS + i] * ctx->h_r2[i];
            const u64 lo = (u64)T, hi = (u64)(T >> 64), mh = (u64)(((u128)(lo * qinv) * q) >> 64);
            A.res[t][i] = hi >= mh ? hi - mh : hi + (q - mh);
        }
    }
    for (int i = 0; i <= level; i++) A.cst[i] = cst[i];
    A.n_terms = n;
    pdl_launch(lincomb_kernel, dim3(ctx->n / TB, level + 1, 2), TB, 0, s, ctx->kp, A, out, out_ps);
    LAUNCH_CHECK();
    return HE_OK;
}

// rescale of m ciphertexts laid out at a uniform stride (poly p of ct i at base + (2i + p) ps)
// The same for m <= HE_NTT_TAB / 2 ciphertexts at unrelated addresses: polys[2j], polys[2j + 1]
// are c0, c1 of ciphertext j (c1 = c0 + its poly stride); one launch set for all of them.
int k_rescale_tab(const he_ctx *ctx, u64 *const *polys, int m, int level, u64 *t, cudaStream_t s) {
    if (m <= 0) return HE_OK;
    if (m > HE_NTT_TAB / 2) { he_set_error("rescale: at most %d ciphertexts per table", HE_NTT_TAB / 2); return HE_EINVAL; }
    if (!(ctx->logn >= 12 && ctx->logn <= 16)) {           // small rings: one ciphertext at a time
        for (int j = 0; j < m; j++)
            HE_TRY(k_rescale_many(ctx, polys[2 * j], (size_t)(polys[2 * j + 1] - polys[2 * j]), 1, level, t, s));
        return HE_OK;
    }
    ntt_job top{nullptr, 0, level, 1, level + 1, 0, 2 * m, 0};
    for (int p = 0; p < 2 * m; p++) top.tab[p] = polys[p];
    HE_TRY(k_ntt(ctx, top, true, s));
    const u64 *cb = ctx->d_consts + ctx->np + 2 * (ctx->L + 1);
    const u64 *inv = cb + (size_t)level * 2 * (ctx->L + 1);
    RescaleFuse F{nullptr, 0, level, inv, inv + (ctx->L + 1)};
    for (int p = 0; p < 2 * m; p++) F.ctab[p] = polys[p];
    ntt_job tj{t, (size_t)level * ctx->n, 0, level, level, 0, 2 * m, 0};
    const int R = ctx->n / ROW, TC = 4096 / R;
    dim3 gA(ROW / TC, level, 2 * m), gB(R / 16, level, 2 * m);
    TraceScope tr("rescale", s, (double)m * level * ctx->n * 8 * 6, (double)m * level * ctx->n * 2);
    if (ntt_onepass(ctx)) return ntt_onepass_launch<false, true>(ctx, tj, F, s);
    if (ntt_shfl(ctx) && ntt_nc(ctx)) {
        pdl_launch(ntt16_cols<false, true, true>, gA, 256, 0, s, ctx->kp, tj, F);
        LAUNCH_CHECK();
        pdl_launch(ntt16_rows_shfl<false, true, true>, gB, 256, 0, s, ctx->kp, tj, F);
        LAUNCH_CHECK();
    } else if (ntt_shfl(ctx)) {
        pdl_launch(ntt16_cols<false, true>, gA, 256, 0, s, ctx->kp, tj, F);
        LAUNCH_CHECK();
        pdl_launch(ntt16_rows_shfl<false, true>, gB, 256, 0, s, ctx->kp, tj, F);
        LAUNCH_CHECK();
    } else if (ntt_nc(ctx)) {
        pdl_launch(ntt16_cols<false, true, true>, gA, 256, 0, s, ctx->kp, tj, F);
        LAUNCH_CHECK();
        pdl_launch(ntt16_rows<false, true, true>, gB, 256, 0, s, ctx->kp, tj, F);
        LAUNCH_CHECK();
    } else {
        pdl_launch(ntt16_cols<false, true>, gA, 256, 0, s, ctx->kp, tj, F);
        LAUNCH_CHECK();
        pdl_launch(ntt16_rows<false, true>, gB, 256, 0, s, ctx->kp, tj, F);
        LAUNCH_CHECK();
    }
    return HE_OK;
}

int k_rescale_many(const he_ctx *ctx, u64 *base, size_t ps, int m, int level, u64 *t, cudaStream_t s) {
    ntt_job top{base, ps, level, 1, level + 1, 0, 2 * m, 0};
    HE_TRY(k_ntt(ctx, top, true, s));
    if (ctx->logn >= 12 && ctx->logn <= 16) {
        // the correction term's reduction and the final combine ride in the NTT's two passes
        const u64 *cb = ctx->d_consts + ctx->np + 2 * (ctx->L + 1);
        const u64 *inv = cb + (size_t)level * 2 * (ctx->L + 1);
        RescaleFuse F{base, ps, level, inv, inv + (ctx->L + 1)};
        ntt_job tj{t, (size_t)level * ctx->n, 0, level, level, 0, 2 * m, 0};
        const int R = ctx->n / ROW, TC = 4096 / R;
        dim3 gA(ROW / TC, level, 2 * m), gB(R / 16, level, 2 * m);
        TraceScope tr("rescale", s, (double)m * level * ctx->n * 8 * 6, (double)m * level * ctx->n * 2);
        if (ntt_onepass(ctx)) return ntt_onepass_launch<false, true>(ctx, tj, F, s);
        if (ntt_shfl(ctx) && ntt_nc(ctx)) {
            pdl_launch(ntt16_cols<false, true, true>, gA, 256, 0, s, ctx->kp, tj, F);
            LAUNCH_CHECK();
            pdl_launch(ntt16_rows_shfl<false, true, true>, gB, 256, 0, s, ctx->kp, tj, F);
            LAUNCH_CHECK();
        } else if (ntt_shfl(ctx)) {
            pdl_launch(ntt16_cols<false, true>, gA, 256, 0, s, ctx->kp, tj, F);
            LAUNCH_CHECK();
            pdl_launch(ntt16_rows_shfl<false, true>, gB, 256, 0, s, ctx->kp, tj, F);
            LAUNCH_CHECK();
        } else if (ntt_nc(ctx)) {
            pdl_launch(ntt16_cols<false, true, true>, gA, 256, 0, s, ctx->kp, tj, F);
            LAUNCH_CHECK();
            pdl_launch(ntt16_rows<false, true, true>, gB, 256, 0, s, ctx->kp, tj, F);
            LAUNCH_CHECK();
        } else {
            pdl_launch(ntt16_cols<false, true>, gA, 256, 0, s, ctx->kp, tj, F);
            LAUNCH_CHECK();
            pdl_launch(ntt16_rows<false, true>, gB, 256, 0, s, ctx->kp, tj, F);
            LAUNCH_CHECK();
        }
        return HE_OK;
    }
    pdl_launch(rescale_prep_kernel, dim3(ctx->n / TB, level, 2 * m), TB, 0, s, ctx->kp, base + (size_t)level * ctx->n, ps, t, level);
    LAUNCH_CHECK();
    ntt_job tj{t, (size_t)level * ctx->n, 0, level, level, 0, 2 * m, 0};
    HE_TRY(k_ntt(ctx, tj, false, s));
    const u64 *cb = ctx->d_consts + ctx->np + 2 * (ctx->L + 1);
    const u64 *inv = cb + (size_t)level * 2 * (ctx->L + 1);
    const u64 *invs = inv + (ctx->L + 1);
    TraceScope tr("rescale", s, (double)m * level * ctx->n * 8 * 6, (double)m * level * ctx->n * 2);
    pdl_launch(rescale_combine_kernel, dim3(ctx->n / TB, level, 2 * m), TB, 0, s, ctx->kp, base, ps, t, level, inv, invs);
    LAUNCH_CHECK();
    return HE_OK;
}

double k_bench_mac(int blocks, int iters, cudaStream_t s) {
    u64 *sink;
    if (he_malloc(&sink, 8) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    pdl_launch(bench_mac_kernel, blocks, 256, 0, s, 0xfedcba9876543211ull, 16, sink);   // warm-up
    cudaEventRecord(e0, s);
    pdl_launch(bench_mac_kernel, blocks, 256, 0, s, 0xfedcba9876543211ull, iters, sink);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    he_count_launch(2);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    he_free(sink);
    return (double)blocks * 256.0 * 8.0 * iters / (ms * 1e-3);
}

double k_bench_modmul(const he_ctx *ctx, int blocks, int iters, cudaStream_t s) {
    u64 *sink;
    if (he_malloc(&sink, 8) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const u64 q = ctx->primes[0];
    pdl_launch(bench_modmul_kernel, blocks, 256, 0, s, q, ctx->h_qinv[0], 16, sink);   // warm-up
    cudaEventRecord(e0, s);
    pdl_launch(bench_modmul_kernel, blocks, 256, 0, s, q, ctx->h_qinv[0], iters, sink);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    he_count_launch(2);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    he_free(sink);
    return (double)blocks * 256.0 * 2.0 * iters / (ms * 1e-3);
}
