// Word-sized modular arithmetic on the integer pipes (primes < 2^61, uint64 limbs).
//
// Three reductions, each with the precondition it needs:
//   mul_shoup  a * w mod q for a fixed w with w' = floor(w 2^64 / q); any a < 2^64 -> [0, q)
//   redc       Montgomery: T 2^-64 mod q for T < q 2^64 with qinv = q^-1 mod 2^64 -> [0, q)
//   reduce64   x mod q for any 64-bit x with mu = floor(2^64 / q)
// No floating point is used anywhere.
#pragma once
#include <stdint.h>

typedef uint64_t u64;
typedef unsigned __int128 u128;

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) {
    return a >= b ? a - b : a + q - b;
}
__device__ __forceinline__ u64 mul_shoup(u64 a, u64 w, u64 ws, u64 q) {
    u64 h = __umul64hi(a, ws);
    u64 r = a * w - h * q;
    return r >= q ? r - q : r;
}
__device__ __forceinline__ u64 redc(u128 T, u64 q, u64 qinv) {
    u64 lo = (u64)T, hi = (u64)(T >> 64);
    u64 m = lo * qinv;
    u64 mh = __umul64hi(m, q);
    return hi >= mh ? hi - mh : hi + (q - mh);
}
__device__ __forceinline__ u64 mul_mont(u64 a, u64 bm, u64 q, u64 qinv) {
    return redc((u128)a * bm, q, qinv);
}
// a * b mod q for two normal-form operands (two Montgomery reductions)
__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, u64 q, u64 qinv, u64 r2) {
    return redc((u128)redc((u128)a * b, q, qinv) * r2, q, qinv);
}
__device__ __forceinline__ u64 reduce64(u64 x, u64 q, u64 mu) {
    u64 h = __umul64hi(x, mu);
    u64 r = x - h * q;
    if (r >= q) r -= q;
    if (r >= q) r -= q;
    return r;
}
__device__ __forceinline__ u64 to_mont(u64 x, u64 q, u64 qinv, u64 r2) {
    return redc((u128)x * r2, q, qinv);
}

// NTT-domain index of the Galois automorphism X -> X^g.  With the forward transform used
// here, slot k holds a(psi^(2 brev(k) + 1)); (a o X^g)(psi^e) = a(psi^(e g)), so the output
// slot k reads input slot brev(((2 brev(k) + 1) g mod 2n - 1) / 2).
__device__ __forceinline__ int autom_index(int k, u64 g, int logn) {
    unsigned bk = __brev((unsigned)k) >> (32 - logn);
    u64 e = ((2 * (u64)bk + 1) * g) & ((2ull << logn) - 1);
    unsigned src = (unsigned)((e - 1) >> 1);
    return (int)(__brev(src) >> (32 - logn));
}

// SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014) used as a counter-based
// generator keyed by (seed, stream): word(idx) = mix(mix(seed ^ stream*gamma) + (idx+1)*gamma).
__host__ __device__ __forceinline__ u64 sm64_mix(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ u64 sm64_word(u64 seed, u64 stream, u64 idx) {
    const u64 gamma = 0x9E3779B97F4A7C15ull;
    return sm64_mix(sm64_mix(seed ^ (stream * gamma)) + (idx + 1) * gamma);
}
