// Arithmetic in GF(p), p < 2^31, for the CUDA kernels.
//
// Residues are canonical uint32 values in [0, p). Products of two residues are
// below 2^62, so any sum of two products fits in 64 bits and is reduced with
// one Barrett step: with mu = floor((2^64 - 1) / p), q = hi64(x * mu) is at
// most two below floor(x / p) for every x < 2^64, so x - q p lies in [0, 3p)
// and two conditional subtractions finish the reduction.
#pragma once
#include <cstdint>

struct ModP {
    uint32_t p;
    uint32_t r64;     // 2^64 mod p
    uint64_t mu;      // floor((2^64 - 1) / p)
    uint32_t pneg;    // -p^{-1} mod 2^32 (odd p): Montgomery reduction with R = 2^32
    uint32_t r2;      // R^2 mod p
};

static inline ModP make_modp(uint32_t p)
{
    ModP M;
    M.p = p;
    M.mu = ~0ull / p;
    M.r64 = (uint32_t)((~0ull % p + 1) % p);
    // Newton iteration for p^{-1} mod 2^32 (p odd): x <- x (2 - p x) doubles the correct bits
    uint32_t x = p;
    for (int i = 0; i < 5; ++i) x *= 2u - p * x;
    M.pneg = (p & 1u) ? (uint32_t)(0u - x) : 0u;
    uint64_t r = (1ull << 32) % p;
    M.r2 = (uint32_t)(r * r % p);
    return M;
}

__device__ __forceinline__ uint32_t red64(uint64_t x, const ModP &M)
{
    uint64_t q = __umul64hi(x, M.mu);
    uint64_t r = x - q * (uint64_t)M.p;
    if (r >= M.p) r -= M.p;
    if (r >= M.p) r -= M.p;
    return (uint32_t)r;
}

__device__ __forceinline__ uint32_t mulm(uint32_t a, uint32_t b, const ModP &M)
{
    return red64((uint64_t)a * b, M);
}

__device__ __forceinline__ uint32_t addm(uint32_t a, uint32_t b, const ModP &M)
{
    uint32_t s = a + b;               // < 2^32 since a, b < 2^31
    return s >= M.p ? s - M.p : s;
}

__device__ __forceinline__ uint32_t subm(uint32_t a, uint32_t b, const ModP &M)
{
    return a >= b ? a - b : a + (M.p - b);
}

// (f * x - m * y) mod p for residues f, x, m, y: both products are below 2^62,
// so f x + (p - m) y < 2^63 is reduced once.
__device__ __forceinline__ uint32_t ffupd(uint32_t f, uint32_t x, uint32_t m, uint32_t y, const ModP &M)
{
    uint32_t nm = m ? M.p - m : 0u;
    return red64((uint64_t)f * x + (uint64_t)nm * y, M);
}

// Montgomery reduction (odd p, R = 2^32): for T < p R returns T R^{-1} mod p.
// T + m p < 2 p R <= 2^64 for p < 2^31, and the result before the final
// subtraction is below 2p.
__device__ __forceinline__ uint32_t redc(uint64_t T, const ModP &M)
{
    const uint32_t m = (uint32_t)T * M.pneg;
    const uint32_t t = (uint32_t)((T + (uint64_t)m * M.p) >> 32);
    return t >= M.p ? t - M.p : t;
}

// R^{-1} (f x - m y) mod p with one reduction: f x + (p - m) y < 2 p^2 < p R.
__device__ __forceinline__ uint32_t ffupd_mont(uint32_t f, uint32_t x, uint32_t m, uint32_t y, const ModP &M)
{
    const uint32_t nm = m ? M.p - m : 0u;
    return redc((uint64_t)f * x + (uint64_t)nm * y, M);
}

// a^(p-2) mod p with Montgomery products (odd p): the inverse of a nonzero residue.
__device__ __forceinline__ uint32_t invm_mont(uint32_t a, const ModP &M)
{
    uint32_t b = redc((uint64_t)a * M.r2, M);            // a R
    uint32_t r = redc((uint64_t)M.r2, M);                // R (one in Montgomery form)
    for (uint32_t e = M.p - 2; e; e >>= 1) {
        if (e & 1u) r = redc((uint64_t)r * b, M);
        b = redc((uint64_t)b * b, M);
    }
    return redc((uint64_t)r, M);                         // back from Montgomery form
}

// a^(p-2) mod p (Fermat), the inverse of a nonzero residue.
__device__ __forceinline__ uint32_t invm(uint32_t a, const ModP &M)
{
    uint32_t e = M.p - 2, r = 1u % M.p, b = a;
    while (e) {
        if (e & 1u) r = mulm(r, b, M);
        b = mulm(b, b, M);
        e >>= 1;
    }
    return r;
}

// A 128-bit-safe accumulator of products below 2^62: the low 64 bits and a
// count of wraps. value = hi * 2^64 + lo.
struct Acc {
    uint64_t lo;
    uint32_t hi;
};

__device__ __forceinline__ void acc_add(Acc &a, uint64_t x)
{
    uint64_t s = a.lo + x;
    a.hi += (s < x);
    a.lo = s;
}

__device__ __forceinline__ uint32_t acc_red(const Acc &a, const ModP &M)
{
    // hi * (2^64 mod p) + (lo mod p) < 2^32 * 2^31 + 2^31 < 2^64
    return red64((uint64_t)a.hi * M.r64 + red64(a.lo, M), M);
}
