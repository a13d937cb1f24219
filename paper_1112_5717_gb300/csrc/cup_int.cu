// Multi-modular integer determinant and rank (the homomorphic-imaging use of
// exact elimination over GF(p), Sec. 1): an integer matrix is reduced modulo
// several primes on the device, each image is factored by CUP (Algorithm 6),
// and the residues are lifted on the host by the Chinese remainder theorem.
//
// This file holds the two device kernels of that path (the reduction to
// residues and the row norms of the Hadamard bound) and its host arithmetic
// (prime generation, mixed-radix CRT into a signed multi-word integer).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include "cup_internal.cuh"

// R[k][i][j] = A[i][j] mod primes[k], the least non-negative residue, for all
// k < K. A is int64 m x n (lda); plane k starts at R + k * plane, row stride ldr.
// Each thread reads an entry once and writes its K residues (coalesced per plane).
__global__ void __launch_bounds__(256)
k_reduce_multi(const int64_t *__restrict__ A, int64_t lda, int64_t m, int64_t n,
               const uint32_t *__restrict__ primes, int K, uint32_t *__restrict__ R, int64_t ldr,
               int64_t plane)
{
    const int64_t total = m * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n, j = e - i * n;
        const int64_t a = A[i * lda + j];
        const bool neg = a < 0;
        // |a| without overflow at INT64_MIN
        const uint64_t mag = neg ? (uint64_t)(-(a + 1)) + 1ull : (uint64_t)a;
        uint32_t *out = R + i * ldr + j;
        for (int k = 0; k < K; ++k) {
            const uint32_t p = primes[k];
            uint32_t r = (uint32_t)(mag % p);
            if (neg && r) r = p - r;
            out[(int64_t)k * plane] = r;
        }
    }
}

cudaError_t launch_reduce_multi(const int64_t *A, int64_t lda, int64_t m, int64_t n, const uint32_t *d_primes,
                                int K, uint32_t *R, int64_t ldr, int64_t plane, cudaStream_t st)
{
    if (m <= 0 || n <= 0 || K <= 0) return cudaSuccess;
    int64_t nb = (m * n + 255) / 256;
    if (nb > 152 * 16) nb = 152 * 16;
    k_reduce_multi<<<(unsigned)nb, 256, 0, st>>>(A, lda, m, n, d_primes, K, R, ldr, plane);
    return cudaGetLastError();
}

// out[i] = log2 of the Euclidean norm of row i of the int64 matrix A (rounded
// up: the double sum of squares is inflated by its worst relative error), or
// -1e300 for a zero row. One CTA per row (grid-stride over rows).
__global__ void __launch_bounds__(256)
k_row_log2norm(const int64_t *__restrict__ A, int64_t lda, int64_t m, int64_t n, double *__restrict__ out)
{
    __shared__ double part[8];
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
        double s = 0.0;
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
            const double v = (double)A[i * lda + j];
            s += v * v;
        }
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
            // every term and partial sum carries at most (n + 8) roundings of 2^-53 each,
            // and the int64 -> double conversion one more per entry
            const double up = 1.0 + (double)(n + 40) * 0x1p-50;
            out[i] = t > 0.0 ? 0.5 * log2(t * up) + 1e-12 : -1e300;
        }
        __syncthreads();
    }
}

cudaError_t launch_row_log2norm(const int64_t *A, int64_t lda, int64_t m, int64_t n, double *out, cudaStream_t st)
{
    if (m <= 0) return cudaSuccess;
    const int64_t nb = m < 152 * 8 ? m : 152 * 8;
    k_row_log2norm<<<(unsigned)nb, 256, 0, st>>>(A, lda, m, n, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Host arithmetic
// ---------------------------------------------------------------------------
namespace {

uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)((unsigned __int128)a * b % p); }

uint64_t powmod(uint64_t b, uint64_t e, uint64_t p)
{
    uint64_t r = 1 % p;
    b %= p;
    while (e) {
        if (e & 1) r = mulmod(r, b, p);
        b = mulmod(b, b, p);
        e >>= 1;
    }
    return r;
}

// x <- x * f + a on little-endian base-2^32 words
void big_muladd(std::vector<uint32_t> &x, uint32_t f, uint32_t a)
{
    uint64_t carry = a;
    for (auto &w : x) {
        const uint64_t t = (uint64_t)w * f + carry;
        w = (uint32_t)t;
        carry = t >> 32;
    }
    if (carry) x.push_back((uint32_t)carry);
}

void big_trim(std::vector<uint32_t> &x)
{
    while (!x.empty() && x.back() == 0) x.pop_back();
}

// -1, 0, 1 as a < b, a == b, a > b (trimmed operands)
int big_cmp(const std::vector<uint32_t> &a, const std::vector<uint32_t> &b)
{
    if (a.size() != b.size()) return a.size() < b.size() ? -1 : 1;
    for (size_t i = a.size(); i-- > 0;)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}

// a - b for a >= b (trimmed result)
std::vector<uint32_t> big_sub(const std::vector<uint32_t> &a, const std::vector<uint32_t> &b)
{
    std::vector<uint32_t> r(a.size());
    int64_t borrow = 0;
    for (size_t i = 0; i < a.size(); ++i) {
        int64_t t = (int64_t)a[i] - borrow - (i < b.size() ? (int64_t)b[i] : 0);
        borrow = t < 0;
        r[i] = (uint32_t)(t + (borrow << 32));
    }
    big_trim(r);
    return r;
}

}  // namespace

bool cup_internal_crt(const uint32_t *res, const uint32_t *pr, int64_t K, std::vector<uint32_t> &mag, int &sign)
{
    // Mixed radix digits (Garner): x = v0 + v1 p0 + v2 p0 p1 + ..., 0 <= vi < pi
    std::vector<uint32_t> v((size_t)K);
    for (int64_t i = 0; i < K; ++i) {
        const uint64_t p = pr[i];
        uint64_t acc = 0, prod = 1 % p;
        for (int64_t j = i - 1; j >= 0; --j) acc = (mulmod(acc, pr[j], p) + v[(size_t)j]) % p;
        for (int64_t j = 0; j < i; ++j) prod = mulmod(prod, pr[j], p);
        if (prod == 0) return false;                       // primes not pairwise distinct
        const uint64_t diff = (res[i] % p + p - acc) % p;
        v[(size_t)i] = (uint32_t)mulmod(diff, powmod(prod, p - 2, p), p);
    }
    std::vector<uint32_t> x, M(1, 1u);
    for (int64_t i = K - 1; i >= 0; --i) big_muladd(x, pr[i], v[(size_t)i]);
    for (int64_t i = 0; i < K; ++i) big_muladd(M, pr[i], 0);
    big_trim(x);
    big_trim(M);
    // symmetric range: x > M / 2 stands for x - M
    std::vector<uint32_t> x2 = x;
    big_muladd(x2, 2u, 0u);
    big_trim(x2);
    if (big_cmp(x2, M) > 0) {
        mag = big_sub(M, x);
        sign = mag.empty() ? 0 : -1;
    } else {
        mag = x;
        sign = mag.empty() ? 0 : 1;
    }
    return true;
}

bool cup_internal_is_prime(uint32_t n)
{
    if (n < 2) return false;
    for (uint32_t q : {2u, 3u, 5u, 7u})
        if (n % q == 0) return n == q;
    uint32_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; ++s; }
    for (uint32_t a : {2u, 3u, 5u, 7u}) {             // deterministic below 3.2e9
        uint64_t x = powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < s; ++i) {
            x = mulmod(x, x, n);
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

int64_t cup_internal_primes_below(uint32_t bound, int64_t count, uint32_t *out)
{
    int64_t got = 0;
    for (uint32_t q = bound; q > 2 && got < count;) {
        --q;
        if (cup_internal_is_prime(q)) out[got++] = q;
    }
    return got;
}
