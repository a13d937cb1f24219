// Batched CUP of many independent matrices, each over its own prime field
// (the multi-modular setting of Sec. 1: one integer problem reduced modulo
// many primes), in one persistent launch.
//
// Each CTA takes the next matrix from a device counter and factors it in
// place with the pivot rule of Algorithm 6 (rows in order; the pivot is the
// first nonzero of the row's residual at a position >= the current rank,
// transposed with that position): a right-looking fraction-free elimination
// over the matrix in global memory (Montgomery reductions for odd p), then
// the normalisation of C's columns and U's rows and the move of U's rows up
// to rows 0..r-1 (the compaction step of Algorithm 6), leaving [C\U].
// Every per-matrix constant (the modulus, its Montgomery inverse and R^2,
// the Barrett reciprocal) is computed on the device.
#include <climits>
#include "cup_internal.cuh"
#include "../../include/cup_gb300.h"

namespace {

constexpr int BT = 512;          // threads per CTA
constexpr int BMAXR = 2048;      // largest min(m, n) of a batched matrix (pivot bookkeeping in smem)

__device__ bool dev_is_prime(uint32_t n)
{
    if (n < 2) return false;
    const uint32_t small[4] = {2u, 3u, 5u, 7u};
    for (int i = 0; i < 4; ++i)
        if (n % small[i] == 0) return n == small[i];
    uint32_t d = n - 1;
    int s = 0;
    while ((d & 1u) == 0) { d >>= 1; ++s; }
    for (int i = 0; i < 4; ++i) {
        uint64_t x = 1, b = small[i] % n;
        for (uint32_t e = d; e; e >>= 1) {
            if (e & 1u) x = x * b % n;
            b = b * b % n;
        }
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int k = 1; k < s; ++k) {
            x = x * x % n;
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

__device__ ModP dev_modp(uint32_t p)
{
    ModP M;
    M.p = p;
    M.mu = ~0ull / p;
    M.r64 = (uint32_t)((~0ull % p + 1) % p);
    uint32_t x = p;
    for (int i = 0; i < 5; ++i) x *= 2u - p * x;
    M.pneg = (p & 1u) ? (uint32_t)(0u - x) : 0u;
    const uint64_t r = (1ull << 32) % p;
    M.r2 = (uint32_t)(r * r % p);
    return M;
}

template <bool MONT>
__device__ __forceinline__ uint32_t bff(uint32_t f, uint32_t x, uint32_t m, uint32_t y, const ModP &M)
{
    return MONT ? ffupd_mont(f, x, m, y, M) : ffupd(f, x, m, y, M);
}

template <bool MONT>
__device__ void factor_one(const cup_batch_item &it, const ModP M, int64_t *rank_out, uint32_t *det_out,
                           int *s_piv_row, uint32_t *s_f, uint32_t *s_inv, int *s_red)
{
    uint32_t *A = it.A;
    const int64_t m = it.m, n = it.n, lda = it.lda;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t one = 1u % M.p;
    int64_t r = 0;
    uint32_t Sprod = one;
    int nswap = 0;
    for (int64_t i = 0; i < m && r < n; ++i) {
        uint32_t *row = A + i * lda;
        // first nonzero of row i at a position >= r
        if (tid == 0) s_red[0] = INT_MAX;
        __syncthreads();
        for (int64_t q = r + tid; q < n; q += nt)
            if (row[q]) { atomicMin(&s_red[0], (int)q); break; }
        __syncthreads();
        const int c = s_red[0];
        __syncthreads();
        if (c == INT_MAX) continue;                       // row i is not in the profile
        if (c != r) {                                     // transposition T_{r,c} on every row
            for (int64_t k = tid; k < m; k += nt) {
                uint32_t *rk = A + k * lda;
                const uint32_t x = rk[r];
                rk[r] = rk[c];
                rk[c] = x;
            }
            ++nswap;
            __syncthreads();
        }
        const uint32_t f = row[r];
        if (tid == 0) {
            it.ipiv[r] = c;
            it.profile[r] = i;
            s_piv_row[r] = (int)i;
            s_f[r] = f;
        }
        // rows below: x <- f x - m y over positions > r (warps along rows, lanes along columns)
        for (int64_t ii = i + 1 + warp; ii < m; ii += nt / 32) {
            uint32_t *rw = A + ii * lda;
            const uint32_t mm = rw[r];
            for (int64_t q = r + 1 + lane; q < n; q += 32) rw[q] = bff<MONT>(f, rw[q], mm, row[q], M);
        }
        __syncthreads();
        Sprod = MONT ? redc((uint64_t)Sprod * f, M) : mulm(Sprod, f, M);
        ++r;
    }
    // scale of step t is mu_t = f_t (R^{-1} f_t for Montgomery): C[., t] carries prod_{t'<t} mu,
    // the pivot row of step t carries f_t
    for (int64_t t = tid; t < r; t += nt) {
        const uint32_t mu = MONT ? redc((uint64_t)s_f[t], M) : s_f[t];
        s_inv[t] = invm(mu, M);                          // mu_t^{-1}
    }
    __syncthreads();
    if (warp == 0) {
        // exclusive prefix products Sinv_t = prod_{t'<t} mu_{t'}^{-1}
        uint32_t carry = one;
        for (int64_t base = 0; base < r; base += 32) {
            const int64_t t = base + lane;
            uint32_t v = (t < r) ? s_inv[t] : one;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v = mulm(v, u, M);
            }
            uint32_t ex = __shfl_up_sync(0xffffffffu, v, 1);
            if (lane == 0) ex = one;
            if (t < r) {
                // pivot-row inverse f_t^{-1} = mu_t^{-1} R^{-1} (Montgomery); Sinv_t into s_inv
                const uint32_t finv = MONT ? redc((uint64_t)s_inv[t], M) : s_inv[t];
                s_f[t] = finv;
                s_inv[t] = mulm(carry, ex, M);
            }
            carry = mulm(carry, __shfl_sync(0xffffffffu, v, 31), M);
        }
    }
    __syncthreads();
    // normalise: C[i][t] = W[i][t] Sinv_t for i >= i_t; U_t = W[i_t][j] f_t^{-1} for j > t
    for (int64_t t = warp; t < r; t += nt / 32) {
        const int64_t it_ = s_piv_row[t];
        const uint32_t sinv = s_inv[t], finv = s_f[t];
        for (int64_t i = it_ + lane; i < m; i += 32) A[i * lda + t] = mulm(A[i * lda + t], sinv, M);
        uint32_t *pr = A + it_ * lda;
        for (int64_t j = t + 1 + lane; j < n; j += 32) pr[j] = mulm(pr[j], finv, M);
    }
    __syncthreads();
    // move U's rows up: row i_t's entries right of t go to row t (then cleared in row i_t)
    for (int64_t t = 0; t < r; ++t) {
        const int64_t it_ = s_piv_row[t];
        if (it_ != t) {
            uint32_t *src = A + it_ * lda, *dst = A + t * lda;
            for (int64_t j = t + 1 + tid; j < n; j += nt) {
                const uint32_t v = src[j];
                src[j] = 0u;
                dst[j] = v;
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        *rank_out = r;
        if (det_out) {
            uint32_t d = 0u;
            if (m == n && r == n) {
                d = one;
                for (int64_t t = 0; t < n; ++t) d = mulm(d, A[t * lda + t], M);
                if ((nswap & 1) && d) d = M.p - d;
            }
            *det_out = d;
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(BT)
k_cup_batched(const cup_batch_item *__restrict__ items, int64_t count, int64_t *__restrict__ ranks,
              uint32_t *__restrict__ dets, unsigned long long *__restrict__ next)
{
    __shared__ int s_piv_row[BMAXR];
    __shared__ uint32_t s_f[BMAXR], s_inv[BMAXR];
    __shared__ int s_red[2];
    __shared__ long long s_b;
    for (;;) {
        if (threadIdx.x == 0) s_b = (long long)atomicAdd(next, 1ull);
        __syncthreads();
        const long long b = s_b;
        __syncthreads();
        if (b >= count) break;
        const cup_batch_item it = items[b];
        const int64_t k = it.m < it.n ? it.m : it.n;
        const bool ok = it.A && it.m >= 0 && it.n >= 0 && it.lda >= (it.n > 0 ? it.n : 1) && k <= BMAXR &&
                        (k == 0 || (it.profile && it.ipiv)) && dev_is_prime(it.p) && it.p < (1u << 31);
        if (!ok) {
            if (threadIdx.x == 0) {
                ranks[b] = -1;
                if (dets) dets[b] = 0u;
            }
            continue;
        }
        const ModP M = dev_modp(it.p);
        if (it.p & 1u) factor_one<true>(it, M, ranks + b, dets ? dets + b : nullptr, s_piv_row, s_f, s_inv, s_red);
        else factor_one<false>(it, M, ranks + b, dets ? dets + b : nullptr, s_piv_row, s_f, s_inv, s_red);
    }
}

}  // namespace

cudaError_t launch_cup_batched(const cup_batch_item *items, int64_t count, int64_t *ranks, uint32_t *dets,
                               unsigned long long *next, int grid, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_cup_batched<<<grid, BT, 0, st>>>(items, count, ranks, dets, next);
    return cudaGetLastError();
}
