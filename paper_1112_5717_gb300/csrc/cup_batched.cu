// Batched CUP of many independent matrices, each over its own prime field
// (the multi-modular setting of Sec. 1: one integer problem reduced modulo
// many primes), in one persistent launch.
//
// Each CTA takes the next matrix from a device work list (largest first) and
// factors it in place with the pivot rule of Algorithm 6 (rows in order; the
// pivot is the first nonzero of the row's residual at a position >= the current
// rank, transposed with that position), leaving [C\U]. Every per-matrix
// constant (the modulus, its Montgomery inverse and R^2, the Barrett
// reciprocal) is computed on the device.
//
// Matrices up to NB_MAXW columns are factored blocked, as Algorithm 6 does at
// one level of its recursion with a 32-row top block: the panel's rows are
// eliminated in shared memory over the whole width (fraction-free, scales
// divided out at the end, so no field inversion sits on the per-row path and no
// row needs speculation), then every row below takes the panel's transpositions,
// its C entries by forward substitution against the panel's unit upper block
// (the TRSM step), and the rank-32 update of its remaining columns (the MM step)
// with the panel's U rows held in registers and 64-bit sums reduced every NR
// products. Wider matrices take an unblocked right-looking elimination in
// global memory.
#include <climits>
#include "cup_internal.cuh"
#include "../../include/cup_gb300.h"

namespace {

constexpr int BT = 512;          // threads per CTA
constexpr int BMAXR = 2048;      // largest min(m, n) of a batched matrix (pivot bookkeeping in smem)
constexpr int NB_PB = 32;        // panel rows of the blocked path
constexpr int NB_MAXW = 1024;    // widest matrix of the blocked path (its panel lives in shared memory)
constexpr int NB_LDP = NB_MAXW + 1;   // panel row stride (odd: column accesses hit distinct banks)
constexpr int NB_LDC = NB_PB + 1;     // stride of the trailing rows' C entries
// dynamic shared memory: panel | C entries of BT trailing rows | pivot rows | small arrays
constexpr size_t NB_OFF_C = (size_t)NB_PB * NB_LDP * 4;
constexpr size_t NB_OFF_PIV = NB_OFF_C + (size_t)BT * NB_LDC * 4;
constexpr size_t NB_OFF_SMALL = NB_OFF_PIV + (size_t)BMAXR * 4;
constexpr size_t NB_SMEM = NB_OFF_SMALL + 8 * NB_PB * 4 + 64;
static_assert(2 * (size_t)BMAXR * 4 <= NB_OFF_C, "the unblocked path's arrays fit in the panel's space");

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

// sum_t a[t] b[t] mod p for 32 residues each (zeros past the panel's pivots): 64-bit
// sums of NR products (NR (p-1)^2 < 2^64), each reduced once
template <int NR>
__device__ __forceinline__ uint32_t dot32(const uint32_t *a, const uint32_t (&b)[NB_PB], const ModP &M)
{
    uint32_t acc = 0u;
#pragma unroll
    for (int t0 = 0; t0 < NB_PB; t0 += NR) {
        uint64_t s = 0;
#pragma unroll
        for (int t = t0; t < t0 + NR && t < NB_PB; ++t) s += (uint64_t)a[t] * b[t];
        acc = addm(acc, red64(s, M), M);
    }
    return acc;
}

template <bool MONT, int NR>
__device__ void factor_blocked(const cup_batch_item &it, const ModP M, int64_t *rank_out, uint32_t *det_out,
                               uint8_t *smem)
{
    uint32_t *P = (uint32_t *)smem;                          // panel: NB_PB rows x NB_LDP
    uint32_t *Cb = (uint32_t *)(smem + NB_OFF_C);            // C entries of up to BT trailing rows
    int *s_piv_row = (int *)(smem + NB_OFF_PIV);             // row of every pivot of the matrix
    int *s_prow = (int *)(smem + NB_OFF_SMALL);              // panel row of the panel's pivot t
    int *s_swp = s_prow + NB_PB;                             // position exchanged with position t
    int *s_rowpiv = s_swp + NB_PB;                           // pivot index of panel row k, or -1
    uint32_t *s_f = (uint32_t *)(s_rowpiv + NB_PB);          // pivot of step t as stored (scaled)
    uint32_t *s_finv = s_f + NB_PB;                          // its inverse
    uint32_t *s_muinv = s_finv + NB_PB;                      // inverse of the row scale of step t
    uint32_t *s_Sinv = s_muinv + NB_PB;                      // prod_{t' < t} of those
    int *s_misc = (int *)(s_Sinv + NB_PB);                   // search results (two slots)
    uint32_t *A = it.A;
    const int64_t m = it.m, n = it.n, lda = it.lda;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const uint32_t one = 1u % M.p;
    int64_t r = 0;
    int nswap = 0;
    for (int64_t i0 = 0; i0 < m && r < n; i0 += NB_PB) {
        const int rows = (int)((m - i0) < NB_PB ? (m - i0) : NB_PB);
        const int W = (int)(n - r);
        for (int k = warp; k < rows; k += nw) {
            const uint32_t *src = A + (i0 + k) * lda + r;
            for (int q = lane; q < W; q += 32) P[k * NB_LDP + q] = src[q];
        }
        if (tid < NB_PB) s_rowpiv[tid] = -1;
        __syncthreads();
        // (1) the panel's rows in order, fraction-free: x <- f x - x[rr] y over positions > rr
        int rr = 0;
        for (int i = 0; i < rows && rr < W; ++i) {
            if (warp == 0) {
                int c = -1;
                for (int q0 = rr; q0 < W; q0 += 32) {
                    const int q = q0 + lane;
                    const unsigned bal = __ballot_sync(0xffffffffu, q < W && P[i * NB_LDP + q] != 0u);
                    if (bal) { c = q0 + __ffs(bal) - 1; break; }
                }
                if (lane == 0) s_misc[i & 1] = c;
            }
            __syncthreads();
            const int c = s_misc[i & 1];
            if (c < 0) continue;                              // row i's residual is zero: not in the profile
            if (c != rr) {                                    // transposition of positions rr and c
                for (int k = tid; k < rows; k += nt) {
                    const uint32_t x = P[k * NB_LDP + rr];
                    P[k * NB_LDP + rr] = P[k * NB_LDP + c];
                    P[k * NB_LDP + c] = x;
                }
                ++nswap;
                __syncthreads();
            }
            const uint32_t f = P[i * NB_LDP + rr];
            if (tid == 0) {
                s_swp[rr] = c;
                s_prow[rr] = i;
                s_rowpiv[i] = rr;
                s_f[rr] = f;
                s_piv_row[r + rr] = (int)(i0 + i);
                it.ipiv[r + rr] = r + c;
                it.profile[r + rr] = i0 + i;
            }
            const uint32_t *y = P + i * NB_LDP;
            for (int k = i + 1 + warp; k < rows; k += nw) {
                uint32_t *xk = P + k * NB_LDP;
                const uint32_t mk = xk[rr];
                for (int q = rr + 1 + lane; q < W; q += 32) xk[q] = bff<MONT>(f, xk[q], mk, y[q], M);
            }
            __syncthreads();
            ++rr;
        }
        const int pb = rr;
        if (pb == 0) continue;          // no pivot: the rows' residuals (already in A) are zero past r
        // (2) scales: step t multiplied the rows below its pivot row by mu_t (f_t, or R^{-1} f_t
        // with Montgomery steps), so a C entry of column t carries prod_{t' < t} mu_t' and
        // the pivot row of step t carries f_t
        for (int t = tid; t < pb; t += nt) {
            const uint32_t mu = MONT ? redc((uint64_t)s_f[t], M) : s_f[t];
            const uint32_t mi = MONT ? invm_mont(mu, M) : invm(mu, M);
            s_muinv[t] = mi;
            s_finv[t] = MONT ? redc((uint64_t)mi, M) : mi;
        }
        __syncthreads();
        if (warp == 0) {
            uint32_t v = (lane < pb) ? s_muinv[lane] : one;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v = mulm(v, u, M);
            }
            uint32_t ex = __shfl_up_sync(0xffffffffu, v, 1);
            if (lane == 0) ex = one;
            if (lane < pb) s_Sinv[lane] = ex;
        }
        __syncthreads();
        // (3) normalise the panel: C entries (positions t <= the row's own pivot) times Sinv_t,
        // U entries (right of the row's pivot) times f^{-1}; dependent rows are zero past
        // their C entries. Then write it back.
        for (int k = warp; k < rows; k += nw) {
            const int tk = s_rowpiv[k];
            uint32_t *xk = P + k * NB_LDP;
            uint32_t *dst = A + (i0 + k) * lda + r;
            for (int q = lane; q < W; q += 32) {
                uint32_t v = xk[q];
                if (q < pb && k >= s_prow[q]) v = mulm(v, s_Sinv[q], M);
                else if (tk >= 0) v = mulm(v, s_finv[tk], M);
                xk[q] = v;
                dst[q] = v;
            }
        }
        __syncthreads();
        // (4) the panel's transpositions on the earlier pivot rows (their U entries) and on
        // every row below the panel
        bool any = false;
        for (int t = 0; t < pb; ++t) any |= s_swp[t] != t;
        const int64_t below0 = i0 + rows, nbelow = m - below0;
        if (any) {
            for (int64_t x = tid; x < r + nbelow; x += nt) {
                const int64_t g = x < r ? (int64_t)s_piv_row[x] : below0 + (x - r);
                uint32_t *row = A + g * lda + r;
                for (int t = 0; t < pb; ++t) {
                    const int c = s_swp[t];
                    if (c != t) {
                        const uint32_t v = row[t];
                        row[t] = row[c];
                        row[c] = v;
                    }
                }
            }
            __syncthreads();
        }
        // (5) rows below, BT at a time: C entries c = y U_pp^{-1} (y = the row at the
        // pivot positions, U_pp the panel's unit upper block) by forward substitution,
        // one thread a row; then x <- x - c U over the positions right of the pivots, one
        // thread per column with the U entries of its columns in registers
        const int j0 = pb + tid, j1 = pb + tid + nt;
        for (int64_t c0 = below0; c0 < m; c0 += BT) {
            const int cnt = (int)((m - c0) < BT ? (m - c0) : BT);
            if (tid < cnt) {
                uint32_t *row = A + (c0 + tid) * lda + r;
                uint32_t cv[NB_PB];
#pragma unroll
                for (int t = 0; t < NB_PB; ++t) cv[t] = (t < pb) ? row[t] : 0u;
#pragma unroll
                for (int t = 1; t < NB_PB; ++t) {
                    if (t < pb) {
                        uint32_t acc = 0u;
#pragma unroll
                        for (int t0 = 0; t0 < t; t0 += NR) {
                            uint64_t sum = 0;
#pragma unroll
                            for (int tp = t0; tp < t0 + NR && tp < t; ++tp)
                                sum += (uint64_t)cv[tp] * P[s_prow[tp] * NB_LDP + t];
                            acc = addm(acc, red64(sum, M), M);
                        }
                        cv[t] = subm(cv[t], acc, M);
                    }
                }
                uint32_t *cb = Cb + tid * NB_LDC;
#pragma unroll
                for (int t = 0; t < NB_PB; ++t) {
                    cb[t] = cv[t];
                    if (t < pb) row[t] = cv[t];
                }
            }
            __syncthreads();
            // one column at a time (its 32 U entries in registers), both passes over the rows
            for (int j = j0; j < W && j < j1 + 1; j += nt) {
                uint32_t u[NB_PB];
#pragma unroll
                for (int t = 0; t < NB_PB; ++t) u[t] = t < pb ? P[s_prow[t] * NB_LDP + j] : 0u;
                for (int k = 0; k < cnt; ++k) {
                    uint32_t *row = A + (c0 + k) * lda + r;
                    row[j] = subm(row[j], dot32<NR>(Cb + k * NB_LDC, u, M), M);
                }
            }
            __syncthreads();
        }
        r += pb;
    }
    // U's rows up to rows 0 .. r-1 (row i_t's entries right of t go to row t, then cleared
    // in row i_t): a move may read a row that an earlier move wrote, so they run in order
    for (int64_t t = 0; t < r; ++t) {
        const int64_t it_ = s_piv_row[t];
        if (it_ != t) {
            uint32_t *src = A + it_ * lda, *dst = A + t * lda;
            for (int64_t j = t + 1 + tid; j < n; j += nt) {
                const uint32_t v = src[j];
                src[j] = 0u;
                dst[j] = v;
            }
            __syncthreads();
        }
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

__global__ void __launch_bounds__(BT, 1)
k_cup_batched(const cup_batch_item *__restrict__ items, int64_t count, int64_t *__restrict__ ranks,
              uint32_t *__restrict__ dets, unsigned long long *__restrict__ next, const int *__restrict__ order)
{
    extern __shared__ __align__(16) uint8_t bsm[];
    int *s_piv_row = (int *)(bsm + NB_OFF_PIV);
    uint32_t *s_f = (uint32_t *)bsm, *s_inv = s_f + BMAXR;     // unblocked path: inside the panel's space
    int *s_red = (int *)(bsm + NB_OFF_SMALL);
    __shared__ long long s_b;
    for (;;) {
        if (threadIdx.x == 0) s_b = (long long)atomicAdd(next, 1ull);
        __syncthreads();
        const long long bi = s_b;
        __syncthreads();
        if (bi >= count) break;
        const long long b = order ? (long long)order[bi] : bi;
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
        uint32_t *dp = dets ? dets + b : nullptr;
        if (it.n <= NB_MAXW) {
            // products summed in 64 bits before a reduction: NR (p - 1)^2 < 2^64
            const uint64_t q = (uint64_t)(it.p - 1) * (it.p - 1);
            const bool odd = it.p & 1u;
            if (q <= ~0ull / 32) {
                if (odd) factor_blocked<true, 32>(it, M, ranks + b, dp, bsm);
                else factor_blocked<false, 32>(it, M, ranks + b, dp, bsm);
            } else if (q <= ~0ull / 16) {
                factor_blocked<true, 16>(it, M, ranks + b, dp, bsm);
            } else {
                factor_blocked<true, 4>(it, M, ranks + b, dp, bsm);
            }
        } else if (it.p & 1u) {
            factor_one<true>(it, M, ranks + b, dp, s_piv_row, s_f, s_inv, s_red);
        } else {
            factor_one<false>(it, M, ranks + b, dp, s_piv_row, s_f, s_inv, s_red);
        }
    }
}

// Work order of the batched launch: items by decreasing cost (m n min(m, n), in
// buckets of powers of two), so the largest factorisations start first and the
// small ones fill in behind them. One CTA; invalid items cost nothing here (the
// factor kernel rejects them).
__global__ void __launch_bounds__(1024)
k_batched_order(const cup_batch_item *__restrict__ items, int64_t count, int *__restrict__ order)
{
    constexpr int NBK = 64;
    __shared__ int cnt[NBK], base[NBK];
    if (threadIdx.x < NBK) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t b = threadIdx.x; b < count; b += blockDim.x) {
        const cup_batch_item it = items[b];
        const double k = (double)(it.m < it.n ? it.m : it.n);
        const double c = (it.m > 0 && it.n > 0) ? (double)it.m * (double)it.n * k : 1.0;
        int e = 0;
        frexp(c, &e);
        const int bk = NBK - 1 - (e < 0 ? 0 : (e > NBK - 1 ? NBK - 1 : e));   // larger cost, earlier bucket
        atomicAdd(&cnt[bk], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int i = 0; i < NBK; ++i) { base[i] = acc; acc += cnt[i]; }
    }
    __syncthreads();
    for (int64_t b = threadIdx.x; b < count; b += blockDim.x) {
        const cup_batch_item it = items[b];
        const double k = (double)(it.m < it.n ? it.m : it.n);
        const double c = (it.m > 0 && it.n > 0) ? (double)it.m * (double)it.n * k : 1.0;
        int e = 0;
        frexp(c, &e);
        const int bk = NBK - 1 - (e < 0 ? 0 : (e > NBK - 1 ? NBK - 1 : e));
        order[atomicAdd(&base[bk], 1)] = (int)b;
    }
}

}  // namespace

cudaError_t launch_cup_batched(const cup_batch_item *items, int64_t count, int64_t *ranks, uint32_t *dets,
                               unsigned long long *next, int *order, int grid, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    if (count > INT_MAX) return cudaErrorInvalidValue;
    static PerDeviceOnce attr;
    cudaError_t e = once_per_device(attr, [] {
        return cudaFuncSetAttribute(k_cup_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NB_SMEM);
    });
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (order) {
        k_batched_order<<<1, 1024, 0, st>>>(items, count, order);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_cup_batched<<<grid, BT, NB_SMEM, st>>>(items, count, ranks, dets, next, order);
    return cudaGetLastError();
}
