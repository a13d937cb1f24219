// Triangular building blocks of Sec. 3.2 at their base (blocks of at most 64),
// plus the small data-movement kernels the derived problems need.
//
// k_tri_right: B <- B T^{-1} or B <- B T   (one warp per row of B)
// k_tri_left:  B <- T^{-1} B or B <- T B   (one thread per column of B)
// with T upper or lower, unit or non-unit diagonal. The recursive drivers in
// cup_api.cu split larger triangles in halves and hand the off-diagonal
// products to the Schur-update engine (Algorithm 2 and its variants, TRMM,
// Algorithm 3 TRTRI, Algorithm 4 TRULM).
#include "cup_internal.cuh"

#define TRI_MAX 64

template <bool MONT>
__device__ __forceinline__ uint32_t mmul(uint32_t a, uint32_t bm, const ModP &M)
{
    // bm is in Montgomery form (b R mod p) when MONT
    return MONT ? redc((uint64_t)a * bm, M) : mulm(a, bm, M);
}

template <bool MONT>
__device__ __forceinline__ uint32_t to_mont(uint32_t b, const ModP &M)
{
    return MONT ? redc((uint64_t)b * M.r2, M) : b;
}

// Load the n x n triangle (only the triangle that is read) and its diagonal:
// sD[k] = 1 for unit, T[k][k] for multiply, T[k][k]^{-1} for solve.
template <bool UPPER, bool UNIT, bool SOLVE, bool MONT>
__device__ void load_tri(const uint32_t *T, int64_t ldt, int n, const ModP &M,
                         uint32_t (*sT)[TRI_MAX + 1], uint32_t *sD)
{
    for (int base = threadIdx.x; base < TRI_MAX * TRI_MAX; base += 8 * blockDim.x) {
        uint32_t v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int idx = base + e * blockDim.x;
            const int k = idx / TRI_MAX, j = idx - k * TRI_MAX;
            const bool in = idx < TRI_MAX * TRI_MAX && (k < n && j < n) && (UPPER ? (j > k) : (j < k));
            v[e] = in ? T[k * ldt + j] : 0u;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int idx = base + e * blockDim.x;
            if (idx < TRI_MAX * TRI_MAX) sT[idx / TRI_MAX][idx % TRI_MAX] = to_mont<MONT>(v[e], M);
        }
    }
    for (int k = threadIdx.x; k < TRI_MAX; k += blockDim.x) {
        uint32_t d = 1u % M.p;
        if (!UNIT && k < n) {
            d = T[k * ldt + k];
            if (SOLVE) d = MONT ? invm_mont(d, M) : invm(d, M);
        }
        sD[k] = to_mont<MONT>(d, M);
    }
}

template <bool UPPER, bool UNIT, bool SOLVE, bool MONT>
__global__ void __launch_bounds__(256)
k_tri_right(const TriDesc d, ModP M)
{
    pdl_enter();
    const int n = (int)d.n.eval();
    if (n <= 0) return;
    const int64_t m = d.rows, ldt = d.ldt, ldb = d.ldb;
    const uint32_t *__restrict__ T = d.T + d.trow.eval() * ldt + d.tcol.eval();
    uint32_t *__restrict__ B = d.B + d.brow.eval() * ldb + d.bcol.eval();
    __shared__ uint32_t sT[TRI_MAX][TRI_MAX + 1];
    __shared__ uint32_t sD[TRI_MAX];
    load_tri<UPPER, UNIT, SOLVE, MONT>(T, ldt, n, M, sT, sD);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < m; i += nw) {
        uint32_t *row = B + i * ldb;
        uint32_t x0 = (lane < n) ? row[lane] : 0u;
        uint32_t x1 = (lane + 32 < n) ? row[lane + 32] : 0u;
        if (SOLVE) {
            // X T = B: columns in dependency order, each finalised then broadcast
            for (int s = 0; s < n; ++s) {
                const int k = UPPER ? s : n - 1 - s;
                if (!UNIT) {
                    if (lane == (k & 31)) {
                        if (k < 32) x0 = mmul<MONT>(x0, sD[k], M);
                        else x1 = mmul<MONT>(x1, sD[k], M);
                    }
                }
                const uint32_t xk = __shfl_sync(0xffffffffu, k < 32 ? x0 : x1, k & 31);
                if (xk) {
                    x0 = subm(x0, mmul<MONT>(xk, sT[k][lane], M), M);
                    x1 = subm(x1, mmul<MONT>(xk, sT[k][lane + 32], M), M);
                }
            }
        } else {
            // Y = B T: y_j = sum_k b_k t_kj over the triangle, plus the diagonal
            uint32_t y0 = mmul<MONT>(x0, sD[lane], M), y1 = mmul<MONT>(x1, sD[lane + 32], M);
            for (int k = 0; k < n; ++k) {
                const uint32_t xk = __shfl_sync(0xffffffffu, k < 32 ? x0 : x1, k & 31);
                if (xk) {
                    y0 = addm(y0, mmul<MONT>(xk, sT[k][lane], M), M);
                    y1 = addm(y1, mmul<MONT>(xk, sT[k][lane + 32], M), M);
                }
            }
            x0 = y0;
            x1 = y1;
        }
        if (lane < n) row[lane] = x0;
        if (lane + 32 < n) row[lane + 32] = x1;
    }
}

// B <- T^{-1} B or B <- T B for n <= 64 rows of B: a CTA takes 32 columns, loads the
// 64 x 32 tile row by row (coalesced) into shared memory, and each warp works on four
// columns at once with the lanes along the rows (rows lane and lane + 32): a solve
// finalises row i, broadcasts it from its lane and the dependent rows subtract
// t_ki x_i (four independent chains per warp); a product needs no chain.
#define TRI_COLS 32
template <bool UPPER, bool UNIT, bool SOLVE, bool MONT>
__global__ void __launch_bounds__(256)
k_tri_left(const uint32_t *__restrict__ T, int64_t ldt, uint32_t *__restrict__ B, int64_t ldb, int n,
           int64_t k, ModP M)
{
    pdl_enter();
    __shared__ uint32_t sT[TRI_MAX][TRI_MAX + 1];
    __shared__ uint32_t sD[TRI_MAX];
    __shared__ uint32_t sB[TRI_MAX][TRI_COLS + 1];
    load_tri<UPPER, UNIT, SOLVE, MONT>(T, ldt, n, M, sT, sD);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t c0 = (int64_t)blockIdx.x * TRI_COLS;
    for (int i = warp; i < n; i += 8) sB[i][lane] = (c0 + lane < k) ? B[i * ldb + c0 + lane] : 0u;
    __syncthreads();
    // warp w: columns w, w + 8, w + 16, w + 24 of the tile
    uint32_t x[4][2];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = warp + 8 * q;
        x[q][0] = (lane < n) ? sB[lane][c] : 0u;
        x[q][1] = (lane + 32 < n) ? sB[lane + 32][c] : 0u;
    }
    if (SOLVE) {
        for (int s = 0; s < n; ++s) {
            const int i = UPPER ? n - 1 - s : s;
            const int hi = i >> 5, li = i & 31;
            // the row's value is final once its diagonal is divided out
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (!UNIT && lane == li) x[q][hi] = mmul<MONT>(x[q][hi], sD[i], M);
            }
            const uint32_t t0 = sT[lane][i], t1 = sT[lane + 32][i];
            const bool d0 = UPPER ? lane < i : lane > i, d1 = UPPER ? lane + 32 < i : lane + 32 > i;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t xi = __shfl_sync(0xffffffffu, hi ? x[q][1] : x[q][0], li);
                if (xi) {
                    if (d0) x[q][0] = subm(x[q][0], mmul<MONT>(xi, t0, M), M);
                    if (d1) x[q][1] = subm(x[q][1], mmul<MONT>(xi, t1, M), M);
                }
            }
        }
    } else {
        // Y = T B: y_i = d_i x_i + sum over the triangle of t_ij x_j
        uint32_t y[4][2];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            y[q][0] = mmul<MONT>(x[q][0], sD[lane], M);
            y[q][1] = mmul<MONT>(x[q][1], sD[lane + 32], M);
        }
        for (int j = 0; j < n; ++j) {
            const int hj = j >> 5, lj = j & 31;
            const uint32_t t0 = sT[lane][j], t1 = sT[lane + 32][j];
            const bool d0 = UPPER ? lane < j : lane > j, d1 = UPPER ? lane + 32 < j : lane + 32 > j;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t xj = __shfl_sync(0xffffffffu, hj ? x[q][1] : x[q][0], lj);
                if (d0) y[q][0] = addm(y[q][0], mmul<MONT>(xj, t0, M), M);
                if (d1) y[q][1] = addm(y[q][1], mmul<MONT>(xj, t1, M), M);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) { x[q][0] = y[q][0]; x[q][1] = y[q][1]; }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = warp + 8 * q;
        if (lane < n) sB[lane][c] = x[q][0];
        if (lane + 32 < n) sB[lane + 32][c] = x[q][1];
    }
    __syncthreads();
    for (int i = warp; i < n; i += 8)
        if (c0 + lane < k) B[i * ldb + c0 + lane] = sB[i][lane];
}

template <bool UPPER, bool UNIT, bool SOLVE>
static cudaError_t tri_dispatch(bool left, const uint32_t *T, int64_t ldt, uint32_t *B, int64_t ldb,
                                int64_t rows, int64_t cols, int n, ModP M, cudaStream_t st)
{
    const bool mont = (M.p & 1u) != 0;
    if (left) {
        const int64_t nb = (cols + TRI_COLS - 1) / TRI_COLS;
        if (mont) launch_pdl(k_tri_left<UPPER, UNIT, SOLVE, true>, (unsigned)nb, 256, 0, st, T, ldt, B, ldb, n, cols, M);
        else launch_pdl(k_tri_left<UPPER, UNIT, SOLVE, false>, (unsigned)nb, 256, 0, st, T, ldt, B, ldb, n, cols, M);
    } else {
        int64_t nb = (rows + 7) / 8;
        if (nb > 152 * 16) nb = 152 * 16;
        TriDesc d{T, ldt, dconst(0), dconst(0), B, ldb, dconst(0), dconst(0), rows, dconst(n)};
        if (mont) launch_pdl(k_tri_right<UPPER, UNIT, SOLVE, true>, (unsigned)nb, 256, 0, st, d, M);
        else launch_pdl(k_tri_right<UPPER, UNIT, SOLVE, false>, (unsigned)nb, 256, 0, st, d, M);
    }
    return cudaGetLastError();
}

cudaError_t launch_tri_leaf(int flags, const uint32_t *T, int64_t ldt, uint32_t *B, int64_t ldb,
                            int64_t rows, int64_t cols, ModP M, cudaStream_t st)
{
    const bool left = flags & TRI_LEFT, upper = flags & TRI_UPPER, unit = flags & TRI_UNIT,
               solve = flags & TRI_SOLVE;
    const int n = (int)(left ? rows : cols);
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if (n > TRI_MAX) return cudaErrorInvalidValue;
    if (upper) {
        if (unit) return solve ? tri_dispatch<true, true, true>(left, T, ldt, B, ldb, rows, cols, n, M, st)
                               : tri_dispatch<true, true, false>(left, T, ldt, B, ldb, rows, cols, n, M, st);
        return solve ? tri_dispatch<true, false, true>(left, T, ldt, B, ldb, rows, cols, n, M, st)
                     : tri_dispatch<true, false, false>(left, T, ldt, B, ldb, rows, cols, n, M, st);
    }
    if (unit) return solve ? tri_dispatch<false, true, true>(left, T, ldt, B, ldb, rows, cols, n, M, st)
                           : tri_dispatch<false, true, false>(left, T, ldt, B, ldb, rows, cols, n, M, st);
    return solve ? tri_dispatch<false, false, true>(left, T, ldt, B, ldb, rows, cols, n, M, st)
                 : tri_dispatch<false, false, false>(left, T, ldt, B, ldb, rows, cols, n, M, st);
}

// TRSM(Right, Upper, Unit) on blocks of up to 128 columns (the TRSM step of
// Algorithm 6): one warp per row of B, each lane holding columns lane + 32 k;
// at step k the final x_k is broadcast and the later columns subtract x_k u_kj.
#define RUU_MAX 128
#define RUU_LDS (RUU_MAX + 4)   // 16-byte aligned rows
#define TRI_VLD 33               // row stride of the 32 x 32 block inverses
// Montgomery reduction of T < 2 p R (p < 2^24) to [0, p): the raw result is below 3p.
__device__ __forceinline__ uint32_t redc_lazy(uint64_t T, const ModP &M)
{
    const uint32_t m = (uint32_t)T * M.pneg;
    uint32_t t = (uint32_t)((T + (uint64_t)m * M.p) >> 32);
    if (t >= M.p) t -= M.p;
    if (t >= M.p) t -= M.p;
    return t;
}

// x mod p for x < 2^39 and p < 2^16: the bits from 24 up are folded with 2^24 mod p
// (the sum stays below 2^32), then one 32-bit Barrett step with mu32 = floor(2^32 / p).
__device__ __forceinline__ uint32_t red39(uint64_t x, uint32_t p, uint32_t c24, uint32_t mu32)
{
    uint32_t t = (uint32_t)(x >> 24) * c24 + (uint32_t)(x & 0xffffffu);
    t -= __umulhi(t, mu32) * p;
    return t >= p ? t - p : t;
}

// MODE 0: per-step Montgomery products (any odd p); 1: lazy Montgomery accumulation
// (odd p < 2^24, the triangle in Montgomery form); 3: p < 2^16, the triangle as it is,
// each 32-column block solved with the inverse of its diagonal block and plain lazy
// sums (products below 2^32, sums below 2^39).
template <int MODE>
__global__ void __launch_bounds__(256)
k_trsm_ruu128(const TriDesc d, ModP M)
{
    // the triangle's load and block inverses run before the wait when d.pre says
    // the triangle and the extents are older than the predecessor kernel
    const bool pre = d.pre != 0;
    if (!pre) pdl_enter();
    constexpr bool MONT = MODE <= 1, LAZY = MODE == 1;
    extern __shared__ __align__(16) uint32_t sU[];        // RUU_MAX x RUU_LDS
    const int n = (int)d.n.eval();
    if (n <= 0) {
        if (pre) pdl_enter();
        return;
    }
    const int64_t m = d.rows, ldt = d.ldt, ldb = d.ldb;
    const uint32_t *__restrict__ T = d.T + d.trow.eval() * ldt + d.tcol.eval();
    uint32_t *__restrict__ B = d.B + d.brow.eval() * ldb + d.bcol.eval();
    // rows 0 .. n-1 of the triangle by asynchronous copies (16-byte pieces when the
    // rows are 16-byte aligned), then one pass keeping only the strictly upper part
    // (zeros elsewhere; rows >= n are never read), in Montgomery form for MODE <= 1
    if (((uintptr_t)T & 15u) == 0 && (ldt & 3) == 0) {
        const int nv = n >> 2;                            // whole 16-byte pieces per row
        for (int idx = threadIdx.x; idx < n * 32; idx += blockDim.x) {
            const int k = idx >> 5, v = idx & 31;
            if (v < nv) cp_async16(sU + k * RUU_LDS + 4 * v, T + k * ldt + 4 * v);
            else if (v == nv)                             // the ragged end of the row, word by word
                for (int j = 4 * nv; j < n; ++j) cp_async4(sU + k * RUU_LDS + j, T + k * ldt + j);
        }
    } else {
        for (int idx = threadIdx.x; idx < n * RUU_MAX; idx += blockDim.x) {
            const int k = idx >> 7, j = idx & (RUU_MAX - 1);
            if (j < n) cp_async4(sU + k * RUU_LDS + j, T + k * ldt + j);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    // MODE 3 reads only the strictly upper part of rows and columns below n and tolerates
    // anything elsewhere (see the solve), so it skips this pass
    for (int base = threadIdx.x; MODE != 3 && base < n * RUU_MAX; base += 8 * blockDim.x) {
        // eight independent entries per pass (all read before any is written)
        uint32_t v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int idx = base + e * blockDim.x, k = idx >> 7, j = idx & (RUU_MAX - 1);
            v[e] = (idx < n * RUU_MAX && j > k && j < n) ? sU[k * RUU_LDS + j] : 0u;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int idx = base + e * blockDim.x, k = idx >> 7, j = idx & (RUU_MAX - 1);
            if (idx < n * RUU_MAX) sU[k * RUU_LDS + j] = MONT ? to_mont<MONT>(v[e], M) : v[e];
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t c24 = (uint32_t)((1u << 24) % M.p), mu32 = (uint32_t)(0xffffffffu / M.p);
    // MODE 3: V_b = inverse of the b-th 32 x 32 diagonal block (unit upper), in two steps.
    // (1) Warp w inverts the 16 x 16 diagonal block w (lane j keeps column j in registers
    // and runs the back substitution V[k][j] = -sum_{l > k} U[k][l] V[l][j] from the
    // bottom row up; rows at or past n stay identity rows), writing it into its quadrant
    // of V_b. (2) With A, D the two 16 x 16 diagonal blocks of block b and B the block
    // between them, V_b's upper-right quadrant is -A^{-1} (B D^{-1}) (two 16 x 16 x 16
    // products over all threads) and its lower-left quadrant is zero. Entries of U outside
    // the strictly upper n x n part are never combined with a nonzero factor in a valid
    // position, so the unmasked triangle is safe; every sum here has at most 16 products
    // below 2^32.
    uint32_t *const sV = sU + RUU_MAX * RUU_LDS;
    if (MODE == 3) {
        const int nblk = (n + 31) >> 5;
        const int wv = threadIdx.x >> 5;
        if (wv < 2 * nblk) {
            const int b = wv >> 1, h = wv & 1, o = 16 * wv, j = lane & 15;
            const int nsb = n - o;                        // valid rows of this sub-block (may be <= 0)
            uint32_t v[16];
#pragma unroll
            for (int l = 0; l < 16; ++l) v[l] = (l == j) ? 1u : 0u;
            // no branch in the chain: every step's loads are unconditional (rows past n
            // lie inside sU) and its result is kept by selection
#pragma unroll
            for (int k = 14; k >= 0; --k) {
                const uint32_t *uk = sU + (o + k) * RUU_LDS + o;
                uint64_t s4[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
                for (int l = k + 1; l < 16; ++l) s4[l & 3] += (uint64_t)uk[l] * v[l];
                const uint32_t r = red39((s4[0] + s4[1]) + (s4[2] + s4[3]), M.p, c24, mu32);
                v[k] = (k < nsb && k < j) ? (r ? M.p - r : 0u) : v[k];
            }
            uint32_t *V = sV + b * 32 * TRI_VLD + 16 * h * (TRI_VLD + 1);
            if (lane < 16) {
#pragma unroll
                for (int k = 0; k < 16; ++k) V[k * TRI_VLD + j] = v[k];
            } else {
                // the lower-left quadrant of V_b is zero (warp 2b writes it)
                if (h == 0) {
                    uint32_t *Z = sV + b * 32 * TRI_VLD + 16 * TRI_VLD;
#pragma unroll
                    for (int k = 0; k < 16; ++k) Z[k * TRI_VLD + j] = 0u;
                }
            }
        }
        __syncthreads();
        uint32_t *const sY = sV + 4 * 32 * TRI_VLD;       // 4 x 16 x 17: B D^{-1} per block
        for (int idx = threadIdx.x; idx < nblk * 256; idx += blockDim.x) {
            const int b = idx >> 8, l = (idx >> 4) & 15, jj = idx & 15;
            const uint32_t *Bl = sU + (32 * b + l) * RUU_LDS + 32 * b + 16;
            const uint32_t *D = sV + b * 32 * TRI_VLD + 16 * TRI_VLD + 16 + jj;
            uint64_t s4[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
            for (int m2 = 0; m2 < 16; ++m2) s4[m2 & 3] += (uint64_t)Bl[m2] * D[m2 * TRI_VLD];
            sY[(b * 16 + l) * 17 + jj] = red39((s4[0] + s4[1]) + (s4[2] + s4[3]), M.p, c24, mu32);
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < nblk * 256; idx += blockDim.x) {
            const int b = idx >> 8, k = (idx >> 4) & 15, jj = idx & 15;
            const uint32_t *Ak = sV + b * 32 * TRI_VLD + k * TRI_VLD;
            uint64_t s4[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
            for (int l = 0; l < 16; ++l) s4[l & 3] += (uint64_t)Ak[l] * sY[(b * 16 + l) * 17 + jj];
            const uint32_t r = red39((s4[0] + s4[1]) + (s4[2] + s4[3]), M.p, c24, mu32);
            sV[b * 32 * TRI_VLD + k * TRI_VLD + 16 + jj] = r ? M.p - r : 0u;
        }
        __syncthreads();
    }
    if (pre) pdl_enter();
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < m; i += nw) {
        uint32_t *row = B + i * ldb;
        if (MODE == 3) {
            // X_b = (B_b - sum_{a < b} X_a U_ab) V_b: the block's solve is 32 independent
            // products per lane (no dependency chain), then the block's values update the
            // later blocks; plain lazy sums (below 2^39) reduced by the 39-bit fold
            uint64_t acc[4];
            uint32_t xo[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                acc[c] = (lane + 32 * c < n) ? (uint64_t)row[lane + 32 * c] : 0ull;
                xo[c] = 0u;
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if (32 * b >= n) break;
                const uint32_t y = red39(acc[b], M.p, c24, mu32);
                const uint32_t *V = sV + b * 32 * TRI_VLD + lane;
                uint64_t s4[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
                for (int k = 0; k < 32; ++k) s4[k & 3] += (uint64_t)__shfl_sync(0xffffffffu, y, k) * V[k * TRI_VLD];
                // lanes at or past n hold no value (their sums may mix unmasked entries): zero
                const uint32_t x = (32 * b + lane < n) ? red39((s4[0] + s4[1]) + (s4[2] + s4[3]), M.p, c24, mu32)
                                                       : 0u;
                xo[b] = x;
                if (b < 3 && 32 * (b + 1) < n) {
                    const uint32_t nx = x ? M.p - x : 0u;
                    const uint32_t *ub = sU + 32 * b * RUU_LDS + lane;
#pragma unroll 4
                    for (int k = 0; k < 32; ++k) {
                        const uint64_t nk = __shfl_sync(0xffffffffu, nx, k);
#pragma unroll
                        for (int c = b + 1; c < 4; ++c) acc[c] += nk * ub[k * RUU_LDS + 32 * c];
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (lane + 32 * c < n) row[lane + 32 * c] = xo[c];
        } else if (LAZY) {
            // x_j = b_j - sum_{k<j} x_k u_kj accumulated unreduced as R b_j + sum (p - x_k) (R u_kj):
            // only column k is reduced at step k (one Montgomery reduction on the chain).
            // With p < 2^24 the sum stays below p R + 128 p^2 < 2 p R, so the
            // reduction lands in [0, 3p).
            uint64_t acc[4];
#pragma unroll
            for (int c = 0; c < 4; ++c)
                acc[c] = (lane + 32 * c < n) ? ((uint64_t)row[lane + 32 * c] << 32) : 0ull;
#pragma unroll
            for (int cb = 0; cb < 4; ++cb) {
                if (32 * cb >= n) break;
                const int kend = n - 32 * cb < 32 ? n - 32 * cb : 32;
                for (int kk = 0; kk < kend; ++kk) {
                    const int k = 32 * cb + kk;
                    const uint32_t t = redc_lazy(acc[cb], M);
                    const uint32_t xk = __shfl_sync(0xffffffffu, t, kk);
                    const uint32_t nx = xk ? M.p - xk : 0u;
                    const uint32_t *uk = sU + k * RUU_LDS + lane;
#pragma unroll
                    for (int c = cb; c < 4; ++c) acc[c] += (uint64_t)nx * uk[32 * c];
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (lane + 32 * c < n) row[lane + 32 * c] = redc_lazy(acc[c], M);
        } else {
            uint32_t x[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) x[c] = (lane + 32 * c < n) ? row[lane + 32 * c] : 0u;
            for (int k = 0; k < n; ++k) {
                const uint32_t src = (k < 32) ? x[0] : (k < 64) ? x[1] : (k < 96) ? x[2] : x[3];
                const uint32_t xk = __shfl_sync(0xffffffffu, src, k & 31);
                if (xk) {
                    const uint32_t *uk = sU + k * RUU_LDS + lane;
#pragma unroll
                    for (int c = 0; c < 4; ++c) x[c] = subm(x[c], mmul<MONT>(xk, uk[32 * c], M), M);
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (lane + 32 * c < n) row[lane + 32 * c] = x[c];
        }
    }
}

cudaError_t launch_trsm_ruu_desc(const TriDesc &d, ModP M, cudaStream_t st)
{
    if (d.rows <= 0 || d.n.hi <= 0) return cudaSuccess;
    if (d.n.hi > RUU_MAX) return cudaErrorInvalidValue;
    static PerDeviceOnce attr;
    const size_t smem = ((size_t)RUU_MAX * RUU_LDS + 4 * 32 * TRI_VLD + 4 * 16 * 17) * sizeof(uint32_t);
    {
        const cudaError_t e = once_per_device(attr, [&] {
            cudaError_t e2 = cudaFuncSetAttribute(k_trsm_ruu128<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e2 == cudaSuccess)
                e2 = cudaFuncSetAttribute(k_trsm_ruu128<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e2 == cudaSuccess)
                e2 = cudaFuncSetAttribute(k_trsm_ruu128<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            return e2;
        });
        if (e != cudaSuccess) return e;
    }
    // one wave of CTAs (two fit an SM): every CTA loads the triangle and, for p < 2^16,
    // inverts its diagonal blocks, so more rows per CTA spread that fixed cost
    int64_t nb = (d.rows + 7) / 8;
    if (nb > 152 * 2) nb = 152 * 2;
    if (M.p < (1u << 16)) return launch_pdl(k_trsm_ruu128<3>, (unsigned)nb, 256, smem, st, d, M);
    if (M.p < (1u << 24)) return launch_pdl(k_trsm_ruu128<1>, (unsigned)nb, 256, smem, st, d, M);
    return launch_pdl(k_trsm_ruu128<0>, (unsigned)nb, 256, smem, st, d, M);
}

// ---------------------------------------------------------------------------
// Small data-movement kernels
// ---------------------------------------------------------------------------
__global__ void k_negate(uint32_t *__restrict__ B, int64_t ldb, int64_t m, int64_t n, uint32_t p)
{
    pdl_enter();
    const int64_t total = m * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / n, j = idx - i * n;
        const uint32_t v = B[i * ldb + j];
        B[i * ldb + j] = v ? p - v : 0u;
    }
}

cudaError_t launch_negate(uint32_t *B, int64_t ldb, int64_t m, int64_t n, uint32_t p, cudaStream_t st)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    int64_t nb = (m * n + 255) / 256;
    if (nb > 152 * 32) nb = 152 * 32;
    launch_pdl(k_negate, (unsigned)nb, 256, 0, st, B, ldb, m, n, p);
    return cudaGetLastError();
}

// Row transpositions (rows a_t and b_t swapped for t in order; if reverse, in
// reverse order): one thread per column, so each column sees the sequence in
// order. With `prefix`, swap t only touches columns 0..a_t (Algorithm 8's
// loop, where row j and row i_j exchange their first j + 1 entries).
// Pair t is (t + base_a, list[t] + base_b) for t in [0, count).
__global__ void k_row_swaps(uint32_t *__restrict__ A, int64_t lda, int64_t ncols,
                            const int64_t *__restrict__ list, int64_t count, int64_t base_a,
                            int64_t base_b, int reverse, int prefix)
{
    pdl_enter();
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    for (int64_t s = 0; s < count; ++s) {
        const int64_t t = reverse ? count - 1 - s : s;
        const int64_t ra = t + base_a, rb = list[t] + base_b;
        if (ra == rb) continue;
        if (prefix && c > t) continue;
        const uint32_t x = A[ra * lda + c];
        A[ra * lda + c] = A[rb * lda + c];
        A[rb * lda + c] = x;
    }
}

cudaError_t launch_row_swaps(uint32_t *A, int64_t lda, int64_t ncols, const int64_t *list, int64_t count,
                             int64_t base_a, int64_t base_b, int reverse, int prefix, cudaStream_t st)
{
    if (ncols <= 0 || count <= 0) return cudaSuccess;
    launch_pdl(k_row_swaps, (unsigned)((ncols + 255) / 256), 256, 0, st, A, lda, ncols, list, count, base_a, base_b,
                                                                   reverse, prefix);
    return cudaGetLastError();
}

// dst[t][0:ncols) = src[idx[t]][0:ncols) for t < nrows
__global__ void k_gather_rows(uint32_t *__restrict__ dst, int64_t ldd, const uint32_t *__restrict__ src,
                              int64_t lds, const int64_t *__restrict__ idx, int64_t nrows, int64_t ncols)
{
    const int64_t t = blockIdx.y;
    if (t >= nrows) return;
    const uint32_t *s = src + idx[t] * lds;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncols; c += (int64_t)gridDim.x * blockDim.x)
        dst[t * ldd + c] = s[c];
}

cudaError_t launch_gather_rows(uint32_t *dst, int64_t ldd, const uint32_t *src, int64_t lds, const int64_t *idx,
                               int64_t nrows, int64_t ncols, cudaStream_t st)
{
    if (nrows <= 0 || ncols <= 0) return cudaSuccess;
    dim3 g((unsigned)((ncols + 255) / 256 < 64 ? (ncols + 255) / 256 : 64), (unsigned)nrows);
    if (nrows > 65535) return cudaErrorInvalidValue;
    k_gather_rows<<<g, 256, 0, st>>>(dst, ldd, src, lds, idx, nrows, ncols);
    return cudaGetLastError();
}

// B[i][j] = (diag && i == j) ? 1 : 0 on an m x n block
__global__ void k_fill(uint32_t *__restrict__ B, int64_t ldb, int64_t m, int64_t n, int diag)
{
    pdl_enter();
    const int64_t total = m * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / n, j = idx - i * n;
        B[i * ldb + j] = (diag && i == j) ? 1u : 0u;
    }
}

cudaError_t launch_fill(uint32_t *B, int64_t ldb, int64_t m, int64_t n, int diag, cudaStream_t st)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    int64_t nb = (m * n + 255) / 256;
    if (nb > 152 * 32) nb = 152 * 32;
    launch_pdl(k_fill, (unsigned)nb, 256, 0, st, B, ldb, m, n, diag);
    return cudaGetLastError();
}

// flag <- 1 if any entry of the m x n block is nonzero
__global__ void k_any_nonzero(const uint32_t *__restrict__ B, int64_t ldb, int64_t m, int64_t n, int *flag)
{
    const int64_t total = m * n;
    int any = 0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / n, j = idx - i * n;
        any |= (B[i * ldb + j] != 0u);
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicExch(flag, 1);
}

cudaError_t launch_any_nonzero(const uint32_t *B, int64_t ldb, int64_t m, int64_t n, int *flag, cudaStream_t st)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    int64_t nb = (m * n + 255) / 256;
    if (nb > 152 * 8) nb = 152 * 8;
    k_any_nonzero<<<(unsigned)nb, 256, 0, st>>>(B, ldb, m, n, flag);
    return cudaGetLastError();
}

// D (n x m) <- S^T for an m x n block S: 32 x 32 tiles through shared memory, so
// that both the reads and the writes run along rows.
__global__ void __launch_bounds__(256)
k_transpose(uint32_t *__restrict__ D, int64_t ldd, const uint32_t *__restrict__ S, int64_t lds, int64_t m,
            int64_t n)
{
    pdl_enter();
    __shared__ uint32_t t[32][33];
    const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;       // 8 rows of 32
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t i = i0 + ty + 8 * k, j = j0 + tx;
        if (i < m && j < n) t[ty + 8 * k][tx] = S[i * lds + j];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t j = j0 + ty + 8 * k, i = i0 + tx;           // D row j, column i
        if (j < n && i < m) D[j * ldd + i] = t[tx][ty + 8 * k];
    }
}

cudaError_t launch_transpose(uint32_t *D, int64_t ldd, const uint32_t *S, int64_t lds, int64_t m, int64_t n,
                             cudaStream_t st)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    if ((n + 31) / 32 > 0x7fffffff || (m + 31) / 32 > 65535) return cudaErrorInvalidValue;
    dim3 g((unsigned)((n + 31) / 32), (unsigned)((m + 31) / 32));
    launch_pdl(k_transpose, g, 256, 0, st, D, ldd, S, lds, m, n);
    return cudaGetLastError();
}

// Copy an m x n block (non-overlapping).
__global__ void k_copy(uint32_t *__restrict__ D, int64_t ldd, const uint32_t *__restrict__ S, int64_t lds,
                       int64_t m, int64_t n)
{
    pdl_enter();
    const int64_t total = m * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / n, j = idx - i * n;
        D[i * ldd + j] = S[i * lds + j];
    }
}

cudaError_t launch_copy(uint32_t *D, int64_t ldd, const uint32_t *S, int64_t lds, int64_t m, int64_t n,
                        cudaStream_t st)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    int64_t nb = (m * n + 255) / 256;
    if (nb > 152 * 32) nb = 152 * 32;
    launch_pdl(k_copy, (unsigned)nb, 256, 0, st, D, ldd, S, lds, m, n);
    return cudaGetLastError();
}

// One-byte residue storage (p < 2^8) at the ABI: the factorization works on a
// uint32 copy. k_widen copies an m x n block of bytes into 32-bit words, k_narrow
// copies words (residues below 256) back to bytes. A thread moves 16 entries of a
// row: one 16-byte load and four 16-byte stores (or the reverse) when the row
// offsets are aligned, single entries otherwise. Both are HBM-bound copies.
template <bool NARROW>
__global__ void __launch_bounds__(256)
k_widen_narrow(uint8_t *__restrict__ B8, int64_t ld8, uint32_t *__restrict__ W, int64_t ldw, int64_t m, int64_t n)
{
    pdl_enter();
    const int64_t per_row = (n + 15) / 16, total = m * per_row;
    const bool vec = ((ld8 | ldw) & 15) == 0 && (((uintptr_t)B8 | (uintptr_t)W) & 15) == 0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / per_row, j0 = (idx - i * per_row) * 16;
        uint8_t *b = B8 + i * ld8 + j0;
        uint32_t *w = W + i * ldw + j0;
        if (vec && j0 + 16 <= n) {
            if (NARROW) {
                uint32_t v[16];
#pragma unroll
                for (int q = 0; q < 4; ++q) *(uint4 *)&v[4 * q] = ((const uint4 *)w)[q];
                uint4 o;
                o.x = v[0] | v[1] << 8 | v[2] << 16 | v[3] << 24;
                o.y = v[4] | v[5] << 8 | v[6] << 16 | v[7] << 24;
                o.z = v[8] | v[9] << 8 | v[10] << 16 | v[11] << 24;
                o.w = v[12] | v[13] << 8 | v[14] << 16 | v[15] << 24;
                *(uint4 *)b = o;
            } else {
                const uint4 x = *(const uint4 *)b;
                const uint32_t wd[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    ((uint4 *)w)[q] = make_uint4(wd[q] & 255u, (wd[q] >> 8) & 255u, (wd[q] >> 16) & 255u, wd[q] >> 24);
            }
        } else {
            const int cnt = (int)(n - j0 < 16 ? n - j0 : 16);
            for (int c = 0; c < cnt; ++c) {
                if (NARROW) b[c] = (uint8_t)w[c];
                else w[c] = b[c];
            }
        }
    }
}

cudaError_t launch_widen_u8(uint32_t *W, int64_t ldw, const uint8_t *B8, int64_t ld8, int64_t m, int64_t n,
                            cudaStream_t st)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    int64_t nb = (m * ((n + 15) / 16) + 255) / 256;
    if (nb > 152 * 16) nb = 152 * 16;
    return launch_pdl(k_widen_narrow<false>, (unsigned)nb, 256, 0, st, const_cast<uint8_t *>(B8), ld8, W, ldw, m, n);
}

cudaError_t launch_narrow_u8(uint8_t *B8, int64_t ld8, const uint32_t *W, int64_t ldw, int64_t m, int64_t n,
                             cudaStream_t st)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    int64_t nb = (m * ((n + 15) / 16) + 255) / 256;
    if (nb > 152 * 16) nb = 152 * 16;
    return launch_pdl(k_widen_narrow<true>, (unsigned)nb, 256, 0, st, B8, ld8, const_cast<uint32_t *>(W), ldw, m, n);
}

// ---------------------------------------------------------------------------
// TRTRI leaf (Algorithm 3 at its base): in-place inverse of an n x n (n <= 64)
// triangular block, one thread per column j solving T x = e_j.
// ---------------------------------------------------------------------------
template <bool UPPER, bool UNIT, bool MONT>
__global__ void __launch_bounds__(512)
k_trtri_leaf(uint32_t *__restrict__ T, int64_t ldt, int n, ModP M)
{
    pdl_enter();
    // T^{-1} as the solution of T X = I: sixteen warps, four columns each, lanes along
    // the rows; row i is finalised (divided by its diagonal), broadcast from its lane,
    // and the rows that depend on it subtract t_ki x_i
    __shared__ uint32_t sT[TRI_MAX][TRI_MAX + 1];
    __shared__ uint32_t sD[TRI_MAX];
    __shared__ uint32_t sX[TRI_MAX][TRI_MAX + 1];
    load_tri<UPPER, UNIT, true, MONT>(T, ldt, n, M, sT, sD);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t one = 1u % M.p;
    uint32_t x[4][2];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = warp + 16 * q;
        x[q][0] = (lane == c) ? one : 0u;
        x[q][1] = (lane + 32 == c) ? one : 0u;
    }
    for (int s = 0; s < n; ++s) {
        const int i = UPPER ? n - 1 - s : s;
        const int hi = i >> 5, li = i & 31;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (!UNIT && lane == li) x[q][hi] = mmul<MONT>(x[q][hi], sD[i], M);
        }
        const uint32_t t0 = sT[lane][i], t1 = sT[lane + 32][i];
        const bool d0 = UPPER ? lane < i : lane > i, d1 = UPPER ? lane + 32 < i : lane + 32 > i;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t xi = __shfl_sync(0xffffffffu, hi ? x[q][1] : x[q][0], li);
            if (xi) {
                if (d0) x[q][0] = subm(x[q][0], mmul<MONT>(xi, t0, M), M);
                if (d1) x[q][1] = subm(x[q][1], mmul<MONT>(xi, t1, M), M);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = warp + 16 * q;
        sX[lane][c] = x[q][0];
        sX[lane + 32][c] = x[q][1];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, c = idx - i * n;
        const bool strict = UPPER ? (c > i) : (c < i);
        if (strict || (!UNIT && c == i)) T[i * ldt + c] = sX[i][c];
    }
}

cudaError_t launch_trtri_leaf(int upper, int unit, uint32_t *T, int64_t ldt, int n, ModP M, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (n > TRI_MAX) return cudaErrorInvalidValue;
    const bool mont = (M.p & 1u) != 0;
#define TRTRI_CASE(U, D)                                                                     \
    if (mont) launch_pdl(k_trtri_leaf<U, D, true>, 1, 512, 0, st, T, ldt, n, M);                     \
    else launch_pdl(k_trtri_leaf<U, D, false>, 1, 512, 0, st, T, ldt, n, M);
    if (upper && unit) { TRTRI_CASE(true, true) }
    else if (upper) { TRTRI_CASE(true, false) }
    else if (unit) { TRTRI_CASE(false, true) }
    else { TRTRI_CASE(false, false) }
#undef TRTRI_CASE
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// TRULM leaf (Algorithm 4 at its base, the variant with unit upper U stored
// strictly above the diagonal and non-unit lower L on and below it):
// A <- U L for an n x n (n <= 64) block.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_trulm_leaf(uint32_t *__restrict__ A, int64_t lda, int n, ModP M)
{
    pdl_enter();
    __shared__ uint32_t sA[TRI_MAX][TRI_MAX + 1];
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, c = idx - i * n;
        sA[i][c] = A[i * lda + c];
    }
    __syncthreads();
    uint32_t out[(TRI_MAX * TRI_MAX + 255) / 256];
    int cnt = 0;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx - i * n;
        // (U L)[i][j] = L[i][j] [i >= j] + sum_{k > i, k >= j} U[i][k] L[k][j]
        Acc acc = {0ull, 0u};
        if (i >= j) acc_add(acc, (uint64_t)sA[i][j]);
        for (int k = (i + 1 > j ? i + 1 : j); k < n; ++k) acc_add(acc, (uint64_t)sA[i][k] * sA[k][j]);
        out[cnt++] = acc_red(acc, M);
    }
    __syncthreads();
    cnt = 0;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx - i * n;
        A[i * lda + j] = out[cnt++];
    }
}

cudaError_t launch_trulm_leaf(uint32_t *A, int64_t lda, int n, ModP M, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (n > TRI_MAX) return cudaErrorInvalidValue;
    launch_pdl(k_trulm_leaf, 1, 256, 0, st, A, lda, n, M);
    return cudaGetLastError();
}

// TRLUM leaf (Algorithm 5 at its base): A = [L\U], L lower and U upper triangular
// sharing the block, one of them with an implicit unit diagonal (L if UNIT_L, else U,
// the [C\U] convention of CUP); A <- L U for an n x n (n <= 64) block.
template <bool UNIT_L>
__global__ void __launch_bounds__(256)
k_trlum_leaf(uint32_t *__restrict__ A, int64_t lda, int n, ModP M)
{
    pdl_enter();
    __shared__ uint32_t sA[TRI_MAX][TRI_MAX + 1];
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, c = idx - i * n;
        sA[i][c] = A[i * lda + c];
    }
    __syncthreads();
    uint32_t out[(TRI_MAX * TRI_MAX + 255) / 256];
    int cnt = 0;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx - i * n;
        // (L U)[i][j] = sum_{k <= min(i, j)} L[i][k] U[k][j]; the k = min(i, j) term
        // carries the unit diagonal of one factor.
        Acc acc = {0ull, 0u};
        const int kd = i < j ? i : j;
        for (int k = 0; k < kd; ++k) acc_add(acc, (uint64_t)sA[i][k] * sA[k][j]);
        const bool plain = UNIT_L ? (i <= j) : (i >= j);     // the unit factor meets the term
        acc_add(acc, plain ? (uint64_t)sA[i][j] : (uint64_t)sA[i][j] * sA[kd][kd]);
        out[cnt++] = acc_red(acc, M);
    }
    __syncthreads();
    cnt = 0;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx - i * n;
        A[i * lda + j] = out[cnt++];
    }
}

cudaError_t launch_trlum_leaf(uint32_t *A, int64_t lda, int n, int unit_l, ModP M, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (n > TRI_MAX) return cudaErrorInvalidValue;
    if (unit_l) launch_pdl(k_trlum_leaf<true>, 1, 256, 0, st, A, lda, n, M);
    else launch_pdl(k_trlum_leaf<false>, 1, 256, 0, st, A, lda, n, M);
    return cudaGetLastError();
}

// Column transpositions (t, list[t]) for t in [0, count) applied to rows
// 0..nrows-1, in order or (reverse) in reverse order; one thread per row, the
// list staged through shared memory a chunk at a time.
__global__ void __launch_bounds__(256)
k_col_swaps(uint32_t *__restrict__ A, int64_t lda, int64_t nrows, const int64_t *__restrict__ list,
            int64_t count, int reverse)
{
    pdl_enter();
    __shared__ int64_t sl[256];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t *row = A + i * lda;
    for (int64_t b = 0; b < count; b += 256) {
        const int64_t e = (count - b) < 256 ? (count - b) : 256;
        __syncthreads();
        if (threadIdx.x < e) {
            const int64_t s = b + threadIdx.x;
            sl[threadIdx.x] = list[reverse ? count - 1 - s : s];
        }
        __syncthreads();
        if (i < nrows)
            for (int64_t k = 0; k < e; ++k) {
                const int64_t t = reverse ? count - 1 - (b + k) : b + k, c = sl[k];
                if (c == t) continue;
                const uint32_t x = row[t];
                row[t] = row[c];
                row[c] = x;
            }
    }
}

cudaError_t launch_col_swaps(uint32_t *A, int64_t lda, int64_t nrows, const int64_t *list, int64_t count,
                             int reverse, cudaStream_t st)
{
    if (nrows <= 0 || count <= 0) return cudaSuccess;
    launch_pdl(k_col_swaps, (unsigned)((nrows + 255) / 256), 256, 0, st, A, lda, nrows, list, count, reverse);
    return cudaGetLastError();
}

// Zero the strict upper triangle of an n x n block.
__global__ void k_zero_upper(uint32_t *__restrict__ B, int64_t ldb, int64_t n)
{
    pdl_enter();
    const int64_t total = n * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / n, j = idx - i * n;
        if (j > i) B[i * ldb + j] = 0u;
    }
}

cudaError_t launch_zero_upper(uint32_t *B, int64_t ldb, int64_t n, cudaStream_t st)
{
    if (n <= 1) return cudaSuccess;
    int64_t nb = (n * n + 255) / 256;
    if (nb > 152 * 32) nb = 152 * 32;
    launch_pdl(k_zero_upper, (unsigned)nb, 256, 0, st, B, ldb, n);
    return cudaGetLastError();
}
