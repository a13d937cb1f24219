// CUDA-core kernels of the CUP hot path over GF(p):
//   * the row-block base case (a slab of at most CUP_BMAX rows), split into a
//     one-CTA pivot kernel and a grid-wide finish kernel;
//   * column transpositions (the A2 <- A2 P1^T and V1 <- V1 P2^T steps);
//   * the CUDA-core INT64 Schur update C <- C - A B mod p (plain path, and the
//     thin-K fallback of the tensor-core path).
//
// The base case generalises the m = 1 case of Algorithm 6 (Sec. 3.3) to a
// block of rows: rows are taken in order, the pivot of a row is the first
// nonzero entry of its residual at a position >= the current rank, and that
// column is transposed with the leading position. The elimination inside the
// slab is fraction-free (row i' <- f row i' - m row i with f the pivot and m
// the entry below it), so no field inversion sits on the per-row critical
// path; the scale factors are products of the pivots and are divided out once
// at the end with inversions computed in parallel.
#include <climits>
#include <cuda_bf16.h>
#include "cup_internal.cuh"

// ---------------------------------------------------------------------------
// Leaf slab, pivot phase (one CTA).
//
// Window: positions [0, wne) of the slab rows [a, a + brows), columns
// [col0, col0 + w). The window is eliminated in panels of PIV_PB rows: the
// panel's rows are taken one by one (each step updating only the panel), then
// every row below takes the panel's pivots in one fused update whose
// coefficients come from unrolling the fraction-free recurrence, so no field
// inversion is needed there either. The row-operation matrix E (eliminated
// slab = E * slab) is carried alongside; its pivot block gives L^{-1}, so
// that U's rows over the whole width are L^{-1} * (pivot rows of the slab),
// which the finish kernel evaluates as a small matrix product.
//
// A row whose window residual is zero while pivots already exist in this slab
// cannot be classified without its residual beyond the window: the kernel then
// stops and reports i_stop; the caller applies the update of the resolved rows
// to the remaining rows (TRSM + MM, as at an internal node of Algorithm 6) and
// calls the kernel again on them.
// ---------------------------------------------------------------------------
#ifndef PIV_THREADS

#define PIV_THREADS 512
#endif
#define PIV_LDW (CUP_WNMAX + 1)
#define PIV_LDE (CUP_BMAX + 1)
#ifndef PIV_PB
#define PIV_PB 8                    // panel rows of the blocked window elimination
#endif
#define PIV_PW 16                   // warps that eliminate a panel (all of them: 8 column chunks x 2 row parities)
#ifndef PIV_QUIET
#define PIV_QUIET 1                 // pipelined block update: leave warp 0's scheduler to warp 0
#endif

// One fraction-free update f x - m y, scaled by R^{-1} in the Montgomery
// variant (odd p): the common factor only changes the tracked row scales.
template <bool MONT>
__device__ __forceinline__ uint32_t ff(uint32_t f, uint32_t x, uint32_t m, uint32_t y, const ModP &M)
{
    return MONT ? ffupd_mont(f, x, m, y, M) : ffupd(f, x, m, y, M);
}

template <bool MONT>
__device__ __forceinline__ uint32_t scale_mul(uint32_t a, uint32_t b, const ModP &M)
{
    return MONT ? redc((uint64_t)a * b, M) : mulm(a, b, M);
}

template <bool MONT>
__device__ __forceinline__ uint32_t inv_any(uint32_t a, const ModP &M)
{
    return MONT ? invm_mont(a, M) : invm(a, M);
}

// First position q in [r, wne) of window row `row` holding a nonzero, or -1.
// Every warp runs it on the same data, so its result needs no broadcast.
__device__ __forceinline__ int window_search(const uint32_t *row, int r, int wne, int lane)
{
    for (int q0 = r; q0 < wne; q0 += 32) {
        const int q = q0 + lane;
        const uint32_t v = (q < wne) ? row[q] : 0u;
        const unsigned bal = __ballot_sync(0xffffffffu, v != 0u);
        if (bal) return q0 + __ffs(bal) - 1;
    }
    return -1;
}

// Barrier over the warps that eliminate a panel (named barrier 1).
__device__ __forceinline__ void panel_bar()
{
    asm volatile("bar.sync 1, %0;" ::"n"(32 * PIV_PW) : "memory");
}

// Montgomery reduction of T < p R to [0, p) (odd p).
__device__ __forceinline__ uint32_t redc_once(uint64_t T, const ModP &M)
{
    return redc(T, M);
}

template <bool MONT, bool WIDE>
__global__ void __launch_bounds__(PIV_THREADS)
k_slab_pivots(const uint32_t *__restrict__ A, int64_t lda, int64_t a, int brows, const Dyn col0d,
              int64_t n, int wn, int speculate, ModP M, SlabScratch *__restrict__ S,
              int64_t *__restrict__ g_ipiv, int64_t *__restrict__ g_prof, int64_t *__restrict__ rank_next)
{
    // col0 was written by the leaf before (several launches back), so it and the work on
    // shared memory alone (E's identity, the window's column map) precede the dependency
    // wait; the window itself comes from the Schur update just before
    const int64_t col0 = col0d.eval();
    const int64_t w = n - col0;
    if (w <= 0) {
        pdl_enter();
        // every column is already a pivot: the slab's rows are dependent
        if (threadIdx.x == 0) {
            S->r_s = 0; S->i_stop = brows; S->wne = 0; S->ext_pos = -1; S->ext_slot = -1;
            S->n_slot = 0; S->n_spec = 0; S->spec_fail = 0;
            if (rank_next) *rank_next = col0;
        }
        return;
    }
    extern __shared__ uint32_t W[];            // brows x PIV_LDW window, then the row-operation matrix
    uint32_t *const E = W + CUP_BMAX * PIV_LDW; // E (CUP_BMAX x PIV_LDE): eliminated slab = E * slab
    __shared__ int s_wcol[CUP_WNMAX];
    __shared__ int s_prof[CUP_BMAX], s_pos[CUP_BMAX], s_spec[CUP_BMAX];
    __shared__ uint32_t s_f[CUP_BMAX], s_finv[CUP_BMAX], s_muinv[CUP_BMAX], s_Sinv[CUP_BMAX],
        s_Sfwd[CUP_BMAX], s_Spinv[CUP_BMAX + 1];
    __shared__ __align__(16) uint32_t s_coef[CUP_BMAX][PIV_PB];   // -a_kt of the block update, per row below a panel
    __shared__ int s_c, s_ext, s_fast;
    __shared__ unsigned long long s_key;
    __shared__ int s_state[2][6];              // after each panel: rank, stop, spec count, done, rows to update, swaps
    __shared__ uint32_t s_T[PIV_PB][PIV_PB];   // fast panel path: the panel's row operations (fraction-free)
    __shared__ uint32_t s_B[PIV_PB][PIV_PB];   // ... with dependent rows: the eliminated block, kept until verified
    __shared__ int s_dep, s_bpf;                // ... with dependent rows: their mask, and the panel's pivot count
    __shared__ uint32_t s_sprod;
    __shared__ int s_slot[CUP_WNMAX + 1], s_sorig[CUP_WNMAX + 2];

    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int wne = (int)(w < (int64_t)wn ? w : (int64_t)wn);
    const uint32_t one = 1u % M.p;
    // R^{-1} for the Montgomery variant (the factor each fraction-free update carries), else 1
    const uint32_t rinv = MONT ? redc(1ull, M) : one;

    for (int idx = tid; idx < brows * CUP_BMAX; idx += nt) {
        const int i = idx >> 6, j = idx & (CUP_BMAX - 1);
        E[i * PIV_LDE + j] = (i == j) ? one : 0u;
    }
    for (int q = tid; q < wne; q += nt) s_wcol[q] = q;
    if (tid == 0) s_ext = -1;
    pdl_enter();
    // window: every element copied asynchronously, one memory latency for the tile
    for (int i = warp; i < brows; i += nw) {
        const uint32_t *src = A + (a + i) * lda + col0;
        for (int q = lane; q < wne; q += 32) cp_async4(W + i * PIV_LDW + q, src + q);
    }
    cp_async_wait_all();
    __syncthreads();

    // Leading rows while the slab has no pivot (whole CTA): a row whose window
    // is zero is either a zero row or has its first nonzero beyond the window,
    // whose column then moves to position 0 (no elimination has happened yet,
    // so the rows are still the unreduced input). Unless row 0 has a nonzero in its
    // window, all rows are examined at once: the first row with a nonzero in its window
    // (from shared memory), then, among the rows before it, the first one with a nonzero
    // beyond the window and that row's first such column, in one pass over those rows in
    // global memory (32 loads of each lane in flight together; a slab of dependent rows
    // is all such rows).
    int p0 = 0;
    if (window_search(W, 0, wne, lane) < 0) {            // row 0's window is zero (same in every warp)
        if (tid == 0) { s_c = brows; s_key = ~0ull; }
        __syncthreads();
        for (int i = warp; i < brows; i += nw)
            if (window_search(W + i * PIV_LDW, 0, wne, lane) >= 0 && lane == 0) atomicMin(&s_c, i);
        __syncthreads();
        p0 = s_c;
        if ((int64_t)wne < w && p0 > 0) {
            // warp w scans rows w, w + nw, ... below p0 beyond the window, 1024 columns a batch;
            // each lane keeps its first nonzero column, the CTA the smallest (row, column)
            const int span = (int)(w - wne);
            unsigned long long best = ~0ull;
            for (int i = warp; i < p0; i += nw) {
                const uint32_t *row = A + (a + i) * lda + col0 + wne;
                for (int qb = 0; qb < span; qb += 32 * 32) {
                    uint32_t v[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int q = qb + 32 * j + lane;
                        v[j] = q < span ? row[q] : 0u;
                    }
                    int first = INT_MAX;
#pragma unroll
                    for (int j = 31; j >= 0; --j) first = v[j] ? qb + 32 * j + lane : first;
                    if (first != INT_MAX) {
                        const unsigned long long key = ((unsigned long long)i << 32) | (unsigned long long)(wne + first);
                        best = key < best ? key : best;
                    }
                }
            }
            if (best != ~0ull) atomicMin(&s_key, best);
            __syncthreads();
            const unsigned long long key = s_key;
            if (key != ~0ull) {
                const int c = (int)(key & 0xffffffffu);
                p0 = (int)(key >> 32);
                for (int ii = tid; ii < brows; ii += nt) W[ii * PIV_LDW + 0] = A[(a + ii) * lda + col0 + c];
                if (tid == 0) { s_ext = c; s_wcol[0] = c; }
                __syncthreads();
            }
        }
    }
    const int ext0 = s_ext;

    int r = 0, stop = brows, nspec = 0, pc = 0;
    bool done = false, try_fast = true;
    uint32_t Sprod = one;                      // product of the row scales applied so far (every thread)
    bool pre_done = false;                     // this panel's block was eliminated during the last update
    // Warp 0's part of the fast panel path (see below) for the panel of rows [bp0, bp0 + 8)
    // at rank position br0: the fraction-free steps on the 8 x 8 diagonal block in registers,
    // T, the pivots and the running scale; s_fast = 1 when no pivot was zero (otherwise
    // nothing but s_fast is written).
    auto block_elim = [&](const int bp0, const int br0) {
        const int k = lane >> 2, jg = lane & 3, ja = 2 * jg, jb = ja + 1;
        uint32_t b0 = W[(bp0 + k) * PIV_LDW + br0 + ja];
        uint32_t b1 = W[(bp0 + k) * PIV_LDW + br0 + jb];
        uint32_t t0 = (k == ja) ? one : 0u, t1 = (k == jb) ? one : 0u;
        uint32_t fv = 0u;                     // lane t keeps the pivot of step t
        bool zero = false;
        // all eight steps unrolled; a zero pivot (the same value in every lane) is
        // noted and the block's results are then discarded. Every lane computes its four
        // updates and keeps them by selection: no divergent branch between the shuffles.
#pragma unroll
        for (int t = 0; t < PIV_PB; ++t) {
            const int sf = 4 * t + (t >> 1), sm = 4 * k + (t >> 1), sy = 4 * t + jg;
            const uint32_t f = __shfl_sync(0xffffffffu, (t & 1) ? b1 : b0, sf);
            const uint32_t mk = __shfl_sync(0xffffffffu, (t & 1) ? b1 : b0, sm);
            zero |= f == 0u;
            const uint32_t y0 = __shfl_sync(0xffffffffu, b0, sy), y1 = __shfl_sync(0xffffffffu, b1, sy);
            const uint32_t z0 = __shfl_sync(0xffffffffu, t0, sy), z1 = __shfl_sync(0xffffffffu, t1, sy);
            fv = (lane == t) ? f : fv;
            const uint32_t n0 = ff<MONT>(f, b0, mk, y0, M), n1 = ff<MONT>(f, b1, mk, y1, M);
            const uint32_t u0 = ff<MONT>(f, t0, mk, z0, M), u1 = ff<MONT>(f, t1, mk, z1, M);
            const bool rk = k > t;
            b0 = (rk && ja > t) ? n0 : b0;
            b1 = (rk && jb > t) ? n1 : b1;
            t0 = rk ? u0 : t0;
            t1 = rk ? u1 : t1;
        }
        const bool ok = !zero;
        if (ok) {
            W[(bp0 + k) * PIV_LDW + br0 + ja] = b0;
            W[(bp0 + k) * PIV_LDW + br0 + jb] = b1;
            // T R for odd p with narrow sums: the pass applying T then needs one
            // Montgomery reduction per entry
            s_T[k][ja] = (MONT && !WIDE) ? redc((uint64_t)t0 * M.r2, M) : t0;
            s_T[k][jb] = (MONT && !WIDE) ? redc((uint64_t)t1 * M.r2, M) : t1;
            if (lane < PIV_PB) {
                s_f[br0 + lane] = fv;
                s_pos[br0 + lane] = (br0 + lane == 0 && ext0 >= 0) ? ext0 : br0 + lane;
                s_prof[br0 + lane] = bp0 + lane;
            }
            // running scale before each step, S_t = Sprod * mu_0 ... mu_{t-1}, by an inclusive
            // scan of the pivots over lanes 0 .. 7 (the identity is one, R in Montgomery form;
            // every product of k factors carries R^{1-k} either way)
            const uint32_t id = MONT ? redc((uint64_t)M.r2, M) : one;
            uint32_t v = (lane < PIV_PB) ? fv : id;
#pragma unroll
            for (int o = 1; o < PIV_PB; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
                const uint32_t pv = scale_mul<MONT>(v, u, M);
                v = (lane >= o) ? pv : v;
            }
            uint32_t ex = __shfl_up_sync(0xffffffffu, v, 1);
            ex = (lane == 0) ? id : ex;
            const uint32_t Sx = scale_mul<MONT>(Sprod, ex, M);     // S_lane (lane < 8)
            const uint32_t Sall = scale_mul<MONT>(Sprod, __shfl_sync(0xffffffffu, v, PIV_PB - 1), M);
            if (lane < PIV_PB) s_Sfwd[br0 + lane] = Sx;
            if (lane == 0) s_sprod = Sall;
        }
        if (lane == 0) s_fast = ok ? 1 : 3;
    };
    // The same steps when a pivot was zero: row i's candidate is its value at the next rank
    // position rr (the count of pivots so far). If that value is zero and the row's whole
    // block residual (positions >= rr) is zero too, the row is taken as dependent: it
    // takes no rank position and no step. The rest of its window residual is checked
    // when the panel's row operations are applied (speculated rows beyond the window go to
    // the finish kernel's check, as in the stepwise path). A zero candidate with a nonzero
    // elsewhere in the block needs a transposition: s_fast = 0 sends the panel to the
    // stepwise path. The block is left in s_B until the check has passed (s_fast = 2).
    auto block_elim_dep = [&](const int bp0, const int br0) {
        const int k = lane >> 2, jg = lane & 3, ja = 2 * jg, jb = ja + 1;
        uint32_t b0 = W[(bp0 + k) * PIV_LDW + br0 + ja];
        uint32_t b1 = W[(bp0 + k) * PIV_LDW + br0 + jb];
        uint32_t t0 = (k == ja) ? one : 0u, t1 = (k == jb) ? one : 0u;
        uint32_t fv = 0u, prow = 0u;           // lane t keeps the pivot of step t and its row
        unsigned dmask = 0u;
        int rr = 0;
        bool bail = false;
#pragma unroll
        for (int i = 0; i < PIV_PB; ++i) {
            const uint32_t src = (rr & 1) ? b1 : b0;
            const uint32_t f = __shfl_sync(0xffffffffu, src, 4 * i + (rr >> 1));
            if (f != 0u) {                      // the same in every lane
                const uint32_t mk = __shfl_sync(0xffffffffu, src, 4 * k + (rr >> 1));
                const uint32_t y0 = __shfl_sync(0xffffffffu, b0, 4 * i + jg), y1 = __shfl_sync(0xffffffffu, b1, 4 * i + jg);
                const uint32_t z0 = __shfl_sync(0xffffffffu, t0, 4 * i + jg), z1 = __shfl_sync(0xffffffffu, t1, 4 * i + jg);
                fv = (lane == rr) ? f : fv;
                prow = (lane == rr) ? (uint32_t)i : prow;
                const uint32_t n0 = ff<MONT>(f, b0, mk, y0, M), n1 = ff<MONT>(f, b1, mk, y1, M);
                const uint32_t u0 = ff<MONT>(f, t0, mk, z0, M), u1 = ff<MONT>(f, t1, mk, z1, M);
                const bool rk = k > i;
                b0 = (rk && ja > rr) ? n0 : b0;
                b1 = (rk && jb > rr) ? n1 : b1;
                t0 = rk ? u0 : t0;
                t1 = rk ? u1 : t1;
                ++rr;
            } else {
                const bool nz = (k == i) && ((ja >= rr && b0 != 0u) || (jb >= rr && b1 != 0u));
                if (__any_sync(0xffffffffu, nz)) { bail = true; break; }
                dmask |= 1u << i;
            }
        }
        // speculation is needed for dependent rows unless the window is the whole residual
        if (!bail && (int64_t)wne < w && !speculate) bail = true;
        if (!bail) {
            s_B[k][ja] = b0;
            s_B[k][jb] = b1;
            s_T[k][ja] = (MONT && !WIDE) ? redc((uint64_t)t0 * M.r2, M) : t0;
            s_T[k][jb] = (MONT && !WIDE) ? redc((uint64_t)t1 * M.r2, M) : t1;
            if (lane < rr) {
                s_f[br0 + lane] = fv;
                s_pos[br0 + lane] = (br0 + lane == 0 && ext0 >= 0) ? ext0 : br0 + lane;
                s_prof[br0 + lane] = bp0 + (int)prow;
            }
            const uint32_t id = MONT ? redc((uint64_t)M.r2, M) : one;
            uint32_t v = (lane < rr) ? fv : id;
#pragma unroll
            for (int o = 1; o < PIV_PB; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
                const uint32_t pv = scale_mul<MONT>(v, u, M);
                v = (lane >= o) ? pv : v;
            }
            uint32_t ex = __shfl_up_sync(0xffffffffu, v, 1);
            ex = (lane == 0) ? id : ex;
            const uint32_t Sx = scale_mul<MONT>(Sprod, ex, M);
            const uint32_t Sall = scale_mul<MONT>(Sprod, __shfl_sync(0xffffffffu, v, PIV_PB - 1), M);
            if (lane < rr) s_Sfwd[br0 + lane] = Sx;
            if (lane == 0) { s_sprod = Sall; s_dep = (int)dmask; s_bpf = rr; }
        }
        if (lane == 0) s_fast = bail ? 0 : 2;
    };
    for (; p0 < brows && !done; p0 += PIV_PB, ++pc) {
        const int pend = p0 + PIV_PB < brows ? p0 + PIV_PB : brows;
        const int r0 = r, np = pend - p0;
        int lim = brows;
        bool pswap = false;
        // Fast path of a panel: when the residual of every panel row at the current rank
        // position is nonzero, the rule takes that position as the pivot of each row in
        // turn (no transposition, no dependent row), so the panel's steps only combine
        // its rows. Warp 0 then eliminates the np x np diagonal block in registers (the
        // same fraction-free steps) and records the row operations as T (panel rows after
        // = T x panel rows before); one parallel pass applies T to the panel's other
        // columns, instead of np steps separated by barriers. A zero on the diagonal sends
        // this panel, and the rest of the slab, to the stepwise elimination below.
        int code = -1;                         // 1: fast, 2: fast with dependent rows, 0: stepwise
        if (pre_done) {
            // warp 0 eliminated this panel's block while the others finished the last update
            code = s_fast;
            pre_done = false;
        } else if (try_fast && np == PIV_PB && r0 + np <= wne) {
            if (warp == 0) block_elim(p0, r0);
            __syncthreads();
            code = s_fast;
        }
        if (code == 3) {
            if (warp == 0) block_elim_dep(p0, r0);
            __syncthreads();
            code = s_fast;
        }
        bool fast = code == 1 || code == 2;
        if (code == 0) try_fast = false;
        // one entry of a panel row after the panel: row kk of T times the rows before it
        auto tval = [&](const int kk, const uint32_t (&x)[PIV_PB]) -> uint32_t {
            if (MONT && !WIDE) {
                // s_T holds T R; at most eight products, each below p^2, sum below p R
                // (narrow sums mean p < 2^28.8), so one Montgomery reduction gives sum T x
                uint64_t s0 = 0;
#pragma unroll
                for (int j = 0; j < PIV_PB; ++j)
                    if (j <= kk) s0 += (uint64_t)s_T[kk][j] * x[j];
                return redc(s0, M);
            } else {
                uint64_t s0 = 0, s1 = 0;      // at most four products below 2^62 in each
#pragma unroll
                for (int j = 0; j < PIV_PB; ++j) {
                    if (j > kk) continue;
                    if (j < 4) s0 += (uint64_t)s_T[kk][j] * x[j];
                    else s1 += (uint64_t)s_T[kk][j] * x[j];
                }
                return addm(red64(s0, M), red64(s1, M), M);
            }
        };
        if (code == 2) {
            // Dependent rows: the panel's row operations are applied to the columns right of
            // the block and to E, with every dependent row's window values checked to be zero,
            // before anything is written; a nonzero sends the panel to the stepwise path with
            // the slab untouched (the block is still in s_B).
            const unsigned dmask = (unsigned)s_dep;
            const int nwc = wne - (r0 + np), ncol = nwc + pend;    // ncol < CTA size
            const int ci = nt - 1 - tid;
            const bool col = ci < ncol;
            const bool inw = ci < nwc;
            uint32_t *base = inw ? W + r0 + np + ci : E + (ci - nwc);
            const int st = inw ? PIV_LDW : PIV_LDE;
            uint32_t x[PIV_PB], res[PIV_PB];
            bool bad = false;
#pragma unroll
            for (int j = 0; j < PIV_PB; ++j) x[j] = col ? base[(p0 + j) * st] : 0u;
#pragma unroll
            for (int kk = 0; kk < PIV_PB; ++kk) {
                res[kk] = kk == 0 ? x[0] : tval(kk, x);
                if (col && inw && ((dmask >> kk) & 1u) && res[kk] != 0u) bad = true;
            }
            if (__syncthreads_or(bad)) {
                fast = false;
                try_fast = false;
            } else {
                if (col) {
#pragma unroll
                    for (int kk = 1; kk < PIV_PB; ++kk) base[(p0 + kk) * st] = res[kk];
                }
                if (tid < PIV_PB * PIV_PB) W[(p0 + (tid >> 3)) * PIV_LDW + r0 + (tid & 7)] = s_B[tid >> 3][tid & 7];
                if ((int64_t)wne < w) {
                    // speculated dependent rows, checked over the whole width by the finish kernel
                    if (tid == 0) {
                        int q = nspec;
                        for (int i = 0; i < PIV_PB; ++i)
                            if ((dmask >> i) & 1u) s_spec[q++] = p0 + i;
                    }
                    nspec += __popc(dmask);
                }
                r = r0 + s_bpf;
                Sprod = s_sprod;
                __syncthreads();
            }
        } else if (fast) {
            // window positions right of the block, then E columns [0, pend): thread per column,
            // panel rows 1 .. np-1 as sums of T's entries times the rows' values before the panel.
            // Columns go to the last threads, whose warps the multiplier pass below leaves
            // idle unless more than 4 (nw - 2) rows lie below the panel.
            const int nwc = wne - (r0 + np), ncol = nwc + pend;
            for (int ci = nt - 1 - tid; ci < ncol; ci += nt) {
                const bool inw = ci < nwc;
                uint32_t *base = inw ? W + r0 + np + ci : E + (ci - nwc);
                const int st = inw ? PIV_LDW : PIV_LDE;
                uint32_t x[PIV_PB];
#pragma unroll
                for (int j = 0; j < PIV_PB; ++j) x[j] = j < np ? base[(p0 + j) * st] : 0u;
#pragma unroll
                for (int kk = 1; kk < PIV_PB; ++kk) {
                    if (kk < np) {
                        if (MONT && !WIDE) {
                            // s_T holds T R; at most eight products, each below p^2, sum
                            // below p R (narrow sums mean p < 2^28.8), so one Montgomery
                            // reduction gives sum T x
                            uint64_t s0 = 0;
#pragma unroll
                            for (int j = 0; j <= kk; ++j) s0 += (uint64_t)s_T[kk][j] * x[j];
                            base[(p0 + kk) * st] = redc(s0, M);
                        } else {
                            uint64_t s0 = 0, s1 = 0;      // at most four products below 2^62 in each
#pragma unroll
                            for (int j = 0; j <= kk; ++j) {
                                if (j < 4) s0 += (uint64_t)s_T[kk][j] * x[j];
                                else s1 += (uint64_t)s_T[kk][j] * x[j];
                            }
                            base[(p0 + kk) * st] = addm(red64(s0, M), red64(s1, M), M);
                        }
                    }
                }
            }
            // With rows below the panel the block update's multiplier pass runs next without a
            // barrier: it reads those rows and the pivot rows at the block's positions (written
            // by warp 0 before the last barrier) and writes those rows' block positions and
            // E diagonal, none of which this pass touches; its own barrier then publishes both
            // before the fused update reads the panel's rows.
            if (pend >= brows) __syncthreads();
            r = r0 + np;
            Sprod = s_sprod;
        }
        if (!fast) {
        if (warp < PIV_PW) {
            // Panel of rows [p0, pend), eliminated by the first PIV_PW warps (named
            // barrier 1): the rows are taken one by one as in the unblocked
            // elimination, each step updating only the panel's rows. Warp w owns the
            // 32-column chunk w % 8 of (window positions > r, then E columns [0, pend))
            // in every other row below the pivot row.
            int lim = brows;                   // rows that still need this panel's pivots
            bool swapped = false;
            for (int i = p0; i < pend; ++i) {
                if ((int64_t)r >= w) { done = true; break; }   // every column is a pivot: later rows are dependent
                const int c = window_search(W + i * PIV_LDW, r, wne, lane);
                if (c < 0) {
                    // r > 0 here: the first row of the first panel holds a window nonzero
                    if ((int64_t)wne == w) continue;   // whole residual known and zero
                    if (!speculate) { stop = i; lim = i; done = true; break; }
                    if (tid == 0) s_spec[nspec] = i;   // verified by the finish kernel
                    ++nspec;
                    continue;
                }
                if (c != r) {
                    swapped = true;
                    // transposition of positions r and c in the panel's rows (rows below
                    // take it with the block update; rows above never read these positions),
                    // once every warp has searched row i
                    panel_bar();
                    for (int ii = p0 + tid; ii < pend; ii += 32 * PIV_PW) {
                        const uint32_t x = W[ii * PIV_LDW + r];
                        W[ii * PIV_LDW + r] = W[ii * PIV_LDW + c];
                        W[ii * PIV_LDW + c] = x;
                    }
                    if (tid == 0) { const int x = s_wcol[r]; s_wcol[r] = s_wcol[c]; s_wcol[c] = x; }
                    panel_bar();
                }
                const uint32_t f = W[i * PIV_LDW + r];
                if (tid == 0) {
                    s_pos[r] = (r == 0 && ext0 >= 0) ? ext0 : c;
                    s_prof[r] = i; s_f[r] = f; s_Sfwd[r] = Sprod;
                }
                const int nwc = wne - r - 1;
                const int ci = 32 * (warp & 7) + lane;         // 32-column chunk of this warp
                const int h = warp >> 3;                       // rows i + 1 + h, i + 3 + h, ...
                if (ci < nwc + pend) {
                    // every operand of the rows is read before any result is stored
                    const bool inw = ci < nwc;
                    const uint32_t y = inw ? W[i * PIV_LDW + r + 1 + ci] : E[i * PIV_LDE + ci - nwc];
                    uint32_t *xk = inw ? W + (i + 1) * PIV_LDW + r + 1 + ci : E + (i + 1) * PIV_LDE + ci - nwc;
                    const int xs = inw ? PIV_LDW : PIV_LDE;
                    const int nk = pend - 1 - i;
                    constexpr int NJ = PIV_PB / 2;
                    uint32_t mk[NJ], xv[NJ];
#pragma unroll
                    for (int jj = 0; jj < NJ; ++jj) {
                        const int j = h + 2 * jj;
                        if (j < nk) { mk[jj] = W[(i + 1 + j) * PIV_LDW + r]; xv[jj] = xk[j * xs]; }
                    }
#pragma unroll
                    for (int jj = 0; jj < NJ; ++jj) {
                        const int j = h + 2 * jj;
                        if (j < nk) xk[j * xs] = ff<MONT>(f, xv[jj], mk[jj], y, M);
                    }
                }
                panel_bar();
                Sprod = scale_mul<MONT>(Sprod, f, M);
                ++r;
            }
            if (tid == 0) {
                int *st = s_state[pc & 1];
                st[0] = r; st[1] = stop; st[2] = nspec; st[3] = done ? 1 : 0; st[4] = lim;
                st[5] = swapped ? 1 : 0;
            }
        }
        __syncthreads();
        lim = s_state[pc & 1][4];
        r = s_state[pc & 1][0]; stop = s_state[pc & 1][1]; nspec = s_state[pc & 1][2];
        done = s_state[pc & 1][3] != 0;
        pswap = s_state[pc & 1][5] != 0;
        }
        const int bp = r - r0;
        if (bp == 0 || pend >= lim) continue;
        // Rows [pend, lim) take the panel's transpositions, then its bp pivots
        // at once. With g_t the scale of step t (the update is
        // z <- g_t z - R^{-1} m_t y_t), the bp sequential updates unroll to
        //   z = (prod_t g_t) x - sum_t (R^{-1} prod_{t' > t} g_t') m_t y_t,
        // where m_t is the row's entry at pivot position r0 + t just before step t.
        {
            // Every warp forms h_t = R^{-1} prod_{t' > t} g_t' and A0 = prod_t g_t by a
            // suffix scan. For odd p it runs on Montgomery representations, where g_t
            // is represented by f_t itself (g_t R = f_t): the exclusive suffix product
            // is then h_t R^2 and the inclusive one A0 R, the forms the update uses.
            uint32_t h, A0, A0f;
            if (MONT) {
                uint32_t suf = (lane < bp) ? s_f[r0 + lane] : redc((uint64_t)M.r2, M);   // R mod p: one
#pragma unroll
                for (int o = 1; o < PIV_PB; o <<= 1) {
                    const uint32_t u = __shfl_down_sync(0xffffffffu, suf, o);
                    const uint32_t ps = redc((uint64_t)suf * u, M);
                    suf = (lane + o < bp) ? ps : suf;
                }
                const uint32_t oneR = redc((uint64_t)M.r2, M);
                uint32_t ex = __shfl_down_sync(0xffffffffu, suf, 1);
                if (lane + 1 >= bp) ex = oneR;
                const uint32_t incl0 = __shfl_sync(0xffffffffu, suf, 0);
                A0f = redc((uint64_t)incl0, M);                  // A0
                if (!WIDE) {
                    h = ex;                                      // h_t R^2
                    A0 = incl0;                                  // A0 R
                } else {
                    h = redc((uint64_t)redc((uint64_t)ex, M), M); // h_t
                    A0 = A0f;
                }
            } else {
                uint32_t suf = (lane < bp) ? s_f[r0 + lane] : one;
#pragma unroll
                for (int o = 1; o < PIV_PB; o <<= 1) {
                    const uint32_t u = __shfl_down_sync(0xffffffffu, suf, o);
                    const uint32_t ps = mulm(suf, u, M);
                    suf = (lane + o < bp) ? ps : suf;
                }
                h = __shfl_down_sync(0xffffffffu, suf, 1);
                if (lane + 1 >= bp) h = one;
                A0 = __shfl_sync(0xffffffffu, suf, 0);
                A0f = A0;
            }
            // (b) eight lanes per row (four rows per warp): the panel's transpositions, then
            // the multipliers m_t by the recurrence restricted to the panel's pivot
            // positions (lane s holds position r0 + s; step t broadcasts lane t's value),
            // stored where the unblocked elimination leaves them, and the coefficients
            // of the fused update (zero for t >= bp); warps without such rows skip it
            if (4 * warp < lim - pend) {
                const int kr = 4 * warp + (lane >> 3), s = lane & 7;
                const int k = pend + kr;
                const bool vk = k < lim;
                uint32_t *wk = W + (vk ? k : pend) * PIV_LDW;
                if (pswap && vk && s == 0) {
                    for (int t = 0; t < bp; ++t) {
                        const int ct = s_pos[r0 + t];
                        if (ct != r0 + t && ct < wne) {
                            const uint32_t x = wk[r0 + t];
                            wk[r0 + t] = wk[ct];
                            wk[ct] = x;
                        }
                    }
                }
                __syncwarp();
                const uint32_t hs = __shfl_sync(0xffffffffu, h, s);   // h_s, held by lane s
                uint32_t v = (vk && s < bp) ? wk[r0 + s] : 0u;
                uint32_t yv[PIV_PB - 1], fv[PIV_PB - 1];
#pragma unroll
                for (int t = 0; t < PIV_PB - 1; ++t) {
                    const bool u = t < bp && s > t && s < bp;
                    fv[t] = u ? s_f[r0 + t] : 0u;
                    yv[t] = u ? W[s_prof[r0 + t] * PIV_LDW + r0 + s] : 0u;
                }
#pragma unroll
                for (int t = 0; t < PIV_PB - 1; ++t) {
                    // computed by every lane and kept by selection (no branch between shuffles)
                    const uint32_t m = __shfl_sync(0xffffffffu, v, (lane & ~7) | t);
                    const uint32_t nv = ff<MONT>(fv[t], v, m, yv[t], M);
                    v = (t < bp && s > t && s < bp) ? nv : v;
                }
                if (vk) {
                    uint32_t cf = 0u;
                    if (s < bp) {
                        wk[r0 + s] = v;
                        const uint32_t at = (MONT && !WIDE) ? redc_once((uint64_t)v * hs, M) : mulm(v, hs, M);
                        cf = at ? M.p - at : 0u;
                    }
                    s_coef[k][s] = cf;
                    // the row's own column of E only picks up the scale
                    if (s == 0)
                        E[k * PIV_LDE + k] = (MONT && !WIDE) ? redc((uint64_t)E[k * PIV_LDE + k] * A0, M)   // A0 is A0 R here
                                                             : mulm(E[k * PIV_LDE + k], A0f, M);
                }
            }
            __syncthreads();
            // (c) window positions [r, wne) and E columns [0, pend) of rows [pend, lim):
            // a warp takes 32 columns (the panel's pivot-row entries in registers) and
            // 8 rows (coefficients read as broadcast vectors)
            {
                int pr[PIV_PB];
#pragma unroll
                for (int t = 0; t < PIV_PB; ++t) pr[t] = s_prof[r0 + (t < bp ? t : 0)];
                const int nwc = wne - r, ncol = nwc + pend;
                const int nch = (ncol + 31) >> 5, nrg = (lim - pend + 7) >> 3;
                // one entry: x <- A0 x + sum_t cf_t y_t
                auto fused = [&](uint32_t *xp, const uint32_t (&cf)[PIV_PB], const uint32_t (&y)[PIV_PB]) {
                    if (WIDE) {
                        Acc acc = {(uint64_t)A0 * *xp, 0u};
#pragma unroll
                        for (int t = 0; t < PIV_PB; ++t) acc_add(acc, (uint64_t)cf[t] * y[t]);
                        *xp = acc_red(acc, M);
                    } else {
                        uint64_t sum = (uint64_t)A0 * *xp;
#pragma unroll
                        for (int t = 0; t < PIV_PB; ++t) sum += (uint64_t)cf[t] * y[t];
                        *xp = MONT ? redc_once(sum, M) : red64(sum, M);
                    }
                };
                auto coefs = [&](const int k, uint32_t (&cf)[PIV_PB]) {
                    const uint4 c0 = *(const uint4 *)&s_coef[k][0];
                    const uint4 c1 = *(const uint4 *)&s_coef[k][4];
                    cf[0] = c0.x; cf[1] = c0.y; cf[2] = c0.z; cf[3] = c0.w;
                    cf[4] = c1.x; cf[5] = c1.y; cf[6] = c1.z; cf[7] = c1.w;
                };
                // Pipelined with the next panel when both take the fast path: warp 0 updates the
                // next panel's 8 x 8 diagonal block itself and eliminates it at once (block_elim),
                // while the other warps update everything else; the next panel then starts with
                // its block done. A zero pivot there leaves the updated block in place for the
                // stepwise path.
                const bool pipe = fast && try_fast && brows - pend >= PIV_PB && r + PIV_PB <= wne;
                if (pipe && warp == 0) {
                    const int k = pend + (lane >> 2), c0 = r + 2 * (lane & 3);
                    uint32_t cf[PIV_PB];
                    coefs(k, cf);
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        uint32_t y[PIV_PB];
#pragma unroll
                        for (int t = 0; t < PIV_PB; ++t) y[t] = W[pr[t] * PIV_LDW + c0 + e];
                        fused(W + k * PIV_LDW + c0 + e, cf, y);
                    }
                    __syncwarp();
                    block_elim(pend, r);
                } else if (!(pipe && PIV_QUIET && (warp & 3) == 0)) {
                    // With PIV_QUIET the warps that share warp 0's scheduler (warp % 4 == 0
                    // on this GPU) stay out of a pipelined update, so that the block
                    // elimination on warp 0's dependency chain issues without contention.
                    const int w1 = !pipe ? warp : PIV_QUIET ? warp - (warp >> 2) - 1 : warp - 1;
                    const int nw1 = !pipe ? nw : PIV_QUIET ? nw - (nw >> 2) : nw - 1;
                    for (int it = w1; it < nch * nrg; it += nw1) {
                        const int rg = it / nch, ch = it - rg * nch;
                        const int ci = 32 * ch + lane;
                        if (ci >= ncol) continue;
                        const bool inw = ci < nwc;
                        const int col = inw ? r + ci : ci - nwc;
                        const uint32_t *ybase = inw ? W + col : E + col;
                        const int ys = inw ? PIV_LDW : PIV_LDE;
                        uint32_t y[PIV_PB];
#pragma unroll
                        for (int t = 0; t < PIV_PB; ++t) y[t] = ybase[pr[t] * ys];
                        // the next panel's diagonal block is warp 0's when pipelined
                        const int k0 = (pipe && rg == 0 && inw && ci < PIV_PB) ? pend + 8 : pend + 8 * rg;
                        const int k1 = pend + 8 * rg + 8 < lim ? pend + 8 * rg + 8 : lim;
                        uint32_t *xp = (inw ? W : E) + k0 * ys + col;
                        for (int k = k0; k < k1; ++k, xp += ys) {
                            uint32_t cf[PIV_PB];
                            coefs(k, cf);
                            fused(xp, cf, y);
                        }
                    }
                }
                pre_done = pipe;
            }
            __syncthreads();
        }
    }
    const int rs = r;

    // Row scales: step t multiplied the rows below its pivot row by mu_t = f_t (R^{-1} f_t in
    // the Montgomery variant), and s_Sfwd[t] = prod_{t' < t} mu_t' (Sprod is the whole
    // product). One parallel pass inverts every prefix product; mu_t^{-1} =
    // Sfwd[t] / Sfwd[t + 1] is then a single product, so no prefix scan is needed. For odd p
    // Sinv is kept in Montgomery representation (Sinv R), as the C values below expect.
    for (int t = tid; t <= rs; t += nt) s_Spinv[t] = inv_any<MONT>(t < rs ? s_Sfwd[t] : Sprod, M);
    __syncthreads();
    for (int t = tid; t < rs; t += nt) {
        const uint32_t muinv = mulm(s_Sfwd[t], s_Spinv[t + 1], M);
        s_muinv[t] = muinv;
        s_Sinv[t] = MONT ? redc((uint64_t)s_Spinv[t] * M.r2, M) : s_Spinv[t];
        s_finv[t] = MONT ? redc((uint64_t)muinv, M) : muinv;   // f^{-1} = mu^{-1} R^{-1}
    }
    __syncthreads();

    // C values of the resolved rows: W[i][t] carries the scale S_t of step t.
    // L^{-1} for the finish kernel: pivot row t of the eliminated slab is
    // (E X)_t = f_t U_t, so U = diag(1/f) E_pp X over the pivot rows, i.e.
    // L^{-1}[t][u] = E[prof t][prof u] / f_t (zero for u > t). For odd p the
    // factors are Montgomery representations (Sinv R, and f^{-1} R = mu^{-1}),
    // so each entry is one Montgomery step.
    // (512 threads: column t or u = tid % 64, rows g + 8 j for the row group g = tid / 64;
    // each thread's eight values are read from shared memory before any is stored)
    {
        const int t = tid & (CUP_BMAX - 1), g = tid >> 6;
        if (t < rs) {
            const int pt = s_prof[t];
            const uint32_t sinv = s_Sinv[t];
            uint32_t wv[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) wv[j] = W[(g + 8 * j) * PIV_LDW + t];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int i = g + 8 * j;
                if (i < stop)
                    S->Cn[i][t] = (i >= pt) ? (MONT ? redc((uint64_t)wv[j] * sinv, M) : mulm(wv[j], sinv, M)) : 0u;
            }
            const int pu = pt;                 // the same column, as u
            uint32_t ev[8], mv[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int t2 = g + 8 * j;
                const int pr = t2 < rs ? s_prof[t2] : 0;
                ev[j] = E[pr * PIV_LDE + pu];
                mv[j] = MONT ? s_muinv[t2] : s_finv[t2];
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int t2 = g + 8 * j;
                if (t2 < rs) S->Linv[t2][t] = MONT ? redc((uint64_t)ev[j] * mv[j], M) : mulm(ev[j], mv[j], M);
            }
        }
    }
    for (int t = tid; t < rs; t += nt)
        S->pinv[t] = MONT ? redc((uint64_t)s_Sfwd[t] * s_muinv[t], M) : mulm(s_Sfwd[t], s_finv[t], M);
    if (warp == 0) {
        int ns = 0;
        for (int base = 0; base < wne; base += 32) {
            const int q = base + lane;
            const bool disp = (q < wne) && (s_wcol[q] != q);
            const unsigned bal = __ballot_sync(0xffffffffu, disp);
            const int sl = disp ? ns + __popc(bal & ((1u << lane) - 1u)) : -1;
            if (q < wne) {
                S->win_col[q] = s_wcol[q];
                S->win_slot[q] = sl;
                if (disp) s_sorig[sl] = s_wcol[q];
            }
            ns += __popc(bal);
        }
        if (lane == 0) {
            S->ext_pos = s_ext;
            S->ext_slot = -1;
            if (s_ext >= 0) { S->ext_slot = ns; s_sorig[ns] = 0; ++ns; }
            s_slot[0] = ns;
            S->n_slot = ns;
            S->r_s = rs;
            S->i_stop = stop;
            S->wne = wne;
            S->n_spec = nspec;
            S->spec_fail = 0;
            if (rank_next) *rank_next = col0 + rs;
        }
    }
    for (int t = tid; t < rs; t += nt) {
        S->prof[t] = s_prof[t];
        g_ipiv[col0 + t] = col0 + s_pos[t];
        g_prof[col0 + t] = a + s_prof[t];
    }
    for (int k = tid; k < nspec; k += nt) S->spec_rows[k] = s_spec[k];
    __syncthreads();
    // original values of every displaced position, for every slab row
    const int nslot = s_slot[0];
    for (int idx = tid; idx < nslot * brows; idx += nt) {
        int sl = idx / brows, i = idx - sl * brows;
        S->Dorig[sl][i] = A[(a + i) * lda + col0 + s_sorig[sl]];
    }
}

// ---------------------------------------------------------------------------
// Leaf slab, finish phase (grid over column positions).
//
// For each position q of the slab, U's rows at q solve L u = x, with x the
// original pivot-row values of the column now at q (via the recorded
// transpositions) and L the pivot rows of C (lower triangular, pivots on the
// diagonal): a forward substitution done by four lanes per column. The final
// [C\U] content is then written with U's rows placed directly at global rows
// col0 .. col0 + r_s (their place in the space-sharing storage of the whole
// matrix) and C in the slab rows. Rows taken as dependent by a speculating
// pivot kernel are checked here: their residual x - C u must vanish.
// ---------------------------------------------------------------------------
#define FIN_LD 72   // bf16 row stride of the digit planes (144 bytes: conflict-free fragment loads)

// MODE 0 / 1: U = Linv X by 64-bit CUDA-core products (1: wide sums); MODE 2 + l:
// by tensor-core bf16 products of l-limb digits (fp32 partial sums stay exact:
// 64 * l * 2^14 < 2^24), recombined in 64 bits.
template <int MODE>
__global__ void __launch_bounds__(256)
k_slab_finish(uint32_t *__restrict__ A, int64_t lda, int64_t a, int brows, const Dyn col0d, int64_t n, ModP M,
              SlabScratch *__restrict__ S, int *__restrict__ err, uint64_t off)
{
    constexpr bool WIDE = MODE == 1;
    constexpr int TCL = MODE >= 2 ? MODE - 1 : 0;
    constexpr int TL = TCL > 0 ? TCL : 1;            // array extent for the digit code
    // The launch just before this one is the slab's pivot kernel, which writes the
    // scratch S but not A, and col0 comes from the leaf before: the slab rows' values
    // in this tile's columns (the pivot rows' original values, except at displaced
    // positions, which S->Dorig keeps) are copied in before the dependency wait.
    const int64_t col0 = col0d.eval();
    const int64_t w = n - col0;
    const int64_t q0 = (int64_t)blockIdx.x * CUP_QT;
    if (q0 >= w) {
        pdl_enter();
        return;
    }
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nq = (int)((w - q0) < CUP_QT ? (w - q0) : CUP_QT);
    extern __shared__ __align__(16) uint8_t fdyn[];
    uint32_t (*sTile)[CUP_QT + 1] = (uint32_t (*)[CUP_QT + 1])(fdyn + (TCL > 0 ? 2 * TCL * CUP_BMAX * FIN_LD * 2 : 0));
    for (int idx = tid; idx < brows * CUP_QT; idx += nt) {
        const int i = idx >> 6, qq = idx & (CUP_QT - 1);
        if (qq < nq) cp_async4(&sTile[i][qq], A + (a + i) * lda + col0 + q0 + qq);
    }
    cp_async_commit();
    pdl_enter();
    __shared__ uint32_t sL[CUP_BMAX][CUP_BMAX + 1];
    __shared__ uint32_t sX[CUP_BMAX][CUP_QT + 1];
    __shared__ uint32_t sPinv[CUP_BMAX];
    __shared__ int sOrig[CUP_QT], sSlot[CUP_QT], sProf[CUP_BMAX];

    // Every read of the scratch is issued at once (its arrays have fixed sizes, so each
    // read is in bounds); the slab's counts only select among the values afterwards.
    const int u = tid & 63, t0 = tid >> 6;          // 4 row groups
    uint32_t lv[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) lv[k] = S->Linv[t0 + 4 * k][u];
    int prof_v = 0, wcol_v = 0, wslot_v = -1;
    uint32_t pinv_v = 0u;
    if (tid < CUP_BMAX) { prof_v = S->prof[tid]; pinv_v = S->pinv[tid]; }
    if (tid < CUP_QT && q0 + tid < CUP_WNMAX) { wcol_v = S->win_col[q0 + tid]; wslot_v = S->win_slot[q0 + tid]; }
    const int rs = S->r_s, stop = S->i_stop, wne = S->wne;
    const int ext_pos = S->ext_pos, ext_slot = S->ext_slot;
    if (TCL > 0 && q0 == 0) {
        // the first tile also writes the slab's C values (positions < r_s <= CUP_QT);
        // the tensor-core product leaves sL unused, so their copy into it starts now
        // and lands while the product runs
        for (int idx = tid; idx < CUP_BMAX * CUP_BMAX; idx += nt) {
            const int i = idx >> 6, t = idx & 63;
            if (i < stop && t < rs) cp_async4(&sL[i][t], &S->Cn[i][t]);
        }
    }
    cp_async_commit();

    if (tid < rs) { sProf[tid] = prof_v; sPinv[tid] = pinv_v; }      // rs <= CUP_BMAX <= blockDim
    if (tid < nq) {
        const int64_t q = q0 + tid;
        int orig, slot;
        if (q < wne) { orig = wcol_v; slot = wslot_v; }
        else if (q == ext_pos) { orig = 0; slot = ext_slot; }
        else { orig = (int)q; slot = -1; }
        sOrig[tid] = orig;
        sSlot[tid] = slot;
    }
    cp_async_wait_prior<1>();                         // the tile (the C values may still fly)
    __syncthreads();
    {
        // X from the tile (or the displaced values; a position that is not displaced holds
        // its own column), Linv as read above
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int t = t0 + 4 * k;
            lv[k] = (t < rs && u < rs) ? lv[k] : 0u;
        }
        if (TCL == 0) {
            const int slot = sSlot[u];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int t = t0 + 4 * k;
                uint32_t xv = 0u;
                if (t < rs && u < nq) xv = (slot >= 0) ? S->Dorig[slot][sProf[t]] : sTile[sProf[t]][u];
                sL[t][u] = lv[k];
                sX[t][u] = xv;
            }
        } else {
            // digit planes: Linv row-major (k = u contiguous), X transposed (n = u rows, k = t
            // contiguous). X is taken by warp w for columns w + 8 m with the lanes along t, so
            // its transposed stores are consecutive (the tile's rows are padded to 65 words,
            // so reading a column of it is conflict-free too).
            __nv_bfloat16 *Ld = (__nv_bfloat16 *)fdyn;
            __nv_bfloat16 *Xt = Ld + TL * CUP_BMAX * FIN_LD;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int t = t0 + 4 * k;
                __nv_bfloat16 dl[TL];
                limb_digits<TL>(lv[k], M.p, dl);
#pragma unroll
                for (int l = 0; l < TCL; ++l) Ld[(l * CUP_BMAX + t) * FIN_LD + u] = dl[l];
            }
            const int wx = tid >> 5, lx = tid & 31;
            uint32_t xw[16];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int u2 = wx + 8 * m, slot2 = sSlot[u2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int t2 = lx + 32 * h;
                    const int pr = t2 < rs ? sProf[t2] : 0;
                    uint32_t x = 0u;
                    if (t2 < rs && u2 < nq) x = (slot2 >= 0) ? S->Dorig[slot2][pr] : sTile[pr][u2];
                    xw[2 * m + h] = x;
                }
            }
#pragma unroll
            for (int m = 0; m < 8; ++m)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    __nv_bfloat16 dx[TL];
                    limb_digits<TL>(xw[2 * m + h], M.p, dx);
#pragma unroll
                    for (int l = 0; l < TCL; ++l) Xt[(l * CUP_BMAX + wx + 8 * m) * FIN_LD + lx + 32 * h] = dx[l];
                }
        }
    }
    __syncthreads();
    if (TCL > 0) {
        // U tile = Linv X on the tensor cores: warp (mt, nh) owns rows 16 mt .. + 15 and
        // columns 32 nh .. + 31 (four 16 x 8 tiles); shift s = i + j collects the digit
        // products A_i B_j
        constexpr int NS = 2 * TL - 1;
        const __nv_bfloat16 *Ld = (const __nv_bfloat16 *)fdyn;
        const __nv_bfloat16 *Xt = Ld + TL * CUP_BMAX * FIN_LD;
        const int warp = tid >> 5, lane = tid & 31;
        const int mt = warp & 3, nh = warp >> 2, g = lane >> 2, tq = lane & 3;
        float acc[NS][4][4];
#pragma unroll
        for (int s2 = 0; s2 < NS; ++s2)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[s2][j][e] = 0.f;
        const int nks = (rs + 15) >> 4;
        for (int ks = 0; ks < nks; ++ks) {
            const int k0 = 16 * ks + 2 * tq;
            uint32_t af[TL][4];
#pragma unroll
            for (int i = 0; i < TCL; ++i) {
                const __nv_bfloat16 *ar = Ld + (i * CUP_BMAX + 16 * mt + g) * FIN_LD + k0;
                af[i][0] = *(const uint32_t *)ar;
                af[i][1] = *(const uint32_t *)(ar + 8 * FIN_LD);
                af[i][2] = *(const uint32_t *)(ar + 8);
                af[i][3] = *(const uint32_t *)(ar + 8 * FIN_LD + 8);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
                for (int j = 0; j < TCL; ++j) {
                    const __nv_bfloat16 *br = Xt + (j * CUP_BMAX + 32 * nh + 8 * nt + g) * FIN_LD + k0;
                    const uint32_t b0 = *(const uint32_t *)br, b1 = *(const uint32_t *)(br + 8);
#pragma unroll
                    for (int i = 0; i < TCL; ++i) mma_16816(acc[i + j][nt], af[i], b0, b1);
                }
            }
        }
        __syncthreads();                                   // every digit read is done
        const uint32_t mu32 = (uint32_t)(M.mu >> 32);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int t = 16 * mt + g + 8 * (e >> 1), qq = 32 * nh + 8 * nt + 2 * tq + (e & 1);
                int64_t v = 0;
#pragma unroll
                for (int s2 = NS - 1; s2 >= 0; --s2) v = v * 256 + (int64_t)__float2int_rn(acc[s2][nt][e]);
                const uint64_t x = (uint64_t)(v + (int64_t)off);
                uint32_t rr;
                if (M.p & 1u) {
                    const uint32_t m = (uint32_t)x * M.pneg;
                    uint32_t tt = (uint32_t)((x + (uint64_t)m * M.p) >> 32);   // x R^{-1} + (< p), below 2^32
                    tt -= __umulhi(tt, mu32) * M.p;
                    if (tt >= M.p) tt -= M.p;
                    rr = redc((uint64_t)tt * M.r2, M);                       // times R
                } else {
                    rr = red64(x, M);
                }
                if (t < rs) sX[t][qq] = rr;
            }
    } else {
    // U tile = Linv X: each thread a 4 x 4 block (rows ty + 16 i, columns tx + 16 j)
    {
        const int tx = tid & 15, ty = tid >> 4;
        uint64_t lo[4][4];
        uint32_t hi[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) { lo[i][j] = 0ull; hi[i][j] = 0u; }
        for (int u = 0; u < rs; ++u) {
            uint32_t av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = sL[ty + 16 * i][u];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = sX[u][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint64_t pr = (uint64_t)av[i] * bv[j];
                    if (WIDE) {
                        const uint64_t s2 = lo[i][j] + pr;
                        hi[i][j] += (s2 < pr);
                        lo[i][j] = s2;
                    } else {
                        lo[i][j] += pr;
                    }
                }
        }
        __syncthreads();                                   // every read of sX is done
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int t = ty + 16 * i;
                if (t < rs) {
                    Acc acc = {lo[i][j], hi[i][j]};
                    sX[t][tx + 16 * j] = acc_red(acc, M);
                }
            }
    }
    }
    __syncthreads();
    // rows taken as dependent: residual x_i - sum_t C[i][t] u_t must be zero at every position
    const int nspec = S->n_spec;
    if (nspec > 0) {
        int bad = 0;
        for (int idx = tid; idx < nspec * nq; idx += nt) {
            const int k = idx / nq, qq = idx - k * nq;
            const int i = S->spec_rows[k];
            const int slot = sSlot[qq];
            const uint32_t x = (slot >= 0) ? S->Dorig[slot][i] : A[(a + i) * lda + col0 + sOrig[qq]];
            Acc acc = {0ull, 0u};
            for (int t = 0; t < rs; ++t) acc_add(acc, (uint64_t)S->Cn[i][t] * sX[t][qq]);
            if (acc_red(acc, M) != x) bad = 1;
        }
        if (__syncthreads_or(bad) && tid == 0) {
            atomicExch(&S->spec_fail, 1);
            if (err) atomicCAS(err, 0, CUP_DEVERR_SPECULATION);
        }
    }
    // C values for the first tile: already in sL with tensor-core digits, else read now
    // (sL is free again after the CUDA-core product)
    if (TCL > 0 && q0 == 0) cp_async_wait_all();
    if (TCL == 0 && q0 == 0) {
        __syncthreads();
        const int t = tid & 63, i0 = tid >> 6;
        uint32_t cv[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) cv[k] = (i0 + 4 * k < stop && t < rs) ? S->Cn[i0 + 4 * k][t] : 0u;
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (i0 + 4 * k < stop && t < rs) sL[i0 + 4 * k][t] = cv[k];
    }
    __syncthreads();
    // rows: U rows col0 + t (t < rs), then slab rows a + i (i < stop) that are not U rows.
    // Thread (column qq, row group g; 256 threads) takes rows g + 4 j of each kind: all 16
    // values of a kind are gathered from shared memory before its stores (indices clamped
    // into the arrays, the selections made on the values).
    {
        const int qq = tid & (CUP_QT - 1), g = tid >> 6;
        if (qq < nq) {
            const int64_t q = q0 + qq;
            const int qc = q < rs ? (int)q : 0;
            uint32_t *colp = A + col0 + q;
            uint32_t vu[16], vs[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int k = g + 4 * j;
                const int64_t rho = col0 + k;
                const int ri = rho >= a ? (int)(rho - a) : 0;
                const uint32_t x = sX[k][qq], c = sL[ri][qc];
                vu[j] = (q > k) ? x : (rho >= a && q < rs) ? c : 0u;
                const uint32_t cs = sL[k][qc];
                vs[j] = q < rs ? cs : 0u;
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int k = g + 4 * j;
                if (k < rs) colp[(col0 + k) * lda] = vu[j];
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int i = g + 4 * j;
                const int64_t rho = a + i;
                if (i < stop && rho >= col0 + rs) colp[rho * lda] = vs[j];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Column transpositions. The recorded pivots ipiv[t] (absolute positions) are
// first compacted to the nontrivial ones, in order; then every row applies
// them in sequence (Sec. 1.1: right multiplication by P^T permutes columns).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_swaplist(const int64_t *__restrict__ ipiv, const Dyn k0d, const Dyn k1d, int2 *__restrict__ pairs,
           int *__restrict__ count)
{
    const int64_t k0 = k0d.eval(), k1 = k1d.eval();
    __shared__ int warp_cnt[32], warp_excl[32];
    __shared__ int chunk_total, base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) base = 0;
    __syncthreads();
    for (int64_t c0 = k0; c0 < k1; c0 += 1024) {
        int64_t t = c0 + tid;
        int64_t c = (t < k1) ? ipiv[t] : t;
        bool nz = (t < k1) && (c != t);
        unsigned bal = __ballot_sync(0xffffffffu, nz);
        if (lane == 0) warp_cnt[warp] = __popc(bal);
        __syncthreads();
        if (warp == 0) {
            int v = warp_cnt[lane];
            int incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            warp_excl[lane] = incl - v;
            if (lane == 31) chunk_total = incl;
        }
        __syncthreads();
        if (nz) {
            int off = base + warp_excl[warp] + __popc(bal & ((1u << lane) - 1u));
            pairs[off] = make_int2((int)t, (int)c);
        }
        __syncthreads();
        if (tid == 0) base += chunk_total;
        __syncthreads();
    }
    if (tid == 0) *count = base;
}

__global__ void __launch_bounds__(256)
k_laswp(uint32_t *__restrict__ A, int64_t lda, const Dyn row0d, const Dyn nrowsd,
        const int2 *__restrict__ pairs, const int *__restrict__ count)
{
    const int64_t row0 = row0d.eval(), nrows = nrowsd.eval();
    __shared__ int2 sp[256];
    const int n = *count;
    if (n == 0) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t *row = A + (row0 + i) * lda;
    for (int b = 0; b < n; b += 256) {
        __syncthreads();
        if (b + (int)threadIdx.x < n) sp[threadIdx.x] = pairs[b + threadIdx.x];
        __syncthreads();
        if (i < nrows) {
            int e = (n - b) < 256 ? (n - b) : 256;
            for (int k = 0; k < e; ++k) {
                int2 pr = sp[k];
                uint32_t x = row[pr.x];
                row[pr.x] = row[pr.y];
                row[pr.y] = x;
            }
        }
    }
}

// Transpositions (t, ipiv[t]) for t in [k0, k1), compacted to the nontrivial
// ones by every CTA itself (in order, a chunk of 256 at a time), then applied
// to this CTA's rows: one launch, no separate list.
__global__ void __launch_bounds__(256)
k_laswp_fused(uint32_t *__restrict__ A, int64_t lda, const Dyn row0d, const Dyn nrowsd,
              const int64_t *__restrict__ ipiv, const Dyn k0d, const Dyn k1d)
{
    pdl_enter();
    const int64_t row0 = row0d.eval(), nrows = nrowsd.eval();
    const int64_t k0 = k0d.eval(), k1 = k1d.eval();
    if (k1 <= k0 || nrows <= 0 || (int64_t)blockIdx.x * blockDim.x >= nrows) return;
    __shared__ int2 sp[256];
    __shared__ int wcnt[8], wex[8], tot;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + tid;
    uint32_t *row = A + (row0 + i) * lda;
    {
        // usually every transposition of the range is trivial: check the whole range
        // with independent loads (one memory latency) before the ordered pass
        bool any = false;
        for (int64_t t = k0 + tid; t < k1; t += blockDim.x) any |= ipiv[t] != t;
        if (!__syncthreads_or(any)) return;
    }
    for (int64_t c0 = k0; c0 < k1; c0 += 256) {
        const int64_t t = c0 + tid;
        const int64_t c = (t < k1) ? ipiv[t] : t;
        const bool nz = (t < k1) && (c != t);
        const unsigned bal = __ballot_sync(0xffffffffu, nz);
        if (lane == 0) wcnt[warp] = __popc(bal);
        __syncthreads();
        if (tid == 0) {
            int acc = 0;
            for (int w = 0; w < 8; ++w) { wex[w] = acc; acc += wcnt[w]; }
            tot = acc;
        }
        __syncthreads();
        if (nz) sp[wex[warp] + __popc(bal & ((1u << lane) - 1u))] = make_int2((int)t, (int)c);
        __syncthreads();
        if (i < nrows)
            for (int k = 0; k < tot; ++k) {
                const int2 pr = sp[k];
                const uint32_t x = row[pr.x];
                row[pr.x] = row[pr.y];
                row[pr.y] = x;
            }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Plain CUDA-core Schur update C <- C - A B mod p (Algorithm 1, alpha = -1,
// beta = 1). 64 x 64 tiles, 4 x 4 outputs per thread, exact 64-bit products;
// when K (p-1)^2 may reach 2^64 the accumulators also count wraps.
// ---------------------------------------------------------------------------
#define GB_M 64
#define GB_N 64
#define GB_K 16
template <bool WIDE>
__global__ void __launch_bounds__(256)
k_gemm_sub_cc(const GemmDesc d, ModP Mp)
{
    pdl_enter();
    const int64_t Mr = d.M, N = d.N.eval(), K = d.K.eval();
    if ((int64_t)blockIdx.x * GB_N >= N || K <= 0) return;
    const int add = d.add;
    const int64_t lda = d.lda, ldb = d.ldb, ldc = d.ldc;
    const uint32_t *__restrict__ A = d.A + d.arow.eval() * lda + d.acol.eval();
    const uint32_t *__restrict__ B = d.B + d.brow.eval() * ldb + d.bcol.eval();
    uint32_t *__restrict__ C = d.C + d.crow.eval() * ldc + d.ccol.eval();
    __shared__ uint32_t As[GB_K][GB_M + 4];
    __shared__ uint32_t Bs[GB_K][GB_N + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * GB_M, n0 = (int64_t)blockIdx.x * GB_N;
    uint64_t acc[4][4];
    uint32_t hi[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { acc[i][j] = 0ull; hi[i][j] = 0u; }

    for (int64_t k0 = 0; k0 < K; k0 += GB_K) {
        for (int idx = threadIdx.x; idx < GB_M * GB_K; idx += 256) {
            int r = idx / GB_K, kk = idx - r * GB_K;
            int64_t gr = m0 + r, gk = k0 + kk;
            As[kk][r] = (gr < Mr && gk < K) ? A[gr * lda + gk] : 0u;
        }
        for (int idx = threadIdx.x; idx < GB_K * GB_N; idx += 256) {
            int kk = idx / GB_N, c = idx - kk * GB_N;
            int64_t gk = k0 + kk, gc = n0 + c;
            Bs[kk][c] = (gk < K && gc < N) ? B[gk * ldb + gc] : 0u;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            uint32_t av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    uint64_t pr = (uint64_t)av[i] * bv[j];
                    if (WIDE) {
                        uint64_t s = acc[i][j] + pr;
                        hi[i][j] += (s < pr);
                        acc[i][j] = s;
                    } else {
                        acc[i][j] += pr;
                    }
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t gr = m0 + ty + 16 * i, gc = n0 + tx + 16 * j;
            if (gr < Mr && gc < N) {
                Acc a = {acc[i][j], hi[i][j]};
                uint32_t v = acc_red(a, Mp);
                uint32_t *cp = C + gr * ldc + gc;
                *cp = add ? addm(*cp, v, Mp) : subm(*cp, v, Mp);
            }
        }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_slab_pivots(const uint32_t *A, int64_t lda, int64_t a, int brows, Dyn col0, int64_t n,
                               int wn, int speculate, ModP M, SlabScratch *S, int64_t *ipiv, int64_t *prof,
                               int64_t *rank_next, cudaStream_t st)
{
    static PerDeviceOnce attr;
    // window rows, then the row-operation matrix
    const size_t smem = ((size_t)CUP_BMAX * PIV_LDW + (size_t)CUP_BMAX * PIV_LDE) * sizeof(uint32_t);
    (void)brows;
    {
        const cudaError_t e = once_per_device(attr, [&] {
            const int mx = (int)smem;
            cudaError_t e2 = cudaFuncSetAttribute(k_slab_pivots<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
            if (e2 == cudaSuccess)
                e2 = cudaFuncSetAttribute(k_slab_pivots<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
            if (e2 == cudaSuccess)
                e2 = cudaFuncSetAttribute(k_slab_pivots<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
            return e2;
        });
        if (e != cudaSuccess) return e;
    }
    // The block update sums PIV_PB + 1 products below p^2 in 64 bits when that cannot wrap;
    // for odd p that sum is reduced by one Montgomery step, which needs it below p 2^32
    // (p < 2^28.8). Larger p take the wide accumulators.
    const uint64_t pm1 = M.p - 1u;
    const bool wide = pm1 * pm1 > ~0ull / (uint64_t)(PIV_PB + 1) ||
                      ((M.p & 1u) && (unsigned __int128)(PIV_PB + 1) * pm1 * pm1 >= ((unsigned __int128)M.p << 32));
    if (M.p & 1u) {
        if (wide)
            return launch_pdl(k_slab_pivots<true, true>, 1, PIV_THREADS, smem, st, A, lda, a, brows, col0, n, wn,
                              speculate, M, S, ipiv, prof, rank_next);
        else
            return launch_pdl(k_slab_pivots<true, false>, 1, PIV_THREADS, smem, st, A, lda, a, brows, col0, n, wn,
                              speculate, M, S, ipiv, prof, rank_next);
    } else {
        return launch_pdl(k_slab_pivots<false, false>, 1, PIV_THREADS, smem, st, A, lda, a, brows, col0, n, wn,
                          speculate, M, S, ipiv, prof, rank_next);
    }
    return cudaGetLastError();
}

cudaError_t launch_slab_finish(uint32_t *A, int64_t lda, int64_t a, int brows, Dyn col0, int64_t n, ModP M,
                               const SlabScratch *S, int *err, cudaStream_t st, bool tensor)
{
    const int64_t wmax = n - col0.lo;
    int64_t nb = (wmax + CUP_QT - 1) / CUP_QT;
    if (nb <= 0) return cudaSuccess;
    if (brows < 1 || brows > CUP_BMAX) return cudaErrorInvalidValue;
    // dynamic shared memory: the digit planes (tensor modes), then the slab tile
    constexpr int tile = CUP_BMAX * (CUP_QT + 1) * 4;
    auto smem_of = [](int l) { return 2 * l * CUP_BMAX * FIN_LD * 2 + tile; };
    static PerDeviceOnce attr;
    const cudaError_t e = once_per_device(attr, [&] {
        cudaError_t e2 = cudaFuncSetAttribute(k_slab_finish<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_of(0));
        if (e2 == cudaSuccess)
            e2 = cudaFuncSetAttribute(k_slab_finish<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_of(0));
        if (e2 == cudaSuccess)
            e2 = cudaFuncSetAttribute(k_slab_finish<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_of(1));
        if (e2 == cudaSuccess)
            e2 = cudaFuncSetAttribute(k_slab_finish<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_of(2));
        if (e2 == cudaSuccess)
            e2 = cudaFuncSetAttribute(k_slab_finish<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_of(3));
        return e2;
    });
    if (e != cudaSuccess) return e;
    const uint32_t p = M.p;
    SlabScratch *Sm = const_cast<SlabScratch *>(S);
    if (tensor && p < (1u << 24)) {
        // tensor-core product of l-limb digits; the recombined value is below 2^55 in size
        const int l = p < (1u << 8) ? 1 : p < (1u << 16) ? 2 : 3;
        const uint64_t off = ((1ull << 55) / p + 1) * p;
        if (l == 1)
            return launch_pdl(k_slab_finish<2>, (unsigned)nb, 256, smem_of(1), st, A, lda, a, brows, col0, n, M, Sm, err, off);
        if (l == 2)
            return launch_pdl(k_slab_finish<3>, (unsigned)nb, 256, smem_of(2), st, A, lda, a, brows, col0, n, M, Sm, err, off);
        return launch_pdl(k_slab_finish<4>, (unsigned)nb, 256, smem_of(3), st, A, lda, a, brows, col0, n, M, Sm, err, off);
    }
    // a row of Linv times a column of X sums CUP_BMAX products: wide sums unless CUP_BMAX (p-1)^2 < 2^64
    const bool wide = (long double)CUP_BMAX * (M.p - 1) * (long double)(M.p - 1) >= 18446744073709551615.0L;
    if (wide)
        return launch_pdl(k_slab_finish<1>, (unsigned)nb, 256, smem_of(0), st, A, lda, a, brows, col0, n, M, Sm, err,
                          (uint64_t)0);
    return launch_pdl(k_slab_finish<0>, (unsigned)nb, 256, smem_of(0), st, A, lda, a, brows, col0, n, M, Sm, err,
                      (uint64_t)0);
}

cudaError_t launch_swaplist(const int64_t *ipiv, Dyn k0, Dyn k1, int2 *pairs, int *count, cudaStream_t st)
{
    k_swaplist<<<1, 1024, 0, st>>>(ipiv, k0, k1, pairs, count);
    return cudaGetLastError();
}

cudaError_t launch_laswp(uint32_t *A, int64_t lda, Dyn row0, Dyn nrows, const int2 *pairs, const int *count,
                         cudaStream_t st)
{
    if (nrows.hi <= 0) return cudaSuccess;
    int64_t nb = (nrows.hi + 255) / 256;
    k_laswp<<<(unsigned)nb, 256, 0, st>>>(A, lda, row0, nrows, pairs, count);
    return cudaGetLastError();
}

cudaError_t launch_laswp_fused(uint32_t *A, int64_t lda, Dyn row0, Dyn nrows, const int64_t *ipiv, Dyn k0, Dyn k1,
                               cudaStream_t st)
{
    if (nrows.hi <= 0 || k1.hi <= k0.lo) return cudaSuccess;
    int64_t nb = (nrows.hi + 255) / 256;
    return launch_pdl(k_laswp_fused, (unsigned)nb, 256, 0, st, A, lda, row0, nrows, ipiv, k0, k1);
}

cudaError_t launch_gemm_cc_desc(const GemmDesc &d, ModP M, cudaStream_t st)
{
    if (d.M <= 0 || d.N.hi <= 0 || d.K.hi <= 0) return cudaSuccess;
    dim3 grid((unsigned)((d.N.hi + GB_N - 1) / GB_N), (unsigned)((d.M + GB_M - 1) / GB_M));
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    // K (p-1)^2 < 2^64 means the 64-bit sum of products cannot wrap
    long double bound = (long double)d.K.hi * (long double)(M.p - 1) * (long double)(M.p - 1);
    if (bound < 18446744073709551615.0L)
        launch_pdl(k_gemm_sub_cc<false>, grid, 256, 0, st, d, M);
    else
        launch_pdl(k_gemm_sub_cc<true>, grid, 256, 0, st, d, M);
    return cudaGetLastError();
}

cudaError_t launch_gemm_sub_cc(const uint32_t *A, int64_t lda, const uint32_t *B, int64_t ldb,
                               uint32_t *C, int64_t ldc, int64_t Mr, int64_t N, int64_t K, ModP M,
                               cudaStream_t st, int add)
{
    GemmDesc d{A, lda, dconst(0), dconst(0), B, ldb, dconst(0), dconst(0), C, ldc, dconst(0), dconst(0),
               Mr, dconst(N), dconst(K), add};
    return launch_gemm_cc_desc(d, M, st);
}

// ---------------------------------------------------------------------------
// Determinant from a full-rank CUP: the product of C's diagonal (the pivots,
// stored on A's diagonal by [C\U]) times (-1)^(number of nontrivial
// transpositions) (Sec. 4.4; for rank n the profile is 0..n-1, so pivot t sits
// at (t, t)). One CTA, tree product modulo p.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_det_reduce(const uint32_t *__restrict__ A, int64_t lda, int64_t n, const int64_t *__restrict__ ipiv,
             ModP M, uint32_t *__restrict__ out)
{
    __shared__ uint32_t sp[1024];
    __shared__ int sneg[1024];
    uint32_t prod = 1u % M.p;
    int neg = 0;
    for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
        prod = mulm(prod, A[t * lda + t], M);
        neg ^= (ipiv[t] != t);
    }
    sp[threadIdx.x] = prod;
    sneg[threadIdx.x] = neg;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sp[threadIdx.x] = mulm(sp[threadIdx.x], sp[threadIdx.x + s], M);
            sneg[threadIdx.x] ^= sneg[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        uint32_t d = sp[0];
        *out = (sneg[0] && d) ? M.p - d : d;
    }
}

cudaError_t launch_det_reduce(const uint32_t *A, int64_t lda, int64_t n, const int64_t *ipiv, ModP M,
                              uint32_t *out, cudaStream_t st)
{
    k_det_reduce<<<1, 1024, 0, st>>>(A, lda, n, ipiv, M, out);
    return cudaGetLastError();
}
