/*
 * Plain CPU oracle for CUP over a prime field GF(p), p < 2^31.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path links, loads or calls
 * this file. It is used by the tests, by the smoke check and by the CPU
 * baseline leg of the benchmark. It shares no code, header or table with the
 * CUDA library: it is written from the definitions of Jeannerod, Pernet and
 * Storjohann, "Rank-profile revealing Gaussian elimination and the CUP matrix
 * decomposition", with plain loops, 64-bit integers and one `% p` per update.
 *
 * Conventions (Sec. 1.1): zero-based indices, half-open ranges, row-major
 * storage with a leading dimension. Entries are canonical residues in [0, p).
 *
 * Parity pins: every function below is checked by the CPU tests against
 * something other than itself (brute-force span tests for rank and profile,
 * Schur-complement minors for C and U, Leibniz determinants, A*A^{-1} = I,
 * uniqueness of the reduced column echelon form, exact big-integer products).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef uint32_t u32;
typedef uint64_t u64;
typedef int64_t i64;

int cupo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* a * b mod p, a, b in [0, p). */
static u32 mulm(u32 a, u32 b, u32 p) { return (u32)(((u64)a * b) % p); }

/* a - b mod p, a, b in [0, p). */
static u32 subm(u32 a, u32 b, u32 p) { return (u32)(((u64)a + p - b) % p); }

/* Inverse of a in GF(p) by the extended Euclidean algorithm; 0 if a == 0. */
u32 cupo_modinv(u32 a, u32 p)
{
    i64 r0 = p, r1 = a % p, s0 = 0, s1 = 1;
    if (r1 == 0) return 0;
    while (r1 != 0) {
        i64 q = r0 / r1, t;
        t = r0 - q * r1; r0 = r1; r1 = t;
        t = s0 - q * s1; s0 = s1; s1 = t;
    }
    /* r0 == gcd == 1 for prime p; s0 * a == 1 (mod p) */
    s0 %= (i64)p;
    if (s0 < 0) s0 += p;
    return (u32)s0;
}

/*
 * CUP decomposition by iterative Gaussian elimination with the pivot rule of
 * the recursive algorithm (Algorithm 6 and its base case): rows are taken in
 * order; for row i the pivot is the first column position c >= r (in the
 * current column order) where the residual of row i is nonzero; columns r and
 * c are transposed (T_{r,c}); U's row r is the residual divided by the pivot;
 * the rows below are eliminated (Sec. 2.2, iterative Gaussian elimination).
 *
 * Outputs (all caller-allocated):
 *   C       m x n (ldc), column echelon form; columns >= r are zero;
 *           C[i][t] = residual of row i at pivot t's column when pivot t was
 *           taken, for i >= profile[t], and 0 above profile[t].
 *   U       n x n (ldu), unit upper triangular; rows >= r are identity rows.
 *   ipiv    r entries, ipiv[t] = position swapped with t (LAPACK style);
 *           P = T_{r-1,ipiv[r-1]} ... T_{0,ipiv[0]} and A P^T = C U.
 *   profile r entries, the row rank profile.
 * Returns the rank r.
 */
i64 cupo_cup(const u32 *A, i64 m, i64 n, i64 lda, u32 p,
             u32 *C, i64 ldc, u32 *U, i64 ldu, i64 *ipiv, i64 *profile)
{
    u32 *W = (u32 *)malloc((size_t)(m > 0 ? m : 1) * (size_t)(n > 0 ? n : 1) * sizeof(u32));
    if (!W) return -1;
    for (i64 i = 0; i < m; ++i)
        memcpy(W + i * n, A + i * lda, (size_t)n * sizeof(u32));
    for (i64 i = 0; i < n; ++i)
        for (i64 j = 0; j < n; ++j)
            U[i * ldu + j] = (i == j) ? 1u : 0u;

    i64 r = 0;
    for (i64 i = 0; i < m && r < n; ++i) {
        u32 *row = W + i * n;
        i64 c = -1;
        for (i64 j = r; j < n; ++j)
            if (row[j] != 0) { c = j; break; }
        if (c < 0) continue;               /* row i is not in the rank profile */
        if (c != r) {                      /* transposition T_{r,c} on all columns */
#pragma omp parallel for schedule(static)
            for (i64 k = 0; k < m; ++k) {
                u32 t = W[k * n + r]; W[k * n + r] = W[k * n + c]; W[k * n + c] = t;
            }
            for (i64 k = 0; k < r; ++k) {
                u32 t = U[k * ldu + r]; U[k * ldu + r] = U[k * ldu + c]; U[k * ldu + c] = t;
            }
        }
        ipiv[r] = c;
        profile[r] = i;
        u32 inv = cupo_modinv(row[r], p);
        u32 *Ur = U + r * ldu;
        for (i64 j = r + 1; j < n; ++j)
            Ur[j] = mulm(row[j], inv, p);
#pragma omp parallel for schedule(static)
        for (i64 k = i + 1; k < m; ++k) {
            u32 *w = W + k * n;
            u32 f = w[r];
            if (f == 0) continue;
            for (i64 j = r + 1; j < n; ++j)
                w[j] = subm(w[j], mulm(f, Ur[j], p), p);
        }
        ++r;
    }
    for (i64 i = 0; i < m; ++i)
        for (i64 t = 0; t < n; ++t)
            C[i * ldc + t] = (t < r && i >= profile[t]) ? W[i * n + t] : 0u;
    free(W);
    return r;
}

/*
 * Space-sharing storage [C\U] of a CUP decomposition (Sec. 3.1): rows 0..r-1
 * hold U strictly above the diagonal; C's first r columns are stored on and
 * below the diagonal; everything else is zero.
 */
void cupo_pack(const u32 *C, i64 ldc, const u32 *U, i64 ldu, i64 m, i64 n, i64 r,
               u32 *out, i64 ldo)
{
    for (i64 i = 0; i < m; ++i)
        for (i64 j = 0; j < n; ++j) {
            u32 v = 0;
            if (i < r && j > i) v = U[i * ldu + j];
            else if (j < r && j <= i) v = C[i * ldc + j];
            out[i * ldo + j] = v;
        }
}

/* Apply column transpositions T_{t, ipiv[t]} for t = k0..k1-1, in order, to
 * rows 0..m-1 of A (A <- A P^T restricted to those transpositions). */
void cupo_laswp_cols(u32 *A, i64 m, i64 lda, const i64 *ipiv, i64 k0, i64 k1)
{
    for (i64 t = k0; t < k1; ++t) {
        i64 c = ipiv[t];
        if (c == t) continue;
        for (i64 i = 0; i < m; ++i) {
            u32 x = A[i * lda + t]; A[i * lda + t] = A[i * lda + c]; A[i * lda + c] = x;
        }
    }
}

/* Algorithm 1 with alpha = -1, beta = 1: C <- C - A B mod p.
 * A is M x K (lda), B is K x N (ldb), C is M x N (ldc). */
void cupo_mm_sub(u32 *Cm, i64 ldc, const u32 *A, i64 lda, const u32 *B, i64 ldb,
                 i64 M, i64 N, i64 K, u32 p)
{
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < M; ++i)
        for (i64 j = 0; j < N; ++j) {
            u32 acc = Cm[i * ldc + j];
            for (i64 k = 0; k < K; ++k)
                acc = subm(acc, mulm(A[i * lda + k], B[k * ldb + j], p), p);
            Cm[i * ldc + j] = acc;
        }
}

/* TRSM(Right, Upper, Unit): B <- B U^{-1}, U n x n unit upper triangular
 * (its diagonal and lower part are not read), B m x n. Row by row forward
 * substitution x_j = b_j - sum_{k<j} x_k u_{kj} (Algorithm 2, unit variant). */
void cupo_trsm_ruu(const u32 *Um, i64 ldu, u32 *B, i64 ldb, i64 m, i64 n, u32 p)
{
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < m; ++i) {
        u32 *x = B + i * ldb;
        for (i64 j = 0; j < n; ++j) {
            u32 acc = x[j];
            for (i64 k = 0; k < j; ++k)
                acc = subm(acc, mulm(x[k], Um[k * ldu + j], p), p);
            x[j] = acc;
        }
    }
}

/* TRSM(Left, Upper, Unit): B <- U^{-1} B, U n x n unit upper, B n x k.
 * Backward substitution by rows. */
void cupo_trsm_luu(const u32 *Um, i64 ldu, u32 *B, i64 ldb, i64 n, i64 k, u32 p)
{
    for (i64 i = n - 1; i >= 0; --i)
        for (i64 l = i + 1; l < n; ++l) {
            u32 f = Um[i * ldu + l];
            if (f == 0) continue;
            for (i64 j = 0; j < k; ++j)
                B[i * ldb + j] = subm(B[i * ldb + j], mulm(f, B[l * ldb + j], p), p);
        }
}

/* TRSM(Left, Lower, NonUnit): B <- L^{-1} B, L n x n lower triangular with
 * nonzero diagonal, B n x k. Forward substitution by rows. */
void cupo_trsm_lln(const u32 *L, i64 ldl, u32 *B, i64 ldb, i64 n, i64 k, u32 p)
{
    for (i64 i = 0; i < n; ++i) {
        for (i64 l = 0; l < i; ++l) {
            u32 f = L[i * ldl + l];
            if (f == 0) continue;
            for (i64 j = 0; j < k; ++j)
                B[i * ldb + j] = subm(B[i * ldb + j], mulm(f, B[l * ldb + j], p), p);
        }
        u32 inv = cupo_modinv(L[i * ldl + i], p);
        for (i64 j = 0; j < k; ++j)
            B[i * ldb + j] = mulm(B[i * ldb + j], inv, p);
    }
}

/*
 * Reduced column echelon form R of A (Sec. 2.2, Proposition 1) by column
 * Gauss-Jordan elimination, independent of the CUP routine: for each row in
 * order, if the row has a nonzero entry among the columns not yet used as
 * pivots, the first such column is moved to position r, scaled so that the
 * pivot is 1, and eliminated from every other column. R is unique, so the
 * choice of pivot column does not affect it.
 *
 * R (m x n, ldr) receives the form (columns >= rank are zero). If X is not
 * NULL it receives an n x n transform with A X = R (the same column
 * operations applied to the identity). profile (>= min(m,n) entries) receives
 * the row rank profile. Returns the rank.
 */
i64 cupo_rref(const u32 *A, i64 m, i64 n, i64 lda, u32 p, u32 *R, i64 ldr,
              u32 *X, i64 ldx, i64 *profile)
{
    u32 *W = (u32 *)malloc((size_t)(m > 0 ? m : 1) * (size_t)(n > 0 ? n : 1) * sizeof(u32));
    if (!W) return -1;
    for (i64 i = 0; i < m; ++i) memcpy(W + i * n, A + i * lda, (size_t)n * sizeof(u32));
    if (X)
        for (i64 i = 0; i < n; ++i)
            for (i64 j = 0; j < n; ++j) X[i * ldx + j] = (i == j);
    i64 r = 0;
    for (i64 i = 0; i < m && r < n; ++i) {
        i64 c = -1;
        for (i64 j = r; j < n; ++j)
            if (W[i * n + j] != 0) { c = j; break; }
        if (c < 0) continue;
        if (c != r) {
            for (i64 k = 0; k < m; ++k) { u32 t = W[k * n + r]; W[k * n + r] = W[k * n + c]; W[k * n + c] = t; }
            if (X) for (i64 k = 0; k < n; ++k) { u32 t = X[k * ldx + r]; X[k * ldx + r] = X[k * ldx + c]; X[k * ldx + c] = t; }
        }
        profile[r] = i;
        u32 inv = cupo_modinv(W[i * n + r], p);
        for (i64 k = 0; k < m; ++k) W[k * n + r] = mulm(W[k * n + r], inv, p);
        if (X) for (i64 k = 0; k < n; ++k) X[k * ldx + r] = mulm(X[k * ldx + r], inv, p);
        for (i64 j = 0; j < n; ++j) {
            if (j == r) continue;
            u32 f = W[i * n + j];
            if (f == 0) continue;
#pragma omp parallel for schedule(static)
            for (i64 k = 0; k < m; ++k) W[k * n + j] = subm(W[k * n + j], mulm(f, W[k * n + r], p), p);
            if (X) for (i64 k = 0; k < n; ++k) X[k * ldx + j] = subm(X[k * ldx + j], mulm(f, X[k * ldx + r], p), p);
        }
        ++r;
    }
    for (i64 i = 0; i < m; ++i) memcpy(R + i * ldr, W + i * n, (size_t)n * sizeof(u32));
    free(W);
    return r;
}

/* Determinant of an n x n matrix by textbook row-echelon elimination with
 * row interchanges (independent of CUP): product of the pivots times the sign
 * of the row permutation. */
u32 cupo_det(const u32 *A, i64 n, i64 lda, u32 p)
{
    u32 *W = (u32 *)malloc((size_t)(n > 0 ? n : 1) * (size_t)(n > 0 ? n : 1) * sizeof(u32));
    for (i64 i = 0; i < n; ++i) memcpy(W + i * n, A + i * lda, (size_t)n * sizeof(u32));
    u32 det = 1 % p;
    for (i64 c = 0; c < n; ++c) {
        i64 piv = -1;
        for (i64 i = c; i < n; ++i) if (W[i * n + c]) { piv = i; break; }
        if (piv < 0) { det = 0; break; }
        if (piv != c) {
            for (i64 j = 0; j < n; ++j) { u32 t = W[c * n + j]; W[c * n + j] = W[piv * n + j]; W[piv * n + j] = t; }
            det = subm(0, det, p);
        }
        det = mulm(det, W[c * n + c], p);
        u32 inv = cupo_modinv(W[c * n + c], p);
#pragma omp parallel for schedule(static)
        for (i64 i = c + 1; i < n; ++i) {
            u32 f = mulm(W[i * n + c], inv, p);
            if (!f) continue;
            for (i64 j = c; j < n; ++j) W[i * n + j] = subm(W[i * n + j], mulm(f, W[c * n + j], p), p);
        }
    }
    free(W);
    return det;
}

/* Inverse of an n x n matrix by Gauss-Jordan elimination on [A | I] with row
 * interchanges. Returns 0 and writes Ainv on success, 1 if A is singular. */
int cupo_inverse(const u32 *A, i64 n, i64 lda, u32 p, u32 *Ainv, i64 ldi)
{
    i64 w = 2 * n;
    u32 *W = (u32 *)malloc((size_t)(n > 0 ? n : 1) * (size_t)(w > 0 ? w : 1) * sizeof(u32));
    for (i64 i = 0; i < n; ++i) {
        memcpy(W + i * w, A + i * lda, (size_t)n * sizeof(u32));
        for (i64 j = 0; j < n; ++j) W[i * w + n + j] = (i == j) ? 1u % p : 0u;
    }
    int singular = 0;
    for (i64 c = 0; c < n; ++c) {
        i64 piv = -1;
        for (i64 i = c; i < n; ++i) if (W[i * w + c]) { piv = i; break; }
        if (piv < 0) { singular = 1; break; }
        if (piv != c)
            for (i64 j = 0; j < w; ++j) { u32 t = W[c * w + j]; W[c * w + j] = W[piv * w + j]; W[piv * w + j] = t; }
        u32 inv = cupo_modinv(W[c * w + c], p);
        for (i64 j = 0; j < w; ++j) W[c * w + j] = mulm(W[c * w + j], inv, p);
#pragma omp parallel for schedule(static)
        for (i64 i = 0; i < n; ++i) {
            if (i == c) continue;
            u32 f = W[i * w + c];
            if (!f) continue;
            for (i64 j = 0; j < w; ++j) W[i * w + j] = subm(W[i * w + j], mulm(f, W[c * w + j], p), p);
        }
    }
    if (!singular)
        for (i64 i = 0; i < n; ++i) memcpy(Ainv + i * ldi, W + i * w + n, (size_t)n * sizeof(u32));
    free(W);
    return singular;
}

/*
 * Particular solution of A x = B (A m x n, B m x k, X n x k) whose entries
 * outside the pivot columns of the CUP decomposition are zero (Sec. 4.4 lists
 * system solving among the problems reduced to CUP; the paper does not fix a
 * particular solution, this choice is the one a CUP-based solver produces).
 * The pivot column set S is read from `ipiv` (r transpositions, as returned by
 * cupo_cup); the columns A[:, S] are independent, so the solution supported
 * on S is unique when it exists. It is found by row-echelon elimination on
 * [A[:, S] | B] with row interchanges and back substitution.
 * Returns 0 on success, 2 if the system has no solution.
 */
int cupo_solve(const u32 *A, i64 m, i64 n, i64 lda, const u32 *B, i64 k, i64 ldb,
               const i64 *ipiv, i64 r, u32 p, u32 *X, i64 ldx)
{
    i64 *perm = (i64 *)malloc((size_t)(n > 0 ? n : 1) * sizeof(i64));
    for (i64 j = 0; j < n; ++j) perm[j] = j;
    for (i64 t = 0; t < r; ++t) { i64 c = ipiv[t]; i64 x = perm[t]; perm[t] = perm[c]; perm[c] = x; }
    i64 w = r + k;
    u32 *W = (u32 *)malloc((size_t)(m > 0 ? m : 1) * (size_t)(w > 0 ? w : 1) * sizeof(u32));
    for (i64 i = 0; i < m; ++i) {
        for (i64 t = 0; t < r; ++t) W[i * w + t] = A[i * lda + perm[t]];
        for (i64 j = 0; j < k; ++j) W[i * w + r + j] = B[i * ldb + j];
    }
    int status = 0;
    for (i64 c = 0; c < r; ++c) {
        i64 piv = -1;
        for (i64 i = c; i < m; ++i) if (W[i * w + c]) { piv = i; break; }
        if (piv < 0) { status = 3; break; }   /* cannot happen: columns independent */
        if (piv != c)
            for (i64 j = 0; j < w; ++j) { u32 t = W[c * w + j]; W[c * w + j] = W[piv * w + j]; W[piv * w + j] = t; }
        u32 inv = cupo_modinv(W[c * w + c], p);
        for (i64 j = 0; j < w; ++j) W[c * w + j] = mulm(W[c * w + j], inv, p);
        for (i64 i = 0; i < m; ++i) {
            if (i == c) continue;
            u32 f = W[i * w + c];
            if (!f) continue;
            for (i64 j = 0; j < w; ++j) W[i * w + j] = subm(W[i * w + j], mulm(f, W[c * w + j], p), p);
        }
    }
    if (status == 0)
        for (i64 i = r; i < m && status == 0; ++i)
            for (i64 j = 0; j < k; ++j)
                if (W[i * w + r + j]) { status = 2; break; }
    if (status == 0) {
        for (i64 j = 0; j < n; ++j)
            for (i64 l = 0; l < k; ++l) X[j * ldx + l] = 0;
        for (i64 t = 0; t < r; ++t)
            for (i64 l = 0; l < k; ++l) X[perm[t] * ldx + l] = W[t * w + r + l];
    }
    free(W);
    free(perm);
    return status;
}

/* Field-operation count of the iterative elimination in cupo_cup for a
 * matrix with the given profile (Sec. 4.2 counts multiplications, additions,
 * inversions and comparisons with zero alike): per pivot t at row i_t, one
 * inversion, n-t-1 multiplications for U's row, and two operations per entry
 * of the (m-i_t-1) x (n-t-1) trailing update. Zero tests are not counted. */
double cupo_opcount(i64 m, i64 n, const i64 *profile, i64 r)
{
    double ops = 0.0;
    for (i64 t = 0; t < r; ++t) {
        double rows = (double)(m - profile[t] - 1), cols = (double)(n - t - 1);
        ops += 1.0 + cols + 2.0 * rows * cols;
    }
    return ops;
}
