/*
 * cup_gb300.h — C ABI of the GB300 (sm_103a) CUP library over prime fields.
 *
 * The library computes the rank-profile revealing CUP decomposition of
 * Jeannerod, Pernet and Storjohann ("Rank-profile revealing Gaussian
 * elimination and the CUP matrix decomposition") and the problems the paper
 * reduces to it, over GF(p) for a prime p < 2^31, with hand-written CUDA
 * kernels on one GPU.
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Matrices are caller-owned DEVICE buffers of uint32 residues in [0, p),
 *   row-major with a leading dimension ld >= number of columns (zero-based
 *   indices and half-open ranges, Sec. 1.1). The library never frees them.
 *   The *_u8 entry points take one-byte residues for p < 2^8 instead.
 * - Index outputs (rank profile, pivots) are caller-owned DEVICE int64 arrays.
 * - Scalars returned through plain pointers (rank, determinant) are HOST
 *   pointers; a call that returns one synchronises `stream` before returning.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream). Work is enqueued on it; buffers must stay valid until it drains.
 * - The handle owns all temporary device memory (the pivot-phase scratch of
 *   the base case, the transposition lists and the 8-bit limb planes of the
 *   tensor-core products), as Definition 1 allows for matrix products. Calls on
 *   one handle must not overlap: use one handle per concurrent stream.
 * - Nothing throws across the ABI; every call returns a cup_status. On an
 *   error the contents of output buffers are unspecified, except that
 *   CUP_SINGULAR from cup_inverse leaves A holding the [C\U] factors.
 */
#ifndef CUP_GB300_H
#define CUP_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CUP_OK = 0,
    CUP_SINGULAR = 1,          /* square input of rank < n (cup_inverse) */
    CUP_INCONSISTENT = 2,      /* cup_solve: the right-hand side is not in the column space */
    CUP_ERR_ARG = -1,          /* bad size, leading dimension, null pointer or option */
    CUP_ERR_PRIME = -2,        /* p is not a prime below 2^31 */
    CUP_ERR_VALUE = -3,        /* an entry >= p (only checked when validation is on) */
    CUP_ERR_CUDA = -4,         /* a CUDA call failed (see cup_last_cuda_error) */
    CUP_ERR_TIMEOUT = -5,      /* a bounded device-side wait expired */
    CUP_ERR_NOMEM = -6,        /* workspace allocation failed */
    CUP_ERR_UNSUPPORTED = -7,  /* valid request the library does not serve */
    CUP_ERR_TOO_LARGE = -8     /* cup_mm_sub_noalloc: the product needs more scratch than it has */
} cup_status;

typedef struct cup_handle cup_handle;

/* Engine used for the Schur update C <- C - A B mod p (Algorithm 1 with
 * alpha = -1, beta = 1, Sec. 3.2): */
enum {
    CUP_ENGINE_PLAIN = 0,      /* CUDA-core 64-bit integer multiply and reduce */
    CUP_ENGINE_TENSOR = 1      /* tcgen05 tensor cores on exact 8-bit limbs */
};

/* Options for cup_set_option. */
enum {
    CUP_OPT_ENGINE = 0,        /* CUP_ENGINE_PLAIN or CUP_ENGINE_TENSOR (default TENSOR) */
    CUP_OPT_LEAF_ROWS = 1,     /* rows of a base-case slab, 1..64 (default 64) */
    CUP_OPT_WINDOW = 2,        /* pivot-search window of the base case, 1..128 (default 96) */
    CUP_OPT_TC_MIN_K = 3,      /* smallest inner dimension sent to the tensor engine (default 64) */
    CUP_OPT_VALIDATE = 4,      /* nonzero: check inputs are canonical residues (slow) */
    CUP_OPT_PROFILE = 5,       /* 1: time every Schur-update launch with CUDA events; 2: every launch */
    CUP_OPT_SCHEDULE = 6,      /* cup_factor schedule: 1 (default) device-resident, replayed as a CUDA
                                  graph when a call repeats; 2 device-resident without graphs; 0 host-driven
                                  (reads each block's rank back before launching the next) */
    CUP_OPT_INT_PATH = 7,      /* images of cup_int_det / cup_int_rank: 0 (default) by a cost model,
                                  1 the batched launch (min(m, n) <= 2048), 2 one full-device CUP per prime */
    CUP_OPT_SHORT_K = 8        /* tensor-engine Schur updates with K at most this (0..256, default 128),
                                  p < 2^24 and at most 2^21 entries of C run as one launch of
                                  mma.sync digit products formed in shared memory instead of a digit
                                  split plus a tcgen05 launch; 0 sends every update to tcgen05 */
};

/* Counters of the work a handle has enqueued since the last cup_reset_stats.
 * Device times are filled only while CUP_OPT_PROFILE is on; they are CUDA
 * event intervals recorded on the launch stream around each Schur-update
 * kernel and read after the call that launched it synchronised. */
typedef struct {
    int64_t launches;          /* kernels launched by the library */
    int64_t host_syncs;        /* stream synchronisations made by the host driver */
    int64_t tc_launches;       /* tcgen05 Schur-update kernels */
    double tc_ms;              /* their summed device time */
    double tc_limb_flops;      /* 2 L^2 M N K over those launches (bf16 tensor-core work) */
    double tc_field_flops;     /* 2 M N K over those launches (field multiply + add) */
    int64_t cc_launches;       /* CUDA-core Schur-update kernels */
    double cc_ms;
    double cc_field_flops;
    double tc_alg_bytes;       /* algorithmic HBM bytes of the tcgen05 launches: limb planes read
                                  (2 L (M + N) K) plus C read and written (8 M N), summed */
    int64_t sk_launches;       /* short-K tensor updates (CUP_OPT_SHORT_K) */
    double sk_ms;              /* their summed device time */
    double sk_field_flops;     /* 2 M N K over those launches */
} cup_stats;

/* Create a handle bound to CUDA device `device` (the device is made current
 * for the duration of each call). */
cup_status cup_create(cup_handle **handle, int device);

/* Release a handle and all its workspace. */
cup_status cup_destroy(cup_handle *handle);

/* Set an option (see the CUP_OPT_* list). */
cup_status cup_set_option(cup_handle *handle, int option, int64_t value);

/* Tuning table of the schedule options (no counterpart in the paper: the
 * recursion's leaf size, the base case's pivot window and the smallest inner
 * dimension sent to the tensor engine only change how fast a factorization
 * runs, never its result). `table` is JSON text {"entries": [rule, ...]}; each
 * rule is an object with numeric fields: the keys "limbs" (1..4, the tensor
 * engine's limb count of p), "tall" (1: m >= 2n, 0: otherwise), "min_lo" and
 * "min_hi" (min(m, n) in [min_lo, min_hi)) select calls (an absent key matches
 * every call), and "leaf_rows", "window", "tc_min_k" give the options. Each
 * factorization (cup_factor and every call built on it) takes the first rule
 * that matches; options set with cup_set_option take precedence. Other keys
 * (timings, notes) are ignored. NULL clears the table. The text is parsed and
 * copied: CUP_ERR_ARG if it is malformed (the previous table is kept). The
 * tuner paper_1112_5717_gb300/tune.py writes such a table from measured times. */
cup_status cup_set_tuning(cup_handle *handle, const char *table);

/* Text of the last CUDA error seen by this handle (static storage). */
const char *cup_last_cuda_error(cup_handle *handle);

/*
 * CUP decomposition in place (Algorithm 6, Sec. 3.3; Ensures: A <- [C\U]).
 *   A        m x n device matrix (lda), overwritten by the space-sharing
 *            storage [C\U] of Sec. 3.1: rows 0..r-1 hold U strictly above the
 *            diagonal (U is unit upper triangular, its diagonal implicit); C's
 *            first r columns are stored on and below the diagonal; all other
 *            entries are zero. A P^T = C U with U embedded in an n x n unit
 *            upper triangular matrix.
 *   d_profile device int64[min(m,n)]: entries 0..r-1 receive the row rank
 *            profile i_0 < ... < i_{r-1} (Sec. 2).
 *   d_ipiv   device int64[min(m,n)]: entries 0..r-1 receive the column
 *            transpositions, LAPACK style: P = T_{r-1,ipiv[r-1]} ... T_{0,ipiv[0]},
 *            i.e. A P^T applies the swaps (t, ipiv[t]) to columns for
 *            t = 0, 1, ..., r-1 in order, with ipiv[t] >= t.
 *   rank     host int64*: receives r (the call synchronises `stream`).
 * The pivot of each row is the first nonzero of its residual at a position
 * >= the current rank, transposed with that position (the rule of
 * Algorithm 6's base case), so C, U and P are those that rule defines.
 */
cup_status cup_factor(cup_handle *handle, uint32_t *A, int64_t m, int64_t n, int64_t lda,
                      uint32_t p, int64_t *d_profile, int64_t *d_ipiv, int64_t *rank,
                      void *stream);

/* cup_factor with the input and the result in HOST memory: hA (m x n, leading
 * dimension ldh, ideally page-locked) is factored, [C\U] is written to hOut (may
 * equal hA), and A (DEVICE, m x n, lda) is the working copy, holding [C\U] too on
 * return; d_profile, d_ipiv and *rank as in cup_factor. The input is copied in row
 * chunks (one leaf, one leaf, then doubling) on a second stream, and the
 * factorization waits for a chunk only when it first reaches its rows, so the
 * copy overlaps the elimination of the rows above it; the copy back starts when
 * the factorization ends. Repeated calls with the same buffers on a non-default
 * stream are replayed as one CUDA graph, copies included. Synchronises `stream`. */
cup_status cup_factor_host(cup_handle *handle, const uint32_t *hA, int64_t ldh, uint32_t *hOut, uint32_t *A,
                           int64_t m, int64_t n, int64_t lda, uint32_t p, int64_t *d_profile, int64_t *d_ipiv,
                           int64_t *rank, void *stream);

/* ---- One-byte residue storage (p < 2^8) ----
 * The same operations for matrices stored as uint8 residues in [0, p), row-major
 * with leading dimension lda (in entries, i.e. bytes), for a prime p below 2^8
 * (CUP_ERR_ARG otherwise). The matrix keeps its one-byte storage at the
 * boundary and in the caller's buffers: the call widens it into a uint32 working
 * copy owned by the handle (4 m n bytes, kept for later calls), runs the uint32
 * path on it, and narrows the result (residues below p fit a byte) back into A.
 * Outputs, pivots, profile and rank are those of the uint32 calls on the same
 * values. Each call synchronises `stream` before returning. */

/* cup_factor on a one-byte matrix: A <- [C\U] (Algorithm 6). */
cup_status cup_factor_u8(cup_handle *handle, uint8_t *A, int64_t m, int64_t n, int64_t lda, uint32_t p,
                         int64_t *d_profile, int64_t *d_ipiv, int64_t *rank, void *stream);

/* cup_factor_host on a one-byte matrix: hA (HOST, m x n, ldh bytes a row) is
 * copied in row chunks into A (DEVICE bytes, lda), each chunk widened on the
 * copy stream as it lands, so the copies overlap the elimination; the result is
 * narrowed into A and copied to hOut (may equal hA). Moves m n bytes each way. */
cup_status cup_factor_host_u8(cup_handle *handle, const uint8_t *hA, int64_t ldh, uint8_t *hOut, uint8_t *A,
                              int64_t m, int64_t n, int64_t lda, uint32_t p, int64_t *d_profile, int64_t *d_ipiv,
                              int64_t *rank, void *stream);

/* cup_det on a one-byte square matrix (A receives the [C\U] factors). */
cup_status cup_det_u8(cup_handle *handle, uint8_t *A, int64_t n, int64_t lda, uint32_t p, uint32_t *det,
                      void *stream);

/* cup_inverse on a one-byte square matrix: A <- A^{-1} (Algorithm 8), or
 * CUP_SINGULAR with A holding the [C\U] factors. */
cup_status cup_inverse_u8(cup_handle *handle, uint8_t *A, int64_t n, int64_t lda, uint32_t p, void *stream);

/*
 * Rank and row rank profile (Sec. 2; Prop. 3). A is destroyed (it receives
 * the [C\U] factors). d_profile as in cup_factor.
 */
cup_status cup_rank_profile(cup_handle *handle, uint32_t *A, int64_t m, int64_t n, int64_t lda,
                            uint32_t p, int64_t *d_profile, int64_t *rank, void *stream);

/*
 * Determinant of a square matrix (Sec. 4.4: CUP suffices). A is destroyed.
 * *det receives det(A) mod p: 0 if the rank is below n, otherwise the
 * product of C's diagonal (the pivots) times (-1)^(number of nontrivial
 * transpositions).
 */
cup_status cup_det(cup_handle *handle, uint32_t *A, int64_t n, int64_t lda, uint32_t p,
                   uint32_t *det, void *stream);

/*
 * In-place inverse of a square matrix (Algorithm 8 via Algorithm 7 and the
 * TRSM/TRTRI/TRULM building blocks, Sec. 3.4, 3.5 and 4.3). On success A
 * holds A^{-1}. Returns CUP_SINGULAR (A holds the [C\U] factors) if the rank
 * is below n.
 */
cup_status cup_inverse(cup_handle *handle, uint32_t *A, int64_t n, int64_t lda, uint32_t p,
                       void *stream);

/*
 * Reduced column echelon form (Proposition 1, Algorithm 8): A (m x n) is
 * overwritten by R, the unique reduced column echelon form of A (columns
 * >= r zero). d_profile as in cup_factor. If X is not NULL it is an n x n
 * device matrix (ldx) that receives the transform with A X = R
 * (X = P^T [X1 X2; 0 I] of Algorithm 8, unique given P).
 */
cup_status cup_rref(cup_handle *handle, uint32_t *A, int64_t m, int64_t n, int64_t lda, uint32_t p,
                    int64_t *d_profile, int64_t *rank, uint32_t *X, int64_t ldx, void *stream);

/*
 * PLE decomposition (Sec. 5, Algorithm 10): the row echelon twin of CUP. A (m x n)
 * is overwritten by [L\E] such that A = P L E, where E (r x n, rows 0 .. r-1 of A,
 * on and right of each row's first nonzero) is in row echelon form revealing the
 * column rank profile, L (m x r, strictly below the diagonal of A's first r
 * columns) is unit lower triangular, and P is a row permutation stored as
 * transpositions: exchanging rows t and d_ipiv[t] of the input, in order
 * t = 0 .. r-1, gives L E (so A = P L E). d_profile receives the column rank
 * profile. (E^T, L^T, P^T) is the CUP decomposition of
 * A^T that cup_factor computes, and this is how it is computed: CUP of a
 * transposed copy (m n uint32 of scratch owned by the call), transposed back.
 */
cup_status cup_ple(cup_handle *handle, uint32_t *A, int64_t m, int64_t n, int64_t lda, uint32_t p,
                   int64_t *d_profile, int64_t *d_ipiv, int64_t *rank, void *stream);

/*
 * Basis of the right nullspace {x : A x = 0} (the echelon transform of Sec. 3.4
 * and 3.5 gives it, Sec. 4.4): with A X = R for the transform X of cup_rref,
 * R's columns r .. n-1 are zero, so X's columns r .. n-1 are a basis. A (m x n)
 * is destroyed (it holds the CUP factors and the echelon work). Nb is a
 * caller-owned n x ldn device matrix, ldn >= n: on success its first n - r
 * columns hold the basis P^T [X2; I_{n-r}] (its other columns are untouched)
 * and *rank = r. n - r = 0 writes nothing.
 */
cup_status cup_nullspace(cup_handle *handle, uint32_t *A, int64_t m, int64_t n, int64_t lda, uint32_t p,
                         uint32_t *Nb, int64_t ldn, int64_t *rank, void *stream);

/*
 * Linear system A X = B (Sec. 4.4: solving reduces to CUP). A (m x n) is
 * destroyed; B (m x k, ldb) is read and destroyed; X (n x k, ldx) receives
 * the solution whose entries outside the CUP pivot columns are zero
 * (x = P^T [U1^{-1} L1^{-1} b_profile; 0]). Returns CUP_INCONSISTENT when no
 * solution exists. *rank receives r.
 */
cup_status cup_solve(cup_handle *handle, uint32_t *A, int64_t m, int64_t n, int64_t lda,
                     uint32_t *B, int64_t k, int64_t ldb, uint32_t *X, int64_t ldx, uint32_t p,
                     int64_t *rank, void *stream);

/* Read (and keep) the counters of a handle. */
cup_status cup_get_stats(cup_handle *handle, cup_stats *out);

/* Device time per kernel class, filled while CUP_OPT_PROFILE >= 2 (every
 * launch bracketed by events): out8[0] tensor-core Schur update, [1]
 * CUDA-core Schur update, [2] base-case pivot kernel, [3] base-case finish
 * kernel, [4] TRSM leaf, [5] column transpositions, [6..7] unused. */
cup_status cup_class_ms(cup_handle *handle, double *out8);

/* Zero the counters of a handle. */
cup_status cup_reset_stats(cup_handle *handle);

/* One matrix of a batched call (all pointers are DEVICE pointers). */
typedef struct {
    uint32_t *A;           /* m x n row-major (lda), residues in [0, p); receives [C\U] */
    int64_t m, n, lda;
    uint32_t p;            /* this matrix's prime, below 2^31 */
    uint32_t reserved;
    int64_t *profile;      /* min(m, n) entries: row rank profile (first rank valid) */
    int64_t *ipiv;         /* min(m, n) entries: column transpositions as in cup_factor */
} cup_batch_item;

/*
 * Batched CUP (Algorithm 6's output for each matrix, as cup_factor) of
 * `count` independent matrices, each over its own prime field, in one
 * persistent launch (one CTA per SM, each factoring one matrix at a time,
 * the largest first); nothing is read back to the host, so the call is
 * asynchronous. A repeated call with the same arguments on a stream other
 * than the legacy default stream replays one CUDA graph (the items are read
 * when it runs, so their contents may change between calls). Matrices with
 * min(m, n) <= 2048 are supported; those with at most 1024 columns are
 * factored in 32-row panels held in shared memory.
 *   d_items  device array of `count` items.
 *   d_rank   device int64[count]: the rank of each matrix, or -1 if its item
 *            was invalid (bad sizes or pointers, p not a prime below 2^31,
 *            min(m, n) > 2048).
 *   d_det    device uint32[count] or NULL: det(A) mod p for square matrices
 *            (0 when singular or not square).
 */
cup_status cup_factor_batched(cup_handle *handle, const cup_batch_item *d_items, int64_t count,
                              int64_t *d_rank, uint32_t *d_det, void *stream);

/* ---- Integer matrices by multi-modular reduction (Sec. 1: computations over
 * Z reduce to linear algebra over prime fields by homomorphic imaging) ----
 * The integer matrix is reduced modulo several primes on the device, each
 * image is factored by CUP (Algorithm 6; the batched launch for images with
 * min(m, n) <= 512, one full-device factorisation per prime otherwise), and
 * the residues are combined on the host by the Chinese remainder theorem.
 * A is a DEVICE int64 matrix, row-major with leading dimension lda >= n;
 * `primes` is a HOST array of K distinct primes below 2^31, or NULL to let
 * the library take the largest primes below 2^31, as many as the bound
 * requires. Integer results are returned as a sign (-1, 0, 1) and the
 * magnitude in little-endian 32-bit words. All calls synchronise the stream. */

/* log2 of the product of the Euclidean norms of the nonzero rows of A (m x n):
 * bounds |det A| (Hadamard's inequality) and every minor of A. */
cup_status cup_int_bound(cup_handle *handle, const int64_t *A, int64_t m, int64_t n, int64_t lda,
                         double *log2_bound, void *stream);

/* det A for square integer A (n x n). *sign and words[0 .. *nwords) receive
 * the integer congruent to det A modulo the product M of the primes used, in
 * (-M/2, M/2]; *certified is 1 when M > 2 * (Hadamard bound), so that this is
 * det A exactly. *rank receives the largest rank over the primes (a lower
 * bound on the rank over Q, exact when certified) and *nprimes (if not NULL)
 * the number of primes used. Returns CUP_ERR_TOO_LARGE, with *nwords set, when
 * cap words are too few (size cap from cup_int_bound: ceil((bound + 1) / 32) + 1
 * always suffices for a certified result). */
cup_status cup_int_det(cup_handle *handle, const int64_t *A, int64_t n, int64_t lda, const uint32_t *primes,
                       int64_t K, uint32_t *words, int64_t cap, int64_t *nwords, int *sign, int64_t *rank,
                       int *certified, int64_t *nprimes, void *stream);

/* rank over Q of the integer matrix A (m x n): the largest rank of its images.
 * *certified is 1 when the product of the primes exceeds the minor bound of
 * cup_int_bound: then no nonzero maximal minor vanishes modulo all of them,
 * so the rank is exact. */
cup_status cup_int_rank(cup_handle *handle, const int64_t *A, int64_t m, int64_t n, int64_t lda,
                        const uint32_t *primes, int64_t K, int64_t *rank, int *certified, int64_t *nprimes,
                        void *stream);

/* Host only. The integer x with x = residues[i] (mod primes[i]) for all i < K,
 * in the symmetric range (-M/2, M/2] of M = product of the primes (mixed-radix
 * Chinese remaindering). Primes must be distinct primes below 2^31
 * (CUP_ERR_PRIME / CUP_ERR_ARG otherwise); CUP_ERR_TOO_LARGE with *nwords set
 * when cap words are too few. */
cup_status cup_crt(const uint32_t *residues, const uint32_t *primes, int64_t K, uint32_t *words, int64_t cap,
                   int64_t *nwords, int *sign);

/* Host only. The `count` largest primes below `bound`, descending, into out;
 * *found receives how many exist (fewer when bound is small). */
cup_status cup_primes_below(uint32_t bound, int64_t count, uint32_t *out, int64_t *found);

/* ---- Building blocks of the hot path (exposed for testing and reuse) ---- */

/* Schur update (Algorithm 1, alpha = -1, beta = 1): C <- C - A B mod p.
 * A is M x K (lda), B is K x N (ldb), C is M x N (ldc); C must not overlap A
 * or B. `engine` selects CUP_ENGINE_PLAIN or CUP_ENGINE_TENSOR. */
cup_status cup_mm_sub(cup_handle *handle, uint32_t *C, int64_t ldc, const uint32_t *A, int64_t lda,
                      const uint32_t *B, int64_t ldb, int64_t M, int64_t N, int64_t K, uint32_t p,
                      int engine, void *stream);

/* TRSM(Right, Upper, Unit) (Algorithm 2, unit-diagonal variant, as used by
 * Algorithm 6's TRSM step): B <- B U^{-1}. U is n x n (ldu); only its strict
 * upper triangle is read. B is m x n (ldb). */
cup_status cup_trsm_ruu(cup_handle *handle, const uint32_t *U, int64_t ldu, uint32_t *B,
                        int64_t ldb, int64_t m, int64_t n, uint32_t p, void *stream);

/* Triangle selection for cup_trsm / cup_trmm / cup_trtri (bit flags). */
enum {
    CUP_LEFT = 1,              /* set: B <- op(T) B; clear: B <- B op(T) */
    CUP_UPPER = 2,             /* set: T upper triangular; clear: lower */
    CUP_UNIT = 4               /* set: unit diagonal (the stored diagonal is not read) */
};

/* TRSM in any of its eight variants (Sec. 3.2; Algorithm 2 is Right, Upper,
 * NonUnit): B <- T^{-1} B (CUP_LEFT) or B <- B T^{-1}. T is n x n (ldt), only
 * its selected triangle (and diagonal unless CUP_UNIT) is read; n = rows of B
 * for CUP_LEFT, columns of B otherwise. B is rows x cols (ldb), overwritten. */
cup_status cup_trsm(cup_handle *handle, int flags, const uint32_t *T, int64_t ldt, uint32_t *B,
                    int64_t ldb, int64_t rows, int64_t cols, uint32_t p, void *stream);

/* TRMM (Sec. 3.2, same eight variants): B <- T B (CUP_LEFT) or B <- B T. */
cup_status cup_trmm(cup_handle *handle, int flags, const uint32_t *T, int64_t ldt, uint32_t *B,
                    int64_t ldb, int64_t rows, int64_t cols, uint32_t p, void *stream);

/* TRTRI (Algorithm 3 and its variants): T <- T^{-1} in place for an n x n
 * triangle selected by CUP_UPPER / CUP_UNIT (CUP_LEFT ignored); entries outside
 * the triangle (and the diagonal when CUP_UNIT) are not touched. The diagonal
 * of a non-unit triangle must be nonzero. */
cup_status cup_trtri(cup_handle *handle, int flags, uint32_t *T, int64_t ldt, int64_t n, uint32_t p,
                     void *stream);

/* TRULM (Algorithm 4): A = [L\U] n x n with U unit upper triangular stored
 * strictly above the diagonal and L lower triangular stored on and below it;
 * A <- U L in place. */
cup_status cup_trulm(cup_handle *handle, uint32_t *A, int64_t lda, int64_t n, uint32_t p, void *stream);

/* TRLUM (Algorithm 5): A = [L\U] n x n with L unit lower triangular stored
 * strictly below the diagonal and U upper triangular stored on and above it;
 * A <- L U in place (the product of LU factors, e.g. to rebuild a matrix). */
cup_status cup_trlum(cup_handle *handle, uint32_t *A, int64_t lda, int64_t n, uint32_t p, void *stream);

/* InPlaceMM (Algorithm 9): B <- A B for A m x m (leading dimension lda >= m) and
 * B m x n (ldb >= n), row-major device buffers, without an m x n temporary.
 * A is factored in place by CUP (A = C U P), B is multiplied by P, U and C in
 * turn (two TRMMs), and A is rebuilt as (C U) P through TRLUM with the unit
 * diagonal on U; on CUP_OK A holds its original entries again. A may be
 * singular: the zero blocks of [C\U] storage make the same steps exact.
 * *rank receives rank(A). Stream-ordered; returns after the work is queued and
 * the device error word is checked (one synchronisation). A and B must not
 * overlap. Allocates 2 m int64 words of scratch for the permutation. */
cup_status cup_inplace_mm(cup_handle *handle, uint32_t *A, int64_t m, int64_t lda, uint32_t *B, int64_t n,
                          int64_t ldb, uint32_t p, int64_t *rank, void *stream);

/* Allocation-free Schur update: C <- C - A B mod p on the tensor engine,
 * like cup_mm_sub with CUP_ENGINE_TENSOR, for callers that cannot call
 * cudaMalloc: a process whose device memory is all reserved up front by its
 * own fixed-size pool (a further cudaMalloc would fail, or would take memory
 * the pool has promised elsewhere), code that has given up allocation after
 * start-up (cudaMalloc and cudaFree may synchronise the whole device, which a
 * latency-bound loop sharing the GPU with other streams cannot afford), or a
 * host whose rules forbid dynamic allocation outside initialisation. The
 * paper has no counterpart: this is a packaging choice.
 *   - No handle and no allocation: the 8-bit limb planes live in one fixed
 *     scratch array of 16 MiB that the library holds on every GPU where it
 *     is loaded, until the process exits. A product needs
 *     L * (M + N) * roundup(K, 64) * 2 bytes of it (L = 1, 2, 3, 4 limbs for
 *     p below 2^8, 2^16, 2^24, 2^31); larger products return
 *     CUP_ERR_TOO_LARGE without touching C. The call allocates nothing itself
 *     and calls no allocating library routine.
 *   - Runs on the current CUDA device. The first call on each device does the
 *     set-up, with that device current: it looks up the scratch array's device
 *     address (cudaGetSymbolAddress) and raises the kernel's shared-memory
 *     limit on that device. Make that first call before any stream capture.
 *   - Every call on a device shares the one scratch array and its error word:
 *     calls that can overlap on the GPU (different streams, or several host
 *     threads) race and must be serialised by the caller. Each call rewrites
 *     the part of the scratch it reads and clears the error word first.
 *   - Synchronises `stream` before returning; CUP_ERR_TIMEOUT if a bounded
 *     device-side wait expired. Arguments as for cup_mm_sub. */
cup_status cup_mm_sub_noalloc(uint32_t *C, int64_t ldc, const uint32_t *A, int64_t lda,
                              const uint32_t *B, int64_t ldb, int64_t M, int64_t N, int64_t K,
                              uint32_t p, void *stream);

/* Self-test of failure detection (no counterpart in the paper): one device
 * thread waits, with the same bounded wait the tensor-core kernels use, on an
 * mbarrier that nothing arrives at. After limit_us microseconds (1 .. 10^7)
 * the wait gives up, records its site in the handle's device error word and
 * the kernel returns; the call then reads the word like every other call and
 * returns CUP_ERR_TIMEOUT with "device wait expired (site 99)" in
 * cup_last_cuda_error. The word is cleared again, so the handle and the CUDA
 * context stay usable. Synchronises `stream`. */
cup_status cup_selftest_wait(cup_handle *handle, int64_t limit_us, void *stream);

/* Peak-rate probe of a tensor instruction on CUDA device `device` (no
 * counterpart in the paper: it measures the exact-integer tensor paths the
 * library could use, to justify the choice of engine). Every SM runs `iters`
 * iterations of back-to-back instructions on operands held in registers or
 * shared memory; *tflops receives the rate in 10^12 operations per second
 * (a multiply and an add count as two), from CUDA events around the launch
 * after a shorter warm-up launch. kind 0: mma.sync m16n8k32 s8 x s8 -> s32;
 * 1: mma.sync m16n8k16 bf16 -> f32; 2: tcgen05.mma kind::f16 with M = 128,
 * N = 256, bf16 operands in shared memory and the fp32 accumulator in TMEM
 * (the instruction of the tensor engine). Allocates and frees a few bytes;
 * synchronises the device's work it launched. CUP_ERR_TIMEOUT if the bounded
 * wait for the tcgen05 instructions expired. */
cup_status cup_probe_tensor_peak(int device, int kind, int64_t iters, double *tflops);

/* Column transpositions (Sec. 1.1): for t = k0..k1-1 in order, swap columns t
 * and d_ipiv[t] of rows row0..row0+nrows-1 of A (A <- A P^T restricted to
 * those transpositions). d_ipiv is a device array indexed by absolute
 * position. */
cup_status cup_laswp_cols(cup_handle *handle, uint32_t *A, int64_t lda, int64_t row0,
                          int64_t nrows, const int64_t *d_ipiv, int64_t k0, int64_t k1,
                          void *stream);

#ifdef __cplusplus
}
#endif
#endif /* CUP_GB300_H */
