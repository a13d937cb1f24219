// Host driver and C ABI of the CUP library (declared in include/cup_gb300.h).
//
// cup_factor follows the row-recursive structure of Algorithm 6 (Sec. 3.3):
// split the rows, factor the top block (rec1), transpose the bottom block's
// columns (A2 <- A2 P1^T), TRSM(Right, Upper, Unit) on its first r1 columns,
// Schur update H <- A22 - G V1, factor H (rec2), transpose V1's columns
// (V1 <- V1 P2^T). The leaves are slabs of at most CUP_BMAX rows factored by
// the base-case kernels. Differences from the printed algorithm, all of which
// leave C, U, P, the rank and the profile unchanged:
//   * U's rows are written by the leaves straight to their final rows of the
//     [C\U] storage (global rows col0..col0+r-1, where col0 is the rank of
//     the rows above), so the row-move loop of Algorithm 6 is not needed;
//   * the split point is aligned to the leaf size instead of floor(m/2), and a
//     leaf may split itself again where its pivot window runs out (any split
//     point yields the same decomposition);
//   * P and the rank profile are stored with absolute indices as they are
//     found, so P <- Diag(I_r1, P2) P1 and the profile offsets need no work.
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <new>
#include <string>
#include <vector>
#include "cup_internal.cuh"
#include "../../include/cup_gb300.h"

struct cup_handle {
    int device = 0;
    int engine = CUP_ENGINE_TENSOR;
    int leaf_rows = 64;
    int window = 96;
    int64_t tc_min_k = 64;
    int64_t short_k = 128;          // largest K of the one-launch short-K tensor update (0: never;
                                    // K = 256 is supported but measured slower than tcgen05 there)
    bool user_set[3] = {false, false, false};   // leaf_rows, window, tc_min_k set by cup_set_option
    struct TuneRule {
        int64_t limbs = -1, tall = -1, min_lo = 0, min_hi = INT64_MAX;
        int64_t leaf_rows = 0, window = 0, tc_min_k = 0;
    };
    std::vector<TuneRule> tuning;  // from cup_set_tuning: the first matching rule applies
    int validate = 0;
    SlabScratch *d_slab = nullptr;
    int2 *d_pairs = nullptr;
    int64_t pairs_cap = 0;
    int *d_count = nullptr;
    int *h_pinned = nullptr;
    int *d_err = nullptr;          // device-side error word of the tensor-core kernels
    unsigned long long *d_next = nullptr;   // work counter of the batched kernel
    int *d_order = nullptr;                 // its work order (largest matrices first)
    int64_t order_cap = 0;
    struct BatchGraph {
        const cup_batch_item *items; int64_t count; int64_t *rank; uint32_t *det; cudaStream_t st;
        int64_t gen; cudaGraphExec_t exec; bool no_capture;
    };
    std::vector<BatchGraph> bgraphs;         // batched calls replayed as graphs
    void *d_ws = nullptr;          // limb planes of the tensor-core Schur update
    size_t ws_bytes = 0;
    int profile = 0;
    int schedule = 1;              // 0: host-driven recursion, 1: device-resident (+ graph replay)
    int int_path = 0;              // multi-modular images: 0 cost model, 1 batched launch, 2 per prime
    cudaStream_t copy = nullptr;   // host-to-device copies of cup_factor_host, overlapping the factorization
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> chunk_ev;  // one per row chunk of a host input
    int use_graph = 1;
    int64_t *d_rank_at = nullptr;  // device-resident schedule: rank before each leaf
    int64_t rank_at_cap = 0;
    uint32_t *d_backup = nullptr;  // input copy for the exact fallback
    size_t backup_bytes = 0;
    uint32_t *d_wide = nullptr;    // uint32 working copy of a one-byte-storage matrix
    size_t wide_bytes = 0;
    int64_t *h_rank = nullptr;     // pinned copy of rank_at after a device-resident run
    int64_t h_rank_cap = 0;
    struct Timed;
    struct GraphEntry {
        uint32_t *A; int64_t m, n, lda; uint32_t p; int64_t *prof, *ipiv; cudaStream_t st;
        int leaf_rows, window, engine; int64_t tc_min_k; int64_t gen; cudaGraphExec_t exec;
        int64_t launches;                 // kernels per replay
        bool no_capture;                  // capture failed once: stay eager
        std::vector<int> timed;           // indices into graph_timed, read after each replay
        std::vector<GemmDesc> gemms;      // the Schur updates it runs (extents resolved per replay)
        const void *hA = nullptr;         // host input copied in by the graph (cup_factor_host)
        int64_t ldh = 0;
        const uint8_t *dev8 = nullptr;    // one-byte input (or its staging copy) widened by the graph
        int64_t ld8 = 0;
        int esize = 4;
        int64_t short_k = 0;
    };
    int64_t gen = 0;                   // bumped whenever a buffer a graph may reference moves
    std::vector<GraphEntry> graphs;
    cup_stats stats = {};
    struct Timed { cudaEvent_t e0, e1; double limb_flops, field_flops; int cls; };
    std::vector<Timed> graph_timed;    // event pairs baked into captured graphs
    double cls_ms[9] = {0};        // per kernel class, profile level >= 2 (8: short-K updates)
    std::vector<Timed> pending;    // recorded intervals not yet read
    std::vector<cudaEvent_t> evpool;
    char err[256] = {0};
};

namespace {

cup_status cuda_ok(cup_handle *h, cudaError_t e)
{
    if (e == cudaSuccess) return CUP_OK;
    snprintf(h->err, sizeof(h->err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return (e == cudaErrorMemoryAllocation) ? CUP_ERR_NOMEM : CUP_ERR_CUDA;
}

#define CK(x)                                  \
    do {                                       \
        cup_status _s = (x);                   \
        if (_s != CUP_OK) return _s;           \
    } while (0)
#define CU(x) CK(cuda_ok(h, (x)))

uint64_t powmod64(uint64_t b, uint64_t e, uint64_t m)
{
    uint64_t r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1) r = (uint64_t)((unsigned __int128)r * b % m);
        b = (uint64_t)((unsigned __int128)b * b % m);
        e >>= 1;
    }
    return r;
}

// Deterministic Miller-Rabin for 32-bit n (bases 2, 3, 5, 7 suffice below 3.2e9).
bool is_prime32(uint32_t n)
{
    if (n < 2) return false;
    for (uint32_t q : {2u, 3u, 5u, 7u}) {
        if (n % q == 0) return n == q;
    }
    uint32_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; ++s; }
    for (uint32_t a : {2u, 3u, 5u, 7u}) {
        uint64_t x = powmod64(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < s; ++i) {
            x = x * x % n;
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

cup_status check_prime(uint32_t p)
{
    if (p >= (1u << 31) || !is_prime32(p)) return CUP_ERR_PRIME;
    return CUP_OK;
}

struct Ctx {
    cup_handle *h;
    uint32_t *A;
    int64_t lda, n;
    ModP M;
    int64_t *ipiv, *prof;
    cudaStream_t st;
};

cudaEvent_t take_event(cup_handle *h)
{
    if (!h->evpool.empty()) {
        cudaEvent_t e = h->evpool.back();
        h->evpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Fold recorded intervals into the counters; the stream they were recorded on
// must have drained.
void flush_timings(cup_handle *h)
{
    for (auto &t : h->pending) {
        float ms = 0.f;
        if (t.e0 && t.e1 && cudaEventElapsedTime(&ms, t.e0, t.e1) == cudaSuccess) {
            if (t.cls == 0) h->stats.tc_ms += ms;
            else if (t.cls == 1) h->stats.cc_ms += ms;
            else if (t.cls == 8) h->stats.sk_ms += ms;
            h->cls_ms[t.cls] += ms;
        }
        if (t.e0) h->evpool.push_back(t.e0);
        if (t.e1) h->evpool.push_back(t.e1);
    }
    h->pending.clear();
}

cup_status sync_stream(cup_handle *h, cudaStream_t st)
{
    CU(cudaStreamSynchronize(st));
    ++h->stats.host_syncs;
    flush_timings(h);
    return CUP_OK;
}

// Interval of one kernel class (profile level >= 2): classes 2 = base-case
// pivots, 3 = base-case finish, 4 = TRSM leaf, 5 = transpositions, 6 = a whole
// tcgen05 update (limb split and product).
struct ClassTimer {
    cup_handle *h;
    cudaStream_t st;
    int cls;
    cudaEvent_t e0 = nullptr;
    ClassTimer(cup_handle *h_, cudaStream_t st_, int cls_) : h(h_), st(st_), cls(cls_)
    {
        if (h->profile >= 2 && (e0 = take_event(h))) cudaEventRecord(e0, st);
    }
    ~ClassTimer()
    {
        if (!e0) return;
        cudaEvent_t e1 = take_event(h);
        if (e1) cudaEventRecord(e1, st);
        h->pending.push_back({e0, e1, 0.0, 0.0, cls});
    }
};

cup_status ensure_pairs(cup_handle *h, int64_t need)
{
    if (need <= h->pairs_cap) return CUP_OK;
    if (h->d_pairs) cudaFree(h->d_pairs);
    h->d_pairs = nullptr;
    h->pairs_cap = 0;
    CU(cudaMalloc(&h->d_pairs, (size_t)need * sizeof(int2)));
    h->pairs_cap = need;
    ++h->gen;
    return CUP_OK;
}

cup_status ensure_base(cup_handle *h)
{
    if (!h->d_slab) CU(cudaMalloc(&h->d_slab, sizeof(SlabScratch)));
    if (!h->d_count) CU(cudaMalloc(&h->d_count, sizeof(int)));
    if (!h->h_pinned) CU(cudaMallocHost(&h->h_pinned, 16 * sizeof(int)));
    if (!h->d_err) {
        CU(cudaMalloc(&h->d_err, sizeof(int)));
        CU(cudaMemset(h->d_err, 0, sizeof(int)));
    }
    return CUP_OK;
}

cup_status ensure_ws(cup_handle *h, size_t bytes)
{
    if (bytes <= h->ws_bytes) return CUP_OK;
    if (h->d_ws) cudaFree(h->d_ws);
    h->d_ws = nullptr;
    h->ws_bytes = 0;
    CU(cudaMalloc(&h->d_ws, bytes));
    h->ws_bytes = bytes;
    ++h->gen;
    return CUP_OK;
}

// Reads the device error word after `st` drains; a set word means a bounded
// device-side wait gave up.
cup_status check_device_error(cup_handle *h, cudaStream_t st)
{
    CU(cudaMemcpyAsync(h->h_pinned + 8, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(sync_stream(h, st));
    if (h->h_pinned[8] != 0) {
        snprintf(h->err, sizeof(h->err), "device wait expired (site %d)", h->h_pinned[8]);
        cudaMemsetAsync(h->d_err, 0, sizeof(int), st);
        return CUP_ERR_TIMEOUT;
    }
    return CUP_OK;
}

cup_status laswp(Ctx &c, int64_t row0, int64_t nrows, int64_t k0, int64_t k1)
{
    cup_handle *h = c.h;
    if (nrows <= 0 || k1 <= k0) return CUP_OK;
    CK(ensure_pairs(h, k1 - k0));
    ClassTimer tm(h, c.st, 5);
    CU(launch_swaplist(c.ipiv, dconst(k0), dconst(k1), h->d_pairs, h->d_count, c.st));
    CU(launch_laswp(c.A, c.lda, dconst(row0), dconst(nrows), h->d_pairs, h->d_count, c.st));
    h->stats.launches += 2;
    return CUP_OK;
}

cup_status mm_sub(cup_handle *h, uint32_t *C, int64_t ldc, const uint32_t *A, int64_t lda,
                  const uint32_t *B, int64_t ldb, int64_t M, int64_t N, int64_t K, const ModP &Mp,
                  int engine, cudaStream_t st, int add = 0)
{
    if (M <= 0 || N <= 0 || K <= 0) return CUP_OK;
    if (engine == CUP_ENGINE_TENSOR && K >= h->tc_min_k && gemm_short_ok(Mp.p, M, N, K, h->short_k)) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (h->profile) { e0 = take_event(h); e1 = take_event(h); if (e0) cudaEventRecord(e0, st); }
        GemmDesc d{A, lda, dconst(0), dconst(0), B, ldb, dconst(0), dconst(0), C, ldc, dconst(0), dconst(0),
                   M, dconst(N), dconst(K), add};
        CU(launch_gemm_short_desc(d, Mp, st));
        if (e1) cudaEventRecord(e1, st);
        const double f = 2.0 * (double)M * (double)N * (double)K;
        h->stats.launches += 1;
        h->stats.sk_launches += 1;
        h->stats.sk_field_flops += f;
        if (h->profile) h->pending.push_back({e0, e1, 0.0, f, 8});
        return CUP_OK;
    }
    if (engine == CUP_ENGINE_TENSOR && K >= h->tc_min_k) {
        CK(ensure_base(h));
        CK(ensure_ws(h, tc_workspace_bytes(Mp.p, M, N, K)));
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (h->profile) { e0 = take_event(h); e1 = take_event(h); }
        CU(launch_gemm_sub_tc(A, lda, B, ldb, C, ldc, M, N, K, Mp, h->d_ws, h->d_err, st, e0, e1, add));
        const int L = tc_limbs(Mp.p);
        const double f = 2.0 * (double)M * (double)N * (double)K;
        h->stats.launches += 3;
        h->stats.tc_launches += 1;
        h->stats.tc_field_flops += f;
        h->stats.tc_limb_flops += f * L * L;
        h->stats.tc_alg_bytes += 2.0 * L * (double)(M + N) * (double)K + 8.0 * (double)M * (double)N;
        if (h->profile) h->pending.push_back({e0, e1, f * L * L, f, 0});
        return CUP_OK;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->profile) { e0 = take_event(h); e1 = take_event(h); if (e0) cudaEventRecord(e0, st); }
    CU(launch_gemm_sub_cc(A, lda, B, ldb, C, ldc, M, N, K, Mp, st, add));
    if (e1) cudaEventRecord(e1, st);
    h->stats.launches += 1;
    h->stats.cc_launches += 1;
    h->stats.cc_field_flops += 2.0 * (double)M * (double)N * (double)K;
    if (h->profile) h->pending.push_back({e0, e1, 0.0, 2.0 * (double)M * (double)N * (double)K, 1});
    return CUP_OK;
}

cup_status trsm_ruu(cup_handle *h, const uint32_t *U, int64_t ldu, uint32_t *B, int64_t ldb,
                    int64_t m, int64_t n, const ModP &M, int engine, cudaStream_t st)
{
    if (m <= 0 || n <= 0) return CUP_OK;
    if (n <= 128) {
        ClassTimer tm(h, st, 4);
        TriDesc d{U, ldu, dconst(0), dconst(0), B, ldb, dconst(0), dconst(0), m, dconst(n)};
        CU(launch_trsm_ruu_desc(d, M, st));
        h->stats.launches += 1;
        return CUP_OK;
    }
    // Algorithm 2: B1 <- B1 U1^{-1}; B2 <- B2 - B1 V; B2 <- B2 U2^{-1}
    int64_t k = ((n / 2) + 127) / 128 * 128;
    CK(trsm_ruu(h, U, ldu, B, ldb, m, k, M, engine, st));
    CK(mm_sub(h, B + k, ldb, B, ldb, U + k, ldu, m, n - k, k, M, engine, st));
    CK(trsm_ruu(h, U + k * ldu + k, ldu, B + k, ldb, m, n - k, M, engine, st));
    return CUP_OK;
}

// Triangular solve or multiply with an n x n triangle T (Sec. 3.2): right side
// B (rows x n) <- B T^{-1} or B T; left side B (n x cols) <- T^{-1} B or T B.
// Halves the triangle (Algorithm 2 and its mirror images; TRMM in the same
// way) and sends the off-diagonal products to the Schur-update engine.
cup_status tri_op(cup_handle *h, int flags, const uint32_t *T, int64_t ldt, uint32_t *B, int64_t ldb,
                  int64_t rows, int64_t cols, const ModP &M, int engine, cudaStream_t st)
{
    const bool left = flags & TRI_LEFT, upper = flags & TRI_UPPER, solve = flags & TRI_SOLVE;
    const int64_t n = left ? rows : cols;
    if (rows <= 0 || cols <= 0) return CUP_OK;
    if (n <= 64) {
        ClassTimer tm(h, st, 4);
        CU(launch_tri_leaf(flags, T, ldt, B, ldb, rows, cols, M, st));
        h->stats.launches += 1;
        return CUP_OK;
    }
    const int64_t k = ((n / 2) + 63) / 64 * 64;
    const uint32_t *T11 = T, *T12 = T + k, *T21 = T + k * ldt, *T22 = T + k * ldt + k;
    if (!left) {
        uint32_t *B1 = B, *B2 = B + k;
        const int64_t m = rows, n2 = n - k;
        if (solve && upper) {
            CK(tri_op(h, flags, T11, ldt, B1, ldb, m, k, M, engine, st));
            CK(mm_sub(h, B2, ldb, B1, ldb, T12, ldt, m, n2, k, M, engine, st, 0));
            CK(tri_op(h, flags, T22, ldt, B2, ldb, m, n2, M, engine, st));
        } else if (solve) {
            CK(tri_op(h, flags, T22, ldt, B2, ldb, m, n2, M, engine, st));
            CK(mm_sub(h, B1, ldb, B2, ldb, T21, ldt, m, k, n2, M, engine, st, 0));
            CK(tri_op(h, flags, T11, ldt, B1, ldb, m, k, M, engine, st));
        } else if (upper) {
            CK(tri_op(h, flags, T22, ldt, B2, ldb, m, n2, M, engine, st));
            CK(mm_sub(h, B2, ldb, B1, ldb, T12, ldt, m, n2, k, M, engine, st, 1));
            CK(tri_op(h, flags, T11, ldt, B1, ldb, m, k, M, engine, st));
        } else {
            CK(tri_op(h, flags, T11, ldt, B1, ldb, m, k, M, engine, st));
            CK(mm_sub(h, B1, ldb, B2, ldb, T21, ldt, m, k, n2, M, engine, st, 1));
            CK(tri_op(h, flags, T22, ldt, B2, ldb, m, n2, M, engine, st));
        }
    } else {
        uint32_t *B1 = B, *B2 = B + k * ldb;
        const int64_t c = cols, n2 = n - k;
        if (solve && upper) {
            CK(tri_op(h, flags, T22, ldt, B2, ldb, n2, c, M, engine, st));
            CK(mm_sub(h, B1, ldb, T12, ldt, B2, ldb, k, c, n2, M, engine, st, 0));
            CK(tri_op(h, flags, T11, ldt, B1, ldb, k, c, M, engine, st));
        } else if (solve) {
            CK(tri_op(h, flags, T11, ldt, B1, ldb, k, c, M, engine, st));
            CK(mm_sub(h, B2, ldb, T21, ldt, B1, ldb, n2, c, k, M, engine, st, 0));
            CK(tri_op(h, flags, T22, ldt, B2, ldb, n2, c, M, engine, st));
        } else if (upper) {
            CK(tri_op(h, flags, T11, ldt, B1, ldb, k, c, M, engine, st));
            CK(mm_sub(h, B1, ldb, T12, ldt, B2, ldb, k, c, n2, M, engine, st, 1));
            CK(tri_op(h, flags, T22, ldt, B2, ldb, n2, c, M, engine, st));
        } else {
            CK(tri_op(h, flags, T22, ldt, B2, ldb, n2, c, M, engine, st));
            CK(mm_sub(h, B2, ldb, T21, ldt, B1, ldb, n2, c, k, M, engine, st, 1));
            CK(tri_op(h, flags, T11, ldt, B1, ldb, k, c, M, engine, st));
        }
    }
    return CUP_OK;
}

// TRTRI (Algorithm 3 and its lower-triangular mirror): T <- T^{-1} in place.
// Upper: V <- V U2^{-1}, V <- U1^{-1} V, V <- -V, then recurse on U1, U2.
// Lower: W <- L2^{-1} W, W <- W L1^{-1}, W <- -W, then recurse.
cup_status trtri(cup_handle *h, bool upper, bool unit, uint32_t *T, int64_t ldt, int64_t n, const ModP &M,
                 int engine, cudaStream_t st)
{
    if (n <= 0) return CUP_OK;
    if (n <= 64) {
        ClassTimer tm(h, st, 4);
        CU(launch_trtri_leaf(upper, unit, T, ldt, (int)n, M, st));
        h->stats.launches += 1;
        return CUP_OK;
    }
    const int64_t k = ((n / 2) + 63) / 64 * 64, n2 = n - k;
    uint32_t *T11 = T, *T12 = T + k, *T21 = T + k * ldt, *T22 = T + k * ldt + k;
    const int base = (upper ? TRI_UPPER : 0) | (unit ? TRI_UNIT : 0) | TRI_SOLVE;
    if (upper) {
        CK(tri_op(h, base, T22, ldt, T12, ldt, k, n2, M, engine, st));
        CK(tri_op(h, base | TRI_LEFT, T11, ldt, T12, ldt, k, n2, M, engine, st));
        CU(launch_negate(T12, ldt, k, n2, M.p, st));
    } else {
        CK(tri_op(h, base | TRI_LEFT, T22, ldt, T21, ldt, n2, k, M, engine, st));
        CK(tri_op(h, base, T11, ldt, T21, ldt, n2, k, M, engine, st));
        CU(launch_negate(T21, ldt, n2, k, M.p, st));
    }
    h->stats.launches += 1;
    CK(trtri(h, upper, unit, T11, ldt, k, M, engine, st));
    CK(trtri(h, upper, unit, T22, ldt, n2, M, engine, st));
    return CUP_OK;
}

// TRULM (Algorithm 4) for A = [L\U] with U unit upper (strictly above the
// diagonal) and L non-unit lower (on and below it): A <- U L in place.
cup_status trulm(cup_handle *h, uint32_t *A, int64_t lda, int64_t n, const ModP &M, int engine, cudaStream_t st)
{
    if (n <= 0) return CUP_OK;
    if (n <= 64) {
        ClassTimer tm(h, st, 4);
        CU(launch_trulm_leaf(A, lda, (int)n, M, st));
        h->stats.launches += 1;
        return CUP_OK;
    }
    const int64_t k = ((n / 2) + 63) / 64 * 64, n2 = n - k;
    uint32_t *A11 = A, *A12 = A + k, *A21 = A + k * lda, *A22 = A + k * lda + k;
    CK(trulm(h, A11, lda, k, M, engine, st));                                           // U1 L1
    CK(mm_sub(h, A11, lda, A12, lda, A21, lda, k, k, n2, M, engine, st, 1));            // + U2 L2
    CK(tri_op(h, 0, A22, lda, A12, lda, k, n2, M, engine, st));                         // U2 L3
    CK(tri_op(h, TRI_LEFT | TRI_UPPER | TRI_UNIT, A22, lda, A21, lda, n2, k, M, engine, st));  // U3 L2
    CK(trulm(h, A22, lda, n2, M, engine, st));                                          // U3 L3
    return CUP_OK;
}

// TRLUM (Algorithm 5): A = [L\U] with L lower and U upper triangular; A <- L U.
// unit_l: L has the implicit unit diagonal (Algorithm 5 as stated); otherwise U
// has it, as in the [C\U] factors of CUP (Algorithm 9). The halves are done in
// the order that reads every operand before it is overwritten.
cup_status trlum(cup_handle *h, uint32_t *A, int64_t lda, int64_t n, int unit_l, const ModP &M, int engine,
                 cudaStream_t st)
{
    if (n <= 0) return CUP_OK;
    if (n <= 64) {
        ClassTimer tm(h, st, 4);
        CU(launch_trlum_leaf(A, lda, (int)n, unit_l, M, st));
        h->stats.launches += 1;
        return CUP_OK;
    }
    const int64_t k = ((n / 2) + 63) / 64 * 64, n2 = n - k;
    const int lu = unit_l ? TRI_UNIT : 0, uu = unit_l ? 0 : TRI_UNIT;
    uint32_t *A11 = A, *A12 = A + k, *A21 = A + k * lda, *A22 = A + k * lda + k;
    CK(trlum(h, A22, lda, n2, unit_l, M, engine, st));                                  // L3 U3
    CK(mm_sub(h, A22, lda, A21, lda, A12, lda, n2, n2, k, M, engine, st, 1));           // + L2 U2
    CK(tri_op(h, TRI_LEFT | lu, A11, lda, A12, lda, k, n2, M, engine, st));             // L1 U2
    CK(tri_op(h, TRI_UPPER | uu, A11, lda, A21, lda, n2, k, M, engine, st));            // L2 U1
    CK(trlum(h, A11, lda, k, unit_l, M, engine, st));                                   // L1 U1
    return CUP_OK;
}

// Algorithms 7 and 8 on the [C\U] factors of rank r: leaves A as
// [X1 X2; R2 0] with the rows of C reordered by the profile loop, i.e. the
// reduced column echelon transform up to that row permutation.
cup_status red_col_ech(cup_handle *h, uint32_t *A, int64_t m, int64_t n, int64_t lda, int64_t r,
                       const int64_t *d_prof, const ModP &M, int engine, cudaStream_t st)
{
    if (r <= 0) return CUP_OK;
    // Algorithm 7: M <- U1^{-1} U2, N <- -M, U1 <- U1^{-1}
    if (r < n) {
        CK(tri_op(h, TRI_LEFT | TRI_UPPER | TRI_UNIT | TRI_SOLVE, A, lda, A + r, lda, r, n - r, M, engine, st));
        CU(launch_negate(A + r, lda, r, n - r, M.p, st));
        h->stats.launches += 1;
    }
    CK(trtri(h, true, true, A, lda, r, M, engine, st));
    // Algorithm 8: bring the profile rows of C to the top (first j+1 entries of
    // rows j and i_j exchanged, j increasing), R2 <- L2 L1^{-1}, L1 <- L1^{-1},
    // X1 <- T1 L1^{-1}
    CU(launch_row_swaps(A, lda, r, d_prof, r, 0, 0, 0, 1, st));
    h->stats.launches += 1;
    if (m > r) CK(tri_op(h, TRI_SOLVE, A, lda, A + r * lda, lda, m - r, r, M, engine, st));
    CK(trtri(h, false, false, A, lda, r, M, engine, st));
    CK(trulm(h, A, lda, r, M, engine, st));
    return CUP_OK;
}

cup_status cup_rec(Ctx &c, int64_t a, int64_t mrows, int64_t col0, int64_t *r_out)
{
    cup_handle *h = c.h;
    const int64_t w = c.n - col0;
    *r_out = 0;
    if (w <= 0 || mrows <= 0) return CUP_OK;
    int64_t k, r1;
    if (mrows <= h->leaf_rows) {
        {
        ClassTimer tm(h, c.st, 2);
        CU(launch_slab_pivots(c.A, c.lda, a, (int)mrows, dconst(col0), c.n, h->window, 0, c.M, h->d_slab,
                              c.ipiv, c.prof, nullptr, c.st));
        }
        CU(cudaMemcpyAsync(h->h_pinned, h->d_slab, 2 * sizeof(int), cudaMemcpyDeviceToHost, c.st));
        {
        ClassTimer tm(h, c.st, 3);
        CU(launch_slab_finish(c.A, c.lda, a, (int)mrows, dconst(col0), c.n, c.M, h->d_slab, nullptr, c.st,
                              h->engine == CUP_ENGINE_TENSOR));
        }
        h->stats.launches += 2;
        CK(sync_stream(h, c.st));
        r1 = h->h_pinned[0];
        k = h->h_pinned[1];
        if (k == mrows) { *r_out = r1; return CUP_OK; }
    } else {
        int64_t nl = (mrows + h->leaf_rows - 1) / h->leaf_rows;
        k = ((nl + 1) / 2) * h->leaf_rows;
        CK(cup_rec(c, a, k, col0, &r1));
    }
    const int64_t a2 = a + k, m2 = mrows - k;
    if (r1 > 0) {
        uint32_t *A = c.A;
        const int64_t lda = c.lda;
        CK(laswp(c, a2, m2, col0, col0 + r1));
        CK(trsm_ruu(h, A + col0 * lda + col0, lda, A + a2 * lda + col0, lda, m2, r1, c.M,
                    h->engine, c.st));
        if (col0 + r1 < c.n)
            CK(mm_sub(h, A + a2 * lda + col0 + r1, lda, A + a2 * lda + col0, lda,
                      A + col0 * lda + col0 + r1, lda, m2, c.n - col0 - r1, r1, c.M, h->engine,
                      c.st));
    }
    int64_t r2 = 0;
    CK(cup_rec(c, a2, m2, col0 + r1, &r2));
    if (r1 > 0 && r2 > 0) CK(laswp(c, col0, r1, col0 + r1, col0 + r1 + r2));
    *r_out = r1 + r2;
    return CUP_OK;
}

// ---------------------------------------------------------------------------
// Device-resident schedule of Algorithm 6. The recursion tree over rows is
// fixed by m and the leaf size; what depends on the data (the rank of the
// rows above a block, col0, and of its top half, mid) is read by every kernel
// from rank_at[], which the base-case kernels fill in as they run. Nothing is
// read back until the end, so the whole factorisation is one stream of
// launches (and one CUDA graph when replayed). Rows whose pivot-window
// residual vanishes are taken as dependent and checked by the finish kernel;
// if a check fails the call is redone host-driven from a copy of the input.
// ---------------------------------------------------------------------------
struct DevCtx {
    cup_handle *h;
    uint32_t *A;
    int64_t lda, m, n;
    ModP M;
    int64_t *ipiv, *prof, *rank_at;
    cudaStream_t st;
    int nleaf;
    std::vector<GemmDesc> *gemms;     // every Schur update enqueued (extents resolved after the run)
    // host input arriving in row chunks: chunk i starts at row chunk_row[i] and has
    // landed at chunk_ev[i]; rows of chunks before next_chunk are known to be there
    const int64_t *chunk_row = nullptr;
    const cudaEvent_t *chunk_ev = nullptr;
    int nchunk = 0, next_chunk = 0;
};

// The stream waits for every chunk of a host input that holds a row below y.
cup_status need_rows(DevCtx &c, int64_t y)
{
    cup_handle *h = c.h;
    while (c.next_chunk < c.nchunk && y > c.chunk_row[c.next_chunk]) {
        CU(cudaStreamWaitEvent(c.st, c.chunk_ev[c.next_chunk], 0));
        ++c.next_chunk;
    }
    return CUP_OK;
}

// Host evaluation of a Dyn whose pointers point into the device array dbase,
// given a host copy hbase of that array.
int64_t host_eval(const Dyn &d, const int64_t *dbase, const int64_t *hbase)
{
    int64_t v = d.s;
    if (d.p0) v += d.c0 * hbase[d.p0 - dbase];
    if (d.p1) v += d.c1 * hbase[d.p1 - dbase];
    return v < d.lo ? d.lo : (v > d.hi ? d.hi : v);
}

cup_status dev_gemm(DevCtx &c, const GemmDesc &g)
{
    cup_handle *h = c.h;
    if (g.M <= 0 || g.N.hi <= 0 || g.K.hi <= 0) return CUP_OK;
    const bool tc = h->engine == CUP_ENGINE_TENSOR && g.K.hi >= h->tc_min_k;
    const bool sk = tc && gemm_short_ok(c.M.p, g.M, g.N.hi, g.K.hi, h->short_k);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->profile) { e0 = take_event(h); e1 = take_event(h); }
    if (sk) {
        if (e0) cudaEventRecord(e0, c.st);
        CU(launch_gemm_short_desc(g, c.M, c.st));
        if (e1) cudaEventRecord(e1, c.st);
        h->stats.launches += 1;
    } else if (tc) {
        ClassTimer tm(h, c.st, 6);
        CU(launch_gemm_tc_desc(g, c.M, h->d_ws, h->d_err, c.st, e0, e1));
        h->stats.launches += 3;
    } else {
        if (e0) cudaEventRecord(e0, c.st);
        CU(launch_gemm_cc_desc(g, c.M, c.st));
        if (e1) cudaEventRecord(e1, c.st);
        h->stats.launches += 1;
    }
    if (h->profile) h->pending.push_back({e0, e1, 0.0, 0.0, sk ? 8 : tc ? 0 : 1});
    GemmDesc rec = g;
    rec.add = sk ? 2 : tc ? 1 : 0;      // reused as the engine tag in the record
    c.gemms->push_back(rec);
    return CUP_OK;
}

cup_status dev_laswp(DevCtx &c, Dyn row0, Dyn nrows, Dyn k0, Dyn k1)
{
    cup_handle *h = c.h;
    if (nrows.hi <= 0 || k1.hi <= k0.lo) return CUP_OK;
    ClassTimer tm(h, c.st, 5);
    CU(launch_laswp_fused(c.A, c.lda, row0, nrows, c.ipiv, k0, k1, c.st));
    h->stats.launches += 1;
    return CUP_OK;
}

// TRSM(Right, Upper, Unit) on columns [j0, j0 + len) of the block [col0, mid):
// Algorithm 2 with the split fixed by the static bound len and every extent
// clamped to r1 = mid - col0 on the device.
cup_status dev_trsm(DevCtx &c, const int64_t *col0p, const int64_t *midp, int64_t a2, int64_t m2, int64_t j0,
                    int64_t len)
{
    cup_handle *h = c.h;
    if (len <= 0) return CUP_OK;
    if (len <= 128) {
        // the triangle U1 comes from the top half's finish kernels; the launch just
        // before this one is the bottom half's transpositions or a TRSM product,
        // neither of which writes U1 or the ranks
        TriDesc d{c.A, c.lda, dvar(j0, col0p, 1, nullptr, 0, 0, c.n), dvar(j0, col0p, 1, nullptr, 0, 0, c.n),
                  c.A, c.lda, dconst(a2), dvar(j0, col0p, 1, nullptr, 0, 0, c.n), m2,
                  dvar(-j0, midp, 1, col0p, -1, 0, len), 1};
        ClassTimer tm(h, c.st, 4);
        CU(launch_trsm_ruu_desc(d, c.M, c.st));
        h->stats.launches += 1;
        return CUP_OK;
    }
    const int64_t k = ((len / 2) + 127) / 128 * 128;
    CK(dev_trsm(c, col0p, midp, a2, m2, j0, k));
    GemmDesc g{c.A, c.lda, dconst(a2), dvar(j0, col0p, 1, nullptr, 0, 0, c.n),
               c.A, c.lda, dvar(j0, col0p, 1, nullptr, 0, 0, c.n), dvar(j0 + k, col0p, 1, nullptr, 0, 0, c.n),
               c.A, c.lda, dconst(a2), dvar(j0 + k, col0p, 1, nullptr, 0, 0, c.n),
               m2, dvar(-j0 - k, midp, 1, col0p, -1, 0, len - k), dvar(-j0, midp, 1, col0p, -1, 0, k), 0,
               1};   // the launch before is the TRSM leaf that wrote A (G's first columns) only
    CK(dev_gemm(c, g));
    CK(dev_trsm(c, col0p, midp, a2, m2, j0 + k, len - k));
    return CUP_OK;
}

cup_status dev_rec(DevCtx &c, int64_t a, int64_t mrows)
{
    cup_handle *h = c.h;
    if (mrows <= 0) return CUP_OK;
    if (mrows <= h->leaf_rows) {
        CK(need_rows(c, a + mrows));
        const int L = c.nleaf++;
        const Dyn col0 = dvar(0, c.rank_at + L, 1, nullptr, 0, 0, c.n);
        {
            ClassTimer tm(h, c.st, 2);
            CU(launch_slab_pivots(c.A, c.lda, a, (int)mrows, col0, c.n, h->window, 1, c.M, h->d_slab, c.ipiv,
                                  c.prof, c.rank_at + L + 1, c.st));
        }
        {
            ClassTimer tm(h, c.st, 3);
            CU(launch_slab_finish(c.A, c.lda, a, (int)mrows, col0, c.n, c.M, h->d_slab, h->d_err, c.st,
                                  h->engine == CUP_ENGINE_TENSOR));
        }
        h->stats.launches += 2;
        return CUP_OK;
    }
    const int64_t nl = (mrows + h->leaf_rows - 1) / h->leaf_rows;
    const int64_t k = ((nl + 1) / 2) * h->leaf_rows;
    const int L0 = c.nleaf;
    CK(dev_rec(c, a, k));
    const int Lm = c.nleaf;
    const int64_t *col0p = c.rank_at + L0, *midp = c.rank_at + Lm;
    const int64_t a2 = a + k, m2 = mrows - k, kmax = k < c.n ? k : c.n;
    CK(need_rows(c, a2 + m2));
    // A2 <- A2 P1^T
    CK(dev_laswp(c, dconst(a2), dconst(m2), dvar(0, col0p, 1, nullptr, 0, 0, c.n), dvar(0, midp, 1, nullptr, 0, 0, c.n)));
    // G <- A21 U1^{-1}
    CK(dev_trsm(c, col0p, midp, a2, m2, 0, kmax));
    // H <- A22 - G V1
    GemmDesc g{c.A, c.lda, dconst(a2), dvar(0, col0p, 1, nullptr, 0, 0, c.n),
               c.A, c.lda, dvar(0, col0p, 1, nullptr, 0, 0, c.n), dvar(0, midp, 1, nullptr, 0, 0, c.n),
               c.A, c.lda, dconst(a2), dvar(0, midp, 1, nullptr, 0, 0, c.n),
               m2, dvar(c.n, midp, -1, nullptr, 0, 0, c.n), dvar(0, midp, 1, col0p, -1, 0, kmax), 0,
               1};   // the launch before is the TRSM leaf that wrote A (G) only
    CK(dev_gemm(c, g));
    CK(dev_rec(c, a2, m2));
    const int L1 = c.nleaf;
    const int64_t *endp = c.rank_at + L1;
    // V1 <- V1 P2^T
    CK(dev_laswp(c, dvar(0, col0p, 1, nullptr, 0, 0, c.n), dvar(0, midp, 1, col0p, -1, 0, kmax),
                 dvar(0, midp, 1, nullptr, 0, 0, c.n), dvar(0, endp, 1, nullptr, 0, 0, c.n)));
    return CUP_OK;
}

int64_t count_leaves(int64_t mrows, int leaf_rows)
{
    if (mrows <= 0) return 0;
    if (mrows <= leaf_rows) return 1;
    const int64_t nl = (mrows + leaf_rows - 1) / leaf_rows;
    const int64_t k = ((nl + 1) / 2) * leaf_rows;
    return count_leaves(k, leaf_rows) + count_leaves(mrows - k, leaf_rows);
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

bool cup_internal_prime_ok(uint32_t p) { return check_prime(p) == CUP_OK; }

cudaError_t launch_cup_batched(const cup_batch_item *items, int64_t count, int64_t *ranks, uint32_t *dets,
                               unsigned long long *next, int *order, int grid, cudaStream_t st);

#define CUP_ERR_SPECULATION_INTERNAL ((cup_status)-100)

namespace {

// Where the input of a factorization comes from. By default it is already in A
// (uint32, on the device). With `host` it is a host matrix of esize-byte entries
// (4: uint32, 1: uint8) copied in by the call; a one-byte host input lands in the
// device bytes dev8 first. With dev8 and no host it is a device matrix of bytes.
// One-byte inputs are widened into A, the call's uint32 working copy.
struct InputSrc {
    const void *host = nullptr;
    int64_t ldh = 0;
    int esize = 4;
    uint8_t *dev8 = nullptr;
    int64_t ld8 = 0;
};

// Rows [r0, r1) of the input into A, on stream `st`.
cup_status load_rows(cup_handle *h, uint32_t *A, int64_t lda, int64_t n, int64_t r0, int64_t r1, const InputSrc &src,
                     cudaStream_t st)
{
    if (r1 <= r0) return CUP_OK;
    if (src.host && src.esize == 4) {
        CU(cudaMemcpy2DAsync(A + r0 * lda, (size_t)lda * 4, (const uint32_t *)src.host + r0 * src.ldh,
                             (size_t)src.ldh * 4, (size_t)n * 4, (size_t)(r1 - r0), cudaMemcpyHostToDevice, st));
        return CUP_OK;
    }
    if (src.host)
        CU(cudaMemcpy2DAsync(src.dev8 + r0 * src.ld8, (size_t)src.ld8, (const uint8_t *)src.host + r0 * src.ldh,
                             (size_t)src.ldh, (size_t)n, (size_t)(r1 - r0), cudaMemcpyHostToDevice, st));
    if (src.dev8) {
        CU(launch_widen_u8(A + r0 * lda, lda, src.dev8 + r0 * src.ld8, src.ld8, r1 - r0, n, st));
        h->stats.launches += 1;
    }
    return CUP_OK;
}

// A host input is copied into A in row chunks on a second stream, and the
// factorization waits for a chunk only when it first touches one of its rows (the
// recursion reaches the rows in order); a device byte input is widened into A by
// the first launch.
cup_status factor_device(cup_handle *h, uint32_t *A, int64_t m, int64_t n, int64_t lda, uint32_t p,
                         int64_t *d_profile, int64_t *d_ipiv, int64_t *rank, cudaStream_t st,
                         const InputSrc &src)
{
    const void *hA = src.host;
    const int64_t ldh = src.ldh;
    const int64_t nleaves = count_leaves(m, h->leaf_rows);
    if (nleaves + 1 > h->rank_at_cap) {
        if (h->d_rank_at) cudaFree(h->d_rank_at);
        h->d_rank_at = nullptr;
        h->rank_at_cap = 0;
        CU(cudaMalloc(&h->d_rank_at, (size_t)(nleaves + 1) * sizeof(int64_t)));
        h->rank_at_cap = nleaves + 1;
        ++h->gen;
    }
    // the exact fallback restarts from a copy of a device input (a host input is
    // simply copied in again), so only device inputs need the m n backup
    const size_t bbytes = (size_t)m * (size_t)n * 4;
    const bool backup = !hA && !src.dev8;
    if (backup && bbytes > h->backup_bytes) {
        if (h->d_backup) cudaFree(h->d_backup);
        h->d_backup = nullptr;
        h->backup_bytes = 0;
        CU(cudaMalloc(&h->d_backup, bbytes));
        h->backup_bytes = bbytes;
        ++h->gen;
    }
    CK(ensure_pairs(h, n));
    if (h->engine == CUP_ENGINE_TENSOR) {
        // the largest product: rows below the first split, all columns, inner size up to that split
        const int64_t nl = (m + h->leaf_rows - 1) / h->leaf_rows;
        const int64_t ktop = m > h->leaf_rows ? ((nl + 1) / 2) * h->leaf_rows : 0;
        if (ktop > 0) CK(ensure_ws(h, tc_workspace_bytes(p, m, n, ktop < n ? ktop : n)));
    }
    if (nleaves + 1 > h->h_rank_cap) {
        if (h->h_rank) cudaFreeHost(h->h_rank);
        h->h_rank = nullptr;
        h->h_rank_cap = 0;
        CU(cudaMallocHost(&h->h_rank, (size_t)(nleaves + 1) * sizeof(int64_t)));
        h->h_rank_cap = nleaves + 1;
        ++h->gen;
    }
    const ModP M = make_modp(p);
    // graph replay for a repeated call with the same buffers and options
    cup_handle::GraphEntry *ge = nullptr;
    for (auto &e : h->graphs)
        if (e.A == A && e.m == m && e.n == n && e.lda == lda && e.p == p && e.prof == d_profile && e.hA == hA &&
            e.ldh == ldh && e.dev8 == src.dev8 && e.ld8 == src.ld8 && e.esize == src.esize &&
            e.ipiv == d_ipiv && e.st == st && e.leaf_rows == h->leaf_rows && e.window == h->window &&
            e.engine == h->engine && e.tc_min_k == h->tc_min_k && e.short_k == h->short_k)
            ge = &e;
    if (ge && ge->gen != h->gen) {
        if (ge->exec) cudaGraphExecDestroy(ge->exec);
        ge->exec = nullptr;
        ge->gen = h->gen;
    }
    // row chunks of a host input: one leaf, one leaf, then doubling (the first rows
    // the recursion's leftmost path reaches beyond each split)
    std::vector<int64_t> chunk_row;
    if (hA) {
        for (int64_t r0 = 0, len = h->leaf_rows; r0 < m; r0 += len, len = (r0 > len ? r0 : len))
            chunk_row.push_back(r0);
        if (!h->copy) CU(cudaStreamCreateWithFlags(&h->copy, cudaStreamNonBlocking));
        if (!h->ev_fork) CU(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        while (h->chunk_ev.size() < chunk_row.size()) {
            cudaEvent_t e = nullptr;
            CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            h->chunk_ev.push_back(e);
        }
    }
    auto enqueue = [&](std::vector<GemmDesc> &gl) -> cup_status {
        DevCtx c{h, A, lda, m, n, M, d_ipiv, d_profile, h->d_rank_at, st, 0, &gl};
        if (hA) {
            CU(cudaEventRecord(h->ev_fork, st));
            CU(cudaStreamWaitEvent(h->copy, h->ev_fork, 0));
            for (size_t i = 0; i < chunk_row.size(); ++i) {
                const int64_t r0 = chunk_row[i], r1 = i + 1 < chunk_row.size() ? chunk_row[i + 1] : m;
                CK(load_rows(h, A, lda, n, r0, r1, src, h->copy));
                CU(cudaEventRecord(h->chunk_ev[i], h->copy));
            }
            c.chunk_row = chunk_row.data();
            c.chunk_ev = h->chunk_ev.data();
            c.nchunk = (int)chunk_row.size();
        } else if (src.dev8) {
            CK(load_rows(h, A, lda, n, 0, m, src, st));
        } else {
            CU(cudaMemcpy2DAsync(h->d_backup, (size_t)n * 4, A, (size_t)lda * 4, (size_t)n * 4, (size_t)m,
                                 cudaMemcpyDeviceToDevice, st));
        }
        CU(cudaMemsetAsync(h->d_rank_at, 0, sizeof(int64_t), st));
        CU(cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
        CK(dev_rec(c, 0, m));
        CK(need_rows(c, INT64_MAX));          // every copy joined (a capture needs the copy stream joined)
        CU(cudaMemcpyAsync(h->h_rank, h->d_rank_at, (size_t)(nleaves + 1) * sizeof(int64_t),
                           cudaMemcpyDeviceToHost, st));
        CU(cudaMemcpyAsync(h->h_pinned + 8, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        return CUP_OK;
    };
    const int64_t launches0 = h->stats.launches;
    // the legacy default stream cannot be captured
    const bool capturable = st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread && h->profile == 0;
    std::vector<GemmDesc> gl_local;
    const std::vector<GemmDesc> *glist = &gl_local;
    const std::vector<int> *timed_now = nullptr;
    if (ge && ge->exec && capturable) {
        CU(cudaGraphLaunch(ge->exec, st));
        h->stats.launches += ge->launches;
        glist = &ge->gemms;
        timed_now = &ge->timed;
    } else if (ge && h->use_graph && capturable && !ge->no_capture) {
        const size_t pend0 = h->pending.size();
        ge->gemms.clear();
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cup_status s = CUP_ERR_CUDA;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            s = enqueue(ge->gemms);
            cudaError_t e = cudaStreamEndCapture(st, &graph);
            if (s == CUP_OK && e == cudaSuccess && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
                exec = nullptr;
            if (graph) cudaGraphDestroy(graph);
        }
        if (!exec) {
            // capture is not available here: run this and later identical calls eagerly
            cudaGetLastError();
            ge->no_capture = true;
            for (size_t i = pend0; i < h->pending.size(); ++i) {
                if (h->pending[i].e0) h->evpool.push_back(h->pending[i].e0);
                if (h->pending[i].e1) h->evpool.push_back(h->pending[i].e1);
            }
            h->pending.resize(pend0);
            h->stats.launches = launches0;
            ge->gemms.clear();
            return factor_device(h, A, m, n, lda, p, d_profile, d_ipiv, rank, st, src);
        }
        ge->exec = exec;
        ge->launches = h->stats.launches - launches0;
        // event pairs recorded during capture stay with the graph
        ge->timed.clear();
        for (size_t i = pend0; i < h->pending.size(); ++i) {
            ge->timed.push_back((int)h->graph_timed.size());
            h->graph_timed.push_back(h->pending[i]);
        }
        h->pending.resize(pend0);
        CU(cudaGraphLaunch(exec, st));
        glist = &ge->gemms;
        timed_now = &ge->timed;
    } else {
        if (!ge && h->use_graph && capturable) {
            // remember the call; the next identical one is captured and replayed
            cup_handle::GraphEntry e{A, m, n, lda, p, d_profile, d_ipiv, st, h->leaf_rows, h->window, h->engine,
                                     h->tc_min_k, h->gen, nullptr, 0, false, {}, {}, hA, ldh, src.dev8, src.ld8,
                                     src.esize, h->short_k};
            if (h->graphs.size() > 16) {
                if (h->graphs.front().exec) cudaGraphExecDestroy(h->graphs.front().exec);
                h->graphs.erase(h->graphs.begin());
            }
            h->graphs.push_back(e);
        }
        CK(enqueue(gl_local));
    }
    CK(sync_stream(h, st));
    if (timed_now)
        for (int ti : *timed_now) {
            auto &t = h->graph_timed[ti];
            float ms = 0.f;
            if (t.e0 && t.e1 && cudaEventElapsedTime(&ms, t.e0, t.e1) == cudaSuccess) {
                if (t.cls == 0) h->stats.tc_ms += ms;
                else if (t.cls == 1) h->stats.cc_ms += ms;
                else if (t.cls == 8) h->stats.sk_ms += ms;
                h->cls_ms[t.cls] += ms;
            } else {
                cudaGetLastError();          // an interval the graph could not time: leave it out
                h->cls_ms[7] += 1.0;         // count of such intervals
            }
        }
    const int64_t r = h->h_rank[nleaves];
    const int err = h->h_pinned[8];
    if (err == 0) {
        // the extents each Schur update actually had, from the ranks this run produced
        const int L = tc_limbs(p);
        for (const auto &g : *glist) {
            const double gn = (double)host_eval(g.N, h->d_rank_at, h->h_rank),
                         gk = (double)host_eval(g.K, h->d_rank_at, h->h_rank);
            const double f = 2.0 * (double)g.M * gn * gk;
            if (g.add == 2) {
                h->stats.sk_launches += 1;
                h->stats.sk_field_flops += f;
            } else if (g.add) {
                h->stats.tc_launches += 1;
                h->stats.tc_field_flops += f;
                h->stats.tc_limb_flops += f * L * L;
                h->stats.tc_alg_bytes += 2.0 * L * ((double)g.M + gn) * gk + 8.0 * (double)g.M * gn;
            } else {
                h->stats.cc_launches += 1;
                h->stats.cc_field_flops += f;
            }
        }
    }
    if (err == CUP_DEVERR_SPECULATION) {
        CU(cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
        return CUP_ERR_SPECULATION_INTERNAL;
    }
    if (err != 0) {
        snprintf(h->err, sizeof(h->err), "device wait expired (site %d)", err);
        CU(cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
        return CUP_ERR_TIMEOUT;
    }
    *rank = r;
    return CUP_OK;
}

cup_status ensure_wide(cup_handle *h, size_t bytes)
{
    if (bytes <= h->wide_bytes) return CUP_OK;
    if (h->d_wide) cudaFree(h->d_wide);
    h->d_wide = nullptr;
    h->wide_bytes = 0;
    CU(cudaMalloc(&h->d_wide, bytes));
    h->wide_bytes = bytes;
    ++h->gen;
    return CUP_OK;
}

// CUP of the input described by src into A (m x n, lda): the device-resident
// schedule (schedule 1), or the host-driven one (schedule 0, and the exact
// fallback when a row taken as dependent was not), which first loads the input
// again: from the host, from the device bytes, or from the backup copy that the
// device-resident run made of a uint32 device input.
// The handle's schedule options for one factorization: the first rule of the tuning
// table that matches the call's limb count and shape sets those the caller did not set
// with cup_set_option; the handle's own values come back when the call returns.
struct TunedOptions {
    cup_handle *h;
    int leaf_rows, window;
    int64_t tc_min_k;
    TunedOptions(cup_handle *h_, int64_t m, int64_t n, uint32_t p)
        : h(h_), leaf_rows(h_->leaf_rows), window(h_->window), tc_min_k(h_->tc_min_k)
    {
        const int64_t L = tc_limbs(p), k = m < n ? m : n, tall = m >= 2 * n ? 1 : 0;
        for (const auto &r : h->tuning) {
            if ((r.limbs >= 0 && r.limbs != L) || (r.tall >= 0 && r.tall != tall) || k < r.min_lo || k >= r.min_hi)
                continue;
            if (!h->user_set[0] && r.leaf_rows >= 1 && r.leaf_rows <= CUP_BMAX) h->leaf_rows = (int)r.leaf_rows;
            if (!h->user_set[1] && r.window >= 1 && r.window <= CUP_WNMAX) h->window = (int)r.window;
            if (!h->user_set[2] && r.tc_min_k >= 1) h->tc_min_k = r.tc_min_k;
            break;
        }
    }
    ~TunedOptions()
    {
        h->leaf_rows = leaf_rows;
        h->window = window;
        h->tc_min_k = tc_min_k;
    }
};

cup_status factor_impl(cup_handle *h, uint32_t *A, int64_t m, int64_t n, int64_t lda, uint32_t p,
                       int64_t *d_profile, int64_t *d_ipiv, int64_t *rank, cudaStream_t st, const InputSrc &src)
{
    TunedOptions tuned(h, m, n, p);
    cup_status s = CUP_ERR_SPECULATION_INTERNAL;
    if (h->schedule == 1) s = factor_device(h, A, m, n, lda, p, d_profile, d_ipiv, rank, st, src);
    if (s != CUP_ERR_SPECULATION_INTERNAL) return s;
    if (src.host || src.dev8) {
        CK(load_rows(h, A, lda, n, 0, m, src, st));
    } else if (h->schedule == 1) {
        CU(cudaMemcpy2DAsync(A, (size_t)lda * 4, h->d_backup, (size_t)n * 4, (size_t)n * 4, (size_t)m,
                             cudaMemcpyDeviceToDevice, st));
    }
    if (h->schedule == 1) ++h->stats.host_syncs;
    Ctx c{h, A, lda, n, make_modp(p), d_ipiv, d_profile, st};
    int64_t r = 0;
    CK(cup_rec(c, 0, m, 0, &r));
    CK(check_device_error(h, st));
    *rank = r;
    return CUP_OK;
}

// Determinant from the factorization of the input described by src into A (n x n).
cup_status det_impl(cup_handle *h, uint32_t *A, int64_t n, int64_t lda, uint32_t p, uint32_t *det, cudaStream_t st,
                    const InputSrc &src)
{
    int64_t *d_idx = nullptr;
    uint32_t *d_out = nullptr;
    CU(cudaMalloc(&d_idx, 2 * (size_t)n * sizeof(int64_t)));
    int64_t r = 0;
    cup_status s = factor_impl(h, A, n, n, lda, p, d_idx, d_idx + n, &r, st, src);
    if (s == CUP_OK) {
        if (r < n) {
            *det = 0;
        } else {
            s = cuda_ok(h, cudaMalloc(&d_out, sizeof(uint32_t)));
            if (s == CUP_OK) s = cuda_ok(h, launch_det_reduce(A, lda, n, d_idx + n, make_modp(p), d_out, st));
            if (s == CUP_OK)
                s = cuda_ok(h, cudaMemcpyAsync(h->h_pinned, d_out, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            if (s == CUP_OK) s = sync_stream(h, st);
            h->stats.launches += 1;
            if (s == CUP_OK) *det = (uint32_t)h->h_pinned[0];
        }
    }
    cudaFree(d_idx);
    if (d_out) cudaFree(d_out);
    return s;
}

// In-place inverse (Algorithm 8 via Algorithm 7) of the input described by src, in A.
cup_status inverse_impl(cup_handle *h, uint32_t *A, int64_t n, int64_t lda, uint32_t p, cudaStream_t st,
                        const InputSrc &src)
{
    int64_t *d_idx = nullptr;
    CU(cudaMalloc(&d_idx, 2 * (size_t)n * sizeof(int64_t)));
    int64_t r = 0;
    const ModP M = make_modp(p);
    cup_status s = factor_impl(h, A, n, n, lda, p, d_idx, d_idx + n, &r, st, src);
    if (s == CUP_OK && r < n) s = CUP_SINGULAR;
    if (s == CUP_OK) s = red_col_ech(h, A, n, n, lda, r, d_idx, M, h->engine, st);
    // A^{-1} = P^T X1: row swaps (j, ipiv[j]) for j = n-1 down to 0
    if (s == CUP_OK) s = cuda_ok(h, launch_row_swaps(A, lda, n, d_idx + n, n, 0, 0, 1, 0, st));
    if (s == CUP_OK) s = check_device_error(h, st);
    cudaFree(d_idx);
    return s;
}

// Checks shared by the one-byte entry points: p below 2^8 and prime.
cup_status check_u8(uint32_t p)
{
    if (p >= 256u) return CUP_ERR_ARG;
    return check_prime(p);
}

}  // namespace



extern "C" {

cup_status cup_create(cup_handle **handle, int device)
{
    if (!handle) return CUP_ERR_ARG;
    *handle = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return CUP_ERR_ARG;
    cup_handle *h = new (std::nothrow) cup_handle();
    if (!h) return CUP_ERR_NOMEM;
    h->device = device;
    *handle = h;
    return CUP_OK;
}

cup_status cup_destroy(cup_handle *h)
{
    if (!h) return CUP_ERR_ARG;
    {
        DeviceGuard g(h->device);
        if (h->d_slab) cudaFree(h->d_slab);
        if (h->d_pairs) cudaFree(h->d_pairs);
        if (h->d_count) cudaFree(h->d_count);
        if (h->h_pinned) cudaFreeHost(h->h_pinned);
        if (h->d_err) cudaFree(h->d_err);
        if (h->d_next) cudaFree(h->d_next);
        if (h->d_order) cudaFree(h->d_order);
        for (auto &b : h->bgraphs)
            if (b.exec) cudaGraphExecDestroy(b.exec);
        if (h->d_ws) cudaFree(h->d_ws);
        if (h->copy) cudaStreamDestroy(h->copy);
        if (h->ev_fork) cudaEventDestroy(h->ev_fork);
        for (cudaEvent_t e : h->chunk_ev) cudaEventDestroy(e);
        if (h->d_rank_at) cudaFree(h->d_rank_at);
        if (h->d_backup) cudaFree(h->d_backup);
        if (h->d_wide) cudaFree(h->d_wide);
        if (h->h_rank) cudaFreeHost(h->h_rank);
        for (auto &g2 : h->graphs)
            if (g2.exec) cudaGraphExecDestroy(g2.exec);
        flush_timings(h);
        for (auto e : h->evpool) cudaEventDestroy(e);
    }
    delete h;
    return CUP_OK;
}

cup_status cup_set_option(cup_handle *h, int option, int64_t value)
{
    if (!h) return CUP_ERR_ARG;
    switch (option) {
    case CUP_OPT_ENGINE:
        if (value != CUP_ENGINE_PLAIN && value != CUP_ENGINE_TENSOR) return CUP_ERR_ARG;
        h->engine = (int)value;
        return CUP_OK;
    case CUP_OPT_LEAF_ROWS:
        if (value < 1 || value > CUP_BMAX) return CUP_ERR_ARG;
        h->leaf_rows = (int)value;
        h->user_set[0] = true;
        return CUP_OK;
    case CUP_OPT_WINDOW:
        if (value < 1 || value > CUP_WNMAX) return CUP_ERR_ARG;
        h->window = (int)value;
        h->user_set[1] = true;
        return CUP_OK;
    case CUP_OPT_TC_MIN_K:
        if (value < 1) return CUP_ERR_ARG;
        h->tc_min_k = value;
        h->user_set[2] = true;
        return CUP_OK;
    case CUP_OPT_VALIDATE:
        h->validate = value != 0;
        return CUP_OK;
    case CUP_OPT_PROFILE:
        h->profile = (int)value;
        return CUP_OK;
    case CUP_OPT_SCHEDULE:
        if (value < 0 || value > 2) return CUP_ERR_ARG;
        h->schedule = value ? 1 : 0;
        h->use_graph = value == 1;
        return CUP_OK;
    case CUP_OPT_INT_PATH:
        if (value < 0 || value > 2) return CUP_ERR_ARG;
        h->int_path = (int)value;
        return CUP_OK;
    case CUP_OPT_SHORT_K:
        if (value < 0 || value > SHORT_K_MAX) return CUP_ERR_ARG;
        h->short_k = value;
        return CUP_OK;
    default:
        return CUP_ERR_ARG;
    }
}

cup_status cup_get_stats(cup_handle *h, cup_stats *out)
{
    if (!h || !out) return CUP_ERR_ARG;
    *out = h->stats;
    return CUP_OK;
}

cup_status cup_class_ms(cup_handle *h, double *out8)
{
    if (!h || !out8) return CUP_ERR_ARG;
    for (int i = 0; i < 8; ++i) out8[i] = h->cls_ms[i];
    return CUP_OK;
}

cup_status cup_reset_stats(cup_handle *h)
{
    if (!h) return CUP_ERR_ARG;
    flush_timings(h);
    h->stats = cup_stats{};
    for (int i = 0; i < 8; ++i) h->cls_ms[i] = 0.0;
    return CUP_OK;
}

const char *cup_last_cuda_error(cup_handle *h)
{
    return h ? h->err : "null handle";
}

cup_status cup_factor(cup_handle *h, uint32_t *A, int64_t m, int64_t n, int64_t lda, uint32_t p,
                      int64_t *d_profile, int64_t *d_ipiv, int64_t *rank, void *stream)
{
    if (!h || !rank || m < 0 || n < 0 || lda < (n > 0 ? n : 1)) return CUP_ERR_ARG;
    CK(check_prime(p));
    *rank = 0;
    if (m == 0 || n == 0) return CUP_OK;
    if (!A || !d_profile || !d_ipiv) return CUP_ERR_ARG;
    if (n >= (int64_t)1 << 31) return CUP_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    CK(ensure_base(h));
    return factor_impl(h, A, m, n, lda, p, d_profile, d_ipiv, rank, (cudaStream_t)stream, InputSrc{});
}

cup_status cup_factor_host(cup_handle *h, const uint32_t *hA, int64_t ldh, uint32_t *hOut, uint32_t *A, int64_t m,
                           int64_t n, int64_t lda, uint32_t p, int64_t *d_profile, int64_t *d_ipiv, int64_t *rank,
                           void *stream)
{
    if (!h || !rank || m < 0 || n < 0 || lda < (n > 0 ? n : 1) || ldh < (n > 0 ? n : 1)) return CUP_ERR_ARG;
    CK(check_prime(p));
    *rank = 0;
    if (m == 0 || n == 0) return CUP_OK;
    if (!hA || !hOut || !A || !d_profile || !d_ipiv) return CUP_ERR_ARG;
    if (n >= (int64_t)1 << 31) return CUP_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    CK(ensure_base(h));
    cudaStream_t st = (cudaStream_t)stream;
    InputSrc src;
    src.host = hA;
    src.ldh = ldh;
    CK(factor_impl(h, A, m, n, lda, p, d_profile, d_ipiv, rank, st, src));
    CU(cudaMemcpy2DAsync(hOut, (size_t)ldh * 4, A, (size_t)lda * 4, (size_t)n * 4, (size_t)m, cudaMemcpyDeviceToHost,
                         st));
    return sync_stream(h, st);
}

cup_status cup_factor_u8(cup_handle *h, uint8_t *A, int64_t m, int64_t n, int64_t lda, uint32_t p,
                         int64_t *d_profile, int64_t *d_ipiv, int64_t *rank, void *stream)
{
    if (!h || !rank || m < 0 || n < 0 || lda < (n > 0 ? n : 1)) return CUP_ERR_ARG;
    CK(check_u8(p));
    *rank = 0;
    if (m == 0 || n == 0) return CUP_OK;
    if (!A || !d_profile || !d_ipiv) return CUP_ERR_ARG;
    if (n >= (int64_t)1 << 31) return CUP_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    CK(ensure_base(h));
    CK(ensure_wide(h, (size_t)m * (size_t)n * 4));
    cudaStream_t st = (cudaStream_t)stream;
    InputSrc src;
    src.esize = 1;
    src.dev8 = A;
    src.ld8 = lda;
    CK(factor_impl(h, h->d_wide, m, n, n, p, d_profile, d_ipiv, rank, st, src));
    CU(launch_narrow_u8(A, lda, h->d_wide, n, m, n, st));
    h->stats.launches += 1;
    return sync_stream(h, st);
}

cup_status cup_factor_host_u8(cup_handle *h, const uint8_t *hA, int64_t ldh, uint8_t *hOut, uint8_t *A, int64_t m,
                              int64_t n, int64_t lda, uint32_t p, int64_t *d_profile, int64_t *d_ipiv, int64_t *rank,
                              void *stream)
{
    if (!h || !rank || m < 0 || n < 0 || lda < (n > 0 ? n : 1) || ldh < (n > 0 ? n : 1)) return CUP_ERR_ARG;
    CK(check_u8(p));
    *rank = 0;
    if (m == 0 || n == 0) return CUP_OK;
    if (!hA || !hOut || !A || !d_profile || !d_ipiv) return CUP_ERR_ARG;
    if (n >= (int64_t)1 << 31) return CUP_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    CK(ensure_base(h));
    CK(ensure_wide(h, (size_t)m * (size_t)n * 4));
    cudaStream_t st = (cudaStream_t)stream;
    InputSrc src;
    src.host = hA;
    src.ldh = ldh;
    src.esize = 1;
    src.dev8 = A;
    src.ld8 = lda;
    CK(factor_impl(h, h->d_wide, m, n, n, p, d_profile, d_ipiv, rank, st, src));
    CU(launch_narrow_u8(A, lda, h->d_wide, n, m, n, st));
    h->stats.launches += 1;
    CU(cudaMemcpy2DAsync(hOut, (size_t)ldh, A, (size_t)lda, (size_t)n, (size_t)m, cudaMemcpyDeviceToHost, st));
    return sync_stream(h, st);
}

cup_status cup_rank_profile(cup_handle *h, uint32_t *A, int64_t m, int64_t n, int64_t lda,
                            uint32_t p, int64_t *d_profile, int64_t *rank, void *stream)
{
    if (!h) return CUP_ERR_ARG;
    int64_t k = m < n ? m : n;
    if (k <= 0) return cup_factor(h, A, m, n, lda, p, d_profile, d_profile, rank, stream);
    int64_t *d_ipiv = nullptr;
    {
        DeviceGuard g(h->device);
        CU(cudaMalloc(&d_ipiv, (size_t)k * sizeof(int64_t)));
    }
    cup_status s = cup_factor(h, A, m, n, lda, p, d_profile, d_ipiv, rank, stream);
    {
        DeviceGuard g(h->device);
        cudaFree(d_ipiv);
    }
    return s;
}

cup_status cup_mm_sub(cup_handle *h, uint32_t *C, int64_t ldc, const uint32_t *A, int64_t lda,
                      const uint32_t *B, int64_t ldb, int64_t M, int64_t N, int64_t K, uint32_t p,
                      int engine, void *stream)
{
    if (!h || M < 0 || N < 0 || K < 0) return CUP_ERR_ARG;
    if (engine != CUP_ENGINE_PLAIN && engine != CUP_ENGINE_TENSOR) return CUP_ERR_ARG;
    CK(check_prime(p));
    if (M == 0 || N == 0 || K == 0) return CUP_OK;
    if (!C || !A || !B || ldc < N || lda < K || ldb < N) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    CK(ensure_base(h));
    CK(mm_sub(h, C, ldc, A, lda, B, ldb, M, N, K, make_modp(p), engine, (cudaStream_t)stream));
    CK(check_device_error(h, (cudaStream_t)stream));
    return CUP_OK;
}

cup_status cup_trsm_ruu(cup_handle *h, const uint32_t *U, int64_t ldu, uint32_t *B, int64_t ldb,
                        int64_t m, int64_t n, uint32_t p, void *stream)
{
    if (!h || m < 0 || n < 0) return CUP_ERR_ARG;
    CK(check_prime(p));
    if (m == 0 || n == 0) return CUP_OK;
    if (!U || !B || ldu < n || ldb < n) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    CK(ensure_base(h));
    CK(trsm_ruu(h, U, ldu, B, ldb, m, n, make_modp(p), h->engine, (cudaStream_t)stream));
    CK(check_device_error(h, (cudaStream_t)stream));
    return CUP_OK;
}

cup_status cup_laswp_cols(cup_handle *h, uint32_t *A, int64_t lda, int64_t row0, int64_t nrows,
                          const int64_t *d_ipiv, int64_t k0, int64_t k1, void *stream)
{
    if (!h || row0 < 0 || nrows < 0 || k0 < 0 || k1 < k0) return CUP_ERR_ARG;
    if (nrows == 0 || k1 == k0) return CUP_OK;
    if (!A || !d_ipiv || lda < 1) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    CK(ensure_base(h));
    Ctx c{h, A, lda, lda, make_modp(2), const_cast<int64_t *>(d_ipiv), nullptr, (cudaStream_t)stream};
    CK(laswp(c, row0, nrows, k0, k1));
    return CUP_OK;
}

cup_status cup_det(cup_handle *h, uint32_t *A, int64_t n, int64_t lda, uint32_t p, uint32_t *det,
                   void *stream)
{
    if (!h || !det || n < 0 || lda < (n > 0 ? n : 1)) return CUP_ERR_ARG;
    CK(check_prime(p));
    if (n == 0) { *det = 1u % p; return CUP_OK; }
    if (!A) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    CK(ensure_base(h));
    return det_impl(h, A, n, lda, p, det, (cudaStream_t)stream, InputSrc{});
}

cup_status cup_det_u8(cup_handle *h, uint8_t *A, int64_t n, int64_t lda, uint32_t p, uint32_t *det, void *stream)
{
    if (!h || !det || n < 0 || lda < (n > 0 ? n : 1)) return CUP_ERR_ARG;
    CK(check_u8(p));
    if (n == 0) { *det = 1u % p; return CUP_OK; }
    if (!A) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    CK(ensure_base(h));
    CK(ensure_wide(h, (size_t)n * (size_t)n * 4));
    cudaStream_t st = (cudaStream_t)stream;
    InputSrc src;
    src.esize = 1;
    src.dev8 = A;
    src.ld8 = lda;
    CK(det_impl(h, h->d_wide, n, n, p, det, st, src));
    CU(launch_narrow_u8(A, lda, h->d_wide, n, n, n, st));
    h->stats.launches += 1;
    return sync_stream(h, st);
}

cup_status cup_inverse(cup_handle *h, uint32_t *A, int64_t n, int64_t lda, uint32_t p, void *stream)
{
    if (!h || n < 0 || lda < (n > 0 ? n : 1)) return CUP_ERR_ARG;
    CK(check_prime(p));
    if (n == 0) return CUP_OK;
    if (!A) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    CK(ensure_base(h));
    return inverse_impl(h, A, n, lda, p, (cudaStream_t)stream, InputSrc{});
}

cup_status cup_inverse_u8(cup_handle *h, uint8_t *A, int64_t n, int64_t lda, uint32_t p, void *stream)
{
    if (!h || n < 0 || lda < (n > 0 ? n : 1)) return CUP_ERR_ARG;
    CK(check_u8(p));
    if (n == 0) return CUP_OK;
    if (!A) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    CK(ensure_base(h));
    CK(ensure_wide(h, (size_t)n * (size_t)n * 4));
    cudaStream_t st = (cudaStream_t)stream;
    InputSrc src;
    src.esize = 1;
    src.dev8 = A;
    src.ld8 = lda;
    const cup_status s = inverse_impl(h, h->d_wide, n, n, p, st, src);
    if (s != CUP_OK && s != CUP_SINGULAR) return s;
    // the inverse, or the [C\U] factors of a singular input
    CU(launch_narrow_u8(A, lda, h->d_wide, n, n, n, st));
    h->stats.launches += 1;
    CK(sync_stream(h, st));
    return s;
}

cup_status cup_rref(cup_handle *h, uint32_t *A, int64_t m, int64_t n, int64_t lda, uint32_t p,
                    int64_t *d_profile, int64_t *rank, uint32_t *X, int64_t ldx, void *stream)
{
    if (!h || !rank || m < 0 || n < 0 || lda < (n > 0 ? n : 1)) return CUP_ERR_ARG;
    if (X && ldx < (n > 0 ? n : 1)) return CUP_ERR_ARG;
    CK(check_prime(p));
    *rank = 0;
    if (m == 0 || n == 0) {
        if (X && n > 0) {
            DeviceGuard g(h->device);
            CU(launch_fill(X, ldx, n, n, 1, (cudaStream_t)stream));
            CU(cudaStreamSynchronize((cudaStream_t)stream));
        }
        return CUP_OK;
    }
    if (!A || !d_profile) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t kmn = m < n ? m : n;
    int64_t *d_ipiv = nullptr;
    CU(cudaMalloc(&d_ipiv, (size_t)kmn * sizeof(int64_t)));
    int64_t r = 0;
    const ModP M = make_modp(p);
    cup_status s = cup_factor(h, A, m, n, lda, p, d_profile, d_ipiv, &r, stream);
    if (s == CUP_OK) s = red_col_ech(h, A, m, n, lda, r, d_profile, M, h->engine, st);
    if (s == CUP_OK && X) {
        // X = P^T [X1 X2; 0 I]
        s = cuda_ok(h, launch_copy(X, ldx, A, lda, r, n, st));
        if (s == CUP_OK) s = cuda_ok(h, launch_fill(X + r * ldx, ldx, n - r, r, 0, st));
        if (s == CUP_OK) s = cuda_ok(h, launch_fill(X + r * ldx + r, ldx, n - r, n - r, 1, st));
        if (s == CUP_OK) s = cuda_ok(h, launch_row_swaps(X, ldx, n, d_ipiv, r, 0, 0, 1, 0, st));
    }
    if (s == CUP_OK) {
        // R = [I_r 0; R2 0] with the profile loop undone (swaps in reverse order)
        s = cuda_ok(h, launch_fill(A, lda, r, n, 1, st));
        if (s == CUP_OK) s = cuda_ok(h, launch_row_swaps(A, lda, n, d_profile, r, 0, 0, 1, 0, st));
    }
    if (s == CUP_OK) s = check_device_error(h, st);
    if (s == CUP_OK) *rank = r;
    cudaFree(d_ipiv);
    return s;
}

cup_status cup_ple(cup_handle *h, uint32_t *A, int64_t m, int64_t n, int64_t lda, uint32_t p, int64_t *d_profile,
                   int64_t *d_ipiv, int64_t *rank, void *stream)
{
    if (!h || !rank || m < 0 || n < 0 || lda < (n > 0 ? n : 1)) return CUP_ERR_ARG;
    CK(check_prime(p));
    *rank = 0;
    if (m == 0 || n == 0) return CUP_OK;
    if (!A || !d_profile || !d_ipiv) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *T = nullptr;
    CU(cudaMalloc(&T, (size_t)m * (size_t)n * sizeof(uint32_t)));
    int64_t r = 0;
    cup_status s = cuda_ok(h, launch_transpose(T, m, A, lda, m, n, st));          // T = A^T (n x m)
    if (s == CUP_OK) s = cup_factor(h, T, n, m, m, p, d_profile, d_ipiv, &r, stream);
    if (s == CUP_OK) s = cuda_ok(h, launch_transpose(A, lda, T, m, n, m, st));   // [L\E] = [C\U]^T
    if (s == CUP_OK) s = cuda_ok(h, cudaStreamSynchronize(st));
    if (s == CUP_OK) *rank = r;
    cudaFree(T);
    return s;
}

cup_status cup_nullspace(cup_handle *h, uint32_t *A, int64_t m, int64_t n, int64_t lda, uint32_t p,
                         uint32_t *Nb, int64_t ldn, int64_t *rank, void *stream)
{
    if (!h || !rank || m < 0 || n < 0 || lda < (n > 0 ? n : 1) || ldn < (n > 0 ? n : 1)) return CUP_ERR_ARG;
    CK(check_prime(p));
    *rank = 0;
    if (n == 0) return CUP_OK;
    if (!Nb) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (m == 0) {
        // every vector is in the nullspace: the identity
        CU(launch_fill(Nb, ldn, n, n, 1, st));
        CU(cudaStreamSynchronize(st));
        return CUP_OK;
    }
    if (!A) return CUP_ERR_ARG;
    const int64_t kmn = m < n ? m : n;
    int64_t *d_ipiv = nullptr, *d_prof = nullptr;
    CU(cudaMalloc(&d_ipiv, (size_t)kmn * sizeof(int64_t)));
    if (cudaMalloc(&d_prof, (size_t)kmn * sizeof(int64_t)) != cudaSuccess) {
        cudaFree(d_ipiv);
        return CUP_ERR_NOMEM;
    }
    int64_t r = 0;
    const ModP M = make_modp(p);
    cup_status s = cup_factor(h, A, m, n, lda, p, d_prof, d_ipiv, &r, stream);
    if (s == CUP_OK) s = red_col_ech(h, A, m, n, lda, r, d_prof, M, h->engine, st);
    if (s == CUP_OK && r < n) {
        // columns r .. n-1 of X = P^T [X1 X2; 0 I]: P^T [X2; I_{n-r}]
        s = cuda_ok(h, launch_copy(Nb, ldn, A + r, lda, r, n - r, st));
        if (s == CUP_OK) s = cuda_ok(h, launch_fill(Nb + r * ldn, ldn, n - r, n - r, 1, st));
        if (s == CUP_OK) s = cuda_ok(h, launch_row_swaps(Nb, ldn, n - r, d_ipiv, r, 0, 0, 1, 0, st));
    }
    if (s == CUP_OK) s = check_device_error(h, st);
    if (s == CUP_OK) *rank = r;
    cudaFree(d_ipiv);
    cudaFree(d_prof);
    return s;
}

cup_status cup_inplace_mm(cup_handle *h, uint32_t *A, int64_t m, int64_t lda, uint32_t *B, int64_t n,
                          int64_t ldb, uint32_t p, int64_t *rank, void *stream)
{
    if (!h || !rank || m < 0 || n < 0 || lda < (m > 0 ? m : 1) || ldb < (n > 0 ? n : 1)) return CUP_ERR_ARG;
    CK(check_prime(p));
    *rank = 0;
    if (m == 0 || n == 0) return CUP_OK;
    if (!A || !B) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    int64_t *d_ipiv = nullptr, *d_prof = nullptr;
    CU(cudaMalloc(&d_ipiv, (size_t)m * sizeof(int64_t)));
    if (cudaMalloc(&d_prof, (size_t)m * sizeof(int64_t)) != cudaSuccess) {
        cudaFree(d_ipiv);
        return CUP_ERR_NOMEM;
    }
    int64_t r = 0;
    const ModP M = make_modp(p);
    // A = C U P with A <- [C\U]; the zero blocks of that storage make C an m x m
    // lower and U an m x m unit upper triangle, so A B = C (U (P B)).
    cup_status s = cup_factor(h, A, m, m, lda, p, d_prof, d_ipiv, &r, stream);
    if (s == CUP_OK) s = cuda_ok(h, launch_row_swaps(B, ldb, n, d_ipiv, r, 0, 0, 0, 0, st));    // B <- P B
    if (s == CUP_OK) s = tri_op(h, TRI_LEFT | TRI_UPPER | TRI_UNIT, A, lda, B, ldb, m, n, M, h->engine, st);
    if (s == CUP_OK) s = tri_op(h, TRI_LEFT, A, lda, B, ldb, m, n, M, h->engine, st);          // B <- C B
    if (s == CUP_OK) s = trlum(h, A, lda, m, 0, M, h->engine, st);                              // A <- C U
    if (s == CUP_OK) s = cuda_ok(h, launch_col_swaps(A, lda, m, d_ipiv, r, 1, st));             // A <- A P
    if (s == CUP_OK) s = check_device_error(h, st);
    if (s == CUP_OK) *rank = r;
    cudaFree(d_ipiv);
    cudaFree(d_prof);
    return s;
}

cup_status cup_solve(cup_handle *h, uint32_t *A, int64_t m, int64_t n, int64_t lda, uint32_t *B,
                     int64_t k, int64_t ldb, uint32_t *X, int64_t ldx, uint32_t p, int64_t *rank,
                     void *stream)
{
    if (!h || !rank || m < 0 || n < 0 || k < 0 || lda < (n > 0 ? n : 1)) return CUP_ERR_ARG;
    if (ldb < (k > 0 ? k : 1) || ldx < (k > 0 ? k : 1)) return CUP_ERR_ARG;
    CK(check_prime(p));
    *rank = 0;
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (k == 0) return CUP_OK;
    if (n > 0 && !X) return CUP_ERR_ARG;
    if (m == 0 || n == 0) {
        if (n > 0) CU(launch_fill(X, ldx, n, k, 0, st));
        int *d_flag = nullptr;
        CU(cudaMalloc(&d_flag, sizeof(int)));
        CU(cudaMemsetAsync(d_flag, 0, sizeof(int), st));
        cup_status s = cuda_ok(h, launch_any_nonzero(B, ldb, m, k, d_flag, st));
        int hf = 0;
        if (s == CUP_OK) s = cuda_ok(h, cudaMemcpyAsync(&hf, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        if (s == CUP_OK) s = cuda_ok(h, cudaStreamSynchronize(st));
        cudaFree(d_flag);
        if (s == CUP_OK && hf) s = CUP_INCONSISTENT;
        return s;
    }
    if (!A || !B) return CUP_ERR_ARG;
    const int64_t kmn = m < n ? m : n;
    const ModP M = make_modp(p);
    int64_t *d_idx = nullptr;
    uint32_t *d_L = nullptr, *d_Y = nullptr, *d_C = nullptr;
    int *d_flag = nullptr;
    CU(cudaMalloc(&d_idx, 2 * (size_t)kmn * sizeof(int64_t)));
    int64_t r = 0;
    cup_status s = cup_factor(h, A, m, n, lda, p, d_idx, d_idx + kmn, &r, stream);
    const int64_t *d_prof = d_idx, *d_ipiv = d_idx + kmn;
    const int64_t rr = r > 0 ? r : 1;
    if (s == CUP_OK) s = cuda_ok(h, cudaMalloc(&d_L, (size_t)rr * rr * sizeof(uint32_t)));
    if (s == CUP_OK) s = cuda_ok(h, cudaMalloc(&d_Y, (size_t)rr * k * sizeof(uint32_t)));
    if (s == CUP_OK) s = cuda_ok(h, cudaMalloc(&d_C, (size_t)m * rr * sizeof(uint32_t)));
    if (s == CUP_OK) s = cuda_ok(h, cudaMalloc(&d_flag, sizeof(int)));
    if (s == CUP_OK) s = cuda_ok(h, cudaMemsetAsync(d_flag, 0, sizeof(int), st));
    if (s == CUP_OK && r > 0) {
        // y1 = L1^{-1} b[profile], L1 = the profile rows of C (lower triangular)
        s = cuda_ok(h, launch_gather_rows(d_L, r, A, lda, d_prof, r, r, st));
        if (s == CUP_OK) s = cuda_ok(h, launch_gather_rows(d_Y, k, B, ldb, d_prof, r, k, st));
        if (s == CUP_OK) s = tri_op(h, TRI_LEFT | TRI_SOLVE, d_L, r, d_Y, k, r, k, M, h->engine, st);
        // consistency: b - C[:, 0:r] y1 must vanish (C without U's part above the diagonal)
        if (s == CUP_OK) s = cuda_ok(h, launch_copy(d_C, r, A, lda, m, r, st));
        if (s == CUP_OK) s = cuda_ok(h, launch_zero_upper(d_C, r, r, st));
        if (s == CUP_OK) s = mm_sub(h, B, ldb, d_C, r, d_Y, k, m, k, r, M, h->engine, st, 0);
        // z1 = U1^{-1} y1
        if (s == CUP_OK) s = tri_op(h, TRI_LEFT | TRI_UPPER | TRI_UNIT | TRI_SOLVE, A, lda, d_Y, k, r, k, M,
                                    h->engine, st);
    }
    if (s == CUP_OK) s = cuda_ok(h, launch_any_nonzero(B, ldb, m, k, d_flag, st));
    // x = P^T [z1; 0]
    if (s == CUP_OK && r > 0) s = cuda_ok(h, launch_copy(X, ldx, d_Y, k, r, k, st));
    if (s == CUP_OK) s = cuda_ok(h, launch_fill(X + r * ldx, ldx, n - r, k, 0, st));
    if (s == CUP_OK) s = cuda_ok(h, launch_row_swaps(X, ldx, k, d_ipiv, r, 0, 0, 1, 0, st));
    int hf = 0;
    if (s == CUP_OK) s = cuda_ok(h, cudaMemcpyAsync(h->h_pinned + 4, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (s == CUP_OK) s = check_device_error(h, st);
    if (s == CUP_OK) hf = h->h_pinned[4];
    if (s == CUP_OK) {
        *rank = r;
        if (hf) s = CUP_INCONSISTENT;
    }
    cudaFree(d_idx);
    if (d_L) cudaFree(d_L);
    if (d_Y) cudaFree(d_Y);
    if (d_C) cudaFree(d_C);
    if (d_flag) cudaFree(d_flag);
    return s;
}

static int tri_flags(int flags, bool solve)
{
    return ((flags & CUP_LEFT) ? TRI_LEFT : 0) | ((flags & CUP_UPPER) ? TRI_UPPER : 0) |
           ((flags & CUP_UNIT) ? TRI_UNIT : 0) | (solve ? TRI_SOLVE : 0);
}

static cup_status tri_entry(cup_handle *h, int flags, bool solve, const uint32_t *T, int64_t ldt, uint32_t *B,
                            int64_t ldb, int64_t rows, int64_t cols, uint32_t p, void *stream)
{
    if (!h || rows < 0 || cols < 0 || (flags & ~7)) return CUP_ERR_ARG;
    CK(check_prime(p));
    if (rows == 0 || cols == 0) return CUP_OK;
    const int64_t n = (flags & CUP_LEFT) ? rows : cols;
    if (!T || !B || ldt < n || ldb < cols) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    CK(ensure_base(h));
    CK(tri_op(h, tri_flags(flags, solve), T, ldt, B, ldb, rows, cols, make_modp(p), h->engine,
              (cudaStream_t)stream));
    CK(check_device_error(h, (cudaStream_t)stream));
    return CUP_OK;
}

cup_status cup_trsm(cup_handle *h, int flags, const uint32_t *T, int64_t ldt, uint32_t *B, int64_t ldb,
                    int64_t rows, int64_t cols, uint32_t p, void *stream)
{
    return tri_entry(h, flags, true, T, ldt, B, ldb, rows, cols, p, stream);
}

cup_status cup_trmm(cup_handle *h, int flags, const uint32_t *T, int64_t ldt, uint32_t *B, int64_t ldb,
                    int64_t rows, int64_t cols, uint32_t p, void *stream)
{
    return tri_entry(h, flags, false, T, ldt, B, ldb, rows, cols, p, stream);
}

cup_status cup_trtri(cup_handle *h, int flags, uint32_t *T, int64_t ldt, int64_t n, uint32_t p, void *stream)
{
    if (!h || n < 0 || (flags & ~7)) return CUP_ERR_ARG;
    CK(check_prime(p));
    if (n == 0) return CUP_OK;
    if (!T || ldt < n) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    CK(ensure_base(h));
    CK(trtri(h, (flags & CUP_UPPER) != 0, (flags & CUP_UNIT) != 0, T, ldt, n, make_modp(p), h->engine,
             (cudaStream_t)stream));
    CK(check_device_error(h, (cudaStream_t)stream));
    return CUP_OK;
}

cup_status cup_trulm(cup_handle *h, uint32_t *A, int64_t lda, int64_t n, uint32_t p, void *stream)
{
    if (!h || n < 0) return CUP_ERR_ARG;
    CK(check_prime(p));
    if (n == 0) return CUP_OK;
    if (!A || lda < n) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    CK(ensure_base(h));
    CK(trulm(h, A, lda, n, make_modp(p), h->engine, (cudaStream_t)stream));
    CK(check_device_error(h, (cudaStream_t)stream));
    return CUP_OK;
}

cup_status cup_trlum(cup_handle *h, uint32_t *A, int64_t lda, int64_t n, uint32_t p, void *stream)
{
    if (!h || n < 0) return CUP_ERR_ARG;
    CK(check_prime(p));
    if (n == 0) return CUP_OK;
    if (!A || lda < n) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    CK(ensure_base(h));
    CK(trlum(h, A, lda, n, 1, make_modp(p), h->engine, (cudaStream_t)stream));
    CK(check_device_error(h, (cudaStream_t)stream));
    return CUP_OK;
}

// Reads the tuning table {"entries": [{"key": number, ...}, ...]}: every object of the
// entries array is one rule; numbers are read as integers (fractions dropped), string,
// array and object values are skipped, unknown keys are ignored.
static bool parse_tuning(const char *t, std::vector<cup_handle::TuneRule> &out)
{
    const char *e = strstr(t, "\"entries\"");
    if (!e) return false;
    const char *c = strchr(e, '[');
    if (!c) return false;
    ++c;
    auto ws = [&]() { while (*c == ' ' || *c == '\n' || *c == '\r' || *c == '\t' || *c == ',') ++c; };
    auto skip_value = [&]() -> bool {
        if (*c == '"') {
            for (++c; *c && *c != '"'; ++c)
                if (*c == '\\' && c[1]) ++c;
            if (!*c) return false;
            ++c;
            return true;
        }
        if (*c == '[' || *c == '{') {
            int depth = 0;
            bool str = false;
            for (; *c; ++c) {
                if (str) { if (*c == '\\' && c[1]) ++c; else if (*c == '"') str = false; continue; }
                if (*c == '"') str = true;
                else if (*c == '[' || *c == '{') ++depth;
                else if ((*c == ']' || *c == '}') && --depth == 0) { ++c; return true; }
            }
            return false;
        }
        for (const char *lit : {"true", "false", "null"}) {
            const size_t k = strlen(lit);
            if (strncmp(c, lit, k) == 0) {
                c += k;
                return true;
            }
        }
        return false;
    };
    for (;;) {
        ws();
        if (*c == ']') return true;
        if (*c != '{') return false;
        ++c;
        cup_handle::TuneRule r;
        for (;;) {
            ws();
            if (*c == '}') { ++c; break; }
            if (*c != '"') return false;
            const char *k0 = ++c;
            while (*c && *c != '"') ++c;
            if (!*c) return false;
            const std::string key(k0, (size_t)(c - k0));
            ++c;
            ws();
            if (*c != ':') return false;
            ++c;
            ws();
            if (*c == '-' || (*c >= '0' && *c <= '9')) {
                char *endp = nullptr;
                const double v = strtod(c, &endp);
                if (endp == c) return false;
                c = endp;
                const int64_t iv = (int64_t)v;
                if (key == "limbs") r.limbs = iv;
                else if (key == "tall") r.tall = iv;
                else if (key == "min_lo") r.min_lo = iv;
                else if (key == "min_hi") r.min_hi = iv;
                else if (key == "leaf_rows") r.leaf_rows = iv;
                else if (key == "window") r.window = iv;
                else if (key == "tc_min_k") r.tc_min_k = iv;
            } else if (!skip_value()) {
                return false;
            }
        }
        out.push_back(r);
    }
}

cup_status cup_set_tuning(cup_handle *h, const char *table)
{
    if (!h) return CUP_ERR_ARG;
    if (!table) {
        h->tuning.clear();
        return CUP_OK;
    }
    std::vector<cup_handle::TuneRule> rules;
    if (!parse_tuning(table, rules)) return CUP_ERR_ARG;
    h->tuning.swap(rules);
    return CUP_OK;
}

cup_status cup_selftest_wait(cup_handle *h, int64_t limit_us, void *stream)
{
    if (!h || limit_us < 1 || limit_us > 10000000) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    CK(ensure_base(h));
    cudaStream_t st = (cudaStream_t)stream;
    CU(cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
    CU(launch_selftest_wait(h->d_err, (uint64_t)limit_us * 1000ull, CUP_DEVERR_SELFTEST, st));
    h->stats.launches += 1;
    return check_device_error(h, st);
}

cup_status cup_factor_batched(cup_handle *h, const cup_batch_item *d_items, int64_t count, int64_t *d_rank,
                              uint32_t *d_det, void *stream)
{
    if (!h || count < 0) return CUP_ERR_ARG;
    if (count == 0) return CUP_OK;
    if (!d_items || !d_rank) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    if (count > INT32_MAX) return CUP_ERR_UNSUPPORTED;
    if (!h->d_next) CU(cudaMalloc(&h->d_next, sizeof(unsigned long long)));
    if (count > h->order_cap) {
        if (h->d_order) cudaFree(h->d_order);
        h->d_order = nullptr;
        h->order_cap = 0;
        CU(cudaMalloc(&h->d_order, (size_t)count * sizeof(int)));
        h->order_cap = count;
        ++h->gen;
    }
    int nsm = 0;
    CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    // one CTA per SM (each holds a 32-row panel of up to 1024 columns in shared memory)
    const int64_t grid = count < (int64_t)nsm ? count : (int64_t)nsm;
    cudaStream_t st = (cudaStream_t)stream;
    // a repeated call with the same arguments on a stream of its own replays one graph
    // (work counter reset, work order, factor kernel)
    const bool capturable = st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
    cup_handle::BatchGraph *bg = nullptr;
    for (auto &e : h->bgraphs)
        if (e.items == d_items && e.count == count && e.rank == d_rank && e.det == d_det && e.st == st) bg = &e;
    if (bg && bg->gen != h->gen) {
        if (bg->exec) cudaGraphExecDestroy(bg->exec);
        bg->exec = nullptr;
        bg->gen = h->gen;
    }
    if (bg && capturable && !bg->exec && !bg->no_capture) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const cudaError_t e1 = launch_cup_batched(d_items, count, d_rank, d_det, h->d_next, h->d_order, (int)grid, st);
            const cudaError_t e2 = cudaStreamEndCapture(st, &graph);
            if (e1 == cudaSuccess && e2 == cudaSuccess && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
                exec = nullptr;
            if (graph) cudaGraphDestroy(graph);
        }
        if (!exec) {
            cudaGetLastError();
            bg->no_capture = true;
        }
        bg->exec = exec;
    }
    if (bg && bg->exec && capturable) {
        CU(cudaGraphLaunch(bg->exec, st));
    } else {
        if (!bg && capturable) {
            if (h->bgraphs.size() > 16) {
                if (h->bgraphs.front().exec) cudaGraphExecDestroy(h->bgraphs.front().exec);
                h->bgraphs.erase(h->bgraphs.begin());
            }
            h->bgraphs.push_back(cup_handle::BatchGraph{d_items, count, d_rank, d_det, st, h->gen, nullptr, false});
        }
        CU(launch_cup_batched(d_items, count, d_rank, d_det, h->d_next, h->d_order, (int)grid, st));
    }
    h->stats.launches += 2;
    return CUP_OK;
}

// ---------------------------------------------------------------------------
// Multi-modular integer determinant and rank (Sec. 1: reduction to prime fields)
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

// log2 of the product of the Euclidean norms of the nonzero rows of A: a bound
// on |det A| (Hadamard) and on every minor of A.
cup_status int_bound(cup_handle *h, const int64_t *A, int64_t m, int64_t n, int64_t lda, double *out, cudaStream_t st)
{
    *out = 0.0;
    if (m == 0 || n == 0) return CUP_OK;
    double *d = nullptr;
    CU(cudaMalloc(&d, (size_t)m * sizeof(double)));
    std::vector<double> v((size_t)m);
    cup_status s = cuda_ok(h, launch_row_log2norm(A, lda, m, n, d, st));
    if (s == CUP_OK)
        s = cuda_ok(h, cudaMemcpyAsync(v.data(), d, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (s == CUP_OK) s = sync_stream(h, st);
    cudaFree(d);
    CK(s);
    double sum = 0.0;
    for (double x : v)
        if (x > 0.0) sum += x;            // zero rows (-1e300) and unit rows add nothing
    *out = sum * (1.0 + 1e-12) + 1e-9;    // the host sum's rounding, upward
    return CUP_OK;
}

// The primes to use: the caller's (checked: prime, below 2^31, pairwise distinct),
// or, if none are given, the largest primes below 2^31 until their product exceeds
// 2^need.
cup_status int_primes(const uint32_t *given, int64_t K, double need, std::vector<uint32_t> &out)
{
    out.clear();
    if (given) {
        if (K <= 0) return CUP_ERR_ARG;
        out.assign(given, given + K);
        for (uint32_t q : out) CK(check_prime(q));
        std::vector<uint32_t> srt = out;
        std::sort(srt.begin(), srt.end());
        for (size_t i = 1; i < srt.size(); ++i)
            if (srt[i] == srt[i - 1]) return CUP_ERR_ARG;
        return CUP_OK;
    }
    double have = 0.0;
    uint32_t q = 1u << 31;
    while (out.empty() || have <= need) {
        uint32_t nx = 0;
        if (cup_internal_primes_below(q, 1, &nx) != 1) return CUP_ERR_UNSUPPORTED;
        out.push_back(nx);
        have += std::log2((double)nx);
        q = nx;
    }
    return CUP_OK;
}

double log2_product(const std::vector<uint32_t> &pr)
{
    double s = 0.0;
    for (uint32_t q : pr) s += std::log2((double)q);
    return s * (1.0 - 1e-12);             // downward
}

// rank (and det, square A) of A mod each prime: batched CUP for small images,
// one full-device CUP per prime otherwise.
cup_status int_residues(cup_handle *h, const int64_t *A, int64_t m, int64_t n, int64_t lda,
                        const std::vector<uint32_t> &pr, int64_t *ranks, uint32_t *dets, cudaStream_t st)
{
    const int64_t K = (int64_t)pr.size();
    const int64_t kmn = m < n ? m : n;
    const size_t plane = (size_t)m * (size_t)n;
    uint32_t *d_pr = nullptr;
    CU(cudaMalloc(&d_pr, (size_t)K * sizeof(uint32_t)));
    cup_status s = cuda_ok(h, cudaMemcpyAsync(d_pr, pr.data(), (size_t)K * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    // Cost model (GB300 measurements): the batched launch runs two images per SM at
    // about 2.3 G field ops/s each; one full-device CUP per prime runs at about
    // 450 G ops/s at 1024^2 plus about a millisecond of launches and syncs.
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
    const double ops = 2.0 * (double)m * n * kmn - (double)(m + n) * kmn * kmn + 2.0 / 3.0 * (double)kmn * kmn * kmn;
    const double waves = std::ceil((double)K / (2.0 * nsm));
    const double t_batch = waves * ops / 2.3e9;
    const double t_seq = (double)K * (ops / 4.5e11 + 1.0e-3);
    const bool fits = kmn <= 2048 && (double)K * (double)plane * 4.0 <= 64.0 * (1ull << 30);
    const bool batched = fits && (h->int_path == 1 || (h->int_path == 0 && t_batch < t_seq));
    if (h->int_path == 1 && !fits) {
        cudaFree(d_pr);
        return CUP_ERR_UNSUPPORTED;
    }
    if (s == CUP_OK && batched) {
        // one allocation: residue planes | profile+ipiv per image | items | ranks | dets
        const size_t b_res = (size_t)K * plane * 4, b_idx = (size_t)K * 2 * (size_t)kmn * 8,
                     b_items = (size_t)K * sizeof(cup_batch_item), b_rank = (size_t)K * 8, b_det = (size_t)K * 4;
        auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
        char *base = nullptr;
        s = cuda_ok(h, cudaMalloc(&base, up(b_res) + up(b_idx) + up(b_items) + up(b_rank) + up(b_det)));
        if (s == CUP_OK) {
            uint32_t *R = (uint32_t *)base;
            int64_t *d_idx = (int64_t *)(base + up(b_res));
            cup_batch_item *d_items = (cup_batch_item *)(base + up(b_res) + up(b_idx));
            int64_t *d_rank = (int64_t *)((char *)d_items + up(b_items));
            uint32_t *d_det = (uint32_t *)((char *)d_rank + up(b_rank));
            std::vector<cup_batch_item> items((size_t)K);
            for (int64_t k = 0; k < K; ++k) {
                cup_batch_item &it = items[(size_t)k];
                memset(&it, 0, sizeof(it));
                it.A = R + (size_t)k * plane;
                it.m = m;
                it.n = n;
                it.lda = n;
                it.p = pr[(size_t)k];
                it.profile = d_idx + (size_t)k * 2 * (size_t)kmn;
                it.ipiv = it.profile + kmn;
            }
            std::vector<int64_t> hr((size_t)K);
            std::vector<uint32_t> hd((size_t)K);
            s = cuda_ok(h, launch_reduce_multi(A, lda, m, n, d_pr, (int)K, R, n, (int64_t)plane, st));
            if (s == CUP_OK)
                s = cuda_ok(h, cudaMemcpyAsync(d_items, items.data(), b_items, cudaMemcpyHostToDevice, st));
            if (s == CUP_OK) s = cup_factor_batched(h, d_items, K, d_rank, dets ? d_det : nullptr, st);
            if (s == CUP_OK) s = cuda_ok(h, cudaMemcpyAsync(hr.data(), d_rank, b_rank, cudaMemcpyDeviceToHost, st));
            if (s == CUP_OK && dets)
                s = cuda_ok(h, cudaMemcpyAsync(hd.data(), d_det, b_det, cudaMemcpyDeviceToHost, st));
            if (s == CUP_OK) s = sync_stream(h, st);
            h->stats.launches += 1;
            for (int64_t k = 0; s == CUP_OK && k < K; ++k) {
                if (hr[(size_t)k] < 0) s = CUP_ERR_CUDA;
                ranks[k] = hr[(size_t)k];
                if (dets) dets[k] = hd[(size_t)k];
            }
            cudaFree(base);
        }
    } else if (s == CUP_OK) {
        uint32_t *buf = nullptr, *d_out = nullptr;
        int64_t *d_idx = nullptr;
        s = cuda_ok(h, cudaMalloc(&buf, plane * 4));
        if (s == CUP_OK) s = cuda_ok(h, cudaMalloc(&d_idx, 2 * (size_t)kmn * sizeof(int64_t)));
        if (s == CUP_OK) s = cuda_ok(h, cudaMalloc(&d_out, sizeof(uint32_t)));
        for (int64_t k = 0; s == CUP_OK && k < K; ++k) {
            const uint32_t q = pr[(size_t)k];
            int64_t r = 0;
            s = cuda_ok(h, launch_reduce_multi(A, lda, m, n, d_pr + k, 1, buf, n, (int64_t)plane, st));
            h->stats.launches += 1;
            if (s == CUP_OK) s = cup_factor(h, buf, m, n, n, q, d_idx, d_idx + kmn, &r, st);
            if (s != CUP_OK) break;
            ranks[k] = r;
            if (!dets) continue;
            if (m != n || r < n) {
                dets[k] = 0;
                continue;
            }
            s = cuda_ok(h, launch_det_reduce(buf, n, n, d_idx + kmn, make_modp(q), d_out, st));
            h->stats.launches += 1;
            if (s == CUP_OK)
                s = cuda_ok(h, cudaMemcpyAsync(h->h_pinned, d_out, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            if (s == CUP_OK) s = sync_stream(h, st);
            if (s == CUP_OK) dets[k] = (uint32_t)h->h_pinned[0];
        }
        if (buf) cudaFree(buf);
        if (d_idx) cudaFree(d_idx);
        if (d_out) cudaFree(d_out);
    }
    cudaFree(d_pr);
    return s;
}

}  // namespace

extern "C" {

cup_status cup_primes_below(uint32_t bound, int64_t count, uint32_t *out, int64_t *found)
{
    if (!found || count < 0 || (count > 0 && !out)) return CUP_ERR_ARG;
    *found = cup_internal_primes_below(bound, count, out);
    return CUP_OK;
}

cup_status cup_crt(const uint32_t *residues, const uint32_t *primes, int64_t K, uint32_t *words, int64_t cap,
                   int64_t *nwords, int *sign)
{
    if (!residues || !primes || !nwords || !sign || K <= 0 || cap < 0 || (cap > 0 && !words)) return CUP_ERR_ARG;
    for (int64_t i = 0; i < K; ++i) CK(check_prime(primes[i]));
    std::vector<uint32_t> mag;
    int sg = 0;
    if (!cup_internal_crt(residues, primes, K, mag, sg)) return CUP_ERR_ARG;
    *nwords = (int64_t)mag.size();
    *sign = sg;
    if ((int64_t)mag.size() > cap) return CUP_ERR_TOO_LARGE;
    if (!mag.empty()) memcpy(words, mag.data(), mag.size() * sizeof(uint32_t));
    return CUP_OK;
}

cup_status cup_int_bound(cup_handle *h, const int64_t *A, int64_t m, int64_t n, int64_t lda, double *log2_bound,
                         void *stream)
{
    if (!h || !log2_bound || m < 0 || n < 0 || lda < (n > 0 ? n : 1)) return CUP_ERR_ARG;
    if (m > 0 && n > 0 && !A) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    return int_bound(h, A, m, n, lda, log2_bound, (cudaStream_t)stream);
}

cup_status cup_int_det(cup_handle *h, const int64_t *A, int64_t n, int64_t lda, const uint32_t *primes, int64_t K,
                       uint32_t *words, int64_t cap, int64_t *nwords, int *sign, int64_t *rank, int *certified,
                       int64_t *nprimes, void *stream)
{
    if (!h || !nwords || !sign || !rank || !certified || n < 0 || lda < (n > 0 ? n : 1) || cap < 0 ||
        (cap > 0 && !words))
        return CUP_ERR_ARG;
    *rank = 0;
    *certified = 0;
    if (nprimes) *nprimes = 0;
    if (n == 0) {
        *nwords = 1;
        *sign = 1;
        *certified = 1;
        if (cap < 1) return CUP_ERR_TOO_LARGE;
        words[0] = 1;
        return CUP_OK;
    }
    if (!A) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    double bound = 0.0;
    CK(int_bound(h, A, n, n, lda, &bound, st));
    std::vector<uint32_t> pr;
    CK(int_primes(primes, K, bound + 1.0, pr));     // the symmetric range needs M > 2 |det|
    const int64_t Kp = (int64_t)pr.size();
    std::vector<int64_t> ranks((size_t)Kp);
    std::vector<uint32_t> dets((size_t)Kp);
    CK(ensure_base(h));
    CK(int_residues(h, A, n, n, lda, pr, ranks.data(), dets.data(), st));
    int64_t r = 0;
    for (int64_t x : ranks) r = x > r ? x : r;
    std::vector<uint32_t> mag;
    int sg = 0;
    if (!cup_internal_crt(dets.data(), pr.data(), Kp, mag, sg)) return CUP_ERR_ARG;
    *rank = r;
    *certified = log2_product(pr) > bound + 1.0;
    if (nprimes) *nprimes = Kp;
    *nwords = (int64_t)mag.size();
    *sign = sg;
    if ((int64_t)mag.size() > cap) return CUP_ERR_TOO_LARGE;
    if (!mag.empty()) memcpy(words, mag.data(), mag.size() * sizeof(uint32_t));
    return CUP_OK;
}

cup_status cup_int_rank(cup_handle *h, const int64_t *A, int64_t m, int64_t n, int64_t lda, const uint32_t *primes,
                        int64_t K, int64_t *rank, int *certified, int64_t *nprimes, void *stream)
{
    if (!h || !rank || !certified || m < 0 || n < 0 || lda < (n > 0 ? n : 1)) return CUP_ERR_ARG;
    *rank = 0;
    *certified = 1;
    if (nprimes) *nprimes = 0;
    if (m == 0 || n == 0) return CUP_OK;
    if (!A) return CUP_ERR_ARG;
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    double bound = 0.0;
    CK(int_bound(h, A, m, n, lda, &bound, st));
    std::vector<uint32_t> pr;
    CK(int_primes(primes, K, bound, pr));           // not every prime can divide a nonzero minor
    std::vector<int64_t> ranks(pr.size());
    CK(ensure_base(h));
    CK(int_residues(h, A, m, n, lda, pr, ranks.data(), nullptr, st));
    int64_t r = 0;
    for (int64_t x : ranks) r = x > r ? x : r;
    *rank = r;
    *certified = log2_product(pr) > bound;
    if (nprimes) *nprimes = (int64_t)pr.size();
    return CUP_OK;
}

}  // extern "C"
