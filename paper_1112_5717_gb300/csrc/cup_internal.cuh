// Internal declarations shared by the CUDA translation units of the CUP library.
#pragma once
#include <atomic>
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>
#include "modp.cuh"

// A value known on the host or only on the device: s + c0 *p0 + c1 *p1,
// clamped to [lo, hi]. The device-resident schedule passes the running rank
// (and the rank at the middle of a node) by pointer; host-driven calls pass
// constants (p0 = p1 = null). hi is also the host's bound for grid sizes.
struct Dyn {
    int64_t s;
    const int64_t *p0, *p1;
    int64_t c0, c1;
    int64_t lo, hi;
    __host__ __device__ __forceinline__ int64_t eval() const
    {
        int64_t v = s;
        if (p0) v += c0 * *p0;
        if (p1) v += c1 * *p1;
        return v < lo ? lo : (v > hi ? hi : v);
    }
};

#ifdef __CUDACC__
// Asynchronous 4-byte global -> shared copies (no register staging, so every
// copy of a tile is in flight at once); cp_async_wait_all() waits for this
// thread's copies, a __syncthreads() after it publishes them to the block.
__device__ __forceinline__ void cp_async4(uint32_t *smem, const uint32_t *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t *smem, const uint32_t *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}
// Close the group of this thread's copies issued so far; cp_async_wait_prior<N>() then
// waits until at most the N most recent groups are still in flight.
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait_prior()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
#endif

#ifdef __CUDACC__
// Programmatic dependent launch. The kernels of the factorisation's launch chain
// are launched with launch_pdl, so each may become resident while the previous
// kernel of its stream is still running; every one of them starts with
// pdl_enter(), which waits for that kernel's completion and memory (nothing is
// read before it) and then lets the next kernel of the stream be launched. A
// kernel launched the ordinary way passes both instructions at once.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// Data written two or more launches back is complete when a dependent kernel
// starts (its predecessor passed its own pdl_enter before releasing it), so a
// prologue that reads only such data may run before pdl_enter; every CTA must
// still pass pdl_enter before it exits, which keeps the chain ordered.
#endif

#ifdef __CUDACC__
#include <cuda_bf16.h>
// Centred base-256 digits of a residue: x = sum_l d_l 256^l (mod p), |d_l| <= 128,
// exact in bf16.
template <int L>
__device__ __forceinline__ void limb_digits(uint32_t x, uint32_t p, __nv_bfloat16 (&d)[L])
{
    int32_t v = (x > (p >> 1)) ? (int32_t)(x - p) : (int32_t)x;
#pragma unroll
    for (int l = 0; l < L - 1; ++l) {
        const int32_t dl = ((v + 128) & 255) - 128;
        d[l] = __int2bfloat16_rn(dl);
        v = (v - dl) >> 8;
    }
    d[L - 1] = __int2bfloat16_rn(v);
}

// D += A B for one 16 x 8 tile: A 16 x 16 (row), B 16 x 8 (col), bf16 in, fp32 accumulate.
__device__ __forceinline__ void mma_16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
#endif

template <typename... KArgs, typename... Args>
static inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                     Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, ((KArgs)args)...);
}

// One-time setup per CUDA device (kernel attributes such as the raised dynamic
// shared-memory limit belong to each device's context): `setup` runs, with the
// device current, the first time a launcher is used on that device, and again
// after a failure. Thread safe; the common path is one atomic load.
struct PerDeviceOnce {
    static constexpr int kMaxDev = 128;
    std::atomic<uint64_t> done[kMaxDev / 64] = {};
    std::mutex mu;
};
template <typename F>
static inline cudaError_t once_per_device(PerDeviceOnce &o, F setup)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= PerDeviceOnce::kMaxDev) return setup();
    const uint64_t bit = 1ull << (dev & 63);
    std::atomic<uint64_t> &w = o.done[dev >> 6];
    if (w.load(std::memory_order_acquire) & bit) return cudaSuccess;
    std::lock_guard<std::mutex> lock(o.mu);
    if (w.load(std::memory_order_relaxed) & bit) return cudaSuccess;
    e = setup();
    if (e == cudaSuccess) w.fetch_or(bit, std::memory_order_release);
    return e;
}

static inline Dyn dconst(int64_t v) { return Dyn{v, nullptr, nullptr, 0, 0, v, v}; }
static inline Dyn dvar(int64_t s, const int64_t *p0, int64_t c0, const int64_t *p1, int64_t c1, int64_t lo,
                       int64_t hi)
{
    return Dyn{s, p0, p1, c0, c1, lo, hi};
}

// One Schur update C <- C -/+ A B mod p where the operands are blocks of
// row-major matrices: element (i, j) of X is X.base[(X.row + i) ld + X.col + j].
// M is fixed; N and K may be dynamic (K.hi and N.hi bound them).
struct GemmDesc {
    const uint32_t *A;
    int64_t lda;
    Dyn arow, acol;
    const uint32_t *B;
    int64_t ldb;
    Dyn brow, bcol;
    uint32_t *C;
    int64_t ldc;
    Dyn crow, ccol;
    int64_t M;
    Dyn N, K;
    int add;
    // 1: B, C and the extents were written at least two launches back on the stream (the
    // launch just before writes only A), so a kernel launched with launch_pdl may read
    // them before waiting for its predecessor
    int pre = 0;
};

// A right-side triangular operation B <- B T^{-1} (or B T) with B rows x n and
// T n x n (n <= 64) given as blocks of row-major matrices at dynamic offsets.
struct TriDesc {
    const uint32_t *T;
    int64_t ldt;
    Dyn trow, tcol;
    uint32_t *B;
    int64_t ldb;
    Dyn brow, bcol;
    int64_t rows;
    Dyn n;
    // 1: T and the extents were written at least two launches back on the stream
    // (never by the kernel launched just before), so a kernel launched with
    // launch_pdl may read them before waiting for its predecessor
    int pre = 0;
};

#define CUP_BMAX 64        // most rows a leaf slab may hold
#define CUP_WNMAX 128      // widest pivot-search window of a leaf
#define CUP_NSLOT (CUP_WNMAX + 2)
#define CUP_QT 64          // column positions per CTA in the leaf finish kernel

// What the leaf pivot kernel hands to the leaf finish kernel (device memory).
// Positions are relative to the slab's first active column col0; rows are
// relative to the slab's first row.
struct SlabScratch {
    int r_s;                 // pivots found
    int i_stop;              // rows resolved (the rest need the node update first)
    int wne;                 // window width used
    int ext_pos;             // position >= wne that received window column 0, or -1
    int ext_slot;            // slot of ext_pos in Dorig
    int n_slot;
    int n_spec;              // rows taken as dependent because their window residual vanished
    int spec_fail;           // set by the finish kernel if such a row has a nonzero residual
    int spec_rows[CUP_BMAX];
    int prof[CUP_BMAX];      // slab-relative row of pivot t
    int win_col[CUP_WNMAX];  // original position held by window position q
    int win_slot[CUP_WNMAX]; // Dorig slot of window position q, or -1 if not displaced
    uint32_t pinv[CUP_BMAX];             // 1 / C[prof t][t]
    uint32_t Linv[CUP_BMAX][CUP_BMAX];   // inverse of L = (C[prof t][u])_{t,u}: U rows = Linv X
    uint32_t Cn[CUP_BMAX][CUP_BMAX];     // C[i][t] for slab rows i < i_stop, t < r_s
    uint32_t Dorig[CUP_NSLOT][CUP_BMAX]; // original values of displaced positions, per slab row
};

// Kernel launchers (cup_kernels.cu). All are asynchronous on `st`.
#define CUP_DEVERR_SPECULATION 100   // device error word: a row taken as dependent was not

cudaError_t launch_slab_pivots(const uint32_t *A, int64_t lda, int64_t a, int brows, Dyn col0, int64_t n,
                               int wn, int speculate, ModP M, SlabScratch *S, int64_t *ipiv, int64_t *prof,
                               int64_t *rank_next, cudaStream_t st);
// tensor: U = L^{-1} X by bf16 digit products on mma.sync for p < 2^24 (the tensor
// engine); otherwise, and for the plain engine, by 64-bit CUDA-core products.
cudaError_t launch_slab_finish(uint32_t *A, int64_t lda, int64_t a, int brows, Dyn col0, int64_t n, ModP M,
                               const SlabScratch *S, int *err, cudaStream_t st, bool tensor);
cudaError_t launch_swaplist(const int64_t *ipiv, Dyn k0, Dyn k1, int2 *pairs, int *count, cudaStream_t st);
cudaError_t launch_laswp(uint32_t *A, int64_t lda, Dyn row0, Dyn nrows, const int2 *pairs, const int *count,
                         cudaStream_t st);
cudaError_t launch_laswp_fused(uint32_t *A, int64_t lda, Dyn row0, Dyn nrows, const int64_t *ipiv, Dyn k0, Dyn k1,
                               cudaStream_t st);
cudaError_t launch_gemm_sub_cc(const uint32_t *A, int64_t lda, const uint32_t *B, int64_t ldb,
                               uint32_t *C, int64_t ldc, int64_t Mr, int64_t N, int64_t K, ModP M,
                               cudaStream_t st, int add = 0);
cudaError_t launch_gemm_cc_desc(const GemmDesc &d, ModP M, cudaStream_t st);
cudaError_t launch_det_reduce(const uint32_t *A, int64_t lda, int64_t n, const int64_t *ipiv, ModP M,
                              uint32_t *out, cudaStream_t st);

// Tensor-core Schur update (cup_tc.cu).
int tc_limbs(uint32_t p);

// One-launch short-K tensor update (cup_short.cu): mma.sync on digits made in
// shared memory, for K up to the handle's bound (at most SHORT_K_MAX), p < 2^24
// and at most SHORT_MAX_OUTPUTS entries of C (beyond that the tcgen05 path's
// throughput wins).
#define SHORT_K_MAX 256
#define SHORT_MAX_OUTPUTS (1ll << 21)
bool gemm_short_ok(uint32_t p, int64_t M, int64_t Nhi, int64_t Khi, int64_t kmax);
cudaError_t launch_gemm_short_desc(const GemmDesc &d, ModP M, cudaStream_t st);
size_t tc_workspace_bytes(uint32_t p, int64_t M, int64_t N, int64_t K);
cudaError_t launch_gemm_tc_desc(const GemmDesc &d, ModP Mp, void *ws, int *err, cudaStream_t st,
                                cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr);
cudaError_t launch_gemm_sub_tc(const uint32_t *A, int64_t lda, const uint32_t *B, int64_t ldb, uint32_t *C,
                               int64_t ldc, int64_t M, int64_t N, int64_t K, ModP Mp, void *ws, int *err,
                               cudaStream_t st, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr,
                               int add = 0);

// Bounded-wait self-test (cup_tc.cu): a wait that nothing completes, given up
// after limit_ns with `code` recorded in *err.
#define CUP_DEVERR_SELFTEST 99
cudaError_t launch_selftest_wait(int *err, uint64_t limit_ns, int code, cudaStream_t st);

// Triangular building blocks (cup_tri.cu). Flags of launch_tri_leaf: the
// triangle T is n x n with n = rows (left) or cols (right) of B, n <= 64.
enum { TRI_LEFT = 1, TRI_UPPER = 2, TRI_UNIT = 4, TRI_SOLVE = 8 };
cudaError_t launch_tri_leaf(int flags, const uint32_t *T, int64_t ldt, uint32_t *B, int64_t ldb,
                            int64_t rows, int64_t cols, ModP M, cudaStream_t st);
// Right, upper, unit solve on a TriDesc (the TRSM step of the device-resident CUP).
cudaError_t launch_trsm_ruu_desc(const TriDesc &d, ModP M, cudaStream_t st);
cudaError_t launch_trtri_leaf(int upper, int unit, uint32_t *T, int64_t ldt, int n, ModP M, cudaStream_t st);
cudaError_t launch_trulm_leaf(uint32_t *A, int64_t lda, int n, ModP M, cudaStream_t st);
cudaError_t launch_trlum_leaf(uint32_t *A, int64_t lda, int n, int unit_l, ModP M, cudaStream_t st);
cudaError_t launch_col_swaps(uint32_t *A, int64_t lda, int64_t nrows, const int64_t *list, int64_t count,
                             int reverse, cudaStream_t st);
cudaError_t launch_negate(uint32_t *B, int64_t ldb, int64_t m, int64_t n, uint32_t p, cudaStream_t st);
cudaError_t launch_row_swaps(uint32_t *A, int64_t lda, int64_t ncols, const int64_t *list, int64_t count,
                             int64_t base_a, int64_t base_b, int reverse, int prefix, cudaStream_t st);
cudaError_t launch_gather_rows(uint32_t *dst, int64_t ldd, const uint32_t *src, int64_t lds, const int64_t *idx,
                               int64_t nrows, int64_t ncols, cudaStream_t st);
cudaError_t launch_fill(uint32_t *B, int64_t ldb, int64_t m, int64_t n, int diag, cudaStream_t st);
cudaError_t launch_any_nonzero(const uint32_t *B, int64_t ldb, int64_t m, int64_t n, int *flag, cudaStream_t st);
cudaError_t launch_transpose(uint32_t *D, int64_t ldd, const uint32_t *S, int64_t lds, int64_t m, int64_t n,
                             cudaStream_t st);
cudaError_t launch_copy(uint32_t *D, int64_t ldd, const uint32_t *S, int64_t lds, int64_t m, int64_t n,
                        cudaStream_t st);
cudaError_t launch_zero_upper(uint32_t *B, int64_t ldb, int64_t n, cudaStream_t st);
// One-byte residue storage: W (uint32, ldw) <- B8 (uint8, ld8) and back, m x n.
cudaError_t launch_widen_u8(uint32_t *W, int64_t ldw, const uint8_t *B8, int64_t ld8, int64_t m, int64_t n,
                            cudaStream_t st);
cudaError_t launch_narrow_u8(uint8_t *B8, int64_t ld8, const uint32_t *W, int64_t ldw, int64_t m, int64_t n,
                             cudaStream_t st);

// Prime check shared by the entry points (cup_api.cu).
bool cup_internal_prime_ok(uint32_t p);

// Batched CUP (cup_batched.cu).

// Multi-modular integer path (cup_int.cu).
#include <vector>
cudaError_t launch_reduce_multi(const int64_t *A, int64_t lda, int64_t m, int64_t n, const uint32_t *d_primes,
                                int K, uint32_t *R, int64_t ldr, int64_t plane, cudaStream_t st);
cudaError_t launch_row_log2norm(const int64_t *A, int64_t lda, int64_t m, int64_t n, double *out, cudaStream_t st);
// x = CRT(res mod pr) in the symmetric range, as sign and little-endian 32-bit magnitude
// words; false if two primes coincide.
bool cup_internal_crt(const uint32_t *res, const uint32_t *pr, int64_t K, std::vector<uint32_t> &mag, int &sign);
bool cup_internal_is_prime(uint32_t n);
int64_t cup_internal_primes_below(uint32_t bound, int64_t count, uint32_t *out);
