// Short-K Schur update C <- C - A B (or C + A B) mod p: the MM step of
// Algorithm 6 (Sec. 3.2, alpha = -1, beta = 1) at the lowest levels of the row
// recursion and of Algorithm 2's TRSM, where the inner dimension is one to four
// base-case slabs (K <= 256) and the product itself is at most a few GFLOP.
//
// There the tcgen05 path costs a separate digit-split launch plus the fixed
// part of its own launch (TMEM allocation, barrier setup, TMA and MMA
// latency), far more than the arithmetic. This kernel does the whole update in
// one launch: every CTA loads its 64 x K block of A, K x 64 block of B and
// 64 x 64 block of C as residues (all loads of a 128-column pass in flight at
// once), writes the
// centred base-256 digits of A and B (L = 1..3 limbs for p < 2^24, bf16) to
// shared memory, forms the L^2 digit products with mma.sync m16n8k16 (fp32
// accumulation: at most K L 2^14 < 2^24 in magnitude, so every partial sum is
// exact), recombines the products by their shift, reduces once and updates C.
#include "cup_internal.cuh"

#define SK_BM 64
#define SK_BN 64

template <int L, int KP>
__global__ void __launch_bounds__(256)
k_gemm_short(const GemmDesc d, ModP Mp, uint64_t off)
{
    // With d.pre the B and C blocks are read before the dependency wait (only A comes
    // from the launch just before); otherwise everything waits.
    const bool pre = d.pre != 0;
    if (!pre) pdl_enter();
    const int64_t Mr = d.M, N = d.N.eval(), K = d.K.eval();
    const int64_t m0 = (int64_t)blockIdx.y * SK_BM, n0 = (int64_t)blockIdx.x * SK_BN;
    if (n0 >= N || m0 >= Mr || K <= 0) {
        if (pre) pdl_enter();
        return;
    }
    const int64_t lda = d.lda, ldb = d.ldb, ldc = d.ldc;
    const uint32_t *__restrict__ A = d.A + (d.arow.eval() + m0) * lda + d.acol.eval();
    const uint32_t *__restrict__ B = d.B + d.brow.eval() * ldb + d.bcol.eval() + n0;
    uint32_t *__restrict__ C = d.C + (d.crow.eval() + m0) * ldc + d.ccol.eval() + n0;
    const int mr = (int)((Mr - m0) < SK_BM ? (Mr - m0) : SK_BM);
    const int nc = (int)((N - n0) < SK_BN ? (N - n0) : SK_BN);
    const int kk = (int)K;                      // K <= KP
    // bf16 row stride of the digit planes: KP + 8 (rows 16-byte aligned, fragment loads of
    // eight rows on distinct banks); K is staged in passes of KC <= 128 columns
    constexpr int SK_LD = KP + 8, KC = KP < 128 ? KP : 128;
    extern __shared__ __align__(16) uint8_t sk_smem[];
    __nv_bfloat16 *As = (__nv_bfloat16 *)sk_smem;        // [L][SK_BM][SK_LD], k contiguous
    __nv_bfloat16 *Bt = As + L * SK_BM * SK_LD;          // [L][SK_BN][SK_LD], k contiguous
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int mt = warp & 3, nh = warp >> 2, g = lane >> 2, tq = lane & 3;

    // A: thread (k = tid % KC) takes rows tid / KC + (256 / KC) j; B: thread (n = tid % 64)
    // takes rows k = tid / 64 + 4 j; C: the 16 entries this thread's MMA tiles produce.
    // Every load of a pass is issued before any use.
    constexpr int RG = 256 / KC, NA = SK_BM / RG, NB = KC / 4;
    uint32_t xa[NA], xb[NB], cv[4][4];
    auto load_b = [&](const int kc) {
        const int n = tid & (SK_BN - 1), k0 = kc + (tid >> 6);
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const int k2 = k0 + 4 * j;
            xb[j] = (k2 < kk && n < nc) ? B[(int64_t)k2 * ldb + n] : 0u;
        }
    };
    auto load_a = [&](const int kc) {
        const int k = kc + (tid & (KC - 1)), i0 = tid / KC;
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            const int i = i0 + RG * j;
            xa[j] = (i < mr && k < kk) ? A[(int64_t)i * lda + k] : 0u;
        }
    };
    auto store_digits = [&](const int kc) {
        const int k = kc + (tid & (KC - 1)), i0 = tid / KC;
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            __nv_bfloat16 dg[L];
            limb_digits<L>(xa[j], Mp.p, dg);
#pragma unroll
            for (int l = 0; l < L; ++l) As[(l * SK_BM + i0 + RG * j) * SK_LD + k] = dg[l];
        }
        const int n = tid & (SK_BN - 1), k0 = kc + (tid >> 6);
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            __nv_bfloat16 dg[L];
            limb_digits<L>(xb[j], Mp.p, dg);
#pragma unroll
            for (int l = 0; l < L; ++l) Bt[(l * SK_BN + n) * SK_LD + k0 + 4 * j] = dg[l];
        }
    };
    load_b(0);
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = 16 * mt + g + 8 * (e >> 1), j = 32 * nh + 8 * nt + 2 * tq + (e & 1);
            cv[nt][e] = (i < mr && j < nc) ? C[(int64_t)i * ldc + j] : 0u;
        }
    if (pre) pdl_enter();
    load_a(0);
    store_digits(0);
#pragma unroll
    for (int kc = KC; kc < KP; kc += KC) {
        if (kc >= kk) break;
        load_b(kc);
        load_a(kc);
        store_digits(kc);
    }
    __syncthreads();

    // warp (mt, nh) owns rows 16 mt .. + 15 and columns 32 nh .. + 31 (four 16 x 8 tiles);
    // shift s = i + j collects the digit products A_i B_j
    constexpr int NS = 2 * L - 1;
    float acc[NS][4][4];
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[s][j][e] = 0.f;
    const int nks = (kk + 15) >> 4;
#pragma unroll
    for (int ks = 0; ks < KP / 16; ++ks) {
        if (ks >= nks) break;
        const int k0 = 16 * ks + 2 * tq;
        uint32_t af[L][4];
#pragma unroll
        for (int i = 0; i < L; ++i) {
            const __nv_bfloat16 *ar = As + (i * SK_BM + 16 * mt + g) * SK_LD + k0;
            af[i][0] = *(const uint32_t *)ar;
            af[i][1] = *(const uint32_t *)(ar + 8 * SK_LD);
            af[i][2] = *(const uint32_t *)(ar + 8);
            af[i][3] = *(const uint32_t *)(ar + 8 * SK_LD + 8);
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
            for (int j = 0; j < L; ++j) {
                const __nv_bfloat16 *br = Bt + (j * SK_BN + 32 * nh + 8 * nt + g) * SK_LD + k0;
                const uint32_t b0 = *(const uint32_t *)br, b1 = *(const uint32_t *)(br + 8);
#pragma unroll
                for (int i = 0; i < L; ++i) mma_16816(acc[i + j][nt], af[i], b0, b1);
            }
        }
    }
    // v = sum_s acc_s 256^s is the integer product of the centred representatives,
    // |v| <= K (p / 2)^2 < 2^54; off is a multiple of p at least that large
    const int add = d.add;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = 16 * mt + g + 8 * (e >> 1), j = 32 * nh + 8 * nt + 2 * tq + (e & 1);
            if (i < mr && j < nc) {
                int64_t v = 0;
#pragma unroll
                for (int s = NS - 1; s >= 0; --s) v = v * 256 + (int64_t)__float2int_rn(acc[s][nt][e]);
                const uint32_t r = red64((uint64_t)(v + (int64_t)off), Mp);
                C[(int64_t)i * ldc + j] = add ? addm(cv[nt][e], r, Mp) : subm(cv[nt][e], r, Mp);
            }
        }
}

template <int L, int KP>
static size_t short_smem()
{
    return (size_t)L * (SK_BM + SK_BN) * (KP + 8) * sizeof(__nv_bfloat16);
}

bool gemm_short_ok(uint32_t p, int64_t M, int64_t Nhi, int64_t Khi, int64_t kmax)
{
    return kmax > 0 && Khi <= kmax && Khi <= SHORT_K_MAX && p < (1u << 24) && M > 0 && Nhi > 0 &&
           M * Nhi <= SHORT_MAX_OUTPUTS;
}

cudaError_t launch_gemm_short_desc(const GemmDesc &d, ModP M, cudaStream_t st)
{
    if (d.M <= 0 || d.N.hi <= 0 || d.K.hi <= 0) return cudaSuccess;
    if (d.K.hi > SHORT_K_MAX || M.p >= (1u << 24)) return cudaErrorInvalidValue;
    static PerDeviceOnce once;
    cudaError_t e = once_per_device(once, [] {
        cudaError_t e2 = cudaSuccess;
#define SK_ATTR(L, KP)                                                                                         \
    if (e2 == cudaSuccess)                                                                                     \
        e2 = cudaFuncSetAttribute(k_gemm_short<L, KP>, cudaFuncAttributeMaxDynamicSharedMemorySize,            \
                                  (int)short_smem<L, KP>());
        SK_ATTR(1, 64) SK_ATTR(2, 64) SK_ATTR(3, 64) SK_ATTR(1, 128) SK_ATTR(2, 128) SK_ATTR(3, 128)
        SK_ATTR(1, 256) SK_ATTR(2, 256) SK_ATTR(3, 256)
#undef SK_ATTR
        return e2;
    });
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((d.N.hi + SK_BN - 1) / SK_BN), (unsigned)((d.M + SK_BM - 1) / SK_BM));
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    const int L = tc_limbs(M.p);
    // a multiple of p no smaller than K (p / 2)^2 (< 2^54 for K <= 256, p < 2^24)
    const uint64_t half = (uint64_t)(M.p / 2 + 1);
    const uint64_t bound = (uint64_t)d.K.hi * half * half;
    const uint64_t off = (bound / M.p + 1) * (uint64_t)M.p;
    const bool k64 = d.K.hi <= 64, k128 = d.K.hi <= 128;
#define SK_GO(LL, KP) return launch_pdl(k_gemm_short<LL, KP>, grid, 256, short_smem<LL, KP>(), st, d, M, off)
    if (L == 1) { if (k64) SK_GO(1, 64); if (k128) SK_GO(1, 128); SK_GO(1, 256); }
    if (L == 2) { if (k64) SK_GO(2, 64); if (k128) SK_GO(2, 128); SK_GO(2, 256); }
    if (k64) SK_GO(3, 64);
    if (k128) SK_GO(3, 128);
    SK_GO(3, 256);
#undef SK_GO
}
