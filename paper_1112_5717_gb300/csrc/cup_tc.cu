// Tensor-core Schur update over GF(p): C <- C - A B mod p (Algorithm 1 with
// alpha = -1, beta = 1, the MM step of Algorithm 6 and of Algorithm 2's TRSM).
//
// Exact integer products on tcgen05 (sm_103a has no integer tcgen05 kind):
//   * every residue x in [0, p) is centred (x - p when x > (p-1)/2) and split
//     into L signed base-256 digits d_l in [-128, 128] (L = 1, 2, 3, 4 for
//     p below 2^8, 2^16, 2^24, 2^31); |d| <= 256 is exact in bf16;
//   * limb products are accumulated by tcgen05.mma kind::f16 (bf16 in,
//     fp32 accumulate in TMEM), one accumulator D_s per digit shift s = i + j,
//     D_s = sum_{i+j=s} A_i B_j^T. Every term is at most 2^14 in magnitude and
//     a shift collects at most L products per k, so a chunk of kc values of k
//     with L * kc * 2^14 <= 2^24 keeps every partial sum an exact fp32
//     integer;
//   * after each chunk the epilogue warps read the accumulators from TMEM,
//     recombine sum_s D_s 256^s in 64-bit integers, reduce mod p and add to a
//     running residue per output; the last chunk's result is subtracted from C.
// Operands reach shared memory by TMA (cp.async.bulk.tensor, 128-byte swizzle)
// from limb planes written by the split kernels below.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <mutex>
#include "cup_internal.cuh"
#include "../../include/cup_gb300.h"

namespace tc {

constexpr int BM = 128;       // rows per tile (tcgen05 M)
constexpr int BK = 64;        // k per pipeline stage: one 128-byte swizzle row of bf16
constexpr int NEPI = 16;      // epilogue warps (four per TMEM lane quarter)
constexpr int NTHREADS = 32 * (2 + NEPI);
constexpr int SMEM_BUDGET = 200 * 1024;
constexpr int GROUP_M = 16;   // tile rows walked together by consecutive CTAs

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: gives up after limit_ns of wall time (2 s in the kernels), or as
// soon as another thread has recorded a failure, and records the failure.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err, int code,
                                          uint64_t limit_ns = 2000000000ull)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255u) == 0u) {
            if (*(volatile int *)err != 0) return false;
            if (globaltimer() - t0 > limit_ns) {
                atomicCAS(err, 0, code);
                return false;
            }
        }
    }
}

// Self-test of the timeout path: one thread waits, with the kernels' bounded
// wait, on an mbarrier that nothing arrives at; the wait gives up after
// limit_ns, records `code` in the error word and the kernel returns normally.
__global__ void k_selftest_wait(int *err, uint64_t limit_ns, int code)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_wait(smem_u32(&bar), 0u, err, code, limit_ns);
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor of tcgen05 for a K-major operand in the
// 128-byte swizzled layout TMA writes: 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);          // start address
    d |= (uint64_t)1 << 16;                            // leading byte offset (unused for SW128 K-major)
    d |= (uint64_t)(1024 >> 4) << 32;                  // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                            // descriptor version
    d |= (uint64_t)2 << 61;                            // 128-byte swizzle
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: bf16 A and B, fp32 D,
// both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_bf16(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
                 "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
                 : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
        "%13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Barrier over the epilogue warps only (named barrier 1).
__device__ __forceinline__ void epi_bar()
{
    asm volatile("bar.sync 1, %0;" ::"n"(32 * NEPI) : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Montgomery step without the final subtraction: for x < 2^61, (x + m p) / R < 2^29 + p.
__device__ __forceinline__ uint32_t redc_raw(uint64_t x, const ModP &M)
{
    const uint32_t m = (uint32_t)x * M.pneg;
    return (uint32_t)((x + (uint64_t)m * M.p) >> 32);
}


template <int L, int BNX = 0>
struct Cfg {
    static constexpr int NACC = 2 * L - 1;
    static constexpr int BN = BNX ? BNX : ((NACC * 128 <= 512) ? 128 : 64);
    // 256-column tiles keep the partial sums of earlier K chunks in the epilogue
    // threads' registers (64 one-byte residues, four to a register) instead of TMEM,
    // and do not prefetch C
    static constexpr bool REGP = BN > 128;
    static_assert(!REGP || L == 1, "register partial sums hold one-byte residues (p < 2^8)");
    // two accumulator sets (the MMAs of chunk c + 1 run while chunk c is drained) when
    // they fit in TMEM next to the partial sums
    static constexpr int NBUF = (2 * NACC * BN + (REGP ? 0 : BN) <= 512) ? 2 : 1;
    static constexpr int STAGE_A = BM * BK * 2;
    static constexpr int STAGE_B = BN * BK * 2;
    static constexpr int STAGE = L * (STAGE_A + STAGE_B);
    static constexpr int NSTAGE = (SMEM_BUDGET / STAGE) < 8 ? (SMEM_BUDGET / STAGE) : 8;
    static constexpr int CBUF = REGP ? 0 : BM * BN * 4;       // a C tile (prefetch when K is short)
    static constexpr int SMEMUSE = (NSTAGE * STAGE > (NSTAGE - 1) * STAGE + CBUF) ? NSTAGE * STAGE
                                                                                   : (NSTAGE - 1) * STAGE + CBUF;
    static_assert(BM * BN * 4 <= NSTAGE * STAGE, "the staged result tile fits in the stage memory");
    static_assert(NBUF * NACC * BN + (REGP ? 0 : BN) <= 512, "accumulators fit in TMEM");
    static constexpr int SMEM = SMEMUSE + 1024;
    static constexpr int KCHUNK = (1024 / L) / BK * BK;      // L * kc * 2^14 <= 2^24
    static constexpr int COLS_PER_WARP = BN / 2;
};

// C[M x N] -= A B (mod p) from limb planes: Al is (L, M, Kp), Bl is (L, N, Kp), bf16, K-major.
template <int L, int BNX>
__global__ void __launch_bounds__(NTHREADS, 1)
k_limb_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            const GemmDesc d, ModP Mp, uint64_t off, uint32_t sh32, int *__restrict__ err)
{
    // The launch just before this one is always this product's k_split, so only the
    // limb planes depend on it: the extents, C and the setup are read or done
    // before pdl_enter (C and the ranks come from earlier launches).
    const int M = (int)d.M, N = (int)d.N.eval(), K = (int)d.K.eval();
    const int Kp = (K + BK - 1) / BK * BK;
    const int add = d.add;
    const int64_t ldc = d.ldc;
    using CF = Cfg<L, BNX>;
    // Tile of this CTA: the grid is one-dimensional and walks groups of GROUP_M tile
    // rows, tile row fastest within a group, so the CTAs resident at a time share a
    // few A and B tiles (read from L2) instead of all of B's planes.
    const int mt = (M + BM - 1) / BM, ntl = gridDim.x / mt;
    const int id = blockIdx.x, grp = id / (GROUP_M * ntl), first = grp * GROUP_M;
    const int gsz = (mt - first) < GROUP_M ? (mt - first) : GROUP_M;
    const int inr = id - grp * GROUP_M * ntl;
    const int tm = first + inr % gsz, tn = inr / gsz;
    if (tn * CF::BN >= N || K <= 0) {                          // outside this call's extents
        pdl_enter();
        return;
    }
    uint32_t *C = d.C + d.crow.eval() * ldc + d.ccol.eval();
    constexpr int BN = CF::BN, NACC = CF::NACC, NSTAGE = CF::NSTAGE, NBUF = CF::NBUF;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[NSTAGE], empty_bar[NSTAGE], accf_bar[NBUF], acce_bar[NBUF];
    __shared__ uint32_t tmem_base_sh;

    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = tm * BM, n0 = tn * BN;
    const int nkb = Kp / BK;
    const int kb_chunk = CF::KCHUNK / BK;
    const int nchunk = (nkb + kb_chunk - 1) / kb_chunk;
    // a short K uses fewer stages; the C tile is then prefetched into the spare space
    const int nst = nkb < NSTAGE ? nkb : NSTAGE;
    const bool pref = CF::CBUF > 0 && nkb < NSTAGE;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(smem_u32(&accf_bar[b]), 1);
            mbar_init(smem_u32(&acce_bar[b]), NEPI);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // With a short K the epilogue warps copy the C tile asynchronously (coalesced)
    // into the shared memory the unused stages leave; it lands while the MMAs run.
    uint32_t *cbuf = (uint32_t *)(smem + CF::SMEMUSE - CF::CBUF);
    if (pref && warp >= 2) {
        constexpr int PER = BM * BN / (32 * NEPI);
        const int et = threadIdx.x - 64;
#pragma unroll 8
        for (int i = 0; i < PER; ++i) {
            const int e = et + 32 * NEPI * i, rr = e / BN, cc = e % BN;
            if (m0 + rr < M && n0 + cc < N) cp_async4(cbuf + e, C + (int64_t)(m0 + rr) * ldc + n0 + cc);
        }
    }
    pdl_enter();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int issued = 0;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % nst;
                const uint32_t ph = (uint32_t)(kb / nst) & 1u;
                if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u, err, 1)) break;
                const uint32_t fb = smem_u32(&full_bar[s]);
                mbar_expect_tx(fb, CF::STAGE);
                const uint32_t st = sbase + s * CF::STAGE;
#pragma unroll
                for (int l = 0; l < L; ++l) tma_load_3d(st + l * CF::STAGE_A, &tmA, kb * BK, m0, l, fb);
#pragma unroll
                for (int l = 0; l < L; ++l)
                    tma_load_3d(st + L * CF::STAGE_A + l * CF::STAGE_B, &tmB, kb * BK, n0, l, fb);
                ++issued;
            }
            // before leaving, let every issued copy land (bounded)
            for (int kb = (issued > nst ? issued - nst : 0); kb < issued; ++kb)
                mbar_wait(smem_u32(&full_bar[kb % nst]), (uint32_t)(kb / nst) & 1u, err, 2);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(BN);
            int kb = 0;
            bool ok = true;
            for (int c = 0; c < nchunk && ok; ++c) {
                // accumulator set c % NBUF must have been drained (chunk c - NBUF)
                const int buf = c % NBUF;
                if (c >= NBUF &&
                    !mbar_wait(smem_u32(&acce_bar[buf]), (uint32_t)((c - NBUF) / NBUF) & 1u, err, 3)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dbase = tmem + (uint32_t)(buf * NACC * BN);
                const int kb_first = kb;
                const int kb_end = (kb + kb_chunk < nkb) ? kb + kb_chunk : nkb;
                for (; kb < kb_end; ++kb) {
                    const int s = kb % nst;
                    const uint32_t ph = (uint32_t)(kb / nst) & 1u;
                    if (!mbar_wait(smem_u32(&full_bar[s]), ph, err, 4)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t st = sbase + s * CF::STAGE;
#pragma unroll
                    for (int i = 0; i < L; ++i)
#pragma unroll
                        for (int j = 0; j < L; ++j) {
                            const int sh = i + j;
                            const int ifirst = sh - (L - 1) > 0 ? sh - (L - 1) : 0;
                            const uint32_t a_addr = st + i * CF::STAGE_A;
                            const uint32_t b_addr = st + L * CF::STAGE_A + j * CF::STAGE_B;
#pragma unroll
                            for (int kk = 0; kk < BK / 16; ++kk) {
                                const uint32_t acc = (kb == kb_first && i == ifirst && kk == 0) ? 0u : 1u;
                                mma_bf16(dbase + sh * BN, sw128_desc(a_addr + kk * 32),
                                         sw128_desc(b_addr + kk * 32), idesc, acc);
                            }
                        }
                    mma_commit(smem_u32(&empty_bar[s]));
                }
                if (ok) mma_commit(smem_u32(&accf_bar[buf]));
            }
        }
    } else {
        // ---------------- epilogue warps ----------------
        // (1) With a short K the C tile was prefetched into cbuf (above).
        // (2) Per chunk, warp w reads TMEM lane quarter w % 4 (one row per thread)
        // and a quarter of the columns, recombines the shift accumulators in 64 bits and
        // reduces them; partial sums of earlier chunks wait in the TMEM columns
        // after the accumulators. (3) The reduced tile goes through stage 0 (free
        // once the last MMA has completed; XOR-swizzled rows keep both access
        // patterns free of bank conflicts) back to the coalesced layout, and C is
        // updated with the lanes along the columns.
        const int et = threadIdx.x - 64;                  // 0 .. 32 NEPI - 1
        constexpr int PER = BM * BN / (32 * NEPI);        // C entries per thread
        const int q = warp & 3;                           // TMEM lane quarter this warp may access
        const int cg = (warp - 2) >> 2;                   // which quarter of the BN columns
        constexpr int CPW = BN / 4;                       // columns per thread
        constexpr int CW = 8;                             // columns per TMEM load
        const uint32_t trow = (uint32_t)(32 * q) << 16;
        const int srow = 32 * q + lane;                   // this thread's row of the tile
        // Odd p with L <= 3: A's digits carry the factor R (the split stores A R mod p),
        // so one Montgomery step of the recombined value v < 2^61 gives the product
        // itself, below 2^29 + p, and a 32-bit Barrett step finishes the reduction.
        const bool mont = (L <= 3) && (Mp.p & 1u);
        const uint32_t mu32 = (uint32_t)(Mp.mu >> 32);    // floor(2^32 / p) for odd p
        uint32_t *tile = (uint32_t *)smem;
        bool ok = true;
        uint32_t runr[CF::REGP ? CPW / 4 : 1];            // partial sums of earlier chunks (REGP), packed bytes
        for (int c = 0; c < nchunk; ++c) {
            const int buf = c % NBUF;
            if (!mbar_wait(smem_u32(&accf_bar[buf]), (uint32_t)(c / NBUF) & 1u, err, 5)) { ok = false; break; }
            tc_fence_after();
            const bool last = c == nchunk - 1;
#pragma unroll
            for (int cb = 0; cb < CPW / CW; ++cb) {
                const int col = cg * CPW + cb * CW;
                const uint32_t tbase = tmem + trow + (uint32_t)(buf * NACC * BN + col);
                const uint32_t pbase = tmem + trow + (uint32_t)(NBUF * NACC * BN + col);   // partial sums
                float d[NACC][CW];
#pragma unroll
                for (int s = 0; s < NACC; ++s) tmem_ld8(tbase + s * BN, d[s]);
                uint32_t run[CW];
                if (CF::REGP) {
#pragma unroll
                    for (int e = 0; e < CW; ++e) run[e] = (runr[(cb * CW + e) >> 2] >> (8 * ((cb * CW + e) & 3))) & 255u;
                } else if (c > 0) {
                    float rf[CW];
                    tmem_ld8(pbase, rf);
#pragma unroll
                    for (int e = 0; e < CW; ++e) run[e] = __float_as_uint(rf[e]);
                }
                tmem_wait_ld();
#pragma unroll
                for (int e = 0; e < CW; ++e) {
                    uint32_t r;
                    if (L <= 3) {
                        int64_t v = 0;
#pragma unroll
                        for (int s = NACC - 1; s >= 0; --s) v = v * 256 + (int64_t)__float2int_rn(d[s][e]);
                        const uint64_t x = (uint64_t)(v + (int64_t)off);
                        if (mont) {
                            uint32_t t = redc_raw(x, Mp);
                            t -= __umulhi(t, mu32) * Mp.p;
                            r = t >= Mp.p ? t - Mp.p : t;
                        } else {
                            r = red64(x, Mp);
                        }
                    } else {
                        int64_t lo = 0, hi = 0;
#pragma unroll
                        for (int s = 3; s >= 0; --s) lo = lo * 256 + (int64_t)__float2int_rn(d[s][e]);
#pragma unroll
                        for (int s = NACC - 1; s >= 4; --s) hi = hi * 256 + (int64_t)__float2int_rn(d[s][e]);
                        uint32_t rl = red64((uint64_t)(lo + (int64_t)off), Mp);
                        uint32_t rh = red64((uint64_t)(hi + (int64_t)off), Mp);
                        r = red64((uint64_t)rh * sh32 + rl, Mp);
                    }
                    run[e] = (c > 0) ? addm(run[e], r, Mp) : r;
                }
                if (!last) {
                    if (CF::REGP) {
#pragma unroll
                        for (int e = 0; e < CW; e += 4)
                            runr[(cb * CW + e) >> 2] = run[e] | run[e + 1] << 8 | run[e + 2] << 16 | run[e + 3] << 24;
                    } else {
                        tmem_st8(pbase, run);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < CW; ++e) tile[srow * BN + ((col + e) ^ (srow & 31))] = run[e];
                }
            }
            if (!last && !CF::REGP) tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acce_bar[buf]));
        }
        if (pref) cp_async_wait_all();
        // every epilogue warp has staged its rows (or given up)
        epi_bar();
        if (ok) {
            // thread et owns column cc of rows rr0, rr0 + RPI, ...: addresses advance by a fixed step
            constexpr int RPI = 32 * NEPI / BN, B2 = 8;
            const int rr0 = et / BN, cc = et % BN;
            const bool colok = n0 + cc < N;
            const int64_t step = (int64_t)RPI * ldc;
            uint32_t *cp = C + (int64_t)(m0 + rr0) * ldc + n0 + cc;
#pragma unroll
            for (int i0 = 0; i0 < PER; i0 += B2) {
                uint32_t cv[B2];
                const uint32_t *lp = cp;
#pragma unroll
                for (int i = 0; i < B2; ++i, lp += step) {
                    const bool in = colok && m0 + rr0 + RPI * (i0 + i) < M;
                    cv[i] = !in ? 0u : pref ? cbuf[et + 32 * NEPI * (i0 + i)] : *lp;
                }
#pragma unroll
                for (int i = 0; i < B2; ++i, cp += step) {
                    const int rr = rr0 + RPI * (i0 + i);
                    if (colok && m0 + rr < M) {
                        const uint32_t v = tile[rr * BN + (cc ^ (rr & 31))];
                        *cp = add ? addm(cv[i], v, Mp) : subm(cv[i], v, Mp);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Limb split: residues -> L planes of centred signed base-256 digits in bf16.
// A (M x K, lda) -> Al[l][i][k], Kp columns (zero padded); B (K x N, ldb) ->
// Bl[l][j][k] (transposed, K-major).
// ---------------------------------------------------------------------------
template <int L>
__device__ __forceinline__ void split_digits(uint32_t x, uint32_t p, uint32_t half, __nv_bfloat16 (&d)[L])
{
    int32_t v = (x > half) ? (int32_t)(x - p) : (int32_t)x;
#pragma unroll
    for (int l = 0; l < L - 1; ++l) {
        int32_t dl = ((v + 128) & 255) - 128;
        d[l] = __int2bfloat16_rn(dl);
        v = (v - dl) >> 8;
    }
    d[L - 1] = __int2bfloat16_rn(v);
}

// One launch splits both operands: blocks [0, nbA) take rows of A (one thread:
// 8 consecutive k of a row; planes (L, M, Kp_stride)), the rest take 32 x 32 tiles
// of B through shared memory (planes (L, N_stride, Kp_stride), K-major). With
// `mont`, A's residues are first multiplied by R (Montgomery form), which the
// GEMM epilogue's single Montgomery reduction then removes.
template <int L>
__global__ void __launch_bounds__(256)
k_split(const GemmDesc d, int Kp_stride, int N_stride, int nbA, int gxB, ModP Mp, int mont,
        __nv_bfloat16 *__restrict__ outA, __nv_bfloat16 *__restrict__ outB)
{
    pdl_enter();
    __shared__ uint32_t t[32][33];
    const uint32_t p = Mp.p, half = (p - 1) / 2;
    const int K = (int)d.K.eval();
    const int Kp = (K + BK - 1) / BK * BK;
    if ((int)blockIdx.x < nbA) {
        const int M = (int)d.M;
        const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const int kv = Kp_stride / 8;
        const int64_t i = idx / kv;
        const int k0 = (int)(idx - i * kv) * 8;
        if (i >= M || k0 >= Kp) return;
        const uint32_t *A = d.A + (d.arow.eval() + i) * d.lda + d.acol.eval();
        uint32_t x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = (k0 + e < K) ? A[k0 + e] : 0u;
        __align__(16) __nv_bfloat16 buf[L][8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const uint32_t v = mont ? redc((uint64_t)x[e] * Mp.r2, Mp) : x[e];
            __nv_bfloat16 dg[L];
            split_digits<L>(v, p, half, dg);
#pragma unroll
            for (int l = 0; l < L; ++l) buf[l][e] = dg[l];
        }
        const int64_t plane = (int64_t)M * Kp_stride;
#pragma unroll
        for (int l = 0; l < L; ++l)
            *(uint4 *)(outA + l * plane + i * Kp_stride + k0) = *(const uint4 *)buf[l];
        return;
    }
    const int bb = (int)blockIdx.x - nbA;
    const int N = (int)d.N.eval();
    const int k0 = (bb / gxB) * 32, n0 = (bb % gxB) * 32;
    if (k0 >= Kp || n0 >= N) return;
    const uint32_t *B = d.B + d.brow.eval() * d.ldb + d.bcol.eval();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 8 rows of 32
    uint32_t v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int k = k0 + ty + 8 * j, n = n0 + tx;
        v[j] = (k < K && n < N) ? B[(int64_t)k * d.ldb + n] : 0u;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) t[ty + 8 * j][tx] = v[j];
    __syncthreads();
    const int64_t plane = (int64_t)N_stride * Kp_stride;
    for (int r = ty; r < 32; r += 8) {
        const int n = n0 + r, k = k0 + tx;
        if (n < N && k < Kp) {
            __nv_bfloat16 dg[L];
            split_digits<L>(t[tx][r], p, half, dg);
#pragma unroll
            for (int l = 0; l < L; ++l) outB[l * plane + (int64_t)n * Kp_stride + k] = dg[l];
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

bool make_map(CUtensorMap *map, void *base, int kp, int rows, int L, int box_rows)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)kp, (cuuint64_t)rows, (cuuint64_t)L};
    cuuint64_t strides[2] = {(cuuint64_t)kp * 2, (cuuint64_t)kp * 2 * (cuuint64_t)rows};
    cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int L, int BNX>
cudaError_t run_cfg(const GemmDesc &d, ModP Mp, void *ws, int *err, cudaStream_t st, cudaEvent_t ev0,
                    cudaEvent_t ev1)
{
    using CF = Cfg<L, BNX>;
    const int M = (int)d.M, Nmax = (int)d.N.hi, Kmax = (int)d.K.hi;
    const int Kp = (Kmax + BK - 1) / BK * BK;                    // plane row stride
    __nv_bfloat16 *Al = (__nv_bfloat16 *)ws;
    __nv_bfloat16 *Bl = Al + (size_t)L * M * Kp;
    {
        const int64_t nthr = (int64_t)M * (Kp / 8);
        const int nbA = (int)((nthr + 255) / 256);
        const int gxB = (Nmax + 31) / 32, gyB = (Kp + 31) / 32;
        const int mont = (L <= 3) && (Mp.p & 1u);
        const cudaError_t e = launch_pdl(k_split<L>, (unsigned)(nbA + gxB * gyB), 256, 0, st, d, Kp, Nmax, nbA, gxB,
                                         Mp, mont, Al, Bl);
        if (e != cudaSuccess) return e;
    }
    CUtensorMap ta, tb;
    if (!make_map(&ta, Al, Kp, M, L, BM) || !make_map(&tb, Bl, Kp, Nmax, L, CF::BN))
        return cudaErrorInvalidValue;
    static PerDeviceOnce attr;
    {
        const cudaError_t e = once_per_device(attr, [] {
            return cudaFuncSetAttribute(k_limb_gemm<L, BNX>, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM);
        });
        if (e != cudaSuccess) return e;
    }
    // offset making the recombined chunk value nonnegative: a multiple of p above its bound
    const int bound_bits = (L <= 3) ? 60 : 52;
    const uint64_t off = ((1ull << bound_bits) / Mp.p + 1) * Mp.p;
    const uint32_t sh32 = (uint32_t)((1ull << 32) % Mp.p);
    const int64_t tiles = (int64_t)((Nmax + CF::BN - 1) / CF::BN) * ((M + BM - 1) / BM);
    if (tiles > INT32_MAX) return cudaErrorInvalidValue;
    dim3 grid((unsigned)tiles);
    if (ev0) cudaEventRecord(ev0, st);
    cudaError_t e = launch_pdl(k_limb_gemm<L, BNX>, grid, NTHREADS, CF::SMEM, st, ta, tb, d, Mp, off, sh32, err);
    if (ev1) cudaEventRecord(ev1, st);
    return e;
}

// (64-column tiles would let two-limb accumulators double-buffer too, but they need
// half again the operand traffic per product and measured slower than 128 columns.)
template <int L>
cudaError_t run(const GemmDesc &d, ModP Mp, void *ws, int *err, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1)
{
    // one limb and a long K: 128 x 256 tiles read half again fewer operand bytes per product
    if constexpr (L == 1) {
        if (d.K.hi >= 1024) return run_cfg<L, 256>(d, Mp, ws, err, st, ev0, ev1);
    }
    return run_cfg<L, 0>(d, Mp, ws, err, st, ev0, ev1);
}

// ---------------------------------------------------------------------------
// Peak-rate probes of the tensor instructions an exact integer product could use
// on this GPU (measurement support for the choice of engine; no counterpart in the
// paper): back-to-back instructions on operands resident in registers or shared
// memory, so each instruction's own rate is timed.
//   kind 0: mma.sync m16n8k32 s8 x s8 -> s32 (8192 integer ops each)
//   kind 1: mma.sync m16n8k16 bf16 x bf16 -> f32 (4096 flops each)
//   kind 2: tcgen05.mma kind::f16, M = 128, N = 256, K = 16, bf16 operands in
//           shared memory, fp32 accumulator in TMEM (1,048,576 flops each)
// ---------------------------------------------------------------------------
template <int KIND>
__global__ void __launch_bounds__(256) k_probe_mma_sync(int64_t iters, uint32_t *sink)
{
    const uint32_t s = threadIdx.x * 0x01010101u + 0x01020304u;
    const uint32_t a[4] = {s, s ^ 0x11111111u, s ^ 0x22222222u, s ^ 0x33333333u};
    const uint32_t b0 = s ^ 0x44444444u, b1 = s ^ 0x55555555u;
    uint32_t c[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) c[j][e] = 0u;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (KIND == 0)
                asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                             "{%8,%9}, {%0,%1,%2,%3};"
                             : "+r"(c[j][0]), "+r"(c[j][1]), "+r"(c[j][2]), "+r"(c[j][3])
                             : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
            else
                asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                             "{%8,%9}, {%0,%1,%2,%3};"
                             : "+r"(c[j][0]), "+r"(c[j][1]), "+r"(c[j][2]), "+r"(c[j][3])
                             : "r"(a[0] & 0x3f803f80u), "r"(a[1] & 0x3f803f80u), "r"(a[2] & 0x3f803f80u),
                               "r"(a[3] & 0x3f803f80u), "r"(b0 & 0x3f803f80u), "r"(b1 & 0x3f803f80u));
        }
    }
    uint32_t x = 0u;
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) x ^= c[j][e];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = x;
}

__global__ void __launch_bounds__(128, 1) k_probe_tcgen05(int64_t iters, int *err)
{
    extern __shared__ uint8_t praw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_sh;
    uint8_t *smem = (uint8_t *)(((uintptr_t)praw + 1023) & ~(uintptr_t)1023);
    constexpr int A_BYTES = BM * BK * 2, B_BYTES = 256 * BK * 2;
    for (int i = threadIdx.x; i < (A_BYTES + B_BYTES) / 16; i += blockDim.x) ((uint4 *)smem)[i] = make_uint4(0, 0, 0, 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes, read by the tensor core
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                     "r"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh;
    if (threadIdx.x == 0) {
        constexpr uint32_t idesc = idesc_bf16(256);
        const uint32_t sa = smem_u32(smem), sb = sa + A_BYTES;
        for (int64_t it = 0; it < iters; ++it)
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
                mma_bf16(tmem, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32), idesc, (it | kk) ? 1u : 0u);
        mma_commit(smem_u32(&bar));
        mbar_wait(smem_u32(&bar), 0u, err, 98);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
}

}  // namespace tc

extern "C" cup_status cup_probe_tensor_peak(int device, int kind, int64_t iters, double *tflops)
{
    if (!tflops || kind < 0 || kind > 2 || iters < 1 || iters > (int64_t)1 << 30) return CUP_ERR_ARG;
    *tflops = 0.0;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return CUP_ERR_ARG;
    int nsm = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int *err = nullptr;
    uint32_t *sink = nullptr;
    cup_status s = CUP_OK;
    float ms = 0.f;
    // the tcgen05 probe asks for more shared memory than two CTAs could share, so each
    // SM runs one (its operand tiles take 49 KB of it)
    const size_t psmem = 120 * 1024;
    const int nthr = kind == 2 ? 128 : 256;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&sink, (size_t)nsm * 2 * 256 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess ||
        (kind == 2 && cudaFuncSetAttribute(tc::k_probe_tcgen05, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)psmem) != cudaSuccess)) {
        s = CUP_ERR_CUDA;
    }
    const int grid = kind == 2 ? nsm : 2 * nsm;
    for (int rep = 0; rep < 2 && s == CUP_OK; ++rep) {       // the first launch warms up
        const int64_t n = rep ? iters : (iters + 9) / 10;
        cudaEventRecord(e0, st);
        if (kind == 0) tc::k_probe_mma_sync<0><<<grid, nthr, 0, st>>>(n, sink);
        else if (kind == 1) tc::k_probe_mma_sync<1><<<grid, nthr, 0, st>>>(n, sink);
        else tc::k_probe_tcgen05<<<grid, nthr, psmem, st>>>(n, err);
        cudaEventRecord(e1, st);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) s = CUP_ERR_CUDA;
        if (s == CUP_OK && rep) {
            if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) s = CUP_ERR_CUDA;
            const double per = kind == 0 ? 8.0 * 8192.0 * (nthr / 32) : kind == 1 ? 8.0 * 4096.0 * (nthr / 32)
                                                                         : 4.0 * 2.0 * tc::BM * 256.0 * 16.0;
            if (s == CUP_OK) *tflops = per * (double)grid * (double)n / (ms * 1e-3) / 1e12;
        }
    }
    int herr = 0;
    if (s == CUP_OK && cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && herr)
        s = CUP_ERR_TIMEOUT;
    if (sink) cudaFree(sink);
    if (err) cudaFree(err);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (prev >= 0) cudaSetDevice(prev);
    return s;
}

cudaError_t launch_selftest_wait(int *err, uint64_t limit_ns, int code, cudaStream_t st)
{
    tc::k_selftest_wait<<<1, 32, 0, st>>>(err, limit_ns, code);
    return cudaGetLastError();
}

int tc_limbs(uint32_t p)
{
    if (p < (1u << 8)) return 1;
    if (p < (1u << 16)) return 2;
    if (p < (1u << 24)) return 3;
    return 4;
}

size_t tc_workspace_bytes(uint32_t p, int64_t M, int64_t N, int64_t K)
{
    const int L = tc_limbs(p);
    const int64_t Kp = (K + tc::BK - 1) / tc::BK * tc::BK;
    return (size_t)L * (size_t)(M + N) * (size_t)Kp * 2;
}

cudaError_t launch_gemm_tc_desc(const GemmDesc &d, ModP Mp, void *ws, int *err, cudaStream_t st, cudaEvent_t ev0,
                                cudaEvent_t ev1)
{
    if (d.M <= 0 || d.N.hi <= 0 || d.K.hi <= 0) return cudaSuccess;
    if (d.M > INT32_MAX / 2 || d.N.hi > INT32_MAX / 2 || d.K.hi > INT32_MAX / 2) return cudaErrorInvalidValue;
    switch (tc_limbs(Mp.p)) {
    case 1: return tc::run<1>(d, Mp, ws, err, st, ev0, ev1);
    case 2: return tc::run<2>(d, Mp, ws, err, st, ev0, ev1);
    case 3: return tc::run<3>(d, Mp, ws, err, st, ev0, ev1);
    default: return tc::run<4>(d, Mp, ws, err, st, ev0, ev1);
    }
}

cudaError_t launch_gemm_sub_tc(const uint32_t *A, int64_t lda, const uint32_t *B, int64_t ldb, uint32_t *C,
                               int64_t ldc, int64_t M, int64_t N, int64_t K, ModP Mp, void *ws, int *err,
                               cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1, int add)
{
    GemmDesc d{A, lda, dconst(0), dconst(0), B, ldb, dconst(0), dconst(0), C, ldc, dconst(0), dconst(0),
               M, dconst(N), dconst(K), add};
    return launch_gemm_tc_desc(d, Mp, ws, err, st, ev0, ev1);
}

// ---------------------------------------------------------------------------
// Allocation-free Schur update (cup_mm_sub_noalloc): the limb planes live in a
// fixed scratch array of the module instead of handle-owned memory.
// ---------------------------------------------------------------------------
#define CUP_NOALLOC_SCRATCH_BYTES (16u << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[CUP_NOALLOC_SCRATCH_BYTES];
static __device__ __align__(256) int g_noalloc_err[64];

namespace {
struct NoallocDev {
    bool ready = false;
    void *scratch = nullptr;
    int *err = nullptr;
};
constexpr int kNoallocDevs = 64;
NoallocDev g_noalloc_dev[kNoallocDevs];
std::mutex g_noalloc_mu;
}  // namespace

extern "C" cup_status cup_mm_sub_noalloc(uint32_t *C, int64_t ldc, const uint32_t *A, int64_t lda,
                                         const uint32_t *B, int64_t ldb, int64_t M, int64_t N, int64_t K,
                                         uint32_t p, void *stream)
{
    if (M < 0 || N < 0 || K < 0) return CUP_ERR_ARG;
    if (!cup_internal_prime_ok(p)) return CUP_ERR_PRIME;
    if (M == 0 || N == 0 || K == 0) return CUP_OK;
    if (!C || !A || !B || ldc < N || lda < K || ldb < N) return CUP_ERR_ARG;
    if (tc_workspace_bytes(p, M, N, K) > (size_t)CUP_NOALLOC_SCRATCH_BYTES) return CUP_ERR_TOO_LARGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocDevs) return CUP_ERR_CUDA;
    NoallocDev &d = g_noalloc_dev[dev];
    {
        // once per device, with that device current: device addresses of the scratch
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!d.ready) {
            void *ws = nullptr, *err = nullptr;
            if (cudaGetSymbolAddress(&ws, g_noalloc_scratch) != cudaSuccess) return CUP_ERR_CUDA;
            if (cudaGetSymbolAddress(&err, g_noalloc_err) != cudaSuccess) return CUP_ERR_CUDA;
            d.scratch = ws;
            d.err = (int *)err;
            d.ready = true;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(d.err, 0, sizeof(int), st) != cudaSuccess) return CUP_ERR_CUDA;
    if (launch_gemm_sub_tc(A, lda, B, ldb, C, ldc, M, N, K, make_modp(p), d.scratch, d.err, st) != cudaSuccess)
        return CUP_ERR_CUDA;
    int herr = 0;
    if (cudaMemcpyAsync(&herr, d.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return CUP_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CUP_ERR_CUDA;
    return herr ? CUP_ERR_TIMEOUT : CUP_OK;
}
