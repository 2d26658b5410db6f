// chi[f][G][G'] = sum_b w[f][b] M[G][b] conj(M[G'][b])   (Eq. chi)  --  BF16x3 on tcgen05.
//
// Real form of the complex product: with b running over pairs and the real index
// k' = 2b + {0,1} interleaving (re, im), the stored row M[G][.] is the interleaved real row, and
// for each frequency f and each G' the weighted operand w_f conj(M[G']) contributes two rows:
//   re-row (P, Q), im-row (-Q, P)  with  P = wr mr + wi mi,  Q = wr mi - wi mr,
// so that  <re-row G', row G> = Re chi_f[G][G'],  <im-row G', row G> = Im chi_f[G][G'].
// Each real operand x is split x = hi + lo into two bf16 and the product is
// a_hi b_hi + a_hi b_lo + a_lo b_hi (three MMAs), accumulated in FP32 in tensor memory over a
// window of TC_FLUSH_STAGES stages and then added into the FP64 result.
//
// Tile (one tcgen05.mma M = 128, N = BN, K = 16 per step): the 128 rows of the MMA's A side are
// built in shared memory from 32 rows M[G'] and the weights of two frequencies
// (re f0 | im f0 | re f1 | im f1, 32 rows each); the BN rows of the B side are raw rows M[G],
// loaded by TMA.  BN (160 .. 256, a template parameter) is chosen per NG by the launcher (least
// padding of NG to a multiple of BN, or a measured choice); NG pads to multiples of 32 and BN
// only.  A job is a pair of such
// tiles (four frequencies, the same 32 G' and the same 208 G) over one accumulation window: each
// stage of raw rows, the operand every tile re-reads from L2, feeds both tiles, and one load of
// M[G'] feeds four frequencies.  The two tiles have their own accumulators in tensor memory and
// their own built buffer, so the builders make one tile while the tensor core multiplies the
// other.  The windows of a tile are added into chi with FP64 atomics, so jobs spread evenly over
// the SMs.  A tile whose two frequencies both lie beyond nf (the last group when nf = 4 n + 2, or
// nf <= 2) is not built, multiplied or flushed; each role counts the stages and jobs of each tile
// separately, so the barrier phases stay paired.
//
// CTA: 14 warps.  warp 0 = TMA producer (raw rows M[G], rows M[G'], the stage's weights of the four
// frequencies; the stages two ahead are prefetched into L2), warp 1 = MMA issuer, warps 2-9 =
// builders of the weighted rows (scale by w, split, write the 128B-swizzled K-major tile), warps
// 10-13 = epilogue (tcgen05.ld -> FP64 atomics).
// Every wait is bounded; a wait that gives up (after the caller's limit, 2 s by default) records
// where in err_flag[1] and the CTA leaves through the common teardown: its copies and MMAs in
// flight are waited for (with the fixed 2 s limit), then TMEM is freed.
#include <cuda.h>
#include <cuda_bf16.h>

#include "rp_internal.h"

namespace rp {

#define TC_NS 2                 // load stages (two, plus L2 prefetch of the stages ahead)
#define TC_BM 128               // built rows per tile (MMA M)
#define TC_GN 32                // G' per tile and frequency
#define TC_BK 64                // reals per stage
#define TC_FLUSH_STAGES 128     // stages per FP32 accumulation window (8192 reals)
#define TC_BUILD_SPLIT 0        // 1: each tile has its own TC_NBUILD / 2 builder threads
#define TC_NBUILD 256           // builder threads (warps 2 ..), one 16-B chunk of a stage's rows each
#define TC_EPI_WARPS 4          // epilogue warps (4: one per TMEM lane quarter; 8: two, half the columns each)
#define TC_THREADS (64 + TC_NBUILD + 32 * TC_EPI_WARPS)
#define TC_TMEM_COLS 512        // the accumulators of the two tiles, BN columns each, 256 apart
#define TC_NF 4                 // frequencies per job (two tiles of two)

#define TC_R_BYTES (TC_GN * TC_BK * 2)            // 4 KB
#define TC_W_BYTES (TC_BK / 2 * 8)                // 32 complex float weights = 256 B
#define TC_B_BYTES (TC_BM * TC_BK * 2)            // 16 KB (128 built rows)

// shared-memory layout for BN raw rows per tile; every swizzled buffer starts on 1024 B
template <int BN>
struct TcL {
    static constexpr int RAW = BN * TC_BK * 2;                       // one bf16 half of the raw rows
    static constexpr int OFF_R = 2 * RAW;
    static constexpr int OFF_W = 2 * RAW + 2 * TC_R_BYTES;
    static constexpr int STAGE_LOAD = 2 * RAW + 2 * TC_R_BYTES + TC_NF * TC_W_BYTES;
    static constexpr int STAGE = OFF_W + 1024;
    static constexpr int B0 = TC_NS * STAGE;
    static constexpr int BAR = B0 + 2 * 2 * TC_B_BYTES;
    static constexpr int TOTAL = BAR + 256 + 1024;
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "MMA N: a multiple of 16 up to 256");
    static_assert(RAW % 1024 == 0 && OFF_W % 1024 == 0, "swizzle atoms aligned");
    static_assert(256 + BN <= TC_TMEM_COLS, "two accumulators fit the allocation");
    static_assert(TOTAL <= 232448, "shared memory per CTA");
    static_assert(TC_NF * TC_W_BYTES <= STAGE - OFF_W, "weights of a stage fit their region");
};

#define TC_WAIT_NS 2000000000ULL   // default limit of a wait, and the limit of the teardown's drains

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false (and err_flag set to `code`) if the phase does not complete within limit_ns;
// a zero limit makes one non-blocking test
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code,
                                          uint64_t limit_ns = TC_WAIT_NS) {
    if (limit_ns == 0) {
        if (mbar_test(bar, parity)) return true;
        atomicExch(err, code);
        return false;
    }
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (true) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try(bar, parity)) return true;
        if (gtimer() - t0 > limit_ns) break;
    }
    atomicExch(err, code);
    return false;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"((uint64_t)src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global [%0, {%1, %2}];" ::"l"((uint64_t)map), "r"(x), "r"(y)
                 : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// shared-memory matrix descriptor: K-major, 128B swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// kind::f16 instruction descriptor: D f32, A bf16, B bf16, both K-major, M = 128, N = BN
template <int BN>
__host__ __device__ constexpr uint32_t tc_idesc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}

template <int BN>
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(tc_idesc<BN>()), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ uint32_t sw128_off(int row, int chunk) {
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void split2(float x, float& hi, float& lo) {
    hi = __bfloat162float(__float2bfloat16_rn(x));
    lo = x - hi;
}

struct TcArgs {
    const float2* w32;      // [TC_NF * nfq][kp2/2] complex float weights of this block (zero padded)
    long long K;
    int ng, nf, nfq, nblk, mt, nst, nwin;
    double2* chi;
    int* err;
    unsigned long long wait_ns;   // limit of the pipeline's waits (the teardown drains use TC_WAIT_NS)
};

// tcgen05.ld of 32 or 16 consecutive accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld32(uint32_t src, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(src));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t src, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(src));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_contract_bf16x3(const __grid_constant__ CUtensorMap raw_hi, const __grid_constant__ CUtensorMap raw_lo,
                      const __grid_constant__ CUtensorMap row_hi, const __grid_constant__ CUtensorMap row_lo,
                      TcArgs args) {
    using L = TcL<BN>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + L::BAR;
    // barriers: full[NS], empty[NS], and per tile t: bready, bfree (its built buffer), accf, acce
    // (its accumulator); done
    auto full = [&](int s) { return bar0 + 8 * s; };
    auto empty = [&](int s) { return bar0 + 8 * (TC_NS + s); };
    auto bready = [&](int t) { return bar0 + 8 * (2 * TC_NS + t); };
    auto bfree = [&](int t) { return bar0 + 8 * (2 * TC_NS + 2 + t); };
    auto accf = [&](int t) { return bar0 + 8 * (2 * TC_NS + 4 + t); };
    auto acce = [&](int t) { return bar0 + 8 * (2 * TC_NS + 6 + t); };
    const uint32_t done_bar = bar0 + 8 * (2 * TC_NS + 8);
    uint32_t* taddr_slot = (uint32_t*)(smem + L::BAR + 8 * (2 * TC_NS + 9));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_NS; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), TC_NBUILD + 1);
        }
        for (int t = 0; t < 2; ++t) {
            mbar_init(bready(t), TC_BUILD_SPLIT ? TC_NBUILD / 2 : TC_NBUILD);
            mbar_init(bfree(t), 1);
            mbar_init(accf(t), 1);
            mbar_init(acce(t), 32 * TC_EPI_WARPS);
        }
        mbar_init(done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(taddr_slot)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *taddr_slot;

    const int ntile = args.nfq * args.nblk * args.mt;
    const int njobs = ntile * args.nwin;
    const int nst = args.nst;
    int* err = args.err;
    const uint64_t lim = args.wait_ns;
    // job -> (accumulation window, group of four frequencies, G' block, G tile); consecutive jobs
    // share a window.  The last block and tile are moved back to end at ng, so that (for ng >=
    // BN) every box lies inside the arrays; a block or tile writes only the rows from its own
    // start (nown, mown) on, so rows covered twice are added once.
    // tile t of a job in frequency group fq holds frequencies 4 fq + 2 t, + 1: it is live if the first is
    auto live_tile = [&](int fq, int t) { return TC_NF * fq + 2 * t < args.nf; };
    auto job_tile = [&](int job, int& w0, int& w1, int& fq, int& n0, int& m0, int& nown, int& mown) {
        const int win = job / ntile, t = job % ntile;
        fq = t / (args.nblk * args.mt);
        const int r = t % (args.nblk * args.mt);
        nown = (r / args.mt) * TC_GN;
        mown = (r % args.mt) * BN;
        n0 = min(nown, max(0, args.ng - TC_GN));
        m0 = min(mown, max(0, args.ng - BN));
        w0 = win * TC_FLUSH_STAGES;
        w1 = min(nst, w0 + TC_FLUSH_STAGES);
    };

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            long long sg = 0;
            bool ok = true;
            const long long kpad = (long long)nst * (TC_BK / 2);
            for (int job = blockIdx.x; job < njobs && ok; job += gridDim.x) {
                int w0, w1, fq, n0, m0, nown, mown;
                job_tile(job, w0, w1, fq, n0, m0, nown, mown);
                // L2 prefetch only of boxes that lie inside the arrays
                const bool pf_raw = m0 + BN <= args.ng, pf_row = n0 + TC_GN <= args.ng;
                const float2* wrow = args.w32 + (size_t)(TC_NF * fq) * kpad;
                for (int st = w0; st < w1; ++st, ++sg) {
                    const int s = (int)(sg % TC_NS);
                    const uint32_t ph = (uint32_t)((sg / TC_NS) & 1);
                    if (st + 2 < w1) {
                        const int xp = (st + 2) * TC_BK;
                        if (pf_raw) {
                            tma_prefetch_2d(&raw_hi, xp, m0);
                            tma_prefetch_2d(&raw_lo, xp, m0);
                        }
                        if (pf_row) {
                            tma_prefetch_2d(&row_hi, xp, n0);
                            tma_prefetch_2d(&row_lo, xp, n0);
                        }
                    }
                    if (!(ok = mbar_wait(empty(s), ph ^ 1, err, 101, lim))) break;
                    const uint32_t base = sbase + s * L::STAGE;
                    mbar_expect_tx(full(s), L::STAGE_LOAD);
#pragma unroll
                    for (int fi = 0; fi < TC_NF; ++fi)
                        bulk_load(base + L::OFF_W + fi * TC_W_BYTES, wrow + (size_t)fi * kpad + (size_t)st * (TC_BK / 2),
                                  TC_W_BYTES, full(s));
                    const int x = st * TC_BK;
                    tma_load_2d(base, &raw_hi, x, m0, full(s));
                    tma_load_2d(base + L::RAW, &raw_lo, x, m0, full(s));
                    tma_load_2d(base + L::OFF_R, &row_hi, x, n0, full(s));
                    tma_load_2d(base + L::OFF_R + TC_R_BYTES, &row_lo, x, n0, full(s));
                }
            }
            // copies still in flight land before the CTA leaves
            for (long long k = (sg > TC_NS ? sg - TC_NS : 0); k < sg; ++k)
                mbar_wait(full((int)(k % TC_NS)), (uint32_t)((k / TC_NS) & 1), err, 102);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            long long sg = 0, cs[2] = {0, 0}, cj[2] = {0, 0};   // stages; per tile: live stages, live jobs
            bool ok = true;
            for (int job = blockIdx.x; job < njobs && ok; job += gridDim.x) {
                int w0, w1, fq, n0, m0, nown, mown;
                job_tile(job, w0, w1, fq, n0, m0, nown, mown);
                const bool lv[2] = {live_tile(fq, 0), live_tile(fq, 1)};
                // the live accumulators drained by the epilogue of their previous job
                for (int t = 0; t < 2 && ok; ++t)
                    if (lv[t]) ok = mbar_wait(acce(t), (uint32_t)((cj[t] & 1) ^ 1), err, 111, lim);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int st = w0; st < w1; ++st, ++sg) {
                    const int s = (int)(sg % TC_NS);
                    if (!(ok = mbar_wait(full(s), (uint32_t)((sg / TC_NS) & 1), err, 112, lim))) break;
                    const uint32_t g_hi = sbase + s * L::STAGE, g_lo = g_hi + L::RAW;
                    for (int t = 0; t < 2; ++t) {
                        if (!lv[t]) continue;
                        if (!(ok = mbar_wait(bready(t), (uint32_t)(cs[t] & 1), err, 113, lim))) break;
                        ++cs[t];
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t d = tmem + (uint32_t)(t * 256);
                        const uint32_t b_hi = sbase + L::B0 + t * 2 * TC_B_BYTES, b_lo = b_hi + TC_B_BYTES;
#pragma unroll
                        for (int kk = 0; kk < TC_BK / 16; ++kk) {
                            const uint32_t off = kk * 32;
                            const uint32_t first = (st == w0 && kk == 0) ? 0u : 1u;
                            mma_bf16<BN>(d, sw128_desc(b_hi + off), sw128_desc(g_hi + off), first);
                            mma_bf16<BN>(d, sw128_desc(b_hi + off), sw128_desc(g_lo + off), 1u);
                            mma_bf16<BN>(d, sw128_desc(b_lo + off), sw128_desc(g_hi + off), 1u);
                        }
                        mma_commit(bfree(t));
                    }
                    if (!ok) break;
                    mma_commit(empty(s));
                }
                if (ok)
                    for (int t = 0; t < 2; ++t)
                        if (lv[t]) {
                            mma_commit(accf(t));
                            ++cj[t];
                        }
            }
            // all issued MMAs complete before teardown
            mma_commit(done_bar);
            mbar_wait(done_bar, 0, err, 114);
        }
    } else if (warp < 2 + TC_NBUILD / 32) {
        // ---------------- builders of the weighted rows (TC_NBUILD threads, one 16-B chunk each) ----
        const int tid = (threadIdx.x - 64) % 256;
        const int tsel = TC_BUILD_SPLIT ? (threadIdx.x - 64) / 256 : -1;   // the one tile built (split)
        const int r = tid >> 3, c = tid & 7;
        long long sg = 0, cs[2] = {0, 0};
        bool ok = true;
        for (int job = blockIdx.x; job < njobs && ok; job += gridDim.x) {
            int w0, w1, fq, n0, m0, nown, mown;
            job_tile(job, w0, w1, fq, n0, m0, nown, mown);
            const bool lv[2] = {live_tile(fq, 0), live_tile(fq, 1)};
            for (int st = w0; st < w1 && ok; ++st, ++sg) {
                const int s = (int)(sg % TC_NS);
                if (!(ok = mbar_wait(full(s), (uint32_t)((sg / TC_NS) & 1), err, 121, lim))) break;
                const unsigned char* stage = smem + s * L::STAGE;
                const unsigned char* rhi = stage + L::OFF_R;
                const unsigned char* rlo = rhi + TC_R_BYTES;
                const uint32_t o = sw128_off(r, c);
                const uint4 vh = *reinterpret_cast<const uint4*>(rhi + o);
                const uint4 vl = *reinterpret_cast<const uint4*>(rlo + o);
                const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&vh);
                const __nv_bfloat162* l2 = reinterpret_cast<const __nv_bfloat162*>(&vl);
                float mr[4], mi[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float2 hh = __bfloat1622float2(h2[i]);
                    const float2 ll = __bfloat1622float2(l2[i]);
                    mr[i] = hh.x + ll.x;
                    mi[i] = hh.y + ll.y;
                }
                for (int t = 0; t < 2; ++t) {
                    if (!lv[t] || (TC_BUILD_SPLIT && t != tsel)) continue;
                    if (!(ok = mbar_wait(bfree(t), (uint32_t)((cs[t] & 1) ^ 1), err, 122, lim))) break;
                    ++cs[t];
                    unsigned char* bhi = smem + L::B0 + t * 2 * TC_B_BYTES;
                    unsigned char* blo = bhi + TC_B_BYTES;
#pragma unroll
                    for (int fq2 = 0; fq2 < 2; ++fq2) {
                        const float2* ws =
                            reinterpret_cast<const float2*>(stage + L::OFF_W + (2 * t + fq2) * TC_W_BYTES);
                        const float4 w01 = *reinterpret_cast<const float4*>(ws + 4 * c);
                        const float4 w23 = *reinterpret_cast<const float4*>(ws + 4 * c + 2);
                        const float wr[4] = {w01.x, w01.z, w23.x, w23.z};
                        const float wi[4] = {w01.y, w01.w, w23.y, w23.w};
                        uint32_t reh[4], rel[4], imh[4], iml[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float P = wr[i] * mr[i] + wi[i] * mi[i];
                            const float Q = wr[i] * mi[i] - wi[i] * mr[i];
                            float ph, pl, qh, ql;
                            split2(P, ph, pl);
                            split2(Q, qh, ql);
                            reh[i] = pack_bf16(ph, qh);
                            rel[i] = pack_bf16(pl, ql);
                            imh[i] = pack_bf16(-qh, ph);
                            iml[i] = pack_bf16(-ql, pl);
                        }
                        const int rre = fq2 * 2 * TC_GN + r, rim = rre + TC_GN;
                        *reinterpret_cast<uint4*>(bhi + sw128_off(rre, c)) = make_uint4(reh[0], reh[1], reh[2], reh[3]);
                        *reinterpret_cast<uint4*>(blo + sw128_off(rre, c)) = make_uint4(rel[0], rel[1], rel[2], rel[3]);
                        *reinterpret_cast<uint4*>(bhi + sw128_off(rim, c)) = make_uint4(imh[0], imh[1], imh[2], imh[3]);
                        *reinterpret_cast<uint4*>(blo + sw128_off(rim, c)) = make_uint4(iml[0], iml[1], iml[2], iml[3]);
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_arrive(bready(t));
                }
                if (!ok) break;
                mbar_arrive(empty(s));
            }
        }
    } else {
        // ---------------- epilogue (128 threads, TMEM lanes by warp % 4) ----------------
        // lane quarter q4: 0 = Re f0, 1 = Im f0, 2 = Re f1, 3 = Im f1 of a tile; lane = G' - n0
        constexpr int NCH = BN / 32;                 // 32-column loads, then one of 16 if BN % 32 = 16
        constexpr bool REM = (BN % 32) == 16;
        static_assert(BN % 32 == 0 || REM, "BN is a multiple of 16");
        const int q4 = warp & 3;
        // columns of this warp: chunks [c0e, c1e) (and the 16-column remainder with the second half)
        const int half = TC_EPI_WARPS == 8 ? (warp - (2 + TC_NBUILD / 32)) / 4 : -1;
        const int c0e = half == 1 ? NCH / 2 : 0, c1e = half == 0 ? NCH / 2 : NCH;
        const bool rem_here = REM && half != 0;
        long long cj[2] = {0, 0};
        bool ok = true;
        double* chi = reinterpret_cast<double*>(args.chi);
        for (int job = blockIdx.x; job < njobs && ok; job += gridDim.x) {
            int w0, w1, fq, n0, m0, nown, mown;
            job_tile(job, w0, w1, fq, n0, m0, nown, mown);
            const int gp = n0 + lane;
            const size_t ldo = (size_t)args.ng * 2;
            const int gmin = mown - m0;
            const int gmax = min(BN, args.ng - m0);   // columns [gmin, gmax) are this tile's
            for (int t = 0; t < 2 && ok; ++t) {
                if (!live_tile(fq, t)) continue;
                const int f = TC_NF * fq + 2 * t + (q4 >> 1), comp = q4 & 1;
                const bool live = f < args.nf && gp >= nown && gp < args.ng;
                double* out = chi + (((size_t)f * args.ng + m0) * args.ng + gp) * 2 + comp;
                if (!(ok = mbar_wait(accf(t), (uint32_t)(cj[t] & 1), err, 131, lim))) break;
                ++cj[t];
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t src = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(t * 256);
#pragma unroll 1
                for (int ch = c0e; ch < c1e; ++ch) {
                    uint32_t v[32];
                    tmem_ld32(src + (uint32_t)(ch * 32), v);
                    if (!rem_here && ch == c1e - 1) {
                        // the accumulator is read: the MMA of the next job may overwrite it
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                        mbar_arrive(acce(t));
                    }
                    if (live) {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (ch * 32 + j >= gmin && ch * 32 + j < gmax)
                                atomicAdd(out + (size_t)(ch * 32 + j) * ldo, (double)__uint_as_float(v[j]));
                    }
                }
                if (rem_here) {
                    constexpr int ch = NCH;
                    uint32_t v[16];
                    tmem_ld16(src + (uint32_t)(ch * 32), v);
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    mbar_arrive(acce(t));
                    if (live) {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (ch * 32 + j >= gmin && ch * 32 + j < gmax)
                                atomicAdd(out + (size_t)(ch * 32 + j) * ldo, (double)__uint_as_float(v[j]));
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// hi/lo bf16 split of M (complex double [ng][ldm] from column col0, K columns) into
// real arrays [ng][kp2] (kp2 = 2 * K rounded up to 64), zero padded
template <typename CI>
__global__ void k_split_bf16(const CI* __restrict__ M, long long ldm, long long col0, long long K, int ng,
                             long long kp2, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long half = kp2 / 2;
    if (t >= (long long)ng * half) return;
    const int g = (int)(t / half);
    const long long b = t % half;
    float x = 0.f, y = 0.f;
    if (b < K) {
        const CI v = M[(size_t)g * ldm + col0 + b];
        x = (float)v.x;
        y = (float)v.y;
    }
    const __nv_bfloat16 hx = __float2bfloat16_rn(x), hy = __float2bfloat16_rn(y);
    const __nv_bfloat16 lx = __float2bfloat16_rn(x - __bfloat162float(hx));
    const __nv_bfloat16 ly = __float2bfloat16_rn(y - __bfloat162float(hy));
    __nv_bfloat162 h2, l2;
    h2.x = hx; h2.y = hy;
    l2.x = lx; l2.y = ly;
    reinterpret_cast<__nv_bfloat162*>(hi)[t] = h2;
    reinterpret_cast<__nv_bfloat162*>(lo)[t] = l2;
}

// complex float copy of the weights of this block: w32[f][b] = w[f][col0 + b], b < kpad, for
// f < nrow (rows f >= nf and columns b >= K are zero)
__global__ void k_weights32(const double2* __restrict__ w, long long ldw, long long col0, long long K, int nf,
                            int nrow, long long kpad, float2* __restrict__ w32) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nrow * kpad) return;
    const int f = (int)(t / kpad);
    const long long b = t % kpad;
    float2 v = make_float2(0.f, 0.f);
    if (f < nf && b < K) {
        const double2 d = w[(size_t)f * ldw + col0 + b];
        v = make_float2((float)d.x, (float)d.y);
    }
    w32[t] = v;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

static bool make_map(CUtensorMap* map, void* base, int ng, long long kp2, int rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)kp2, (cuuint64_t)ng};
    cuuint64_t strides[1] = {(cuuint64_t)kp2 * 2};
    cuuint32_t box[2] = {TC_BK, (cuuint32_t)rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

long long tc_kp2(long long K) { return ((2 * K + TC_BK - 1) / TC_BK) * TC_BK; }
int tc_wrows(int nf) { return (nf + TC_NF - 1) / TC_NF * TC_NF; }

cudaError_t launch_split_bf16(const void* M, bool m32, long long ldm, long long col0, long long K, int ng, void* hi,
                              void* lo, cudaStream_t st) {
    const long long kp2 = tc_kp2(K);
    const long long n = (long long)ng * (kp2 / 2);
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (m32)
        k_split_bf16<float2><<<grid, 256, 0, st>>>((const float2*)M, ldm, col0, K, ng, kp2, (__nv_bfloat16*)hi,
                                                   (__nv_bfloat16*)lo);
    else
        k_split_bf16<double2><<<grid, 256, 0, st>>>((const double2*)M, ldm, col0, K, ng, kp2, (__nv_bfloat16*)hi,
                                                    (__nv_bfloat16*)lo);
    return cudaGetLastError();
}

// chi (+)= ... over the K pairs whose bf16 split is in hi/lo ([ng][kp2]); chi must be zeroed by
// the caller before the first accumulation
cudaError_t launch_weights32(long long K, const double2* w, long long ldw, long long col0, int nf, void* w32,
                             cudaStream_t st) {
    const long long kpad = tc_kp2(K) / 2;
    const int nrow = tc_wrows(nf);
    const long long nw = (long long)nrow * kpad;
    k_weights32<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(w, ldw, col0, K, nf, nrow, kpad, (float2*)w32);
    return cudaGetLastError();
}

cudaError_t launch_contract_bf16x3(const void* hi, const void* lo, long long K, int ng, const double2* w,
                                   long long ldw, long long col0, int nf, void* w32, double2* chi, int* err,
                                   int num_sms, cudaStream_t st) {
    cudaError_t e = launch_weights32(K, w, ldw, col0, nf, w32, st);
    if (e != cudaSuccess) return e;
    return launch_contract_bf16x3_core(hi, lo, K, ng, nf, w32, chi, err, num_sms, TC_WAIT_NS, st, 0);
}

// tile widths the kernel is built for
static const int kTcBn[] = {160, 192, 208, 224, 256};

bool tc_bn_supported(int bn) {
    for (int b : kTcBn)
        if (b == bn) return true;
    return false;
}

int tc_bn_candidates(int* out) {
    const int n = (int)(sizeof(kTcBn) / sizeof(kTcBn[0]));
    if (out)
        for (int i = 0; i < n; ++i) out[i] = kTcBn[i];
    return n;
}

__global__ void k_fill_tune(__nv_bfloat16* hi, __nv_bfloat16* lo, long long n, float2* w, long long nw) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n + nw; i += (long long)gridDim.x * blockDim.x) {
        // a hash of the index, scaled into [-1, 1)
        unsigned x = (unsigned)(i * 2654435761ull) ^ (unsigned)(i >> 29);
        x ^= x >> 15; x *= 2246822519u; x ^= x >> 13;
        const float v = (float)(x & 0xffffff) * (2.0f / 16777216.0f) - 1.0f;
        if (i < n) {
            hi[i] = __float2bfloat16_rn(v);
            lo[i] = __float2bfloat16_rn(v * (1.0f / 512.0f));
        } else {
            w[i - n] = make_float2(v, -0.5f * v);
        }
    }
}

cudaError_t launch_fill_tune_operands(void* hi, void* lo, long long n_bf16, void* w32, long long n_w32,
                                      cudaStream_t st) {
    k_fill_tune<<<1024, 256, 0, st>>>((__nv_bfloat16*)hi, (__nv_bfloat16*)lo, n_bf16, (float2*)w32, n_w32);
    return cudaGetLastError();
}

// least padded rows ceil(ng / BN) BN; on a tie the wider tile (fewer raw-row reloads per flop)
int tc_pick_bn(int ng) {
    int best = 208;
    long long best_rows = -1;
    for (int b : kTcBn) {
        const long long rows = (long long)((ng + b - 1) / b) * b;
        if (best_rows < 0 || rows < best_rows || (rows == best_rows && b > best)) {
            best = b;
            best_rows = rows;
        }
    }
    return best;
}

template <int BN>
static cudaError_t launch_bn(const CUtensorMap& mraw_hi, const CUtensorMap& mraw_lo, const CUtensorMap& mrow_hi,
                             const CUtensorMap& mrow_lo, const TcArgs& a, int grid, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_contract_bf16x3<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TcL<BN>::TOTAL);
    if (e != cudaSuccess) return e;
    k_contract_bf16x3<BN><<<grid, TC_THREADS, TcL<BN>::TOTAL, st>>>(mraw_hi, mraw_lo, mrow_hi, mrow_lo, a);
    return cudaGetLastError();
}

cudaError_t launch_contract_bf16x3_core(const void* hi, const void* lo, long long K, int ng, int nf,
                                        const void* w32, double2* chi, int* err, int num_sms,
                                        unsigned long long wait_ns, cudaStream_t st, int bn) {
    if (bn <= 0) bn = tc_pick_bn(ng);
    if (!tc_bn_supported(bn)) return cudaErrorInvalidValue;
    const long long kp2 = tc_kp2(K);
    CUtensorMap mraw_hi, mraw_lo, mrow_hi, mrow_lo;
    if (!make_map(&mraw_hi, const_cast<void*>(hi), ng, kp2, bn) ||
        !make_map(&mraw_lo, const_cast<void*>(lo), ng, kp2, bn) ||
        !make_map(&mrow_hi, const_cast<void*>(hi), ng, kp2, TC_GN) ||
        !make_map(&mrow_lo, const_cast<void*>(lo), ng, kp2, TC_GN))
        return cudaErrorInvalidValue;
    TcArgs a;
    a.w32 = (const float2*)w32; a.K = K;
    a.ng = ng; a.nf = nf; a.nfq = tc_wrows(nf) / TC_NF;
    a.nblk = (ng + TC_GN - 1) / TC_GN;
    a.mt = (ng + bn - 1) / bn;
    a.nst = (int)(kp2 / TC_BK);
    a.nwin = (a.nst + TC_FLUSH_STAGES - 1) / TC_FLUSH_STAGES;
    a.chi = chi; a.err = err;
    a.wait_ns = wait_ns;
    const long long njobs = (long long)a.nfq * a.nblk * a.mt * a.nwin;
    if (njobs > 0x7fffffffLL) return cudaErrorInvalidValue;
    const int grid = njobs < num_sms ? (int)njobs : num_sms;
    switch (bn) {
        case 160: return launch_bn<160>(mraw_hi, mraw_lo, mrow_hi, mrow_lo, a, grid, st);
        case 192: return launch_bn<192>(mraw_hi, mraw_lo, mrow_hi, mrow_lo, a, grid, st);
        case 208: return launch_bn<208>(mraw_hi, mraw_lo, mrow_hi, mrow_lo, a, grid, st);
        case 224: return launch_bn<224>(mraw_hi, mraw_lo, mrow_hi, mrow_lo, a, grid, st);
        default: return launch_bn<256>(mraw_hi, mraw_lo, mrow_hi, mrow_lo, a, grid, st);
    }
}

}  // namespace rp
