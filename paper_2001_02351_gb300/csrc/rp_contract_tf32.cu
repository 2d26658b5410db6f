// chi[f][G][G'] (+)= sum_b w[f][b] M[G][b] conj(M[G'][b])      (Eq. chi), TF32x3 tier.
//
// Same real form as the BF16x3 kernel (K interleaves re, im of each pair; for each G' the
// weighted operand contributes a re-row (P, Q) and an im-row (-Q, P), P = wr mr + wi mi,
// Q = wr mi - wi mr), on the warp-level tensor-core instruction mma.sync m16n8k8 with TF32
// inputs: every real operand is split x = hi + lo (hi = x rounded to TF32, lo = x - hi) and the
// product is a_hi b_hi + a_hi b_lo + a_lo b_hi, accumulated in FP32 registers over one chunk (16
// reals: at most 16 roundings of 2^-23, below the 2^-22 of the split) and added into FP64
// registers after every chunk; the FP64 sums are added into chi at the end.
// CTA: 256 threads, tile 64 G rows x 64 G' (128 weighted rows); K chunk of 16 reals (8 pairs)
// staged in shared memory as TF32 hi / lo.
#include "rp_internal.h"

namespace rp {

#define TF_TM 64                 // G rows per CTA
#define TF_TN 64                 // G' per CTA (128 weighted rows)
#define TF_KC 16                 // reals per chunk
#define TF_LD (TF_KC + 4)        // padded row: conflict-free fragment loads

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// split into TF32 hi (bit pattern) and lo (rounded to TF32 as well)
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}

template <typename CM>
__global__ void __launch_bounds__(256) k_contract_tf32x3(const CM* __restrict__ M, long long ldm, long long K,
                                                         const double2* __restrict__ w, long long ldw,
                                                         long long col0w, int ng, double2* __restrict__ chi,
                                                         int accumulate) {
    __shared__ uint32_t Ah[TF_TM][TF_LD], Al[TF_TM][TF_LD];
    __shared__ uint32_t Bh[2 * TF_TN][TF_LD], Bl[2 * TF_TN][TF_LD];
    const int f = blockIdx.z;
    const int row0 = blockIdx.y * TF_TM, g0 = blockIdx.x * TF_TN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 2) * 32;            // 2 warps along G rows
    const int wn = (warp & 3) * 32;             // 4 warps along the 128 weighted rows
    const int gid = lane >> 2, tig = lane & 3;
    const double2* wf = w + (size_t)f * ldw + col0w;

    float acc[2][4][4];
    double sum[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f, sum[i][j][e] = 0.0;

    const long long nchunk = (2 * K + TF_KC - 1) / TF_KC;
    for (long long c = 0; c < nchunk; ++c) {
        const long long p0 = c * (TF_KC / 2);        // first pair of the chunk
        __syncthreads();
        // A: rows G (TF_TM) x 16 pairs; one pair (re, im) per element
        for (int e = tid; e < TF_TM * (TF_KC / 2); e += 256) {
            const int r = e / (TF_KC / 2), p = e % (TF_KC / 2);
            float2 m = make_float2(0.f, 0.f);
            if (row0 + r < ng && p0 + p < K) {
                const CM v = M[(size_t)(row0 + r) * ldm + p0 + p];
                m = make_float2((float)v.x, (float)v.y);
            }
            uint32_t h0, l0, h1, l1;
            split_tf32(m.x, h0, l0);
            split_tf32(m.y, h1, l1);
            Ah[r][2 * p] = h0; Ah[r][2 * p + 1] = h1;
            Al[r][2 * p] = l0; Al[r][2 * p + 1] = l1;
        }
        // B: for each G' the re-row (P, Q) and the im-row (-Q, P) of w conj(M)
        for (int e = tid; e < TF_TN * (TF_KC / 2); e += 256) {
            const int r = e / (TF_KC / 2), p = e % (TF_KC / 2);
            float P = 0.f, Q = 0.f;
            if (g0 + r < ng && p0 + p < K) {
                const CM mv = M[(size_t)(g0 + r) * ldm + p0 + p];
                const float2 m = make_float2((float)mv.x, (float)mv.y);
                const double2 wv = wf[p0 + p];
                const float wr = (float)wv.x, wi = (float)wv.y;
                P = wr * m.x + wi * m.y;
                Q = wr * m.y - wi * m.x;
            }
            uint32_t ph, pl, qh, ql, nqh, nql;
            split_tf32(P, ph, pl);
            split_tf32(Q, qh, ql);
            nqh = qh ^ 0x80000000u;
            nql = ql ^ 0x80000000u;
            Bh[r][2 * p] = ph; Bh[r][2 * p + 1] = qh;
            Bl[r][2 * p] = pl; Bl[r][2 * p + 1] = ql;
            Bh[TF_TN + r][2 * p] = nqh; Bh[TF_TN + r][2 * p + 1] = ph;
            Bl[TF_TN + r][2 * p] = nql; Bl[TF_TN + r][2 * p + 1] = pl;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < TF_KC; ks += 8) {
            uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + gid;
                ah[i][0] = Ah[r][ks + tig];     ah[i][1] = Ah[r + 8][ks + tig];
                ah[i][2] = Ah[r][ks + tig + 4]; ah[i][3] = Ah[r + 8][ks + tig + 4];
                al[i][0] = Al[r][ks + tig];     al[i][1] = Al[r + 8][ks + tig];
                al[i][2] = Al[r][ks + tig + 4]; al[i][3] = Al[r + 8][ks + tig + 4];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = wn + j * 8 + gid;
                bh[j][0] = Bh[n][ks + tig]; bh[j][1] = Bh[n][ks + tig + 4];
                bl[j][0] = Bl[n][ks + tig]; bl[j][1] = Bl[n][ks + tig + 4];
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    mma_tf32(acc[i][j], ah[i], bh[j]);
                    mma_tf32(acc[i][j], ah[i], bl[j]);
                    mma_tf32(acc[i][j], al[i], bh[j]);
                }
        }
        {
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int e = 0; e < 4; ++e) sum[i][j][e] += (double)acc[i][j][e], acc[i][j][e] = 0.f;
        }
    }
    // fragment (i, j, e): G row wm + 16 i + gid + 8 (e >> 1), weighted row wn + 8 j + 2 tig + (e & 1);
    // weighted rows below TF_TN are Re chi[G][g0 + row], the rest Im chi[G][g0 + row - TF_TN]
    double* out = reinterpret_cast<double*>(chi + (size_t)f * ng * ng);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int r = row0 + wm + 16 * i + gid + 8 * (e >> 1);
                const int wr = wn + 8 * j + 2 * tig + (e & 1);
                const int comp = wr >= TF_TN;
                const int gp = g0 + wr - comp * TF_TN;
                if (r < ng && gp < ng) {
                    double* p = out + ((size_t)r * ng + gp) * 2 + comp;
                    *p = accumulate ? *p + sum[i][j][e] : sum[i][j][e];
                }
            }
}

cudaError_t launch_contract_tf32x3(const void* M, bool m32, long long ldm, long long K, const double2* w,
                                   long long ldw, long long col0w, int nf, int ng, double2* chi, int accumulate,
                                   cudaStream_t st) {
    dim3 grid((ng + TF_TN - 1) / TF_TN, (ng + TF_TM - 1) / TF_TM, nf);
    if (m32)
        k_contract_tf32x3<float2><<<grid, 256, 0, st>>>((const float2*)M, ldm, K, w, ldw, col0w, ng, chi, accumulate);
    else
        k_contract_tf32x3<double2><<<grid, 256, 0, st>>>((const double2*)M, ldm, K, w, ldw, col0w, ng, chi,
                                                         accumulate);
    return cudaGetLastError();
}

}  // namespace rp
