// chi[f][G][G'] (+)= sum_b w[f][b] M[G][b] conj(M[G'][b])      (Eq. chi, FP64)
//
// Native FP64 contraction on the tensor cores with mma.sync m8n8k4 (DMMA).  A CTA owns a
// 64 x 64 tile of one frequency's chi and runs over all pairs b of the block; the
// complex product is four real DMMA per 8x8x4 step (re += ar br - ai bi, im += ar bi + ai br),
// with B = w conj(M) formed while staging the tile in shared memory.
#include "rp_internal.h"

namespace rp {

#define CF_TM 64
#define CF_TK 16

__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(d0), "+d"(d1)
                 : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(128) k_contract_f64(const double2* __restrict__ M, long long ldm, long long K,
                                                      const double2* __restrict__ w, long long ldw, long long col0,
                                                      int ng, double2* __restrict__ chi, int accumulate) {
    __shared__ double Ar[CF_TM][CF_TK + 1], Ai[CF_TM][CF_TK + 1], Br[CF_TM][CF_TK + 1], Bi[CF_TM][CF_TK + 1];
    const int f = blockIdx.z;
    const int row0 = blockIdx.y * CF_TM, col0t = blockIdx.x * CF_TM;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gid = lane >> 2, tig = lane & 3;
    const double2* wf = w + (size_t)f * ldw + col0;

    double accr[4][4][2], acci[4][4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) accr[i][j][0] = accr[i][j][1] = acci[i][j][0] = acci[i][j][1] = 0.0;

    for (long long k0 = 0; k0 < K; k0 += CF_TK) {
        // stage A = M[row tile][k0..k0+16) and B = w * conj(M[col tile][...])
#pragma unroll
        for (int it = 0; it < (CF_TM * CF_TK) / 128; ++it) {
            const int e = tid + it * 128;
            const int r = e / CF_TK, kk = e % CF_TK;
            const long long kg = k0 + kk;
            double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
            if (kg < K) {
                const double2 wv = wf[kg];
                if (row0 + r < ng) a = M[(size_t)(row0 + r) * ldm + kg];
                if (col0t + r < ng) {
                    const double2 m = M[(size_t)(col0t + r) * ldm + kg];
                    // w * conj(m)
                    b = make_double2(wv.x * m.x + wv.y * m.y, wv.y * m.x - wv.x * m.y);
                }
            }
            Ar[r][kk] = a.x; Ai[r][kk] = a.y;
            Br[r][kk] = b.x; Bi[r][kk] = b.y;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < CF_TK; ks += 4) {
            double ar[4], ai[4], nai[4], br[4], bi[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                ar[i] = Ar[wm + i * 8 + gid][ks + tig];
                ai[i] = Ai[wm + i * 8 + gid][ks + tig];
                nai[i] = -ai[i];
                br[i] = Br[wn + i * 8 + gid][ks + tig];
                bi[i] = Bi[wn + i * 8 + gid][ks + tig];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    dmma(accr[i][j][0], accr[i][j][1], ar[i], br[j]);
                    dmma(accr[i][j][0], accr[i][j][1], nai[i], bi[j]);
                    dmma(acci[i][j][0], acci[i][j][1], ar[i], bi[j]);
                    dmma(acci[i][j][0], acci[i][j][1], ai[i], br[j]);
                }
        }
        __syncthreads();
    }
    double2* out = chi + (size_t)f * ng * ng;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int r = row0 + wm + i * 8 + gid;
                const int cidx = col0t + wn + j * 8 + 2 * tig + e;
                if (r < ng && cidx < ng) {
                    double2 v = make_double2(accr[i][j][e], acci[i][j][e]);
                    double2* p = out + (size_t)r * ng + cidx;
                    if (accumulate) { double2 o = *p; v.x += o.x; v.y += o.y; }
                    *p = v;
                }
            }
}

cudaError_t launch_contract_f64(const double2* M, long long ldm, long long K, const double2* w, long long ldw,
                                long long col0, int nf, int ng, double2* chi, int accumulate, cudaStream_t st) {
    dim3 grid((ng + CF_TM - 1) / CF_TM, (ng + CF_TM - 1) / CF_TM, nf);
    k_contract_f64<<<grid, 128, 0, st>>>(M, ldm, K, w, ldw, col0, ng, chi, accumulate);
    return cudaGetLastError();
}

}  // namespace rp
