// Screened direct and exchange integrals between Wannier functions (Sec. 2.4):
//   U_{i0jR}(w) = 1/N_q sum_q e^{-iq.R} [ sum_{G,G' in eps} n_i(q+G) W_GG'(q,w) n_j(q+G')^* + sum_tail n_i v n_j^* ]
//   J_{i0jR}(w) = 1/N_q sum_q           [ sum_{G,G' in eps} p_ijR(q+G) W_GG'   p_ijR(q+G')^* + sum_tail |p_ijR|^2 v ]
// (Eq. matrix_U, Eq. matrix_J with rho = n / |q+G| and W = v^1/2 eps^-1 v^1/2 of Eq. Wq), and the bare
// forms over the whole wave-function sphere with v = 4 pi / (Omega |q+G|^2) (Eq. matrix_V, Eq. matrix_X):
//   n_i(q+G)   = 1/N_k sum_k            <phi~_{i,k+q}| e^{i(q+G).r} |phi~_{i,k}>   (density of Wannier function i)
//   p_ijR(q+G) = 1/N_k sum_k e^{-ik.R}  <phi~_{i,k+q}| e^{i(q+G).r} |phi~_{j,k}>   (pair product phi_i0^* phi_jR)
// The orbital pair densities <phi~_{a,k+q}|e^{i(q+G).r}|phi~_{o,k}> come from the band pair-density
// kernels run on the Wannier coefficient vectors (a band view of nocc = nemp = nw), read back on the
// whole wave-function sphere of q.  Three kernels then:
//   k_wan_density   rows B[b][G] (b < nw: n_b; b = nw + (r nw + i) nw + j: p_ijR_r), a k sum per G;
//   k_wan_wrhs      Y[f][b][g] = sum_g' W_f[g][g'] conj(B[b][eps(g')]) on the epsilon sphere, each W
//                   row read once for every b (FP64, bound by the FP64 pipe for more than a few b);
//   k_wan_reduce    the bilinear forms with the tail (or, bare, the whole sphere), times e^{-iq.R} / N_q,
//                   added into U and J.
#include <cmath>
#include <cstring>

#include "rp_internal.h"

namespace rp {

#define WI_ROWS 8          // W rows per CTA of k_wan_wrhs
#define WI_KC 64           // G' per shared-memory chunk

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {   // a * conj(b)
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// B[b][G] for the nb = nw + nR nw^2 rows; one CTA per G of the wave-function sphere, the row M[G][.]
// (nk nw^2 pair densities) staged through shared memory in chunks of k points
__global__ void __launch_bounds__(256) k_wan_density(const double2* __restrict__ M, long long ldm, int nk, int nw, int nR,
                                                     const double2* __restrict__ phase /* [nR][nk] */, int kc,
                                                     double2* __restrict__ B, int ngp) {
    extern __shared__ double2 row[];
    const int g = blockIdx.x;
    const int nw2 = nw * nw, nb = nw + nR * nw2;
    const double2* src = M + (size_t)g * ldm;
    double2 acc[4];
    for (int i = 0; i < 4; ++i) acc[i] = make_double2(0.0, 0.0);
    for (int k0 = 0; k0 < nk; k0 += kc) {
        const int kn = min(kc, nk - k0);
        __syncthreads();
        for (int e = threadIdx.x; e < kn * nw2; e += blockDim.x) row[e] = src[(size_t)k0 * nw2 + e];
        __syncthreads();
        for (int t = 0; t < 4; ++t) {
            const int b = threadIdx.x + t * blockDim.x;
            if (b >= nb) break;
            double2 a = acc[t];
            if (b < nw) {
                for (int k = 0; k < kn; ++k) {
                    const double2 v = row[k * nw2 + b * nw + b];
                    a.x += v.x;
                    a.y += v.y;
                }
            } else {
                const int x = b - nw, r = x / nw2, ij = x % nw2;
                const double2* ph = phase + (size_t)r * nk + k0;
                for (int k = 0; k < kn; ++k) {
                    const double2 v = cmul(ph[k], row[k * nw2 + ij]);
                    a.x += v.x;
                    a.y += v.y;
                }
            }
            acc[t] = a;
        }
    }
    const double s = 1.0 / nk;
    for (int t = 0; t < 4; ++t) {
        const int b = threadIdx.x + t * blockDim.x;
        if (b < nb) B[(size_t)b * ngp + g] = make_double2(acc[t].x * s, acc[t].y * s);
    }
}

// Y[f][b][g] = sum_g' W[f][g][g'] conj(B[b][pe[g']]) for the epsilon-sphere rows g of this CTA
__global__ void __launch_bounds__(256) k_wan_wrhs(const double2* __restrict__ W, int ng, const double2* __restrict__ B,
                                                  int ngp, const int* __restrict__ pe, int nb, double2* __restrict__ Y) {
    __shared__ double2 ws[WI_ROWS][WI_KC];
    extern __shared__ double2 bs[];                     // [nb][WI_KC]
    const int f = blockIdx.y, g0 = blockIdx.x * WI_ROWS;
    const double2* Wf = W + (size_t)f * ng * ng;
    const int nout = WI_ROWS * nb;
    double2 acc[8];
    for (int i = 0; i < 8; ++i) acc[i] = make_double2(0.0, 0.0);
    for (int c0 = 0; c0 < ng; c0 += WI_KC) {
        const int cn = min(WI_KC, ng - c0);
        __syncthreads();
        for (int e = threadIdx.x; e < WI_ROWS * WI_KC; e += blockDim.x) {
            const int r = e / WI_KC, c = e % WI_KC;
            ws[r][c] = (g0 + r < ng && c < cn) ? Wf[(size_t)(g0 + r) * ng + c0 + c] : make_double2(0.0, 0.0);
        }
        for (int e = threadIdx.x; e < nb * WI_KC; e += blockDim.x) {
            const int b = e / WI_KC, c = e % WI_KC;
            bs[e] = c < cn ? B[(size_t)b * ngp + pe[c0 + c]] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        for (int t = 0; t < 8; ++t) {
            const int o = threadIdx.x + t * blockDim.x;
            if (o >= nout) break;
            const int r = o / nb, b = o % nb;
            double2 a = acc[t];
            for (int c = 0; c < cn; ++c) {
                const double2 v = cmulc(ws[r][c], bs[b * WI_KC + c]);
                a.x += v.x;
                a.y += v.y;
            }
            acc[t] = a;
        }
    }
    for (int t = 0; t < 8; ++t) {
        const int o = threadIdx.x + t * blockDim.x;
        if (o >= nout) break;
        const int r = o / nb, b = o % nb;
        if (g0 + r < ng) Y[((size_t)f * nb + b) * ng + g0 + r] = acc[t];
    }
}

// one CTA per (f, output): U[f][r][i][j] or J[f][r][i][j] (+)= its bilinear form / N_q (U with e^{-iq.R})
__global__ void __launch_bounds__(256) k_wan_reduce(const double2* __restrict__ B, int ngp, const double* __restrict__ v,
                                                    const unsigned char* __restrict__ in_eps,
                                                    const int* __restrict__ pe, int ng, const double2* __restrict__ Y,
                                                    int nw, int nR, const double2* __restrict__ qph, double inv_nq,
                                                    int accumulate, double2* __restrict__ U, double2* __restrict__ J) {
    __shared__ double2 red[256];
    const int nw2 = nw * nw, nb = nw + nR * nw2;
    const int f = blockIdx.y;
    const int o = blockIdx.x;                         // [0, nR nw2): U entries, then [nR nw2, 2 nR nw2): J
    const bool isJ = o >= nR * nw2;
    const int x = isJ ? o - nR * nw2 : o, r = x / nw2, ij = x % nw2, i = ij / nw, j = ij % nw;
    const int ba = isJ ? nw + x : i, bb = isJ ? nw + x : j;
    double2 a = make_double2(0.0, 0.0);
    // the epsilon sphere through W (Y holds W conj(B) there); without W the whole sphere is bare
    if (Y) {
        const double2* y = Y + ((size_t)f * nb + bb) * ng;
        for (int g = threadIdx.x; g < ng; g += blockDim.x) {
            const double2 t = cmul(B[(size_t)ba * ngp + pe[g]], y[g]);
            a.x += t.x;
            a.y += t.y;
        }
    }
    for (int g = threadIdx.x; g < ngp; g += blockDim.x) {
        if (Y && in_eps[g]) continue;
        const double2 t = cmulc(B[(size_t)ba * ngp + g], B[(size_t)bb * ngp + g]);
        a.x += t.x * v[g];
        a.y += t.y * v[g];
    }
    red[threadIdx.x] = a;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[threadIdx.x].x += red[threadIdx.x + s].x;
            red[threadIdx.x].y += red[threadIdx.x + s].y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double2 t = red[0];
        if (!isJ) t = cmul(qph[r], t);
        t.x *= inv_nq;
        t.y *= inv_nq;
        double2* out = (isJ ? J : U) + ((size_t)f * nR + r) * nw2 + ij;
        if (accumulate) {
            out->x += t.x;
            out->y += t.y;
        } else {
            *out = t;
        }
    }
}

cudaError_t launch_wan_density(const double2* M, long long ldm, int nk, int nw, int nR, const double2* phase,
                               double2* B, int ngp, cudaStream_t st) {
    const int nw2 = nw * nw;
    const int kc = std::max(1, std::min(nk, 4096 / nw2));
    const size_t smem = (size_t)kc * nw2 * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(k_wan_density, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_wan_density<<<ngp, 256, smem, st>>>(M, ldm, nk, nw, nR, phase, kc, B, ngp);
    return cudaGetLastError();
}

cudaError_t launch_wan_wrhs(const double2* W, int ng, int nf, const double2* B, int ngp, const int* pe, int nb,
                            double2* Y, cudaStream_t st) {
    const size_t smem = (size_t)nb * WI_KC * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(k_wan_wrhs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_wan_wrhs<<<dim3((ng + WI_ROWS - 1) / WI_ROWS, nf), 256, smem, st>>>(W, ng, B, ngp, pe, nb, Y);
    return cudaGetLastError();
}

cudaError_t launch_wan_reduce(const double2* B, int ngp, const double* v, const unsigned char* in_eps, const int* pe,
                              int ng, const double2* Y, int nw, int nR, int nf, const double2* qph, double inv_nq,
                              int accumulate, double2* U, double2* J, cudaStream_t st) {
    k_wan_reduce<<<dim3(2 * nR * nw * nw, nf), 256, 0, st>>>(B, ngp, v, in_eps, pe, ng, Y, nw, nR, qph, inv_nq,
                                                            accumulate, U, J);
    return cudaGetLastError();
}

}  // namespace rp
