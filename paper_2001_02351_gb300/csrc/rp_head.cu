// Head row of the pair densities at q -> 0 for an insulator (Sec. 2.3, Eq. eps00, Eq. momentum):
//   u_b = qhat.p_ao(k) / (E_ak - E_ok),   p_ao(k) = sum_G conj(C_a(k+G)) (k+G) C_o(k+G)
// (the k.p limit of M^{G=0}_ao(k+q, k) / |q| along the unit direction qhat; exact for a local
// potential).  Appended as an extra row of the pair-density block, it makes the contraction of
// Eq. chi produce the head (lim chi_00 / q^2) and the wings (lim chi_G0 / |q|, chi_0G / |q|) with the
// body.  Per k it is a small complex product U = C_emp^* diag(qhat.(k+G)) C_occ^T over the k point's
// plane waves: one CTA per (k, 32 empty bands, 32 occupied bands), the G sum staged through shared
// memory in chunks of 32, four outputs per thread.
#include "rp_internal.h"

namespace rp {

#define HR_T 32     // bands per tile side
#define HR_GC 32    // plane waves per chunk

template <typename R>
struct HrC;
template <>
struct HrC<float> {
    using C = float2;
    __device__ static C mk(float x, float y) { return make_float2(x, y); }
};
template <>
struct HrC<double> {
    using C = double2;
    __device__ static C mk(double x, double y) { return make_double2(x, y); }
};

__device__ __forceinline__ void store_c(float2* p, double x, double y) { *p = make_float2((float)x, (float)y); }
__device__ __forceinline__ void store_c(double2* p, double x, double y) { *p = make_double2(x, y); }

template <typename R, typename CO>
__global__ void __launch_bounds__(256) k_head_row(const double2* __restrict__ coef, const int* __restrict__ miller,
                                                  const int* __restrict__ npw, int npw_max, int nband, int nocc,
                                                  int nemp, const double* __restrict__ energy, int k0, int n1, int n2,
                                                  int n3, double r00, double r01, double r02, double r10, double r11,
                                                  double r12, double r20, double r21, double r22, double qx, double qy,
                                                  double qz, CO* __restrict__ M, long long col0) {
    using C = typename HrC<R>::C;
    __shared__ C sa[HR_T][HR_GC + 1], so[HR_T][HR_GC + 1];
    __shared__ R ss[HR_GC];
    const int k = k0 + blockIdx.z;
    const int a0 = blockIdx.x * HR_T, o0 = blockIdx.y * HR_T;
    const int i1 = k / (n2 * n3), i2 = (k / n3) % n2, i3 = k % n3;
    const double kf0 = (double)i1 / n1, kf1 = (double)i2 / n2, kf2 = (double)i3 / n3;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;         // outputs (a0 + ty + 16 j, o0 + tx + 16 i)
    R acc[2][2][2] = {};
    const int np = npw[k];
    const double2* ck = coef + (size_t)k * nband * npw_max;
    for (int g0 = 0; g0 < np; g0 += HR_GC) {
        __syncthreads();
        if (threadIdx.x < HR_GC) {
            const int g = g0 + threadIdx.x;
            R s = 0;
            if (g < np) {
                const int* m = miller + ((size_t)k * npw_max + g) * 3;
                const double f0 = m[0] + kf0, f1 = m[1] + kf1, f2 = m[2] + kf2;
                // qhat . (k + G) with k + G = f B (rows of B the reciprocal vectors)
                const double cx = f0 * r00 + f1 * r10 + f2 * r20;
                const double cy = f0 * r01 + f1 * r11 + f2 * r21;
                const double cz = f0 * r02 + f1 * r12 + f2 * r22;
                s = (R)(qx * cx + qy * cy + qz * cz);
            }
            ss[threadIdx.x] = s;
        }
        for (int e = threadIdx.x; e < HR_T * HR_GC; e += 256) {
            const int r = e / HR_GC, c = e % HR_GC, g = g0 + c;
            const int a = a0 + r, o = o0 + r;
            double2 va = make_double2(0.0, 0.0), vo = make_double2(0.0, 0.0);
            if (g < np && a < nemp) va = ck[(size_t)(nocc + a) * npw_max + g];
            if (g < np && o < nocc) vo = ck[(size_t)o * npw_max + g];
            sa[r][c] = HrC<R>::mk((R)va.x, (R)va.y);
            so[r][c] = HrC<R>::mk((R)vo.x, (R)vo.y);
        }
        __syncthreads();
#pragma unroll 4
        for (int c = 0; c < HR_GC; ++c) {
            const R s = ss[c];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const C a = sa[ty + 16 * j][c];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const C o = so[tx + 16 * i][c];
                    // conj(a) * s * o
                    acc[j][i][0] += s * (a.x * o.x + a.y * o.y);
                    acc[j][i][1] += s * (a.x * o.y - a.y * o.x);
                }
            }
        }
    }
    const double* ek = energy + (size_t)k * nband;
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int a = a0 + ty + 16 * j, o = o0 + tx + 16 * i;
            if (a < nemp && o < nocc) {
                const double d = ek[nocc + a] - ek[o];
                const long long b = ((long long)blockIdx.z * nemp + a) * nocc + o;
                store_c(M + col0 + b, (double)acc[j][i][0] / d, (double)acc[j][i][1] / d);
            }
        }
}

cudaError_t launch_head_row(rp_ctx* c, int k0, int nkb, const double qhat[3], bool fp32, void* M, long long col0,
                            cudaStream_t st) {
    const dim3 grid((c->nemp + HR_T - 1) / HR_T, (c->nocc + HR_T - 1) / HR_T, nkb);
    const double* b = c->recip;
    if (fp32)
        k_head_row<float, float2><<<grid, 256, 0, st>>>(
            (const double2*)c->d_coef.p, (const int*)c->d_miller.p, (const int*)c->d_npw.p, c->npw_max, c->nband,
            c->nocc, c->nemp, (const double*)c->d_energy.p, k0, c->kmesh[0], c->kmesh[1], c->kmesh[2], b[0], b[1], b[2],
            b[3], b[4], b[5], b[6], b[7], b[8], qhat[0], qhat[1], qhat[2], (float2*)M, col0);
    else
        k_head_row<double, double2><<<grid, 256, 0, st>>>(
            (const double2*)c->d_coef.p, (const int*)c->d_miller.p, (const int*)c->d_npw.p, c->npw_max, c->nband,
            c->nocc, c->nemp, (const double*)c->d_energy.p, k0, c->kmesh[0], c->kmesh[1], c->kmesh[2], b[0], b[1], b[2],
            b[3], b[4], b[5], b[6], b[7], b[8], qhat[0], qhat[1], qhat[2], (double2*)M, col0);
    return cudaGetLastError();
}

}  // namespace rp
