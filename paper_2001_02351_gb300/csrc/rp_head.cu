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

// ---------------------------------------------------------------------------------------------
// Intraband plasma frequency (Sec. 2.3, Eq. plasma), a Fermi-surface integral over all loaded bands:
//   (w_pl^2)^{mu nu} = (4 pi / Omega) (2 / N_k) sum_k sum_a (1 - T_ak^2) x_ak p^mu_aa(k) p^nu_aa(k),
// p_aa(k) = sum_G |C_a(k+G)|^2 (k+G) and x_ak the delta(E_F - E) weight of mesh point k over the 24
// tetrahedra around it: each tetrahedron adds (1/6) g[d1, d2, d3, d4, d_j], g(x) = (x - E_F)^3_+ , which
// is a quarter of the cubic B-spline on those five knots evaluated at E_F (Curry-Schoenberg; the
// Cox-de Boor recursion below has only non-negative terms).  One warp per (k, band): lanes over the
// plane waves for p, lane 0 for the weight; the six tensor components are added with FP64 atomics.

__device__ double bspline4_at(double t, const double* xs) {
    // normalised cubic B-spline on the sorted knots xs[0..4] at t
    double m[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const double w = xs[i + 1] - xs[i];
        m[i] = (w > 0.0 && t >= xs[i] && t < xs[i + 1]) ? 1.0 / w : 0.0;
    }
#pragma unroll
    for (int k = 2; k <= 4; ++k) {
#pragma unroll
        for (int i = 0; i + k <= 4; ++i) {
            const double w = xs[i + k] - xs[i];
            m[i] = w > 0.0 ? (double)k / ((k - 1) * w) * ((t - xs[i]) * m[i] + (xs[i + k] - t) * m[i + 1]) : 0.0;
        }
    }
    return m[0];
}

__global__ void __launch_bounds__(256) k_plasma(const double2* __restrict__ coef, const int* __restrict__ miller,
                                                const int* __restrict__ npw, int npw_max, int nband,
                                                const double* __restrict__ energy, const double* __restrict__ T,
                                                const int* __restrict__ tets, const int* __restrict__ tetk, int nk,
                                                int n1, int n2, int n3, double r00, double r01, double r02,
                                                double r10, double r11, double r12, double r20, double r21,
                                                double r22, double ef, double scale, double* __restrict__ out) {
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (wid >= nk * nband) return;
    const int k = wid / nband, a = wid % nband;
    // delta weight (lane 0)
    double x = 0.0;
    if (lane == 0) {
        for (int s = 0; s < 24; ++s) {
            const int e = tetk[24 * k + s];
            if (e < 0) continue;
            const int t = e >> 2, j = e & 3;
            double d[5];
#pragma unroll
            for (int i = 0; i < 4; ++i) d[i] = energy[(size_t)tets[4 * t + i] * nband + a];
            d[4] = d[j];
            // sort five values (insertion)
#pragma unroll
            for (int i = 1; i < 5; ++i) {
                const double v = d[i];
                int p = i - 1;
                while (p >= 0 && d[p] > v) { d[p + 1] = d[p]; --p; }
                d[p + 1] = v;
            }
            x += bspline4_at(ef, d) * 0.25 / 6.0;
        }
        if (T) {
            const double tt = T[(size_t)k * nband + a];
            x *= 1.0 - tt * tt;
        }
    }
    x = __shfl_sync(0xffffffffu, x, 0);
    if (x == 0.0) return;                       // the whole warp: nothing on the Fermi surface here
    const int i1 = k / (n2 * n3), i2 = (k / n3) % n2, i3 = k % n3;
    const double kf0 = (double)i1 / n1, kf1 = (double)i2 / n2, kf2 = (double)i3 / n3;
    double p0 = 0.0, p1 = 0.0, p2 = 0.0;
    const double2* c = coef + ((size_t)k * nband + a) * npw_max;
    for (int g = lane; g < npw[k]; g += 32) {
        const int* m = miller + ((size_t)k * npw_max + g) * 3;
        const double f0 = m[0] + kf0, f1 = m[1] + kf1, f2 = m[2] + kf2;
        const double w = c[g].x * c[g].x + c[g].y * c[g].y;
        p0 += w * (f0 * r00 + f1 * r10 + f2 * r20);
        p1 += w * (f0 * r01 + f1 * r11 + f2 * r21);
        p2 += w * (f0 * r02 + f1 * r12 + f2 * r22);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        p0 += __shfl_down_sync(0xffffffffu, p0, off);
        p1 += __shfl_down_sync(0xffffffffu, p1, off);
        p2 += __shfl_down_sync(0xffffffffu, p2, off);
    }
    if (lane == 0) {
        const double s = scale * x;
        atomicAdd(out + 0, s * p0 * p0);
        atomicAdd(out + 1, s * p0 * p1);
        atomicAdd(out + 2, s * p0 * p2);
        atomicAdd(out + 4, s * p1 * p1);
        atomicAdd(out + 5, s * p1 * p2);
        atomicAdd(out + 8, s * p2 * p2);
    }
}

cudaError_t launch_plasma(rp_ctx* c, double ef, double* out, cudaStream_t st) {
    const double* b = c->recip;
    const long long warps = (long long)c->nk * c->nband;
    const double scale = (4.0 * M_PI / c->omega) * (2.0 / c->nk);
    k_plasma<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(
        (const double2*)c->d_coef.p, (const int*)c->d_miller.p, (const int*)c->d_npw.p, c->npw_max, c->nband,
        (const double*)c->d_energy.p, c->T.empty() ? nullptr : (const double*)c->d_T.p, (const int*)c->d_tets.p,
        (const int*)c->d_tetk.p, c->nk, c->kmesh[0], c->kmesh[1], c->kmesh[2], b[0], b[1], b[2], b[3], b[4], b[5], b[6],
        b[7], b[8], ef, scale, out);
    return cudaGetLastError();
}

}  // namespace rp
