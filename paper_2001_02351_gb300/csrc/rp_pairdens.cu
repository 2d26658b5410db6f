// Pair densities M^G_ab(k+q,k) by the Fourier route of Sec. 2.3 (Eq. ism):
//   1. gather C_G(k) of every band into a Miller box (shifted by -G0 for the empty
//      bands taken at k' = k + q - G0),
//   2. inverse transform box -> real-space grid, one axis at a time (Eq. pak on the grid:
//      u(r) = sum_G C_G e^{+iG.r}),
//   3. pointwise product p_ab(r) = conj(u_a(r)) u_b(r),
//   4. forward transform with the same +i sign (the matrix element carries e^{+iG.r}),
//      pruned on every axis to the Miller values present in the epsilon sphere,
//   5. read-back on the sphere and normalisation by 1/(N1 N2 N3).
// Every transform stage is a pruned discrete Fourier sum along one axis written as a
// batched product with a small phase matrix E[out][in].
#include "rp_internal.h"

namespace rp {

template <typename C>
struct CT;
template <>
struct CT<double2> {
    using R = double;
    static __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
};
template <>
struct CT<float2> {
    using R = float;
    static __device__ __forceinline__ float2 make(float a, float b) { return make_float2(a, b); }
};

// Scatter the plane-wave coefficients of the bands of k into boxes [band][B][B][B].
// Slot s < nocc: occupied band s at k.  Slot s >= nocc: empty band s at k' = kp[k],
// placed at Miller index m - G0(k), so that its transform is u~_a(r) = sum C e^{i(G-G0).r}.
__global__ void k_scatter_box(const double2* __restrict__ coef, const int* __restrict__ miller,
                              const int* __restrict__ npw, int npw_max, int nband, int nocc,
                              const int* __restrict__ kp, const int* __restrict__ g0, int k0, int nkb,
                              int lb, double2* __restrict__ box) {
    const int B = 2 * lb + 1;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long total = (long long)nkb * nband * npw_max;
    if (t >= total) return;
    int p = (int)(t % npw_max);
    int s = (int)((t / npw_max) % nband);
    int kl = (int)(t / ((long long)npw_max * nband));
    int k = k0 + kl;
    int ks = (s < nocc) ? k : kp[k];
    if (p >= npw[ks]) return;
    const int* m = miller + ((size_t)ks * npw_max + p) * 3;
    int sh0 = 0, sh1 = 0, sh2 = 0;
    if (s >= nocc) { sh0 = g0[3 * k]; sh1 = g0[3 * k + 1]; sh2 = g0[3 * k + 2]; }
    int i0 = m[0] - sh0 + lb, i1 = m[1] - sh1 + lb, i2 = m[2] - sh2 + lb;
    size_t dst = (((size_t)(kl * nband + s) * B + i0) * B + i1) * B + i2;
    box[dst] = coef[((size_t)ks * nband + s) * npw_max + p];
}

// Y[b][j][c] = sum_i E[j][i] X[b][i][c]   (one output per thread, c fastest)
template <typename C>
__global__ void k_axis_pass(const C* __restrict__ X, C* __restrict__ Y, const C* __restrict__ E,
                            long long nb, int nin, int nout, int nc, long long sxb, long long sxi,
                            long long syb, long long syj) {
    using R = typename CT<C>::R;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long total = nb * nout * nc;
    if (t >= total) return;
    int c = (int)(t % nc);
    int j = (int)((t / nc) % nout);
    long long b = t / ((long long)nc * nout);
    const C* x = X + b * sxb + c;
    const C* e = E + (size_t)j * nin;
    R re = 0, im = 0;
    for (int i = 0; i < nin; ++i) {
        C v = x[i * sxi];
        C w = e[i];
        re += w.x * v.x - w.y * v.y;
        im += w.x * v.y + w.y * v.x;
    }
    Y[b * syb + (long long)j * syj + c] = CT<C>::make(re, im);
}

// p[pa][o][r] = conj(u[nocc + a0 + pa][r]) * u[o][r]
template <typename C>
__global__ void k_pair_product(const C* __restrict__ u, long long nr, int nocc, int a0, int na,
                               C* __restrict__ p) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long total = (long long)na * nocc * nr;
    if (t >= total) return;
    long long r = t % nr;
    int o = (int)((t / nr) % nocc);
    int pa = (int)(t / (nr * nocc));
    C a = u[(size_t)(nocc + a0 + pa) * nr + r];
    C b = u[(size_t)o * nr + r];
    p[t] = CT<C>::make(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// M[g][col0 + pair] = (1/Nr) sum_x Ex[gx(g)][x] T2[pair][x][gy(g)][gz(g)]
template <typename C>
__global__ void k_sphere_readout(const C* __restrict__ T2, const C* __restrict__ Ex,
                                 const int* __restrict__ gpos, int ng, int npair, int n1, int ny,
                                 int nz, typename CT<C>::R scale, double2* __restrict__ M,
                                 long long ldm, long long col0) {
    using R = typename CT<C>::R;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long total = (long long)ng * npair;
    if (t >= total) return;
    int pr = (int)(t % npair);
    int g = (int)(t / npair);
    int gx = gpos[3 * g], gy = gpos[3 * g + 1], gz = gpos[3 * g + 2];
    const C* src = T2 + (size_t)pr * n1 * ny * nz + (size_t)gy * nz + gz;
    const C* e = Ex + (size_t)gx * n1;
    R re = 0, im = 0;
    for (int x = 0; x < n1; ++x) {
        C v = src[(size_t)x * ny * nz];
        C w = e[x];
        re += w.x * v.x - w.y * v.y;
        im += w.x * v.y + w.y * v.x;
    }
    M[(size_t)g * ldm + col0 + pr] = make_double2((double)(re * scale), (double)(im * scale));
}

static inline unsigned grid_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

cudaError_t launch_gather_inverse(rp_ctx* c, int k0, int nkb, cudaStream_t st) {
    const int B = 2 * c->lb + 1;
    const int N1 = c->fft[0], N2 = c->fft[1], N3 = c->fft[2];
    const long long nbands = (long long)nkb * c->nband;
    const size_t box = (size_t)nbands * B * B * B, u1 = (size_t)nbands * N1 * B * B,
                 u2 = (size_t)nbands * N1 * N2 * B, uu = (size_t)nbands * c->nr;
    if (ensure(c, c->s_box, box * sizeof(double2)) || ensure(c, c->s_u1, u1 * sizeof(double2)) ||
        ensure(c, c->s_u2, u2 * sizeof(double2)) || ensure(c, c->s_u, uu * sizeof(double2)))
        return cudaErrorMemoryAllocation;
    double2* dbox = (double2*)c->s_box.p;
    cudaError_t e = cudaMemsetAsync(dbox, 0, box * sizeof(double2), st);
    if (e != cudaSuccess) return e;
    const int bs = 256;
    long long n = (long long)nkb * c->nband * c->npw_max;
    k_scatter_box<<<grid_for(n, bs), bs, 0, st>>>((const double2*)c->d_coef.p, (const int*)c->d_miller.p,
                                                  (const int*)c->d_npw.p, c->npw_max, c->nband, c->nocc,
                                                  (const int*)c->plan.d_kp.p, (const int*)c->plan.d_g0.p, k0,
                                                  nkb, c->lb, dbox);
    // m1 -> x
    n = nbands * N1 * (long long)B * B;
    k_axis_pass<double2><<<grid_for(n, bs), bs, 0, st>>>(dbox, (double2*)c->s_u1.p, (const double2*)c->d_einv[0].p,
                                                         nbands, B, N1, B * B, (long long)B * B * B, (long long)B * B,
                                                         (long long)N1 * B * B, (long long)B * B);
    // m2 -> y
    n = nbands * N1 * (long long)N2 * B;
    k_axis_pass<double2><<<grid_for(n, bs), bs, 0, st>>>((const double2*)c->s_u1.p, (double2*)c->s_u2.p,
                                                         (const double2*)c->d_einv[1].p, nbands * N1, B, N2, B,
                                                         (long long)B * B, (long long)B, (long long)N2 * B,
                                                         (long long)B);
    // m3 -> z
    n = nbands * N1 * (long long)N2 * N3;
    k_axis_pass<double2><<<grid_for(n, bs), bs, 0, st>>>((const double2*)c->s_u2.p, (double2*)c->s_u.p,
                                                         (const double2*)c->d_einv[2].p, nbands * N1 * N2, B, N3, 1,
                                                         (long long)B, 1LL, (long long)N3, 1LL);
    return cudaGetLastError();
}

cudaError_t launch_pair_forward(rp_ctx* c, int nkb, double2* M, long long ldm, long long col0, cudaStream_t st,
                                int* nlaunch) {
    const QPlan& P = c->plan;
    const int N1 = c->fft[0], N2 = c->fft[1], N3 = c->fft[2];
    const int nx = P.nset[0], ny = P.nset[1], nz = P.nset[2];
    (void)nx;
    const long long nr = c->nr;
    // empty bands per sub-block: keep the product scratch near 256 MB
    int na = (int)std::max(1LL, std::min((long long)c->nemp, (256LL << 20) / ((long long)c->nocc * nr * 16)));
    const size_t pbytes = (size_t)na * c->nocc * nr * sizeof(double2);
    const size_t t1 = (size_t)na * c->nocc * N1 * N2 * nz * sizeof(double2);
    const size_t t2 = (size_t)na * c->nocc * N1 * ny * nz * sizeof(double2);
    if (ensure(c, c->s_p, pbytes) || ensure(c, c->s_t1, t1) || ensure(c, c->s_t2, t2)) return cudaErrorMemoryAllocation;
    const int bs = 256;
    for (int kl = 0; kl < nkb; ++kl) {
        const double2* u = (const double2*)c->s_u.p + (size_t)kl * c->nband * nr;
        for (int a0 = 0; a0 < c->nemp; a0 += na) {
            int nab = std::min(na, c->nemp - a0);
            long long npair = (long long)nab * c->nocc;
            long long n = npair * nr;
            k_pair_product<double2><<<grid_for(n, bs), bs, 0, st>>>(u, nr, c->nocc, a0, nab, (double2*)c->s_p.p);
            // z -> gz (innermost axis)
            n = npair * N1 * N2 * nz;
            k_axis_pass<double2><<<grid_for(n, bs), bs, 0, st>>>((const double2*)c->s_p.p, (double2*)c->s_t1.p,
                                                                 (const double2*)P.d_efwd[2].p, npair * N1 * N2, N3, nz,
                                                                 1, (long long)N3, 1LL, (long long)nz, 1LL);
            // y -> gy
            n = npair * N1 * ny * nz;
            k_axis_pass<double2><<<grid_for(n, bs), bs, 0, st>>>((const double2*)c->s_t1.p, (double2*)c->s_t2.p,
                                                                 (const double2*)P.d_efwd[1].p, npair * N1, N2, ny, nz,
                                                                 (long long)N2 * nz, (long long)nz,
                                                                 (long long)ny * nz, (long long)nz);
            // x -> gx on the sphere points
            n = (long long)P.ng * npair;
            long long col = col0 + (long long)kl * c->nemp * c->nocc + (long long)a0 * c->nocc;
            k_sphere_readout<double2><<<grid_for(n, bs), bs, 0, st>>>((const double2*)c->s_t2.p,
                                                                      (const double2*)P.d_efwd[0].p,
                                                                      (const int*)P.d_gpos.p, P.ng, (int)npair, N1, ny,
                                                                      nz, 1.0 / (double)nr, M, ldm, col);
            *nlaunch += 4;
        }
    }
    return cudaGetLastError();
}

}  // namespace rp
