// Generalized-tetrahedron pair weights (Eq. Xakqbk, Eq. tetrahedron), FP64.
//
// For one band pair (a empty at k+q, b occupied at k) the vertex weight is
//   x(k) = (1/6) sum over the 24 tetrahedra t containing k of
//          [f_z1 + f_z2][d_1, d_2, d_3, d_4, d_j(k)],
// a fourth-order divided difference (node of k repeated) of f_z(x) = (z-x)^3 log(z-x),
// with d_v = E_a(k_v + q) - E_b(k_v) at the tetrahedron's vertices and
// z1 = w + i d, z2 = -w + i d (time-ordered) or -w - i d (retarded).  Linear
// interpolation of D and of the matrix-element product over a tetrahedron, integrated
// exactly, gives that divided difference (Hermite-Genocchi).
//
// Degeneracy: sorted nodes closer than delta_a + delta_r max(|x|) to their group's
// first node are merged into the group mean.  Numerically, a divided difference over a
// run of nodes whose spread s is at most TAU |z - c| (c its midpoint) is summed from the
// Taylor series f[x_i..x_j] = sum_m f^(m)(c)/m! h_{m-n}(x - c) instead of the recursion;
// when the whole set of five nodes qualifies, only the m >= 4 coefficients appear
// (6 (m-4)!/m! (z-c)^(3-m)) and no logarithm is needed.
#include "rp_internal.h"

namespace rp {

#define TT_TAU 0.5
#define TT_KMAX 40
#define TT_FCH 4

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cinv(double2 a) {
    double d = a.x * a.x + a.y * a.y;
    return make_double2(a.x / d, -a.y / d);
}
__device__ __forceinline__ double2 clog_(double2 a) { return make_double2(log(hypot(a.x, a.y)), atan2(a.y, a.x)); }

// f^(m)(c)/m! = (z-c)^(3-m) * b_m(log(z-c))
__device__ __forceinline__ double2 bcoef(int m, double2 L) {
    switch (m) {
        case 0: return L;
        case 1: return make_double2(-(3.0 * L.x + 1.0), -3.0 * L.y);
        case 2: return make_double2((6.0 * L.x + 5.0) * 0.5, 3.0 * L.y);
        case 3: return make_double2(-(6.0 * L.x + 11.0) / 6.0, -L.y);
        default: return make_double2(6.0 / ((double)m * (m - 1) * (m - 2) * (m - 3)), 0.0);
    }
}

// number of series terms for ratio rho = max|x - c| / |z - c| (rho <= TAU/2)
__device__ __forceinline__ int nterms(double rho) {
    if (rho <= 0.0) return 0;
    int k = (int)ceil(-39.2 / log(rho)) + 6;
    return k > TT_KMAX ? TT_KMAX : k;
}

// divided difference over the sorted run x[i..j] by the Taylor series about its midpoint
__device__ double2 dd_run_series(const double* x, int i, int j, double2 z) {
    const int n = j - i;
    const double c = 0.5 * (x[i] + x[j]);
    const double2 y = make_double2(z.x - c, z.y);
    const double R = hypot(y.x, y.y);
    double tmax = 0.0;
    for (int v = i; v <= j; ++v) tmax = fmax(tmax, fabs(x[v] - c));
    const int K = nterms(tmax / R);
    double h[TT_KMAX + 1];
    h[0] = 1.0;
    for (int k = 1; k <= K; ++k) h[k] = 0.0;
    for (int v = i; v <= j; ++v) {
        const double t = x[v] - c;
        for (int k = 1; k <= K; ++k) h[k] += t * h[k - 1];
    }
    const double2 L = clog_(y);
    const double2 w = cinv(y);
    // sum_k b_{n+k} h_k w^k  by Horner
    double2 S = cscale(bcoef(n + K, L), h[K]);
    for (int k = K - 1; k >= 0; --k) S = cadd(cmul(S, w), cscale(bcoef(n + k, L), h[k]));
    // times y^(3-n)
    double2 p = make_double2(1.0, 0.0);
    if (n <= 3) {
        for (int e = 0; e < 3 - n; ++e) p = cmul(p, y);
    } else {
        for (int e = 0; e < n - 3; ++e) p = cmul(p, w);
    }
    return cmul(S, p);
}

// full divided-difference table (recursion with series for narrow runs)
__device__ double2 dd5_table(const double* x, double2 z) {
    double2 D[5][5];
    for (int i = 0; i < 5; ++i) {
        double2 y = make_double2(z.x - x[i], z.y);
        double2 L = clog_(y);
        D[i][i] = cmul(cmul(cmul(y, y), y), L);
    }
    for (int n = 1; n < 5; ++n)
        for (int i = 0; i + n < 5; ++i) {
            const int j = i + n;
            const double s = x[j] - x[i];
            const double c = 0.5 * (x[i] + x[j]);
            const double R = hypot(z.x - c, z.y);
            if (s <= TT_TAU * R) D[i][j] = dd_run_series(x, i, j, z);
            else D[i][j] = cscale(csub(D[i + 1][j], D[i][j - 1]), 1.0 / s);
        }
    return D[0][4];
}

// One thread per (k, a, o); frequencies in chunks of TT_FCH.
__global__ void k_tetra_weights(const double* __restrict__ E, const double* __restrict__ Tw, int nband, int nocc,
                                int nemp, int nk, const int* __restrict__ kp, const int* __restrict__ tets,
                                const int* __restrict__ tetk, int nf, const double* __restrict__ freq, int axis,
                                int ordering, double delta, double da, double dr, double2* __restrict__ wout) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long K = (long long)nk * nemp * nocc;
    if (t >= K) return;
    const int f_begin = blockIdx.y * TT_FCH;
    const int o = (int)(t % nocc);
    const int a = (int)((t / nocc) % nemp);
    const int k = (int)(t / ((long long)nocc * nemp));
    double pref = 2.0 / (double)nk;
    if (Tw) pref *= 1.0 - Tw[(size_t)kp[k] * nband + nocc + a] * Tw[(size_t)k * nband + o];
    for (int f0 = f_begin; f0 < nf && f0 < f_begin + TT_FCH; f0 += TT_FCH) {
        double2 z[TT_FCH][2];
        double2 acc[TT_FCH];
        for (int q = 0; q < TT_FCH; ++q) {
            acc[q] = make_double2(0.0, 0.0);
            const int f = f0 + q < nf ? f0 + q : nf - 1;
            const double wv = freq[f];
            if (axis == RP_AXIS_REAL) {
                z[q][0] = make_double2(wv, delta);
                z[q][1] = make_double2(-wv, ordering == RP_TIME_ORDERED ? delta : -delta);
            } else {
                z[q][0] = make_double2(0.0, wv + delta);
                z[q][1] = make_double2(0.0, ordering == RP_TIME_ORDERED ? -wv + delta : -wv - delta);
            }
        }
        for (int s = 0; s < 24; ++s) {
            const int code = tetk[24 * k + s];
            const int tt = code >> 2, jv = code & 3;
            double x[5];
            for (int v = 0; v < 4; ++v) {
                const int kv = tets[4 * tt + v];
                x[v] = E[(size_t)kp[kv] * nband + nocc + a] - E[(size_t)kv * nband + o];
            }
            x[4] = x[jv];
            // sort (insertion, 5 elements)
            for (int i = 1; i < 5; ++i) {
                double v = x[i];
                int j = i - 1;
                while (j >= 0 && x[j] > v) { x[j + 1] = x[j]; --j; }
                x[j + 1] = v;
            }
            // merge degenerate groups into their mean
            {
                int gid[5];
                gid[0] = 0;
                double start = x[0];
                for (int i = 1; i < 5; ++i) {
                    const double thr = da + dr * fmax(fabs(start), fabs(x[i]));
                    const bool nw = (x[i] - start) >= thr;
                    gid[i] = gid[i - 1] + (nw ? 1 : 0);
                    if (nw) start = x[i];
                }
                double m[5];
                for (int g = 0; g < 5; ++g) {
                    double sum = 0.0;
                    int cnt = 0;
                    for (int i = 0; i < 5; ++i)
                        if (gid[i] == g) { sum += x[i]; ++cnt; }
                    m[g] = cnt ? sum / cnt : 0.0;
                }
                for (int i = 0; i < 5; ++i) x[i] = m[gid[i]];
            }
            const double c = 0.5 * (x[0] + x[4]);
            const double spread = x[4] - x[0];
            double h[TT_KMAX + 1];
            int hk = -1;   // h_k(x - c) computed up to this order
            for (int q = 0; q < TT_FCH; ++q) {
                if (f0 + q >= nf) break;
                for (int side = 0; side < 2; ++side) {
                    const double2 zz = z[q][side];
                    const double2 y = make_double2(zz.x - c, zz.y);
                    const double R = hypot(y.x, y.y);
                    double2 dd;
                    if (spread <= TT_TAU * R) {
                        const int K = nterms(0.5 * spread / R);
                        if (K > hk) {
                            h[0] = 1.0;
                            for (int kk = 1; kk <= K; ++kk) h[kk] = 0.0;
                            for (int v = 0; v < 5; ++v) {
                                const double tv = x[v] - c;
                                for (int kk = 1; kk <= K; ++kk) h[kk] += tv * h[kk - 1];
                            }
                            hk = K;
                        }
                        const double2 w = cinv(y);
                        double2 S = make_double2(6.0 / ((double)(4 + K) * (3 + K) * (2 + K) * (1 + K)) * h[K], 0.0);
                        for (int kk = K - 1; kk >= 0; --kk) {
                            const double b = 6.0 / ((double)(4 + kk) * (3 + kk) * (2 + kk) * (1 + kk));
                            S = cmul(S, w);
                            S.x += b * h[kk];
                        }
                        dd = cmul(S, w);
                    } else {
                        dd = dd5_table(x, zz);
                    }
                    acc[q] = cadd(acc[q], dd);
                }
            }
        }
        for (int q = 0; q < TT_FCH; ++q) {
            if (f0 + q >= nf) break;
            wout[(size_t)(f0 + q) * K + t] = cscale(acc[q], pref / 6.0);
        }
    }
}

cudaError_t launch_tetra(rp_ctx* c, int axis, int ordering, int nf, const double* d_freq, double delta,
                         double da, double dr, double2* w, cudaStream_t st) {
    const long long K = (long long)c->nk * c->nemp * c->nocc;
    const int bs = 128;
    dim3 grid((unsigned)((K + bs - 1) / bs), (unsigned)((nf + TT_FCH - 1) / TT_FCH));
    k_tetra_weights<<<grid, bs, 0, st>>>(
        (const double*)c->d_energy.p, c->T.empty() ? nullptr : (const double*)c->d_T.p, c->nband, c->nocc,
        c->nemp, c->nk, (const int*)c->plan.d_kp.p, (const int*)c->d_tets.p, (const int*)c->d_tetk.p, nf, d_freq,
        axis, ordering, delta, da, dr, w);
    return cudaGetLastError();
}

}  // namespace rp
