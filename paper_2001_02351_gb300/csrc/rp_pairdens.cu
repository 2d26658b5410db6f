// Pair densities M^G_ab(k+q,k) by the Fourier route of Sec. 2.3 (Eq. ism):
//   1. gather C_G(k) of every band into a Miller box (shifted by -G0 for the empty
//      bands taken at k' = k + q - G0),
//   2. inverse transform box -> real-space grid, one axis at a time (Eq. pak on the grid:
//      u(r) = sum_G C_G e^{+iG.r}),
//   3. pointwise product p_ab(r) = conj(u_a(r)) u_b(r),
//   4. forward transform with the same +i sign (the matrix element carries e^{+iG.r}),
//      pruned on every axis to the Miller values present in the epsilon sphere,
//   5. read-back on the sphere and normalisation by 1/(N1 N2 N3).
// On transform grids of 16, 24 or 32 points the transforms are in-register line FFTs
// (rp_fft.cuh): k_gather_fft (steps 1-2), k_pair_zy (steps 3-4 along z and y, one x plane per
// CTA) and the x read-out (step 5): k_pair_x_w, a line transform of each (pair, yz) point of the
// symmetric residue window (FP32 lines), or k_pair_x, a sum over x for each sphere point (FP64
// lines).  The other grids take the general path, where each stage is a pruned discrete Fourier
// sum along one axis written as a batched product with a small phase matrix E[out][in].
#include "rp_internal.h"
#include "rp_fft.cuh"

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
template <typename C>
__global__ void k_scatter_box(const double2* __restrict__ coef, const int* __restrict__ miller,
                              const int* __restrict__ npw, int npw_max, int nband, int nocc,
                              const int* __restrict__ kp, const int* __restrict__ g0, int k0, int nkb,
                              int lb, C* __restrict__ box) {
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
    const double2 v = coef[((size_t)ks * nband + s) * npw_max + p];
    box[dst] = CT<C>::make((typename CT<C>::R)v.x, (typename CT<C>::R)v.y);
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
template <typename C, typename CO>
__global__ void k_sphere_readout(const C* __restrict__ T2, const C* __restrict__ Ex,
                                 const int* __restrict__ gpos, int ng, int npair, int n1, int ny,
                                 int nz, typename CT<C>::R scale, CO* __restrict__ M,
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
    M[(size_t)g * ldm + col0 + pr] = CT<CO>::make((typename CT<CO>::R)(re * scale), (typename CT<CO>::R)(im * scale));
}

static inline unsigned grid_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// Gather + inverse transform by line FFTs, one CTA per band (grid N^3, Miller box B^3, B <= N).
// The box is scattered into the first B planes of T[x][m2][m3]; the x transform then runs in
// place, each thread on its own (m2, m3) column of every plane (it reads the column's B entries
// into registers before it writes the N outputs), so no other thread's data is touched.  The y
// and z transforms follow for XG = 256 / N planes at a time through U[x][y][m3], and the z lines
// go straight from registers to u.  Frequency n of a line holds Miller value n (n <= lb) or
// n - N (n >= N - lb); with B <= N the two ranges do not meet.
template <typename C, int N>
__global__ void __launch_bounds__(256) k_gather_fft(const double2* __restrict__ coef, const int* __restrict__ miller,
                                                    const int* __restrict__ npw, int npw_max, int nband, int nocc,
                                                    const int* __restrict__ kp, const int* __restrict__ g0, int k0,
                                                    int lb, C* __restrict__ u) {
    using R = typename CT<C>::R;
    constexpr int XG = 256 / N;
    const int B = 2 * lb + 1, BB = B * B;
    extern __shared__ __align__(16) unsigned char sm_gf[];
    C* T = reinterpret_cast<C*>(sm_gf);      // [N][B][B]; its first B planes are the box
    C* U = T + (size_t)N * BB;               // [XG][N][B]
    const int band = blockIdx.x;             // kl * nband + s
    const int kl = band / nband, s = band % nband;
    const int k = k0 + kl;
    const int ks = (s < nocc) ? k : kp[k];
    for (int e = threadIdx.x; e < B * BB; e += 256) T[e] = CT<C>::make(0, 0);
    __syncthreads();
    int sh0 = 0, sh1 = 0, sh2 = 0;
    if (s >= nocc) { sh0 = g0[3 * k]; sh1 = g0[3 * k + 1]; sh2 = g0[3 * k + 2]; }
    for (int p = threadIdx.x; p < npw[ks]; p += 256) {
        const int* m = miller + ((size_t)ks * npw_max + p) * 3;
        const double2 v = coef[((size_t)ks * nband + s) * npw_max + p];
        T[((m[0] - sh0 + lb) * B + (m[1] - sh1 + lb)) * B + (m[2] - sh2 + lb)] = CT<C>::make((R)v.x, (R)v.y);
    }
    __syncthreads();
    // box index of the Miller value at frequency n, or -1
    auto slot = [&](int n) { return n <= lb ? n + lb : (n >= N - lb ? n - N + lb : -1); };
    // x: m1 -> x on every (m2, m3) column, in place
    for (int l = threadIdx.x; l < BB; l += 256) {
        C v[N];
#pragma unroll
        for (int n = 0; n < N; ++n) {
            const int m = slot(n);
            v[n] = m >= 0 ? T[m * BB + l] : CT<C>::make(0, 0);
        }
        LineFFT<C, N>::run(v);
#pragma unroll
        for (int x = 0; x < N; ++x) T[x * BB + l] = v[x];
    }
    C* dst = u + (size_t)band * N * N * N;
    for (int x0 = 0; x0 < N; x0 += XG) {
        const int xg = min(XG, N - x0);
        __syncthreads();
        // y: m2 -> y on the (x, m3) lines of xg planes
        for (int l = threadIdx.x; l < xg * B; l += 256) {
            const int xl = l / B, m3 = l % B;
            const C* src = T + (size_t)(x0 + xl) * BB + m3;
            C v[N];
#pragma unroll
            for (int n = 0; n < N; ++n) {
                const int m = slot(n);
                v[n] = m >= 0 ? src[m * B] : CT<C>::make(0, 0);
            }
            LineFFT<C, N>::run(v);
#pragma unroll
            for (int y = 0; y < N; ++y) U[(xl * N + y) * B + m3] = v[y];
        }
        __syncthreads();
        // z: m3 -> z on the (x, y) lines, written to the grid
        for (int l = threadIdx.x; l < xg * N; l += 256) {
            const C* src = U + (size_t)l * B;
            C v[N];
#pragma unroll
            for (int n = 0; n < N; ++n) {
                const int m = slot(n);
                v[n] = m >= 0 ? src[m] : CT<C>::make(0, 0);
            }
            LineFFT<C, N>::run(v);
            C* d = dst + ((size_t)x0 * N + l) * N;
#pragma unroll
            for (int z = 0; z < N; ++z) d[z] = v[z];
        }
    }
}

// Gather + inverse transform of one band per CTA: the Miller box of the band (shifted by -G0 for
// the empty bands at k' = k + q - G0) is built in shared memory, then every x plane of the
// real-space grid is formed by three small sums (m1 -> x, m2 -> y, m3 -> z) and written once.
template <typename C>
__global__ void __launch_bounds__(256) k_gather_grid(const double2* __restrict__ coef, const int* __restrict__ miller,
                                                     const int* __restrict__ npw, int npw_max, int nband, int nocc,
                                                     const int* __restrict__ kp, const int* __restrict__ g0, int k0,
                                                     int lb, int N1, int N2, int N3, const C* __restrict__ ex,
                                                     const C* __restrict__ ey, const C* __restrict__ ez,
                                                     C* __restrict__ u) {
    using R = typename CT<C>::R;
    const int B = 2 * lb + 1;
    extern __shared__ __align__(16) unsigned char sm_g[];
    C* box = reinterpret_cast<C*>(sm_g);     // [B][B][B]
    C* u1 = box + B * B * B;                 // [B][B]   (m2, m3) of one x
    C* u2 = u1 + B * B;                      // [N2][B]  (y, m3) of one x
    const int band = blockIdx.x;             // kl * nband + s
    const int kl = band / nband, s = band % nband;
    const int k = k0 + kl;
    const int ks = (s < nocc) ? k : kp[k];
    for (int e = threadIdx.x; e < B * B * B; e += blockDim.x) box[e] = CT<C>::make(0, 0);
    __syncthreads();
    int sh0 = 0, sh1 = 0, sh2 = 0;
    if (s >= nocc) { sh0 = g0[3 * k]; sh1 = g0[3 * k + 1]; sh2 = g0[3 * k + 2]; }
    for (int p = threadIdx.x; p < npw[ks]; p += blockDim.x) {
        const int* m = miller + ((size_t)ks * npw_max + p) * 3;
        const double2 v = coef[((size_t)ks * nband + s) * npw_max + p];
        box[((m[0] - sh0 + lb) * B + (m[1] - sh1 + lb)) * B + (m[2] - sh2 + lb)] = CT<C>::make((R)v.x, (R)v.y);
    }
    C* dst = u + (size_t)band * N1 * N2 * N3;
    for (int x = 0; x < N1; ++x) {
        __syncthreads();
        const C* e1 = ex + (size_t)x * B;
        for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
            R re = 0, im = 0;
            for (int m1 = 0; m1 < B; ++m1) {
                const C v = box[m1 * B * B + e], w = e1[m1];
                re += w.x * v.x - w.y * v.y;
                im += w.x * v.y + w.y * v.x;
            }
            u1[e] = CT<C>::make(re, im);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < N2 * B; e += blockDim.x) {
            const int y = e / B, m3 = e % B;
            const C* e2 = ey + (size_t)y * B;
            R re = 0, im = 0;
            for (int m2 = 0; m2 < B; ++m2) {
                const C v = u1[m2 * B + m3], w = e2[m2];
                re += w.x * v.x - w.y * v.y;
                im += w.x * v.y + w.y * v.x;
            }
            u2[e] = CT<C>::make(re, im);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < N2 * N3; e += blockDim.x) {
            const int y = e / N3, z = e % N3;
            const C* e3 = ez + (size_t)z * B;
            const C* src = u2 + y * B;
            R re = 0, im = 0;
            for (int m3 = 0; m3 < B; ++m3) {
                const C v = src[m3], w = e3[m3];
                re += w.x * v.x - w.y * v.y;
                im += w.x * v.y + w.y * v.x;
            }
            dst[(size_t)x * N2 * N3 + e] = CT<C>::make(re, im);
        }
    }
}


// ---- fused pair kernels (line transforms in registers) ----

// product and z transform: one (pair, x, y) line per thread, pruned to the z values of the sphere
// u holds the bands of nkb k points ([kl][band][line][z]).  A CTA takes 32 consecutive lines of
// one empty band (grid.y runs over (kl, pa), pa < nab) and loops over the occupied bands four at
// a time; the lines are staged in shared memory with coalesced loads (rows padded by one element
// against bank conflicts).  T1 pair index (kl * nab + pa) * nocc + o.
template <typename C, int N3>
__global__ void __launch_bounds__(128) k_pair_z(const C* __restrict__ u, int nband, int nocc, int a0, int nab,
                                                int nlines, const int* __restrict__ zmap, int nz,
                                                C* __restrict__ T1) {
    constexpr int LD = N3 + 1;
    extern __shared__ __align__(16) unsigned char sm_z[];
    C* sa = reinterpret_cast<C*>(sm_z);              // [32][LD]
    C* so = sa + 32 * LD;                            // [4][32][LD]
    const int l0 = blockIdx.x * 32;
    const int kl = blockIdx.y / nab, pa = blockIdx.y % nab;
    const int nl = min(32, nlines - l0);
    const C* uk = u + (size_t)kl * nband * nlines * N3;
    const C* ua = uk + ((size_t)(nocc + a0 + pa) * nlines + l0) * N3;
    for (int e = threadIdx.x; e < nl * N3; e += 128) sa[(e / N3) * LD + e % N3] = ua[e];
    const int li = threadIdx.x & 31, oi = threadIdx.x >> 5;
    for (int o0 = 0; o0 < nocc; o0 += 4) {
        __syncthreads();
        for (int q = 0; q < 4 && o0 + q < nocc; ++q) {
            const C* uo = uk + ((size_t)(o0 + q) * nlines + l0) * N3;
            for (int e = threadIdx.x; e < nl * N3; e += 128) so[q * 32 * LD + (e / N3) * LD + e % N3] = uo[e];
        }
        __syncthreads();
        const int o = o0 + oi;
        if (li >= nl || o >= nocc) continue;
        C x[N3];
#pragma unroll
        for (int z = 0; z < N3; ++z) x[z] = c_conjmul(sa[li * LD + z], so[oi * 32 * LD + li * LD + z]);
        LineFFT<C, N3>::run(x);
        C* dst = T1 + ((size_t)(blockIdx.y * nocc + o) * nlines + l0 + li) * nz;
#pragma unroll
        for (int z = 0; z < N3; ++z) {
            const int iz = zmap[z];
            if (iz >= 0) dst[iz] = x[z];
        }
    }
}

// y transform (pruned) of PPC pairs per CTA into shared memory, then the x sum on the sphere points
template <typename C, int N2, int PPC, typename CO>
__global__ void __launch_bounds__(256) k_pair_yx(const C* __restrict__ T1, int npair, int N1, int nz,
                                                 const int* __restrict__ ymap, int ny,
                                                 const C* __restrict__ Ex, const int* __restrict__ gpos, int ng,
                                                 typename Cx<C>::R scale, CO* __restrict__ M, long long ldm,
                                                 long long col0) {
    using R = typename Cx<C>::R;
    extern __shared__ __align__(16) unsigned char sm_yx[];
    C* T2 = (C*)sm_yx;   // [PPC][N1][ny][nz]
    const int p0 = blockIdx.x * PPC;
    const int tile = N1 * ny * nz;
    for (int ln = threadIdx.x; ln < PPC * N1 * nz; ln += blockDim.x) {
        const int j = ln / (N1 * nz);
        const int x = (ln / nz) % N1, iz = ln % nz;
        if (p0 + j >= npair) continue;
        const C* src = T1 + ((size_t)(p0 + j) * N1 + x) * N2 * nz + iz;
        C v[N2];
#pragma unroll
        for (int y = 0; y < N2; ++y) v[y] = src[(size_t)y * nz];
        LineFFT<C, N2>::run(v);
#pragma unroll
        for (int y = 0; y < N2; ++y) {
            const int iy = ymap[y];
            if (iy >= 0) T2[j * tile + (x * ny + iy) * nz + iz] = v[y];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ng * PPC; t += blockDim.x) {
        const int j = t % PPC, g = t / PPC;
        if (p0 + j >= npair) continue;
        const int gx = gpos[3 * g], gy = gpos[3 * g + 1], gz = gpos[3 * g + 2];
        const C* src = T2 + j * tile + gy * nz + gz;
        const C* e = Ex + (size_t)gx * N1;
        R re = 0, im = 0;
        for (int x = 0; x < N1; ++x) {
            const C v = src[x * ny * nz];
            const C w = e[x];
            re += w.x * v.x - w.y * v.y;
            im += w.x * v.y + w.y * v.x;
        }
        M[(size_t)g * ldm + col0 + p0 + j] = CT<CO>::make((typename CT<CO>::R)(re * scale), (typename CT<CO>::R)(im * scale));
    }
}


// ---- plane-wise pair transform: z and y on chip, one x plane per CTA ----
//
// k_pair_zy: CTA = one x plane of one k of the block and A = 128 / N2 empty bands, whose planes
// stay in shared memory while the occupied bands stream through, one plane per step: the plane
// of band o + 1 is fetched with coalesced 16-byte loads into registers while thread (a, y) forms
// conj(u_a) u_o on its z line of band o, transforms it in registers (pruned to the sphere's z
// residues) and parks it in a double-buffered tile.  Then one thread per (a, sphere z) column
// transforms along y in registers and writes the sphere's y residues to T2[pair][x][iy][iz]; the
// warps without a column go straight on to the next band.  One barrier per occupied band.  The
// y and z axes of T2 hold the residues present on the sphere in ascending order: residue r of
// an axis is kept when bit r of its mask is set, at position popc(mask & (2^r - 1)).
// With W > 0 the y and z axes of T2 instead hold the symmetric window of values -W .. W (value g at
// position g + W; every sphere value lies in it, 2 W + 1 <= N): the stores then have compile-time
// offsets, no mask is tested per output, and the outputs outside the window are never formed.
// k_pair_x: the x sum on the sphere points, M[g][col0 + pair] = scale * sum_x Ex[gx][x] T2[...],
// with T2 streamed through shared memory a few pairs at a time (double-buffered cp.async).
// shared-memory layout of k_pair_zy: planes [N2][LD] (FP32 lines: LD even, so a row is read with
// 16-byte loads, conflict-free for N = 16, 24, 32) and the z-transformed lines [2][A][N2][nz]
// (nz = 2 W + 1 with a window); at N = 24, W = 5 four CTAs fit an SM
template <typename C, int N>
struct ZyLayout {
    static constexpr int A = 128 / N;
    static constexpr int LD = sizeof(C) == 8 ? N + 2 : N + 1;
    static size_t smem(int nz) { return sizeof(C) * ((size_t)(A + 2) * N * LD + (size_t)2 * A * N * nz); }
};

template <typename C, int N3, int N2, int W>
__global__ void __launch_bounds__(128, sizeof(C) == 16 ? 1 : 3) k_pair_zy(const C* __restrict__ u, int nband, int nocc, int e0,
                                                 int nemp, int N1, unsigned zmask, int nz_, unsigned ymask, int ny_,
                                                 C* __restrict__ T2) {
    static_assert(W == 0 || (2 * W + 1 <= N2 && 2 * W + 1 <= N3), "window wider than the plane");
    constexpr int NW = 2 * W + 1;
    const int nz = W > 0 ? NW : nz_, ny = W > 0 ? NW : ny_;
    static_assert(N2 == N3, "square planes");
    using L = ZyLayout<C, N3>;
    constexpr int A = L::A;
    constexpr int LD = L::LD;
    constexpr int PER = 16 / sizeof(C);                 // complex values per 16-byte load
    constexpr int NE = N2 * N3 / PER;                   // 16-byte pieces of a plane
    constexpr int NV = (NE + 127) / 128;                // pieces per thread (the last one guarded)
    static_assert(NE * PER == N2 * N3, "plane must split into 16-byte pieces");
    extern __shared__ __align__(16) unsigned char sm_zy[];
    C* sa = reinterpret_cast<C*>(sm_zy);          // [A][N2][LD]
    C* so = sa + A * N2 * LD;                     // [2][N2][LD]
    C* tz = so + 2 * N2 * LD;                     // [2][A][N2][nz]
    const int x = blockIdx.x, a0 = blockIdx.y * A, kl = blockIdx.z;
    const int na = min(A, nemp - a0);
    const size_t plane = (size_t)N2 * N3;
    const C* uk = u + (size_t)kl * nband * N1 * plane + x * plane;
    for (int q = 0; q < na; ++q) {
        const C* ua = uk + (size_t)(nocc + e0 + a0 + q) * N1 * plane;
        for (int e = threadIdx.x; e < N2 * N3; e += 128) sa[(q * N2 + e / N3) * LD + e % N3] = ua[e];
    }
    // occupied plane 0
    for (int e = threadIdx.x; e < N2 * N3; e += 128) so[(e / N3) * LD + e % N3] = uk[e];
    __syncthreads();
    const int y = threadIdx.x % N2, ai = threadIdx.x / N2;
    const int nyz = ny * nz;
    for (int o = 0; o < nocc; ++o) {
        const C* sb = so + (o & 1) * N2 * LD;
        C* tb = tz + (o & 1) * A * N2 * nz;
        // prefetch plane o + 1 (16-byte loads, consecutive threads on consecutive addresses)
        float4 pf[NV];
        const bool more = o + 1 < nocc;
        if (more) {
            const float4* src = reinterpret_cast<const float4*>(uk + (size_t)(o + 1) * N1 * plane);
#pragma unroll
            for (int i = 0; i < NV; ++i)
                if (i * 128 + (int)threadIdx.x < NE) pf[i] = __ldg(src + i * 128 + threadIdx.x);
        }
        if (ai < na) {
            C v[N3];
            if constexpr (sizeof(C) == 8) {
                const float4* ra = reinterpret_cast<const float4*>(sa + (ai * N2 + y) * LD);
                const float4* rb = reinterpret_cast<const float4*>(sb + y * LD);
#pragma unroll
                for (int z2 = 0; z2 < N3 / 2; ++z2) {
                    const float4 p = ra[z2], q = rb[z2];
                    v[2 * z2] = c_conjmul(make_float2(p.x, p.y), make_float2(q.x, q.y));
                    v[2 * z2 + 1] = c_conjmul(make_float2(p.z, p.w), make_float2(q.z, q.w));
                }
            } else {
#pragma unroll
                for (int z = 0; z < N3; ++z) v[z] = c_conjmul(sa[(ai * N2 + y) * LD + z], sb[y * LD + z]);
            }
            LineFFT<C, N3>::run(v);
            if constexpr (W > 0) {
#pragma unroll
                for (int z = 0; z < N3; ++z) {
                    const int r = z <= N3 / 2 ? z : z - N3;     // signed value of residue z
                    if (r >= -W && r <= W) tb[(ai * N2 + y) * NW + r + W] = v[z];
                }
            } else {
#pragma unroll
                for (int z = 0; z < N3; ++z)
                    if ((zmask >> z) & 1u) tb[(ai * N2 + y) * nz + __popc(zmask & ((1u << z) - 1u))] = v[z];
            }
        }
        if (more) {
            C* dst = so + ((o + 1) & 1) * N2 * LD;
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                if (i * 128 + (int)threadIdx.x >= NE) break;
                const C* c = reinterpret_cast<const C*>(&pf[i]);
                const int e0 = (i * 128 + threadIdx.x) * PER;
#pragma unroll
                for (int j = 0; j < PER; ++j) dst[((e0 + j) / N3) * LD + (e0 + j) % N3] = c[j];
            }
        }
        __syncthreads();
        for (int col = threadIdx.x; col < na * nz; col += 128) {
            const int q = col / nz, iz = col % nz;
            C v[N2];
#pragma unroll
            for (int yy = 0; yy < N2; ++yy) v[yy] = tb[(q * N2 + yy) * nz + iz];
            LineFFT<C, N2>::run(v);
            const size_t pair = ((size_t)kl * nemp + a0 + q) * nocc + o;
            C* dst = T2 + (pair * N1 + x) * nyz + iz;
            if constexpr (W > 0) {
#pragma unroll
                for (int yy = 0; yy < N2; ++yy) {
                    const int r = yy <= N2 / 2 ? yy : yy - N2;
                    if (r >= -W && r <= W) dst[(r + W) * NW] = v[yy];
                }
            } else {
#pragma unroll
                for (int yy = 0; yy < N2; ++yy)
                    if ((ymask >> yy) & 1u) dst[__popc(ymask & ((1u << yy) - 1u)) * nz] = v[yy];
            }
        }
    }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// pairs per stage of the x read-out (one stage is PB * N1 * nyz complex values)
template <typename C>
struct PairX { static constexpr int PB = sizeof(C) == 8 ? 2 : 1; };
#define PX_THREADS 256

// persistent: each CTA takes chunks of PB pairs (chunk c, c + gridDim.x, ...); the next chunk's
// slab is copied while the current one is summed
template <typename C, typename CO>
__global__ void __launch_bounds__(PX_THREADS) k_pair_x(const C* __restrict__ T2, long long npair, int N1, int nyz,
                                                       int nz, const C* __restrict__ Ex, int nx,
                                                       const int* __restrict__ gpos, int ng,
                                                       typename Cx<C>::R scale, CO* __restrict__ M, long long ldm,
                                                       long long col0) {
    using R = typename Cx<C>::R;
    constexpr int PB = PairX<C>::PB;
    extern __shared__ __align__(16) unsigned char sm_x[];
    const size_t per = (size_t)N1 * nyz;
    C* slab = reinterpret_cast<C*>(sm_x);         // [2][PB][N1][nyz]
    C* ex = slab + 2 * PB * per;                  // [nx][N1]
    C* out = ex + nx * N1;                        // [ng][PB]
    for (int e = threadIdx.x; e < nx * N1; e += PX_THREADS) ex[e] = Ex[e];
    const long long nchunk = (npair + PB - 1) / PB;
    auto issue = [&](long long c, int b) {
        const long long p0 = c * PB;
        const size_t nbytes = (size_t)min((long long)PB, npair - p0) * per * sizeof(C);   // multiple of 16
        const char* src = reinterpret_cast<const char*>(T2 + (size_t)p0 * per);
        char* dst = reinterpret_cast<char*>(slab + (size_t)b * PB * per);
        for (size_t off = (size_t)threadIdx.x * 16; off < nbytes; off += PX_THREADS * 16) cp_async16(dst + off, src + off);
        cp_async_commit();
    };
    long long c = blockIdx.x;
    if (c < nchunk) issue(c, 0);
    for (int b = 0; c < nchunk; c += gridDim.x, b ^= 1) {
        if (c + gridDim.x < nchunk) issue(c + gridDim.x, b ^ 1);
        else cp_async_commit();                   // an empty group keeps the count uniform
        cp_async_wait<1>();                       // the current chunk's group has landed
        __syncthreads();
        const long long p0 = c * PB;
        const int np = (int)min((long long)PB, npair - p0);
        const C* t = slab + (size_t)b * PB * per;
        for (int g = threadIdx.x; g < ng; g += PX_THREADS) {
            const int gx = gpos[3 * g], gyz = gpos[3 * g + 1] * nz + gpos[3 * g + 2];
            const C* w = ex + gx * N1;
            R re[PB], im[PB];
#pragma unroll
            for (int j = 0; j < PB; ++j) re[j] = im[j] = 0;
#pragma unroll 8
            for (int xx = 0; xx < N1; ++xx) {
                const C cw = w[xx];
#pragma unroll
                for (int j = 0; j < PB; ++j) {
                    const C v = t[j * per + xx * nyz + gyz];
                    re[j] += cw.x * v.x - cw.y * v.y;
                    im[j] += cw.x * v.y + cw.y * v.x;
                }
            }
#pragma unroll
            for (int j = 0; j < PB; ++j) out[g * PB + j] = Cx<C>::mk(re[j] * scale, im[j] * scale);
        }
        __syncthreads();                          // slab b and out are free after this
        for (int e = threadIdx.x; e < ng * np; e += PX_THREADS) {
            const int g = e / np, j = e % np;
            const C v = out[g * PB + j];
            M[(size_t)g * ldm + col0 + p0 + j] = CT<CO>::make((typename CT<CO>::R)v.x, (typename CT<CO>::R)v.y);
        }
    }
    cp_async_wait<0>();
}

// x read-out for the windowed T2 (FP32 lines, half-width W on all three axes): one thread per
// (pair, yz point of the window; a window of more than 256 points is taken 256 points at a time)
// loads the point's N1 values along x (consecutive threads on consecutive points, so each x plane
// is read coalesced), transforms them in registers (the same +i line transform as z and y) and
// parks the outputs that lie on the sphere (colg) in shared memory; then the block writes its PB
// pairs as M[g][col0 + pair], PB consecutive columns per row.
template <int W>
struct PairXW {
    static constexpr int NW = 2 * W + 1, NC = NW * NW;
    static constexpr int TPP = NC >= 256 ? 256 : (NC + 31) / 32 * 32;   // threads per pair
    static constexpr int PB = 256 / TPP;                                // pairs per block
    static constexpr int THREADS = PB * TPP;
};

template <int N, int W, typename CO>
__global__ void __launch_bounds__(PairXW<W>::THREADS) k_pair_x_w(const float2* __restrict__ T2, long long npair,
                                                                const int* __restrict__ colg, int ng, float scale,
                                                                CO* __restrict__ M, long long ldm, long long col0) {
    using X = PairXW<W>;
    static_assert(2 * W + 1 <= N, "window wider than the axis");
    extern __shared__ __align__(16) unsigned char sm_xw[];
    float2* xo = reinterpret_cast<float2*>(sm_xw);            // [ng][PB]
    const int j = threadIdx.x / X::TPP, c = threadIdx.x % X::TPP;
    const long long p0 = (long long)blockIdx.x * X::PB, p = p0 + j;
    for (int cl = c; p < npair && cl < X::NC; cl += X::TPP) {
        float2 v[N];
        const float2* src = T2 + (size_t)p * N * X::NC + cl;
#pragma unroll
        for (int x = 0; x < N; ++x) v[x] = __ldg(src + (size_t)x * X::NC);
        LineFFT<float2, N>::run(v);
#pragma unroll
        for (int r = 0; r < N; ++r) {
            const int gx = r <= N / 2 ? r : r - N;                 // signed value of residue r
            if (gx >= -W && gx <= W) {
                const int g = __ldg(colg + (gx + W) * X::NC + cl);
                if (g >= 0) xo[g * X::PB + j] = make_float2(v[r].x * scale, v[r].y * scale);
            }
        }
    }
    __syncthreads();
    const int np = (int)min((long long)X::PB, npair - p0);
    for (int e = threadIdx.x; e < ng * np; e += X::THREADS) {
        const int g = e / np, jj = e % np;
        const float2 v = xo[g * X::PB + jj];
        M[(size_t)g * ldm + col0 + p0 + jj] = CT<CO>::make((typename CT<CO>::R)v.x, (typename CT<CO>::R)v.y);
    }
}

template <int N, int W, typename CO>
static bool launch_x_w_n(const float2* T2, long long npair, const int* colg, int ng, float scale, CO* M, long long ldm,
                         long long col0, cudaStream_t st) {
    using X = PairXW<W>;
    const size_t smem = (size_t)ng * X::PB * sizeof(float2);
    if (smem > 200 * 1024) return false;
    if (cudaFuncSetAttribute(k_pair_x_w<N, W, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return false;
    const long long nblk = (npair + X::PB - 1) / X::PB;
    k_pair_x_w<N, W, CO><<<(unsigned)nblk, X::THREADS, smem, st>>>(T2, npair, colg, ng, scale, M, ldm, col0);
    return true;
}

template <typename C, int N, int W>
static bool launch_zy_n(const C* u, int nkb, int nband, int nocc, int e0, int nemp, int N1, unsigned zmask, int nz,
                        unsigned ymask, int ny, C* T2, cudaStream_t st) {
    constexpr int A = ZyLayout<C, N>::A;
    if (W > 0) nz = ny = 2 * W + 1;
    const size_t smem = ZyLayout<C, N>::smem(nz);
    if (smem > 200 * 1024) return false;
    if (cudaFuncSetAttribute(k_pair_zy<C, N, N, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return false;
    dim3 grid(N1, (nemp + A - 1) / A, nkb);
    k_pair_zy<C, N, N, W><<<grid, 128, smem, st>>>(u, nband, nocc, e0, nemp, N1, zmask, nz, ymask, ny, T2);
    return true;
}

// half-widths of the symmetric residue windows the FP32 plane kernel is built for, per plane
// length 16, 24, 32, 48 (ascending; the plan takes the narrowest that holds the sphere)
static constexpr int kZyWin[4][5] = {{2, 3, 4, 5, 7}, {3, 5, 6, 7, 11}, {5, 7, 8, 11, 15}, {7, 9, 11, 15, 23}};
template <int N>
static constexpr int zy_row() { return N == 16 ? 0 : N == 24 ? 1 : N == 32 ? 2 : 3; }

int zy_window(int n, int m) {
    const int i = n == 16 ? 0 : n == 24 ? 1 : n == 32 ? 2 : n == 48 ? 3 : -1;
    if (i < 0) return 0;
    for (int w : kZyWin[i])
        if (w >= m) return w;
    return 0;
}

template <int N>
static bool launch_zy_win(int w, const float2* u, int nkb, int nband, int nocc, int e0, int nemp, int N1, float2* T2,
                          cudaStream_t st) {
    constexpr int i = zy_row<N>();
    if (w == kZyWin[i][0]) return launch_zy_n<float2, N, kZyWin[i][0]>(u, nkb, nband, nocc, e0, nemp, N1, 0, 0, 0, 0, T2, st);
    if (w == kZyWin[i][1]) return launch_zy_n<float2, N, kZyWin[i][1]>(u, nkb, nband, nocc, e0, nemp, N1, 0, 0, 0, 0, T2, st);
    if (w == kZyWin[i][2]) return launch_zy_n<float2, N, kZyWin[i][2]>(u, nkb, nband, nocc, e0, nemp, N1, 0, 0, 0, 0, T2, st);
    if (w == kZyWin[i][3]) return launch_zy_n<float2, N, kZyWin[i][3]>(u, nkb, nband, nocc, e0, nemp, N1, 0, 0, 0, 0, T2, st);
    if (w == kZyWin[i][4]) return launch_zy_n<float2, N, kZyWin[i][4]>(u, nkb, nband, nocc, e0, nemp, N1, 0, 0, 0, 0, T2, st);
    return false;
}

template <int N, typename CO>
static bool launch_x_win_n(int w, const float2* T2, long long npair, const int* colg, int ng, float scale, CO* M,
                           long long ldm, long long col0, cudaStream_t st) {
    constexpr int i = zy_row<N>();
    if (w == kZyWin[i][0]) return launch_x_w_n<N, kZyWin[i][0], CO>(T2, npair, colg, ng, scale, M, ldm, col0, st);
    if (w == kZyWin[i][1]) return launch_x_w_n<N, kZyWin[i][1], CO>(T2, npair, colg, ng, scale, M, ldm, col0, st);
    if (w == kZyWin[i][2]) return launch_x_w_n<N, kZyWin[i][2], CO>(T2, npair, colg, ng, scale, M, ldm, col0, st);
    if (w == kZyWin[i][3]) return launch_x_w_n<N, kZyWin[i][3], CO>(T2, npair, colg, ng, scale, M, ldm, col0, st);
    if (w == kZyWin[i][4]) return launch_x_w_n<N, kZyWin[i][4], CO>(T2, npair, colg, ng, scale, M, ldm, col0, st);
    return false;
}

// x read-out of the windowed T2 by line transforms (built for every window; false only when a
// launch attribute is refused, and the caller then uses k_pair_x on the same layout)
template <typename CO>
static bool launch_x_win(int n, int w, const float2* T2, long long npair, const int* colg, int ng, float scale,
                         CO* M, long long ldm, long long col0, cudaStream_t st) {
    switch (n) {
        case 16: return launch_x_win_n<16, CO>(w, T2, npair, colg, ng, scale, M, ldm, col0, st);
        case 24: return launch_x_win_n<24, CO>(w, T2, npair, colg, ng, scale, M, ldm, col0, st);
        case 32: return launch_x_win_n<32, CO>(w, T2, npair, colg, ng, scale, M, ldm, col0, st);
        case 48: return launch_x_win_n<48, CO>(w, T2, npair, colg, ng, scale, M, ldm, col0, st);
        default: return false;
    }
}

// plane-wise path for square planes N2 == N3 of a supported length: the residue masks, or (FP32
// lines, w > 0) the symmetric window of half-width w
// (empty bands e0 .. e0 + nemp - 1 of each k; the masks are 32-bit, so the residue-set form stops at 32)
template <typename C>
static bool launch_zy(int n2, int n3, int w, const C* u, int nkb, int nband, int nocc, int e0, int nemp, int N1,
                      unsigned zmask, int nz, unsigned ymask, int ny, C* T2, cudaStream_t st) {
    if (n2 != n3) return false;
    if constexpr (sizeof(C) == 8) {
        if (w > 0) {
            switch (n3) {
                case 16: return launch_zy_win<16>(w, u, nkb, nband, nocc, e0, nemp, N1, T2, st);
                case 24: return launch_zy_win<24>(w, u, nkb, nband, nocc, e0, nemp, N1, T2, st);
                case 32: return launch_zy_win<32>(w, u, nkb, nband, nocc, e0, nemp, N1, T2, st);
                case 48: return launch_zy_win<48>(w, u, nkb, nband, nocc, e0, nemp, N1, T2, st);
                default: return false;
            }
        }
    } else {
        if (w > 0) return false;
    }
    switch (n3) {
        case 16: return launch_zy_n<C, 16, 0>(u, nkb, nband, nocc, e0, nemp, N1, zmask, nz, ymask, ny, T2, st);
        case 24: return launch_zy_n<C, 24, 0>(u, nkb, nband, nocc, e0, nemp, N1, zmask, nz, ymask, ny, T2, st);
        case 32: return launch_zy_n<C, 32, 0>(u, nkb, nband, nocc, e0, nemp, N1, zmask, nz, ymask, ny, T2, st);
        default: return false;
    }
}

template <typename C, int N3>
static void launch_z(const C* u, int nkb, int nband, int nocc, int a0, int nab, int nlines, const int* zmap, int nz,
                     C* T1, cudaStream_t st) {
    dim3 grid((nlines + 31) / 32, nkb * nab);
    const size_t smem = (size_t)5 * 32 * (N3 + 1) * sizeof(C);
    cudaFuncSetAttribute(k_pair_z<C, N3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_pair_z<C, N3><<<grid, 128, smem, st>>>(u, nband, nocc, a0, nab, nlines, zmap, nz, T1);
}

template <typename C, int N2, typename CO>
static void launch_yx(const C* T1, int npair, int N1, int nz, const int* ymap, int ny, const C* Ex,
                      const int* gpos, int ng, typename Cx<C>::R scale, CO* M, long long ldm, long long col0,
                      cudaStream_t st) {
    constexpr int PPC = sizeof(C) == 8 ? 4 : 2;
    const size_t smem = (size_t)PPC * N1 * ny * nz * sizeof(C);
    cudaFuncSetAttribute(k_pair_yx<C, N2, PPC, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_pair_yx<C, N2, PPC, CO><<<(npair + PPC - 1) / PPC, 256, smem, st>>>(T1, npair, N1, nz, ymap, ny, Ex, gpos,
                                                                         ng, scale, M, ldm, col0);
}

// dispatch on the compile-time line lengths this build instantiates; false if not available
template <typename C>
static bool fused_z(int n, const C* u, int nkb, int nband, int nocc, int a0, int nab, int nlines, const int* zmap,
                    int nz, C* T1, cudaStream_t st) {
    switch (n) {
        case 8: launch_z<C, 8>(u, nkb, nband, nocc, a0, nab, nlines, zmap, nz, T1, st); return true;
        case 12: launch_z<C, 12>(u, nkb, nband, nocc, a0, nab, nlines, zmap, nz, T1, st); return true;
        case 16: launch_z<C, 16>(u, nkb, nband, nocc, a0, nab, nlines, zmap, nz, T1, st); return true;
        case 24: launch_z<C, 24>(u, nkb, nband, nocc, a0, nab, nlines, zmap, nz, T1, st); return true;
        case 32: launch_z<C, 32>(u, nkb, nband, nocc, a0, nab, nlines, zmap, nz, T1, st); return true;
        case 48: launch_z<C, 48>(u, nkb, nband, nocc, a0, nab, nlines, zmap, nz, T1, st); return true;
        default: return false;
    }
}

template <typename C, typename CO>
static bool fused_yx(int n, const C* T1, int npair, int N1, int nz, const int* ymap, int ny,
                     const C* Ex, const int* gpos, int ng, typename Cx<C>::R scale, CO* M, long long ldm,
                     long long col0, cudaStream_t st) {
    constexpr int PPC = sizeof(C) == 8 ? 4 : 2;
    if ((size_t)PPC * N1 * ny * nz * sizeof(C) > 200 * 1024) return false;
    switch (n) {
        case 8: launch_yx<C, 8, CO>(T1, npair, N1, nz, ymap, ny, Ex, gpos, ng, scale, M, ldm, col0, st); return true;
        case 12: launch_yx<C, 12, CO>(T1, npair, N1, nz, ymap, ny, Ex, gpos, ng, scale, M, ldm, col0, st); return true;
        case 16: launch_yx<C, 16, CO>(T1, npair, N1, nz, ymap, ny, Ex, gpos, ng, scale, M, ldm, col0, st); return true;
        case 24: launch_yx<C, 24, CO>(T1, npair, N1, nz, ymap, ny, Ex, gpos, ng, scale, M, ldm, col0, st); return true;
        case 32: launch_yx<C, 32, CO>(T1, npair, N1, nz, ymap, ny, Ex, gpos, ng, scale, M, ldm, col0, st); return true;
        case 48: launch_yx<C, 48, CO>(T1, npair, N1, nz, ymap, ny, Ex, gpos, ng, scale, M, ldm, col0, st); return true;
        default: return false;
    }
}


template <typename C, int N>
static bool gather_fft_n(rp_ctx* c, int k0, long long nbands, cudaStream_t st) {
    const int B = 2 * c->lb + 1;
    const size_t smem = sizeof(C) * ((size_t)N * B * B + (size_t)256 * B);
    if (B > N || smem > 227 * 1024) return false;      // the opt-in maximum per CTA
    if (ensure(c, c->s_u, (size_t)nbands * c->plan.nr * sizeof(C))) return false;
    if (cudaFuncSetAttribute(k_gather_fft<C, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return false;
    k_gather_fft<C, N><<<(unsigned)nbands, 256, smem, st>>>(
        (const double2*)c->d_coef.p, (const int*)c->d_miller.p, (const int*)c->d_npw.p, c->npw_max, c->nband, c->nocc,
        (const int*)c->plan.d_kp.p, (const int*)c->plan.d_g0.p, k0, c->lb, (C*)c->s_u.p);
    return true;
}

template <typename C>
static cudaError_t gather_inverse_t(rp_ctx* c, int k0, int nkb, const C* const einv[3],
                                    cudaStream_t st) {
    const int B = 2 * c->lb + 1;
    const int N1 = c->plan.nfft[0], N2 = c->plan.nfft[1], N3 = c->plan.nfft[2];
    const long long nbands = (long long)nkb * c->nband;
    // line-FFT path on cubic grids of a supported length
    if (N1 == N2 && N2 == N3) {
        bool done = false;
        if (N1 == 16) done = gather_fft_n<C, 16>(c, k0, nbands, st);
        else if (N1 == 24) done = gather_fft_n<C, 24>(c, k0, nbands, st);
        else if (N1 == 32) done = gather_fft_n<C, 32>(c, k0, nbands, st);
        if (done) return cudaGetLastError();
    }
    {   // one CTA per band with the Miller box in shared memory
        const size_t smem = sizeof(C) * ((size_t)B * B * B + (size_t)B * B + (size_t)N2 * B);
        if (smem <= 200 * 1024) {
            if (ensure(c, c->s_u, (size_t)nbands * c->plan.nr * sizeof(C))) return cudaErrorMemoryAllocation;
            cudaError_t e = cudaFuncSetAttribute(k_gather_grid<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            k_gather_grid<C><<<(unsigned)nbands, 256, smem, st>>>(
                (const double2*)c->d_coef.p, (const int*)c->d_miller.p, (const int*)c->d_npw.p, c->npw_max, c->nband,
                c->nocc, (const int*)c->plan.d_kp.p, (const int*)c->plan.d_g0.p, k0, c->lb, N1, N2, N3, einv[0], einv[1],
                einv[2], (C*)c->s_u.p);
            return cudaGetLastError();
        }
    }
    const size_t box = (size_t)nbands * B * B * B, u1 = (size_t)nbands * N1 * B * B,
                 u2 = (size_t)nbands * N1 * N2 * B, uu = (size_t)nbands * c->plan.nr;
    if (ensure(c, c->s_box, box * sizeof(C)) || ensure(c, c->s_u1, u1 * sizeof(C)) ||
        ensure(c, c->s_u2, u2 * sizeof(C)) || ensure(c, c->s_u, uu * sizeof(C)))
        return cudaErrorMemoryAllocation;
    C* dbox = (C*)c->s_box.p;
    cudaError_t e = cudaMemsetAsync(dbox, 0, box * sizeof(C), st);
    if (e != cudaSuccess) return e;
    const int bs = 256;
    long long n = (long long)nkb * c->nband * c->npw_max;
    k_scatter_box<C><<<grid_for(n, bs), bs, 0, st>>>((const double2*)c->d_coef.p, (const int*)c->d_miller.p,
                                                     (const int*)c->d_npw.p, c->npw_max, c->nband, c->nocc,
                                                     (const int*)c->plan.d_kp.p, (const int*)c->plan.d_g0.p, k0,
                                                     nkb, c->lb, dbox);
    // m1 -> x
    n = nbands * N1 * (long long)B * B;
    k_axis_pass<C><<<grid_for(n, bs), bs, 0, st>>>(dbox, (C*)c->s_u1.p, einv[0], nbands, B, N1, B * B,
                                                   (long long)B * B * B, (long long)B * B, (long long)N1 * B * B,
                                                   (long long)B * B);
    // m2 -> y
    n = nbands * N1 * (long long)N2 * B;
    k_axis_pass<C><<<grid_for(n, bs), bs, 0, st>>>((const C*)c->s_u1.p, (C*)c->s_u2.p, einv[1], nbands * N1, B, N2, B,
                                                   (long long)B * B, (long long)B, (long long)N2 * B, (long long)B);
    // m3 -> z
    n = nbands * N1 * (long long)N2 * N3;
    k_axis_pass<C><<<grid_for(n, bs), bs, 0, st>>>((const C*)c->s_u2.p, (C*)c->s_u.p, einv[2], nbands * N1 * N2, B, N3,
                                                   1, (long long)B, 1LL, (long long)N3, 1LL);
    return cudaGetLastError();
}

template <typename C, typename CO>
static cudaError_t pair_forward_t(rp_ctx* c, int nkb, CO* M, long long ldm, long long col0, const C* const efwd[3],
                                  cudaStream_t st, int* nlaunch) {
    const QPlan& P = c->plan;
    const int N1 = c->plan.nfft[0], N2 = c->plan.nfft[1], N3 = c->plan.nfft[2];
    const int ny = P.nset[1], nz = P.nset[2];
    const long long nr = c->plan.nr;
    const int bs = 256;
    // plane-wise path: z and y transforms on chip, then the x sum on the sphere points; FP32 lines
    // use the symmetric residue window when the plan found one
    {
        const int w = sizeof(C) == 8 ? P.zyw : 0;
        const int wy = w > 0 ? 2 * w + 1 : ny, wz = w > 0 ? 2 * w + 1 : nz;
        const size_t per_pair = (size_t)N1 * wy * wz * sizeof(C);
        const size_t budget = c->pair_budget;
        // empty bands per pass: all of them when the k block's plane sums fit the budget, else (a
        // single k point, whose pairs are columns (a, o) in order) chunks of empty bands
        int ne = c->nemp;
        if ((size_t)nkb * c->nemp * c->nocc * per_pair > budget)
            ne = nkb == 1 ? (int)std::min<size_t>((size_t)c->nemp,
                                                  std::max<size_t>(1, budget / ((size_t)c->nocc * per_pair)))
                          : 0;
        constexpr int PB = PairX<C>::PB;
        // shared memory of the x read-out that will run: k_pair_x_w holds only its pairs' outputs
        // (PB pairs per block for the window of half-width w, as PairXW<w>)
        auto xw_pb = [](int hw) {
            const int nc = (2 * hw + 1) * (2 * hw + 1);
            return 256 / (nc >= 256 ? 256 : (nc + 31) / 32 * 32);
        };
        const size_t xsm = w > 0 ? (size_t)P.ng * xw_pb(w) * sizeof(C)
                                          : ((size_t)2 * PB * N1 * wy * wz + (size_t)P.nset[0] * N1 +
                                             (size_t)P.ng * PB) * sizeof(C);
        // the x sum of npair pairs of T2 into columns col .. col + npair - 1
        auto x_readout = [&](long long npair, long long col) -> cudaError_t {
            if constexpr (sizeof(C) == 8) {
                if (w > 0 && launch_x_win<CO>(N1, w, (const float2*)c->s_t2.p, npair, (const int*)P.d_colg.p, P.ng,
                                              (float)(1.0 / (double)nr), M, ldm, col, st))
                    return cudaGetLastError();
            }
            cudaError_t e = cudaFuncSetAttribute(k_pair_x<C, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm);
            if (e != cudaSuccess) return e;
            const long long nchunk = (npair + PB - 1) / PB;
            // as many CTAs per SM as fit: each keeps its own chunk in flight
            int per_sm = 1;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair_x<C, CO>, PX_THREADS, xsm) != cudaSuccess ||
                per_sm < 1) {
                cudaGetLastError();
                per_sm = 1;
            }
            const unsigned grid = (unsigned)std::min<long long>(nchunk, (long long)per_sm * c->num_sms);
            k_pair_x<C, CO><<<grid, PX_THREADS, xsm, st>>>(
                (const C*)c->s_t2.p, npair, N1, wy * wz, wz, efwd[0], P.nset[0],
                (const int*)(w > 0 ? P.d_gpos_w.p : P.d_gpos_r.p), P.ng,
                (typename CT<C>::R)(1.0 / (double)nr), M, ldm, col);
            return cudaGetLastError();
        };
        if (ne > 0 && P.fused && (w > 0 || P.masks) && xsm <= 200 * 1024 &&
            ensure(c, c->s_t2, (size_t)nkb * ne * c->nocc * per_pair) == RP_OK) {
            for (int e0 = 0; e0 < c->nemp; e0 += ne) {
                const int nab = std::min(ne, c->nemp - e0);
                if (!launch_zy<C>(N2, N3, w, (const C*)c->s_u.p, nkb, c->nband, c->nocc, e0, nab, N1, P.zmask, nz,
                                  P.ymask, ny, (C*)c->s_t2.p, st)) {
                    if (e0 == 0) break;             // not built or refused: the paths below
                    return cudaErrorLaunchFailure;  // (the same launch as the first chunk's)
                }
                cudaError_t e = x_readout((long long)nkb * nab * c->nocc, col0 + (long long)e0 * c->nocc);
                if (e != cudaSuccess) return e;
                *nlaunch += 2;
                if (e0 + nab >= c->nemp) return cudaGetLastError();
            }
        }
    }
    // fused path over the whole k block when its partial transforms fit the scratch budget
    {
        const long long npair = (long long)nkb * c->nemp * c->nocc;
        const size_t t1 = (size_t)npair * N1 * N2 * nz * sizeof(C);
        if (P.fused && t1 <= (size_t)12 << 30 && ensure(c, c->s_t1, t1) == RP_OK &&
            fused_z<C>(N3, (const C*)c->s_u.p, nkb, c->nband, c->nocc, 0, c->nemp, N1 * N2, (const int*)P.d_zmap.p,
                       nz, (C*)c->s_t1.p, st)) {
            if (fused_yx<C, CO>(N2, (const C*)c->s_t1.p, (int)npair, N1, nz, (const int*)P.d_ymap.p, ny, efwd[0],
                                (const int*)P.d_gpos.p, P.ng, (typename CT<C>::R)(1.0 / (double)nr), M, ldm, col0,
                                st)) {
                *nlaunch += 2;
                return cudaGetLastError();
            }
            if (ensure(c, c->s_t2, (size_t)npair * N1 * ny * nz * sizeof(C))) return cudaErrorMemoryAllocation;
            long long n = npair * N1 * ny * nz;
            k_axis_pass<C><<<grid_for(n, bs), bs, 0, st>>>((const C*)c->s_t1.p, (C*)c->s_t2.p, efwd[1], npair * N1, N2,
                                                           ny, nz, (long long)N2 * nz, (long long)nz, (long long)ny * nz,
                                                           (long long)nz);
            n = (long long)P.ng * npair;
            k_sphere_readout<C, CO><<<grid_for(n, bs), bs, 0, st>>>((const C*)c->s_t2.p, efwd[0], (const int*)P.d_gpos.p,
                                                                    P.ng, (int)npair, N1, ny, nz,
                                                                    (typename CT<C>::R)(1.0 / (double)nr), M, ldm, col0);
            *nlaunch += 3;
            return cudaGetLastError();
        }
    }
    // empty bands per sub-block: keep the product scratch near 256 MB
    const long long per = (long long)c->nocc * nr * (long long)sizeof(C);
    int na = (int)std::max(1LL, std::min((long long)c->nemp, (256LL << 20) / per));
    const size_t pbytes = (size_t)na * c->nocc * nr * sizeof(C);
    const size_t t1 = (size_t)na * c->nocc * N1 * N2 * nz * sizeof(C);
    const size_t t2 = (size_t)na * c->nocc * N1 * ny * nz * sizeof(C);
    if (ensure(c, c->s_p, pbytes) || ensure(c, c->s_t1, t1) || ensure(c, c->s_t2, t2)) return cudaErrorMemoryAllocation;
    for (int kl = 0; kl < nkb; ++kl) {
        const C* u = (const C*)c->s_u.p + (size_t)kl * c->nband * nr;
        for (int a0 = 0; a0 < c->nemp; a0 += na) {
            int nab = std::min(na, c->nemp - a0);
            long long npair = (long long)nab * c->nocc;
            long long n = npair * nr;
            k_pair_product<C><<<grid_for(n, bs), bs, 0, st>>>(u, nr, c->nocc, a0, nab, (C*)c->s_p.p);
            // z -> gz (innermost axis)
            n = npair * N1 * N2 * nz;
            k_axis_pass<C><<<grid_for(n, bs), bs, 0, st>>>((const C*)c->s_p.p, (C*)c->s_t1.p, efwd[2], npair * N1 * N2,
                                                           N3, nz, 1, (long long)N3, 1LL, (long long)nz, 1LL);
            // y -> gy
            n = npair * N1 * ny * nz;
            k_axis_pass<C><<<grid_for(n, bs), bs, 0, st>>>((const C*)c->s_t1.p, (C*)c->s_t2.p, efwd[1], npair * N1, N2,
                                                           ny, nz, (long long)N2 * nz, (long long)nz, (long long)ny * nz,
                                                           (long long)nz);
            // x -> gx on the sphere points
            n = (long long)P.ng * npair;
            long long col = col0 + (long long)kl * c->nemp * c->nocc + (long long)a0 * c->nocc;
            k_sphere_readout<C, CO><<<grid_for(n, bs), bs, 0, st>>>((const C*)c->s_t2.p, efwd[0],
                                                                    (const int*)P.d_gpos.p, P.ng, (int)npair, N1, ny,
                                                                    nz, (typename CT<C>::R)(1.0 / (double)nr), M, ldm,
                                                                    col);
            *nlaunch += 4;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_gather_inverse(rp_ctx* c, int k0, int nkb, bool fp32, cudaStream_t st) {
    if (fp32) {
        const float2* e[3] = {(const float2*)c->plan.d_einv32[0].p, (const float2*)c->plan.d_einv32[1].p,
                              (const float2*)c->plan.d_einv32[2].p};
        return gather_inverse_t<float2>(c, k0, nkb, e, st);
    }
    const double2* e[3] = {(const double2*)c->plan.d_einv[0].p, (const double2*)c->plan.d_einv[1].p,
                           (const double2*)c->plan.d_einv[2].p};
    return gather_inverse_t<double2>(c, k0, nkb, e, st);
}

cudaError_t launch_pair_forward(rp_ctx* c, int nkb, double2* M, long long ldm, long long col0, cudaStream_t st,
                                int* nlaunch) {
    const QPlan& P = c->plan;
    const double2* e[3] = {(const double2*)P.d_efwd[0].p, (const double2*)P.d_efwd[1].p,
                           (const double2*)P.d_efwd[2].p};
    return pair_forward_t<double2, double2>(c, nkb, M, ldm, col0, e, st, nlaunch);
}

cudaError_t launch_pair_forward32(rp_ctx* c, int nkb, float2* M, long long ldm, long long col0, cudaStream_t st,
                                  int* nlaunch) {
    const QPlan& P = c->plan;
    const float2* e[3] = {(const float2*)P.d_efwd32[0].p, (const float2*)P.d_efwd32[1].p,
                          (const float2*)P.d_efwd32[2].p};
    return pair_forward_t<float2, float2>(c, nkb, M, ldm, col0, e, st, nlaunch);
}

}  // namespace rp
