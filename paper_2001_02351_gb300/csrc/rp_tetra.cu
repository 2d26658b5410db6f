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
// Precision: FP64 throughout for the FP64 tier; for the split-precision tiers FP32, with
// every node set that has a near degeneracy evaluated again in FP64.
#include <algorithm>

#include "rp_internal.h"

namespace rp {

#define TT_TAU 0.5
#define TT_KMAX 48
#define TT_FCH 4

template <typename R>
struct TT;
template <>
struct TT<double> {
    using C = double2;
    static __device__ __forceinline__ C mk(double a, double b) { return make_double2(a, b); }
    static __device__ __forceinline__ double hyp(double a, double b) { return hypot(a, b); }
    static __device__ __forceinline__ C clog(C a) { return make_double2(log(hypot(a.x, a.y)), atan2(a.y, a.x)); }
    static __device__ __forceinline__ double lg(double a) { return log(a); }
    static __device__ __forceinline__ double rsq(double a) { return rsqrt(a); }
};
template <>
struct TT<float> {
    using C = float2;
    static __device__ __forceinline__ C mk(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ float hyp(float a, float b) { return hypotf(a, b); }
    static __device__ __forceinline__ C clog(C a) { return make_float2(logf(hypotf(a.x, a.y)), atan2f(a.y, a.x)); }
    static __device__ __forceinline__ float lg(float a) { return logf(a); }
    static __device__ __forceinline__ float rsq(float a) { return rsqrtf(a); }
};

template <typename C>
__device__ __forceinline__ C tadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C>
__device__ __forceinline__ C tsub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C>
__device__ __forceinline__ C tmul(C a, C b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
template <typename C, typename R>
__device__ __forceinline__ C tscale(C a, R s) { return {a.x * s, a.y * s}; }
template <typename C>
__device__ __forceinline__ C tinv(C a) {
    const auto d = a.x * a.x + a.y * a.y;
    return {a.x / d, -a.y / d};
}

// f^(m)(c)/m! = (z-c)^(3-m) * b_m(log(z-c))  for f(x) = (z-x)^3 log(z-x)
template <typename R>
__device__ __forceinline__ typename TT<R>::C bcoef(int m, typename TT<R>::C L) {
    if (m >= 4) return TT<R>::mk((R)6 / ((R)m * (m - 1) * (m - 2) * (m - 3)), (R)0);
    if (m == 0) return L;
    if (m == 1) return TT<R>::mk(-((R)3 * L.x + (R)1), (R)-3 * L.y);
    if (m == 2) return TT<R>::mk(((R)6 * L.x + (R)5) * (R)0.5, (R)3 * L.y);
    return TT<R>::mk(-((R)6 * L.x + (R)11) / (R)6, -L.y);
}

// number of series terms for ratio rho = max|x - c| / |z - c| (rho <= TAU/2), by precision
template <typename R>
__device__ __forceinline__ int nterms(R rho) {
    if (rho <= (R)0) return 0;
    const R target = sizeof(R) == 8 ? (R)-39.2 : (R)-18.0;
    int k = (int)ceil(target / TT<R>::lg(rho)) + 6;
    return k > TT_KMAX ? TT_KMAX : k;
}

// Divided difference of order n over the m = n+1 centred nodes t (t = x - c) by the Taylor
// series about c:  y^(3-n) sum_k b_{n+k} h_k(t) y^-k,  y = z - c.  With r = |y| the sum is
// taken as sum_k b_{n+k} h_k(t/r) (conj(y)/r)^k, so every power stays on the unit circle.
// The complete homogeneous polynomials h_k come from the recurrence
// h_k = e1 h_{k-1} - e2 h_{k-2} + ... with the elementary symmetric polynomials e_j of the
// scaled nodes, so no array is needed.
template <typename R>
__device__ __forceinline__ typename TT<R>::C dd_series(const R (&t)[5], int m, typename TT<R>::C y, int K) {
    using C = typename TT<R>::C;
    const int n = m - 1;
    const R r = TT<R>::hyp(y.x, y.y);
    const R rinv = (R)1 / r;
    R e[6] = {1, 0, 0, 0, 0, 0};
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        if (v < m) {
            const R tv = t[v] * rinv;
#pragma unroll
            for (int j = 5; j >= 1; --j) e[j] += tv * e[j - 1];
        }
    }
    const C L = (n <= 3) ? TT<R>::clog(y) : TT<R>::mk(0, 0);
    const C u = TT<R>::mk(y.x * rinv, -y.y * rinv);     // conj(y)/r, |u| = 1
    R h1 = 0, h2 = 0, h3 = 0, h4 = 0;                    // h_{k-2} .. h_{k-5}
    R hk = 1;                                            // h_{k-1}
    C uk = TT<R>::mk(1, 0);
    C S = bcoef<R>(n, L);
    for (int k = 1; k <= K; ++k) {
        const R hn = e[1] * hk - e[2] * h1 + e[3] * h2 - e[4] * h3 + e[5] * h4;
        h4 = h3; h3 = h2; h2 = h1; h1 = hk; hk = hn;
        uk = tmul(uk, u);
        S = tadd(S, tscale(tmul(bcoef<R>(n + k, L), uk), hk));
    }
    // times y^(3-n)
    C p = TT<R>::mk(1, 0);
    if (n <= 3) {
        for (int q = 0; q < 3 - n; ++q) p = tmul(p, y);
    } else {
        const C w = tinv(y);
        for (int q = 0; q < n - 3; ++q) p = tmul(p, w);
    }
    return tmul(S, p);
}

// Fourth divided difference over the five nodes c + {-s/2, t1, t2, t3, s/2} by the Taylor series
// about the centre c:  y^-1 sum_k b_{4+k} h_k(t/r) u^k,  y = z - c, r = |y|, u = conj(y)/r,
// b_q = 6 / (q (q-1) (q-2) (q-3)).  With every scaled node within rho = s / (2 r) of zero,
// |h_k| <= C(k+4, 4) rho^k, so |b_{4+k} h_k u^k| <= rho^k / 4 while the sum is at least
// (1 - 2 rho) / (4 (1 - rho)): after K terms the remainder is below 2 rho^(K+1) of the sum for
// rho <= 1/4, and K is the smallest count that puts it under half the unit roundoff.
template <typename R>
__device__ __forceinline__ typename TT<R>::C dd5_series(R t1, R t2, R t3, R s, typename TT<R>::C y) {
    using C = typename TT<R>::C;
    constexpr int KM = sizeof(R) == 8 ? 28 : 13;            // K at rho = 1/4
    const R rinv = TT<R>::rsq(y.x * y.x + y.y * y.y);
    const R rho = (R)0.5 * s * rinv;
    int K = 0;
    if (rho > (R)0) {
        const R target = sizeof(R) == 8 ? (R)-38.5 : (R)-17.5;   // log of half the roundoff, with margin
        K = (int)ceil(target / TT<R>::lg(rho));
        K = K < KM ? K : KM;
    }
    const R nd[5] = {-rho, t1 * rinv, t2 * rinv, t3 * rinv, rho};
    R e1 = 0, e2 = 0, e3 = 0, e4 = 0, e5 = 0;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        e5 += nd[v] * e4;
        e4 += nd[v] * e3;
        e3 += nd[v] * e2;
        e2 += nd[v] * e1;
        e1 += nd[v];
    }
    const C u = TT<R>::mk(y.x * rinv, -y.y * rinv);
    R h1 = 0, h2 = 0, h3 = 0, h4 = 0, hk = 1;
    C uk = TT<R>::mk(1, 0);
    C S = TT<R>::mk((R)0.25, 0);
#pragma unroll
    for (int k = 1; k <= KM; ++k) {
        if (k > K) break;
        const R hn = e1 * hk - e2 * h1 + e3 * h2 - e4 * h3 + e5 * h4;
        h4 = h3; h3 = h2; h2 = h1; h1 = hk; hk = hn;
        uk = tmul(uk, u);
        const R bh = (R)(6.0 / ((double)(k + 4) * (k + 3) * (k + 2) * (k + 1))) * hk;
        S.x += bh * uk.x;
        S.y += bh * uk.y;
    }
    const C p = tmul(S, u);
    return TT<R>::mk(p.x * rinv, p.y * rinv);
}

// 6 / (m (m-1) (m-2) (m-3)) for m = 0 .. 63 (entries below 4 unused)
__constant__ double c_bq[64];

// Divided difference of order n = m - 1 over the sorted run x[i..j] (m nodes) by the Taylor
// series about its first node x_i, whose logarithm L = log(z - x_i) is known:
//   sum_q f^(q)(x_i)/q! h_{q-n}(x - x_i),  f^(q)(x_i)/q! = y^(3-q) b_q(L),  y = z - x_i.
// The sum runs over scaled nodes (x - x_i)/|y| and unit-modulus powers conj(y)/|y|.
template <typename R>
__device__ typename TT<R>::C dd_run_about_node(const R (&x)[5], int i, int j, typename TT<R>::C y,
                                               typename TT<R>::C L, R rho) {
    using C = typename TT<R>::C;
    const int n = j - i;
    const R r = TT<R>::hyp(y.x, y.y);
    const R rinv = (R)1 / r;
    R e[6] = {1, 0, 0, 0, 0, 0};
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        if (v > i && v <= j) {   // node x_i itself contributes a zero offset
            const R tv = (x[v] - x[i]) * rinv;
#pragma unroll
            for (int q = 5; q >= 1; --q) e[q] += tv * e[q - 1];
        }
    }
    const int K = nterms<R>(rho);
    const C u = TT<R>::mk(y.x * rinv, -y.y * rinv);
    R h1 = 0, h2 = 0, h3 = 0, h4 = 0, hk = 1;
    C uk = TT<R>::mk(1, 0);
    C S = bcoef<R>(n, L);
    for (int k = 1; k <= K; ++k) {
        const R hn = e[1] * hk - e[2] * h1 + e[3] * h2 - e[4] * h3 + e[5] * h4;
        h4 = h3; h3 = h2; h2 = h1; h1 = hk; hk = hn;
        uk = tmul(uk, u);
        const int q = n + k;
        const C b = q >= 4 ? TT<R>::mk((R)c_bq[q < 64 ? q : 63], 0) : bcoef<R>(q, L);
        S = tadd(S, tscale(tmul(b, uk), hk));
    }
    C p = TT<R>::mk(1, 0);
    if (n <= 3) {
        for (int q = 0; q < 3 - n; ++q) p = tmul(p, y);
    } else {
        const C w = tinv(y);
        for (int q = 0; q < n - 3; ++q) p = tmul(p, w);
    }
    return tmul(S, p);
}

#define TT_TAU_RUN 0.3

// full divided-difference table: recursion between well separated nodes, closed forms for
// coincident nodes, Taylor series about the run's first node for narrow runs (no logarithm
// beyond the five node logarithms).  *narrow is set when a narrow run of nonzero width occurs.
template <typename R>
__device__ typename TT<R>::C dd5_table(const R (&x)[5], typename TT<R>::C z, bool* narrow) {
    using C = typename TT<R>::C;
    C D[5][5], L[5], Y[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        Y[i] = TT<R>::mk(z.x - x[i], z.y);
        if (i > 0 && x[i] == x[i - 1]) {
            L[i] = L[i - 1];
        } else {
            L[i] = TT<R>::clog(Y[i]);
        }
        D[i][i] = tmul(tmul(tmul(Y[i], Y[i]), Y[i]), L[i]);
    }
#pragma unroll
    for (int n = 1; n < 5; ++n)
#pragma unroll
        for (int i = 0; i + n < 5; ++i) {
            const int j = i + n;
            const R s = x[j] - x[i];
            if (s == (R)0) {
                // confluent: f^(n)(x_i)/n!
                C p = TT<R>::mk(1, 0);
                if (n <= 3) {
                    for (int q = 0; q < 3 - n; ++q) p = tmul(p, Y[i]);
                } else {
                    const C w = tinv(Y[i]);
                    for (int q = 0; q < n - 3; ++q) p = tmul(p, w);
                }
                D[i][j] = tmul(bcoef<R>(n, L[i]), p);
                continue;
            }
            const R Ri = TT<R>::hyp(Y[i].x, Y[i].y);
            if (s <= (R)TT_TAU_RUN * Ri) {
                *narrow = true;
                D[i][j] = dd_run_about_node<R>(x, i, j, Y[i], L[i], s / Ri);
            } else {
                D[i][j] = tscale(tsub(D[i + 1][j], D[i][j - 1]), (R)1 / s);
            }
        }
    return D[0][4];
}

__device__ __forceinline__ void cswap(double& a, double& b) {
    const double lo = fmin(a, b), hi = fmax(a, b);
    a = lo;
    b = hi;
}

// nodes of tetrahedron-vertex entry `code` for pair (a, o): loaded, sorted, degenerate groups
// merged into their mean (Eq. tetrahedron thresholds), all in FP64
__device__ __forceinline__ void tetra_nodes(const double* __restrict__ E, int nband, int nocc, int a, int o,
                                            const int* __restrict__ kp, const int* __restrict__ tets, int code,
                                            double da, double dr, double (&x)[5]) {
    const int tt = code >> 2, jv = code & 3;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int kv = tets[4 * tt + v];
        x[v] = E[(size_t)kp[kv] * nband + nocc + a] - E[(size_t)kv * nband + o];
    }
    x[4] = jv == 0 ? x[0] : jv == 1 ? x[1] : jv == 2 ? x[2] : x[3];
    cswap(x[0], x[1]); cswap(x[3], x[4]); cswap(x[2], x[4]); cswap(x[2], x[3]); cswap(x[0], x[3]);
    cswap(x[0], x[2]); cswap(x[1], x[4]); cswap(x[1], x[3]); cswap(x[1], x[2]);
    bool brk[5];
    brk[0] = true;
    double start = x[0];
#pragma unroll
    for (int i = 1; i < 5; ++i) {
        const double thr = da + dr * fmax(fabs(start), fabs(x[i]));
        brk[i] = (x[i] - start) >= thr;
        if (brk[i]) start = x[i];
    }
    if (brk[1] && brk[2] && brk[3] && brk[4]) return;
    double y[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        double sum = 0.0;
        int cnt = 0;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            bool same = true;
#pragma unroll
            for (int b = 1; b < 5; ++b)
                if (b > (i < j ? i : j) && b <= (i < j ? j : i) && brk[b]) same = false;
            if (same) { sum += x[j]; ++cnt; }
        }
        y[i] = sum / cnt;
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) x[i] = y[i];
}

// one divided difference in FP64 from the nodes themselves (used for near-degenerate sets of
// the FP32 path)
__device__ __noinline__ double2 dd_fp64_entry(const double* __restrict__ E, int nband, int nocc, int a, int o,
                                              const int* __restrict__ kp, const int* __restrict__ tets, int code,
                                              double da, double dr, double2 z) {
    double x[5];
    tetra_nodes(E, nband, nocc, a, o, kp, tets, code, da, dr, x);
    const double c = 0.5 * (x[0] + x[4]);
    const double2 y = make_double2(z.x - c, z.y);
    const double spread = x[4] - x[0];
    if (spread * spread <= TT_TAU * TT_TAU * (y.x * y.x + y.y * y.y))
        return dd5_series<double>(x[1] - c, x[2] - c, x[3] - c, spread, y);
    bool unused = false;
    return dd5_table<double>(x, z, &unused);
}

template <typename R>
__device__ __noinline__ typename TT<R>::C dd_table_entry(const R (&x)[5], typename TT<R>::C z) {
    bool unused = false;
    return dd5_table<R>(x, z, &unused);
}

// nodes of entry `code` relative to the pair's transition energy d0, as the FP32 pass forms them:
// centre ct, offsets tr (outer nodes at -+ spread / 2)
__device__ __forceinline__ void fp32_nodes(const double (&x)[5], double d0, float& ct, float (&tr)[5]) {
    const double cd = 0.5 * (x[0] + x[4]);
    const float spread = (float)(x[4] - x[0]);
    tr[0] = -0.5f * spread;
    tr[1] = (float)(x[1] - cd);
    tr[2] = (float)(x[2] - cd);
    tr[3] = (float)(x[3] - cd);
    tr[4] = 0.5f * spread;
    ct = (float)(cd - d0);
}

// item of the deferred work list: pair t, frequency f, tetrahedron-vertex entry s, pole side,
// kind (0: near-degenerate set, evaluated in FP64; 1: wide set of the FP32 pass, full table in FP32)
__device__ __forceinline__ unsigned long long tetra_item(long long t, int f, int s, int side, int kind) {
    return ((unsigned long long)t << 32) | ((unsigned long long)f << 16) | ((unsigned long long)s << 8) |
           ((unsigned long long)kind << 1) | (unsigned long long)side;
}

// Append a (pair, frequency, tetrahedron-vertex, pole) item to the FP64 work list; when the list
// is full, evaluate it here instead (slower, same result).
template <typename C>
__device__ __forceinline__ void defer_or_eval(unsigned long long* queue, unsigned long long qcap,
                                              unsigned long long* qcount, long long t, int f, int s, int side,
                                              C& sacc, const double* __restrict__ E, int nband, int nocc, int a,
                                              int o, const int* __restrict__ kp, const int* __restrict__ tets,
                                              int code, double da, double dr, double2 zd) {
    const unsigned long long slot = atomicAdd(qcount, 1ULL);
    if (slot < qcap) {
        queue[slot] = tetra_item(t, f, s, side, 0);
        return;
    }
    const double2 r = dd_fp64_entry(E, nband, nocc, a, o, kp, tets, code, da, dr, zd);
    sacc.x += r.x;
    sacc.y += r.y;
}

// Pass over the deferred items: one item per thread, result added to the weight
__global__ void __launch_bounds__(128) k_tetra_fixup(const double* __restrict__ E, const double* __restrict__ Tw,
                                                     int nband, int nocc, int nemp, int nk,
                                                     const int* __restrict__ kp, const int* __restrict__ tets,
                                                     const int* __restrict__ tetk, const double* __restrict__ freq,
                                                     int axis, int ordering, double delta, double da, double dr,
                                                     const unsigned long long* __restrict__ queue,
                                                     const unsigned long long* __restrict__ qcount,
                                                     unsigned long long qcap, double2* __restrict__ wout) {
    const unsigned long long n = min(*qcount, qcap);
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long item = queue[i];
    const long long t = (long long)(item >> 32);
    const int f = (int)((item >> 16) & 0xFFFF), s = (int)((item >> 8) & 0xFF), side = (int)(item & 1);
    const int kind = (int)((item >> 1) & 1);
    const long long K = (long long)nk * nemp * nocc;
    const int o = (int)(t % nocc);
    const int a = (int)((t / nocc) % nemp);
    const int k = (int)(t / ((long long)nocc * nemp));
    double pref = 2.0 / (double)nk;
    if (Tw) pref *= 1.0 - Tw[(size_t)kp[k] * nband + nocc + a] * Tw[(size_t)k * nband + o];
    const double wv = freq[f];
    double2 zd;
    if (axis == RP_AXIS_REAL)
        zd = side == 0 ? make_double2(wv, delta) : make_double2(-wv, ordering == RP_TIME_ORDERED ? delta : -delta);
    else
        zd = side == 0 ? make_double2(0.0, wv + delta)
                       : make_double2(0.0, ordering == RP_TIME_ORDERED ? -wv + delta : -wv - delta);
    double2 r;
    if (kind == 0) {
        r = dd_fp64_entry(E, nband, nocc, a, o, kp, tets, tetk[24 * k + s], da, dr, zd);
    } else {
        double x[5];
        tetra_nodes(E, nband, nocc, a, o, kp, tets, tetk[24 * k + s], da, dr, x);
        const double d0 = E[(size_t)kp[k] * nband + nocc + a] - E[(size_t)k * nband + o];
        float ct, tr[5], xr[5];
        fp32_nodes(x, d0, ct, tr);
#pragma unroll
        for (int j = 0; j < 5; ++j) xr[j] = ct + tr[j];
        const float2 rf = dd_table_entry<float>(xr, make_float2((float)(zd.x - d0), (float)zd.y));
        r = make_double2((double)rf.x, (double)rf.y);
    }
    double* dst = reinterpret_cast<double*>(wout + (size_t)f * K + t);
    atomicAdd(dst, r.x * pref / 6.0);
    atomicAdd(dst + 1, r.y * pref / 6.0);
    }
}

// Weights for one (k, a, o) per thread and a chunk of frequencies per grid row.  The 24
// tetrahedron-vertex node sets are prepared once in FP64 (sort, merge, centre) and kept in
// shared memory; every frequency is then evaluated from them in precision R.  Nodes and poles
// are taken relative to the pair's own transition energy D0 so that R = float keeps its
// resolution.  With R = float every node set is evaluated in FP32 except those with two nodes
// closer than TT_NEAR but not merged (near degeneracy), which go to an FP64 pass.
#define TT_NEAR 1e-5
#define TT_FIELDS 5   // t1, t2, t3, centre - D0, spread (negative: near-degenerate set)

template <typename R>
__global__ void __launch_bounds__(128) k_tetra_weights(const double* __restrict__ E, const double* __restrict__ Tw,
                                                       int nband, int nocc, int nemp, int nk,
                                                       const int* __restrict__ kp, const int* __restrict__ tets,
                                                       const int* __restrict__ tetk, int nf, int fch,
                                                       const double* __restrict__ freq, int axis, int ordering,
                                                       double delta, double da, double dr,
                                                       double2* __restrict__ wout,
                                                       unsigned long long* __restrict__ queue,
                                                       unsigned long long qcap, unsigned long long* qcount) {
    using C = typename TT<R>::C;
    extern __shared__ __align__(16) unsigned char tsm_raw[];
    R* tsm = reinterpret_cast<R*>(tsm_raw);
    const int bd = blockDim.x, tid = threadIdx.x;
    auto fld = [&](int s, int f) -> R& { return tsm[(s * TT_FIELDS + f) * bd + tid]; };
    const long long t = (long long)blockIdx.x * bd + tid;
    const long long K = (long long)nk * nemp * nocc;
    if (t >= K) return;
    const int o = (int)(t % nocc);
    const int a = (int)((t / nocc) % nemp);
    const int k = (int)(t / ((long long)nocc * nemp));
    double pref = 2.0 / (double)nk;
    if (Tw) pref *= 1.0 - Tw[(size_t)kp[k] * nband + nocc + a] * Tw[(size_t)k * nband + o];
    const double d0 = E[(size_t)kp[k] * nband + nocc + a] - E[(size_t)k * nband + o];
    for (int s = 0; s < 24; ++s) {
        double x[5];
        tetra_nodes(E, nband, nocc, a, o, kp, tets, tetk[24 * k + s], da, dr, x);
        const double cd = 0.5 * (x[0] + x[4]);
        bool near = false;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const double g = x[i + 1] - x[i];
            near = near || (g > 0.0 && g < TT_NEAR);
        }
        fld(s, 0) = (R)(x[1] - cd);
        fld(s, 1) = (R)(x[2] - cd);
        fld(s, 2) = (R)(x[3] - cd);
        fld(s, 3) = (R)(cd - d0);
        fld(s, 4) = near ? -(R)(x[4] - x[0]) - (R)1 : (R)(x[4] - x[0]);
    }
    const int f1 = min(nf, (int)(blockIdx.y + 1) * fch);
    for (int f = blockIdx.y * fch; f < f1; ++f) {
        const double wv = freq[f];
        double2 acc = make_double2(0.0, 0.0);
        for (int side = 0; side < 2; ++side) {
            double2 zd;
            if (axis == RP_AXIS_REAL)
                zd = side == 0 ? make_double2(wv, delta) : make_double2(-wv, ordering == RP_TIME_ORDERED ? delta : -delta);
            else
                zd = side == 0 ? make_double2(0.0, wv + delta)
                               : make_double2(0.0, ordering == RP_TIME_ORDERED ? -wv + delta : -wv - delta);
            const C zr = TT<R>::mk((R)(zd.x - d0), (R)zd.y);    // pole relative to D0
            C sacc = TT<R>::mk(0, 0);
            for (int s = 0; s < 24; ++s) {
                const R sp = fld(s, 4);
                const R spread = sp < (R)0 ? -sp - (R)1 : sp;
                R tr[5] = {(R)-0.5 * spread, fld(s, 0), fld(s, 1), fld(s, 2), (R)0.5 * spread};
                const R ct = fld(s, 3);
                if (sizeof(R) == 4 && sp < (R)0) {
                    defer_or_eval(queue, qcap, qcount, t, f, s, side, sacc, E, nband, nocc, a, o, kp, tets,
                                  tetk[24 * k + s], da, dr, zd);
                    continue;
                }
                const C y = TT<R>::mk(zr.x - ct, zr.y);
                if (spread * spread <= (R)(TT_TAU * TT_TAU) * (y.x * y.x + y.y * y.y)) {
                    sacc = tadd(sacc, dd5_series<R>(tr[1], tr[2], tr[3], spread, y));
                } else {
                    // a wide set: in the FP32 pass it goes to the work list (evaluated there with
                    // the full table, so that the warps here stay on the series path)
                    if (sizeof(R) == 4) {
                        const unsigned long long slot = atomicAdd(qcount, 1ULL);
                        if (slot < qcap) {
                            queue[slot] = tetra_item(t, f, s, side, 1);
                            continue;
                        }
                    }
                    R xr[5];
#pragma unroll
                    for (int i = 0; i < 5; ++i) xr[i] = ct + tr[i];
                    sacc = tadd(sacc, dd_table_entry<R>(xr, zr));
                }
            }
            acc.x += (double)sacc.x;
            acc.y += (double)sacc.y;
        }
        wout[(size_t)f * K + t] = make_double2(acc.x * pref / 6.0, acc.y * pref / 6.0);
    }
}

cudaError_t launch_tetra(rp_ctx* c, int axis, int ordering, int nf, const double* d_freq, double delta,
                         double da, double dr, bool fp32, double2* w, cudaStream_t st) {
    {   // series coefficients 6 / (m (m-1) (m-2) (m-3)) of the resonant path
        static double bq[64];
        for (int m = 0; m < 64; ++m) bq[m] = m >= 4 ? 6.0 / ((double)m * (m - 1) * (m - 2) * (m - 3)) : 0.0;
        cudaError_t e = cudaMemcpyToSymbolAsync(c_bq, bq, sizeof(bq), 0, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
    }
    // FP64 work list of the FP32 pass: up to 2% of all evaluations (overflow is evaluated in place)
    const long long Kp = (long long)c->nk * c->nemp * c->nocc;
    unsigned long long qcap = (unsigned long long)std::max(1LL << 16, (long long)(0.02 * 48.0 * nf * Kp));
    if (fp32 && ensure(c, c->s_queue, (qcap + 1) * sizeof(unsigned long long)) != RP_OK)
        return cudaErrorMemoryAllocation;
    unsigned long long* qcount = fp32 ? (unsigned long long*)c->s_queue.p : nullptr;
    unsigned long long* queue = fp32 ? qcount + 1 : nullptr;
    if (fp32) {
        cudaError_t e = cudaMemsetAsync(qcount, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
    }
    const long long K = (long long)c->nk * c->nemp * c->nocc;
    const int bs = 128;
    // frequencies per grid row: all of them when the pairs alone fill the GPU
    const int fch = K >= 4LL * 152 * bs ? nf : std::max(1, (int)((nf * K + 4LL * 152 * bs - 1) / (4LL * 152 * bs)));
    dim3 grid((unsigned)((K + bs - 1) / bs), (unsigned)((nf + fch - 1) / fch));
    const size_t smem = (size_t)24 * TT_FIELDS * bs * (fp32 ? sizeof(float) : sizeof(double));
    if (fp32) {
        cudaFuncSetAttribute(k_tetra_weights<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_tetra_weights<float><<<grid, bs, smem, st>>>(
            (const double*)c->d_energy.p, c->T.empty() ? nullptr : (const double*)c->d_T.p, c->nband, c->nocc,
            c->nemp, c->nk, (const int*)c->plan.d_kp.p, (const int*)c->d_tets.p, (const int*)c->d_tetk.p, nf, fch,
            d_freq, axis, ordering, delta, da, dr, w, queue, qcap, qcount);
        // the deferred items (count read on the device): a grid-stride pass
        k_tetra_fixup<<<c->num_sms * 8, 128, 0, st>>>(
            (const double*)c->d_energy.p, c->T.empty() ? nullptr : (const double*)c->d_T.p, c->nband, c->nocc,
            c->nemp, c->nk, (const int*)c->plan.d_kp.p, (const int*)c->d_tets.p, (const int*)c->d_tetk.p, d_freq,
            axis, ordering, delta, da, dr, queue, qcount, qcap, w);
    } else {
        cudaFuncSetAttribute(k_tetra_weights<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_tetra_weights<double><<<grid, bs, smem, st>>>(
            (const double*)c->d_energy.p, c->T.empty() ? nullptr : (const double*)c->d_T.p, c->nband, c->nocc,
            c->nemp, c->nk, (const int*)c->plan.d_kp.p, (const int*)c->d_tets.p, (const int*)c->d_tetk.p, nf, fch,
            d_freq, axis, ordering, delta, da, dr, w, nullptr, 0, nullptr);
    }
    return cudaGetLastError();
}

}  // namespace rp
