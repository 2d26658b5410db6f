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

// Fourth divided difference over the five nodes c + t_v (t_0 = -s/2, t_4 = s/2, |t_v| <= s/2) by
// the Taylor series about the centre c:  y^-1 sum_k b_{4+k} h_k(t/r) u^k,  y = z - c, r = |y|,
// u = conj(y)/r, b_q = 6 / (q (q-1) (q-2) (q-3)).  The complete homogeneous polynomials h_k of the
// scaled nodes follow from their elementary symmetric polynomials, e_j(t/r) = e_j(t) r^-j, passed
// in unscaled (they do not depend on z).  With every scaled node within rho = s / (2 r) of zero,
// |h_k| <= C(k+4, 4) rho^k, so |b_{4+k} h_k u^k| <= rho^k / 4 while the sum is at least
// (1 - 2 rho) / (4 (1 - rho)): after K terms the remainder is below 2 rho^(K+1) of the sum for
// rho <= 1/4, and K is the smallest count that puts it under half the unit roundoff.  In FP32 the
// count is made uniform over the converged lanes of the warp (the largest of theirs).
template <typename R>
__device__ __forceinline__ typename TT<R>::C dd5_series(const R (&e)[5], R s, typename TT<R>::C y, R r2) {
    using C = typename TT<R>::C;
    constexpr int KM = sizeof(R) == 8 ? 28 : 13;            // K at rho = 1/4
    const R rinv = TT<R>::rsq(r2);
    const R rho = (R)0.5 * s * rinv;
    int K = 0;
    if constexpr (sizeof(R) == 4) {
        if (rho > 0.f) K = (int)ceilf(__fdividef(-25.25f, __log2f(rho)));   // log2 of half the roundoff
        K = K < KM ? K : KM;
        K = __reduce_max_sync(__activemask(), K);
    } else {
        if (rho > 0.0) K = (int)ceil(-38.5 / log(rho));
        K = K < KM ? K : KM;
    }
    const R r_2 = rinv * rinv;
    const R e1 = e[0] * rinv, e2 = e[1] * r_2, e3 = e[2] * r_2 * rinv, e4 = e[3] * r_2 * r_2,
            e5 = e[4] * r_2 * r_2 * rinv;
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

// elementary symmetric polynomials e_1 .. e_5 of five values
template <typename R>
__device__ __forceinline__ void esym5(const R (&t)[5], R (&e)[5]) {
    e[0] = e[1] = e[2] = e[3] = e[4] = 0;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        e[4] += t[v] * e[3];
        e[3] += t[v] * e[2];
        e[2] += t[v] * e[1];
        e[1] += t[v] * e[0];
        e[0] += t[v];
    }
}

// 6 / (m (m-1) (m-2) (m-3)) for m = 0 .. 63 (entries below 4 unused), and the same values rounded
// to float for the FP32 table (no double load or conversion per term)
__constant__ double c_bq[64];
__constant__ float c_bqf[64];

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
        const int qc = q < 64 ? q : 63;
        const C b = q >= 4 ? TT<R>::mk(sizeof(R) == 4 ? (R)c_bqf[qc] : (R)c_bq[qc], 0) : bcoef<R>(q, L);
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

// five nodes sorted, degenerate groups merged into their mean (Eq. tetrahedron thresholds), FP64
__device__ __forceinline__ void sort_merge5(double (&x)[5], double da, double dr) {
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
    sort_merge5(x, da, dr);
}

// nodes of entry `code` for pair (a, o) relative to the pair's transition energy d0, in FP32:
// the vertex energies are differenced in FP64 and rounded once, then sorted and merged (Eq.
// tetrahedron thresholds on the absolute energies d0 + x) in FP32
__device__ __forceinline__ void tetra_nodes_rel32(const double* __restrict__ E, int nband, int nocc, int a, int o,
                                                  const int* __restrict__ kp, const int* __restrict__ tets, int code,
                                                  double d0, float da, float dr, float (&x)[5]) {
    const int tt = code >> 2, jv = code & 3;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int kv = tets[4 * tt + v];
        x[v] = (float)((E[(size_t)kp[kv] * nband + nocc + a] - E[(size_t)kv * nband + o]) - d0);
    }
    x[4] = jv == 0 ? x[0] : jv == 1 ? x[1] : jv == 2 ? x[2] : x[3];
    auto sw = [](float& p, float& q) { const float lo = fminf(p, q), hi = fmaxf(p, q); p = lo; q = hi; };
    sw(x[0], x[1]); sw(x[3], x[4]); sw(x[2], x[4]); sw(x[2], x[3]); sw(x[0], x[3]);
    sw(x[0], x[2]); sw(x[1], x[4]); sw(x[1], x[3]); sw(x[1], x[2]);
    const float d0f = (float)d0;
    bool brk[5];
    brk[0] = true;
    float start = x[0];
#pragma unroll
    for (int i = 1; i < 5; ++i) {
        const float thr = da + dr * fmaxf(fabsf(d0f + start), fabsf(d0f + x[i]));
        brk[i] = (x[i] - start) >= thr;
        if (brk[i]) start = x[i];
    }
    if (brk[1] && brk[2] && brk[3] && brk[4]) return;
    float y[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        float sum = 0.f;
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
    const double r2 = y.x * y.x + y.y * y.y;
    if (spread * spread <= TT_TAU * TT_TAU * r2) {
        const double t[5] = {-0.5 * spread, x[1] - c, x[2] - c, x[3] - c, 0.5 * spread};
        double e[5];
        esym5<double>(t, e);
        return dd5_series<double>(e, spread, y, r2);
    }
    bool unused = false;
    return dd5_table<double>(x, z, &unused);
}

template <typename R>
__device__ __noinline__ typename TT<R>::C dd_table_entry(const R (&x)[5], typename TT<R>::C z) {
    bool unused = false;
    return dd5_table<R>(x, z, &unused);
}

#define TT_NEAR 1e-5  // gap below which unmerged nodes make a set near-degenerate
#define TT_FIELDS 7   // FP64 node sets: e1 .. e5, centre - D0, spread (negative: near-degenerate set)
#define TT_FIELDS32 5 // FP32 node sets: the three inner centred nodes over the half-spread, centre - D0, spread
#define TT_FC 4       // frequencies per node-set read

// pole z of side 0 (w + i d, or i(nu + d)) and side 1 (the second term of Eq. Xakqbk)
__device__ __forceinline__ double2 tetra_pole(const double* __restrict__ freq, int f, int side, int axis,
                                              int ordering, double delta) {
    const double wv = freq[f];
    if (axis == RP_AXIS_REAL)
        return side == 0 ? make_double2(wv, delta) : make_double2(-wv, ordering == RP_TIME_ORDERED ? delta : -delta);
    return side == 0 ? make_double2(0.0, wv + delta)
                     : make_double2(0.0, ordering == RP_TIME_ORDERED ? -wv + delta : -wv - delta);
}

// The 2 TT_FC poles of one FP32 node set (nodes c + t, centre c = ct relative to D0), summed by the
// series of dd5_series with the pole-independent part done once: with sg the half-spread,
//   h_k(t / r) u^k = h_k(t / sg) w^k,  w = sg conj(y) / r^2,  y = z - c,
// so the complete homogeneous polynomials of the half-spread-scaled nodes (e: their elementary
// symmetric polynomials) are formed once for the set, c_k = b_{4+k} h_k, and each pole sums
// 1/4 + sum_k c_k w^k by Horner and multiplies by 1/y.  The term count of a pole is the bound of
// dd5_series (rho = sg / r); the poles of one side take the largest count over their frequencies
// and the converged lanes, so that the four Horner chains of a side run side by side.  A pole whose
// set is too wide for the series (rho > 1/4) marks bit 2 s + side of its frequency's work-list mask.
__device__ __forceinline__ void series_poles32(const float (&e)[5], float spread, float ct,
                                               const float2 (&zr)[TT_FC][2], int nfc, int s,
                                               float2 (&acc)[TT_FC], unsigned long long (&dmask)[TT_FC]) {
    constexpr int KM = 13;                        // the count at rho = 1/4
    const unsigned am = __activemask();
    const float sg = 0.5f * spread;
    float2 g[TT_FC][2], w[TT_FC][2];
    bool use[TT_FC][2];
    int ksd[2] = {0, 0};
#pragma unroll
    for (int fi = 0; fi < TT_FC; ++fi)
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const float yx = zr[fi][side].x - ct, yy = zr[fi][side].y;
            const float r2 = yx * yx + yy * yy;
            const bool live = fi < nfc;
            const bool ok = spread * spread <= (float)(TT_TAU * TT_TAU) * r2;
            if (live && !ok) dmask[fi] |= 1ull << (2 * s + side);
            use[fi][side] = live && ok;
            const float inv = __fdividef(1.f, r2);
            g[fi][side] = make_float2(yx * inv, -yy * inv);
            w[fi][side] = make_float2(sg * g[fi][side].x, sg * g[fi][side].y);
            const float rho2 = sg * sg * inv;
            int K = 0;
            if (live && ok && rho2 > 0.f) K = (int)ceilf(__fdividef(-50.5f, __log2f(rho2)));  // rho^K < 2^-25.25
            K = K < KM ? K : KM;
            ksd[side] = max(ksd[side], __reduce_max_sync(am, K));
        }
    const int ks = max(ksd[0], ksd[1]);
    float c[KM + 1];
    float h1 = 0.f, h2 = 0.f, h3 = 0.f, h4 = 0.f, hk = 1.f;
#pragma unroll
    for (int k = 1; k <= KM; ++k) {
        c[k] = 0.f;
        if (k <= ks) {
            const float hn = (e[0] * hk - e[1] * h1) + (e[2] * h2 - e[3] * h3) + e[4] * h4;
            h4 = h3; h3 = h2; h2 = h1; h1 = hk; hk = hn;
            c[k] = (float)(6.0 / ((double)(k + 4) * (k + 3) * (k + 2) * (k + 1))) * hn;
        }
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        float2 P[TT_FC];
#pragma unroll
        for (int fi = 0; fi < TT_FC; ++fi) P[fi] = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = KM; k >= 1; --k) {
            if (k > ksd[side]) continue;
#pragma unroll
            for (int fi = 0; fi < TT_FC; ++fi) {
                const float px = P[fi].x + c[k];
                P[fi] = make_float2(px * w[fi][side].x - P[fi].y * w[fi][side].y,
                                    px * w[fi][side].y + P[fi].y * w[fi][side].x);
            }
        }
#pragma unroll
        for (int fi = 0; fi < TT_FC; ++fi) {
            if (!use[fi][side]) continue;
            const float sx = 0.25f + P[fi].x, sy = P[fi].y;
            acc[fi].x += sx * g[fi][side].x - sy * g[fi][side].y;
            acc[fi].y += sx * g[fi][side].y + sy * g[fi][side].x;
        }
    }
}

// Work list of the FP32 pass: one item per (pair t, frequency f) that has node sets too wide for the
// series, with the mask of those (tetrahedron-vertex entry s, pole side) as bit 2 s + side.
// x = t << 16 | f, y = mask (48 bits).  Each (t, f) appears at most once, so its pass adds into the
// weight without atomics.
__device__ __forceinline__ ulonglong2 tetra_item(long long t, int f, unsigned long long mask) {
    return make_ulonglong2(((unsigned long long)t << 16) | (unsigned long long)f, mask);
}

// Append an item to the work list with one counter update per warp (the converged lanes that
// push take consecutive slots); false when the list is full.
__device__ __forceinline__ bool queue_push(ulonglong2* queue, unsigned long long qcap, unsigned long long* qcount,
                                           ulonglong2 item) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(qcount, (unsigned long long)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    const unsigned long long slot = base + (unsigned long long)__popc(mask & ((1u << lane) - 1u));
    if (slot >= qcap) return false;
    queue[slot] = item;
    return true;
}

// Sum of the divided differences of the entries in `mask` for pair (k, a, o) at frequency f: each
// node set in FP32 relative to d0 with the full table, or in FP64 when two of its nodes lie closer
// than TT_NEAR without being merged (the FP32 nodes decide, as in the main pass).
__device__ double2 deferred_sum(const double* __restrict__ E, int nband, int nocc, int a, int o, int k,
                                const int* __restrict__ kp, const int* __restrict__ tets,
                                const int* __restrict__ tetk, const double* __restrict__ freq, int f, int axis,
                                int ordering, double delta, double da, double dr, double d0,
                                unsigned long long mask) {
    double2 sum = make_double2(0.0, 0.0);
    while (mask) {
        const int bit = __ffsll((long long)mask) - 1;
        mask &= mask - 1;
        const int s = bit >> 1, side = bit & 1;
        const double2 zd = tetra_pole(freq, f, side, axis, ordering, delta);
        float xr[5];
        tetra_nodes_rel32(E, nband, nocc, a, o, kp, tets, tetk[24 * k + s], d0, (float)da, (float)dr, xr);
        bool near = false;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float g = xr[i + 1] - xr[i];
            near = near || (g > 0.f && g < (float)TT_NEAR);
        }
        double2 r;
        if (near) {
            r = dd_fp64_entry(E, nband, nocc, a, o, kp, tets, tetk[24 * k + s], da, dr, zd);
        } else {
            const float2 rf = dd_table_entry<float>(xr, make_float2((float)(zd.x - d0), (float)zd.y));
            r = make_double2((double)rf.x, (double)rf.y);
        }
        sum.x += r.x;
        sum.y += r.y;
    }
    return sum;
}

// Pass over the work list: one (pair, frequency) per thread, its deferred entries added to the weight
__global__ void __launch_bounds__(128) k_tetra_fixup(const double* __restrict__ E, const double* __restrict__ Tw,
                                                     int nband, int nocc, int nemp, int nk,
                                                     const int* __restrict__ kp, const int* __restrict__ tets,
                                                     const int* __restrict__ tetk, const double* __restrict__ freq,
                                                     int axis, int ordering, double delta, double da, double dr,
                                                     const ulonglong2* __restrict__ queue,
                                                     const unsigned long long* __restrict__ qcount,
                                                     unsigned long long qcap, double2* __restrict__ wout) {
    const unsigned long long n = min(*qcount, qcap);
    const long long K = (long long)nk * nemp * nocc;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const ulonglong2 item = queue[i];
        const long long t = (long long)(item.x >> 16);
        const int f = (int)(item.x & 0xFFFF);
        const int o = (int)(t % nocc);
        const int a = (int)((t / nocc) % nemp);
        const int k = (int)(t / ((long long)nocc * nemp));
        double pref = 2.0 / (double)nk;
        if (Tw) pref *= 1.0 - Tw[(size_t)kp[k] * nband + nocc + a] * Tw[(size_t)k * nband + o];
        const double ps = pref / 6.0;
        const double d0 = E[(size_t)kp[k] * nband + nocc + a] - E[(size_t)k * nband + o];
        const double2 r = deferred_sum(E, nband, nocc, a, o, k, kp, tets, tetk, freq, f, axis, ordering, delta, da,
                                       dr, d0, item.y);
        double2* dst = wout + (size_t)f * K + t;
        double2 v = *dst;
        v.x += r.x * ps;
        v.y += r.y * ps;
        *dst = v;
    }
}

// Weights for one (k, a, o) per thread and a chunk of frequencies per grid row.  The 24
// tetrahedron-vertex node sets are prepared once (sorted, merged, centred; FP64 for R = double,
// FP32 relative to the pair's own transition energy D0 for R = float) and kept in shared memory:
// for R = double their centre, spread and the elementary symmetric polynomials of the centred
// nodes; for R = float (five fields, which with 168 registers lets six 64-thread blocks share an
// SM) their centre, spread and the three inner centred nodes over the half-spread, whose
// symmetric polynomials (with the outer nodes -1 and 1) are formed again at each read.  The
// frequencies are then taken TT_FC at a time, each node set read once for the 2 TT_FC poles.  With
// R = float the node sets too wide for the series go to the work list (there the FP32 table, or
// FP64 when two of the set's nodes lie closer than TT_NEAR without being merged).
template <typename R>
__global__ void __launch_bounds__(64, sizeof(R) == 4 ? 6 : 1) k_tetra_weights(const double* __restrict__ E, const double* __restrict__ Tw,
                                                      int nband, int nocc, int nemp, int nk,
                                                      const int* __restrict__ kp, const int* __restrict__ tets,
                                                      const int* __restrict__ tetk, int nf, int fch,
                                                      const double* __restrict__ freq, int axis, int ordering,
                                                      double delta, double da, double dr,
                                                      double2* __restrict__ wout, ulonglong2* __restrict__ queue,
                                                      unsigned long long qcap, unsigned long long* qcount) {
    using C = typename TT<R>::C;
    extern __shared__ __align__(16) unsigned char tsm_raw[];
    R* tsm = reinterpret_cast<R*>(tsm_raw);
    const int bd = blockDim.x, tid = threadIdx.x;
    constexpr int NFLD = sizeof(R) == 4 ? TT_FIELDS32 : TT_FIELDS;
    auto fld = [&](int s, int f) -> R& { return tsm[(s * NFLD + f) * bd + tid]; };
    const long long t = (long long)blockIdx.x * bd + tid;
    const long long K = (long long)nk * nemp * nocc;
    if (t >= K) return;
    const int o = (int)(t % nocc);
    const int a = (int)((t / nocc) % nemp);
    const int k = (int)(t / ((long long)nocc * nemp));
    double pref = 2.0 / (double)nk;
    if (Tw) pref *= 1.0 - Tw[(size_t)kp[k] * nband + nocc + a] * Tw[(size_t)k * nband + o];
    const double ps = pref / 6.0;
    const double d0 = E[(size_t)kp[k] * nband + nocc + a] - E[(size_t)k * nband + o];
    for (int s = 0; s < 24; ++s) {
        R x[5];
        if constexpr (sizeof(R) == 4) {
            tetra_nodes_rel32(E, nband, nocc, a, o, kp, tets, tetk[24 * k + s], d0, (float)da, (float)dr, x);
        } else {
            double xa[5];
            tetra_nodes(E, nband, nocc, a, o, kp, tets, tetk[24 * k + s], da, dr, xa);
#pragma unroll
            for (int i = 0; i < 5; ++i) x[i] = xa[i] - d0;
        }
        const R cd = (R)0.5 * (x[0] + x[4]);
        const R spread = x[4] - x[0];
        if constexpr (sizeof(R) == 4) {
            // inner centred nodes over the half-spread sg (the outer two are -1 and 1)
            const float sg = 0.5f * spread;
            const float si = sg > 0.f ? 1.f / sg : 0.f;
            fld(s, 0) = (x[1] - cd) * si;
            fld(s, 1) = (x[2] - cd) * si;
            fld(s, 2) = (x[3] - cd) * si;
            fld(s, 3) = cd;
            fld(s, 4) = spread;
        } else {
            bool near = false;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const R g = x[i + 1] - x[i];
                near = near || (g > (R)0 && g < (R)TT_NEAR);
            }
            R e[5];
            const R tc[5] = {(R)-0.5 * spread, x[1] - cd, x[2] - cd, x[3] - cd, (R)0.5 * spread};
            esym5<R>(tc, e);
#pragma unroll
            for (int j = 0; j < 5; ++j) fld(s, j) = e[j];
            fld(s, 5) = cd;
            fld(s, 6) = near ? -spread - (R)1 : spread;
        }
    }
    const int fend = min(nf, (int)(blockIdx.y + 1) * fch);
    for (int f0 = blockIdx.y * fch; f0 < fend; f0 += TT_FC) {
        C zr[TT_FC][2], acc[TT_FC];
        unsigned long long dmask[TT_FC];         // entries of each frequency left to the work list
#pragma unroll
        for (int fi = 0; fi < TT_FC; ++fi) {
            acc[fi] = TT<R>::mk(0, 0);
            dmask[fi] = 0ull;
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const double2 zd = tetra_pole(freq, min(f0 + fi, nf - 1), side, axis, ordering, delta);
                zr[fi][side] = TT<R>::mk((R)(zd.x - d0), (R)zd.y);    // pole relative to D0
            }
        }
        for (int s = 0; s < 24; ++s) {
            if constexpr (sizeof(R) == 4) {
                const float spread = fld(s, 4), ct = fld(s, 3);
                const float one = spread > 0.f ? 1.f : 0.f;
                const float tc[5] = {-one, fld(s, 0), fld(s, 1), fld(s, 2), one};
                float e[5];
                esym5<float>(tc, e);
                series_poles32(e, spread, ct, zr, fend - f0, s, acc, dmask);
            } else {
                const R sp = fld(s, 6);
                const R spread = sp < (R)0 ? -sp - (R)1 : sp;
                const R e[5] = {fld(s, 0), fld(s, 1), fld(s, 2), fld(s, 3), fld(s, 4)};
                const R ct = fld(s, 5);
#pragma unroll
                for (int fi = 0; fi < TT_FC; ++fi) {
                    if (f0 + fi >= fend) break;
#pragma unroll
                    for (int side = 0; side < 2; ++side) {
                        const C y = TT<R>::mk(zr[fi][side].x - ct, zr[fi][side].y);
                        const R r2 = y.x * y.x + y.y * y.y;
                        if (spread * spread <= (R)(TT_TAU * TT_TAU) * r2) {
                            acc[fi] = tadd(acc[fi], dd5_series<R>(e, spread, y, r2));
                            continue;
                        }
                        double xa[5];
                        R xr[5];
                        tetra_nodes(E, nband, nocc, a, o, kp, tets, tetk[24 * k + s], da, dr, xa);
#pragma unroll
                        for (int i = 0; i < 5; ++i) xr[i] = (R)(xa[i] - d0);
                        acc[fi] = tadd(acc[fi], dd_table_entry<R>(xr, zr[fi][side]));
                    }
                }
            }
        }
#pragma unroll
        for (int fi = 0; fi < TT_FC; ++fi) {
            if (f0 + fi >= fend) break;
            double2 extra = make_double2(0.0, 0.0);
            if (sizeof(R) == 4 && dmask[fi] != 0ull &&
                !queue_push(queue, qcap, qcount, tetra_item(t, f0 + fi, dmask[fi])))
                // the list is full: the same evaluation here
                extra = deferred_sum(E, nband, nocc, a, o, k, kp, tets, tetk, freq, f0 + fi, axis, ordering, delta,
                                     da, dr, d0, dmask[fi]);
            wout[(size_t)(f0 + fi) * K + t] = make_double2(((double)acc[fi].x + extra.x) * ps,
                                                           ((double)acc[fi].y + extra.y) * ps);
        }
    }
}

// ---- metals: Fermi-surface clipping -------------------------------------------------------------
// Pieces of a tetrahedron where the linear function with vertex values e is negative, as rows of
// barycentric coordinates of the tetrahedron (out[p][i][j]: sub-vertex i of piece p = sum_j out
// vertex j): none (no vertex below zero), the corner at the lowest vertex (one), a triangular
// prism (two or three: three pieces, (A0 A1 A2 B0), (A1 A2 B0 B1), (A2 B0 B1 B2) for triangles A, B
// with lateral edges A_i B_i), the whole (four).  Zero counts as not negative.
__device__ int clip_negative4(const double (&e)[4], double (&out)[3][4][4]) {
    int s[4] = {0, 1, 2, 3};
    for (int i = 1; i < 4; ++i) {            // stable insertion sort of the vertices by e
        const int v = s[i];
        int j = i - 1;
        while (j >= 0 && e[s[j]] > e[v]) { s[j + 1] = s[j]; --j; }
        s[j + 1] = v;
    }
    int n = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) n += e[i] < 0.0 ? 1 : 0;
    auto unit = [](double (&r)[4], int u) {
#pragma unroll
        for (int j = 0; j < 4; ++j) r[j] = j == u ? 1.0 : 0.0;
    };
    auto cut = [&](double (&r)[4], int u, int v) {   // zero of the edge u-v (e[u] < 0 <= e[v])
        const double t = e[u] / (e[u] - e[v]);
#pragma unroll
        for (int j = 0; j < 4; ++j) r[j] = 0.0;
        r[u] = 1.0 - t;
        r[v] = t;
    };
    auto prism = [&](double (&A)[3][4], double (&B)[3][4]) {
        const double* rows[3][4] = {{A[0], A[1], A[2], B[0]}, {A[1], A[2], B[0], B[1]}, {A[2], B[0], B[1], B[2]}};
        for (int p = 0; p < 3; ++p)
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) out[p][i][j] = rows[p][i][j];
    };
    if (n == 0) return 0;
    if (n == 4) {
        for (int i = 0; i < 4; ++i) unit(out[0][i], i);
        return 1;
    }
    if (n == 1) {
        unit(out[0][0], s[0]);
        cut(out[0][1], s[0], s[1]);
        cut(out[0][2], s[0], s[2]);
        cut(out[0][3], s[0], s[3]);
        return 1;
    }
    double A[3][4], B[3][4];
    if (n == 2) {
        unit(A[0], s[0]); cut(A[1], s[0], s[2]); cut(A[2], s[0], s[3]);
        unit(B[0], s[1]); cut(B[1], s[1], s[2]); cut(B[2], s[1], s[3]);
    } else {
        unit(A[0], s[0]); unit(A[1], s[1]); unit(A[2], s[2]);
        cut(B[0], s[0], s[3]); cut(B[1], s[1], s[3]); cut(B[2], s[2], s[3]);
    }
    prism(A, B);
    return 3;
}

__device__ __forceinline__ double det4(const double (&m)[4][4]) {
    const double a0 = m[2][2] * m[3][3] - m[2][3] * m[3][2], a1 = m[2][1] * m[3][3] - m[2][3] * m[3][1];
    const double a2 = m[2][1] * m[3][2] - m[2][2] * m[3][1], a3 = m[2][0] * m[3][3] - m[2][3] * m[3][0];
    const double a4 = m[2][0] * m[3][2] - m[2][2] * m[3][0], a5 = m[2][0] * m[3][1] - m[2][1] * m[3][0];
    return m[0][0] * (m[1][1] * a0 - m[1][2] * a1 + m[1][3] * a2) -
           m[0][1] * (m[1][0] * a0 - m[1][2] * a3 + m[1][3] * a4) +
           m[0][2] * (m[1][0] * a1 - m[1][1] * a3 + m[1][3] * a5) -
           m[0][3] * (m[1][0] * a2 - m[1][1] * a4 + m[1][2] * a5);
}

// f_z[x0..x4] in FP64 from five nodes (sorted and merged here; the series about the centre for a
// narrow set, else the table)
__device__ __noinline__ double2 dd_fp64_nodes(double (&x)[5], double da, double dr, double2 z) {
    sort_merge5(x, da, dr);
    const double c = 0.5 * (x[0] + x[4]);
    const double2 y = make_double2(z.x - c, z.y);
    const double spread = x[4] - x[0];
    const double r2 = y.x * y.x + y.y * y.y;
    if (spread * spread <= TT_TAU * TT_TAU * r2) {
        const double t[5] = {-0.5 * spread, x[1] - c, x[2] - c, x[3] - c, 0.5 * spread};
        double e[5];
        esym5<double>(t, e);
        return dd5_series<double>(e, spread, y, r2);
    }
    bool unused = false;
    return dd5_table<double>(x, z, &unused);
}

// Metallic weights, FP64, one (k, a, o) per thread: for each of the 24 tetrahedra around k the part
// where band o (at the vertex points) lies below the Fermi energy and band a (at their k + q) above
// it, cut into pieces; a piece F (barycentric rows, volume |det F|) adds |det F| sum_i F[i][j] w_i
// to vertex j, w_i its own vertex-i weight (the unclipped formula with D at its vertices).
__global__ void __launch_bounds__(128) k_tetra_metal(const double* __restrict__ E, const double* __restrict__ Tw,
                                                     int nband, int nocc, int nemp, int nk,
                                                     const int* __restrict__ kp, const int* __restrict__ tets,
                                                     const int* __restrict__ tetk, int nf,
                                                     const double* __restrict__ freq, int axis, int ordering,
                                                     double delta, double da, double dr, double fermi,
                                                     double2* __restrict__ wout) {
    const long long K = (long long)nk * nemp * nocc;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K) return;
    const int o = (int)(t % nocc), a = (int)((t / nocc) % nemp), k = (int)(t / ((long long)nocc * nemp));
    double pref = 2.0 / (double)nk;
    if (Tw) pref *= 1.0 - Tw[(size_t)kp[k] * nband + nocc + a] * Tw[(size_t)k * nband + o];
    const double ps = pref / 6.0;
    for (int f = 0; f < nf; ++f) wout[(size_t)f * K + t] = make_double2(0.0, 0.0);
    for (int s = 0; s < 24; ++s) {
        const int code = tetk[24 * k + s];
        const int tt = code >> 2, jv = code & 3;
        double eo[4], ea[4], d[4], g1[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int kv = tets[4 * tt + v];
            eo[v] = E[(size_t)kv * nband + o];
            ea[v] = E[(size_t)kp[kv] * nband + nocc + a];
            d[v] = ea[v] - eo[v];
            g1[v] = eo[v] - fermi;
        }
        double P1[3][4][4];
        const int n1 = clip_negative4(g1, P1);
        for (int p1 = 0; p1 < n1; ++p1) {
            double g2[4];
            for (int i = 0; i < 4; ++i) {
                g2[i] = 0.0;
                for (int j = 0; j < 4; ++j) g2[i] += P1[p1][i][j] * (fermi - ea[j]);
            }
            double P2[3][4][4];
            const int n2 = clip_negative4(g2, P2);
            for (int p2 = 0; p2 < n2; ++p2) {
                double F[4][4];
                for (int i = 0; i < 4; ++i)
                    for (int j = 0; j < 4; ++j) {
                        double v = 0.0;
                        for (int m = 0; m < 4; ++m) v += P2[p2][i][m] * P1[p1][m][j];
                        F[i][j] = v;
                    }
                const double vol = fabs(det4(F));
                if (vol == 0.0) continue;
                double ds[4];
                for (int i = 0; i < 4; ++i) {
                    ds[i] = 0.0;
                    for (int j = 0; j < 4; ++j) ds[i] += F[i][j] * d[j];
                }
                for (int f = 0; f < nf; ++f) {
                    double2 acc = make_double2(0.0, 0.0);
                    for (int side = 0; side < 2; ++side) {
                        const double2 z = tetra_pole(freq, f, side, axis, ordering, delta);
                        for (int i = 0; i < 4; ++i) {
                            const double cf = F[i][jv];
                            if (cf == 0.0) continue;
                            double x[5] = {ds[0], ds[1], ds[2], ds[3], ds[i]};
                            const double2 w = dd_fp64_nodes(x, da, dr, z);
                            acc.x += cf * w.x;
                            acc.y += cf * w.y;
                        }
                    }
                    double2* dst = wout + (size_t)f * K + t;
                    double2 v = *dst;
                    v.x += vol * acc.x * ps;
                    v.y += vol * acc.y * ps;
                    *dst = v;
                }
            }
        }
    }
}

cudaError_t launch_tetra(rp_ctx* c, int axis, int ordering, int nf, const double* d_freq, double delta,
                         double da, double dr, bool fp32, double2* w, cudaStream_t st) {
    {   // series coefficients 6 / (m (m-1) (m-2) (m-3)) of the resonant path
        static double bq[64];
        static float bqf[64];
        for (int m = 0; m < 64; ++m) {
            bq[m] = m >= 4 ? 6.0 / ((double)m * (m - 1) * (m - 2) * (m - 3)) : 0.0;
            bqf[m] = (float)bq[m];
        }
        cudaError_t e = cudaMemcpyToSymbolAsync(c_bq, bq, sizeof(bq), 0, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_bqf, bqf, sizeof(bqf), 0, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
    }
    if (c->metal) {
        // Fermi-surface clipping in FP64 for every tier (the split tiers convert the weights after)
        const long long K = (long long)c->nk * c->nemp * c->nocc;
        k_tetra_metal<<<(unsigned)((K + 127) / 128), 128, 0, st>>>(
            (const double*)c->d_energy.p, c->T.empty() ? nullptr : (const double*)c->d_T.p, c->nband, c->nocc,
            c->nemp, c->nk, (const int*)c->plan.d_kp.p, (const int*)c->d_tets.p, (const int*)c->d_tetk.p, nf,
            d_freq, axis, ordering, delta, da, dr, c->efermi, w);
        return cudaGetLastError();
    }
    // work list of the FP32 pass: up to a quarter of all (pair, frequency) (overflow is evaluated in
    // place); 16-byte items after a 16-byte counter
    const long long Kp = (long long)c->nk * c->nemp * c->nocc;
    unsigned long long qcap = (unsigned long long)std::max(1LL << 16, (long long)(0.25 * nf * Kp));
    if (fp32 && ensure(c, c->s_queue, (qcap + 1) * sizeof(ulonglong2)) != RP_OK)
        return cudaErrorMemoryAllocation;
    unsigned long long* qcount = fp32 ? (unsigned long long*)c->s_queue.p : nullptr;
    ulonglong2* queue = fp32 ? (ulonglong2*)c->s_queue.p + 1 : nullptr;
    if (fp32) {
        cudaError_t e = cudaMemsetAsync(qcount, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
    }
    const long long K = (long long)c->nk * c->nemp * c->nocc;
    const int bs = 64;
    // frequencies per grid row: all of them when the pairs alone fill the GPU
    const long long fill = 4LL * c->num_sms * bs;
    const int fch = K >= fill ? nf : std::max(1, (int)((nf * K + fill - 1) / fill));
    dim3 grid((unsigned)((K + bs - 1) / bs), (unsigned)((nf + fch - 1) / fch));
    const size_t smem = (size_t)24 * (fp32 ? TT_FIELDS32 : TT_FIELDS) * bs * (fp32 ? sizeof(float) : sizeof(double));
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
