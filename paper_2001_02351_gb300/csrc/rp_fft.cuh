// In-register mixed-radix (4, 3, 2) Fourier transform of one line of N complex values,
// sign +1:  X[k] = sum_j x[j] exp(+2 pi i j k / N).
// Decimation in time; the twiddles W_N^e = exp(2 pi i e / N) are compile-time constants
// (cos and sin of the reduced angle by their Taylor series in double, rounded once to the
// line's precision), so a transform issues no loads.
#pragma once

#include <cuda_runtime.h>

namespace rp {

template <typename C>
struct Cx;
template <>
struct Cx<float2> {
    using R = float;
    static __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
};
template <>
struct Cx<double2> {
    using R = double;
    static __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
};

template <typename C>
__device__ __forceinline__ C c_add(C a, C b) { return Cx<C>::mk(a.x + b.x, a.y + b.y); }
template <typename C>
__device__ __forceinline__ C c_sub(C a, C b) { return Cx<C>::mk(a.x - b.x, a.y - b.y); }
template <typename C>
__device__ __forceinline__ C c_mul(C a, C b) { return Cx<C>::mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// conj(a) * b
template <typename C>
__device__ __forceinline__ C c_conjmul(C a, C b) { return Cx<C>::mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
// i * a
template <typename C>
__device__ __forceinline__ C c_i(C a) { return Cx<C>::mk(-a.y, a.x); }

// cos and sin of 2 pi p / q at compile time: quarter turns exact, otherwise the angle is reduced
// to |x| <= pi/2 and summed from the Taylor series (terms to x^41 / 41!, far below double
// roundoff there)
__host__ __device__ constexpr double ct_cos_series(double x) {
    double term = 1.0, sum = 1.0;
    for (int n = 1; n <= 20; ++n) {
        term *= -x * x / ((double)(2 * n - 1) * (double)(2 * n));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double ct_sin_series(double x) {
    double term = x, sum = x;
    for (int n = 1; n <= 20; ++n) {
        term *= -x * x / ((double)(2 * n) * (double)(2 * n + 1));
        sum += term;
    }
    return sum;
}
constexpr double kCtPi = 3.14159265358979323846264338327950288;
__host__ __device__ constexpr double ct_angle(int p, int q) {   // 2 pi p / q in (-pi, pi]
    const int r = ((p % q) + q) % q;
    return 2.0 * r > q ? 2.0 * kCtPi * (double)(r - q) / (double)q : 2.0 * kCtPi * (double)r / (double)q;
}
__host__ __device__ constexpr double ct_cos2pi(int p, int q) {
    const int r = ((p % q) + q) % q;
    if ((4 * r) % q == 0) {
        const int quarter = 4 * r / q;
        return quarter == 0 ? 1.0 : (quarter == 2 ? -1.0 : 0.0);
    }
    const double x = ct_angle(p, q);
    const double ax = x < 0 ? -x : x;
    return ax > kCtPi / 2 ? -ct_cos_series(kCtPi - ax) : ct_cos_series(x);
}
__host__ __device__ constexpr double ct_sin2pi(int p, int q) {
    const int r = ((p % q) + q) % q;
    if ((4 * r) % q == 0) {
        const int quarter = 4 * r / q;
        return quarter == 1 ? 1.0 : (quarter == 3 ? -1.0 : 0.0);
    }
    const double x = ct_angle(p, q);
    if (x > kCtPi / 2) return ct_sin_series(kCtPi - x);
    if (x < -kCtPi / 2) return -ct_sin_series(kCtPi + x);
    return ct_sin_series(x);
}

// W_N^E = exp(2 pi i E / N) as a constant of the line's precision
template <typename C, int N, int E>
__device__ __forceinline__ C twiddle() {
    using R = typename Cx<C>::R;
    constexpr double c = ct_cos2pi(E, N), s = ct_sin2pi(E, N);
    return Cx<C>::mk((R)c, (R)s);
}

// a * W_N^E; the quarter turns (1, i, -1, -i) are exact swaps and sign changes, so they cost no
// multiplication by a literal zero or one
template <typename C, int N, int E>
__device__ __forceinline__ C tw_mul(C a) {
    constexpr int r = ((E % N) + N) % N;
    if constexpr (r == 0) {
        return a;
    } else if constexpr (4 * r == N) {
        return Cx<C>::mk(-a.y, a.x);
    } else if constexpr (2 * r == N) {
        return Cx<C>::mk(-a.x, -a.y);
    } else if constexpr (4 * r == 3 * N) {
        return Cx<C>::mk(a.y, -a.x);
    } else {
        return c_mul(a, twiddle<C, N, E>());
    }
}

template <int N>
struct Radix {
    static constexpr int value = (N % 4 == 0 && N > 4) ? 4 : (N % 3 == 0 ? 3 : (N % 2 == 0 ? 2 : N));
};

// small DFT of size R in place (R = 2, 3, 4), sign +1
template <typename C>
__device__ __forceinline__ void small_dft(C (&t)[2]) {
    const C a = t[0], b = t[1];
    t[0] = c_add(a, b);
    t[1] = c_sub(a, b);
}
template <typename C>
__device__ __forceinline__ void small_dft(C (&t)[4]) {
    const C s02 = c_add(t[0], t[2]), d02 = c_sub(t[0], t[2]);
    const C s13 = c_add(t[1], t[3]), d13 = c_i(c_sub(t[1], t[3]));
    t[0] = c_add(s02, s13);
    t[2] = c_sub(s02, s13);
    t[1] = c_add(d02, d13);
    t[3] = c_sub(d02, d13);
}
template <typename C>
__device__ __forceinline__ void small_dft(C (&t)[3]) {
    using R = typename Cx<C>::R;
    const R h = (R)0.86602540378443864676;   // sqrt(3)/2
    const C s = c_add(t[1], t[2]);
    const C d = c_sub(t[1], t[2]);
    const C y0 = c_add(t[0], s);
    const C m = Cx<C>::mk(t[0].x - (R)0.5 * s.x, t[0].y - (R)0.5 * s.y);
    const C rd = Cx<C>::mk(-h * d.y, h * d.x);   // i (sqrt3/2) d
    t[0] = y0;
    t[1] = c_add(m, rd);
    t[2] = c_sub(m, rd);
}

template <typename C, int N>
struct LineFFT {
    static constexpr int R = Radix<N>::value;
    static constexpr int M = N / R;
    // butterflies k .. M-1 of the last stage: t_s = W_N^{s k} sub[s][k], R-point DFT, scatter
    template <int K>
    static __device__ __forceinline__ void butterflies(C (&x)[N], C (&sub)[R][M]) {
        if constexpr (K < M) {
            C t[R];
            t[0] = sub[0][K];
            t[1] = tw_mul<C, N, K>(sub[1][K]);
            if constexpr (R > 2) t[2] = tw_mul<C, N, 2 * K>(sub[2][K]);
            if constexpr (R > 3) t[3] = tw_mul<C, N, 3 * K>(sub[3][K]);
            small_dft<C>(t);
#pragma unroll
            for (int q = 0; q < R; ++q) x[K + M * q] = t[q];
            butterflies<K + 1>(x, sub);
        }
    }
    static __device__ __forceinline__ void run(C (&x)[N]) {
        if constexpr (N == 1) {
            return;
        } else if constexpr (M == 1) {
            small_dft<C>(x);
        } else {
            C sub[R][M];
#pragma unroll
            for (int s = 0; s < R; ++s)
#pragma unroll
                for (int j = 0; j < M; ++j) sub[s][j] = x[j * R + s];
#pragma unroll
            for (int s = 0; s < R; ++s) LineFFT<C, M>::run(sub[s]);
            butterflies<0>(x, sub);
        }
    }
};

}  // namespace rp
