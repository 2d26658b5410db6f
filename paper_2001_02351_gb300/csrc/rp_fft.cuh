// In-register mixed-radix (4, 3, 2) Fourier transform of one line of N complex values,
// sign +1:  X[k] = sum_j x[j] exp(+2 pi i j k / N).
// Decimation in time; the twiddles W_N^e = exp(2 pi i e / N) come from a table tw[e],
// e = 0 .. NF-1, of the full line length NF (sub-transforms read it with stride NF/N).
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

template <typename C, int N, int STRIDE>
struct LineFFT {
    static constexpr int R = Radix<N>::value;
    static constexpr int M = N / R;
    static __device__ __forceinline__ void run(C (&x)[N], const C* __restrict__ tw) {
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
            for (int s = 0; s < R; ++s) LineFFT<C, M, STRIDE * R>::run(sub[s], tw);
#pragma unroll
            for (int k = 0; k < M; ++k) {
                C t[R];
                t[0] = sub[0][k];
#pragma unroll
                for (int s = 1; s < R; ++s) t[s] = c_mul(sub[s][k], tw[s * k * STRIDE]);
                small_dft<C>(t);
#pragma unroll
                for (int q = 0; q < R; ++q) x[k + M * q] = t[q];
            }
        }
    }
};

}  // namespace rp
