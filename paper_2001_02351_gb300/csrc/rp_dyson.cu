// Dyson step, FP64 (Eq. epsGG and Eq. Wq):
//   eps = 1 - v^1/2 chi v^1/2,   W = v^1/2 eps^-1 v^1/2,   v^1/2_G = sqrt(4 pi/Omega)/|q+G|.
// One CTA per frequency inverts eps in place by Gauss-Jordan elimination with partial
// pivoting (row swaps recorded and undone as column swaps at the end).  A zero or
// non-finite pivot sets err_flag[0] and leaves that frequency's output unspecified.
#include "rp_internal.h"

namespace rp {

#define DY_THREADS 1024

__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

__global__ void __launch_bounds__(DY_THREADS) k_dyson(const double2* __restrict__ chi, const double* __restrict__ vs,
                                                      int n, double2* __restrict__ Wout, int* err_flag) {
    extern __shared__ unsigned char smem[];
    double2* rowj = (double2*)smem;
    double2* colj = rowj + n;
    int* perm = (int*)(colj + n);
    __shared__ double red_v[32];
    __shared__ int red_i[32];
    __shared__ int s_piv;
    __shared__ int s_bad;
    const int f = blockIdx.x;
    const double2* X = chi + (size_t)f * n * n;
    double2* A = Wout + (size_t)f * n * n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long nn = (long long)n * n;
    for (long long e = tid; e < nn; e += DY_THREADS) {
        const int i = (int)(e / n), j = (int)(e % n);
        const double s = vs[i] * vs[j];
        double2 x = X[e];
        A[e] = make_double2((i == j ? 1.0 : 0.0) - s * x.x, -s * x.y);
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        // partial pivoting: largest |A[i][j]| over i >= j
        double best = -1.0;
        int bi = j;
        for (int i = j + tid; i < n; i += DY_THREADS) {
            const double v = cabs2(A[(size_t)i * n + j]);
            if (v > best || (v == best && i < bi)) { best = v; bi = i; }
        }
        for (int off = 16; off > 0; off >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, best, off);
            const int oi = __shfl_down_sync(0xffffffffu, bi, off);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
        __syncthreads();
        if (warp == 0) {
            best = red_v[lane];
            bi = red_i[lane];
            for (int off = 16; off > 0; off >>= 1) {
                const double ov = __shfl_down_sync(0xffffffffu, best, off);
                const int oi = __shfl_down_sync(0xffffffffu, bi, off);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (lane == 0) {
                s_piv = bi;
                perm[j] = bi;
                if (!(best > 0.0) || !isfinite(best)) s_bad = 1;
            }
        }
        __syncthreads();
        if (s_bad) break;
        const int p = s_piv;
        if (p != j) {
            for (int c = tid; c < n; c += DY_THREADS) {
                double2 t = A[(size_t)j * n + c];
                A[(size_t)j * n + c] = A[(size_t)p * n + c];
                A[(size_t)p * n + c] = t;
            }
            __syncthreads();
        }
        for (int i = tid; i < n; i += DY_THREADS) colj[i] = A[(size_t)i * n + j];
        __syncthreads();
        const double2 piv = colj[j];
        const double d = cabs2(piv);
        const double2 inv = make_double2(piv.x / d, -piv.y / d);
        for (int c = tid; c < n; c += DY_THREADS) {
            double2 v = (c == j) ? make_double2(1.0, 0.0) : A[(size_t)j * n + c];
            double2 r = make_double2(v.x * inv.x - v.y * inv.y, v.x * inv.y + v.y * inv.x);
            rowj[c] = r;
            A[(size_t)j * n + c] = r;
        }
        __syncthreads();
        for (long long e = tid; e < nn; e += DY_THREADS) {
            const int i = (int)(e / n), c = (int)(e % n);
            if (i == j) continue;
            const double2 fi = colj[i];
            const double2 r = rowj[c];
            double2 a = (c == j) ? make_double2(0.0, 0.0) : A[e];
            a.x -= fi.x * r.x - fi.y * r.y;
            a.y -= fi.x * r.y + fi.y * r.x;
            A[e] = a;
        }
        __syncthreads();
    }
    if (s_bad) {
        if (tid == 0) atomicOr(err_flag, 1);
        return;
    }
    // undo the row interchanges as column interchanges, last first
    for (int j = n - 1; j >= 0; --j) {
        const int p = perm[j];
        if (p != j) {
            for (int i = tid; i < n; i += DY_THREADS) {
                double2 t = A[(size_t)i * n + j];
                A[(size_t)i * n + j] = A[(size_t)i * n + p];
                A[(size_t)i * n + p] = t;
            }
        }
        __syncthreads();
    }
    for (long long e = tid; e < nn; e += DY_THREADS) {
        const int i = (int)(e / n), c = (int)(e % n);
        const double s = vs[i] * vs[c];
        double2 a = A[e];
        A[e] = make_double2(a.x * s, a.y * s);
    }
}

cudaError_t launch_dyson(const double2* chi, const double* vs, int ng, int nf, double2* W, int* err_flag,
                         cudaStream_t st) {
    const size_t smem = (size_t)ng * (2 * sizeof(double2) + sizeof(int));
    cudaError_t e = cudaFuncSetAttribute(k_dyson, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_dyson<<<nf, DY_THREADS, smem, st>>>(chi, vs, ng, W, err_flag);
    return cudaGetLastError();
}

}  // namespace rp
