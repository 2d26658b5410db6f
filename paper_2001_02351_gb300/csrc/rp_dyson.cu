// Dyson step, FP64 (Eq. epsGG and Eq. Wq):
//   eps = 1 - v^1/2 chi v^1/2,   W = v^1/2 eps^-1 v^1/2,   v^1/2_G = sqrt(4 pi/Omega)/|q+G|.
// One CTA per frequency inverts eps in place by Gauss-Jordan elimination with partial
// pivoting (row swaps recorded and undone as column swaps at the end).  A zero or
// non-finite pivot sets err_flag[0] and leaves that frequency's output unspecified.
#include <cooperative_groups.h>

#include <algorithm>

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


// Cooperative form: P CTAs per frequency (grid = frequencies of the launch * P, all resident; the
// launcher groups frequencies so that a launch's matrices stay within L2), the columns of each
// frequency's matrix split among its P CTAs.  Per pivot j every CTA finds the same pivot row
// (identical scan of column j), copies column j and the pivot row into shared memory, then after a
// grid-wide sync applies the interchange and the elimination to its own columns; a second sync
// closes the step.  Row interchanges are undone afterwards as column interchanges, row by row.
// The grid barriers are shared by all frequencies, so every CTA passes exactly 2 n + 1 of them
// whatever the data: a frequency that meets a bad pivot keeps passing both barriers of each
// remaining step and skips only the arithmetic.
#define DC_THREADS 512

__global__ void __launch_bounds__(DC_THREADS) k_dyson_coop(const double2* __restrict__ chi,
                                                           const double* __restrict__ vs, int n, int P,
                                                           double2* __restrict__ Wout, int* err_flag) {
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    extern __shared__ unsigned char smem[];
    double2* colj = (double2*)smem;        // column j (rows 0..n-1), after the interchange
    double2* rowj = colj + n;              // pivot row j (all columns), after the interchange
    int* perm = (int*)(rowj + n);
    __shared__ double red_v[DC_THREADS / 32];
    __shared__ int red_i[DC_THREADS / 32];
    __shared__ int s_piv, s_bad;
    const int f = blockIdx.x / P, pc = blockIdx.x % P;
    const int c0 = (int)((long long)n * pc / P), c1 = (int)((long long)n * (pc + 1) / P);
    const double2* X = chi + (size_t)f * n * n;
    double2* A = Wout + (size_t)f * n * n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int w = c1 - c0;
    // eps = 1 - v^1/2 chi v^1/2 on this CTA's columns
    for (long long e = tid; e < (long long)n * w; e += DC_THREADS) {
        const int i = (int)(e / w), jj = c0 + (int)(e % w);
        const double sc = vs[i] * vs[jj];
        const double2 x = X[(size_t)i * n + jj];
        A[(size_t)i * n + jj] = make_double2((i == jj ? 1.0 : 0.0) - sc * x.x, -sc * x.y);
    }
    if (tid == 0) s_bad = 0;
    grid.sync();
    for (int j = 0; j < n; ++j) {
        if (s_bad) {          // read after a barrier: the same value in every thread of the CTA
            grid.sync();
            grid.sync();
            continue;
        }
        double best = -1.0;
        int bi = j;
        for (int i = j + tid; i < n; i += DC_THREADS) {
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
        if (tid == 0) {
            best = red_v[0];
            bi = red_i[0];
            for (int q = 1; q < DC_THREADS / 32; ++q)
                if (red_v[q] > best || (red_v[q] == best && red_i[q] < bi)) { best = red_v[q]; bi = red_i[q]; }
            s_piv = bi;
            perm[j] = bi;
            if (!(best > 0.0) || !isfinite(best)) s_bad = 1;
        }
        __syncthreads();
        if (s_bad) {          // this frequency's CTAs all see the same pivot; the grid keeps going
            grid.sync();
            grid.sync();
            continue;
        }
        const int p = s_piv;
        for (int i = tid; i < n; i += DC_THREADS) {
            const int src = (i == j) ? p : (i == p ? j : i);
            colj[i] = A[(size_t)src * n + j];
        }
        for (int c = tid; c < n; c += DC_THREADS) rowj[c] = A[(size_t)p * n + c];
        __syncthreads();
        grid.sync();
        const double2 piv = colj[j];
        const double d = cabs2(piv);
        const double2 inv = make_double2(piv.x / d, -piv.y / d);
        // interchange rows j and p on this CTA's columns
        if (p != j)
            for (int c = c0 + tid; c < c1; c += DC_THREADS) A[(size_t)p * n + c] = A[(size_t)j * n + c];
        __syncthreads();
        // scaled pivot row on this CTA's columns (position j holds 1/pivot)
        for (int c = c0 + tid; c < c1; c += DC_THREADS) {
            const double2 v = (c == j) ? make_double2(1.0, 0.0) : rowj[c];
            const double2 r = make_double2(v.x * inv.x - v.y * inv.y, v.x * inv.y + v.y * inv.x);
            rowj[c] = r;
            A[(size_t)j * n + c] = r;
        }
        __syncthreads();
        for (long long e = tid; e < (long long)n * w; e += DC_THREADS) {
            const int i = (int)(e / w), c = c0 + (int)(e % w);
            if (i == j) continue;
            const double2 fi = colj[i];
            const double2 r = rowj[c];
            double2 a = (c == j) ? make_double2(0.0, 0.0) : A[(size_t)i * n + c];
            a.x -= fi.x * r.x - fi.y * r.y;
            a.y -= fi.x * r.y + fi.y * r.x;
            A[(size_t)i * n + c] = a;
        }
        grid.sync();
    }
    if (s_bad) {
        if (tid == 0 && pc == 0) atomicOr(err_flag, 1);
        return;
    }
    // undo the interchanges as column interchanges and scale by v^1/2, on this CTA's rows
    const int r0 = (int)((long long)n * pc / P), r1 = (int)((long long)n * (pc + 1) / P);
    for (int i = r0 + warp; i < r1; i += DC_THREADS / 32) {
        double2* row = A + (size_t)i * n;
        if (lane == 0)
            for (int jj = n - 1; jj >= 0; --jj) {
                const int q = perm[jj];
                if (q != jj) { const double2 t = row[jj]; row[jj] = row[q]; row[q] = t; }
            }
        __syncwarp();
        for (int c = lane; c < n; c += 32) {
            const double sc = vs[i] * vs[c];
            const double2 a = row[c];
            row[c] = make_double2(a.x * sc, a.y * sc);
        }
    }
}

cudaError_t launch_dyson(const double2* chi, const double* vs, int ng, int nf, double2* W, int* err_flag,
                         cudaStream_t st) {
    const size_t smem = (size_t)ng * (2 * sizeof(double2) + sizeof(int));
    {   // cooperative form over the whole GPU when it fits
        int dev = 0, nsm = 0, per_sm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaFuncSetAttribute(k_dyson_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dyson_coop, DC_THREADS, smem) == cudaSuccess &&
            per_sm > 0) {
            // frequencies per launch: as many as keep their matrices within ~96 MB of L2, since every
            // pivot step updates the whole of each matrix (rank one); the columns of a matrix are
            // split over P CTAs of at least 16 columns
            const size_t mat = (size_t)ng * ng * sizeof(double2);
            const int g = (int)std::max<size_t>(1, std::min<size_t>((size_t)nf, ((size_t)96 << 20) / mat));
            const int P = std::min(std::max(1, ng / 16), (per_sm * nsm) / g);
            if (P >= 2) {
                cudaError_t e = cudaSuccess;
                for (int f0 = 0; f0 < nf && e == cudaSuccess; f0 += g) {
                    const int fg = std::min(g, nf - f0);
                    int P_ = P, n_ = ng;
                    const double2* chi_ = chi + (size_t)f0 * ng * ng;
                    const double* vs_ = vs;
                    double2* W_ = W + (size_t)f0 * ng * ng;
                    int* err_ = err_flag;
                    void* args[] = {(void*)&chi_, (void*)&vs_, (void*)&n_, (void*)&P_, (void*)&W_, (void*)&err_};
                    e = cudaLaunchCooperativeKernel((const void*)k_dyson_coop, dim3(fg * P), dim3(DC_THREADS), args, smem,
                                                    st);
                    if (e != cudaSuccess && f0 > 0) return e;     // a group already ran: report, no fallback
                }
                if (e == cudaSuccess) return cudaSuccess;
                cudaGetLastError();
            }
        }
        cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(k_dyson, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_dyson<<<nf, DY_THREADS, smem, st>>>(chi, vs, ng, W, err_flag);
    return cudaGetLastError();
}

}  // namespace rp
