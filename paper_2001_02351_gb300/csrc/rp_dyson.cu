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

// a - f r as four fused multiply-adds (the FP64 pipe is the bound: no separate products or sums)
__device__ __forceinline__ double2 cfms(double2 a, double2 f, double2 r) {
    a.x = fma(-f.x, r.x, a.x);
    a.x = fma(f.y, r.y, a.x);
    a.y = fma(-f.x, r.y, a.y);
    a.y = fma(-f.y, r.x, a.y);
    return a;
}

// largest v (then smallest i) over the CTA; every thread gets the result (two barriers)
template <int NT>
__device__ __forceinline__ void block_argmax(double& v, int& i, double* red_v, int* red_i) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, v, off);
        const int oi = __shfl_down_sync(0xffffffffu, i, off);
        if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
    }
    if (lane == 0) { red_v[warp] = v; red_i[warp] = i; }
    __syncthreads();
    v = red_v[0];
    i = red_i[0];
    for (int q = 1; q < NT / 32; ++q)
        if (red_v[q] > v || (red_v[q] == v && red_i[q] < i)) { v = red_v[q]; i = red_i[q]; }
    __syncthreads();
}

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
        for (int i = tid / n, c = tid % n; i < n;) {
            if (i != j) {
                const double2 fi = colj[i];
                double2 a = (c == j) ? make_double2(0.0, 0.0) : A[(size_t)i * n + c];
                A[(size_t)i * n + c] = cfms(a, fi, rowj[c]);
            }
            i += DY_THREADS / n;
            c += DY_THREADS % n;
            if (c >= n) { c -= n; ++i; }
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


// Cooperative form: P CTAs per frequency (grid = frequencies of the launch * P, all resident), the
// columns of each matrix split evenly among its P CTAs.  Pivot j is published through global scratch
// by the CTA that owns column j: in step j - 1 it updates that column first, finds its pivot and
// writes the column and the pivot row index, then updates the rest of its columns; one grid barrier
// closes the step.  Every CTA then reads the column (coalesced), applies the interchange and the
// scaled pivot row to its own columns and eliminates them.  A zero or non-finite pivot is published
// as -1; the CTAs of that frequency keep passing the barriers (exactly n + 1 for every CTA, whatever
// the data) and skip the arithmetic.  Afterwards each CTA undoes the interchanges on its own rows as
// one column gather and scales by v^1/2.
#define DC_THREADS 512
#define DC_UNROLL 4

// CTA pc of the P CTAs of one matrix: X = chi (n x n), A = W, cb = [2][n] published columns, perm =
// [n] pivot rows then [2] published pivots.  nsteps >= n grid barriers after the first (a launch over
// matrices of several sizes runs the largest count; a smaller matrix passes the extra barriers idle).
__device__ __forceinline__ void dyson_coop_body(cooperative_groups::grid_group& grid, const double2* __restrict__ X,
                                                const double* __restrict__ vs, int n, int P, int pc,
                                                double2* __restrict__ A, double2* __restrict__ cb,
                                                int* __restrict__ perm, int nsteps, int* err_flag,
                                                unsigned char* smem) {
    double2* colj = (double2*)smem;        // column j after the interchange (all rows)
    double2* rowj = colj + n;              // scaled pivot row on this CTA's columns; a row in the undo
    int* idx = (int*)(rowj + n);           // column gather of the undo
    __shared__ double red_v[DC_THREADS / 32];
    __shared__ int red_i[DC_THREADS / 32];
    const int c0 = (int)((long long)n * pc / P), c1 = (int)((long long)n * (pc + 1) / P);
    const int w = c1 - c0;
    int* pivb = perm + n;
    const int tid = threadIdx.x;
    // element walk over this CTA's n x w block, row-major, without divisions in the loop
    const int di = DC_THREADS / w, dc = DC_THREADS % w;
    // eps = 1 - v^1/2 chi v^1/2 on this CTA's columns
    for (int i = tid / w, cc = tid % w; i < n;) {
        const int c = c0 + cc;
        const double sc = vs[i] * vs[c];
        const double2 x = X[(size_t)i * n + c];
        A[(size_t)i * n + c] = make_double2((i == c ? 1.0 : 0.0) - sc * x.x, -sc * x.y);
        i += di;
        cc += dc;
        if (cc >= w) { cc -= w; ++i; }
    }
    __syncthreads();
    if (c0 == 0) {       // owner of column 0 publishes it and its pivot
        double best = -1.0;
        int bi = 0;
        for (int i = tid; i < n; i += DC_THREADS) {
            const double2 a = A[(size_t)i * n];
            cb[i] = a;
            const double v = cabs2(a);
            if (v > best || (v == best && i < bi)) { best = v; bi = i; }
        }
        block_argmax<DC_THREADS>(best, bi, red_v, red_i);
        if (tid == 0) {
            perm[0] = bi;
            pivb[0] = (best > 0.0 && isfinite(best)) ? bi : -1;
        }
    }
    grid.sync();
    bool bad = false;                      // uniform over the CTA (read from the same published value)
    for (int j = 0; j < nsteps; ++j) {
        const int cur = j & 1, nxt = cur ^ 1;
        if (j < n && !bad) bad = __ldcg(&pivb[cur]) < 0;
        if (j < n && !bad) {
            const int p = __ldcg(&pivb[cur]);
            for (int i = tid; i < n; i += DC_THREADS) {
                const int src = (i == j) ? p : (i == p ? j : i);
                colj[i] = __ldcg(&cb[(size_t)cur * n + src]);
            }
            for (int c = c0 + tid; c < c1; c += DC_THREADS) rowj[c] = A[(size_t)p * n + c];
            __syncthreads();
            const double2 piv = colj[j];
            const double d = cabs2(piv);
            const double2 inv = make_double2(piv.x / d, -piv.y / d);
            // interchange rows j and p on this CTA's columns; row j becomes the scaled pivot row
            // (position j holds 1 / pivot)
            for (int c = c0 + tid; c < c1; c += DC_THREADS) {
                const double2 v = (c == j) ? make_double2(1.0, 0.0) : rowj[c];
                const double2 r = make_double2(v.x * inv.x - v.y * inv.y, v.x * inv.y + v.y * inv.x);
                if (p != j) A[(size_t)p * n + c] = A[(size_t)j * n + c];
                A[(size_t)j * n + c] = r;
                rowj[c] = r;
            }
            __syncthreads();
            const int jn = j + 1;
            const bool owner = jn < n && jn >= c0 && jn < c1;
            if (owner) {        // column j + 1 first: eliminate, publish, find its pivot
                const double2 r = rowj[jn];
                double best = -1.0;
                int bi = jn;
                for (int i = tid; i < n; i += DC_THREADS) {
                    double2 a;
                    if (i == j) {
                        a = r;
                    } else {
                        a = cfms(A[(size_t)i * n + jn], colj[i], r);
                        A[(size_t)i * n + jn] = a;
                    }
                    cb[(size_t)nxt * n + i] = a;
                    if (i >= jn) {
                        const double v = cabs2(a);
                        if (v > best || (v == best && i < bi)) { best = v; bi = i; }
                    }
                }
                block_argmax<DC_THREADS>(best, bi, red_v, red_i);
                if (tid == 0) {
                    perm[jn] = bi;
                    pivb[nxt] = (best > 0.0 && isfinite(best)) ? bi : -1;
                }
            }
            // the rest of this CTA's block, DC_UNROLL elements per thread in flight (their loads
            // issued before their arithmetic: the block streams from L2 or DRAM every step)
            for (int i = tid / w, cc = tid % w; i < n;) {
                int ei[DC_UNROLL], ec[DC_UNROLL];
                double2 a[DC_UNROLL];
#pragma unroll
                for (int u = 0; u < DC_UNROLL; ++u) {
                    const int c = c0 + cc;
                    const bool act = i < n && i != j && c != jn;
                    ei[u] = act ? i : -1;
                    ec[u] = c;
                    a[u] = (act && c != j) ? A[(size_t)i * n + c] : make_double2(0.0, 0.0);
                    i += di;
                    cc += dc;
                    if (cc >= w) { cc -= w; ++i; }
                }
#pragma unroll
                for (int u = 0; u < DC_UNROLL; ++u)
                    if (ei[u] >= 0) A[(size_t)ei[u] * n + ec[u]] = cfms(a[u], colj[ei[u]], rowj[ec[u]]);
            }
        }
        grid.sync();
    }
    if (bad) {
        if (tid == 0 && pc == 0) atomicOr(err_flag, 1);
        return;
    }
    // the row interchanges undone as column interchanges, last first, composed into one gather:
    // out[c] = row[idx[c]]
    int* pv = (int*)colj;
    for (int i = tid; i < n; i += DC_THREADS) {
        pv[i] = __ldcg(&perm[i]);
        idx[i] = i;
    }
    __syncthreads();
    if (tid == 0)
        for (int jj = n - 1; jj >= 0; --jj) {
            const int q = pv[jj];
            const int t = idx[jj];
            idx[jj] = idx[q];
            idx[q] = t;
        }
    __syncthreads();
    const int r0 = (int)((long long)n * pc / P), r1 = (int)((long long)n * (pc + 1) / P);
    for (int i = r0; i < r1; ++i) {
        double2* row = A + (size_t)i * n;
        for (int c = tid; c < n; c += DC_THREADS) rowj[c] = __ldcg(&row[c]);
        __syncthreads();
        const double vi = vs[i];
        for (int c = tid; c < n; c += DC_THREADS) {
            const double sc = vi * vs[c];
            const double2 a = rowj[idx[c]];
            row[c] = make_double2(a.x * sc, a.y * sc);
        }
        __syncthreads();
    }
}

// Hermitian positive definite eps (chi0 Hermitian and negative semidefinite, as on the imaginary
// axis): the sweep operator on the lower triangle, no pivoting.  Sweeping k maps d = A_kk,
// c = column k (c_i = A_ik, Hermitian: A_kj = conj(c_j)) to
//   A_kk = -1/d,   A_ik = c_i / d,   A_kj = conj(c_j) / d,   A_ij -= c_i conj(c_j) / d  (i, j != k),
// which keeps the matrix Hermitian; after all n sweeps it holds -eps^-1, so W = -v^1/2 A v^1/2.
// Half the flops of Gauss-Jordan (the lower triangle only).  The columns are split among the P CTAs
// by equal element counts of the lower triangle.  Column k of step k is published by every CTA
// (row k of its own columns, conjugated) and by the owner of column k (its part from the diagonal
// down) after the CTA's update of step k - 1; one grid barrier closes each step (n + 1 in all,
// whatever the data).  A pivot d that is not positive and finite (eps not positive definite) marks
// the matrix bad: its CTAs skip the arithmetic and the flag is raised.
__device__ __forceinline__ int herm_split(int n, int P, int p) {
    // smallest c with (elements of columns 0 .. c-1 of the lower triangle) >= p / P of all
    const long long total = (long long)n * (n + 1) / 2;
    const long long target = total * p / P;
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) / 2;
        const long long el = (long long)mid * n - (long long)mid * (mid - 1) / 2;
        if (el >= target) hi = mid; else lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ void dyson_herm_body(cooperative_groups::grid_group& grid, const double2* __restrict__ X,
                                                const double* __restrict__ vs, int n, int P, int pc,
                                                double2* __restrict__ A, double2* __restrict__ cb, int nsteps,
                                                int* err_flag, unsigned char* smem) {
    double2* cc = (double2*)smem;          // column k of the step (all rows)
    double2* uu = cc + n;                  // c_i / d
    const int c0 = herm_split(n, P, pc), c1 = herm_split(n, P, pc + 1);
    const int w = c1 - c0;
    const int tid = threadIdx.x;
    // this CTA's block: rows c0 .. n-1 of its columns (entries above the diagonal skipped)
    const int di = w > 0 ? DC_THREADS / w : 0, dc = w > 0 ? DC_THREADS % w : 0;
    if (w > 0)
        for (int i = c0 + tid / w, cq = tid % w; i < n;) {
            const int j = c0 + cq;
            if (j <= i) {
                const double sc = vs[i] * vs[j];
                const double2 x = X[(size_t)i * n + j];
                A[(size_t)i * n + j] = make_double2((i == j ? 1.0 : 0.0) - sc * x.x, -sc * x.y);
            }
            i += di;
            cq += dc;
            if (cq >= w) { cq -= w; ++i; }
        }
    __syncthreads();
    if (c0 == 0 && w > 0)                  // column 0 for step 0
        for (int i = tid; i < n; i += DC_THREADS) cb[i] = A[(size_t)i * n];
    grid.sync();
    bool bad = false;
    for (int k = 0; k < nsteps; ++k) {
        const int cur = k & 1, nxt = cur ^ 1;
        if (k < n && !bad) {
            for (int i = tid; i < n; i += DC_THREADS) cc[i] = __ldcg(&cb[(size_t)cur * n + i]);
            __syncthreads();
            const double d = cc[k].x;
            if (!(d > 0.0) || !isfinite(d)) bad = true;        // the same value in every CTA of the matrix
        }
        if (k < n && !bad) {
            const double inv = 1.0 / cc[k].x;
            for (int i = tid; i < n; i += DC_THREADS) uu[i] = make_double2(cc[i].x * inv, cc[i].y * inv);
            __syncthreads();
            // the update of one lower-triangle entry (old value a where it is read)
            auto upd = [&](int ii, int jj, double2 a) {
                double2 v;
                if (ii == k && jj == k) v = make_double2(-inv, 0.0);
                else if (ii == k) v = make_double2(uu[jj].x, -uu[jj].y);          // conj(c_j) / d
                else if (jj == k) v = uu[ii];                                      // c_i / d
                else v = cfms(a, uu[ii], make_double2(cc[jj].x, -cc[jj].y));       // - c_i conj(c_j) / d
                A[(size_t)ii * n + jj] = v;
            };
            // rows c1 .. n-1: the full width of this CTA's columns
            if (w > 0 && c1 < n)
                for (int i = c1 + tid / w, cq = tid % w; i < n;) {
                    int ei[DC_UNROLL], ej[DC_UNROLL];
                    double2 a[DC_UNROLL];
#pragma unroll
                    for (int q = 0; q < DC_UNROLL; ++q) {
                        const int j = c0 + cq;
                        ei[q] = i < n ? i : -1;
                        ej[q] = j;
                        a[q] = (i < n && i != k && j != k) ? A[(size_t)i * n + j] : make_double2(0.0, 0.0);
                        i += di;
                        cq += dc;
                        if (cq >= w) { cq -= w; ++i; }
                    }
#pragma unroll
                    for (int q = 0; q < DC_UNROLL; ++q)
                        if (ei[q] >= 0) upd(ei[q], ej[q], a[q]);
                }
            // rows c0 .. c1-1: the triangle j <= i, entry e = r (r + 1) / 2 + (j - c0) for row c0 + r
            {
                const int T = w * (w + 1) / 2;
                for (int e0 = tid; e0 < T; e0 += DC_UNROLL * DC_THREADS) {
                    int ei[DC_UNROLL], ej[DC_UNROLL];
                    double2 a[DC_UNROLL];
#pragma unroll
                    for (int q = 0; q < DC_UNROLL; ++q) {
                        const int e = e0 + q * DC_THREADS;
                        ei[q] = -1;
                        ej[q] = 0;
                        a[q] = make_double2(0.0, 0.0);
                        if (e < T) {
                            int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
                            while (r > 0 && r * (r + 1) / 2 > e) --r;
                            while ((r + 1) * (r + 2) / 2 <= e) ++r;
                            const int i = c0 + r, j = c0 + (e - r * (r + 1) / 2);
                            ei[q] = i;
                            ej[q] = j;
                            if (i != k && j != k) a[q] = A[(size_t)i * n + j];
                        }
                    }
#pragma unroll
                    for (int q = 0; q < DC_UNROLL; ++q)
                        if (ei[q] >= 0) upd(ei[q], ej[q], a[q]);
                }
            }
            __syncthreads();
            // publish column k + 1: row k + 1 of this CTA's columns left of it (conjugated), and the
            // owner of column k + 1 its entries from the diagonal down
            const int kn = k + 1;
            if (kn < n) {
                for (int j = c0 + tid; j < c1 && j < kn; j += DC_THREADS) {
                    const double2 v = A[(size_t)kn * n + j];
                    cb[(size_t)nxt * n + j] = make_double2(v.x, -v.y);
                }
                if (kn >= c0 && kn < c1)
                    for (int i = kn + tid; i < n; i += DC_THREADS) cb[(size_t)nxt * n + i] = A[(size_t)i * n + kn];
            }
        }
        grid.sync();
    }
    if (bad) {
        if (tid == 0 && pc == 0) atomicOr(err_flag, 1);
        return;
    }
    // W = -v^1/2 A v^1/2 on this CTA's columns, both triangles (the upper one from the lower)
    if (w > 0)
        for (int i = c0 + tid / w, cq = tid % w; i < n;) {
            const int j = c0 + cq;
            if (j <= i) {
                const double sc = -vs[i] * vs[j];
                const double2 a = A[(size_t)i * n + j];
                const double2 v = make_double2(a.x * sc, a.y * sc);
                A[(size_t)i * n + j] = v;
                if (i != j) A[(size_t)j * n + i] = make_double2(v.x, -v.y);
            }
            i += di;
            cq += dc;
            if (cq >= w) { cq -= w; ++i; }
        }
}

__global__ void __launch_bounds__(DC_THREADS) k_dyson_coop(const double2* __restrict__ chi,
                                                           const double* __restrict__ vs, int n, int P,
                                                           double2* __restrict__ Wout,
                                                           double2* __restrict__ colbuf, int* __restrict__ ibuf,
                                                           int herm, int* err_flag) {
    cooperative_groups::grid_group grid = cooperative_groups::this_grid();
    extern __shared__ unsigned char smem[];
    const int f = blockIdx.x / P, pc = blockIdx.x % P;
    if (herm) {
        dyson_herm_body(grid, chi + (size_t)f * n * n, vs, n, P, pc, Wout + (size_t)f * n * n,
                        colbuf + (size_t)f * 2 * n, n, err_flag, smem);
        return;
    }
    dyson_coop_body(grid, chi + (size_t)f * n * n, vs, n, P, pc, Wout + (size_t)f * n * n, colbuf + (size_t)f * 2 * n,
                    ibuf + (size_t)f * (n + 2), n, err_flag, smem);
}

// matrices of several sizes in one cooperative launch (the (q, w) members of a batch): CTA b works
// on matrix map[b].x as its CTA map[b].y; every CTA passes nsteps = the largest n barriers
__global__ void __launch_bounds__(DC_THREADS) k_dyson_list(const DysonMat* __restrict__ mats,
                                                           const int2* __restrict__ map, int nsteps, int herm,
                                                           int* err_flag) {
    cooperative_groups::grid_group grid = cooperative_groups::this_grid();
    extern __shared__ unsigned char smem[];
    const int2 mp = map[blockIdx.x];
    const DysonMat m = mats[mp.x];
    if (herm) {
        dyson_herm_body(grid, m.chi, m.vs, m.n, m.P, mp.y, m.W, m.cb, nsteps, err_flag, smem);
        return;
    }
    dyson_coop_body(grid, m.chi, m.vs, m.n, m.P, mp.y, m.W, m.cb, m.ib, nsteps, err_flag, smem);
}

int dyson_list_slots(int nmax) {
    const size_t smem = (size_t)nmax * (2 * sizeof(double2) + sizeof(int));
    int dev = 0, nsm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(k_dyson_list, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dyson_list, DC_THREADS, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * nsm;
}

cudaError_t launch_dyson_list(const DysonMat* d_mats, const int2* d_map, int nblocks, int nmax, bool herm,
                              int* err_flag, cudaStream_t st) {
    const size_t smem = (size_t)nmax * (2 * sizeof(double2) + sizeof(int));
    cudaError_t e = cudaFuncSetAttribute(k_dyson_list, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nsteps = nmax, hm = herm ? 1 : 0;
    void* args[] = {(void*)&d_mats, (void*)&d_map, (void*)&nsteps, (void*)&hm, (void*)&err_flag};
    return cudaLaunchCooperativeKernel((const void*)k_dyson_list, dim3(nblocks), dim3(DC_THREADS), args, smem, st);
}

size_t dyson_scratch_bytes(int ng, int nf) {
    const size_t cols = (size_t)nf * 2 * ng * sizeof(double2);
    return ((cols + 255) / 256) * 256 + (size_t)nf * (ng + 2) * sizeof(int);
}

cudaError_t launch_dyson(const double2* chi, const double* vs, int ng, int nf, double2* W, void* scratch,
                         bool herm, int* err_flag, cudaStream_t st) {
    const size_t smem = (size_t)ng * (2 * sizeof(double2) + sizeof(int));
    {   // cooperative form over the whole GPU when it fits
        int dev = 0, nsm = 0, per_sm = 0;
        if (scratch && cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaFuncSetAttribute(k_dyson_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dyson_coop, DC_THREADS, smem) == cudaSuccess &&
            per_sm > 0) {
            // every frequency in one launch when each can have two CTAs; CTAs as many as are resident,
            // so that every SM holds (nearly) the same number of equal column blocks (the FP64 pipe
            // is the bound), and at least 8 columns per CTA
            const int slots = per_sm * nsm;
            const int g = std::max(1, std::min(nf, slots / 2));
            const int pmax = ng / 8;
            if (pmax >= 2) {
                double2* cb_all = (double2*)scratch;
                int* ib_all = (int*)((char*)scratch + (((size_t)nf * 2 * ng * sizeof(double2) + 255) / 256) * 256);
                cudaError_t e = cudaSuccess;
                for (int f0 = 0; f0 < nf && e == cudaSuccess; f0 += g) {
                    const int fg = std::min(g, nf - f0);
                    int P_ = std::min(pmax, slots / fg), n_ = ng;
                    const double2* chi_ = chi + (size_t)f0 * ng * ng;
                    const double* vs_ = vs;
                    double2* W_ = W + (size_t)f0 * ng * ng;
                    double2* cb_ = cb_all + (size_t)f0 * 2 * ng;
                    int* ib_ = ib_all + (size_t)f0 * (ng + 2);
                    int* err_ = err_flag;
                    int hm = herm ? 1 : 0;
                    void* args[] = {(void*)&chi_, (void*)&vs_, (void*)&n_, (void*)&P_, (void*)&W_,
                                    (void*)&cb_, (void*)&ib_, (void*)&hm, (void*)&err_};
                    e = cudaLaunchCooperativeKernel((const void*)k_dyson_coop, dim3(fg * P_), dim3(DC_THREADS), args,
                                                    smem, st);
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
