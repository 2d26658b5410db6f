// Host side of the C ABI: validation, the per-q plan, scratch management and the
// order of kernel launches for each entry point.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <vector>

#include "rp_internal.h"

namespace rp {

int fail(rp_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(rp_ctx* c, cudaError_t e, const char* where) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    return fail(c, e == cudaErrorMemoryAllocation ? RP_ERR_OOM : RP_ERR_CUDA, buf);
}

void prof_begin(rp_ctx* c, int stage, cudaStream_t st) {
    if (!c->prof) return;
    std::vector<cudaEvent_t>& v = c->prof_ev[stage];
    const int i = 2 * c->prof_used[stage];
    while ((int)v.size() < i + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        v.push_back(e);
    }
    cudaEventRecord(v[i], st);
}

void prof_end(rp_ctx* c, int stage, cudaStream_t st, int launches) {
    c->prof_launches[stage] += launches;
    if (!c->prof) return;
    std::vector<cudaEvent_t>& v = c->prof_ev[stage];
    const int i = 2 * c->prof_used[stage];
    if ((int)v.size() < i + 2) return;
    cudaEventRecord(v[i + 1], st);
    c->prof_used[stage]++;
}

void release(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

int ensure(rp_ctx* c, DevBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return RP_OK;
    release(b);
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        char buf[128];
        snprintf(buf, sizeof(buf), "device allocation of %zu bytes failed", bytes);
        return fail(c, RP_ERR_OOM, buf);
    }
    b.bytes = bytes;
    return RP_OK;
}

static int upload(rp_ctx* c, DevBuf& b, const void* src, size_t bytes) {
    int s = ensure(c, b, bytes);
    if (s) return s;
    cudaError_t e = cudaMemcpy(b.p, src, bytes, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? RP_OK : cuda_fail(c, e, "upload");
}

static bool good_fft(int n) {
    if (n < 4 || n > 128) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

static void cart(const rp_ctx* c, const double f[3], double out[3]) {
    for (int x = 0; x < 3; ++x) out[x] = f[0] * c->recip[0 * 3 + x] + f[1] * c->recip[1 * 3 + x] + f[2] * c->recip[2 * 3 + x];
}

static double half_norm2(const rp_ctx* c, const double q[3], int m1, int m2, int m3) {
    double f[3] = {q[0] + m1, q[1] + m2, q[2] + m3}, v[3];
    cart(c, f, v);
    return 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
}

static void search_box(const rp_ctx* c, double ecut, const double q[3], int nmax[3]) {
    for (int i = 0; i < 3; ++i) {
        double alen = std::sqrt(c->lat[i * 3] * c->lat[i * 3] + c->lat[i * 3 + 1] * c->lat[i * 3 + 1] + c->lat[i * 3 + 2] * c->lat[i * 3 + 2]);
        nmax[i] = (int)std::floor(std::sqrt(2.0 * ecut) * alen / (2.0 * M_PI) + std::fabs(q[i])) + 1;
    }
}

int plan_q(rp_ctx* c, const double q[3]) { return plan_q_cut(c, q, c->ecut_eps); }

int plan_q_cut(rp_ctx* c, const double q[3], double ecut_eps, bool exact) {
    QPlan& P = c->plan;
    if (P.valid && P.q[0] == q[0] && P.q[1] == q[1] && P.q[2] == q[2] && P.ecut == ecut_eps && P.exact == exact)
        return RP_OK;
    P.valid = false;
    if (!(ecut_eps > 0.0) || !(ecut_eps <= c->ecut_psi)) return fail(c, RP_ERR_ARG, "need 0 < Ecut_eps <= Ecut_psi");
    for (int i = 0; i < 3; ++i) {
        if (!std::isfinite(q[i]) || !(std::fabs(q[i]) < 1.0)) return fail(c, RP_ERR_ARG, "q must be finite with |q_i| < 1");
        double v = q[i] * c->kmesh[i];
        long long r = llround(v);
        if (std::fabs(v - (double)r) > 1e-9) return fail(c, RP_ERR_ARG, "q is not a vector of the k mesh");
        P.qi[i] = (int)r;
    }
    // epsilon sphere and tail, lexicographic Miller order
    P.gm.clear(); P.tail.clear(); P.vs.clear(); P.tailv.clear();
    int nmax[3];
    search_box(c, c->ecut_psi, q, nmax);
    const double fourpi_om = 4.0 * M_PI / c->omega;
    for (int m1 = -nmax[0]; m1 <= nmax[0]; ++m1)
        for (int m2 = -nmax[1]; m2 <= nmax[1]; ++m2)
            for (int m3 = -nmax[2]; m3 <= nmax[2]; ++m3) {
                double e = half_norm2(c, q, m1, m2, m3);
                if (e <= ecut_eps && e > 1e-14) {
                    P.gm.push_back(m1); P.gm.push_back(m2); P.gm.push_back(m3);
                    P.vs.push_back(std::sqrt(fourpi_om / (2.0 * e)));
                } else if (e > ecut_eps && e <= c->ecut_psi) {
                    P.tail.push_back(m1); P.tail.push_back(m2); P.tail.push_back(m3);
                    P.tailv.push_back(fourpi_om / (2.0 * e));
                }
            }
    P.ng = (int)P.vs.size();
    P.ntail = (int)P.tailv.size();
    if (P.ng == 0) return fail(c, RP_ERR_ARG, "empty epsilon sphere");
    // umklapp map
    const int n2 = c->kmesh[1], n3 = c->kmesh[2];
    P.kp.assign(c->nk, 0);
    P.g0.assign(3 * c->nk, 0);
    for (int k = 0; k < c->nk; ++k) {
        int i[3] = {k / (n2 * n3), (k / n3) % n2, k % n3};
        int j[3], kk[3];
        for (int a = 0; a < 3; ++a) {
            j[a] = i[a] + P.qi[a];
            int n = c->kmesh[a];
            int g = (j[a] >= 0) ? j[a] / n : -((-j[a] + n - 1) / n);
            P.g0[3 * k + a] = g;
            kk[a] = j[a] - g * n;
        }
        P.kp[k] = (kk[0] * n2 + kk[1]) * n3 + kk[2];
    }
    // index sets of the pruned forward transforms
    P.gpos.assign(3 * P.ng, 0);
    for (int a = 0; a < 3; ++a) {
        std::set<int> s;
        for (int g = 0; g < P.ng; ++g) s.insert(P.gm[3 * g + a]);
        P.setv[a].assign(s.begin(), s.end());
        P.nset[a] = (int)P.setv[a].size();
        for (int g = 0; g < P.ng; ++g)
            P.gpos[3 * g + a] = (int)(std::lower_bound(P.setv[a].begin(), P.setv[a].end(), P.gm[3 * g + a]) - P.setv[a].begin());
    }
    // Transform grid.  The product conj(u_a) u_o has Miller components within
    // +-(2 mu + 1) per axis (mu: largest |m| of the bands; the empty band is shifted by -G0, |G0_i|
    // <= 1) and is read back at |g| <= Lg; on any grid with N >= 2 mu + 2 + Lg no other component
    // of the product folds onto a sphere value, so the transforms give the convolution of Eq. ism
    // exactly.  A cubic requested grid larger than that is replaced by the smallest of the
    // transform sizes with dedicated kernels that qualifies; otherwise (including a requested
    // grid that folds) the requested grid is used as given.
    for (int a = 0; a < 3; ++a) P.nfft[a] = c->fft[a];
    if (c->lb > 0 && c->fft[0] == c->fft[1] && c->fft[1] == c->fft[2]) {
        int need = 0;
        for (int a = 0; a < 3; ++a) {
            int lg = 0;
            for (int v : P.setv[a]) lg = std::max(lg, std::abs(v));
            need = std::max(need, 2 * c->mu[a] + 2 + lg);
        }
        for (int cand : {16, 24, 32, 48})
            if (cand >= need && cand < c->fft[0]) {
                for (int a = 0; a < 3; ++a) P.nfft[a] = cand;
                break;
            }
    }
    if (exact && c->lb > 0) {
        // a grid on which the transforms are the plain convolution: the requested one if nothing folds
        // onto the sphere there, else the smallest size (of 2s and 3s) on which nothing does
        int need = 0;
        for (int a = 0; a < 3; ++a) {
            int lg = 0;
            for (int v : P.setv[a]) lg = std::max(lg, std::abs(v));
            need = std::max(need, 2 * c->mu[a] + 2 + lg);
        }
        if (P.nfft[0] < need || P.nfft[1] < need || P.nfft[2] < need) {
            int n = need;
            while (!good_fft(n)) ++n;
            if (n > 128) return fail(c, RP_ERR_UNSUPPORTED, "exact transform grid above 128");
            for (int a = 0; a < 3; ++a) P.nfft[a] = n;
        }
    }
    P.nr = (long long)P.nfft[0] * P.nfft[1] * P.nfft[2];
    for (int a = 0; a < 3; ++a) {
        // forward phases exp(+2 pi i g x / N): the matrix element of Eq. ism carries e^{+iG.r}
        const int N = P.nfft[a];
        std::vector<double> e(2 * P.nset[a] * N);
        std::vector<float> e32(2 * P.nset[a] * N);
        for (int s_ = 0; s_ < P.nset[a]; ++s_)
            for (int x = 0; x < N; ++x) {
                long long ph = ((long long)P.setv[a][s_] * x) % N;
                if (ph < 0) ph += N;
                double ang = 2.0 * M_PI * (double)ph / (double)N;
                e[2 * (s_ * N + x)] = std::cos(ang);
                e[2 * (s_ * N + x) + 1] = std::sin(ang);
                e32[2 * (s_ * N + x)] = (float)std::cos(ang);
                e32[2 * (s_ * N + x) + 1] = (float)std::sin(ang);
            }
        int st = upload(c, P.d_efwd[a], e.data(), e.size() * sizeof(double));
        if (st) return st;
        st = upload(c, P.d_efwd32[a], e32.data(), e32.size() * sizeof(float));
        if (st) return st;
    }
    // residue maps of the line transforms (sphere index of each transform output, or -1)
    P.fused = true;
    for (int a = 1; a < 3; ++a) {
        const int N = P.nfft[a];
        int st_;
        {
            std::vector<int> map(N, -1);
            for (int s_ = 0; s_ < P.nset[a]; ++s_) {
                int r = ((P.setv[a][s_] % N) + N) % N;
                if (map[r] >= 0) P.fused = false;     // two sphere values on one residue (aliasing)
                map[r] = s_;
            }
            if ((st_ = upload(c, a == 2 ? P.d_zmap : P.d_ymap, map.data(), N * sizeof(int)))) return st_;
        }
    }
    // residue masks and residue-ordered sphere positions (plane-wise pair kernels)
    P.masks = P.fused && P.nfft[1] <= 32 && P.nfft[2] <= 32;
    P.ymask = P.zmask = 0;
    std::vector<int> gpos_r(P.gpos);
    if (P.masks) {
        for (int a = 1; a < 3; ++a) {
            const int N = P.nfft[a];
            unsigned m = 0;
            for (int s_ = 0; s_ < P.nset[a]; ++s_) m |= 1u << (((P.setv[a][s_] % N) + N) % N);
            (a == 1 ? P.ymask : P.zmask) = m;
            for (int g = 0; g < P.ng; ++g) {
                const int r = ((P.gm[3 * g + a] % N) + N) % N;
                gpos_r[3 * g + a] = __builtin_popcount(m & ((1u << r) - 1u));
            }
        }
    }
    // symmetric window for the FP32 pair kernels (cubic grids): the narrowest built half-width
    // that holds every component of the sphere
    P.zyw = 0;
    std::vector<int> gpos_w(P.gpos), colg;
    if (P.fused && P.nfft[0] == P.nfft[1] && P.nfft[1] == P.nfft[2]) {
        int m = 0;
        for (int g = 0; g < 3 * P.ng; ++g) m = std::max(m, std::abs(P.gm[g]));
        P.zyw = zy_window(P.nfft[1], m);
        if (P.zyw > 0) {
            const int W = P.zyw, NW = 2 * W + 1;
            colg.assign((size_t)NW * NW * NW, -1);
            for (int g = 0; g < P.ng; ++g) {
                gpos_w[3 * g + 1] = P.gm[3 * g + 1] + W;
                gpos_w[3 * g + 2] = P.gm[3 * g + 2] + W;
                colg[(size_t)(P.gm[3 * g] + W) * NW * NW + (P.gm[3 * g + 1] + W) * NW + P.gm[3 * g + 2] + W] = g;
            }
        }
    }
    int st;
    // inverse-transform phases exp(+2 pi i m x / N) for m = -lb..lb (Eq. pak on the grid)
    if (c->lb > 0) {
        const int B = 2 * c->lb + 1;
        for (int a = 0; a < 3; ++a) {
            const int N = P.nfft[a];
            std::vector<double> e(2 * (size_t)N * B);
            std::vector<float> e32(2 * (size_t)N * B);
            for (int x = 0; x < N; ++x)
                for (int mi = 0; mi < B; ++mi) {
                    long long ph = ((long long)(mi - c->lb) * x) % N;
                    if (ph < 0) ph += N;
                    double ang = 2.0 * M_PI * (double)ph / (double)N;
                    e[2 * ((size_t)x * B + mi)] = std::cos(ang);
                    e[2 * ((size_t)x * B + mi) + 1] = std::sin(ang);
                    e32[2 * ((size_t)x * B + mi)] = (float)std::cos(ang);
                    e32[2 * ((size_t)x * B + mi) + 1] = (float)std::sin(ang);
                }
            if ((st = upload(c, P.d_einv[a], e.data(), e.size() * sizeof(double)))) return st;
            if ((st = upload(c, P.d_einv32[a], e32.data(), e32.size() * sizeof(float)))) return st;
        }
    }
    if ((st = upload(c, P.d_gpos_r, gpos_r.data(), gpos_r.size() * sizeof(int)))) return st;
    if ((st = upload(c, P.d_gpos_w, gpos_w.data(), gpos_w.size() * sizeof(int)))) return st;
    if (!colg.empty() && (st = upload(c, P.d_colg, colg.data(), colg.size() * sizeof(int)))) return st;
    if ((st = upload(c, P.d_gpos, P.gpos.data(), P.gpos.size() * sizeof(int)))) return st;
    if ((st = upload(c, P.d_kp, P.kp.data(), P.kp.size() * sizeof(int)))) return st;
    if ((st = upload(c, P.d_g0, P.g0.data(), P.g0.size() * sizeof(int)))) return st;
    if ((st = upload(c, P.d_vs, P.vs.data(), P.vs.size() * sizeof(double)))) return st;
    for (int i = 0; i < 3; ++i) P.q[i] = q[i];
    P.ecut = ecut_eps;
    P.exact = exact;
    P.valid = true;
    return RP_OK;
}

// Six tetrahedra per sub-cell sharing the shortest main diagonal (Eq. tetrahedron reading).
static void build_tetrahedra(rp_ctx* c) {
    const int n[3] = {c->kmesh[0], c->kmesh[1], c->kmesh[2]};
    const int starts[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    int best = 0;
    double best_len = 1e300;
    for (int s = 0; s < 4; ++s) {
        double f[3], v[3];
        for (int a = 0; a < 3; ++a) f[a] = (1.0 - 2.0 * starts[s][a]) / n[a];
        cart(c, f, v);
        double len = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (len < best_len * (1.0 - 1e-12)) { best_len = len; best = s; }
    }
    // paths 0 -> e_i -> e_i + e_j -> (1,1,1) over the 6 axis orders, reflected onto the diagonal
    const int order[6][2] = {{0, 1}, {0, 2}, {1, 0}, {1, 2}, {2, 0}, {2, 1}};
    int off[6][4][3];
    for (int t = 0; t < 6; ++t) {
        int v[4][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {1, 1, 1}};
        v[1][order[t][0]] = 1;
        v[2][order[t][0]] = 1;
        v[2][order[t][1]] = 1;
        for (int p = 0; p < 4; ++p)
            for (int a = 0; a < 3; ++a) off[t][p][a] = starts[best][a] ? 1 - v[p][a] : v[p][a];
    }
    c->tets.assign(24 * c->nk, 0);
    c->tetk.assign(24 * c->nk, -1);
    std::vector<int> fill(c->nk, 0);
    int t_index = 0;
    for (int i1 = 0; i1 < n[0]; ++i1)
        for (int i2 = 0; i2 < n[1]; ++i2)
            for (int i3 = 0; i3 < n[2]; ++i3)
                for (int t = 0; t < 6; ++t, ++t_index)
                    for (int p = 0; p < 4; ++p) {
                        int j1 = (i1 + off[t][p][0]) % n[0], j2 = (i2 + off[t][p][1]) % n[1], j3 = (i3 + off[t][p][2]) % n[2];
                        int k = (j1 * n[1] + j2) * n[2] + j3;
                        c->tets[4 * t_index + p] = k;
                        c->tetk[24 * k + fill[k]++] = 4 * t_index + p;
                    }
}

}  // namespace rp

using namespace rp;

extern "C" {

int rp_setup_cell(const double lat[9], const int kmesh[3], const int fft[3], double ecut_psi_ha,
                  double ecut_eps_ha, rp_ctx** out) {
    if (!out || !lat || !kmesh || !fft) return RP_ERR_ARG;
    *out = nullptr;
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(lat[i])) return RP_ERR_ARG;
    for (int i = 0; i < 3; ++i) {
        if (kmesh[i] < 1 || kmesh[i] > 64) return RP_ERR_ARG;
        if (!good_fft(fft[i])) return RP_ERR_ARG;
    }
    if (!(ecut_eps_ha > 0) || !(ecut_psi_ha >= ecut_eps_ha) || !std::isfinite(ecut_psi_ha)) return RP_ERR_ARG;
    rp_ctx* c = new (std::nothrow) rp_ctx();
    if (!c) return RP_ERR_OOM;
    std::memcpy(c->lat, lat, sizeof(c->lat));
    const double* a = lat;
    double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) + a[2] * (a[3] * a[7] - a[4] * a[6]);
    if (!(std::fabs(det) > 1e-12)) { delete c; return RP_ERR_ARG; }
    c->omega = std::fabs(det);
    // b_i = 2 pi (a_j x a_k) / det  (rows), so that a_i . b_j = 2 pi delta_ij
    const double* a1 = a; const double* a2 = a + 3; const double* a3 = a + 6;
    double* b = c->recip;
    auto crossv = [](const double* u, const double* v, double* w) {
        w[0] = u[1] * v[2] - u[2] * v[1]; w[1] = u[2] * v[0] - u[0] * v[2]; w[2] = u[0] * v[1] - u[1] * v[0]; };
    crossv(a2, a3, b); crossv(a3, a1, b + 3); crossv(a1, a2, b + 6);
    for (int i = 0; i < 9; ++i) b[i] *= 2.0 * M_PI / det;
    for (int i = 0; i < 3; ++i) { c->kmesh[i] = kmesh[i]; c->fft[i] = fft[i]; }
    c->nk = kmesh[0] * kmesh[1] * kmesh[2];
    c->nr = (long long)fft[0] * fft[1] * fft[2];
    c->ecut_psi = ecut_psi_ha;
    c->ecut_eps = ecut_eps_ha;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) { delete c; return RP_ERR_CUDA; }
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        delete c;
        return RP_ERR_CUDA;
    }
    if (ensure(c, c->d_err, 16 * sizeof(int)) || cudaMemset(c->d_err.p, 0, 16 * sizeof(int)) != cudaSuccess) {
        delete c;
        return RP_ERR_OOM;
    }
    *out = c;
    return RP_OK;
}

int rp_load_bands(rp_ctx* c, int nk, int nband, int nocc, const int* npw, int npw_max, const int* miller,
                  const double* coef, const double* energy_ha, const double* T) {
    if (!c) return RP_ERR_ARG;
    if (nk != c->nk) return fail(c, RP_ERR_ARG, "nk does not match the k mesh");
    if (nocc < 1 || nband <= nocc) return fail(c, RP_ERR_ARG, "need 1 <= nocc < nband");
    if (!npw || !miller || !coef || !energy_ha || npw_max < nband) return fail(c, RP_ERR_ARG, "bad band arrays");
    int maxm = 0, mu[3] = {0, 0, 0};
    // grid point -> (k + 1) of the last k whose sphere holds it: no clearing between k points
    std::vector<int> mark((size_t)c->nr, 0);
    for (int k = 0; k < nk; ++k) {
        if (npw[k] < nband || npw[k] > npw_max) return fail(c, RP_ERR_ARG, "npw out of range");
        for (int p = 0; p < npw[k]; ++p) {
            long long idx = 0;
            for (int a = 0; a < 3; ++a) {
                const int m = miller[((size_t)k * npw_max + p) * 3 + a], n = c->fft[a];
                maxm = std::max(maxm, std::abs(m));
                mu[a] = std::max(mu[a], std::abs(m));
                int w = m < 0 ? m + n : m;                   // residue of m modulo n when |m| < n
                if (w < 0 || w >= n) w = ((m % n) + n) % n;
                idx = idx * n + w;
            }
            if (mark[idx] == k + 1) return fail(c, RP_ERR_ARG, "wave-function sphere does not fit the FFT grid");
            mark[idx] = k + 1;
        }
    }
    for (long long i = 0; i < (long long)nk * nband; ++i) {
        if (!std::isfinite(energy_ha[i])) return fail(c, RP_ERR_ARG, "energy not finite");
        if (T && !(T[i] >= 0.0 && T[i] <= 1.0)) return fail(c, RP_ERR_ARG, "T outside [0,1]");
    }
    c->loaded = false;
    c->plan.valid = false;
    c->nband = nband; c->nocc = nocc; c->nemp = nband - nocc; c->npw_max = npw_max;
    c->lb = maxm + 1;
    for (int a = 0; a < 3; ++a) c->mu[a] = mu[a];
    if (2 * c->lb + 1 > 4 * std::max(c->fft[0], std::max(c->fft[1], c->fft[2])))
        return fail(c, RP_ERR_ARG, "Miller indices too large for the grid");
    c->npw.assign(npw, npw + nk);
    c->miller.assign(miller, miller + (size_t)nk * npw_max * 3);
    c->energy.assign(energy_ha, energy_ha + (size_t)nk * nband);
    if (T) c->T.assign(T, T + (size_t)nk * nband); else c->T.clear();
    int st;
    if ((st = upload(c, c->d_coef, coef, (size_t)nk * nband * npw_max * 2 * sizeof(double)))) return st;
    if ((st = upload(c, c->d_miller, miller, (size_t)nk * npw_max * 3 * sizeof(int)))) return st;
    if ((st = upload(c, c->d_npw, npw, (size_t)nk * sizeof(int)))) return st;
    if ((st = upload(c, c->d_energy, energy_ha, (size_t)nk * nband * sizeof(double)))) return st;
    if (T) { if ((st = upload(c, c->d_T, T, (size_t)nk * nband * sizeof(double)))) return st; }
    build_tetrahedra(c);
    if ((st = upload(c, c->d_tets, c->tets.data(), c->tets.size() * sizeof(int)))) return st;
    if ((st = upload(c, c->d_tetk, c->tetk.data(), c->tetk.size() * sizeof(int)))) return st;
    c->loaded = true;
    return RP_OK;
}

int rp_sphere_size(rp_ctx* c, const double q[3], int* ng, int* n_tail, int* miller_out, int* tail_out) {
    if (!c) return RP_ERR_ARG;
    return rp_sphere_size_at(c, q, c->ecut_eps, ng, n_tail, miller_out, tail_out);
}

int rp_sphere_size_at(rp_ctx* c, const double q[3], double ecut_eps_ha, int* ng, int* n_tail, int* miller_out,
                      int* tail_out) {
    if (!c || !q) return RP_ERR_ARG;
    int st = plan_q_cut(c, q, ecut_eps_ha);
    if (st) return st;
    if (ng) *ng = c->plan.ng;
    if (n_tail) *n_tail = c->plan.ntail;
    if (miller_out) std::memcpy(miller_out, c->plan.gm.data(), c->plan.gm.size() * sizeof(int));
    if (tail_out) std::memcpy(tail_out, c->plan.tail.data(), c->plan.tail.size() * sizeof(int));
    return RP_OK;
}

static int check_ready_cut(rp_ctx* c, const double q[3], double ecut_eps) {
    if (!c) return RP_ERR_ARG;
    if (!c->loaded) return fail(c, RP_ERR_STATE, "bands not loaded");
    if (!q) return fail(c, RP_ERR_ARG, "q is NULL");
    return plan_q_cut(c, q, ecut_eps);
}
static int check_ready(rp_ctx* c, const double q[3]) { return check_ready_cut(c, q, c ? c->ecut_eps : 0.0); }

int rp_transform_grid(rp_ctx* c, const double q[3], int* n_out, int* window_out) {
    int s = check_ready(c, q);
    if (s) return s;
    if (!n_out) return fail(c, RP_ERR_ARG, "n_out is NULL");
    for (int a = 0; a < 3; ++a) n_out[a] = c->plan.nfft[a];
    if (window_out) *window_out = c->plan.zyw;
    return RP_OK;
}

static int finish(rp_ctx* c, cudaStream_t st, int on_device) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
    c->last_stream = st;
    if (!on_device) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
    }
    return RP_OK;
}

// pair densities of k in [k0, k1) into M (device) with leading dimension ldm, column col0
// M is complex double, or complex float when fp32 (split-precision tiers).  The k points are
// taken in sub-blocks whose real-space grids stay within a scratch budget.
static int pair_density_device(rp_ctx* c, int k0, int k1, void* M, bool fp32, long long ldm, long long col0,
                               cudaStream_t st) {
    const size_t per_k = (size_t)c->nband * c->plan.nr * (fp32 ? sizeof(float2) : sizeof(double2));
    // plane sums of one k point in the windowed (FP32) or residue-set (FP64) layout of the plane-wise
    // pair kernels: the sub-block keeps them within those kernels' budget (one k point at least;
    // its empty bands are then taken in chunks)
    const QPlan& P = c->plan;
    const int W = fp32 ? P.zyw : 0;
    const size_t wyz = W > 0 ? (size_t)(2 * W + 1) * (2 * W + 1) : (size_t)P.nset[1] * P.nset[2];
    const size_t t2_k = (size_t)c->nemp * c->nocc * P.nfft[0] * wyz * (fp32 ? sizeof(float2) : sizeof(double2));
    size_t kb_t2 = std::max<size_t>(1, c->pair_budget / std::max<size_t>(1, t2_k));
    if (!fp32) {
        // the FP64 tier's fused path keeps z-transformed planes of every pair within 12 GB
        const size_t t1_k = (size_t)c->nemp * c->nocc * P.nfft[0] * P.nfft[1] * P.nset[2] * sizeof(double2);
        kb_t2 = std::min<size_t>(kb_t2, std::max<size_t>(1, ((size_t)12 << 30) / std::max<size_t>(1, t1_k)));
    }
    const int kb = (int)std::max<size_t>(
        1, std::min<size_t>(std::min<size_t>((size_t)(k1 - k0), ((size_t)2 << 30) / (3 * per_k)), kb_t2));
    for (int k = k0; k < k1; k += kb) {
        const int nkb = std::min(kb, k1 - k);
        prof_begin(c, 0, st);
        cudaError_t e = launch_gather_inverse(c, k, nkb, fp32, st);
        prof_end(c, 0, st, 1);
        if (e != cudaSuccess) return cuda_fail(c, e, "gather/inverse transform");
        prof_begin(c, 1, st);
        int nl = 0;
        const long long col = col0 + (long long)(k - k0) * c->nemp * c->nocc;
        e = fp32 ? launch_pair_forward32(c, nkb, (float2*)M, ldm, col, st, &nl)
                 : launch_pair_forward(c, nkb, (double2*)M, ldm, col, st, &nl);
        prof_end(c, 1, st, nl);
        if (e != cudaSuccess) return cuda_fail(c, e, "pair transform");
    }
    return RP_OK;
}

int rp_pair_density(rp_ctx* c, const double q[3], int k_begin, int k_end, double* M_out, int on_device, void* stream) {
    int s = check_ready(c, q);
    if (s) return s;
    if (k_begin < 0 || k_end > c->nk || k_begin >= k_end || !M_out) return fail(c, RP_ERR_ARG, "bad k range or output");
    cudaStream_t st = (cudaStream_t)stream;
    const long long kcols = (long long)(k_end - k_begin) * c->nemp * c->nocc;
    const size_t bytes = (size_t)c->plan.ng * kcols * sizeof(double2);
    double2* M = (double2*)M_out;
    if (!on_device) {
        if ((s = ensure(c, c->s_io1, bytes))) return s;
        M = (double2*)c->s_io1.p;
    }
    if ((s = pair_density_device(c, k_begin, k_end, M, false, kcols, 0, st))) return s;
    if (!on_device) {
        cudaError_t e = cudaMemcpyAsync(M_out, M, bytes, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "copy M");
    }
    return finish(c, st, on_device);
}

static int check_freq(rp_ctx* c, int axis, int ordering, int nfreq, const double* freq, double delta,
                      double da, double dr) {
    if (axis != RP_AXIS_REAL && axis != RP_AXIS_IMAG) return fail(c, RP_ERR_ARG, "bad axis");
    if (ordering != RP_TIME_ORDERED && ordering != RP_RETARDED) return fail(c, RP_ERR_ARG, "bad ordering");
    if (nfreq < 1 || !freq) return fail(c, RP_ERR_ARG, "no frequencies");
    if (!(delta >= 0) || !(da >= 0) || !(dr >= 0) || !std::isfinite(delta)) return fail(c, RP_ERR_ARG, "bad broadening/thresholds");
    for (int f = 0; f < nfreq; ++f) {
        if (!std::isfinite(freq[f])) return fail(c, RP_ERR_ARG, "frequency not finite");
        double im1 = (axis == RP_AXIS_REAL) ? delta : freq[f] + delta;
        double im2 = (axis == RP_AXIS_REAL) ? (ordering == RP_TIME_ORDERED ? delta : -delta)
                                            : (ordering == RP_TIME_ORDERED ? -freq[f] + delta : -freq[f] - delta);
        if (im1 == 0.0 || im2 == 0.0) return fail(c, RP_ERR_ARG, "a pole of X lies on the real axis");
    }
    return RP_OK;
}

static int weights_device(rp_ctx* c, int axis, int ordering, int nfreq, const double* freq, double delta,
                          double da, double dr, bool fp32, double2* w, cudaStream_t st) {
    int s = ensure(c, c->s_io3, nfreq * sizeof(double));
    if (s) return s;
    // the frequencies go through a pageable host copy owned by the context: a copy from pageable
    // memory is staged before cudaMemcpyAsync returns, so neither buffer has to outlive the call
    // and the stream is not synchronised (the caller's array might be pinned)
    c->freq_stage.assign(freq, freq + nfreq);
    cudaError_t e = cudaMemcpyAsync(c->s_io3.p, c->freq_stage.data(), nfreq * sizeof(double),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy frequencies");
    prof_begin(c, 2, st);
    e = launch_tetra(c, axis, ordering, nfreq, (const double*)c->s_io3.p, delta, da, dr, fp32, w, st);
    prof_end(c, 2, st, fp32 ? 2 : 1);
    return e == cudaSuccess ? RP_OK : cuda_fail(c, e, "tetrahedron weights");
}

int rp_tetra_weights(rp_ctx* c, const double q[3], int axis, int ordering, int nfreq, const double* freq,
                     double delta, double da, double dr, int precision, double* w_out, int on_device, void* stream) {
    int s = check_ready(c, q);
    if (s) return s;
    if ((s = check_freq(c, axis, ordering, nfreq, freq, delta, da, dr))) return s;
    if (!w_out) return fail(c, RP_ERR_ARG, "w_out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const long long K = (long long)c->nk * c->nemp * c->nocc;
    const size_t bytes = (size_t)nfreq * K * sizeof(double2);
    double2* w = (double2*)w_out;
    if (!on_device) {
        if ((s = ensure(c, c->s_io1, bytes))) return s;
        w = (double2*)c->s_io1.p;
    }
    if (precision != RP_FP64_NATIVE && precision != RP_BF16X3) return fail(c, RP_ERR_UNSUPPORTED, "precision not built");
    if ((s = weights_device(c, axis, ordering, nfreq, freq, delta, da, dr, precision != RP_FP64_NATIVE, w, st))) return s;
    if (!on_device) {
        cudaError_t e = cudaMemcpyAsync(w_out, w, bytes, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "copy w");
    }
    return finish(c, st, on_device);
}

// raw rows per tile of the BF16x3 contraction for this NG: the tuned or set choice, else 0 (the
// launcher's least-padding rule)
static int tile_for(const rp_ctx* c, int ng) {
    auto it = c->tile_bn.find(ng);
    return it == c->tile_bn.end() ? 0 : it->second;
}

// chi (+)= M[:, col0m .. col0m+K) diag(w[f][col0w ..]) M^H with the selected precision.
// For RP_BF16X3 the caller zeroes chi before the first block.
static int contract_block(rp_ctx* c, int precision, const void* M, bool m32, long long ldm, long long col0m,
                          long long K, const double2* w, long long ldw, long long col0w, int nfreq, int ng,
                          double2* chi, int accumulate, cudaStream_t st) {
    cudaError_t e;
    if (precision == RP_FP64_NATIVE) {
        prof_begin(c, 3, st);
        e = launch_contract_f64((const double2*)M + col0m, ldm, K, w, ldw, col0w, nfreq, ng, chi, accumulate, st);
        prof_end(c, 3, st, 1);
        return e == cudaSuccess ? RP_OK : cuda_fail(c, e, "contraction");
    }
    if (precision == RP_TF32X3) {
        prof_begin(c, 3, st);
        const void* Mb = m32 ? (const void*)((const float2*)M + col0m) : (const void*)((const double2*)M + col0m);
        e = launch_contract_tf32x3(Mb, m32, ldm, K, w, ldw, col0w, nfreq, ng, chi, accumulate, st);
        prof_end(c, 3, st, 1);
        return e == cudaSuccess ? RP_OK : cuda_fail(c, e, "TF32x3 contraction");
    }
    const size_t sb = (size_t)ng * tc_kp2(K) * 2;
    int s;
    if ((s = ensure(c, c->s_hi, sb)) || (s = ensure(c, c->s_lo, sb)) ||
        (s = ensure(c, c->s_w32, (size_t)tc_wrows(nfreq) * (tc_kp2(K) / 2) * sizeof(float2))))
        return s;
    prof_begin(c, 5, st);
    e = launch_split_bf16(M, m32, ldm, col0m, K, ng, c->s_hi.p, c->s_lo.p, st);
    if (e == cudaSuccess) e = launch_weights32(K, w, ldw, col0w, nfreq, c->s_w32.p, st);
    prof_end(c, 5, st, 2);
    if (e == cudaSuccess) {
        prof_begin(c, 3, st);
        e = launch_contract_bf16x3_core(c->s_hi.p, c->s_lo.p, K, ng, nfreq, c->s_w32.p, chi, (int*)c->d_err.p + 1,
                                        c->num_sms, c->wait_ns, st, tile_for(c, ng));
        prof_end(c, 3, st, 1);
    }
    return e == cudaSuccess ? RP_OK : cuda_fail(c, e, "bf16x3 contraction");
}

static int check_timeout(rp_ctx* c) {
    int flag = 0;
    if (cudaMemcpy(&flag, (int*)c->d_err.p + 1, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "read timeout flag");
    if (flag) {
        cudaMemset((int*)c->d_err.p + 1, 0, sizeof(int));
        char buf[96];
        snprintf(buf, sizeof(buf), "a bounded device wait gave up (site %d)", flag);
        return fail(c, RP_ERR_TIMEOUT, buf);
    }
    return RP_OK;
}

int rp_contract_chi0(rp_ctx* c, int ng, long long K, int nfreq, const double* M, const double* w, int precision,
                     double* chi_out, int on_device, void* stream) {
    if (!c) return RP_ERR_ARG;
    if (ng < 1 || K < 1 || nfreq < 1 || !M || !w || !chi_out) return fail(c, RP_ERR_ARG, "bad contraction arguments");
    if (precision != RP_FP64_NATIVE && precision != RP_BF16X3 && precision != RP_TF32X3)
        return fail(c, RP_ERR_UNSUPPORTED, "precision not built");
    cudaStream_t st = (cudaStream_t)stream;
    const double2 *dM = (const double2*)M, *dw = (const double2*)w;
    double2* dchi = (double2*)chi_out;
    int s;
    const size_t bm = (size_t)ng * K * sizeof(double2), bw = (size_t)nfreq * K * sizeof(double2);
    const size_t bc = (size_t)nfreq * ng * ng * sizeof(double2);
    if (!on_device) {
        if ((s = ensure(c, c->s_io1, bm)) || (s = ensure(c, c->s_io2, bw)) || (s = ensure(c, c->s_chi, bc))) return s;
        cudaMemcpyAsync(c->s_io1.p, M, bm, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(c->s_io2.p, w, bw, cudaMemcpyHostToDevice, st);
        dM = (const double2*)c->s_io1.p; dw = (const double2*)c->s_io2.p; dchi = (double2*)c->s_chi.p;
    }
    if (precision == RP_BF16X3) {
        cudaError_t e = cudaMemsetAsync(dchi, 0, bc, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "zero chi");
    }
    if ((s = contract_block(c, precision, dM, false, K, 0, K, dw, K, 0, nfreq, ng, dchi, 0, st))) return s;
    if (!on_device) {
        cudaError_t e = cudaMemcpyAsync(chi_out, dchi, bc, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "copy chi");
    }
    if ((s = finish(c, st, on_device))) return s;
    return on_device ? RP_OK : check_timeout(c);
}

// chi0 of q summed over the pairs of the k points in klist[nks] (all k when klist is NULL), with
// weights from the whole mesh's tetrahedra
// With qhat (q = 0 only) the block of pair densities gets a head row u_b = qhat.p_b / D_b above the
// sphere rows, and chi0_out is the extended [nfreq][NG+1][NG+1] matrix (index 0: head and wings).
static int build_chi0(rp_ctx* c, const double q[3], double ecut_eps, int axis, int ordering, int nfreq,
                      const double* freq, double delta, double da, double dr, int precision, double* chi0_out,
                      int on_device, void* stream, int nks = 0, const int* klist = nullptr,
                      const double* qhat = nullptr) {
    int s = check_ready_cut(c, q, ecut_eps);
    if (s) return s;
    if (qhat && (q[0] != 0.0 || q[1] != 0.0 || q[2] != 0.0)) return fail(c, RP_ERR_ARG, "the head row needs q = 0");
    if ((s = check_freq(c, axis, ordering, nfreq, freq, delta, da, dr))) return s;
    if (!chi0_out) return fail(c, RP_ERR_ARG, "chi0_out is NULL");
    // runs of consecutive k points: [runs[2i], runs[2i+1])
    std::vector<int> runs;
    if (klist) {
        if (nks < 1 || nks > c->nk) return fail(c, RP_ERR_ARG, "bad k-point count");
        std::vector<int> ks(klist, klist + nks);
        std::sort(ks.begin(), ks.end());
        for (int i = 0; i < nks; ++i) {
            if (ks[i] < 0 || ks[i] >= c->nk) return fail(c, RP_ERR_ARG, "k index out of range");
            if (i > 0 && ks[i] == ks[i - 1]) return fail(c, RP_ERR_ARG, "repeated k index");
            if (i > 0 && ks[i] == ks[i - 1] + 1) runs.back() = ks[i] + 1;
            else { runs.push_back(ks[i]); runs.push_back(ks[i] + 1); }
        }
    } else {
        runs = {0, c->nk};
    }
    if (precision != RP_FP64_NATIVE && precision != RP_BF16X3 && precision != RP_TF32X3)
        return fail(c, RP_ERR_UNSUPPORTED, "precision not built");
    cudaStream_t st = (cudaStream_t)stream;
    const int ngs = c->plan.ng;                       // sphere rows
    const int ng = qhat ? ngs + 1 : ngs;               // rows of the contraction
    const long long K = (long long)c->nk * c->nemp * c->nocc;
    const long long kcols = (long long)c->nemp * c->nocc;
    // k points per contraction launch: about 64k pair columns
    const int kb = (int)std::max(1LL, std::min((long long)c->nk, 65536LL / kcols));
    if ((s = ensure(c, c->s_w, (size_t)nfreq * K * sizeof(double2)))) return s;
    const bool m32 = precision != RP_FP64_NATIVE;
    if ((s = ensure(c, c->s_m, (size_t)ng * kcols * kb * (m32 ? sizeof(float2) : sizeof(double2))))) return s;
    const size_t bc = (size_t)nfreq * ng * ng * sizeof(double2);
    double2* chi = (double2*)chi0_out;
    if (!on_device) {
        if ((s = ensure(c, c->s_chi, bc))) return s;
        chi = (double2*)c->s_chi.p;
    }
    double2* w = (double2*)c->s_w.p;
    // the FP32 weight pass belongs to the BF16x3 tier; TF32x3 keeps FP64 weights (its own error is
    // far below the FP32 pass's)
    if ((s = weights_device(c, axis, ordering, nfreq, freq, delta, da, dr, precision == RP_BF16X3, w, st))) return s;
    if (precision == RP_BF16X3) {
        cudaError_t e = cudaMemsetAsync(chi, 0, bc, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "zero chi");
    }
    void* M = c->s_m.p;
    bool first = true;
    for (size_t r = 0; r < runs.size(); r += 2)
        for (int k0 = runs[r]; k0 < runs[r + 1]; k0 += kb) {
            const int k1 = std::min(runs[r + 1], k0 + kb);
            const long long cols = (long long)(k1 - k0) * kcols;
            // sphere rows from row 1 when the head row is there
            void* Ms = !qhat ? M : (m32 ? (void*)((float2*)M + cols) : (void*)((double2*)M + cols));
            if ((s = pair_density_device(c, k0, k1, Ms, m32, cols, 0, st))) return s;
            if (qhat) {
                cudaError_t e = launch_head_row(c, k0, k1 - k0, qhat, m32, M, 0, st);
                if (e != cudaSuccess) return cuda_fail(c, e, "head row");
            }
            if ((s = contract_block(c, precision, M, m32, cols, 0, cols, w, K, (long long)k0 * kcols, nfreq, ng, chi,
                                    first ? 0 : 1, st)))
                return s;
            first = false;
        }
    if (!on_device) {
        cudaError_t e = cudaMemcpyAsync(chi0_out, chi, bc, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "copy chi0");
    }
    if ((s = finish(c, st, on_device))) return s;
    return on_device ? RP_OK : check_timeout(c);
}

int rp_check_numeric(rp_ctx* c) {
    if (!c) return RP_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(c->last_stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
    int flag[2] = {0, 0};
    e = cudaMemcpy(flag, c->d_err.p, 2 * sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "read error flags");
    if (flag[0] || flag[1]) cudaMemset(c->d_err.p, 0, 2 * sizeof(int));
    if (flag[1]) {
        char buf[112];
        snprintf(buf, sizeof(buf), "a bounded device wait of an asynchronous contraction gave up (site %d)", flag[1]);
        return fail(c, RP_ERR_TIMEOUT, buf);
    }
    if (flag[0]) return fail(c, RP_ERR_NUMERIC, "zero or non-finite pivot in the Dyson solve");
    return RP_OK;
}

int rp_set_contraction_tile(rp_ctx* c, int ng, int bn) {
    if (!c) return RP_ERR_ARG;
    if (ng < 1) return fail(c, RP_ERR_ARG, "ng < 1");
    if (bn == 0) {
        c->tile_bn.erase(ng);
        return RP_OK;
    }
    if (!tc_bn_supported(bn)) return fail(c, RP_ERR_ARG, "tile width not built");
    c->tile_bn[ng] = bn;
    return RP_OK;
}

int rp_tune_contraction(rp_ctx* c, int ng, long long K, int nfreq, int* bn_out, double* ms_out) {
    if (!c) return RP_ERR_ARG;
    if (ng < 1 || K < 1 || nfreq < 1 || !bn_out) return fail(c, RP_ERR_ARG, "bad tuning shape");
    cudaStream_t st = nullptr;
    const long long kp2 = tc_kp2(K);
    int s;
    if ((s = ensure(c, c->s_hi, (size_t)ng * kp2 * 2)) || (s = ensure(c, c->s_lo, (size_t)ng * kp2 * 2)) ||
        (s = ensure(c, c->s_w32, (size_t)tc_wrows(nfreq) * (kp2 / 2) * sizeof(float2))) ||
        (s = ensure(c, c->s_chi, (size_t)nfreq * ng * ng * sizeof(double2))))
        return s;
    cudaError_t e = launch_fill_tune_operands(c->s_hi.p, c->s_lo.p, (long long)ng * kp2, c->s_w32.p,
                                              (long long)tc_wrows(nfreq) * (kp2 / 2), st);
    if (e != cudaSuccess) return cuda_fail(c, e, "tuning operands");
    int cand[16];
    const int nc = tc_bn_candidates(cand);
    cudaEvent_t ev[2];
    if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "events");
    int best = 0;
    float best_ms = 0.0f;
    for (int i = 0; i < nc && e == cudaSuccess; ++i) {
        float ms = 0.0f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {      // the first run warms up
            e = cudaEventRecord(ev[0], st);
            if (e == cudaSuccess)
                e = launch_contract_bf16x3_core(c->s_hi.p, c->s_lo.p, K, ng, nfreq, c->s_w32.p, (double2*)c->s_chi.p,
                                                (int*)c->d_err.p + 1, c->num_sms, c->wait_ns, st, cand[i]);
            if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        }
        if (ms_out) ms_out[i] = ms;
        if (e == cudaSuccess && (best == 0 || ms < best_ms)) {
            best = cand[i];
            best_ms = ms;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e != cudaSuccess) return cuda_fail(c, e, "tuning run");
    if ((s = check_timeout(c))) return s;
    c->tile_bn[ng] = best;
    *bn_out = best;
    return RP_OK;
}

int rp_set_dyson_hermitian(rp_ctx* c, int on) {
    if (!c) return RP_ERR_ARG;
    c->dyson_herm = on != 0;
    return RP_OK;
}

int rp_set_fermi(rp_ctx* c, double efermi_ha) {
    if (!c) return RP_ERR_ARG;
    if (std::isnan(efermi_ha)) {
        c->metal = false;
        return RP_OK;
    }
    if (!std::isfinite(efermi_ha)) return fail(c, RP_ERR_ARG, "Fermi energy not finite");
    c->metal = true;
    c->efermi = efermi_ha;
    return RP_OK;
}

int rp_set_pair_budget(rp_ctx* c, long long bytes) {
    if (!c) return RP_ERR_ARG;
    if (bytes < 1) return fail(c, RP_ERR_ARG, "pair budget must be positive");
    c->pair_budget = (size_t)bytes;
    return RP_OK;
}

int rp_set_wait_limit(rp_ctx* c, long long limit_ns) {
    if (!c) return RP_ERR_ARG;
    if (limit_ns < 0) return fail(c, RP_ERR_ARG, "negative wait limit");
    c->wait_ns = (unsigned long long)limit_ns;
    return RP_OK;
}

static int solve_w(rp_ctx* c, const double q[3], double ecut_eps, int nfreq, const double* chi0, double* W_out,
                   double* tail_out, int on_device, void* stream) {
    int s = check_ready_cut(c, q, ecut_eps);
    if (s) return s;
    if (nfreq < 1 || !chi0 || !W_out) return fail(c, RP_ERR_ARG, "bad Dyson arguments");
    const int ng = c->plan.ng;
    if (ng > 4096) return fail(c, RP_ERR_UNSUPPORTED, "NG above 4096");
    cudaStream_t st = (cudaStream_t)stream;
    if (on_device && c->last_stream) {
        // a bad pivot of an earlier asynchronous call is reported here
        int flag = 0;
        if (cudaMemcpy(&flag, c->d_err.p, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && flag) {
            cudaMemset(c->d_err.p, 0, sizeof(int));
            return fail(c, RP_ERR_NUMERIC, "zero or non-finite pivot in an earlier Dyson solve");
        }
    }
    const size_t bc = (size_t)nfreq * ng * ng * sizeof(double2);
    const double2* dchi = (const double2*)chi0;
    double2* dW = (double2*)W_out;
    if (!on_device) {
        if ((s = ensure(c, c->s_io1, bc)) || (s = ensure(c, c->s_io2, bc)) ||
            (s = ensure(c, c->s_io3, (size_t)std::max(1, c->plan.ntail) * sizeof(double)))) return s;
        cudaError_t e = cudaMemcpyAsync(c->s_io1.p, chi0, bc, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "copy chi0");
        dchi = (const double2*)c->s_io1.p;
        dW = (double2*)c->s_io2.p;
    }
    if ((s = ensure(c, c->s_dy, dyson_scratch_bytes(ng, nfreq)))) return s;
    prof_begin(c, 4, st);
    cudaError_t e = launch_dyson(dchi, (const double*)c->plan.d_vs.p, ng, nfreq, dW, c->s_dy.p, c->dyson_herm, (int*)c->d_err.p, st);
    prof_end(c, 4, st, 1);
    if (e != cudaSuccess) return cuda_fail(c, e, "Dyson solve");
    if (tail_out && c->plan.ntail > 0) {
        if (on_device) {
            // staged from the plan's pageable vector before the call returns
            e = cudaMemcpyAsync(tail_out, c->plan.tailv.data(), c->plan.ntail * sizeof(double),
                                cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return cuda_fail(c, e, "tail");
        } else {
            std::memcpy(tail_out, c->plan.tailv.data(), c->plan.ntail * sizeof(double));
        }
    }
    if (!on_device) {
        e = cudaMemcpyAsync(W_out, dW, bc, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "copy W");
        if ((s = finish(c, st, 0))) return s;
        return rp_check_numeric(c);
    }
    return finish(c, st, 1);
}

int rp_build_chi0(rp_ctx* c, const double q[3], int axis, int ordering, int nfreq, const double* freq,
                  double delta, double da, double dr, int precision, double* chi0_out, int on_device, void* stream) {
    if (!c) return RP_ERR_ARG;
    return build_chi0(c, q, c->ecut_eps, axis, ordering, nfreq, freq, delta, da, dr, precision, chi0_out, on_device,
                      stream);
}

int rp_build_chi0_q0(rp_ctx* c, const double qhat[3], int axis, int ordering, int nfreq, const double* freq,
                     double delta, double da, double dr, int precision, double* chi0_out, int on_device,
                     void* stream) {
    if (!c) return RP_ERR_ARG;
    if (!qhat) return fail(c, RP_ERR_ARG, "qhat is NULL");
    const double n = std::sqrt(qhat[0] * qhat[0] + qhat[1] * qhat[1] + qhat[2] * qhat[2]);
    if (!(n > 0.0) || !std::isfinite(n)) return fail(c, RP_ERR_ARG, "qhat must be a nonzero direction");
    const double u[3] = {qhat[0] / n, qhat[1] / n, qhat[2] / n};
    const double q0[3] = {0.0, 0.0, 0.0};
    // u = qhat.p / (E_ak - E_ok) needs the lowest empty band above the highest occupied one at every k
    if (c->loaded)
        for (int k = 0; k < c->nk; ++k)
            if (!(c->energy[(size_t)k * c->nband + c->nocc] > c->energy[(size_t)k * c->nband + c->nocc - 1]))
                return fail(c, RP_ERR_ARG, "the q -> 0 head needs a gap between occupied and empty bands at every k");
    return build_chi0(c, q0, c->ecut_eps, axis, ordering, nfreq, freq, delta, da, dr, precision, chi0_out, on_device,
                      stream, 0, nullptr, u);
}

int rp_solve_w_q0(rp_ctx* c, int nfreq, const double* chi0, double* W_out, double* tail_out, int on_device,
                  void* stream) {
    const double q0[3] = {0.0, 0.0, 0.0};
    int s = check_ready(c, q0);
    if (s) return s;
    if (nfreq < 1 || !chi0 || !W_out) return fail(c, RP_ERR_ARG, "bad Dyson arguments");
    const int n = c->plan.ng + 1;
    if (n > 4096) return fail(c, RP_ERR_UNSUPPORTED, "NG above 4096");
    cudaStream_t st = (cudaStream_t)stream;
    // v^1/2 of the extended rows: sqrt(4 pi/Omega) for the head (its 1/|q| is carried by the head row)
    std::vector<double> vx(n);
    vx[0] = std::sqrt(4.0 * M_PI / c->omega);
    for (int g = 1; g < n; ++g) vx[g] = c->plan.vs[g - 1];
    const size_t bc = (size_t)nfreq * n * n * sizeof(double2);
    if ((s = ensure(c, c->s_io3, n * sizeof(double)))) return s;
    cudaError_t e = cudaMemcpyAsync(c->s_io3.p, vx.data(), n * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "v^1/2");
    const double2* dchi = (const double2*)chi0;
    double2* dW = (double2*)W_out;
    if (!on_device) {
        if ((s = ensure(c, c->s_io1, bc)) || (s = ensure(c, c->s_io2, bc))) return s;
        if ((e = cudaMemcpyAsync(c->s_io1.p, chi0, bc, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(c, e, "copy chi0");
        dchi = (const double2*)c->s_io1.p;
        dW = (double2*)c->s_io2.p;
    }
    if ((s = ensure(c, c->s_dy, dyson_scratch_bytes(n, nfreq)))) return s;
    prof_begin(c, 4, st);
    e = launch_dyson(dchi, (const double*)c->s_io3.p, n, nfreq, dW, c->s_dy.p, c->dyson_herm, (int*)c->d_err.p, st);
    prof_end(c, 4, st, 1);
    if (e != cudaSuccess) return cuda_fail(c, e, "Dyson solve");
    if (tail_out && c->plan.ntail > 0) {
        if (on_device) {
            e = cudaMemcpyAsync(tail_out, c->plan.tailv.data(), c->plan.ntail * sizeof(double), cudaMemcpyHostToDevice,
                                st);
            if (e != cudaSuccess) return cuda_fail(c, e, "tail");
        } else {
            std::memcpy(tail_out, c->plan.tailv.data(), c->plan.ntail * sizeof(double));
        }
    }
    if (!on_device) {
        if ((e = cudaMemcpyAsync(W_out, dW, bc, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_fail(c, e, "copy W");
        if ((s = finish(c, st, 0))) return s;
        return rp_check_numeric(c);
    }
    return finish(c, st, 1);
}

int rp_rotate_q(rp_ctx* c, const double q_irr[3], const double q[3], const int S[9], int nfreq, const double* X_irr,
                double* X_out, int on_device, void* stream) {
    if (!c) return RP_ERR_ARG;
    if (!q_irr || !q || !S || nfreq < 1 || !X_irr || !X_out) return fail(c, RP_ERR_ARG, "bad rotation arguments");
    // q* S = q + G_s with G_s integer
    int gs[3];
    for (int j = 0; j < 3; ++j) {
        const double v = q_irr[0] * S[0 * 3 + j] + q_irr[1] * S[1 * 3 + j] + q_irr[2] * S[2 * 3 + j] - q[j];
        gs[j] = (int)llround(v);
        if (std::fabs(v - gs[j]) > 1e-9) return fail(c, RP_ERR_ARG, "q is not the image of q_irr under S");
    }
    // S must be a rotation of the lattice: |(m S) B| = |m B| on the reciprocal basis vectors
    for (int i = 0; i < 3; ++i) {
        double f[3] = {0, 0, 0}, g[3] = {0, 0, 0}, a[3], b[3];
        f[i] = 1.0;
        for (int j = 0; j < 3; ++j) g[j] = S[i * 3 + j];
        cart(c, f, a);
        cart(c, g, b);
        const double na = a[0] * a[0] + a[1] * a[1] + a[2] * a[2], nb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
        if (std::fabs(na - nb) > 1e-9 * na) return fail(c, RP_ERR_ARG, "S is not a rotation of the lattice");
    }
    int s = plan_q(c, q_irr);
    if (s) return s;
    const std::vector<int> gi = c->plan.gm;
    if ((s = plan_q(c, q))) return s;
    const QPlan& P = c->plan;
    const int n = P.ng;
    if ((int)gi.size() != 3 * n) return fail(c, RP_ERR_ARG, "the spheres of q_irr and q differ in size");
    std::map<long long, int> pos;
    auto key = [](long long a, long long b, long long d) { return ((a + 4096) * 8192 + (b + 4096)) * 8192 + (d + 4096); };
    for (int g = 0; g < n; ++g) {
        long long m[3];
        for (int j = 0; j < 3; ++j)
            m[j] = (long long)gi[3 * g] * S[0 * 3 + j] + (long long)gi[3 * g + 1] * S[1 * 3 + j] +
                   (long long)gi[3 * g + 2] * S[2 * 3 + j] + gs[j];
        pos[key(m[0], m[1], m[2])] = g;
    }
    std::vector<int> perm(n);
    for (int g = 0; g < n; ++g) {
        auto it = pos.find(key(P.gm[3 * g], P.gm[3 * g + 1], P.gm[3 * g + 2]));
        if (it == pos.end()) return fail(c, RP_ERR_ARG, "S does not map the sphere of q_irr onto that of q");
        perm[g] = it->second;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bc = (size_t)nfreq * n * n * sizeof(double2);
    if ((s = ensure(c, c->s_io3, n * sizeof(int)))) return s;
    cudaError_t e = cudaMemcpyAsync(c->s_io3.p, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "permutation");
    const double2* din = (const double2*)X_irr;
    double2* dout = (double2*)X_out;
    if (!on_device) {
        if ((s = ensure(c, c->s_io1, bc)) || (s = ensure(c, c->s_io2, bc))) return s;
        if ((e = cudaMemcpyAsync(c->s_io1.p, X_irr, bc, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(c, e, "copy X");
        din = (const double2*)c->s_io1.p;
        dout = (double2*)c->s_io2.p;
    }
    if ((e = launch_rotate(din, (const int*)c->s_io3.p, n, nfreq, dout, c->num_sms, st)) != cudaSuccess)
        return cuda_fail(c, e, "rotation");
    if (!on_device && (e = cudaMemcpyAsync(X_out, dout, bc, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(c, e, "copy X");
    return finish(c, st, on_device);
}

int rp_plasma(rp_ctx* c, double fermi_ha, double* omega2_out) {
    if (!c) return RP_ERR_ARG;
    if (!c->loaded) return fail(c, RP_ERR_STATE, "bands not loaded");
    if (!omega2_out || !std::isfinite(fermi_ha)) return fail(c, RP_ERR_ARG, "bad plasma arguments");
    int s = ensure(c, c->s_io3, 16 * sizeof(double));
    if (s) return s;
    cudaError_t e = cudaMemset(c->s_io3.p, 0, 16 * sizeof(double));
    if (e == cudaSuccess) e = launch_plasma(c, fermi_ha, (double*)c->s_io3.p, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    double t[9];
    if (e == cudaSuccess) e = cudaMemcpy(t, c->s_io3.p, 9 * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "plasma frequency");
    t[3] = t[1]; t[6] = t[2]; t[7] = t[5];
    std::memcpy(omega2_out, t, sizeof(t));
    return RP_OK;
}

int rp_probe_peaks(double* out) {
    if (!out) return RP_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RP_ERR_CUDA;
    return probe_peaks(out, nsm, nullptr);
}

int rp_optics(rp_ctx* c, int nfreq, const double* freq_ha, const double* W00, double* out) {
    if (!c) return RP_ERR_ARG;
    if (nfreq < 1 || !freq_ha || !W00 || !out) return fail(c, RP_ERR_ARG, "bad optics arguments");
    const double s = c->omega / (4.0 * M_PI);
    for (int f = 0; f < nfreq; ++f) {
        const std::complex<double> einv(W00[2 * f] * s, W00[2 * f + 1] * s);
        if (!(std::abs(einv) > 0.0) || !std::isfinite(std::abs(einv))) return fail(c, RP_ERR_NUMERIC, "eps^-1_00 zero or not finite");
        const std::complex<double> em = 1.0 / einv;
        const std::complex<double> r = (1.0 - std::sqrt(einv)) / (1.0 + std::sqrt(einv));
        double* o = out + 5 * f;
        o[0] = em.real();
        o[1] = em.imag();
        o[2] = -einv.imag();
        o[3] = freq_ha[f] / (4.0 * M_PI) * em.imag();
        o[4] = std::norm(r);
    }
    return RP_OK;
}

int rp_build_chi0_kset(rp_ctx* c, const double q[3], int nks, const int* k_list, int axis, int ordering, int nfreq,
                       const double* freq, double delta, double da, double dr, int precision, double* chi0_out,
                       int on_device, void* stream) {
    if (!c) return RP_ERR_ARG;
    if (!k_list) return fail(c, RP_ERR_ARG, "k_list is NULL");
    return build_chi0(c, q, c->ecut_eps, axis, ordering, nfreq, freq, delta, da, dr, precision, chi0_out, on_device,
                      stream, nks, k_list);
}

int rp_solve_w(rp_ctx* c, const double q[3], int nfreq, const double* chi0, double* W_out, double* tail_out,
               int on_device, void* stream) {
    if (!c) return RP_ERR_ARG;
    return solve_w(c, q, c->ecut_eps, nfreq, chi0, W_out, tail_out, on_device, stream);
}

int rp_build_chi0_batched(rp_ctx* c, int nq, const double* q_frac, const double* ecut_eps_per_q, int axis,
                          int ordering, int nfreq, const double* freq, double delta, double da, double dr,
                          int precision, double* const* chi0_out, int on_device, void* stream) {
    if (!c) return RP_ERR_ARG;
    if (nq < 1 || !q_frac || !chi0_out) return fail(c, RP_ERR_ARG, "bad batch arguments");
    for (int i = 0; i < nq; ++i) {
        const double cut = ecut_eps_per_q ? ecut_eps_per_q[i] : c->ecut_eps;
        const int s = build_chi0(c, q_frac + 3 * i, cut, axis, ordering, nfreq, freq, delta, da, dr, precision,
                                 chi0_out[i], on_device, stream);
        if (s) return s;
    }
    return RP_OK;
}

// Device buffers: every (q, w) matrix of the batch, sorted by NG (largest first), goes into
// cooperative launches of k_dyson_list that each fill the GPU.  Consecutive matrices join a launch
// while their summed per-pivot work (sum of NG^2) stays below about a large sphere's frequency set,
// so small spheres share their grid barriers; each matrix gets CTAs in proportion to NG^2 (equal
// work per CTA and step), at least 2 and at most one per 8 columns.
static constexpr int kPerQ = -1;     // solve_w_list: use the per-q solves instead
static int solve_w_list(rp_ctx* c, int nq, const double* q_frac, const double* cuts, int nfreq,
                        const double* const* chi0, double* const* W_out, double* const* tail_out, cudaStream_t st) {
    int s;
    if (c->last_stream) {
        // a bad pivot of an earlier asynchronous call is reported here
        int flag = 0;
        if (cudaMemcpy(&flag, c->d_err.p, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && flag) {
            cudaMemset(c->d_err.p, 0, sizeof(int));
            return fail(c, RP_ERR_NUMERIC, "zero or non-finite pivot in an earlier Dyson solve");
        }
    }
    std::vector<int> ng(nq);
    std::vector<size_t> vofs(nq);
    c->dy_vs.clear();
    for (int i = 0; i < nq; ++i) {
        if ((s = check_ready_cut(c, q_frac + 3 * i, cuts ? cuts[i] : c->ecut_eps))) return s;
        ng[i] = c->plan.ng;
        if (ng[i] > 4096) return fail(c, RP_ERR_UNSUPPORTED, "NG above 4096");
        vofs[i] = c->dy_vs.size();
        c->dy_vs.insert(c->dy_vs.end(), c->plan.vs.begin(), c->plan.vs.end());
        if (tail_out && tail_out[i] && c->plan.ntail > 0) {
            // staged from the plan's pageable vector before the call returns
            cudaError_t e = cudaMemcpyAsync(tail_out[i], c->plan.tailv.data(), c->plan.ntail * sizeof(double),
                                            cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return cuda_fail(c, e, "tail");
        }
    }
    // spheres below 16 points take the per-q solve (at least 8 columns for each of two CTAs)
    if (*std::min_element(ng.begin(), ng.end()) < 16) return kPerQ;
    // matrices, largest sphere first; scratch offsets
    const int nm = nq * nfreq;
    std::vector<int> order(nm);
    for (int m = 0; m < nm; ++m) order[m] = m;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ng[a / nfreq] > ng[b / nfreq]; });
    size_t cb_bytes = 0, ib_bytes = 0;
    for (int i = 0; i < nq; ++i) {
        cb_bytes += (size_t)nfreq * 2 * ng[i] * sizeof(double2);
        ib_bytes += (size_t)nfreq * (ng[i] + 2) * sizeof(int);
    }
    const size_t vs_bytes = c->dy_vs.size() * sizeof(double);
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    // launches: [first, last) of the sorted list, with their CTA counts
    std::vector<int> lb, lcount;
    std::vector<DysonMat> mats(nm);
    std::vector<int2> map;
    {
        const double target = 24.0 * 904.0 * 904.0;
        int m0 = 0;
        while (m0 < nm) {
            const int nmax = ng[order[m0] / nfreq];
            const int slots = dyson_list_slots(nmax);
            if (slots < 2) return fail(c, RP_ERR_CUDA, "batched Dyson kernel cannot be resident");
            double work = 0.0;
            int m1 = m0;
            while (m1 < nm && (m1 - m0 + 1) * 2 <= slots) {
                const double n = ng[order[m1] / nfreq];
                if (m1 > m0 && work + n * n > target) break;
                work += n * n;
                ++m1;
            }
            // two CTAs per matrix, then each further resident slot to the matrix whose CTAs have the
            // most work per step (NG^2 / P), up to one CTA per 8 columns: every slot is used and the
            // CTAs' work is as even as whole CTAs allow
            std::vector<int> P(m1 - m0, 2);
            int used = 2 * (m1 - m0);
            {
                std::vector<std::pair<double, int>> heap;
                for (int t = m0; t < m1; ++t) {
                    const double n = ng[order[t] / nfreq];
                    heap.push_back({n * n / 2.0, t - m0});
                }
                std::make_heap(heap.begin(), heap.end());
                while (used < slots && !heap.empty()) {
                    std::pop_heap(heap.begin(), heap.end());
                    const int i = heap.back().second;
                    heap.pop_back();
                    const int n = ng[order[m0 + i] / nfreq];
                    if (P[i] >= std::max(2, n / 8)) continue;
                    ++P[i];
                    ++used;
                    heap.push_back({(double)n * n / P[i], i});
                    std::push_heap(heap.begin(), heap.end());
                }
            }
            lb.push_back(m0);
            lcount.push_back(used);
            for (int t = m0; t < m1; ++t) {
                mats[t].n = ng[order[t] / nfreq];
                mats[t].P = P[t - m0];
                for (int pc = 0; pc < P[t - m0]; ++pc) map.push_back(make_int2(t, pc));
            }
            m0 = m1;
        }
        lb.push_back(nm);
    }
    const size_t mats_bytes = (size_t)nm * sizeof(DysonMat), map_bytes = map.size() * sizeof(int2);
    const size_t total = up(cb_bytes) + up(ib_bytes) + up(vs_bytes) + up(mats_bytes) + up(map_bytes);
    if ((s = ensure(c, c->s_dy, total))) return s;
    char* base = (char*)c->s_dy.p;
    double2* cb = (double2*)base;
    int* ib = (int*)(base + up(cb_bytes));
    double* dvs = (double*)(base + up(cb_bytes) + up(ib_bytes));
    DysonMat* dmats = (DysonMat*)(base + up(cb_bytes) + up(ib_bytes) + up(vs_bytes));
    int2* dmap = (int2*)((char*)dmats + up(mats_bytes));
    // per-matrix pointers: scratch in the order of q and w
    {
        std::vector<size_t> cbo(nq), ibo(nq);
        size_t a = 0, b = 0;
        for (int i = 0; i < nq; ++i) {
            cbo[i] = a; ibo[i] = b;
            a += (size_t)nfreq * 2 * ng[i];
            b += (size_t)nfreq * (ng[i] + 2);
        }
        for (int t = 0; t < nm; ++t) {
            const int i = order[t] / nfreq, f = order[t] % nfreq;
            const size_t n = (size_t)ng[i];
            mats[t].chi = (const double2*)chi0[i] + (size_t)f * n * n;
            mats[t].W = (double2*)W_out[i] + (size_t)f * n * n;
            mats[t].vs = dvs + vofs[i];
            mats[t].cb = cb + cbo[i] + (size_t)f * 2 * n;
            mats[t].ib = ib + ibo[i] + (size_t)f * (n + 2);
        }
    }
    // the lists go through context-owned pageable copies (staged before each copy call returns)
    c->dy_mats = mats;
    c->dy_map = map;
    cudaError_t e = cudaMemcpyAsync(dvs, c->dy_vs.data(), vs_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dmats, c->dy_mats.data(), mats_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dmap, c->dy_map.data(), map_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "batched Dyson lists");
    prof_begin(c, 4, st);
    int cta0 = 0;
    for (size_t l = 0; l + 1 < lb.size(); ++l) {
        const int nmax = ng[order[lb[l]] / nfreq];
        e = launch_dyson_list(dmats, dmap + cta0, lcount[l], nmax, c->dyson_herm, (int*)c->d_err.p, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "batched Dyson solve");
        cta0 += lcount[l];
    }
    prof_end(c, 4, st, (int)lb.size() - 1);
    return finish(c, st, 1);
}

int rp_solve_w_batched(rp_ctx* c, int nq, const double* q_frac, const double* ecut_eps_per_q, int nfreq,
                       const double* const* chi0, double* const* W_out, double* const* tail_out, int on_device,
                       void* stream) {
    if (!c) return RP_ERR_ARG;
    if (nq < 1 || !q_frac || !chi0 || !W_out) return fail(c, RP_ERR_ARG, "bad batch arguments");
    if (nfreq < 1) return fail(c, RP_ERR_ARG, "bad Dyson arguments");
    if (on_device && nq > 1) {
        if (!c->loaded) return fail(c, RP_ERR_STATE, "bands not loaded");
        for (int i = 0; i < nq; ++i)
            if (!chi0[i] || !W_out[i]) return fail(c, RP_ERR_ARG, "bad Dyson arguments");
        const int s = solve_w_list(c, nq, q_frac, ecut_eps_per_q, nfreq, chi0, W_out, tail_out, (cudaStream_t)stream);
        if (s != kPerQ) return s;
    }
    for (int i = 0; i < nq; ++i) {
        const double cut = ecut_eps_per_q ? ecut_eps_per_q[i] : c->ecut_eps;
        const int s = solve_w(c, q_frac + 3 * i, cut, nfreq, chi0[i], W_out[i], tail_out ? tail_out[i] : nullptr,
                              on_device, stream);
        if (s) return s;
    }
    return RP_OK;
}

int rp_load_wannier(rp_ctx* c, int nw, const double* coef) {
    if (!c) return RP_ERR_ARG;
    if (!c->loaded) return fail(c, RP_ERR_STATE, "bands not loaded");
    if (nw < 1 || nw > 16 || !coef) return fail(c, RP_ERR_ARG, "need 1 <= nw <= 16 and coefficients");
    const size_t row = (size_t)nw * c->npw_max * sizeof(double2);      // one k point's orbitals
    int st = ensure(c, c->d_wcoef, 2 * row * c->nk);
    if (st) return st;
    // each orbital twice: [k][0, nw) is the "occupied" copy at k, [k][nw, 2 nw) the "empty" one at k + q
    for (int half = 0; half < 2; ++half) {
        cudaError_t e = cudaMemcpy2D((char*)c->d_wcoef.p + half * row, 2 * row, coef, row, row, c->nk,
                                     cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(c, e, "upload Wannier coefficients");
    }
    c->nw = nw;
    return RP_OK;
}

int rp_interaction(rp_ctx* c, const double q[3], int nfreq, const double* W, int nR, const int* R_list, double* U_out,
                   double* J_out, int accumulate, int on_device, void* stream) {
    if (!c) return RP_ERR_ARG;
    if (!c->loaded || c->nw < 1) return fail(c, RP_ERR_STATE, "bands and Wannier functions not loaded");
    if (!q || nR < 1 || !R_list || !U_out || !J_out || (W && nfreq < 1))
        return fail(c, RP_ERR_ARG, "bad interaction arguments");
    const int nw = c->nw, nw2 = nw * nw, nb = nw + nR * nw2;
    if (nb > 192) return fail(c, RP_ERR_ARG, "nw + nR nw^2 above 192");
    cudaStream_t st = (cudaStream_t)stream;
    int s;
    // the epsilon sphere of W (the context's cut-off), then the whole wave-function sphere of q
    if ((s = check_ready(c, q))) return s;
    const std::vector<int> eps_m = c->plan.gm;
    const int ng = c->plan.ng;
    if ((s = plan_q_cut(c, q, c->ecut_psi, true))) return s;
    const QPlan& P = c->plan;
    const int ngp = P.ng;
    // positions of the epsilon-sphere members in the (lexicographic) wave-function sphere
    std::vector<int> pe(std::max(ng, 1));
    std::vector<unsigned char> in_eps(ngp, 0);
    {
        int e = 0;
        for (int g = 0; g < ngp && e < ng; ++g)
            if (P.gm[3 * g] == eps_m[3 * e] && P.gm[3 * g + 1] == eps_m[3 * e + 1] && P.gm[3 * g + 2] == eps_m[3 * e + 2]) {
                pe[e++] = g;
                in_eps[g] = 1;
            }
        if (e != ng) return fail(c, RP_ERR_STATE, "epsilon sphere not inside the wave-function sphere");
    }
    // e^{-i k.R} of every mesh point and e^{-i q.R}, v of the sphere
    std::vector<double2> tab((size_t)nR * c->nk + nR);
    for (int r = 0; r < nR; ++r) {
        for (int k = 0; k < c->nk; ++k) {
            const int i1 = k / (c->kmesh[1] * c->kmesh[2]), i2 = (k / c->kmesh[2]) % c->kmesh[1], i3 = k % c->kmesh[2];
            const double t = (double)i1 * R_list[3 * r] / c->kmesh[0] + (double)i2 * R_list[3 * r + 1] / c->kmesh[1] +
                             (double)i3 * R_list[3 * r + 2] / c->kmesh[2];
            tab[(size_t)r * c->nk + k] = make_double2(std::cos(2.0 * M_PI * t), -std::sin(2.0 * M_PI * t));
        }
        const double t = q[0] * R_list[3 * r] + q[1] * R_list[3 * r + 1] + q[2] * R_list[3 * r + 2];
        tab[(size_t)nR * c->nk + r] = make_double2(std::cos(2.0 * M_PI * t), -std::sin(2.0 * M_PI * t));
    }
    std::vector<double> v(ngp);
    for (int g = 0; g < ngp; ++g) v[g] = P.vs[g] * P.vs[g];
    const size_t tab_b = tab.size() * sizeof(double2), v_b = ngp * sizeof(double), pe_b = pe.size() * sizeof(int);
    const size_t aux = tab_b + v_b + pe_b + ngp + 256 * 4;
    const long long ldm = (long long)c->nk * nw2;
    const int nf = W ? nfreq : 1;
    const size_t nout = (size_t)nf * nR * nw2;
    if ((s = ensure(c, c->s_wm, (size_t)ngp * ldm * sizeof(double2))) ||
        (s = ensure(c, c->s_wb, (size_t)nb * ngp * sizeof(double2))) ||
        (s = ensure(c, c->s_wtab, aux)) || (s = ensure(c, c->s_wout, 2 * nout * sizeof(double2))))
        return s;
    char* ax = (char*)c->s_wtab.p;
    double2* d_tab = (double2*)ax;
    double* d_v = (double*)(ax + ((tab_b + 255) / 256) * 256);
    int* d_pe = (int*)((char*)d_v + ((v_b + 255) / 256) * 256);
    unsigned char* d_in = (unsigned char*)((char*)d_pe + ((pe_b + 255) / 256) * 256);
    // pageable sources: staged before each call returns
    cudaError_t e = cudaMemcpyAsync(d_tab, tab.data(), tab_b, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_v, v.data(), v_b, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_pe, pe.data(), pe_b, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_in, in_eps.data(), ngp, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "interaction tables");
    // orbital pair densities through the band kernels, on a band view of the Wannier functions
    {
        rp::DevBuf coef = c->d_coef;
        const int nband = c->nband, nocc = c->nocc, nemp = c->nemp;
        c->d_coef = c->d_wcoef;
        c->nband = 2 * nw; c->nocc = nw; c->nemp = nw;
        s = pair_density_device(c, 0, c->nk, c->s_wm.p, false, ldm, 0, st);
        c->d_coef = coef;
        c->nband = nband; c->nocc = nocc; c->nemp = nemp;
        if (s) return s;
    }
    e = launch_wan_density((const double2*)c->s_wm.p, ldm, c->nk, nw, nR, d_tab, (double2*)c->s_wb.p, ngp, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "Wannier densities");
    const double2* dW = (const double2*)W;
    double2* Y = nullptr;
    if (W) {
        const size_t wb = (size_t)nfreq * ng * ng * sizeof(double2);
        if ((s = ensure(c, c->s_wy, (size_t)nfreq * nb * ng * sizeof(double2)))) return s;
        if (!on_device) {
            if ((s = ensure(c, c->s_io1, wb))) return s;
            if ((e = cudaMemcpyAsync(c->s_io1.p, W, wb, cudaMemcpyHostToDevice, st)) != cudaSuccess)
                return cuda_fail(c, e, "copy W");
            dW = (const double2*)c->s_io1.p;
        }
        Y = (double2*)c->s_wy.p;
        e = launch_wan_wrhs(dW, ng, nfreq, (const double2*)c->s_wb.p, ngp, d_pe, nb, Y, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "W times the densities");
    }
    double2* dU = (double2*)U_out;
    double2* dJ = (double2*)J_out;
    if (!on_device) {
        dU = (double2*)c->s_wout.p;
        dJ = dU + nout;
        if (accumulate) {
            if ((e = cudaMemcpyAsync(dU, U_out, nout * sizeof(double2), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
                (e = cudaMemcpyAsync(dJ, J_out, nout * sizeof(double2), cudaMemcpyHostToDevice, st)) != cudaSuccess)
                return cuda_fail(c, e, "copy U, J");
        }
    }
    e = launch_wan_reduce((const double2*)c->s_wb.p, ngp, d_v, d_in, d_pe, ng, Y, nw, nR, nf, d_tab + (size_t)nR * c->nk,
                          1.0 / c->nk, accumulate, dU, dJ, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "interaction sums");
    if (!on_device) {
        if ((e = cudaMemcpyAsync(U_out, dU, nout * sizeof(double2), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(J_out, dJ, nout * sizeof(double2), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_fail(c, e, "copy U, J");
    }
    return finish(c, st, on_device);
}

int rp_profile_enable(rp_ctx* c, int enable) {
    if (!c) return RP_ERR_ARG;
    c->prof = enable != 0;
    for (int i = 0; i < RP_NSTAGE; ++i) { c->prof_used[i] = 0; c->prof_launches[i] = 0; }
    return RP_OK;
}

int rp_profile_read(rp_ctx* c, double* ms, long long* launches) {
    if (!c || !ms || !launches) return RP_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(c->last_stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
    for (int i = 0; i < RP_NSTAGE; ++i) {
        double tot = 0.0;
        for (int j = 0; j < c->prof_used[i]; ++j) {
            float t = 0.0f;
            e = cudaEventElapsedTime(&t, c->prof_ev[i][2 * j], c->prof_ev[i][2 * j + 1]);
            if (e != cudaSuccess) return cuda_fail(c, e, "event time");
            tot += t;
        }
        ms[i] = tot;
        launches[i] = c->prof_launches[i];
    }
    return RP_OK;
}

const char* rp_last_error(const rp_ctx* c) {
    return c ? c->err.c_str() : "null context";
}

void rp_destroy(rp_ctx* c) {
    if (!c) return;
    DevBuf* bufs[] = {&c->d_coef, &c->d_miller, &c->d_npw, &c->d_energy, &c->d_T, &c->d_tets, &c->d_tetk,
                      &c->plan.d_einv[0], &c->plan.d_einv[1], &c->plan.d_einv[2], &c->plan.d_einv32[0],
                      &c->plan.d_einv32[1], &c->plan.d_einv32[2], &c->d_err, &c->s_box, &c->s_u1, &c->s_u2,
                      &c->s_u, &c->s_p, &c->s_t1, &c->s_t2, &c->s_m, &c->s_w, &c->s_chi, &c->s_io1, &c->s_io2,
                      &c->s_io3, &c->s_hi, &c->s_lo, &c->s_w32, &c->s_queue, &c->plan.d_gpos, &c->plan.d_kp, &c->plan.d_g0, &c->plan.d_vs,
                      &c->plan.d_efwd[0], &c->plan.d_efwd[1], &c->plan.d_efwd[2], &c->plan.d_efwd32[0],
                      &c->plan.d_efwd32[1], &c->plan.d_efwd32[2], &c->plan.d_zmap, &c->plan.d_ymap,
                      &c->plan.d_gpos_r, &c->plan.d_gpos_w, &c->plan.d_colg, &c->d_wcoef, &c->s_wm, &c->s_wb,
                      &c->s_wy, &c->s_wtab, &c->s_wout, &c->s_dy};
    for (DevBuf* b : bufs) release(*b);
    for (int i = 0; i < RP_NSTAGE; ++i)
        for (cudaEvent_t e : c->prof_ev[i]) cudaEventDestroy(e);
    delete c;
}

}  // extern "C"
