// Internal declarations shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "respack_gb300.h"

#define RP_NSTAGE 6

namespace rp {

// Grow-only device allocation owned by a context.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Everything that depends on q: the epsilon sphere and its tail, the umklapp map
// k + q = k' + G0, and the phase tables of the pruned transforms.
struct QPlan {
    bool valid = false;
    double q[3] = {0, 0, 0};
    double ecut = 0;                 // epsilon-sphere cut-off the plan was made for (Ha)
    bool exact = false;              // transform grid chosen so that nothing folds onto the sphere
    int qi[3] = {0, 0, 0};           // q * kmesh (integers)
    int ng = 0, ntail = 0;
    std::vector<int> gm;             // [ng][3]
    std::vector<int> tail;           // [ntail][3]
    std::vector<double> vs;          // [ng] sqrt(4 pi / Omega) / |q+G|
    std::vector<double> tailv;       // [ntail] 4 pi / (Omega |q+G|^2)
    std::vector<int> kp, g0;         // [nk], [nk][3]
    int nset[3] = {0, 0, 0};         // distinct Miller values per axis in the sphere
    std::vector<int> setv[3];        // the values
    std::vector<int> gpos;           // [ng][3] position of each G's components in the sets
    DevBuf d_gpos, d_efwd[3], d_efwd32[3], d_kp, d_g0, d_vs;
    // residue maps (grid index -> position in the axis set, -1 if absent) of the y and z axes for
    // the fused pair kernels; fused is false when two set values share a residue
    bool fused = false;
    DevBuf d_zmap, d_ymap;
    // residue masks of the y and z axes (bit r: residue r present; axes of length <= 32 only) and
    // the sphere positions with the y and z components in ascending residue order, for the
    // plane-wise pair kernels
    bool masks = false;
    unsigned ymask = 0, zmask = 0;
    DevBuf d_gpos_r;
    // symmetric residue window of the FP32 pair kernels (cubic grids): half-width zyw (0: none)
    // holding every sphere component on all three axes; the sphere positions with the y and z
    // components at g + zyw, and the sphere index of each window point (gx, gy, gz) as
    // colg[gx + zyw][(gy + zyw) (2 zyw + 1) + gz + zyw] (-1 off the sphere)
    int zyw = 0;
    DevBuf d_gpos_w, d_colg;
    // grid of the pair-density transforms: the requested grid, or a smaller cubic one on which
    // the transforms are still exact for this sphere (see plan_q), with its inverse-transform
    // phases exp(+2 pi i m x / N) for m = -lb..lb, [N_axis][2 lb + 1] (FP64 and FP32)
    int nfft[3] = {0, 0, 0};
    long long nr = 0;
    DevBuf d_einv[3], d_einv32[3];
};

// one matrix of a batched Dyson launch: chi and W (n x n), v^1/2, its scratch (cb [2][n], ib [n + 2])
// and its CTA count P
struct DysonMat {
    const double2* chi;
    double2* W;
    const double* vs;
    double2* cb;
    int* ib;
    int n, P;
};

}  // namespace rp

struct rp_ctx {
    int device = 0;
    double lat[9], recip[9], omega = 0;
    int kmesh[3] = {1, 1, 1}, nk = 1, fft[3] = {0, 0, 0};
    long long nr = 0;
    double ecut_psi = 0, ecut_eps = 0;

    bool loaded = false;
    int nband = 0, nocc = 0, nemp = 0, npw_max = 0;
    int lb = 0;                       // half width of the Miller box used by the gather
    int mu[3] = {0, 0, 0};            // largest |Miller index| of the bands per axis
    std::vector<int> npw;             // [nk]
    std::vector<int> miller;          // [nk][npw_max][3]
    std::vector<double> energy;       // [nk][nband]
    std::vector<double> T;            // [nk][nband] or empty
    std::vector<int> tets;            // [6 nk][4]
    std::vector<int> tetk;            // [nk][24]: 4 * tetra + vertex position

    rp::DevBuf d_coef, d_miller, d_npw, d_energy, d_T, d_tets, d_tetk;
    rp::DevBuf d_err;                 // int error flags written by kernels
    rp::DevBuf s_dy;                  // scratch of the cooperative Dyson solve
    std::vector<double> dy_vs;        // staging of the batched Dyson solve: v^1/2 of every q,
    std::vector<rp::DysonMat> dy_mats; // the matrix list
    std::vector<int2> dy_map;         // and the CTA map
    // scratch (grow-only)
    rp::DevBuf s_box, s_u1, s_u2, s_u, s_p, s_t1, s_t2, s_m, s_w, s_chi, s_io1, s_io2, s_io3;
    rp::DevBuf s_hi, s_lo;            // bf16 hi/lo split of a block of pair densities
    rp::DevBuf s_w32;                 // complex float weights of that block
    rp::DevBuf s_queue;               // FP64 work list of the FP32 weight pass (count + items)
    // Wannier functions of the interaction step: coefficients [nk][2 nw][npw_max] (each orbital twice,
    // a band view with nocc = nemp = nw), and the scratch of rp_interaction
    int nw = 0;
    rp::DevBuf d_wcoef, s_wm, s_wb, s_wy, s_wtab, s_wout;
    int num_sms = 0;
    unsigned long long wait_ns = 2000000000ULL;   // limit of a bounded device wait (rp_set_wait_limit)
    size_t pair_budget = (size_t)16 << 30;        // plane-sum scratch of the pair stage (rp_set_pair_budget)
    bool metal = false;                           // Fermi-surface clipping of the weights (rp_set_fermi)
    bool dyson_herm = false;                      // Hermitian positive definite Dyson sweep (rp_set_dyson_hermitian)
    double efermi = 0.0;
    std::map<int, int> tile_bn;                   // NG -> raw rows per tile of the BF16x3 contraction
                                                  // (rp_tune_contraction / rp_set_contraction_tile)
    std::vector<double> freq_stage;               // host copy of the frequencies of the last weight pass

    rp::QPlan plan;
    // per-stage timing (CUDA events on the launching stream) and launch counts
    bool prof = false;
    std::vector<cudaEvent_t> prof_ev[RP_NSTAGE];
    int prof_used[RP_NSTAGE] = {0};
    long long prof_launches[RP_NSTAGE] = {0};
    std::string err;
    cudaStream_t last_stream = nullptr;
};

namespace rp {

int fail(rp_ctx* c, int code, const std::string& msg);
void prof_begin(rp_ctx* c, int stage, cudaStream_t st);
void prof_end(rp_ctx* c, int stage, cudaStream_t st, int launches);
int cuda_fail(rp_ctx* c, cudaError_t e, const char* where);
int ensure(rp_ctx* c, DevBuf& b, size_t bytes);
void release(DevBuf& b);
int plan_q(rp_ctx* c, const double q[3]);                  // with the context's cut-off
// (exact: enlarge a requested grid on which the product folds onto the sphere, so that the transforms
// give the plain convolution of Eq. ism)
int plan_q_cut(rp_ctx* c, const double q[3], double ecut_eps, bool exact = false);

// ---- kernel launchers (each returns cudaError_t of the launch) ----
// gather + inverse transform of nb bands into u[nb][N1][N2][N3] (complex double)
cudaError_t launch_gather_inverse(rp_ctx* c, int k0, int nkb, bool fp32, cudaStream_t st);
// pair densities of the bands prepared by launch_gather_inverse into M[ng][ld] at column col0
cudaError_t launch_pair_forward(rp_ctx* c, int nkb, double2* M, long long ldm, long long col0,
                                cudaStream_t st, int* nlaunch);
// the same in FP32 (for the split-precision tiers), M as complex float
// half-width of the FP32 plane kernel's residue window for plane length n holding |g| <= m (0: none)
int zy_window(int n, int m);
cudaError_t launch_pair_forward32(rp_ctx* c, int nkb, float2* M, long long ldm, long long col0,
                                  cudaStream_t st, int* nlaunch);
// tetrahedron weights for all pairs: w[nf][K]
// (fp32: split-precision tiers, FP64 re-evaluation near degeneracies)
cudaError_t launch_tetra(rp_ctx* c, int axis, int ordering, int nf, const double* d_freq,
                         double delta, double delta_a, double delta_r, bool fp32, double2* w,
                         cudaStream_t st);
// chi[f] (+)= M diag(w[f][col0..]) M^H, FP64 tensor cores
cudaError_t launch_contract_f64(const double2* M, long long ldm, long long K, const double2* w,
                                long long ldw, long long col0, int nf, int ng, double2* chi,
                                int accumulate, cudaStream_t st);
// BF16x3 tcgen05 contraction: split, then chi (+)= over the split block (chi zeroed by the caller)
long long tc_kp2(long long K);
int tc_wrows(int nf);   // rows of the float weight scratch (frequencies rounded up to whole jobs)
cudaError_t launch_split_bf16(const void* M, bool m32, long long ldm, long long col0, long long K, int ng,
                              void* hi, void* lo, cudaStream_t st);
// (w32: scratch of tc_wrows(nf) * tc_kp2(K) / 2 complex floats)
cudaError_t launch_contract_bf16x3(const void* hi, const void* lo, long long K, int ng, const double2* w,
                                   long long ldw, long long col0, int nf, void* w32, double2* chi, int* err,
                                   int num_sms, cudaStream_t st);
// the two halves of launch_contract_bf16x3: float copy of the weights, then the tensor-core kernel
cudaError_t launch_weights32(long long K, const double2* w, long long ldw, long long col0, int nf, void* w32,
                             cudaStream_t st);
// (wait_ns: limit of the kernel's pipeline waits; a wait that gives up sets *err and the kernel returns;
// bn: raw rows per tile, one of tc_bn_supported, or <= 0 for tc_pick_bn(ng))
cudaError_t launch_contract_bf16x3_core(const void* hi, const void* lo, long long K, int ng, int nf,
                                        const void* w32, double2* chi, int* err, int num_sms,
                                        unsigned long long wait_ns, cudaStream_t st, int bn);
bool tc_bn_supported(int bn);
int tc_pick_bn(int ng);
int tc_bn_candidates(int* out);     // the supported tile widths (returns their count, out may be NULL)
// seeded finite bf16 operands and float weights for timing runs of the contraction
cudaError_t launch_fill_tune_operands(void* hi, void* lo, long long n_bf16, void* w32, long long n_w32,
                                      cudaStream_t st);
// TF32x3 contraction (mma.sync, FP32 accumulation added into FP64): chi (+)= over K pairs of M
// (complex float when m32, else complex double) from column 0 of the given pointer
cudaError_t launch_contract_tf32x3(const void* M, bool m32, long long ldm, long long K, const double2* w,
                                   long long ldw, long long col0w, int nf, int ng, double2* chi, int accumulate,
                                   cudaStream_t st);
// resident CTAs of the list kernel for matrices of at most nmax rows (0: not available)
int dyson_list_slots(int nmax);
// one cooperative launch of nblocks CTAs over a list of matrices (d_map[b] = {matrix, CTA of it})
// (herm: eps Hermitian positive definite, the lower-triangle sweep without pivoting)
cudaError_t launch_dyson_list(const DysonMat* d_mats, const int2* d_map, int nblocks, int nmax, bool herm,
                              int* err_flag, cudaStream_t st);
// Dyson step; scratch: dyson_scratch_bytes(ng, nf) of device memory (NULL: one CTA per frequency)
size_t dyson_scratch_bytes(int ng, int nf);
cudaError_t launch_dyson(const double2* chi, const double* vs, int ng, int nf, double2* W, void* scratch,
                         bool herm, int* err_flag, cudaStream_t st);
// head row at q -> 0: u_b = qhat.p_b / D_b of the pairs of k in [k0, k0 + nkb) into M[col0 + b] (complex
// float when fp32, else complex double)
cudaError_t launch_head_row(rp_ctx* c, int k0, int nkb, const double qhat[3], bool fp32, void* M, long long col0,
                            cudaStream_t st);
// peak probes: out[0] FP64 FMA, out[1] FP64 mma.sync, out[2] bf16 tcgen05 (TFLOP/s); an rp_status
int probe_peaks(double* out, int num_sms, cudaStream_t st);
// plasma tensor of Eq. plasma added into out[9] (device, zeroed by the caller)
cudaError_t launch_plasma(rp_ctx* c, double ef, double* out, cudaStream_t st);
// rotation of a q matrix: out[f][i][j] = in[f][perm[i]][perm[j]]
cudaError_t launch_rotate(const double2* in, const int* perm, int n, int nf, double2* out, int num_sms,
                          cudaStream_t st);
// interaction step (Sec. 2.4): densities of the Wannier functions, W times their conjugates, bilinear forms
cudaError_t launch_wan_density(const double2* M, long long ldm, int nk, int nw, int nR, const double2* phase,
                               double2* B, int ngp, cudaStream_t st);
cudaError_t launch_wan_wrhs(const double2* W, int ng, int nf, const double2* B, int ngp, const int* pe, int nb,
                            double2* Y, cudaStream_t st);
cudaError_t launch_wan_reduce(const double2* B, int ngp, const double* v, const unsigned char* in_eps, const int* pe,
                              int ng, const double2* Y, int nw, int nR, int nf, const double2* qph, double inv_nq,
                              int accumulate, double2* U, double2* J, cudaStream_t st);

}  // namespace rp
