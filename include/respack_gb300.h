/*
 * respack_gb300.h -- C ABI of the GB300 (sm_103a) polarization / screened-interaction library.
 *
 * The library computes, for one crystal and one k mesh, the plane-wave
 * polarization function chi0_GG'(q, w) of the random-phase approximation and the
 * screened interaction W_GG'(q, w) (Nakamura et al., RESPACK, Comput. Phys.
 * Commun. 2021, arXiv 2001.02351, Sec. 2.3 "Response function with random phase
 * approximation" and Sec. 2.4 "Direct-Coulomb and exchange integrals"):
 *
 *   pair densities   M^G_ab(k+q,k) = <psi_{a,k+q}| e^{i(q+G).r} |psi_{b,k}>      (Eq. ism)
 *   frequency factor X = 1/(w - D + i d) - 1/(w + D - i d),  D = E_{a,k+q} - E_{b,k} (Eq. Xakqbk)
 *                    integrated with generalized-tetrahedron weights x(k)          (Eq. tetrahedron)
 *   polarization     chi_GG' = (2/N_k) sum_{k,a unocc,b occ} (1 - T T) M^G M^G'* x (Eq. chi)
 *   dielectric       eps_GG' = delta_GG' - (4 pi/Omega) chi_GG' / (|q+G||q+G'|)    (Eq. epsGG)
 *   screened         W_GG' = (4 pi/Omega) eps^-1_GG' / (|q+G||q+G'|), plus the bare
 *                    diagonal 4 pi/(Omega |q+G|^2) between the two cut-offs         (Eq. Wq)
 *
 * Units: Hartree atomic units (energies in Ha, lengths in bohr).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Complex arrays are interleaved (re, im) double pairs ("c128"), row-major.
 *  - Ownership: the caller owns every buffer it passes.  rp_load_bands copies the
 *    band data into library-owned device memory; rp_destroy frees it.
 *  - on_device = 1: every array argument marked "[io]" is a device pointer of the
 *    current CUDA device, work is queued on `cuda_stream` (a cudaStream_t, NULL =
 *    legacy default stream) and the call returns without synchronising.
 *    on_device = 0: those arrays are host pointers and the call is synchronous.
 *    Arrays not marked "[io]" are always host pointers.
 *  - Errors: every entry point returns an rp_status.  No exception or abort crosses
 *    the ABI.  rp_last_error(ctx) describes the last failure of that context.  A
 *    context is not thread safe: one thread (one stream) per context at a time.
 *  - k mesh: Gamma-centred, k = (i1/n1, i2/n2, i3/n3) in reciprocal-lattice
 *    coordinates, index k = (i1*n2 + i2)*n3 + i3.  q must be a mesh vector.
 *  - Band pairs: K = N_k * n_emp * n_occ pairs per q, column index
 *    b = (k * n_emp + a) * n_occ + o, with a = alpha - n_occ the empty band at k+q
 *    and o the occupied band at k (bands are 0-based, sorted by energy).
 *  - G lists: the epsilon sphere of q is {G : 0 < 1/2|q+G|^2 <= E_cut^eps} (Sec. 2.3;
 *    G = 0 at q = 0 is left out, the analytic head of Eq. eps00 is not computed),
 *    the tail is {G : E_cut^eps < 1/2|q+G|^2 <= E_cut^psi} (Eq. Wq); both in
 *    lexicographic (m1, m2, m3) Miller order.  NG and N_tail come from rp_sphere_size.
 */
#ifndef RESPACK_GB300_H
#define RESPACK_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rp_ctx rp_ctx;

typedef enum {
    RP_OK = 0,
    RP_ERR_ARG = -1,          /* an argument is out of range or inconsistent        */
    RP_ERR_STATE = -2,        /* called out of order (e.g. no bands loaded)         */
    RP_ERR_OOM = -3,          /* device or host allocation failed                   */
    RP_ERR_CUDA = -4,         /* a CUDA runtime call failed                         */
    RP_ERR_NUMERIC = -5,      /* zero or non-finite pivot in the Dyson solve        */
    RP_ERR_TIMEOUT = -6,      /* a bounded device wait gave up                      */
    RP_ERR_UNSUPPORTED = -7   /* valid request this build does not implement        */
} rp_status;

typedef enum {
    RP_FP64_NATIVE = 0,       /* FP64 pair densities and FP64 tensor-core contraction */
    RP_FP64_EMULATED = 1,     /* reserved (RP_ERR_UNSUPPORTED)                        */
    RP_TF32X3 = 2,            /* FP32 pair densities, FP64 weights, TF32x3 contraction
                                 (mma.sync m16n8k8 TF32, FP32 accumulation added into
                                 FP64 every 16 reals)                                 */
    RP_BF16X3 = 3             /* FP32 pair densities, BF16x3 tcgen05 contraction with
                                 FP32 accumulation flushed to FP64                    */
} rp_precision;

typedef enum { RP_AXIS_REAL = 0, RP_AXIS_IMAG = 1 } rp_axis;          /* w real, or w = i*nu */
typedef enum { RP_TIME_ORDERED = 0, RP_RETARDED = 1 } rp_ordering;
/* RP_TIME_ORDERED is Eq. Xakqbk as printed: X = 1/(w-D+id) - 1/(w+D-id), even in w.
 * RP_RETARDED uses - 1/(w+D+id) for the second term, so that chi(-w) = chi(w)^*. */

/* rp_setup_cell -- crystal, k mesh, FFT grid and cut-offs (Eq. pak; Sec. 2.3).
 *   lat[9]      rows a1, a2, a3 of the direct lattice (bohr).
 *   kmesh[3]    Gamma-centred mesh n1, n2, n3 (each >= 1).
 *   fft[3]      real-space grid N1, N2, N3; each a product of 2s and 3s, 4..128.  It must
 *               hold the wave-function sphere without overlap (checked in rp_load_bands).
 *   ecut_psi_ha wave-function cut-off E_cut^psi (Ha), ecut_eps_ha polarization cut-off
 *               E_cut^eps (Ha), 0 < E_cut^eps <= E_cut^psi.
 *   out         receives a new context (library-owned; free with rp_destroy).
 *   Selects the current CUDA device for the context.  RP_ERR_ARG on bad sizes. */
int rp_setup_cell(const double lat[9], const int kmesh[3], const int fft[3],
                  double ecut_psi_ha, double ecut_eps_ha, rp_ctx** out);

/* rp_load_bands -- Bloch coefficients and energies (Eq. pak; dir-wfn data of Sec. 4).
 *   nk          must equal n1*n2*n3.  nband = nocc + nemp bands per k, nocc >= 1, nemp >= 1.
 *   npw[nk]     number of plane waves at each k;  npw_max >= max(npw) is the row stride.
 *   miller      int [nk][npw_max][3] Miller indices (m1,m2,m3) of k+G, rows past npw ignored.
 *   coef        c128 [nk][nband][npw_max] coefficients C_G,alpha(k), orthonormal per k.
 *   energy_ha   double [nk][nband] band energies (Ha).
 *   T           double [nk][nband] cRPA weights T_alpha,k of Eq. tak in [0,1], or NULL (RPA).
 *   All host pointers; copied to device memory.  RP_ERR_ARG if a sphere does not fit the
 *   FFT grid (two Miller indices congruent modulo the grid). */
int rp_load_bands(rp_ctx* ctx, int nk, int nband, int nocc, const int* npw, int npw_max,
                  const int* miller, const double* coef, const double* energy_ha, const double* T);

/* rp_sphere_size -- epsilon sphere and tail of q.
 *   q_frac[3]   q in reciprocal-lattice coordinates (a k-mesh vector).
 *   ng, n_tail  receive NG and N_tail.  miller_out int [NG][3] or NULL; tail_out int
 *   [N_tail][3] or NULL (host). */
int rp_sphere_size(rp_ctx* ctx, const double q_frac[3], int* ng, int* n_tail,
                   int* miller_out, int* tail_out);

/* rp_transform_grid -- the transform grid the pair densities of q run on (bands loaded, else
 *   RP_ERR_STATE): n_out int[3] (host).  It is the smallest grid with dedicated kernels (16, 24, 32
 *   or 48 points per axis) on which the transforms give the convolution of Eq. ism exactly
 *   (N >= 2 mu + 2 + Lg, mu the bands' largest |Miller| component, Lg the sphere's), when that is
 *   smaller than the cubic grid of rp_setup_cell; else the grid of rp_setup_cell.  window_out:
 *   NULL or the half-width of the residue window of the split tiers' plane kernels (0: none). */
int rp_transform_grid(rp_ctx* ctx, const double q_frac[3], int* n_out, int* window_out);

/* rp_sphere_size_at -- rp_sphere_size for a given epsilon cut-off ecut_eps_ha (0 < ecut_eps_ha
 *   <= Ecut_psi, else RP_ERR_ARG) instead of the context's: the sizes of one member of a batch
 *   with per-q cut-offs (rp_build_chi0_batched). */
int rp_sphere_size_at(rp_ctx* ctx, const double q_frac[3], double ecut_eps_ha, int* ng, int* n_tail,
                      int* miller_out, int* tail_out);

/* rp_pair_density -- M^G_ab(k+q,k) for the pairs of k in [k_begin, k_end) (Eq. ism),
 *   computed as in the paper with Fourier transforms: gather of C onto the real-space
 *   grid, inverse 3D transform, conjugate product, forward 3D transform read back on
 *   the epsilon sphere, normalised by 1/(N1 N2 N3).
 *   M_out [io] c128 [NG][(k_end-k_begin)*nemp*nocc]  (pair columns as above).
 *   FP64 throughout. */
int rp_pair_density(rp_ctx* ctx, const double q_frac[3], int k_begin, int k_end,
                    double* M_out, int on_device, void* cuda_stream);

/* rp_tetra_weights -- pair weights w_b(w) = (2/N_k)(1 - T_{a,k+q} T_{b,k}) x(k; a, b, q, w)
 *   (Eq. chi prefactor times Eq. tetrahedron).
 *   freq_ha[nfreq]  real frequencies (RP_AXIS_REAL) or nu of w = i nu (RP_AXIS_IMAG), Ha.
 *   delta_ha        broadening d of Eq. Xakqbk (>= 0); both poles must stay off the real axis.
 *   delta_a (Ha), delta_r  degeneracy thresholds of Eq. tetrahedron: sorted nodes closer than
 *                   delta_a + delta_r*max(|x|) to their group's first node are merged.
 *   precision       RP_FP64_NATIVE: FP64 throughout.  RP_BF16X3: FP32 evaluation, with every
 *                   node set that has a near degeneracy evaluated again in FP64 (the weights the
 *                   split-precision chi0 path uses).
 *   w_out [io]      c128 [nfreq][K]. */
int rp_tetra_weights(rp_ctx* ctx, const double q_frac[3], int axis, int ordering,
                     int nfreq, const double* freq_ha, double delta_ha, double delta_a,
                     double delta_r, int precision, double* w_out, int on_device, void* cuda_stream);

/* rp_contract_chi0 -- chi[f] = M diag(w[f]) M^H (Eq. chi as a weighted contraction).
 *   ng, K        sizes;  M [io] c128 [ng][K];  w [io] c128 [nfreq][K];
 *   chi_out [io] c128 [nfreq][ng][ng] (overwritten).  precision: RP_FP64_NATIVE, RP_TF32X3
 *   or RP_BF16X3 (M and w are FP64 in all three; the split tiers round them on the device). */
int rp_contract_chi0(rp_ctx* ctx, int ng, long long K, int nfreq, const double* M,
                     const double* w, int precision, double* chi_out, int on_device,
                     void* cuda_stream);

/* rp_build_chi0 -- the whole chi0 path for one q: pair densities, tetrahedron weights and
 *   the contraction, streamed over blocks of k so that M is never held whole.
 *   chi0_out [io] c128 [nfreq][NG][NG].  Other arguments as above.
 *   RP_ERR_TIMEOUT if a bounded wait of the RP_BF16X3 contraction kernel gave up (chi0_out is then
 *   unspecified); with on_device = 1 that status is only known after the stream has run and is
 *   returned by rp_check_numeric. */
int rp_build_chi0(rp_ctx* ctx, const double q_frac[3], int axis, int ordering, int nfreq,
                  const double* freq_ha, double delta_ha, double delta_a, double delta_r,
                  int precision, double* chi0_out, int on_device, void* cuda_stream);

/* rp_build_chi0_kset -- rp_build_chi0 with the k sum of Eq. chi restricted to the nks distinct
 *   mesh points of k_list (host, any order): the pairs (k, a, o) with k in the list contribute, each
 *   with its full-mesh tetrahedron weight, so the chi0 of a partition of the mesh into k sets sums
 *   to the chi0 of the whole mesh.  Used for a sampled reference of a workload too large for a
 *   full FP64 build, and as the unit of a build whose k points are shared out over several GPUs.
 *   chi0_out [io] c128 [nfreq][NG][NG] (overwritten).  RP_ERR_ARG for an index outside [0, N_k) or
 *   a repeated one.  Other arguments and errors as rp_build_chi0. */
int rp_build_chi0_kset(rp_ctx* ctx, const double q_frac[3], int nks, const int* k_list, int axis, int ordering,
                       int nfreq, const double* freq_ha, double delta_ha, double delta_a, double delta_r,
                       int precision, double* chi0_out, int on_device, void* cuda_stream);

/* rp_solve_w -- Dyson step (Eq. epsGG, Eq. Wq) in FP64:
 *   eps = 1 - v^1/2 chi0 v^1/2,  W = v^1/2 eps^-1 v^1/2,  v^1/2_G = sqrt(4 pi/Omega)/|q+G|,
 *   eps^-1 by Gauss-Jordan elimination with partial pivoting, one matrix per frequency.
 *   chi0 [io] c128 [nfreq][NG][NG];  W_out [io] c128 [nfreq][NG][NG];
 *   tail_out [io] double [N_tail] (4 pi/(Omega |q+G|^2) on the tail list) or NULL.
 *   RP_ERR_NUMERIC if a pivot is zero or not finite (W_out is then unspecified); with
 *   on_device = 1 that status is only known after the stream is synchronised and is
 *   returned by the next call of rp_solve_w or by rp_check_numeric. */
int rp_solve_w(rp_ctx* ctx, const double q_frac[3], int nfreq, const double* chi0,
               double* W_out, double* tail_out, int on_device, void* cuda_stream);

/* rp_build_chi0_batched -- rp_build_chi0 for nq q points in one call (the q-point loop of
 *   Eq. chi over the mesh), each with its own epsilon sphere.
 *   q_frac [nq][3] (host); ecut_eps_per_q [nq] Ha (host) or NULL for the context's cut-off;
 *   chi0_out [nq] (host array of pointers), chi0_out[i] [io] c128 [nfreq][NG_i][NG_i] with NG_i
 *   from rp_sphere_size_at.  Frequencies, broadening, thresholds and precision are shared.  The
 *   members are queued in order on cuda_stream; the first failure stops the batch and is
 *   returned (earlier members are complete, later ones untouched). */
int rp_build_chi0_batched(rp_ctx* ctx, int nq, const double* q_frac, const double* ecut_eps_per_q,
                          int axis, int ordering, int nfreq, const double* freq_ha, double delta_ha,
                          double delta_a, double delta_r, int precision, double* const* chi0_out,
                          int on_device, void* cuda_stream);

/* rp_solve_w_batched -- rp_solve_w for the members of a batch: chi0[i], W_out[i] [io] c128
 *   [nfreq][NG_i][NG_i]; tail_out NULL or [nq] pointers (each NULL or double [N_tail,i]);
 *   q_frac and ecut_eps_per_q as in rp_build_chi0_batched.  FP64, errors as rp_solve_w.  Host
 *   buffers: the members are solved one after another and the first failure stops the batch.
 *   Device buffers (on_device = 1, nq > 1, every NG_i >= 16): all (q, w) matrices, largest sphere
 *   first, are packed into a few cooperative launches (consecutive matrices share a launch while
 *   their summed NG^2 stays below about 24 x 904^2; CTAs per matrix in proportion to NG^2); a bad
 *   pivot is reported by rp_check_numeric, the other matrices are still solved.  The Dyson form
 *   (pivoted or Hermitian sweep) follows rp_set_dyson_hermitian. */
int rp_solve_w_batched(rp_ctx* ctx, int nq, const double* q_frac, const double* ecut_eps_per_q, int nfreq,
                       const double* const* chi0, double* const* W_out, double* const* tail_out,
                       int on_device, void* cuda_stream);

/* rp_build_chi0_q0 -- chi0 in the limit q -> 0 along the direction qhat[3] (Cartesian, any length > 0)
 *   for an insulator (band-index occupations), with its head and wings (Sec. 2.3, Eq. eps00 without
 *   the intraband term, Eq. momentum).  The long-wavelength limit of the G = 0 pair density is taken
 *   from k.p: M^0_ao(k+q, k) / |q| -> u_b = qhat.p_ao(k) / (E_ak - E_ok), p_ao = sum_G C_a(k+G)^*
 *   (k+G) C_o(k+G) (exact for a local potential).  RP_ERR_ARG unless the lowest empty band lies above
 *   the highest occupied one at every k.
 *   chi0_out [io] c128 [nfreq][NG+1][NG+1], NG of the epsilon sphere of q = 0 (G != 0): index 0 holds
 *   lim chi_00 / q^2 at [0][0], lim chi_G0 / |q| at [G][0] and lim chi_0G / |q| at [0][G]; indices
 *   1..NG the body, equal to rp_build_chi0 at q = 0.  Other arguments and errors as rp_build_chi0. */
int rp_build_chi0_q0(rp_ctx* ctx, const double qhat[3], int axis, int ordering, int nfreq, const double* freq_ha,
                     double delta_ha, double delta_a, double delta_r, int precision, double* chi0_out,
                     int on_device, void* cuda_stream);

/* rp_solve_w_q0 -- the Dyson step of rp_solve_w for the extended q -> 0 matrix of rp_build_chi0_q0:
 *   eps_00 = 1 - (4 pi/Omega) chi_00/q^2, eps_G0 = -(4 pi/Omega) (chi_G0/|q|) / |G| and its transpose
 *   partner, the body as at q = 0, inverted as one (NG+1) matrix.  W_out [io] c128 [nfreq][NG+1][NG+1]
 *   = v^1/2 eps^-1 v^1/2 with v^1/2 = sqrt(4 pi/Omega) for index 0, so that W_out[f][0][0] is
 *   q^2 W_00 = (4 pi/Omega) eps^-1_00 and W_out[f][G][0] is |q| W_G0 (the q -> 0 divergences taken
 *   out).  tail_out as rp_solve_w at q = 0.  Errors as rp_solve_w. */
int rp_solve_w_q0(rp_ctx* ctx, int nfreq, const double* chi0, double* W_out, double* tail_out, int on_device,
                  void* cuda_stream);

/* rp_rotate_q -- a q matrix at a reducible q from the one at its irreducible q_irr (Sec. 3.1,
 *   Eq. symeps, symmorphic crystal): S int[9] is the rotation as an integer matrix acting on fractional
 *   row vectors (row i holds the image of the i-th reciprocal basis vector), q_irr S = q + G_s with G_s
 *   integer; then X_{G,G'}(q) = X_{G*,G'*}(q_irr) for G = G* S + G_s.  Valid for chi0 (when the k sum
 *   is invariant under S), eps^-1 and W (|q+G| = |q_irr+G*|).  X_irr, X_out [io] c128 [nfreq][NG][NG]
 *   on the epsilon spheres of q_irr and q.  RP_ERR_ARG if S is not a rotation of the lattice, q is
 *   not the image of q_irr or the spheres do not map onto each other. */
int rp_rotate_q(rp_ctx* ctx, const double q_irr[3], const double q_frac[3], const int S[9], int nfreq,
                const double* X_irr, double* X_out, int on_device, void* cuda_stream);

/* rp_plasma -- the intraband plasma frequency of the usual RPA (Sec. 2.3, Eq. plasma), a Fermi-surface
 *   integral over every loaded band:
 *     (w_pl^2)^{mu nu} = (4 pi/Omega)(2/N_k) sum_{k,a} (1 - T_ak^2) p^mu_aa(k) p^nu_aa(k) delta(E_ak - E_F),
 *   p_aa = sum_G |C_a(k+G)|^2 (k+G) (Eq. momentum, local potential), the delta function integrated with
 *   the tetrahedra of the frequency weights (linear interpolation of E_a over each).  omega2_out
 *   double[9] (host, Cartesian, row-major; Ha^2): w_pl^2 for each pair of directions, so that the
 *   Drude term of Eq. eps00 along qhat is qhat.w_pl^2.qhat / (w (w + i delta)).  The bands that cross
 *   E_F must be among the loaded ones.  Synchronous. */
int rp_plasma(rp_ctx* ctx, double fermi_ha, double* omega2_out);

/* rp_optics -- macroscopic optical quantities (Eqs. epsilonM, eels, optical-conductivity,
 *   reflectance) from W00 c128 [nfreq] (host): the elements W_out[f][0][0] of rp_solve_w_q0, i.e.
 *   (4 pi/Omega) eps^-1_00.  out double [nfreq][5] (host): Re eps_M, Im eps_M (eps_M = 1/eps^-1_00),
 *   the loss function -Im eps^-1_00, Re sigma = w Im eps_M / (4 pi) (atomic units; freq_ha[f] real
 *   frequencies) and the normal-incidence reflectivity |(1 - sqrt(eps^-1_00))/(1 + sqrt(eps^-1_00))|^2.
 *   RP_ERR_NUMERIC for a zero or non-finite eps^-1_00.  Host arithmetic only. */
int rp_optics(rp_ctx* ctx, int nfreq, const double* freq_ha, const double* W00, double* out);

/* rp_load_wannier -- Wannier functions of the interaction step (Sec. 2.4): coef c128
 *   [nk][nw][npw_max] (host) holds, for each mesh point k, the plane-wave coefficients of the Bloch
 *   orbitals phi~_ik = sum over lattice vectors R of phi_iR e^{ik.R}, normalised on the crystal like the
 *   bands and given in the plane-wave sets of rp_load_bands (the same Miller lists).  1 <= nw <= 16.
 *   Copied to device memory.  RP_ERR_STATE without bands. */
int rp_load_wannier(rp_ctx* ctx, int nw, const double* coef);

/* rp_interaction -- the term of one q of the screened direct and exchange integrals (Eq. matrix_U,
 *   Eq. matrix_J), or of the bare ones (Eq. matrix_V, Eq. matrix_X) when W is NULL:
 *     U_{i0jR} += (1/N_q) e^{-iq.R} [ sum_{G,G' in eps} n_i(q+G) W_GG' n_j(q+G')^* + sum_{tail} n_i v_G n_j^* ]
 *     J_{i0jR} += (1/N_q)           [ sum_{G,G' in eps} p(q+G) W_GG' p(q+G')^*      + sum_{tail} |p|^2 v_G ]
 *   with n_i(q+G) = (1/N_k) sum_k <phi~_{i,k+q}|e^{i(q+G).r}|phi~_{i,k}> (the Fourier component of
 *   Wannier function i's density), p = p_ijR(q+G) = (1/N_k) sum_k e^{-ik.R} <phi~_{i,k+q}|e^{i(q+G).r}|
 *   phi~_{j,k}> and v_G = 4 pi/(Omega |q+G|^2); W = v^1/2 eps^-1 v^1/2 of rp_solve_w on the epsilon
 *   sphere of q, the tail the rest of the wave-function sphere (bare: the whole sphere with v).
 *   Summing the calls over every q of the mesh gives the integrals.  q = 0, G = 0 is left out.
 *   W [io] c128 [nfreq][NG][NG] or NULL;  R_list int [nR][3] lattice vectors (host, reduced
 *   coordinates);  U_out, J_out [io] c128 [nfreq][nR][nw][nw] ([1][nR][nw][nw] when W is NULL),
 *   overwritten with this q's term (accumulate = 0) or added to (accumulate = 1).  The pair
 *   densities are formed on a transform grid on which nothing folds onto the sphere (the requested
 *   grid, enlarged when needed).  FP64.  nw + nR nw^2 <= 192, else RP_ERR_ARG; RP_ERR_STATE without
 *   rp_load_wannier. */
int rp_interaction(rp_ctx* ctx, const double q_frac[3], int nfreq, const double* W, int nR, const int* R_list,
                   double* U_out, double* J_out, int accumulate, int on_device, void* cuda_stream);

/* rp_check_numeric -- synchronises the context's last stream and reports what the asynchronous
 *   (on_device = 1) calls since the previous check left in the context's device flags:
 *   RP_ERR_TIMEOUT if a bounded device wait of a contraction gave up (its chi0 is unspecified),
 *   else RP_ERR_NUMERIC if an rp_solve_w met a bad pivot, else RP_OK.  Both flags are cleared. */
int rp_check_numeric(rp_ctx* ctx);

/* rp_tune_contraction -- tile autotuner of the RP_BF16X3 contraction kernel (no counterpart in the
 *   paper).  The kernel multiplies tiles of 128 weighted rows by BN rows of M (BN one of 160, 192,
 *   208, 224, 256); for the shape ng x K pairs x nfreq it times one launch of each BN on seeded
 *   synthetic operands in library scratch (CUDA events, after a warm-up launch), records the fastest
 *   for this ng in the context (used by every later RP_BF16X3 contraction with this NG) and
 *   returns it in *bn_out.  ms_out: NULL or double[5], the times of the candidates in the order
 *   above.  Synchronous.  Without a tuned or set choice the kernel takes the BN that pads NG
 *   least (the wider on a tie). */
int rp_tune_contraction(rp_ctx* ctx, int ng, long long K, int nfreq, int* bn_out, double* ms_out);

/* rp_set_contraction_tile -- records BN for contractions with this ng (a choice cached from an
 *   earlier rp_tune_contraction); bn = 0 removes the entry.  RP_ERR_ARG for a BN not built. */
int rp_set_contraction_tile(rp_ctx* ctx, int ng, int bn);

/* rp_probe_peaks -- measurement aid with no counterpart in the paper: the device's FP64 FMA rate,
 *   FP64 tensor (mma.sync m8n8k4) rate and bf16 tcgen05 (M 128, N 256, f32 accumulation) rate in
 *   TFLOP/s, out double[3] (host), each from a small register- or shared-memory-only kernel timed
 *   with CUDA events after a warm-up launch on the current device.  Synchronous.  RP_ERR_TIMEOUT if
 *   the tcgen05 probe's bounded wait gave up. */
int rp_probe_peaks(double* out);

/* rp_set_dyson_hermitian -- on != 0: the Dyson steps of the context (rp_solve_w, rp_solve_w_batched,
 *   rp_solve_w_q0) take eps = 1 - v^1/2 chi0 v^1/2 as Hermitian positive definite, which it is on
 *   the imaginary axis (chi0 Hermitian, negative semidefinite; Eq. epsGG), and invert it by the sweep
 *   operator on its lower triangle without pivoting (half the FP64 work of the pivoted
 *   Gauss-Jordan solve; the upper triangle of chi0 is not read).  A pivot that is not positive
 *   (eps not positive definite, e.g. chi0 of the real axis) is reported like a bad pivot
 *   (RP_ERR_NUMERIC, that frequency's W unspecified).  on = 0: pivoted Gauss-Jordan (the default). */
int rp_set_dyson_hermitian(rp_ctx* ctx, int on);

/* rp_set_fermi -- metals (Sec. 2.3; Eq. Xakqbk with the occupations of a metal): with a Fermi energy
 *   set, the tetrahedron weights of a pair (a, o) integrate each tetrahedron only over its part where
 *   band o (at k) lies below efermi_ha and band a (at k + q) above it, both interpolated linearly
 *   (Fermi-surface clipping: the part is cut into sub-tetrahedra and the generalized tetrahedron
 *   formula applied on each), evaluated in FP64 for every precision tier.  A metal's band list
 *   (rp_load_bands) holds its partly filled bands in both ranges: the first nocc entries are the
 *   bands that may be occupied, the next ones those that may be empty, so a partly filled band is
 *   passed twice and (a, o) of one band with itself is an intraband term.  NaN turns the clipping
 *   off (band-index occupations, the default).  RP_ERR_ARG for an infinite value. */
int rp_set_fermi(rp_ctx* ctx, double efermi_ha);

/* rp_set_pair_budget -- bytes of device scratch the pair-density stage may give to the plane sums of
 *   its pair kernels (default 16 GiB).  The k points are taken in sub-blocks whose plane sums fit;
 *   when one k point's do not, its empty bands are taken in chunks that fit (the pair densities are
 *   the same either way).  bytes >= 1, else RP_ERR_ARG. */
int rp_set_pair_budget(rp_ctx* ctx, long long bytes);

/* rp_set_wait_limit -- testing aid with no counterpart in the paper: the time after which a
 *   bounded device wait of the context's RP_BF16X3 contraction kernel gives up (default 2e9 ns).
 *   A wait that gives up sets the context's timeout flag and the kernel returns through its
 *   teardown (copies and tensor-core operations in flight are drained with the fixed 2 s limit,
 *   tensor memory is freed), so a short limit exercises that path without hanging the device.
 *   limit_ns >= 0, else RP_ERR_ARG. */
int rp_set_wait_limit(rp_ctx* ctx, long long limit_ns);

/* rp_contract_chi0_static -- the RP_BF16X3 contraction of rp_contract_chi0 without any
 *   device allocation, for callers that cannot allocate device memory when they need chi0
 *   (for example a host program that hands the whole device memory budget to its own pool at
 *   start-up and forbids later cudaMalloc calls, or a loop that must not risk the device-wide
 *   synchronisation an allocation can cause).  The paper has no counterpart; this is an
 *   interface variant only.  No context is needed.
 *   ng, K, nfreq  sizes;  M c128 [ng][K], w c128 [nfreq][K] and chi_out c128 [nfreq][ng][ng] are
 *                 device pointers of the current device owned by the caller; work is queued on
 *                 cuda_stream and the call returns without synchronising.
 *   Scratch: a 64 MiB array inside the library, held by every GPU that loads it until the
 *   process exits.  Limits: with kp2 = 2 K rounded up to a multiple of 64,
 *   ng * kp2 <= 12582912 and 4 * ceil(nfreq / 4) * kp2 / 2 <= 1048576; larger requests return RP_ERR_ARG
 *   before anything is queued.  The first call on a device looks up the array's device address
 *   (once per device); make that first call before any stream capture.  Every call uses the
 *   same array: calls whose work overlaps on the GPU (other streams, other threads) race and
 *   must be serialised by the caller.  A device-side wait that gives up leaves chi_out
 *   unspecified and sets a flag in the array; rp_contract_chi0_static_status reports it.
 *   Returns RP_OK, RP_ERR_ARG or RP_ERR_CUDA. */
int rp_contract_chi0_static(int ng, long long K, int nfreq, const double* M, const double* w,
                            double* chi_out, void* cuda_stream);

/* rp_contract_chi0_static_status -- synchronises cuda_stream and returns RP_ERR_TIMEOUT if the
 *   last rp_contract_chi0_static on the current device had a device-side wait give up (the flag
 *   in the library's array is then cleared), RP_OK if not, RP_ERR_CUDA if the synchronisation or
 *   the read failed.  Allocates nothing.  Call it after the call it checks and before the next
 *   one (each call clears the flag when it starts).  No counterpart in the paper. */
int rp_contract_chi0_static_status(void* cuda_stream);

/* rp_profile_enable -- measurement aid (no counterpart in the paper).  enable = 1 starts
 *   recording a CUDA event pair on the launching stream around every stage of the path and
 *   counting kernel launches per stage; enable = 0 stops.  Either call resets the totals.
 * rp_profile_read -- synchronises the context's last stream and returns, per stage,
 *   the summed device time (ms) and the number of kernels launched since the last reset.
 *   Stages: 0 gather + inverse transform, 1 pair product + forward transform + read-back,
 *   2 tetrahedron weights, 3 chi0 contraction kernel, 4 Dyson solve, 5 operands of the split
 *   contraction (bf16 split of M and float weights of each block).  ms[6], launches[6] (host). */
int rp_profile_enable(rp_ctx* ctx, int enable);
int rp_profile_read(rp_ctx* ctx, double* ms, long long* launches);

/* rp_last_error -- text of the last failure of ctx (valid until the next call on ctx). */
const char* rp_last_error(const rp_ctx* ctx);

/* rp_destroy -- frees the context and all library-owned device memory. */
void rp_destroy(rp_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
