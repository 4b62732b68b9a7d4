/*
 * ap.h -- C-ABI of the GB300 adaptive-precision EAM/ACE force evaluation.
 *
 * Method: "Adaptive-precision potentials for large-scale atomistic simulations"
 * (arXiv 2411.03002).  Each atom i carries a switching parameter lambda_i in [0,1]
 * (the fast weight): E_i = lambda_i E_i^(f) + (1 - lambda_i) E_i^(p) (Eq. energy_hyb),
 * with E^(f) an embedded-atom model (Eq. energy_eam) and E^(p) a linear atomic
 * cluster expansion (Eq. energy_ace).  lambda_i comes from the time-averaged
 * centro-symmetry parameter (Eq. csp_1_i, Appendix A) through the switching
 * function of Appendix B (Eqs. csp_2_i, lambda_1_i .. lambda_4_i).  Forces are
 * the fixed-lambda gradient F_i^d (Eq. F_i_d, section 2.3); time integration is
 * velocity Verlet with the lambda step (Eq. vv).
 *
 * Conventions for every entry point:
 *   - Return value: ap_status, AP_OK (0) on success.  Nothing throws across the
 *     ABI.  ap_last_error(ctx) returns a message for the last failure.
 *   - Pointers named d_* are caller-owned DEVICE pointers (contiguous, CUDA
 *     global memory of the current device); pointers named h_* are caller-owned
 *     HOST pointers.  The library never frees caller memory.  It owns only the
 *     scratch held in the context (neighbour lists, histories, queues), which it
 *     allocates on first use and grows when a larger n arrives.
 *   - Arrays of 3-vectors are row-major [n][3] (x0 y0 z0 x1 ...).
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream) unless a comment says the call synchronises.
 *   - A context is bound to one device and is not thread-safe.
 *   - lambda is always the paper's lambda (1 = fast/EAM, 0 = precise/ACE).
 *   - Units: eV, Angstrom, fs, amu.
 */
#ifndef AP_H
#define AP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ap_status;

#define AP_OK 0
#define AP_ERR_ARG 1        /* invalid argument (null pointer, bad size, bad config)   */
#define AP_ERR_CUDA 2       /* a CUDA runtime call failed                              */
#define AP_ERR_CAPACITY 3   /* a neighbour row exceeded its capacity; see ap_need()    */
#define AP_ERR_NONFINITE 4  /* NaN/Inf found in positions or forces                    */
#define AP_ERR_TIMEOUT 5    /* a bounded device wait gave up (the kernel returned early) */
#define AP_ERR_STATE 6      /* call order violated (e.g. evaluation before neighbours) */
#define AP_ERR_RADICAND 7   /* a local-thermostat correction had a negative radicand   */
#define AP_ERR_BOX 8        /* an atom lies outside a non-periodic box dimension       */
#define AP_ERR_SKIN 9       /* an atom moved more than skin/2 between list rebuilds    */

#define AP_PREC_FP64 0      /* all potential arithmetic in FP64                        */
#define AP_PREC_MIXED 1     /* FP32 potentials; FP64 integration and energy sums       */

#define AP_DETECT_CSP 0      /* f_cut argument from the averaged centro-symmetry (Eq. lambda_1_i) */
#define AP_DETECT_SELECTOR 1 /* f_cut argument from the averaged selector score p (ap_sel_*)     */

#define AP_SEL_NFEAT 24      /* selector features per atom                              */
#define AP_SEL_NHID 64       /* hidden width of the selector MLP                        */
#define AP_SEL_NPARAMS 5825  /* 24*64 + 64 + 64*64 + 64 + 64 + 1                        */

#define AP_EAM_ANALYTIC 0   /* eam_type: the analytic synthetic EAM (eam_beta .. eam_h)     */
#define AP_EAM_MISHIN 1     /* eam_type: Mishin EAM2 copper (Appendix E), eam_mishin[]      */

#define AP_REBUILD_SKIN (-1) /* rebuild_every: rebuild on the skin criterion (see ap_config) */

#define AP_FCUT_PRINTED 0   /* f_cut(x) = 1 - 1.875x + 1.25x^3 - 0.375x^5 as printed    */
#define AP_FCUT_C2 1        /* C2-symmetric reading 0.5*p(2x-1)                         */

/* Orthorhombic box: lo <= x < hi in periodic dimensions (positions may be
 * unwrapped; the library works with images); in non-periodic dimensions every
 * atom must satisfy lo <= x < hi, else AP_ERR_BOX. */
typedef struct {
  double lo[3];
  double hi[3];
  int32_t periodic[3];
} ap_box;

/* Every parameter of one run.  Plain data; copied by ap_create. */
typedef struct {
  /* EAM (Eq. energy_eam) with the analytic forms
   *   zeta(r) = exp(-beta (r/r0 - 1)) psi((r - rc)/h),
   *   xi(rho) = -A sqrt(rho),
   *   Phi(r)  = D [exp(-2 alpha (r - rp)) - 2 exp(-alpha (r - rp))] psi((r - rc)/h),
   *   psi(x)  = x^4/(1 + x^4) for x < 0, else 0. */
  double eam_beta, eam_alpha, eam_A, eam_D, eam_rp, eam_r0, eam_rc, eam_h;
  /* Linear ACE (Eq. energy_ace): E_i = sum_v c_v B_iv.  Radial basis
   * g_k(r) = T_k(2r/rc - 1) f_cut(r/rc), R_nl = sum_k W[l][n][k] g_k (n,k < 8,
   * l <= 4); A_nlm = (1/n0) sum_j R_nl Y_lm; B: nu = 1, 2 (all n1 <= n2, l) and 3
   * (n <= 2, l <= 3, Gaunt-coupled), 325 functions ordered nu = 1 by n, nu = 2 by
   * (n1, n2, l), nu = 3 by (p1 <= p2 <= p3) with p = 4n + l (ap_ace_basis_desc lists
   * them).  ace_c holds ace_nc >= 325 coefficients (extra ignored). */
  double ace_W[5 * 8 * 8];
  double ace_c[512];
  int32_t ace_nc;
  double ace_rc, ace_n0;
  /* Switching function (Appendix B, Table model_parameters). */
  double csp_lo, csp_hi;     /* Angstrom^2 */
  double r_lo, r_hi;         /* lambda spread radii, Angstrom */
  double dlam_min;           /* minimum lambda step */
  int32_t n_csp_avg;         /* samples in the CSP moving average */
  int32_t n_lam_avg;         /* samples in the lambda_min moving average */
  int32_t fcut_mode;         /* AP_FCUT_* */
  /* Neighbour lists: radius = potential cutoff + skin.  cap_* = entries per row
   * (0 selects 160 for EAM and 288 for ACE). */
  double skin;
  int32_t cap_eam, cap_ace;
  int32_t precision;         /* AP_PREC_* */
  /* Molecular dynamics (ap_step). */
  double dt;                 /* fs */
  int32_t lambda_every;      /* lambda update and list rebuild period (steps) */
  int32_t indenter_on;       /* 1: spherical indenter F = k (R - r)^2 (x - c)/r, r < R */
  double ind_c0[3], ind_v[3], ind_R, ind_k;   /* centre at t=0 (A), velocity (A/fs), R (A), k (eV/A^3) */
  int32_t rebuild_every;     /* neighbour rebuild period (steps); 0 = lambda_every.  Every
                                lambda update also rebuilds, so the CSP sees fresh rows.
                                AP_REBUILD_SKIN: ap_step reads the largest displacement
                                since the last build after every drift (a stream sync
                                per step) and rebuilds when it exceeds skin/2; a lambda
                                update keeps the lists while it is at most 0.45 skin
                                and takes the CSP from them where they decide it (12
                                candidates inside r_search - 2 x that displacement; any
                                atom that fails this makes the update rebuild after
                                all).  The precise queue's ACE rows (ace_rc + skin)
                                are checked the same way against their own build and
                                rebuilt alone when needed.  Lambda and the forces equal
                                those of a rebuild at the update.  Lists are kept only with
                                AP_DETECT_CSP, without the local thermostat, and when
                                every periodic dimension of every system holds at least
                                2 ceil((ace_rc + 2 skin)/h) + 1 cells (h the cell
                                edge) or the offsets are stored; otherwise each update
                                rebuilds (the per-step check stays). */
  /* Detector behind lambda_0 (Appendix B allows any detector whose f_cut argument
   * is 0 for precise and 1 for fast atoms).  AP_DETECT_SELECTOR pushes the
   * selector's p_i in [0,1] into the history in place of CSP_i and uses
   * lambda_0 = 1 - f_cut((sel_p_hi - p_avg)/(sel_p_hi - sel_p_lo)); it needs a
   * model (ap_sel_set_model).  Ignored with AP_DETECT_CSP. */
  int32_t detector;
  double sel_p_lo, sel_p_hi;
  /* Local thermostat (section 2.3 and Appendix C), used by ap_step on every lambda
   * update when 1.  With lambda^c the values before the update and lambda^d after
   * it, each mobile atom's energy error
   *   Delta E_i = Delta T_i + Delta V_i,
   *   Delta V_i = (lambda_i^c - lambda_i^d)(E_i^f - E_i^p)                  (Eq. Delta_V_i)
   *   Delta T_i = sum_a [dt^2/(8 m_i)(F^c_ia^2 - F^d_ia^2) + (F^c_ia - F^d_ia) v_ia(t+dt/2) dt/2]
   * (interatomic forces only) is corrected at the end of the step by rescaling the
   * relative momenta of Omega_i = {i} + the distinct mobile atoms of its EAM row:
   * v_j <- v_cm + beta (v_j - v_cm), beta = sqrt(Delta E_i / K_rel + 1) (Eqs.
   * p_resc_omega, beta_omega_i).  Rows hold at most cap_eam atoms, below the
   * paper's 800, so no random draw is made.  Corrections run in an 8-colour sweep
   * over cells of edge >= 2 (eam_rc + 2 skin) (ascending index inside a cell),
   * the sub-domain order the paper leaves open; groups in cells of one colour are
   * disjoint.  A negative radicand skips that correction and makes ap_step return
   * AP_ERR_RADICAND.  One system only (not with ap_build_neighbors_batch). */
  int32_t thermostat_on;
  /* Finnis-Sinclair ACE form (Eq. energy_ace, nonlinear part): with ace_fs_on = 1,
   * E_i^(p) = phi_i^(1) + F(phi_i^(2)), phi^(1) = sum c_v B_iv (ace_c) and
   * phi^(2) = sum c2_v B_iv (ace_c2, the same basis and ace_nc), and the embedding
   * F(phi) = sign(phi) (sqrt(|phi| + eps^2) - eps), eps = ace_fs_eps > 0: the paper's
   * sqrt(phi) up to the constant -eps and O(eps^2/sqrt(phi)), defined and C1 for every
   * real phi.  0 = linear ACE (E = phi^(1)). */
  int32_t ace_fs_on;
  double ace_fs_eps;
  double ace_c2[512];
  /* Fast potential.  AP_EAM_ANALYTIC: the analytic forms above.  AP_EAM_MISHIN: the
   * EAM2 forms of Appendix E with
   *   Phi(r)  = (E1 M(r; r01, a1) + E2 M(r; r02, a2) + delta) psi((r - rc)/h)
   *             - sum_{n=1..3} [r <= rs_n] S_n (rs_n - r)^4,
   *             M(r; r0, a) = exp(-2a(r - r0)) - 2 exp(-a(r - r0)),
   *   zeta(r) = (a exp(-b1 (r - r03)^2) + exp(-b2 (r - r04))) psi((r - rc)/h),
   *   xi(x)   = F0 + xi0 + xi2/2 y^2 + q1 y^3 + q2 y^4 + q3 y^5 + q4 y^6   (x <= 1),
   *           = F0 + (xi0 + xi2/2 y^2 + q1 y^3 + Q1 y^4)/(1 + Q2 y^3)    (x > 1),  y = x - 1,
   * and eam_mishin holding E1, E2, delta, F0, xi0, xi2, h, q1, q2, q3, q4, Q1, Q2,
   * S1, S2, S3, a, a1, a2, b1, b2, r01, r02, r03, r04, rs1, rs2, rs3, rc in that order
   * (eV, Angstrom).  The EAM neighbour rows still use eam_rc + skin, so eam_rc must be
   * >= the Mishin rc; eam_beta .. eam_h other than eam_rc are then unused.  The
   * selector detector and ap_eval_eam_static accept AP_EAM_ANALYTIC only. */
  int32_t eam_type;
  double eam_mishin[29];
  /* ACE force reduction.  0: each neighbour pair's contribution is scattered with
   * floating-point atomics (FP32 vector atomics in mixed precision), so the summation
   * order, and with it the last bits of the forces, varies from run to run.  1: each
   * contribution is rounded to a multiple of 2^-36 eV/A (an error of at most 2^-37 per
   * contribution) and summed with 64-bit integer atomics, which are exact and
   * independent of the order: forces, and ap_step trajectories, are bitwise
   * reproducible on one GPU model.  Accumulated forces must stay below 2^27 eV/A. */
  int32_t ace_deterministic;
} ap_config;

typedef struct ap_ctx ap_ctx;

/* Statistics written by ap_step (host struct). */
typedef struct {
  int64_t step;              /* MD steps done by this context so far */
  int64_t n_precise;         /* |{i : lambda_i < 1}| after the last update */
  int64_t n_detected;        /* |{i : lambda_0,i < 1}| after the last update */
  int64_t rebuilds;          /* neighbour-list rebuilds so far */
  double e_pot;              /* sum_i E_i (Eq. energy_hyb) + indenter energy, FP64 */
  double e_kin;              /* sum_i m v^2 / 2, FP64 */
  double max_disp;           /* largest displacement since the last rebuild (A) */
  int32_t error_bits;        /* OR of 1 << AP_ERR_* seen on the device */
  int64_t th_corrected;      /* local-thermostat corrections applied so far */
  int64_t th_refused;        /* corrections refused for a negative radicand so far */
  double th_energy;          /* sum of the corrected Delta E so far (eV) */
  int64_t kept;              /* lambda updates that kept the lists (AP_REBUILD_SKIN) so far */
  int64_t ace_rebuilds;      /* ACE row builds between lambda updates (AP_REBUILD_SKIN) so far */
} ap_step_stats;

/* ----------------------------------------------------------------- lifetime */

/* Create a context on the current CUDA device.  Builds the ACE coupling tables
 * on the host (real Gaunt coefficients from the Racah formula).  Synchronous.
 * Errors: AP_ERR_ARG for a null pointer or an invalid config. */
ap_status ap_create(const ap_config* h_cfg, ap_ctx** out);

/* Free all library-owned device memory.  Synchronises the device. */
void ap_destroy(ap_ctx* ctx);

/* Static message of the last error of ctx (never NULL). */
const char* ap_last_error(const ap_ctx* ctx);

/* Required capacity after AP_ERR_CAPACITY (largest row count seen). */
int64_t ap_need(const ap_ctx* ctx);

/* Number of ACE B-functions (325) and their description: h_desc[v*7 + 0..6] =
 * nu, n1, n2, n3, l1, l2, l3 (unused slots 0). */
int32_t ap_ace_nbasis(const ap_ctx* ctx);
ap_status ap_ace_basis_desc(const ap_ctx* ctx, int32_t* h_desc);

/* Real Gaunt coefficients used by the nu = 3 couplings, computed on the host
 * from the Racah 3j formula: h_out[((((l1*7+m1+3)*4+l2)*7+m2+3)*4+l3)*7+m3+3]. */
ap_status ap_ace_gaunt(const ap_ctx* ctx, double* h_out);

/* ----------------------------------------------------------------- neighbours */

/* Cell list (section 2.4: per-domain neighbour search) and full neighbour rows
 * at eam_rc + skin for every atom: j in row i iff (j,s) != (i,0) and
 * |x_j + s L - x_i|^2 < (eam_rc + skin)^2 in FP64 (the defining arithmetic; FP32
 * is only a pre-filter with a guard band).  d_x [n][3] FP64 positions, possibly
 * unwrapped.  d_species may be NULL (single species; nonzero entries are an
 * error).  Synchronises to check capacity; grows the rows and rebuilds once if a
 * row overflowed.  Errors: AP_ERR_ARG, AP_ERR_BOX, AP_ERR_CAPACITY, AP_ERR_CUDA. */
ap_status ap_build_neighbors(ap_ctx* ctx, int64_t n, const double* d_x, const int32_t* d_species,
                             const ap_box* h_box, void* stream);

/* Same for n_sys independent systems concatenated in d_x: system s owns atoms
 * [h_offsets[s], h_offsets[s+1]) and box h_boxes[s].  No pair crosses systems. */
ap_status ap_build_neighbors_batch(ap_ctx* ctx, int32_t n_sys, const int64_t* h_offsets, const ap_box* h_boxes,
                                   const double* d_x, const int32_t* d_species, void* stream);

/* Export the neighbour rows (which = 0: EAM rows of all atoms; 1: ACE rows of
 * the last precise queue, radius ace_rc + skin).  d_cnt [rows], d_idx
 * [rows][cap], d_shift [rows][cap][3] = s of each entry relative to the d_x of
 * the build.  *h_rows receives the number of rows.  Synchronises.  An EAM row
 * lists the entries inside the potential's cutoff at the build (by an FP32 test)
 * before the skin entries; within each part the order is the build's own. */
ap_status ap_get_neighbors(ap_ctx* ctx, int32_t which, int32_t* d_cnt, int32_t* d_idx, int32_t* d_shift, int64_t cap,
                           int64_t* h_rows);

/* The atoms in the spatial order of the last neighbour build: d_order[k] (int32, [n]
 * device) is the k-th atom of the cell list, cells in raster order (x fastest) and
 * atoms of a cell by index; with batched systems each system's atoms stay in its own
 * range.  Applying this permutation to the caller's per-atom arrays (x_new = x[order],
 * and the same for v, masses, lambda ...) puts neighbours close in memory, which the
 * EAM and ACE gathers depend on: a randomly ordered 4M-atom slab runs 33 % slower than the
 * same slab in this order.  No paper counterpart (LAMMPS sorts atoms for the same
 * reason).  Errors: AP_ERR_STATE before ap_build_neighbors, AP_ERR_ARG for a null
 * pointer. */
ap_status ap_spatial_order(ap_ctx* ctx, int32_t* d_order, void* stream);

/* Total number of entries in the current EAM rows (which = 0) or ACE rows (which = 1,
 * the precise queue's rows), or the EAM row prefixes that the last EAM force pass
 * walked (which = 2: per atom, one past the last entry that the density pass found
 * inside the potential's cutoff), summed on the device by one reduction kernel;
 * *h_total is a host pointer.  Synchronises the legacy default stream.  No paper
 * counterpart: instrumentation (the EAM density pass reads the which = 0 entries, the
 * force pass the which = 2 ones, every MD step).  Errors: AP_ERR_STATE before
 * ap_build_neighbors, or for which = 2 before an EAM evaluation on the current rows;
 * AP_ERR_ARG for a null pointer or another `which`. */
ap_status ap_neighbor_total(ap_ctx* ctx, int32_t which, int64_t* h_total);

/* ----------------------------------------------------------------- lambda */

/* One lambda update (Appendix B) from the current neighbour rows, in FP64 with
 * the arithmetic order of the definitions (bit-reproducible sets):
 *   CSP_i: 12 nearest neighbours within eam_rc + skin (fewer -> +inf), the 6
 *     smallest |r_a + r_b|^2 summed in ascending order (Eq. csp_1_i, Appendix A);
 *   CSP_avg: mean of the last n_csp_avg samples incl. this one (Eq. csp_2_i);
 *   lambda_0 = 1 - f_cut((csp_hi - CSP_avg)/(csp_hi - csp_lo)) (Eq. lambda_1_i);
 *   lambda_min: minimum over detected atoms within r_hi (Eq. lambda_2_i);
 *   lambda_avg: mean of the last n_lam_avg lambda_min samples (Eq. lambda_3_i);
 *   lambda = lambda_avg,msz (Eq. lambda_4_i).
 * d_changeable [n] uint8 (NULL = all changeable; 0 = lambda fixed at 1).
 * sample_now = 1: the update above, pushing this call's CSP and lambda_min samples
 * into the histories; sample_now = 0: no sample, the lambda of the last update and
 * its queue are returned (d_x unused; AP_ERR_STATE without an earlier update).
 * Outputs: d_lam [n] FP64; d_precise_idx [n] int32 = ascending indices with
 * lambda < 1 (the precise work queue); d_n_precise device int64 (may be NULL).
 * The first sampling call after creation or ap_reset_lambda fills the histories
 * with its sample.  Requires a neighbour build at the same positions for exact
 * CSP candidates. */
ap_status ap_classify(ap_ctx* ctx, int64_t n, const double* d_x, const uint8_t* d_changeable, int32_t sample_now,
                      double* d_lam, int32_t* d_precise_idx, int64_t* d_n_precise, void* stream);

/* The precise work queue of a given lambda (section 2.4: only atoms with
 * lambda_i < 1 need the precise potential): d_queue[0..k) = the ascending
 * indices i with d_lam[i] < 1, *d_n_queue (device int64) = k.  d_lam [n] FP64,
 * d_queue [n] int32.  Uses the context's scratch: needs a neighbour build on at
 * least n atoms before (AP_ERR_STATE otherwise). */
ap_status ap_precise_queue(ap_ctx* ctx, int64_t n, const double* d_lam, int32_t* d_queue, int64_t* d_n_queue,
                           void* stream);

/* Forget the CSP/lambda histories and the previous lambda. */
ap_status ap_reset_lambda(ap_ctx* ctx);

/* Copy intermediate arrays of the last ap_classify (any pointer may be NULL):
 * CSP sample, CSP_avg, lambda_0, lambda_min, lambda_avg (each [n] FP64). */
ap_status ap_get_lambda_state(ap_ctx* ctx, double* d_csp, double* d_csp_avg, double* d_lam0, double* d_lam_min,
                              double* d_lam_avg, void* stream);

/* ----------------------------------------------------------------- potentials */

/* EAM for every atom (Eq. energy_eam) with lambda weights (Eq. F_i_d):
 *   d_e_fast[i] = xi(rho_i) + 1/2 sum_j Phi(r_ij)              (written, FP64)
 *   d_f[i]     += -grad_i sum_k lambda_k E_k^(f)  at fixed lambda (accumulated)
 * d_lam [n] FP64 (NULL = all 1).  d_feat [n][24] FP32 (may be NULL): the
 * selector's EAM-level features of every atom (ap_sel_features with all atoms
 * changeable; analytic EAM only, AP_ERR_ARG otherwise); computing them replaces the
 * CSP sample that ap_get_lambda_state returns.  Requires ap_build_neighbors on the
 * same n. */
ap_status ap_eval_eam(ap_ctx* ctx, int64_t n, const double* d_x, const double* d_lam, double* d_e_fast, double* d_f,
                      float* d_feat, void* stream);

/* Linear ACE for the atoms of the precise queue (Eq. energy_ace) with weights
 * w_i = 1 - lambda_i:
 *   d_e_prec[i] = E_i^(p) for i in the queue, 0 for every other atom  (written)
 *   d_f[k]     += -grad_k sum_i w_i E_i^(p)                           (accumulated)
 * d_precise_idx [*d_n_precise] int32 atom indices (e.g. from ap_classify);
 * d_n_precise is a DEVICE int64.  Builds the ACE rows (ace_rc + skin) for the
 * queue; the ACE storage (rows, pair records, per-atom scratch) is sized for the
 * queue's length, read back with one synchronisation of the stream, and grows
 * when a longer queue arrives.  d_f may be NULL (energies only). */
ap_status ap_eval_ace(ap_ctx* ctx, int64_t n, const double* d_x, const double* d_lam, const int32_t* d_precise_idx,
                      const int64_t* d_n_precise, double* d_e_prec, double* d_f, void* stream);

/* Blend (Eq. energy_hyb): d_e_atom[i] = lambda_i e_fast_i + (1 - lambda_i) e_prec_i
 * (FP64) and d_e_total (device double) = sum_i d_e_atom[i] by a fixed-order
 * tree reduction (bitwise reproducible).  d_e_atom may be NULL. */
ap_status ap_blend_forces(ap_ctx* ctx, int64_t n, const double* d_lam, const double* d_e_fast, const double* d_e_prec,
                          double* d_e_atom, double* d_e_total, void* stream);

/* ----------------------------------------------------------------- dynamics */

/* nsteps of velocity Verlet with the lambda step (Eq. vv), all on the device:
 * half kick, drift, [every lambda_every steps: wrap, neighbour rebuild, lambda
 * update, precise queue], EAM + ACE forces at the new lambda, indenter, half kick.
 * Fixed atoms (d_fixed[i] != 0) keep v = 0, do not move and keep lambda = 1.
 * On the first call the context prepares neighbours, lambda and F(x(0)) itself.
 * d_x, d_v, d_f [n][3] FP64 in/out; d_mass [n] FP64; d_fixed [n] uint8 or NULL;
 * d_lam [n] FP64 out.  h_stats (may be NULL) is filled at the end.  The call
 * synchronises the stream at its end and at every rebuild: there it checks the
 * error bits so far (an error ends the call), grows the EAM rows if one overflowed,
 * and reads the new precise queue's length to size the ACE storage for it.  With
 * rebuild_every = AP_REBUILD_SKIN it also synchronises after every drift.
 * Errors: as above plus AP_ERR_SKIN (an atom moved more than skin/2 before a
 * rebuild; never with AP_REBUILD_SKIN) and AP_ERR_NONFINITE. */
ap_status ap_step(ap_ctx* ctx, int64_t n, double* d_x, double* d_v, double* d_f, const double* d_mass,
                  const uint8_t* d_fixed, double* d_lam, int64_t nsteps, ap_step_stats* h_stats, void* stream);

/* ----------------------------------------------------------------- selector */

/* The selector is a learned detection score that can replace the centro-symmetry
 * argument of f_cut (Appendix B: any detector whose argument is 0 for atoms to be
 * computed precisely and 1 for atoms to be computed fast).  The paper prescribes no
 * detector of this kind; its definition is this library's:
 *   features (24 per atom, FP32, from the EAM rows; N = pairs with r < 5.5 A,
 *   S1 r < 3.09, S2 3.09 <= r < 4.02, S3 4.02 <= r < 4.77 A; empty sets give 0):
 *     0 rho_i  1 xi(rho_i)  2 xi'(rho_i)  3 1/2 sum_N Phi  4-6 |S1| |S2| |S3|
 *     7 min(CSP_i, 100)  8 sum_{j in S2} min(r_j^2, min_{k in S2\j} |r_j + r_k|^2)
 *     9-11 |sum r_j| over S1, S2, N  12 |sum_N zeta'(r_j) r_j/r_j|
 *     13 rho_i - mean_{S1} rho_j  14-17 mean, std, min, max of r over S1
 *     18-21 mean, std, third and fourth central moments of r over N  22 |N|
 *     23 mean_N xi'_j - xi'_i
 *   network: x~ = bf16((x - mu) * inv_sigma) (FP32 arithmetic);
 *     h1 = bf16(relu(x~ W1 + b1)); h2 = relu(h1 W2 + b2); z = h2 . w3 + b3;
 *     p = 1/(1 + exp(-z)), with W1, W2, w3 used as bf16 and FP32 accumulation
 *     (tcgen05 tensor cores for the two hidden layers).
 *   training: loss = sum_b w_b [softplus(z_b) - y_b z_b] (weights as given, e.g.
 *     normalised to sum 1), gradient straight through the bf16 roundings, Adam
 *     with bias correction on FP32 master weights (m = b1 m + (1-b1) g,
 *     v = b2 v + (1-b2) g^2, theta -= lr (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps)).
 * Flat parameter layout (AP_SEL_NPARAMS floats): W1 [24][64] (input-major), b1 [64],
 * W2 [64][64] (input-major), b2 [64], w3 [64], b3. */

/* Load a model: h_params [AP_SEL_NPARAMS], h_mu [24], h_inv_sigma [24] (host FP32,
 * finite).  Resets the Adam state.  Synchronises.  Errors: AP_ERR_ARG. */
ap_status ap_sel_set_model(ap_ctx* ctx, const float* h_params, const float* h_mu, const float* h_inv_sigma);

/* Copy the FP32 master parameters (and mu, inv_sigma; any pointer may be NULL)
 * to host memory.  Synchronises.  Errors: AP_ERR_STATE without a model. */
ap_status ap_sel_get_model(ap_ctx* ctx, float* h_params, float* h_mu, float* h_inv_sigma);

/* Raw features d_feat [n][24] FP32 of every atom at positions d_x.  Requires
 * ap_build_neighbors on the same n and positions.  Computes the CSP sample of
 * every changeable atom (d_changeable as in ap_classify) on the way, which
 * replaces the one ap_get_lambda_state returns.  Errors: AP_ERR_STATE without
 * neighbours, AP_ERR_ARG with eam_type other than AP_EAM_ANALYTIC (the features
 * are the analytic EAM's pair terms). */
ap_status ap_sel_features(ap_ctx* ctx, int64_t n, const double* d_x, const uint8_t* d_changeable, float* d_feat,
                          void* stream);

/* p = sigmoid(z) of n raw feature rows d_feat [n][24]: d_p [n] FP32 (may be NULL),
 * d_logit [n] FP32 (may be NULL).  Errors: AP_ERR_STATE without a model. */
ap_status ap_sel_predict(ap_ctx* ctx, int64_t n, const float* d_feat, float* d_p, float* d_logit, void* stream);

/* One Adam step on a batch of b samples: rows d_idx[0..b) of d_feat [*][24],
 * d_label [*] (0 or 1) and d_weight [*] (d_idx NULL: rows 0..b).  d_loss (device
 * float, may be NULL) receives the batch loss before the step.  The gradient is
 * reduced in a fixed order (bitwise reproducible on one GPU model).
 * Errors: AP_ERR_STATE without a model, AP_ERR_ARG for b < 1. */
ap_status ap_sel_train_step(ap_ctx* ctx, int64_t b, const float* d_feat, const int32_t* d_idx, const float* d_label,
                            const float* d_weight, float lr, float beta1, float beta2, float eps, float* d_loss,
                            void* stream);

/* Gradient (h_grad [AP_SEL_NPARAMS], may be NULL) and loss (*h_loss, may be NULL)
 * of the last ap_sel_train_step.  Synchronises; reports AP_ERR_TIMEOUT if a
 * tensor-core wait gave up. */
ap_status ap_sel_get_grad(ap_ctx* ctx, float* h_grad, float* h_loss);

/* ----------------------------------------------------------------- allocation-free EAM */

/* The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory at all (for instance code that runs inside a
 * process whose device memory belongs to another runtime's pool, or a
 * deployment whose memory budget is fixed before it starts).  It computes what
 * ap_eval_eam computes -- d_e_fast[i] = xi(rho_i) + 1/2 sum_j Phi(r_ij) (written)
 * and d_f[i] += -grad_i sum_k lambda_k E_k^(f) at fixed lambda (accumulated) --
 * for one system of at most 32768 atoms, in FP64, with pairs found by brute force
 * over all atoms and periodic images (O(n^2): meant for small systems).  It needs
 * no context and calls no allocator.  Only the EAM fields of h_cfg are read.
 * d_x [n][3], d_lam [n] (NULL = all 1), d_e_fast [n], d_f [n][3]: device
 * pointers owned by the caller; h_cfg, h_box: host.
 * Scratch: one fixed array of 32768 x 3 doubles (768 KiB) inside the library,
 * held by every GPU that loads the library until the process exits.  All calls
 * share it, so calls whose kernels overlap on the GPU (e.g. on two streams)
 * race: serialise them.  The first call on each device looks up the array's
 * device address (with that device current); make that first call before any
 * stream capture.  `stream` must belong to the current device (NULL: the legacy
 * default stream).  Errors: AP_ERR_ARG for n > 32768, n < 0, null pointers, a
 * stream of another device or a bad box/config (including eam_type other than
 * AP_EAM_ANALYTIC); AP_ERR_CUDA if the address lookup or a launch fails. */
ap_status ap_eval_eam_static(const ap_config* h_cfg, int64_t n, const double* d_x, const ap_box* h_box,
                             const double* d_lam, double* d_e_fast, double* d_f, void* stream);

/* ----------------------------------------------------------------- profiling */

/* Phases timed by ap_step when profiling is on (CUDA events on the call's stream). */
#define AP_PHASE_NEIGHBORS 0   /* wrap, cell list, shadows, EAM rows              */
#define AP_PHASE_CLASSIFY 1    /* CSP, lambda_0, spread, averages, queue, ACE rows */
#define AP_PHASE_EAM 2         /* EAM density + force kernels                      */
#define AP_PHASE_ACE 3         /* fused ACE energy/adjoint/force kernel           */
#define AP_PHASE_OTHER 4       /* integrator, finalize, indenter, reductions      */
#define AP_PHASE_THERMOSTAT 5  /* local thermostat: difference forces, Delta E, corrections */
#define AP_PHASE_ACE_ADJOINT 6 /* k_ace_adjoint alone (the force stage; also counted in ACE) */
#define AP_PHASE_EAM_FORCE 7   /* k_eam_force alone (the force pass; also counted in EAM)   */
#define AP_PHASE_ACE_BASIS 8   /* k_ace_basis alone (rows, G, A, nu = 1, 2; also counted in ACE) */
#define AP_NUM_PHASES 9

/* Turn per-phase event timing in ap_step on (1) or off (0) and clear the totals.
 * No paper counterpart: instrumentation of this implementation. */
ap_status ap_profile_enable(ap_ctx* ctx, int32_t on);

/* Accumulated device milliseconds and launch counts per phase since the last
 * ap_profile_enable (h_ms, h_calls: AP_NUM_PHASES entries each), the number of
 * this library's kernels launched by ap_step (*h_kernels), and the neighbour
 * pairs within ace_rc (*h_ace_pairs) and precise atoms (*h_ace_atoms) that the
 * ACE kernel processed, as of the last synchronising call.  Host pointers; any
 * may be NULL. */
ap_status ap_profile_read(ap_ctx* ctx, double* h_ms, int64_t* h_calls, int64_t* h_kernels, int64_t* h_ace_pairs,
                          int64_t* h_ace_atoms);

/* Tensor-core work counted since the last ap_profile_enable, as of the last
 * synchronising call: the m16n8k8 TF32 MMA tiles (2 x 16 x 8 x 8 flops each) that
 * the ACE basis kernel issued (mixed precision; 0 in FP64).  *h_mma is a host
 * pointer.  No paper counterpart: instrumentation.  Errors: AP_ERR_ARG. */
ap_status ap_profile_mma(ap_ctx* ctx, int64_t* h_mma);

/* Throughput peak of the current device, measured: which = 0 the FP32 FFMA rate
 * (eight independent FFMA chains per thread on 4 x 256 threads per SM), which = 1
 * the warp-level TF32 tensor-core rate (mma m16n8k8, eight independent accumulator
 * tiles per warp), in TFLOP/s (*h_tflops; an FMA counts 2 flops), and the SM clock
 * during the best of `reps` runs (*h_sm_mhz, may be NULL: SM cycle counter over the
 * global nanosecond timer).  reps in [2, 100]; the first run is a warm-up and is not
 * counted.  Allocates and frees a small device buffer; synchronises the stream.  No
 * paper counterpart: the denominators of the arithmetic rooflines.
 * Errors: AP_ERR_ARG (which, reps, null h_tflops), AP_ERR_CUDA. */
ap_status ap_probe_peak(int32_t which, int32_t reps, void* stream, double* h_tflops, double* h_sm_mhz);

/* ----------------------------------------------------------------- checkpoint */

/* Serialise the lambda histories, previous lambda, ring positions and step
 * counter into a host buffer.  With h_buf == NULL only *h_len (bytes) is set.
 * Synchronises. */
ap_status ap_state_export(ap_ctx* ctx, void* h_buf, size_t* h_len);
ap_status ap_state_import(ap_ctx* ctx, const void* h_buf, size_t h_len);

#ifdef __cplusplus
}
#endif

#endif /* AP_H */
