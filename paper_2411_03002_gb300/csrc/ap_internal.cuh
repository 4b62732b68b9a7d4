// Internal declarations of the GB300 adaptive-precision library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ap.h"

namespace ap {

// ------------------------------------------------------------------ geometry
// One simulation cell.  Cells of the search grid have edge h[d] = L[d]/nc[d] >=
// (largest list radius)/2, so every list needs a stencil half-width of 2 cells.
struct SysInfo {
  double lo[3];
  double L[3];       // hi - lo, computed once on the host
  double h[3];       // cell edge
  float hf[3];       // FP32 copy of h
  int nc[3];         // cells per dimension (<= 1023)
  int periodic[3];
  int cell_base;     // first global cell id of this system
  int org[3];        // offsets of this system's cell origins lo + c h in the origin table, per dimension
};

constexpr int kMaxCellsPerDim = 1023;
// Skin criterion (rebuild_every = AP_REBUILD_SKIN): a lambda update keeps the lists while
// the largest displacement since the build is at most this fraction of the skin
// (compile-time tuning; at most 0.5, the lists' own limit).
#ifndef AP_KEEP_FRAC
#define AP_KEEP_FRAC 0.45
#endif
constexpr double kKeepFrac = AP_KEEP_FRAC;
static_assert(kKeepFrac > 0.0 && kKeepFrac <= 0.5, "kept lists need m <= skin/2");
constexpr int kStencil = 2;          // cell half-width of the EAM and ACE list stencils

// Packed wrapped cell coordinates (10 bits each) carried in the shadow .w.
__host__ __device__ inline int pack_cell(int cx, int cy, int cz) { return cx | (cy << 10) | (cz << 20); }
__host__ __device__ inline int cell_x(int c) { return c & 1023; }
__host__ __device__ inline int cell_y(int c) { return (c >> 10) & 1023; }
__host__ __device__ inline int cell_z(int c) { return (c >> 20) & 1023; }

#ifdef __CUDACC__
// Cell-relative shadow s = x - o of a position in its unwrapped cell c, o = lo + c h the
// cell's origin (FP64; the FP32 shadow rounds s).  The origins of the wrapped cells come
// from a table (org, offsets S.org), so a shadow costs one FP64 subtraction per
// component, FP64 arithmetic being slow on this GPU; an unwrapped cell adds whole periods.
__device__ inline void cell_shadow(const SysInfo& S, const double* __restrict__ org, const int4& c,
                                   const double x[3], double s[3]) {
  const int cw[3] = {c.w & 1023, (c.w >> 10) & 1023, (c.w >> 20) & 1023};
  const int cu[3] = {c.x, c.y, c.z};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double v = x[d] - org[S.org[d] + cw[d]];
    if (cu[d] != cw[d]) v -= (double)((cu[d] - cw[d]) / S.nc[d]) * S.L[d];
    s[d] = v;
  }
}
#endif

// Stored per-entry cell offsets k (small boxes): 8 bits per component, biased by 128.
__host__ __device__ inline int pack_off(int kx, int ky, int kz) { return (kx + 128) | ((ky + 128) << 8) | ((kz + 128) << 16); }
__host__ __device__ inline int off_x(int p) { return (p & 255) - 128; }
__host__ __device__ inline int off_y(int p) { return ((p >> 8) & 255) - 128; }
__host__ __device__ inline int off_z(int p) { return ((p >> 16) & 255) - 128; }

// Cell offset of a pair from the wrapped cells (valid when nc >= 2*kStencil+1 in
// every periodic dimension, i.e. when offsets are not stored).
__device__ inline int wrap_off(int dc, int nc, int periodic) {
  if (periodic) {
    if (dc > nc / 2) dc -= nc;
    else if (dc < -(nc / 2)) dc += nc;
  }
  return dc;
}

// ------------------------------------------------------------------ error bits
enum : int {
  kErrCapacity = 1 << AP_ERR_CAPACITY,
  kErrNonfinite = 1 << AP_ERR_NONFINITE,
  kErrBox = 1 << AP_ERR_BOX,
  kErrSkin = 1 << AP_ERR_SKIN,
  kErrArg = 1 << AP_ERR_ARG,
  kErrTimeout = 1 << AP_ERR_TIMEOUT,
  kErrRadicand = 1 << AP_ERR_RADICAND,
};

// ------------------------------------------------------------------ device buffers
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
};

// Device-side scalars of one context.
struct DevScalars {
  int err;            // OR of error bits
  int need_eam;       // largest EAM row count seen
  int need_ace;       // largest ACE row count seen
  int n_detected;     // |D|
  int n_precise;      // |P| (int32 copy used by kernels)
  int work_counter;   // persistent-kernel work counter
  int work_counter2;  // second persistent-kernel work counter (right after work_counter)
  int n_csp_slow;     // atoms handed from the FP32 CSP kernel to the exact one
  int ace_row_max;    // longest ACE row of the last ACE row build
  int n_stale_bad;    // atoms whose CSP the rows of an earlier build cannot decide (stale rows)
  int n_det1;         // detected atoms the lambda spread's second pass visits
  unsigned long long row_total;   // ap_neighbor_total's result
  unsigned int max_disp2_bits;  // float bits of the largest squared displacement
  unsigned int max_dispa2_bits; // the same since the last ACE row build of the precise queue (skin criterion)
  long long n_precise64;
  double e_total;
  double e_kin;
  double e_ind;
  unsigned long long ace_pairs;   // neighbour pairs within the ACE cutoff processed (cumulative)
  unsigned long long ace_atoms;   // precise atoms processed by the ACE kernel (cumulative)
  unsigned long long ace_mma;     // m16n8k8 TF32 tensor-core MMAs issued by k_ace_basis (cumulative)
  int n_th_k;                     // local thermostat: |{Delta lambda != 0}| of the last update
  int n_th_e;                     // local thermostat: |{Delta E != 0}| of the last update
  unsigned long long th_n;        // corrections applied (cumulative)
  unsigned long long th_bad;      // corrections refused for a negative radicand (cumulative)
  double th_e;                    // sum of the corrected Delta E (cumulative, eV)
};

// ------------------------------------------------------------------ ACE tables
struct AceTables {
  int nb = 0;
  std::vector<int> desc;         // nb * 7
  std::vector<double> gaunt;     // 4*7*4*7*4*7
  // Flattened product terms of E = sum_v c_v B_v, each t: coef * A[a1] * A[a2] * A[a3]
  // (a2 = a3 = 255 for nu = 1 and a3 = 255 for nu = 2).
  std::vector<int> term_idx;     // packed a1 | a2 << 8 | a3 << 16
  std::vector<double> term_coef;
  int n_terms = 0;
  std::vector<double> c1;        // [8] nu = 1 coefficients
  std::vector<double> m2;        // [5][8][8] nu = 2 symmetric coupling matrices
  // nu = 3 merged monomials coef * A_a A_b A_c over the 48 entries with n <= 2,
  // l <= 3 (a <= b <= c, key c | b << 6 | a << 12, ascending keys); the
  // lane-per-atom kernel's straight-line code (ace_nu3.inc) is generated from nu3_key.
  std::vector<uint32_t> nu3_key;
  std::vector<double> nu3_coef;
  // second coefficient set phi^(2) of the Finnis-Sinclair form (zeros unless ace_fs_on)
  std::vector<double> c1b, m2b, nu3_coef2;
};
void build_ace_tables(const ap_config& cfg, AceTables& t);

// ------------------------------------------------------------------ selector model
// Device image of the selector MLP 24-64-64-1.  Flat FP32 parameter layout (the
// ABI's): W1 [24][64] input-major, b1 [64], W2 [64][64], b2 [64], w3 [64], b3.
struct SelDev {
  static constexpr int kParams = AP_SEL_NPARAMS;
  static constexpr int kOffB1 = 24 * 64, kOffW2 = kOffB1 + 64, kOffB2 = kOffW2 + 64 * 64, kOffW3 = kOffB2 + 64,
                       kOffB3 = kOffW3 + 64;
  // FP32 vectors: w3 (bf16-valued), b1, b2, b3, mu, 1/sigma
  static constexpr int kW3 = 0, kB1 = 64, kB2 = 128, kB3 = 192, kMu = 196, kInvS = 220, kVec = 244;
  // bf16 operand images in the canonical no-swizzle K-major layout: W1^T (64 x 32,
  // K padded with zeros) then W2^T (64 x 64); core matrix (row block rb, K block kb)
  // at (kb * 8 + rb) * 128 bytes.
  alignas(16) uint8_t img[4096 + 8192];
  alignas(16) float vec[256];
  alignas(16) float W2r[64 * 64];   // bf16-valued W2 [k][n] for the backward pass
};
static_assert(SelDev::kOffB3 + 1 == SelDev::kParams, "selector parameter layout");

// ------------------------------------------------------------------ context
}  // namespace ap

struct ap_ctx {
  ap_config cfg;
  int device = 0;
  std::string err_msg = "no error";
  int64_t need = 0;
  ap::AceTables ace;

  // systems
  int n_sys = 0;
  std::vector<ap::SysInfo> h_sys;
  std::vector<int64_t> h_offsets;
  ap::SysInfo* d_sys = nullptr;
  int* d_atom_sys = nullptr;     // null when n_sys == 1
  int n_cells = 0;
  bool stored_off = false;
  bool lim_valid = false;        // d_lim_eam holds the prefixes of an EAM pass on the current rows
  float split_rpf2 = 0.f;        // r_c^2 (FP32) at which the EAM rows were split
  int sten_spread[3] = {0, 0, 0};
  int sten_spread_stale[3] = {0, 0, 0};   // the spread's stencil with cells up to skin/2 old
  bool cells_stale = false;      // the atoms moved since the cell build (ap_step skipped a rebuild)
  double stale_m = 0.0;          // with cells_stale: the largest displacement since the cell build
  bool stale_ok = false;         // rows and cells may be kept past a lambda update (pair offsets unwrap)

  // capacity
  int64_t n_cap = 0;             // per-atom arrays sized for this many atoms
  int64_t n = 0;                 // atoms of the last build
  int cells_cap = 0;
  int cap_eam = 0, cap_ace = 0;
  bool built = false;
  bool lam_ready = false;        // a classification exists for the current n
  int64_t rebuilds = 0;
  int64_t kept = 0;              // lambda updates that kept the lists (skin criterion)
  int64_t ace_rebuilds = 0;      // ACE row builds between lambda updates (skin criterion)

  // per-atom state (device)
  int* d_cell = nullptr;         // global cell id (wrapped)
  int4* d_cunw = nullptr;        // unwrapped cell coords (x,y,z) + packed wrapped code (w)
  int* d_cell_start = nullptr;   // [n_cells + 1]
  int* d_cell_count = nullptr;   // [n_cells]
  int* d_cell_atoms = nullptr;   // [n]
  int* d_slot = nullptr;         // [n] slot inside cell
  float4* d_sh32 = nullptr;      // FP32 cell-relative shadow
  float4* d_sh32c = nullptr;     // the same in cell order (the EAM row build's candidate stream)
  double4_32a* d_sh64 = nullptr;     // FP64 cell-relative shadow
  float4* d_sh32b = nullptr;     // [n] the FP32 shadows at the last build (displacement check)
  float4* d_sh32a = nullptr;     // [n] the FP32 shadows at the last ACE row build (skin criterion only)
  double* d_org = nullptr;       // cell origins lo + c h of every system and dimension (SysInfo::org)
  double* d_vscale = nullptr;    // [n] 0.5 dt ACC / m_i of the current ap_step call
  int* d_nbr_eam = nullptr;      // [n][cap_eam]
  int* d_off_eam = nullptr;      // [n][cap_eam] (stored offsets only)
  int* d_cnt_eam = nullptr;      // [n]
  int* d_lim_eam = nullptr;      // [n] the row build's in-range count, then (after each EAM density
                                 //     pass) one past the last entry found inside r_c
  int* d_split_eam = nullptr;    // [n] the row build's in-range count, kept until the next build
                                 //     (rebuild_every = AP_REBUILD_SKIN only)
  int* d_nbr_ace = nullptr;      // [ace_q_cap][cap_ace] rows in queue order
  int* d_off_ace = nullptr;
  int* d_cnt_ace = nullptr;      // [ace_q_cap]
  int64_t ace_q_cap = 0;         // queue positions held by the ACE rows and the ACE scratch below
  int ace_rec_cap = 0;           // pair-record slots per queue position (>= the longest ACE row)

  // lambda state (FP64)
  double* d_csp = nullptr;       // sample
  int* d_csp_slow = nullptr;     // [n] atoms whose CSP needs the exact selection
  double* d_csp_avg = nullptr;
  double* d_lam0 = nullptr;
  double* d_lam_min = nullptr;
  double* d_lam_avg = nullptr;
  double* d_lam_prev = nullptr;
  double* d_csp_hist = nullptr;  // [n_csp_avg][n]
  double* d_lam_hist = nullptr;  // [n_lam_avg][n]
  int csp_pos = -1, lam_pos = -1;
  bool hist_started = false;
  int* d_flag = nullptr;         // [n] compaction flags
  int* d_scan = nullptr;         // [n + 1] scan output
  int* d_detected = nullptr;     // [n] detected queue
  float* d_vmin_f = nullptr;     // [n] FP32 minima of the lambda spread's first pass
  int* d_det1 = nullptr;         // [n] detected atoms the spread's second pass visits
  int* d_precise = nullptr;      // [n] internal precise queue
  double* d_lam_int = nullptr;   // [n] internal lambda (ap_step)

  // potentials scratch
  void* d_q = nullptr;           // [n] (lambda xi', lambda) as float2 or double2
  double* d_xi = nullptr;        // [n] xi(rho)
  float4* d_facc32 = nullptr;    // [n] ACE force accumulator (mixed)
  double* d_facc64 = nullptr;    // [n][3] ACE force accumulator (FP64)
  unsigned long long* d_faccfix = nullptr;   // [n][3] fixed-point ACE force accumulator (ace_deterministic)
  double* d_efast = nullptr;     // [n] internal (ap_step)
  double* d_eprec = nullptr;     // [n] internal (ap_step)
  double* d_eatom = nullptr;     // [n] internal (ap_step)
  double* d_eext = nullptr;      // [n] indenter energy per atom (ap_step)
  uint8_t* d_changeable = nullptr;  // [n] complement of the fixed mask (ap_step)
  bool restart_pending = false;  // lambda state imported; next ap_step reuses it
  float* d_W32 = nullptr;        // [W (320) | M2 (320) | C1 (8)]
  double* d_W64 = nullptr;
  // ACE scratch per precise-queue position q < ace_q_cap (working precision)
  void* d_ace_list = nullptr;       // [q][ace_rec_cap] in-range (d_x, d_y, d_z, j) records
  int* d_ace_nin = nullptr;         // [q]
  void* d_ace_a48 = nullptr;        // [q][48]
  void* d_ace_dA = nullptr;         // [q][200]
  double* d_ace_e12 = nullptr;      // [q]
  void* d_ace_de3 = nullptr;        // [q][48]
  double* d_ace_e3 = nullptr;       // [q]
  void* d_ace_dAb = nullptr;        // [q][200] (Finnis-Sinclair form)
  double* d_ace_e12b = nullptr;     // [q]
  double* d_ace_fs = nullptr;       // [q][2]

  // scan scratch
  int* d_scan_tmp = nullptr;
  size_t scan_tmp_cap = 0;
  double* d_red = nullptr;       // reduction partials
  int red_cap = 0;

  // selector (learned detection score)
  ap::SelDev* d_sel_model = nullptr;
  float* d_sel_master = nullptr;   // [kParams] FP32 master weights
  float* d_sel_m1 = nullptr;       // Adam first moments
  float* d_sel_m2 = nullptr;       // Adam second moments
  float* d_sel_grad = nullptr;     // [kParams + 1] gradient and loss of the last training step
  float* d_sel_partial = nullptr;  // [2 * num_sms][kParams + 1]
  float2* d_sel_rho = nullptr;     // [n] FP32 (rho, xi'(rho)) of the feature pre-pass
  float* d_sel_feat = nullptr;     // [n][24] features of the classification path
  double* d_sel_score = nullptr;   // [n] selector score p of the classification path
  float* d_sel_z = nullptr;        // [train_cap] logits of the last training forward pass
  void* d_sel_h1 = nullptr;        // [train_cap][64] bf16 hidden layer 1
  float* d_sel_h2 = nullptr;       // [train_cap][64] FP32 hidden layer 2
  int64_t sel_train_cap = 0;
  int64_t sel_feat_cap = 0;
  bool sel_ready = false;
  int64_t sel_t = 0;               // Adam steps taken

  // local thermostat scratch (allocated when thermostat_on)
  double* d_th_lamc = nullptr;   // [n] lambda^c (the values before the update)
  double* d_th_dlam = nullptr;   // [n] Delta lambda = lambda^c - lambda^d
  double* d_th_w = nullptr;      // [n] ACE weights of the difference force (-Delta lambda)
  double* d_th_df = nullptr;     // [n][3] F^c - F^d
  double* d_th_ep = nullptr;     // [n] E^p of the atoms with Delta lambda != 0
  double* d_th_de = nullptr;     // [n] Delta E
  int* d_th_qk = nullptr;        // [n] atoms with Delta lambda != 0
  int* d_th_qe = nullptr;        // [n] atoms with Delta E != 0
  int* d_th_cellof = nullptr;    // [n]
  int* d_th_atoms = nullptr;     // [n]
  int* d_th_ccount = nullptr;    // [cells]
  int* d_th_cstart = nullptr;    // [cells + 1]
  int64_t th_cap = 0, th_cells_cap = 0;

  ap::DevScalars* d_sc = nullptr;
  ap::DevScalars* h_sc = nullptr;  // pinned mirror

  // MD
  int64_t step = 0;
  bool md_ready = false;
  int num_sms = 0;

  // profiling (ap_profile_enable / ap_profile_read)
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;   // reusable events
  struct EvSpan {
    int phase, start, end;
  };
  std::vector<EvSpan> ev_pairs_phase;   // (phase, start event, end event)
  int ev_used = 0;
  double prof_ms[AP_NUM_PHASES] = {};
  int64_t prof_calls[AP_NUM_PHASES] = {};
  int64_t kernels = 0;                // kernels launched by ap_step since the last enable
};

namespace ap {

// ------------------------------------------------------------------ launchers
// scan.cu / k_neighbors.cu
size_t scan_tmp_bytes(int n);
// d_out has n+1 entries; returns the number of kernels launched
int scan_exclusive(const int* d_in, int* d_out, int n, int* d_tmp, cudaStream_t s);
void launch_bin(ap_ctx* c, const double* d_x, const int32_t* d_species, cudaStream_t s);
void launch_cell_sort(ap_ctx* c, cudaStream_t s);
void launch_shadow(ap_ctx* c, const double* d_x, cudaStream_t s);
void launch_build_eam(ap_ctx* c, const double* d_x, cudaStream_t s);
void launch_row_total(ap_ctx* c, int which, int rows, cudaStream_t s);   // -> c->d_sc->row_total
void launch_build_ace(ap_ctx* c, const double* d_x, const int* d_queue, const int* d_nq, cudaStream_t s);
void launch_export_rows(ap_ctx* c, int which, int rows, int cap_out, int* d_cnt, int* d_idx, int* d_shift,
                        cudaStream_t s);
void launch_wrap_positions(ap_ctx* c, double* d_x, cudaStream_t s);

// ap_api.cu: profiling marks (event index, or -1 when profiling is off) and spans
int prof_mark(ap_ctx* c, cudaStream_t s);
void prof_add(ap_ctx* c, int phase, int start, int end);

// k_classify.cu
// fresh_rows: the EAM rows were built at d_x (the CSP may stop after their in-range part);
// stale_disp > 0: the rows are older than d_x, every atom having moved at most stale_disp
// since the build; atoms whose selection the rows cannot guarantee are counted in
// DevScalars::n_stale_bad.
void launch_csp(ap_ctx* c, const double* d_x, const uint8_t* d_ch, cudaStream_t s, bool fresh_rows = false,
                double stale_disp = 0.0);
void launch_lambda0(ap_ctx* c, const uint8_t* d_ch, const double* d_score, double lo, double hi, cudaStream_t s);
void launch_spread(ap_ctx* c, const double* d_x, const uint8_t* d_ch, cudaStream_t s);
void launch_lambda_final(ap_ctx* c, const uint8_t* d_ch, double* d_lam, int* d_queue, int64_t* d_nq64,
                         cudaStream_t s);

// k_eam.cu
void launch_eam(ap_ctx* c, const double* d_lam, double* d_e_fast, double* d_f, bool accumulate, cudaStream_t s);

// k_ace.cu
void upload_ace_tables(ap_ctx* c);
bool ace_nu3_matches(const AceTables& t);
// d_wgt: explicit ACE weights w_i (NULL: w_i = 1 - lambda_i); d_count: device queue
// length (NULL: the context's precise count).
void launch_ace(ap_ctx* c, const double* d_lam, const int* d_queue, double* d_e_prec, bool forces, cudaStream_t s,
                const double* d_wgt = nullptr, const int* d_count = nullptr);
void launch_ace_finalize(ap_ctx* c, double* d_f, cudaStream_t s);

// k_selector.cu
void launch_sel_features(ap_ctx* c, float* d_feat, cudaStream_t s);   // needs c->d_csp of the same positions
cudaError_t sel_mlp_attr();
void launch_sel_mlp(ap_ctx* c, int64_t n, const float* d_feat, const int* d_idx, float* d_p, double* d_score,
                    float* d_z, void* d_h1, float* d_h2, cudaStream_t s);
int sel_bwd_parts(ap_ctx* c, int64_t b);
void launch_sel_backward(ap_ctx* c, int64_t b, const float* d_feat, const int* d_idx, const float* d_label,
                         const float* d_weight, cudaStream_t s);
void launch_sel_adam(ap_ctx* c, bool update, float lr, float beta1, float beta2, float eps, float inv_bc1,
                     float inv_bc2, cudaStream_t s);
size_t sel_partial_floats(ap_ctx* c);

// k_thermostat.cu
int th_cell_count(const ap_ctx* c);
void launch_th_delta(ap_ctx* c, const double* d_lam_c, const double* d_lam_d, cudaStream_t s);
void launch_th_energy(ap_ctx* c, const double* d_f, const double* d_v, const double* d_mass, const uint8_t* d_fixed,
                      cudaStream_t s);
void launch_th_correct(ap_ctx* c, const int* d_q, const int* d_m, const double* d_x, const uint8_t* d_fixed,
                       const double* d_mass, double* d_v, cudaStream_t s);

// k_md.cu
void launch_vscale(ap_ctx* c, const double* d_mass, cudaStream_t s);
void launch_vv_first(ap_ctx* c, double* d_x, double* d_v, const double* d_f, const double* d_mass,
                     const uint8_t* d_fixed, cudaStream_t s);
void launch_vv_second(ap_ctx* c, double* d_v, const double* d_f, const double* d_mass, const uint8_t* d_fixed,
                      cudaStream_t s);
void launch_indenter(ap_ctx* c, const double* d_x, double* d_f, double t, cudaStream_t s);
void launch_blend(ap_ctx* c, const double* d_lam, const double* d_ef, const double* d_ep, const double* d_e_ext,
                  double* d_e_atom, double* d_e_total, cudaStream_t s);
void launch_kinetic(ap_ctx* c, const double* d_v, const double* d_mass, double* d_out, cudaStream_t s);
void launch_fill_lambda(ap_ctx* c, double* d_lam, double value, cudaStream_t s);

}  // namespace ap
